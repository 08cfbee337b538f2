// Serving: a stream of placement jobs with continuous batching (see the
// serving section of include/fftpl.h).  Host-side scheduler: a FIFO queue, an
// HBM-budget admission test, one stream per active job, latency records.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "fftpl_internal.cuh"
#include "loop_ctrl.cuh"

using namespace fftpl;

namespace {

struct Job {
    int64_t id = 0;
    int32_t state = FFTPL_JOB_QUEUED;
    // deep copies of the submission
    fftpl_region region{};
    int32_t n = 0, m_mov = 0, m_fix = 0, E = 0;
    int64_t P = 0;
    std::vector<float> w, h, fx, fy, dx, dy, x0, y0, xr, yr;
    std::vector<int32_t> net_ptr, pin_cell;
    fftpl_options opt{};
    int32_t iters = 0, launched = 0;
    double t_submit = 0, t_admit = 0, t_done = 0, hpwl = 0, tau = 0;
    double t_prev = -1.0;   // end of the tick that ran the job's previous iterations
    size_t est_bytes = 0, dev_bytes = 0;
    fftpl_t handle = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
};

double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    double pos = q * (double)(v.size() - 1);
    size_t i = (size_t)pos;
    double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct fftpl_server {
    fftpl_server_options opt{};
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    std::deque<Job*> queue;
    std::vector<Job*> active;
    int64_t next_id = 1, submitted = 0, completed = 0, failed = 0;
    size_t used = 0, peak_bytes = 0;
    int32_t peak_active = 0;
    double injected = -1.0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double first_submit = -1.0, last_done = 0.0;
    std::vector<double> iter_ms, job_ms;
    std::string err;

    double now() const {
        if (injected >= 0.0) return injected;
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

fftpl_status fail(fftpl_server* s, fftpl_status st, const std::string& m) {
    s->err = m;
    set_global_error(m);
    return st;
}

void release(Job* j) {
    if (j->handle) fftpl_destroy(j->handle);
    j->handle = nullptr;
    if (j->ev) cudaEventDestroy(j->ev);
    j->ev = nullptr;
    if (j->stream) cudaStreamDestroy(j->stream);
    j->stream = nullptr;
}

// Creates the job's handle on its own stream and starts its placement run.
fftpl_status admit(fftpl_server* s, Job* j) {
    if (s->opt.dry_run) {
        j->dev_bytes = j->est_bytes;
        return FFTPL_OK;
    }
    if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(s, FFTPL_ECUDA, "stream or event creation failed");
    }
    fftpl_cells cells{j->m_mov, j->m_fix, j->w.data(), j->h.data(),
                      j->m_fix ? j->fx.data() : nullptr, j->m_fix ? j->fy.data() : nullptr};
    fftpl_nets nets{j->E, j->net_ptr.data()};
    fftpl_pins pins{j->P, j->pin_cell.data(), j->dx.data(), j->dy.data()};
    fftpl_status st = fftpl_create(&j->region, j->n, &cells, &nets, &pins, &j->opt, j->stream,
                                   &j->handle);
    if (st != FFTPL_OK) return st;
    Ctx& c = *j->handle;
    // start positions through the handle's host-staging buffer
    size_t m = (size_t)j->m_mov;
    if (!c.hx) {
        st = FFTPL_OK;
        float* p = nullptr;
        if (cudaMalloc((void**)&p, std::max<size_t>(2 * m, 1) * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(s, FFTPL_ENOMEM, "start-position buffer");
        }
        c.dev_allocs.push_back(p);
        c.dev_bytes += std::max<size_t>(2 * m, 1) * sizeof(float);
        c.hx = p;
        c.hy = p + m;
    }
    if (m) {
        cudaMemcpyAsync(c.hx, j->x0.data(), m * sizeof(float), cudaMemcpyHostToDevice, j->stream);
        cudaMemcpyAsync(c.hy, j->y0.data(), m * sizeof(float), cudaMemcpyHostToDevice, j->stream);
    }
    st = fftpl_place_init(j->handle, c.hx, c.hy);
    if (st != FFTPL_OK) return st;
    st = loop_records(c, j->iters, 0.0);
    if (st != FFTPL_OK) return st;
    j->dev_bytes = fftpl_device_bytes(j->handle);
    return FFTPL_OK;
}

// Copies the result of a finished job and frees its device resources.
fftpl_status retire(fftpl_server* s, Job* j) {
    if (!s->opt.dry_run) {
        Ctx& c = *j->handle;
        size_t m = (size_t)j->m_mov;
        j->xr.resize(m);
        j->yr.resize(m);
        double k = 0.0;
        if (cudaMemcpy(&k, c.ctrl + C_K, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(s, FFTPL_ECUDA, "reading the job's iteration count");
        int last = (int)k - 1;
        if (last >= 0 && last < c.recs_cap) {
            double r[kRecFields];
            cudaMemcpy(r, c.recs + (size_t)last * kRecFields, sizeof(r), cudaMemcpyDeviceToHost);
            j->hpwl = r[1];
            j->tau = r[3];
        }
        if (m) {
            cudaMemcpy(j->xr.data(), c.u, m * sizeof(float), cudaMemcpyDeviceToHost);
            cudaMemcpy(j->yr.data(), c.u + m, m * sizeof(float), cudaMemcpyDeviceToHost);
        }
        j->launched = (int)k;
        if (cudaGetLastError() != cudaSuccess) return fail(s, FFTPL_ECUDA, "copying a result");
    }
    release(j);
    return FFTPL_OK;
}

}  // namespace

extern "C" {

void fftpl_server_default_options(fftpl_server_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = (size_t)150 << 30;
    o->max_active = 64;
    o->iters_per_tick = 1;
}

size_t fftpl_estimate_bytes(int32_t n, int32_t m_mov, int32_t m_fix, int32_t E, int64_t P,
                            int32_t iters, int32_t deterministic) {
    (void)E;
    size_t nn = (size_t)n * n, m = (size_t)std::max(m_mov, 0), f = (size_t)std::max(m_fix, 0);
    size_t slots = (size_t)(1.15 * (double)std::max<int64_t>(P, 0)) + 32 * 64;
    size_t b = 32 * nn + (deterministic ? 4 * nn : 0) + 16 * (size_t)n + 64;
    b += 8 * (m + f) + 8 * f + 40 * m;                 // sizes, fixed centres, gN, gW, gW2, pos2
    b += 20 * slots + (deterministic ? 4 * slots + 8 * (size_t)P + 4 * m : 0);
    b += 40 * m + 8 * m;                               // loop vectors, start positions
    b += 64 * (size_t)std::max(iters, 1) + 8192;       // records, sums, control
    if (deterministic) b += 16 * (std::max(nn / 4, 2 * m / 256) + slots / 256) + 64;
    return b;
}

fftpl_status fftpl_server_create(const fftpl_server_options* opt, fftpl_server_t* out) {
    if (!out) return FFTPL_EINVAL;
    *out = nullptr;
    fftpl_server* s = new (std::nothrow) fftpl_server();
    if (!s) return FFTPL_ENOMEM;
    if (opt) s->opt = *opt;
    else fftpl_server_default_options(&s->opt);
    if (s->opt.max_active < 1 || s->opt.iters_per_tick < 1 || s->opt.hbm_budget_bytes == 0) {
        delete s;
        set_global_error("server options: max_active, iters_per_tick and the budget must be > 0");
        return FFTPL_EINVAL;
    }
    *out = s;
    return FFTPL_OK;
}

void fftpl_server_destroy(fftpl_server_t s) {
    if (!s) return;
    for (Job* j : s->active) release(j);
    delete s;
}

fftpl_status fftpl_server_set_clock(fftpl_server_t s, double now_s) {
    if (!s) return FFTPL_EINVAL;
    s->injected = now_s;
    return FFTPL_OK;
}

fftpl_status fftpl_server_submit(fftpl_server_t s, const fftpl_region* region, int32_t n,
                                 const fftpl_cells* cells, const fftpl_nets* nets,
                                 const fftpl_pins* pins, const fftpl_options* opt,
                                 const float* x0, const float* y0, int32_t iters, int64_t* id) {
    if (!s || !region || !cells || !nets || !pins || !id) return FFTPL_EINVAL;
    if (iters < 1) return fail(s, FFTPL_EINVAL, "iters must be >= 1");
    if (cells->m_mov > 0 && (!x0 || !y0)) return fail(s, FFTPL_EINVAL, "null start positions");
    if (cells->m_mov < 0 || cells->m_fix < 0 || nets->E < 0 || pins->P < 0 || !nets->net_ptr)
        return fail(s, FFTPL_EINVAL, "bad job sizes");
    auto j = std::make_unique<Job>();
    j->id = s->next_id++;
    j->region = *region;
    j->n = n;
    j->m_mov = cells->m_mov;
    j->m_fix = cells->m_fix;
    j->E = nets->E;
    j->P = pins->P;
    size_t mt = (size_t)cells->m_mov + cells->m_fix;
    if (mt && (!cells->w || !cells->h)) return fail(s, FFTPL_EINVAL, "null cell sizes");
    j->w.assign(cells->w, cells->w + mt);
    j->h.assign(cells->h, cells->h + mt);
    if (cells->m_fix) {
        if (!cells->fix_x || !cells->fix_y) return fail(s, FFTPL_EINVAL, "null fixed centres");
        j->fx.assign(cells->fix_x, cells->fix_x + cells->m_fix);
        j->fy.assign(cells->fix_y, cells->fix_y + cells->m_fix);
    }
    j->net_ptr.assign(nets->net_ptr, nets->net_ptr + nets->E + 1);
    if (pins->P) {
        if (!pins->pin_cell || !pins->dx || !pins->dy) return fail(s, FFTPL_EINVAL, "null pins");
        j->pin_cell.assign(pins->pin_cell, pins->pin_cell + pins->P);
        j->dx.assign(pins->dx, pins->dx + pins->P);
        j->dy.assign(pins->dy, pins->dy + pins->P);
    }
    if (opt) j->opt = *opt;
    else fftpl_default_options(&j->opt);
    if (s->opt.deterministic) j->opt.deterministic = 1;
    j->opt.use_graphs = 0;
    j->x0.assign(x0, x0 + cells->m_mov);
    j->y0.assign(y0, y0 + cells->m_mov);
    j->iters = iters;
    j->est_bytes = fftpl_estimate_bytes(n, cells->m_mov, cells->m_fix, nets->E, pins->P, iters,
                                        j->opt.deterministic);
    j->t_submit = s->now();
    if (s->first_submit < 0) s->first_submit = j->t_submit;
    *id = j->id;
    s->queue.push_back(j.get());
    s->jobs[j->id] = std::move(j);
    s->submitted++;
    return FFTPL_OK;
}

fftpl_status fftpl_server_tick(fftpl_server_t s, int32_t* active, int32_t* queued) {
    if (!s) return FFTPL_EINVAL;
    fftpl_status status = FFTPL_OK;
    // admit in arrival order while the budget and the slots allow
    while (!s->queue.empty() && (int)s->active.size() < s->opt.max_active) {
        Job* j = s->queue.front();
        bool fits = s->used + j->est_bytes <= s->opt.hbm_budget_bytes;
        if (!fits && !s->active.empty()) break;   // wait for memory to free up
        s->queue.pop_front();
        if (!fits) {                              // larger than the whole budget
            j->state = FFTPL_JOB_FAILED;
            s->failed++;
            status = fail(s, FFTPL_ENOMEM, "job exceeds the HBM budget");
            continue;
        }
        fftpl_status st = admit(s, j);
        if (st != FFTPL_OK) {
            release(j);
            j->state = FFTPL_JOB_FAILED;
            s->failed++;
            status = st;
            continue;
        }
        j->state = FFTPL_JOB_ACTIVE;
        j->t_admit = s->now();
        s->used += j->dev_bytes;
        s->active.push_back(j);
    }
    s->peak_active = std::max(s->peak_active, (int32_t)s->active.size());
    s->peak_bytes = std::max(s->peak_bytes, s->used);
    // one round: iters_per_tick iterations of every active job, concurrently
    double t_start = s->now();
    std::vector<int> ran(s->active.size(), 0);
    for (size_t k = 0; k < s->active.size(); ++k) {
        Job* j = s->active[k];
        int todo = std::min(s->opt.iters_per_tick, j->iters - j->launched);
        if (!s->opt.dry_run) {
            for (int t = 0; t < todo; ++t) {
                fftpl_status st = loop_enqueue(*j->handle);
                if (st != FFTPL_OK) {
                    status = st;
                    todo = t;
                    break;
                }
            }
            cudaEventRecord(j->ev, j->handle->stream);
        }
        j->launched += todo;
        ran[k] = todo;
    }
    if (!s->opt.dry_run) {
        for (Job* j : s->active) {
            if (cudaEventSynchronize(j->ev) != cudaSuccess) {
                cudaGetLastError();
                status = fail(s, FFTPL_ECUDA, "a job's iterations failed");
            }
        }
    }
    double t_end = s->now();
    // per-iteration latency seen by a job: time since its previous iterations
    // completed (waiting behind the other jobs included), per iteration
    for (size_t k = 0; k < s->active.size(); ++k) {
        Job* j = s->active[k];
        if (ran[k] > 0) {
            double since = j->t_prev >= 0.0 ? j->t_prev : t_start;
            s->iter_ms.push_back(1e3 * (t_end - since) / ran[k]);
            j->t_prev = t_end;
        }
    }
    // retire finished jobs
    std::vector<Job*> keep;
    for (Job* j : s->active) {
        if (j->launched >= j->iters) {
            fftpl_status st = retire(s, j);
            s->used -= j->dev_bytes;
            if (st != FFTPL_OK) {
                j->state = FFTPL_JOB_FAILED;
                s->failed++;
                status = st;
                continue;
            }
            j->state = FFTPL_JOB_DONE;
            j->t_done = s->now();
            s->job_ms.push_back(1e3 * (j->t_done - j->t_submit));
            s->completed++;
            s->last_done = j->t_done;
        } else {
            keep.push_back(j);
        }
    }
    s->active.swap(keep);
    if (active) *active = (int32_t)s->active.size();
    if (queued) *queued = (int32_t)s->queue.size();
    return status;
}

fftpl_status fftpl_server_job(fftpl_server_t s, int64_t id, fftpl_job_info* info, float* x,
                              float* y) {
    if (!s) return FFTPL_EINVAL;
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return fail(s, FFTPL_EINVAL, "unknown job id");
    Job* j = it->second.get();
    if (info) {
        info->id = j->id;
        info->state = j->state;
        info->iters_done = j->launched;
        info->m_mov = j->m_mov;
        info->n = j->n;
        info->t_submit = j->t_submit;
        info->t_admit = j->t_admit;
        info->t_done = j->t_done;
        info->hpwl = j->hpwl;
        info->tau = j->tau;
        info->device_bytes = j->dev_bytes;
    }
    if ((x || y) && j->state == FFTPL_JOB_DONE && !s->opt.dry_run) {
        if (x) std::copy(j->xr.begin(), j->xr.end(), x);
        if (y) std::copy(j->yr.begin(), j->yr.end(), y);
    } else if ((x || y) && j->state != FFTPL_JOB_DONE) {
        return fail(s, FFTPL_ESTATE, "job not done");
    }
    return FFTPL_OK;
}

fftpl_status fftpl_server_report(fftpl_server_t s, fftpl_server_stats* o) {
    if (!s || !o) return FFTPL_EINVAL;
    memset(o, 0, sizeof(*o));
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->failed = s->failed;
    o->active = (int32_t)s->active.size();
    o->queued = (int32_t)s->queue.size();
    o->peak_active = s->peak_active;
    o->peak_device_bytes = s->peak_bytes;
    o->wall_s = s->first_submit >= 0 ? s->last_done - s->first_submit : 0.0;
    o->jobs_per_s = o->wall_s > 0 ? (double)s->completed / o->wall_s : 0.0;
    o->iter_p50_ms = pct(s->iter_ms, 0.50);
    o->iter_p99_ms = pct(s->iter_ms, 0.99);
    o->job_p50_ms = pct(s->job_ms, 0.50);
    o->job_p99_ms = pct(s->job_ms, 0.99);
    return FFTPL_OK;
}

}  // extern "C"
