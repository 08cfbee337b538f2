// Serving: a stream of placement jobs with continuous batching (see the
// serving section of include/fftpl.h).
//
// Job life: QUEUED -> (admitted by budget and slot) created on a worker
// thread -> ACTIVE: its iterations are launched in chunks on its own stream,
// each chunk as soon as the job's previous chunk has completed, so that no
// job waits for another -> retired on a worker thread (results copied to the
// host, device memory returned to the pool in stream order) -> DONE.  The
// tick thread never blocks on the device: it launches and polls events.
// Handle creation (host layout work, device set-up) and retirement run on
// worker threads so that they overlap the running jobs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fftpl_internal.cuh"
#include "loop_ctrl.cuh"

using namespace fftpl;

namespace {

enum Phase { PH_QUEUED, PH_CREATING, PH_ACTIVE, PH_RETIRING, PH_DONE, PH_FAILED };

struct Job {
    int64_t id = 0;
    std::atomic<int> phase{PH_QUEUED};
    // deep copies of the submission (inputs dropped once the handle exists)
    fftpl_region region{};
    int32_t n = 0, m_mov = 0, m_fix = 0, E = 0;
    int64_t P = 0;
    std::vector<float> w, h, fx, fy, dx, dy, x0, y0, xr, yr;
    std::vector<int32_t> net_ptr, pin_cell;
    fftpl_options opt{};
    int32_t iters = 0, launched = 0, completed_iters = 0, in_flight = 0;
    double t_submit = 0, t_admit = 0, t_done = 0, hpwl = 0, tau = 0;
    double t_prev = -1.0;   // completion of the job's previous chunk of iterations
    size_t est_bytes = 0, dev_bytes = 0, held = 0;
    fftpl_t handle = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    fftpl_status status = FFTPL_OK;
    std::string err;
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
    std::vector<Job*> creating, active, retiring;
    int64_t next_id = 1, submitted = 0, completed = 0, failed = 0;
    size_t used = 0, peak_bytes = 0;
    int32_t peak_active = 0;
    std::atomic<double> injected{-1.0};
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double first_submit = -1.0, last_done = 0.0;
    std::vector<double> iter_ms, job_ms;
    std::string err;
    int device = 0;
    // worker threads: handle creation and retirement
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> tasks;
    bool stop = false;
    std::vector<std::thread> workers;

    double now() const {
        double inj = injected.load();
        if (inj >= 0.0) return inj;
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

void drop_inputs(Job* j) {
    std::vector<float>().swap(j->w);
    std::vector<float>().swap(j->h);
    std::vector<float>().swap(j->fx);
    std::vector<float>().swap(j->fy);
    std::vector<float>().swap(j->dx);
    std::vector<float>().swap(j->dy);
    std::vector<float>().swap(j->x0);
    std::vector<float>().swap(j->y0);
    std::vector<int32_t>().swap(j->net_ptr);
    std::vector<int32_t>().swap(j->pin_cell);
}

// Creates the job's handle on its own stream, loads its start positions,
// initialises the loop and captures the loop graph (worker thread).
fftpl_status create_job(Job* j) {
    if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        j->err = "stream or event creation failed";
        return FFTPL_ECUDA;
    }
    fftpl_cells cells{j->m_mov, j->m_fix, j->w.data(), j->h.data(),
                      j->m_fix ? j->fx.data() : nullptr, j->m_fix ? j->fy.data() : nullptr};
    fftpl_nets nets{j->E, j->net_ptr.data()};
    fftpl_pins pins{j->P, j->pin_cell.data(), j->dx.data(), j->dy.data()};
    fftpl_status st = fftpl_create(&j->region, j->n, &cells, &nets, &pins, &j->opt, j->stream,
                                   &j->handle);
    if (st != FFTPL_OK) {
        const char* e = fftpl_last_error(nullptr);
        j->err = e ? e : "fftpl_create failed";
        return st;
    }
    st = serve_prepare(*j->handle, j->x0.data(), j->y0.data(), j->iters);
    if (st != FFTPL_OK) {
        j->err = j->handle->last_error;
        return st;
    }
    j->dev_bytes = fftpl_device_bytes(j->handle);
    return FFTPL_OK;
}

// Copies a finished job's result to the host and frees its device
// resources (worker thread; waits for the job's own stream only).
fftpl_status retire_job(Job* j) {
    Ctx& c = *j->handle;
    cudaStream_t s = j->stream;
    const size_t m = (size_t)j->m_mov;
    j->xr.resize(m);
    j->yr.resize(m);
    double k = 0.0;
    double r[kRecFields] = {};
    cudaMemcpyAsync(&k, c.ctrl + C_K, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (m) {
        cudaMemcpyAsync(j->xr.data(), c.u, m * sizeof(float), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(j->yr.data(), c.u + m, m * sizeof(float), cudaMemcpyDeviceToHost, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        j->err = "reading the job's result";
        return FFTPL_ECUDA;
    }
    const int last = (int)k - 1;
    if (last >= 0 && last < c.recs_cap) {
        cudaMemcpyAsync(r, c.recs + (size_t)last * kRecFields, sizeof(r), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        j->hpwl = r[1];
        j->tau = r[3];
    }
    j->launched = (int)k;
    if (cudaGetLastError() != cudaSuccess) {
        j->err = "copying a result";
        return FFTPL_ECUDA;
    }
    release(j);
    return FFTPL_OK;
}

void worker_main(fftpl_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->tasks.empty(); });
            if (s->stop && s->tasks.empty()) return;
            j = s->tasks.front();
            s->tasks.pop_front();
        }
        const int ph = j->phase.load();
        if (ph == PH_CREATING) {
            fftpl_status st = create_job(j);
            if (st == FFTPL_OK) drop_inputs(j);
            j->status = st;
            j->phase.store(st == FFTPL_OK ? PH_ACTIVE : PH_FAILED);
        } else if (ph == PH_RETIRING) {
            fftpl_status st = retire_job(j);
            j->status = st;
            j->t_done = s->now();
            j->phase.store(st == FFTPL_OK ? PH_DONE : PH_FAILED);
        }
    }
}

void push_task(fftpl_server* s, Job* j) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->tasks.push_back(j);
    }
    s->cv.notify_one();
}

// A chunk of iterations of an active job: launched on its stream, then
// marked by its event (dry run: complete at once).
fftpl_status launch_chunk(fftpl_server* s, Job* j) {
    const int todo = std::min(s->opt.iters_per_tick, j->iters - j->launched);
    if (!s->opt.dry_run) {
        for (int t = 0; t < todo; ++t) {
            fftpl_status st = loop_iter(*j->handle, true);
            if (st != FFTPL_OK) return st;
        }
        if (cudaEventRecord(j->ev, j->stream) != cudaSuccess) {
            cudaGetLastError();
            return FFTPL_ECUDA;
        }
    }
    j->launched += todo;
    j->in_flight = todo;
    if (j->t_prev < 0.0) j->t_prev = s->now();
    return FFTPL_OK;
}

// 1 when the job's in-flight chunk has completed (dry run: always).
int chunk_done(fftpl_server* s, Job* j, fftpl_status* status) {
    if (s->opt.dry_run) return 1;
    cudaError_t e = cudaEventQuery(j->ev);
    if (e == cudaErrorNotReady) return 0;
    if (e != cudaSuccess) {
        cudaGetLastError();
        *status = fail(s, FFTPL_ECUDA, "a job's iterations failed");
    }
    return 1;
}

void finish(fftpl_server* s, Job* j, bool ok) {
    s->used -= j->held;
    j->held = 0;
    if (ok) {
        s->job_ms.push_back(1e3 * (j->t_done - j->t_submit));
        s->completed++;
        s->last_done = std::max(s->last_done, j->t_done);
    } else {
        s->failed++;
    }
}

}  // namespace

extern "C" {

void fftpl_server_default_options(fftpl_server_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = (size_t)150 << 30;
    o->max_active = 64;
    o->iters_per_tick = 1;
    o->workers = 4;
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
    if (s->opt.max_active < 1 || s->opt.iters_per_tick < 1 || s->opt.hbm_budget_bytes == 0 ||
        s->opt.workers < 0) {
        delete s;
        set_global_error("server options: max_active, iters_per_tick and the budget must be > 0");
        return FFTPL_EINVAL;
    }
    if (!s->opt.dry_run) {
        if (cudaGetDevice(&s->device) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            set_global_error("no CUDA device for the server");
            return FFTPL_ECUDA;
        }
        const int nw = s->opt.workers > 0 ? s->opt.workers : 4;
        for (int k = 0; k < nw; ++k) s->workers.emplace_back(worker_main, s);
    }
    *out = s;
    return FFTPL_OK;
}

void fftpl_server_destroy(fftpl_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (std::thread& t : s->workers) t.join();
    for (Job* j : s->creating) release(j);
    for (Job* j : s->active) release(j);
    for (Job* j : s->retiring) release(j);
    delete s;
}

fftpl_status fftpl_server_set_clock(fftpl_server_t s, double now_s) {
    if (!s) return FFTPL_EINVAL;
    s->injected.store(now_s);
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
    // each iteration replays the job's captured loop graph
    j->opt.use_graphs = 1;
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
    // 1. jobs whose handles the workers finished creating start running
    {
        std::vector<Job*> keep;
        for (Job* j : s->creating) {
            const int ph = j->phase.load();
            if (ph == PH_CREATING) {
                keep.push_back(j);
                continue;
            }
            if (ph == PH_FAILED) {
                release(j);
                finish(s, j, false);
                status = fail(s, j->status, "job creation failed: " + j->err);
                continue;
            }
            // the estimate reserved at admission becomes the actual footprint
            s->used = s->used - j->held + j->dev_bytes;
            j->held = j->dev_bytes;
            j->t_admit = s->now();
            s->active.push_back(j);
        }
        s->creating.swap(keep);
    }
    // 2. admit in arrival order while the budget and the slots allow
    while (!s->queue.empty() &&
           (int)(s->active.size() + s->creating.size()) < s->opt.max_active) {
        Job* j = s->queue.front();
        bool fits = s->used + j->est_bytes <= s->opt.hbm_budget_bytes;
        if (!fits && (!s->active.empty() || !s->creating.empty() || !s->retiring.empty()))
            break;                                // wait for memory to free up
        s->queue.pop_front();
        if (!fits) {                              // larger than the whole budget
            j->phase.store(PH_FAILED);
            s->failed++;
            status = fail(s, FFTPL_ENOMEM, "job exceeds the HBM budget");
            continue;
        }
        s->used += j->est_bytes;
        j->held = j->est_bytes;
        if (s->opt.dry_run) {
            j->dev_bytes = j->est_bytes;
            j->phase.store(PH_ACTIVE);
            j->t_admit = s->now();
            s->active.push_back(j);
        } else {
            j->phase.store(PH_CREATING);
            s->creating.push_back(j);
            push_task(s, j);
        }
    }
    s->peak_bytes = std::max(s->peak_bytes, s->used);
    // 3. every active job: record a completed chunk, launch the next one or
    // hand the job to retirement; no job waits for another
    {
        std::vector<Job*> keep;
        for (Job* j : s->active) {
            if (j->in_flight > 0) {
                if (!chunk_done(s, j, &status)) {
                    keep.push_back(j);
                    continue;
                }
                const double t = s->now();
                s->iter_ms.push_back(1e3 * (t - j->t_prev) / j->in_flight);
                j->t_prev = t;
                j->completed_iters += j->in_flight;
                j->in_flight = 0;
            }
            if (j->launched < j->iters) {
                fftpl_status st = launch_chunk(s, j);
                if (st != FFTPL_OK) {
                    status = fail(s, st, "launching a job's iterations failed");
                    release(j);
                    j->phase.store(PH_FAILED);
                    finish(s, j, false);
                    continue;
                }
                if (s->opt.dry_run) {
                    // a dry chunk completes within the tick that launched it
                    const double t = s->now();
                    s->iter_ms.push_back(1e3 * (t - j->t_prev) / j->in_flight);
                    j->t_prev = t;
                    j->completed_iters += j->in_flight;
                    j->in_flight = 0;
                    if (j->launched < j->iters) {
                        keep.push_back(j);
                        continue;
                    }
                } else {
                    keep.push_back(j);
                    continue;
                }
            }
            // all iterations done
            if (s->opt.dry_run) {
                j->t_done = s->now();
                j->phase.store(PH_DONE);
                finish(s, j, true);
            } else {
                j->phase.store(PH_RETIRING);
                s->retiring.push_back(j);
                push_task(s, j);
            }
        }
        s->active.swap(keep);
    }
    s->peak_active = std::max(s->peak_active, (int32_t)s->active.size());
    // 4. retired jobs release their budget
    {
        std::vector<Job*> keep;
        for (Job* j : s->retiring) {
            const int ph = j->phase.load();
            if (ph == PH_RETIRING) {
                keep.push_back(j);
                continue;
            }
            const bool ok = ph == PH_DONE;
            if (!ok) status = fail(s, j->status, "retiring a job failed: " + j->err);
            finish(s, j, ok);
        }
        s->retiring.swap(keep);
    }
    if (active) *active = (int32_t)(s->active.size() + s->creating.size() + s->retiring.size());
    if (queued) *queued = (int32_t)s->queue.size();
    return status;
}

fftpl_status fftpl_server_job(fftpl_server_t s, int64_t id, fftpl_job_info* info, float* x,
                              float* y) {
    if (!s) return FFTPL_EINVAL;
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return fail(s, FFTPL_EINVAL, "unknown job id");
    Job* j = it->second.get();
    const int ph = j->phase.load();
    // a job finishing on a worker is reported once the tick has seen it
    const bool retiring = std::find(s->retiring.begin(), s->retiring.end(), j) != s->retiring.end();
    const bool creating = std::find(s->creating.begin(), s->creating.end(), j) != s->creating.end();
    int32_t state = FFTPL_JOB_QUEUED;
    if (ph == PH_FAILED && !creating && !retiring) state = FFTPL_JOB_FAILED;
    else if (ph == PH_DONE && !retiring) state = FFTPL_JOB_DONE;
    else if (ph == PH_ACTIVE || ph == PH_RETIRING || retiring || (ph != PH_QUEUED && creating))
        state = FFTPL_JOB_ACTIVE;
    if (info) {
        info->id = j->id;
        info->state = state;
        info->iters_done = state == FFTPL_JOB_DONE ? j->launched : j->completed_iters;
        info->m_mov = j->m_mov;
        info->n = j->n;
        info->t_submit = j->t_submit;
        info->t_admit = j->t_admit;
        info->t_done = j->t_done;
        info->hpwl = j->hpwl;
        info->tau = j->tau;
        info->device_bytes = state == FFTPL_JOB_ACTIVE ? j->held : j->dev_bytes;
    }
    if ((x || y) && state == FFTPL_JOB_DONE && !s->opt.dry_run) {
        if (x) std::copy(j->xr.begin(), j->xr.end(), x);
        if (y) std::copy(j->yr.begin(), j->yr.end(), y);
    } else if ((x || y) && state != FFTPL_JOB_DONE) {
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
    o->active = (int32_t)(s->active.size() + s->creating.size() + s->retiring.size());
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
