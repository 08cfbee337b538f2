// C ABI of libfftpl (include/fftpl.h): validation, resource management and
// the orchestration of one objective-gradient evaluation.
//
// One evaluation (Algorithm 1: f, density, FFT solve, gradient) runs as
//   main stream: zero sums, zero D, scatter -> rows_fwd -> cols -> rows_inv
//   side stream: (zero gW) -> WA                       (forked, concurrent)
//   main stream: join -> cells (gather + pin sums + norms)
// (with host outputs the WA branch writes grad W~ itself and the main
// stream ends with the field gather before the join)
// and, when use_graphs is set, is replayed from a captured CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "fftpl_internal.cuh"
#include "loop_ctrl.cuh"

using namespace fftpl;

namespace {

thread_local std::string g_create_error;
std::atomic<int> g_fail_after{0};

struct Fail {
    fftpl_status st;
};

#define CK(call)                                                                    \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            c.last_error = std::string(#call) + ": " + cudaGetErrorString(e_);      \
            return (e_ == cudaErrorMemoryAllocation) ? FFTPL_ENOMEM : FFTPL_ECUDA;  \
        }                                                                           \
    } while (0)

fftpl_status set_err(Ctx& c, fftpl_status st, const std::string& msg) {
    c.last_error = msg;
    return st;
}

// Device memory of every handle comes from one stream-ordered pool per
// device that keeps freed blocks for reuse (release threshold: never), so
// that creating and destroying handles allocates with cudaMallocFromPoolAsync
// and frees with cudaFreeAsync on the handle's stream: no call here waits
// for the whole device (cudaMalloc / cudaFree synchronise it), and a server
// retiring one job does not stall the others.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};

cudaError_t device_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = ~0ULL;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// The small pinned host mirror of a handle's FP64 sums, from a process-wide
// arena (page-locked allocations and frees synchronise the device, so the
// slots are recycled instead).
constexpr size_t kHostSlot = kAccDoubles * sizeof(double);
std::mutex g_host_mu;
std::vector<double*> g_host_free;

cudaError_t host_slot(double** p) {
    std::lock_guard<std::mutex> lk(g_host_mu);
    if (g_host_free.empty()) {
        constexpr int kSlots = 256;
        char* block = nullptr;
        cudaError_t e = cudaMallocHost((void**)&block, kSlots * kHostSlot);
        if (e != cudaSuccess) return e;
        for (int k = kSlots - 1; k >= 0; --k)
            g_host_free.push_back(reinterpret_cast<double*>(block + k * kHostSlot));
    }
    *p = g_host_free.back();
    g_host_free.pop_back();
    return cudaSuccess;
}

void host_slot_release(double* p) {
    std::lock_guard<std::mutex> lk(g_host_mu);
    g_host_free.push_back(p);
}

template <typename T>
fftpl_status dalloc(Ctx& c, T** p, size_t count) {
    *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    int k = g_fail_after.load();
    if (k > 0) {
        if (g_fail_after.fetch_sub(1) == 1) {
            return set_err(c, FFTPL_ENOMEM, "injected allocation failure");
        }
    }
    cudaError_t e = pool_alloc((void**)p, bytes, c.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, FFTPL_ENOMEM,
                       std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
    }
    c.dev_allocs.push_back((void*)*p);
    c.dev_bytes += bytes;
    return FFTPL_OK;
}

// Device temporaries of one create call, freed (in stream order) when it
// returns.
struct TempDev {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit TempDev(cudaStream_t st) : s(st) {}
    ~TempDev() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        *p = nullptr;
        cudaError_t e = pool_alloc((void**)p, std::max<size_t>(count, 1) * sizeof(T), s);
        if (e == cudaSuccess) ptrs.push_back((void*)*p);
        else cudaGetLastError();
        return e;
    }
};

#define TRY(x)                              \
    do {                                    \
        fftpl_status s_ = (x);              \
        if (s_ != FFTPL_OK) return s_;      \
    } while (0)

bool finite_pos(float v) { return isfinite(v) && v > 0.0f; }

// Waits for the handle's own streams only, then returns its device memory
// to the pool in stream order.
void free_ctx(fftpl_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->eval_graph) cudaGraphExecDestroy(c->eval_graph);
    if (c->loop_graph) cudaGraphExecDestroy(c->loop_graph);
    for (void* p : c->dev_allocs) cudaFreeAsync(p, c->stream);
    if (!c->dev_allocs.empty() && c->stream) cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    tc_free(*c);
    tcr_free(*c);
    if (c->acc_host) host_slot_release(c->acc_host);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

// ---------------------------------------------------------------- validation
fftpl_status validate(Ctx& c, const fftpl_region* R, int n, const fftpl_cells* cells,
                      const fftpl_nets* nets, const fftpl_pins* pins, const fftpl_options* opt) {
    if (!R || !cells || !nets || !pins) return set_err(c, FFTPL_EINVAL, "null argument");
    if (n < FFTPL_MIN_N || n > FFTPL_MAX_N || (n & (n - 1)) != 0)
        return set_err(c, FFTPL_EINVAL, "n must be a power of two in [16, 4096]");
    if (!(isfinite(R->x0) && isfinite(R->y0) && isfinite(R->x1) && isfinite(R->y1)) ||
        !(R->x1 > R->x0) || !(R->y1 > R->y0))
        return set_err(c, FFTPL_EINVAL, "region must be finite with x1 > x0 and y1 > y0");
    // every bin edge must be exact in float32, computed as x0 + k * wb
    double lo[2] = {R->x0, R->y0}, hi[2] = {R->x1, R->y1};
    for (int a = 0; a < 2; ++a) {
        double step = (hi[a] - lo[a]) / n;
        float lof = (float)lo[a], stf = (float)step;
        if ((double)lof != lo[a] || (double)stf != step)
            return set_err(c, FFTPL_EINVAL, "region corner and bin size must be exact in float32");
        for (int k = 0; k <= n; ++k) {
            volatile float e = lof + (float)k * stf;
            if ((double)e != lo[a] + k * step)
                return set_err(c, FFTPL_EINVAL, "bin edges must be exact in float32");
        }
        if ((double)(float)hi[a] != hi[a])
            return set_err(c, FFTPL_EINVAL, "region corner must be exact in float32");
    }
    if (cells->m_mov < 0 || cells->m_fix < 0) return set_err(c, FFTPL_EINVAL, "negative cell count");
    long long mt = (long long)cells->m_mov + cells->m_fix;
    if (mt > 0 && (!cells->w || !cells->h)) return set_err(c, FFTPL_EINVAL, "null cell sizes");
    if (cells->m_fix > 0 && (!cells->fix_x || !cells->fix_y))
        return set_err(c, FFTPL_EINVAL, "null fixed-cell positions");
    for (long long i = 0; i < mt; ++i)
        if (!finite_pos(cells->w[i]) || !finite_pos(cells->h[i]))
            return set_err(c, FFTPL_EINVAL, "cell sizes must be finite and > 0");
    for (int i = 0; i < cells->m_fix; ++i)
        if (!isfinite(cells->fix_x[i]) || !isfinite(cells->fix_y[i]))
            return set_err(c, FFTPL_EINVAL, "fixed-cell positions must be finite");
    if (nets->E < 0) return set_err(c, FFTPL_EINVAL, "negative net count");
    if (pins->P < 0 || pins->P > 0x7fffffffLL) return set_err(c, FFTPL_EINVAL, "bad pin count");
    if (!nets->net_ptr) return set_err(c, FFTPL_EINVAL, "null net_ptr");
    if (nets->net_ptr[0] != 0 || (long long)nets->net_ptr[nets->E] != pins->P)
        return set_err(c, FFTPL_EINVAL, "net_ptr must start at 0 and end at P");
    for (int e = 0; e < nets->E; ++e)
        if (nets->net_ptr[e + 1] < nets->net_ptr[e])
            return set_err(c, FFTPL_EINVAL, "net_ptr must be non-decreasing");
    if (pins->P > 0 && (!pins->pin_cell || !pins->dx || !pins->dy))
        return set_err(c, FFTPL_EINVAL, "null pin arrays");
    for (long long p = 0; p < pins->P; ++p) {
        if (pins->pin_cell[p] < 0 || pins->pin_cell[p] >= mt)
            return set_err(c, FFTPL_EINVAL, "pin_cell out of range");
        if (!isfinite(pins->dx[p]) || !isfinite(pins->dy[p]))
            return set_err(c, FFTPL_EINVAL, "pin offsets must be finite");
    }
    if (opt) {
        if (!(opt->target_density > 0.0) || !isfinite(opt->target_density))
            return set_err(c, FFTPL_EINVAL, "target_density must be > 0");
        if (opt->solve_path != FFTPL_SOLVE_FFT && opt->solve_path != FFTPL_SOLVE_TC_BF16X3 &&
            opt->solve_path != FFTPL_SOLVE_TC_RADIX)
            return set_err(c, FFTPL_EINVAL, "unknown solve_path");
        if (opt->solve_path == FFTPL_SOLVE_TC_BF16X3 && n < FFTPL_TC_MIN_N)
            return set_err(c, FFTPL_EINVAL, "the tensor-core solve path needs n >= 128");
        if (opt->solve_path == FFTPL_SOLVE_TC_RADIX && n < FFTPL_TCR_MIN_N)
            return set_err(c, FFTPL_EINVAL, "the radix tensor-core solve path needs n >= 256");
        if (!(opt->dw_ref > 0.0)) return set_err(c, FFTPL_EINVAL, "dw_ref must be > 0");
        if (opt->wirelength != FFTPL_WL_WA && opt->wirelength != FFTPL_WL_LSE)
            return set_err(c, FFTPL_EINVAL, "unknown wirelength model");
        if (opt->optimizer != FFTPL_OPT_NESTEROV && opt->optimizer != FFTPL_OPT_CG)
            return set_err(c, FFTPL_EINVAL, "unknown optimizer");
        if (!(opt->helmholtz_eps >= 0.0) || !isfinite(opt->helmholtz_eps))
            return set_err(c, FFTPL_EINVAL, "helmholtz_eps must be finite and >= 0");
        if (!(opt->alpha_max_cap_bins >= 0.0) || !isfinite(opt->alpha_max_cap_bins))
            return set_err(c, FFTPL_EINVAL, "alpha_max_cap_bins must be finite and >= 0");
    }
    return FFTPL_OK;
}

// ---------------------------------------------------------------- profiling
void prof_begin(Ctx& c, int stage, cudaStream_t s, int* slot) {
    *slot = -1;
    if (!c.profiling) return;
    if (c.prof_used + 2 > (int)c.prof_ev.size()) {
        // ring full: fold the recorded pairs into the totals
        cudaDeviceSynchronize();
        for (int i = 0; i + 1 < c.prof_used; i += 2) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, c.prof_ev[i], c.prof_ev[i + 1]) == cudaSuccess)
                c.stage_ms[c.prof_stage[i / 2]] += ms;
        }
        c.prof_used = 0;
    }
    *slot = c.prof_used;
    c.prof_stage[c.prof_used / 2] = stage;
    c.stage_launches[stage]++;
    cudaEventRecord(c.prof_ev[c.prof_used], s);
    c.prof_used += 2;
}

void prof_end(Ctx& c, int slot, cudaStream_t s) {
    if (slot < 0) return;
    cudaEventRecord(c.prof_ev[slot + 1], s);
}

struct Stage {
    Ctx& c;
    cudaStream_t s;
    int slot;
    Stage(Ctx& c_, int id, cudaStream_t s_) : c(c_), s(s_) { prof_begin(c, id, s, &slot); }
    ~Stage() { prof_end(c, slot, s); }
};

// Spectral solve of the current D (and M) into psi and E2, with the overflow,
// charge and energy sums: stages 1-3 of the profile.
fftpl_status enqueue_solve(Ctx& c, cudaStream_t s) {
    if (c.tcr) {
        { Stage st(c, 1, s); CK(launch_tcr(c, 0, s)); }
        { Stage st(c, 2, s); CK(launch_tcr(c, 1, s)); }
        { Stage st(c, 3, s); CK(launch_tcr(c, 2, s)); }
    } else if (c.tc) {
        { Stage st(c, 1, s); CK(launch_tc(c, 0, s)); CK(launch_tc(c, 1, s)); }
        { Stage st(c, 2, s); CK(launch_tc(c, 2, s)); }
        { Stage st(c, 3, s); CK(launch_tc(c, 3, s)); }
    } else {
        { Stage st(c, 1, s); CK(launch_rows_fwd(c, s)); }
        { Stage st(c, 2, s); CK(launch_cols_spectral(c, s)); }
        { Stage st(c, 3, s); CK(launch_rows_inv(c, s)); }
    }
    return FFTPL_OK;
}

// The overflow and charge sums of the current D alone.
cudaError_t launch_tau(Ctx& c, cudaStream_t s) {
    if (c.tcr) return launch_tcr(c, 3, s);
    return c.tc ? launch_tc(c, 0, s) : launch_rows_fwd(c, s);
}

// ---------------------------------------------------------------- evaluation
// EV_HOST: the gradient arrays are pinned host memory written over the link
enum { EV_DENSITY = 1, EV_WA = 2, EV_ADJOINT = 4, EV_NO_GATHER = 8, EV_HOST = 16 };

// Enqueues one evaluation; gradients must be non-null device arrays.
// stage (2 m_mov floats, or null): x, y may be pinned host memory; the
// scatter reads them once and leaves a device copy there for the later
// kernels.
fftpl_status enqueue_eval(Ctx& c, const float* x, const float* y, float gamma, int what,
                          float* gNx, float* gNy, float* gWx, float* gWy,
                          float* stage = nullptr) {
    cudaStream_t s = c.stream;
    size_t nn = (size_t)c.n * c.n;
    CK(cudaMemsetAsync(c.acc, 0, kAccDoubles * sizeof(double), s));
    bool dens = (what & EV_DENSITY) != 0, wa = (what & EV_WA) != 0;
    const bool grads = !(what & EV_NO_GATHER);
    // with both branches the scatter also writes the WA kernel's positions,
    // and the WA branch forks after it.  Device outputs: after the join one
    // cell kernel writes both gradients (measured 18 % faster than a
    // separate WA gradient pass beside the chain).  Host outputs (and the
    // other combinations): the WA branch ends with its own gradient pass, so
    // that its writes over the host link overlap the density chain (5 %
    // faster end to end).
    const bool pos_from_scatter = dens && wa;
    const bool fused = dens && wa && grads && !(what & (EV_ADJOINT | EV_HOST));
    auto wa_branch = [&](bool interleave) -> fftpl_status {
        CK(cudaEventRecord(c.ev_fork, s));
        CK(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
        {
            Stage st(c, 4, c.side);
            if (!c.opt.deterministic)
                CK(cudaMemsetAsync(c.gW2, 0, (size_t)c.m_mov * sizeof(float2), c.side));
            CK(launch_wa_impl(c, x, y, gamma, nullptr, nullptr, interleave, c.side));
            if (grads && !fused) CK(launch_pin_sum(c, gWx, gWy, c.side));
        }
        CK(cudaEventRecord(c.ev_join, c.side));
        return FFTPL_OK;
    };
    if (wa && !pos_from_scatter) TRY(wa_branch(true));
    if (dens) {
        {
            Stage st(c, 0, s);
            if (c.opt.deterministic) CK(cudaMemsetAsync(c.Dq, 0, nn * sizeof(long long), s));
            else CK(cudaMemsetAsync(c.D, 0, nn * sizeof(float), s));
            CK(launch_scatter_mov(c, x, y, pos_from_scatter, stage, s));
        }
        if (pos_from_scatter) TRY(wa_branch(false));
        TRY(enqueue_solve(c, s));
    }
    const float* xs = stage ? stage : x;
    const float* ys = stage ? stage + c.m_mov : y;
    if (fused) {
        CK(cudaStreamWaitEvent(s, c.ev_join, 0));
        Stage st(c, 5, s);
        CK(launch_cells(c, xs, ys, gNx, gNy, gWx, gWy, s));
    } else {
        if (dens && grads) {
            if ((what & EV_ADJOINT) && !c.tc) CK(launch_rows_psi(c, s));
            Stage st(c, 5, s);
            CK(launch_gather(c, xs, ys, gNx, gNy, (what & EV_ADJOINT) != 0, s));
        }
        if (wa) CK(cudaStreamWaitEvent(s, c.ev_join, 0));
    }
    c.rho_valid = false;
    c.split_valid = false;
    c.fields_valid = dens;
    // the tensor-core solve writes psi; the adjoint gather formed it above
    c.psi_valid = dens && (c.tc != nullptr || (what & EV_ADJOINT));
    return FFTPL_OK;
}

// psi for the current fields: the transform path forms it from PT on demand.
fftpl_status ensure_psi(Ctx& c, cudaStream_t s) {
    if (!c.psi_valid) {
        CK(launch_rows_psi(c, s));
        c.psi_valid = true;
    }
    return FFTPL_OK;
}

// total of one striped accumulator
double acc_total(const double* acc, int q) {
    double s = 0.0;
    for (int k = 0; k < kAccStripes; ++k) s += acc[k * kAccStride + q];
    return s;
}

void fill_report(const Ctx& c, const double* acc, fftpl_eval_report* rep) {
    rep->N = 0.5 * c.Ab * acc_total(acc, ACC_N);
    rep->W = acc_total(acc, ACC_W);
    rep->hpwl = acc_total(acc, ACC_HPWL);
    rep->tau = c.mov_area > 0 ? acc_total(acc, ACC_TAU) / c.mov_area : 0.0;
    rep->gN_l1 = acc_total(acc, ACC_GN_L1);
    rep->gW_l1 = acc_total(acc, ACC_GW_L1);
    rep->charge = acc_total(acc, ACC_CHARGE);
    rep->mov_area = c.mov_area;
}

fftpl_status read_report(Ctx& c, fftpl_eval_report* rep) {
    CK(cudaMemcpyAsync(c.acc_host, c.acc, kAccDoubles * sizeof(double), cudaMemcpyDeviceToHost,
                       c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (rep) fill_report(c, c.acc_host, rep);
    return FFTPL_OK;
}

// internal gradient scratch for NULL outputs
float* scratch(Ctx& c, int which) { return (which < 2 ? c.gN : c.gW) + (which & 1) * c.m_mov; }

}  // namespace

void fftpl::set_global_error(const std::string& msg) { g_create_error = msg; }

// =========================================================================
extern "C" {

int32_t fftpl_version(void) { return FFTPL_VERSION; }

void fftpl_default_options(fftpl_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->target_density = 1.0;
    o->solve_path = FFTPL_SOLVE_FFT;
    o->deterministic = 0;
    o->lambda0 = 0.0;
    o->gamma_fixed = 0.0;
    o->dw_ref = 3.5e5;
    o->alpha_max0_bins = 0.044;
    o->tau_stop = 0.1;
    o->stop_on_tau = 0;
    o->use_graphs = 0;
    o->wirelength = FFTPL_WL_WA;
    o->optimizer = FFTPL_OPT_NESTEROV;
    o->helmholtz_eps = 0.0;
    o->alpha_max_cap_bins = 16.0;
}

fftpl_status fftpl_fillers(const fftpl_region* R, const fftpl_cells* cells,
                           double target_density, int64_t* count, float* filler_w,
                           float* filler_h) {
    if (!R || !cells || !count || !filler_w || !filler_h || cells->m_mov < 0 ||
        cells->m_fix < 0 || (cells->m_mov + cells->m_fix > 0 && (!cells->w || !cells->h)) ||
        (cells->m_fix > 0 && (!cells->fix_x || !cells->fix_y)) ||
        !(target_density > 0.0) || !std::isfinite(target_density)) {
        set_global_error("fftpl_fillers: null or invalid argument");
        return FFTPL_EINVAL;
    }
    const int m = cells->m_mov, k = cells->m_fix;
    for (int i = 0; i < m + k; ++i)
        if (!finite_pos(cells->w[i]) || !finite_pos(cells->h[i])) {
            set_global_error("fftpl_fillers: cell sizes must be finite and > 0");
            return FFTPL_EINVAL;
        }
    double area = (R->x1 - R->x0) * (R->y1 - R->y0), fixed = 0.0, mov = 0.0, sw = 0.0, sh = 0.0;
    for (int f = 0; f < k; ++f) {
        const double hw = 0.5 * cells->w[m + f], hh = 0.5 * cells->h[m + f];
        const double ox = std::min(R->x1, (double)cells->fix_x[f] + hw) -
                          std::max(R->x0, (double)cells->fix_x[f] - hw);
        const double oy = std::min(R->y1, (double)cells->fix_y[f] + hh) -
                          std::max(R->y0, (double)cells->fix_y[f] - hh);
        if (ox > 0.0 && oy > 0.0) fixed += ox * oy;
    }
    for (int i = 0; i < m; ++i) {
        mov += (double)cells->w[i] * (double)cells->h[i];
        sw += cells->w[i];
        sh += cells->h[i];
    }
    *count = 0;
    *filler_w = 0.0f;
    *filler_h = 0.0f;
    if (m <= 0) return FFTPL_OK;
    const float mw = (float)(sw / m), mh = (float)(sh / m);
    const double fill = target_density * (area - fixed) - mov;
    *filler_w = mw;
    *filler_h = mh;
    if (fill > 0.0) *count = (int64_t)std::floor(fill / ((double)mw * (double)mh));
    return FFTPL_OK;
}

void fftpl_debug_fail_alloc_after(int32_t k) { g_fail_after.store(k > 0 ? k : 0); }

fftpl_status fftpl_debug_transpose_stores(fftpl_t h, int32_t tma) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (tma && !c.spec_maps_ok) return set_err(c, FFTPL_ESTATE, "tensor maps not available");
    CK(cudaStreamSynchronize(c.stream));
    if (c.eval_graph) {
        cudaGraphExecDestroy(c.eval_graph);
        c.eval_graph = nullptr;
    }
    if (c.loop_graph) {
        cudaGraphExecDestroy(c.loop_graph);
        c.loop_graph = nullptr;
    }
    c.spec_tma = tma != 0;
    return FFTPL_OK;
}

fftpl_status fftpl_debug_tc_gemm(const void* a_hi, const void* a_lo, const void* b_hi,
                                 const void* b_lo, int32_t M, int32_t N, int32_t K, float* d,
                                 int32_t nsplit, int32_t no_loads, int32_t* err, void* stream) {
    auto al16 = [](const void* p) { return p && ((uintptr_t)p & 15u) == 0; };
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64 ||
        (nsplit != 1 && nsplit != 3) || !al16(a_hi) || !al16(a_lo) || !al16(b_hi) ||
        !al16(b_lo) || !al16(d) || !err) {
        set_global_error("fftpl_debug_tc_gemm: bad sizes, split or pointers");
        return FFTPL_EINVAL;
    }
    cudaError_t e = tc_debug_gemm(a_hi, a_lo, b_hi, b_lo, M, N, K, d, nsplit, no_loads, err,
                                  (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_global_error(std::string("fftpl_debug_tc_gemm: ") + cudaGetErrorString(e));
        return FFTPL_ECUDA;
    }
    return FFTPL_OK;
}

const char* fftpl_last_error(fftpl_t h) {
    if (!h) return g_create_error.c_str();
    return h->last_error.c_str();
}

// Re-lays the netlist for the WA kernel.
//  1. Internal cell numbers (label rounds on the device, k_setup.cu; then
//     cells ordered by (label, distance, index) with two counting sorts).
//  2. Nets of degree >= 2 ordered by their lowest cell number (counting
//     sort), grouped by degree, largest first, into slabs of up to 32 nets;
//     pin k of slab net j at slot base + 32 k + j.  Degrees kBigMin..kBigMax
//     instead take L = grp_lanes(d) lanes per net, 32 / L nets per slab:
//     pin k of slab net j at base + 32 (k / L) + j L + k % L.  Degree-1 nets
//     have no wirelength and are left out.
//  3. The pin records written in slab layout on the device.
// In deterministic mode also the cell-ordered pin slots (pins of each cell,
// by internal number, contiguous and in net order).
static fftpl_status build_slabs(Ctx& c, const fftpl_nets* nets, const fftpl_pins* pins) {
    const int32_t* np = nets->net_ptr;
    const int32_t* pc = pins->pin_cell;
    const int m = c.m_mov, E = c.E;
    const int64_t P = c.P;
    cudaStream_t s = c.stream;
    TempDev tmp(s);
    int *d_np = nullptr, *d_pc = nullptr, *d_key = nullptr, *d_slot = nullptr,
        *d_lanes = nullptr;
    float *d_dx = nullptr, *d_dy = nullptr;
    CK(tmp.alloc(&d_np, (size_t)E + 1));
    CK(tmp.alloc(&d_pc, (size_t)P));
    CK(tmp.alloc(&d_dx, (size_t)P));
    CK(tmp.alloc(&d_dy, (size_t)P));
    CK(tmp.alloc(&d_key, (size_t)E));
    CK(tmp.alloc(&d_slot, (size_t)E));
    CK(tmp.alloc(&d_lanes, (size_t)E));
    CK(cudaMemcpyAsync(d_np, np, ((size_t)E + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (P > 0) {
        CK(cudaMemcpyAsync(d_pc, pc, (size_t)P * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_dx, pins->dx, (size_t)P * sizeof(float), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_dy, pins->dy, (size_t)P * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    // 1. internal cell numbers
    std::vector<int32_t> rank((size_t)m);
    if (m > 0) {
        int *lab = nullptr, *next = nullptr, *dist = nullptr, *netlab = nullptr;
        CK(tmp.alloc(&lab, (size_t)m));
        CK(tmp.alloc(&next, (size_t)m));
        CK(tmp.alloc(&dist, (size_t)m));
        CK(tmp.alloc(&netlab, (size_t)E));
        CK(launch_label_rounds(m, E, d_np, d_pc, lab, next, dist, netlab, s));
        std::vector<int32_t> hl((size_t)m), hd((size_t)m);
        CK(cudaMemcpyAsync(hl.data(), lab, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hd.data(), dist, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // stable counting sorts: by distance, then by label (unreached cells,
        // label and distance "infinite", last in index order)
        const int nd = kLabelRounds + 2;
        std::vector<int32_t> cnt((size_t)std::max(nd, m + 1) + 1, 0), o1((size_t)m), o2((size_t)m);
        auto dkey = [&](int i) { return hd[i] > kLabelRounds ? kLabelRounds + 1 : hd[i]; };
        auto lkey = [&](int i) { return hl[i] >= m ? m : hl[i]; };
        for (int i = 0; i < m; ++i) cnt[dkey(i) + 1]++;
        for (int k = 0; k < nd; ++k) cnt[k + 1] += cnt[k];
        for (int i = 0; i < m; ++i) o1[cnt[dkey(i)]++] = i;
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int i = 0; i < m; ++i) cnt[lkey(i) + 1]++;
        for (int k = 0; k <= m; ++k) cnt[k + 1] += cnt[k];
        for (int q = 0; q < m; ++q) o2[cnt[lkey(o1[q])]++] = o1[q];
        for (int q = 0; q < m; ++q) rank[o2[q]] = q;
        TRY(dalloc(c, &c.cell_rank, (size_t)m));
        CK(cudaMemcpyAsync(c.cell_rank, rank.data(), (size_t)m * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
    }
    // 2. nets by lowest cell number, then slabs by degree
    std::vector<int32_t> key((size_t)E);
    CK(launch_net_key(m, E, d_np, d_pc, c.cell_rank, d_key, s));
    if (E > 0)
        CK(cudaMemcpyAsync(key.data(), d_key, (size_t)E * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int maxd = 0;
    for (int e = 0; e < E; ++e) maxd = std::max(maxd, np[e + 1] - np[e]);
    std::vector<int32_t> kcnt((size_t)m + 2, 0);
    for (int e = 0; e < E; ++e)
        if (np[e + 1] - np[e] >= 2) kcnt[key[e] + 1]++;
    for (int k = 0; k <= m; ++k) kcnt[k + 1] += kcnt[k];
    std::vector<int32_t> by_key((size_t)kcnt[m + 1]);
    for (int e = 0; e < E; ++e)
        if (np[e + 1] - np[e] >= 2) by_key[kcnt[key[e]]++] = e;
    std::vector<int32_t> dcnt((size_t)maxd + 2, 0);
    for (int e : by_key) dcnt[np[e + 1] - np[e]]++;
    // heaviest slabs first: the long nets start early and overlap with the
    // many short ones instead of forming a tail
    std::vector<int4> slabs;
    std::vector<int64_t> first_slab((size_t)maxd + 1, 0);
    int64_t slots = 0;
    auto lanes_of = [](int d) { return d >= kBigMin && d <= kBigMax ? grp_lanes(d) : 1; };
    for (int d = maxd; d >= 2; --d) {
        first_slab[d] = (int64_t)slabs.size();
        const int L = lanes_of(d), G = 32 / L;
        for (int s0 = 0; s0 < dcnt[d]; s0 += G) {
            slabs.push_back(make_int4((int)slots, d, std::min(G, dcnt[d] - s0), L > 1 ? L : 0));
            slots += 32LL * ((d + L - 1) / L);
        }
    }
    if (slots > 0x7fffffffLL) return set_err(c, FFTPL_EINVAL, "too many pins");
    c.nslabs = (int)slabs.size();
    c.slab_slots = slots;
    std::vector<int32_t> net_slot((size_t)E, -1), net_lanes((size_t)E, 1),
        seen((size_t)maxd + 1, 0);
    for (int e : by_key) {
        const int d = np[e + 1] - np[e], j = seen[d]++, L = lanes_of(d), G = 32 / L;
        net_slot[e] = slabs[(size_t)(first_slab[d] + j / G)].x + (j % G) * L;
        net_lanes[e] = L;
    }
    // the slabs of degree kBigMin..kBigMax first (k_wa_grp), the others
    // after them in the same order (k_wa); the slot layout is unchanged
    auto is_big = [](const int4& sl) { return sl.y >= kBigMin && sl.y <= kBigMax; };
    std::stable_partition(slabs.begin(), slabs.end(), is_big);
    c.nbig = (int)std::count_if(slabs.begin(), slabs.end(), is_big);
    // cell-ordered slots (by internal cell number) for the deterministic
    // reduction
    std::vector<int32_t> cslot;
    int* d_cslot = nullptr;
    if (c.opt.deterministic) {
        std::vector<int32_t> cnt((size_t)m + 1, 0);
        for (int e = 0; e < E; ++e) {
            if (np[e + 1] - np[e] < 2) continue;
            for (int p = np[e]; p < np[e + 1]; ++p)
                if (pc[p] < m) cnt[rank[pc[p]] + 1]++;
        }
        for (int i = 0; i < m; ++i) cnt[i + 1] += cnt[i];
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        cslot.assign((size_t)P, -1);
        for (int e = 0; e < E; ++e) {
            if (np[e + 1] - np[e] < 2) continue;
            for (int p = np[e]; p < np[e + 1]; ++p)
                if (pc[p] < m) cslot[p] = fill[rank[pc[p]]]++;
        }
        CK(cudaMemcpyAsync(c.cell_pin_ptr, cnt.data(), cnt.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
        CK(tmp.alloc(&d_cslot, (size_t)P));
        if (P > 0)
            CK(cudaMemcpyAsync(d_cslot, cslot.data(), (size_t)P * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));
    }
    // 3. pin records in slab layout (padding slots: cell -1, offsets 0)
    const size_t ns = (size_t)std::max<int64_t>(slots, 1);
    TRY(dalloc(c, &c.slabs, std::max<size_t>(slabs.size(), 1)));
    TRY(dalloc(c, &c.pin_cell, ns));
    TRY(dalloc(c, &c.pin_dx, ns));
    TRY(dalloc(c, &c.pin_dy, ns));
    // pxy: scratch of the runtime-degree WA body, which only the slabs above
    // kBigMax use; slots go out heaviest first, so theirs are [0, hi_slots)
    int64_t hi_slots = 0;
    for (const int4& sl : slabs)
        if (sl.y > kBigMax) hi_slots += 32LL * sl.y;
    TRY(dalloc(c, &c.pxy, (size_t)std::max<int64_t>(hi_slots, 1)));
    if (c.opt.deterministic) TRY(dalloc(c, &c.pin_slot, ns));
    if (!slabs.empty())
        CK(cudaMemcpyAsync(c.slabs, slabs.data(), slabs.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c.pin_cell, 0xff, ns * sizeof(int32_t), s));
    CK(cudaMemsetAsync(c.pin_dx, 0, ns * sizeof(float), s));
    CK(cudaMemsetAsync(c.pin_dy, 0, ns * sizeof(float), s));
    if (c.pin_slot) CK(cudaMemsetAsync(c.pin_slot, 0xff, ns * sizeof(int32_t), s));
    if (E > 0) {
        CK(cudaMemcpyAsync(d_slot, net_slot.data(), (size_t)E * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_lanes, net_lanes.data(), (size_t)E * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
    }
    CK(launch_fill_slabs(m, E, d_np, d_pc, d_dx, d_dy, c.cell_rank, c.fix_x, c.fix_y, d_slot,
                         d_lanes, d_cslot, c.pin_cell, c.pin_dx, c.pin_dy, c.pin_slot, s));
    CK(cudaStreamSynchronize(s));
    return FFTPL_OK;
}

static fftpl_status create_impl(Ctx& c, const fftpl_region* R, int32_t n, const fftpl_cells* cells,
                                const fftpl_nets* nets, const fftpl_pins* pins,
                                const fftpl_options* opt, void* stream) {
    TRY(validate(c, R, n, cells, nets, pins, opt));
    if (opt) c.opt = *opt;
    else fftpl_default_options(&c.opt);
    c.n = n;
    c.logn = 0;
    while ((1 << c.logn) < n) c.logn++;
    c.m_mov = cells->m_mov;
    c.m_fix = cells->m_fix;
    c.E = nets->E;
    c.P = pins->P;
    c.x0 = R->x0; c.y0 = R->y0; c.x1 = R->x1; c.y1 = R->y1;
    c.Lx = R->x1 - R->x0;
    c.Ly = R->y1 - R->y0;
    c.wb = c.Lx / n;
    c.hb = c.Ly / n;
    c.Ab = c.wb * c.hb;
    c.grid.n = n;
    c.grid.x0 = (float)c.x0;
    c.grid.y0 = (float)c.y0;
    c.grid.wb = (float)c.wb;
    c.grid.hb = (float)c.hb;
    c.grid.inv_wb = (float)(1.0 / c.wb);
    c.grid.inv_hb = (float)(1.0 / c.hb);
    c.grid.guard = (float)((n + 1) * ldexp(1.0, -20));
    c.mov_area = 0.0;
    for (int i = 0; i < c.m_mov; ++i) c.mov_area += (double)cells->w[i] * (double)cells->h[i];
    for (int e = 0; e < c.E; ++e)
        c.wa_max_degree = std::max(c.wa_max_degree, nets->net_ptr[e + 1] - nets->net_ptr[e]);

    c.stream = (cudaStream_t)stream;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev));
    if (!c.stream) {
        // a blocking stream of our own: ordered with the legacy default
        // stream (implicit synchronisation) yet capturable into graphs
        CK(cudaStreamCreate(&c.own_stream));
        c.stream = c.own_stream;
    }
    CK(cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
    CK(host_slot(&c.acc_host));

    size_t nn = (size_t)n * n;
    int mt = c.m_mov + c.m_fix;
    TRY(dalloc(c, &c.w, mt));
    TRY(dalloc(c, &c.h, mt));
    TRY(dalloc(c, &c.fix_x, c.m_fix));
    TRY(dalloc(c, &c.fix_y, c.m_fix));
    TRY(dalloc(c, &c.M, nn));
    if (c.opt.deterministic) TRY(dalloc(c, &c.Dq, nn));
    else TRY(dalloc(c, &c.D, nn));
    TRY(dalloc(c, &c.T1, nn));
    TRY(dalloc(c, &c.PT, nn));
    TRY(dalloc(c, &c.RT, nn));
    spec_maps_init(c);
    TRY(dalloc(c, &c.psi, nn));
    TRY(dalloc(c, &c.E2, nn));
    TRY(dalloc(c, &c.tw, n));
    TRY(dalloc(c, &c.ph, n + 1));
    TRY(dalloc(c, &c.acc, kAccDoubles));
    TRY(dalloc(c, &c.err, 1));
    TRY(dalloc(c, &c.gN, 2 * (size_t)c.m_mov));
    TRY(dalloc(c, &c.gW, 2 * (size_t)c.m_mov));
    TRY(dalloc(c, &c.gW2, (size_t)c.m_mov));
    TRY(dalloc(c, &c.pos2, (size_t)c.m_mov));
    if (c.opt.deterministic) {
        TRY(dalloc(c, &c.cell_pin_ptr, (size_t)c.m_mov + 1));
        TRY(dalloc(c, &c.gpin, c.P));
    }
    cudaStream_t s = c.stream;
    CK(cudaMemcpyAsync(c.w, cells->w, mt * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c.h, cells->h, mt * sizeof(float), cudaMemcpyHostToDevice, s));
    if (c.m_fix) {
        CK(cudaMemcpyAsync(c.fix_x, cells->fix_x, c.m_fix * sizeof(float), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c.fix_y, cells->fix_y, c.m_fix * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    // transform tables (FP64 on the host, rounded once): FFT twiddles
    // exp(-2 pi i k / n) and cosine-transform twiddles exp(-i pi u / 2n)
    std::vector<float2> tw(n), ph(n + 1);
    for (int k = 0; k < n; ++k) {
        double a = 2.0 * M_PI * k / n;
        tw[k] = make_float2((float)cos(a), (float)-sin(a));
    }
    for (int u = 0; u <= n; ++u) {
        double a = M_PI * u / (2.0 * n);
        ph[u] = make_float2((float)cos(a), (float)-sin(a));
    }
    CK(cudaMemcpyAsync(c.tw, tw.data(), n * sizeof(float2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c.ph, ph.data(), (n + 1) * sizeof(float2), cudaMemcpyHostToDevice, s));
    TRY(build_slabs(c, nets, pins));
    if (c.opt.deterministic) {
        // capacity in blocks of every kernel that reduces on each stream
        long long cap0 = std::max<long long>((long long)n / 4, (2LL * c.m_mov + kCellThreads - 1) / kCellThreads);
        if (c.opt.solve_path == FFTPL_SOLVE_TC_BF16X3)
            cap0 = std::max<long long>(cap0, std::max<long long>((long long)n * n / 1024,
                                                                 (long long)(n / 128) * (n / 128)));
        if (c.opt.solve_path == FFTPL_SOLVE_TC_RADIX)
            cap0 = std::max<long long>(cap0, ((long long)(n / 2) * (n / 2 + 1) + 255) / 256);
        long long cap1 = std::max<long long>(
            ((long long)(c.nslabs - c.nbig) + kWaThreads / 32 - 1) / (kWaThreads / 32),
            ((long long)c.nbig + kWaThreads / 32 - 1) / (kWaThreads / 32));
        cap1 = std::max<long long>(cap1, ((long long)c.m_mov + kCellThreads - 1) / kCellThreads);
        c.det_cap[0] = (int)std::max<long long>(cap0, 1);
        c.det_cap[1] = (int)std::max<long long>(cap1, 1);
        TRY(dalloc(c, &c.det_part, 2 * ((size_t)c.det_cap[0] + c.det_cap[1])));
        TRY(dalloc(c, &c.det_ticket, 4));
        CK(cudaMemsetAsync(c.det_ticket, 0, 4 * sizeof(unsigned), s));
    }
    // fixed-cell map M = rho_t F (Section III-B), order-free int64 sums
    {
        long long* q = nullptr;
        CK(pool_alloc((void**)&q, nn * sizeof(long long), s));
        cudaError_t e = cudaMemsetAsync(q, 0, nn * sizeof(long long), s);
        if (e == cudaSuccess && c.m_fix > 0)
            e = launch_scatter(c, c.fix_x, c.fix_y, c.w + c.m_mov, c.h + c.m_mov, c.m_fix, nullptr, q, s);
        if (e == cudaSuccess) e = launch_q_to_f(q, (float)c.opt.target_density, c.M, (int)nn, s);
        cudaFreeAsync(q, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        CK(e);
    }
    CK(cudaMemsetAsync(c.err, 0, sizeof(int), s));
    prepare_spectral(c.logn);
    if (c.opt.solve_path == FFTPL_SOLVE_TC_BF16X3) {
        uint16_t* block = nullptr;
        TRY(dalloc(c, &block, tc_elems(n)));
        cudaError_t e = tc_setup(c, block, s);
        if (e == cudaErrorInvalidValue)
            return set_err(c, FFTPL_ECUDA, "cuTensorMapEncodeTiled unavailable or failed");
        CK(e);
    }
    if (c.opt.solve_path == FFTPL_SOLVE_TC_RADIX) {
        uint16_t* block = nullptr;
        float2* zv = nullptr;
        TRY(dalloc(c, &block, tcr_elems(n)));
        TRY(dalloc(c, &zv, 2 * nn));
        cudaError_t e = tcr_setup(c, block, zv, s);
        if (e == cudaErrorInvalidValue)
            return set_err(c, FFTPL_ECUDA, "cuTensorMapEncodeTiled unavailable or failed");
        CK(e);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return FFTPL_OK;
}

fftpl_status fftpl_create(const fftpl_region* region, int32_t n, const fftpl_cells* cells,
                          const fftpl_nets* nets, const fftpl_pins* pins, const fftpl_options* opt,
                          void* cuda_stream, fftpl_t* out) {
    if (!out) {
        g_create_error = "null output handle";
        return FFTPL_EINVAL;
    }
    *out = nullptr;
    fftpl_ctx* c = new (std::nothrow) fftpl_ctx();
    if (!c) {
        g_create_error = "host allocation failed";
        return FFTPL_ENOMEM;
    }
    fftpl_status st = create_impl(*c, region, n, cells, nets, pins, opt, cuda_stream);
    if (st != FFTPL_OK) {
        g_create_error = c->last_error;
        free_ctx(c);
        return st;
    }
    g_create_error.clear();
    *out = c;
    return FFTPL_OK;
}

void fftpl_destroy(fftpl_t h) { free_ctx(h); }

size_t fftpl_device_bytes(fftpl_t h) { return h ? h->dev_bytes : 0; }

fftpl_status fftpl_check(fftpl_t h) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    CK(cudaStreamSynchronize(c.stream));
    CK(cudaStreamSynchronize(c.side));
    int err = 0;
    CK(cudaMemcpy(&err, c.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & ERR_TIMEOUT) return set_err(c, FFTPL_ETIMEOUT, "a device wait timed out");
    if (err) return set_err(c, FFTPL_ECUDA, "device error word set");
    return FFTPL_OK;
}

fftpl_status fftpl_density(fftpl_t h, const float* x, const float* y, double* N, float* gx,
                           float* gy) {
    if (!h || (h->m_mov > 0 && (!x || !y))) return h ? set_err(*h, FFTPL_EINVAL, "null positions") : FFTPL_EINVAL;
    Ctx& c = *h;
    TRY(enqueue_eval(c, x, y, 0.0f, EV_DENSITY, gx ? gx : scratch(c, 0), gy ? gy : scratch(c, 1),
                     nullptr, nullptr));
    if (N) {
        fftpl_eval_report r;
        TRY(read_report(c, &r));
        *N = r.N;
    }
    return FFTPL_OK;
}

fftpl_status fftpl_density_adjoint(fftpl_t h, const float* x, const float* y, double* N,
                                   float* gx, float* gy) {
    if (!h || (h->m_mov > 0 && (!x || !y))) return h ? set_err(*h, FFTPL_EINVAL, "null positions") : FFTPL_EINVAL;
    Ctx& c = *h;
    TRY(enqueue_eval(c, x, y, 0.0f, EV_DENSITY | EV_ADJOINT, gx ? gx : scratch(c, 0),
                     gy ? gy : scratch(c, 1), nullptr, nullptr));
    if (N) {
        fftpl_eval_report r;
        TRY(read_report(c, &r));
        *N = r.N;
    }
    return FFTPL_OK;
}

fftpl_status fftpl_energy(fftpl_t h, const float* x, const float* y, double* N) {
    if (!h || (h->m_mov > 0 && (!x || !y))) return h ? set_err(*h, FFTPL_EINVAL, "null positions") : FFTPL_EINVAL;
    Ctx& c = *h;
    TRY(enqueue_eval(c, x, y, 0.0f, EV_DENSITY | EV_NO_GATHER, nullptr, nullptr, nullptr, nullptr));
    if (N) {
        fftpl_eval_report r;
        TRY(read_report(c, &r));
        *N = r.N;
    }
    return FFTPL_OK;
}

fftpl_status fftpl_gather(fftpl_t h, const float* x, const float* y, int32_t mode, float* gx,
                          float* gy) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (c.m_mov > 0 && (!x || !y || !gx || !gy)) return set_err(c, FFTPL_EINVAL, "null argument");
    if (mode != 0 && mode != 1) return set_err(c, FFTPL_EINVAL, "mode must be 0 or 1");
    if (!c.fields_valid) return set_err(c, FFTPL_ESTATE, "no density evaluation yet");
    if (mode == 1) TRY(ensure_psi(c, c.stream));
    CK(launch_gather(c, x, y, gx, gy, mode == 1, c.stream));
    return FFTPL_OK;
}

fftpl_status fftpl_wa(fftpl_t h, const float* x, const float* y, float gamma, double* W,
                      float* gx, float* gy) {
    if (!h || (h->m_mov > 0 && (!x || !y))) return h ? set_err(*h, FFTPL_EINVAL, "null positions") : FFTPL_EINVAL;
    Ctx& c = *h;
    if (!(gamma > 0.0f) || !isfinite(gamma)) return set_err(c, FFTPL_EINVAL, "gamma must be > 0");
    TRY(enqueue_eval(c, x, y, gamma, EV_WA, nullptr, nullptr, gx ? gx : scratch(c, 2),
                     gy ? gy : scratch(c, 3)));
    if (W) {
        fftpl_eval_report r;
        TRY(read_report(c, &r));
        *W = r.W;
    }
    return FFTPL_OK;
}

// One full evaluation through the captured graph when use_graphs is set
// (the graph is keyed by the buffers, gamma and the staging buffer).
static fftpl_status eval_impl(Ctx& c, const float* x, const float* y, float gamma, float* gNx,
                              float* gNy, float* gWx, float* gWy, float* stage) {
    // a staging buffer means x, y and the gradients are pinned host memory
    const int what = EV_DENSITY | EV_WA | (stage ? EV_HOST : 0);
    if (c.opt.use_graphs && !c.profiling) {
        float gk = gamma;
        const void* key[8] = {x, y, gNx, gNy, gWx, gWy, nullptr, stage};
        memcpy(&key[6], &gk, sizeof(float));
        if (!c.eval_graph || memcmp(key, c.graph_key, sizeof(key)) != 0) {
            if (c.eval_graph) {
                cudaGraphExecDestroy(c.eval_graph);
                c.eval_graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
            int64_t before = c.launches;
            fftpl_status st = enqueue_eval(c, x, y, gamma, what, gNx, gNy, gWx, gWy, stage);
            cudaError_t ee = cudaStreamEndCapture(c.stream, &g);
            if (st != FFTPL_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            CK(ee);
            cudaError_t ie = cudaGraphInstantiate(&c.eval_graph, g, 0);
            cudaGraphDestroy(g);
            CK(ie);
            memcpy(c.graph_key, key, sizeof(key));
            c.graph_nkernels = c.launches - before;
            c.launches = before;  // counted at replay
        }
        CK(cudaGraphLaunch(c.eval_graph, c.stream));
        c.launches += c.graph_nkernels;
        c.fields_valid = true;
        c.rho_valid = false;
        c.split_valid = false;
        c.psi_valid = c.tc != nullptr;
        return FFTPL_OK;
    }
    return enqueue_eval(c, x, y, gamma, what, gNx, gNy, gWx, gWy, stage);
}

fftpl_status fftpl_eval(fftpl_t h, const float* x, const float* y, float gamma, float* gNx,
                        float* gNy, float* gWx, float* gWy, fftpl_eval_report* rep) {
    if (!h || (h->m_mov > 0 && (!x || !y))) return h ? set_err(*h, FFTPL_EINVAL, "null positions") : FFTPL_EINVAL;
    Ctx& c = *h;
    if (!(gamma > 0.0f) || !isfinite(gamma)) return set_err(c, FFTPL_EINVAL, "gamma must be > 0");
    gNx = gNx ? gNx : scratch(c, 0);
    gNy = gNy ? gNy : scratch(c, 1);
    gWx = gWx ? gWx : scratch(c, 2);
    gWy = gWy ? gWy : scratch(c, 3);
    TRY(eval_impl(c, x, y, gamma, gNx, gNy, gWx, gWy, nullptr));
    if (rep) TRY(read_report(c, rep));
    return FFTPL_OK;
}

// Device address of pinned (page-locked, mapped) host memory, or null for
// any other pointer (pageable host memory is not handed to kernels).
static void* mapped_host(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

fftpl_status fftpl_eval_host(fftpl_t h, const float* x_host, const float* y_host, float gamma,
                             float* gNx_host, float* gNy_host, float* gWx_host, float* gWy_host,
                             fftpl_eval_report* rep) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (c.m_mov > 0 && (!x_host || !y_host)) return set_err(c, FFTPL_EINVAL, "null positions");
    if (!(gamma > 0.0f) || !isfinite(gamma)) return set_err(c, FFTPL_EINVAL, "gamma must be > 0");
    size_t m = (size_t)c.m_mov;
    if (!c.hx) {
        TRY(dalloc(c, &c.hx, 2 * m));
        TRY(dalloc(c, &c.hg, 4 * m));
        c.hy = c.hx + m;
    }
    cudaStream_t s = c.stream;
    // all six buffers pinned: the kernels read the positions and write the
    // gradients over the host link themselves (the scatter reads x, y once
    // and stages a device copy; the cell kernel writes the gradients), so the
    // transfers overlap the computation instead of preceding and following it
    void* xd = mapped_host(x_host);
    void* yd = mapped_host(y_host);
    void* gd[4] = {mapped_host(gNx_host), mapped_host(gNy_host), mapped_host(gWx_host),
                   mapped_host(gWy_host)};
    if (m > 0 && xd && yd && gd[0] && gd[1] && gd[2] && gd[3]) {
        TRY(eval_impl(c, (const float*)xd, (const float*)yd, gamma, (float*)gd[0], (float*)gd[1],
                      (float*)gd[2], (float*)gd[3], c.hx));
        return read_report(c, rep);
    }
    CK(cudaMemcpyAsync(c.hx, x_host, m * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c.hy, y_host, m * sizeof(float), cudaMemcpyHostToDevice, s));
    TRY(eval_impl(c, c.hx, c.hy, gamma, c.hg, c.hg + m, c.hg + 2 * m, c.hg + 3 * m, nullptr));
    float* outs[4] = {gNx_host, gNy_host, gWx_host, gWy_host};
    for (int k = 0; k < 4; ++k)
        if (outs[k])
            CK(cudaMemcpyAsync(outs[k], c.hg + k * m, m * sizeof(float), cudaMemcpyDeviceToHost, s));
    return read_report(c, rep);
}

fftpl_status fftpl_report(fftpl_t h, fftpl_eval_report* rep) {
    if (!h || !rep) return FFTPL_EINVAL;
    return read_report(*h, rep);
}

fftpl_status fftpl_fields(fftpl_t h, const float** rho, const float** psi, const float** ex,
                          const float** ey) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (!c.fields_valid) return set_err(c, FFTPL_ESTATE, "no density evaluation yet");
    if (rho) {
        if (!c.rho) TRY(dalloc(c, &c.rho, (size_t)c.n * c.n));
        if (!c.rho_valid) {
            CK(launch_rho(c, c.stream));
            c.rho_valid = true;
        }
        *rho = c.rho;
    }
    if (psi) {
        TRY(ensure_psi(c, c.stream));
        *psi = c.psi;
    }
    if (ex || ey) {
        if (!c.ex) {
            TRY(dalloc(c, &c.ex, (size_t)c.n * c.n));
            TRY(dalloc(c, &c.ey, (size_t)c.n * c.n));
        }
        if (!c.split_valid) {
            CK(launch_split_field(c, c.stream));
            c.split_valid = true;
        }
        if (ex) *ex = c.ex;
        if (ey) *ey = c.ey;
    }
    CK(cudaStreamSynchronize(c.stream));
    return FFTPL_OK;
}

fftpl_status fftpl_fields_q(fftpl_t h, const int64_t** q) {
    if (!h || !q) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (!c.opt.deterministic || !c.fields_valid)
        return set_err(c, FFTPL_ESTATE, "no deterministic density evaluation yet");
    CK(cudaStreamSynchronize(c.stream));
    *q = reinterpret_cast<const int64_t*>(c.Dq);
    return FFTPL_OK;
}

fftpl_status fftpl_bin_ranges(fftpl_t h, const float* x, const float* y, int32_t* ranges,
                              int64_t* pairs) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (c.m_mov > 0 && (!x || !y || !ranges)) return set_err(c, FFTPL_EINVAL, "null argument");
    CK(cudaMemsetAsync(c.acc, 0, kAccDoubles * sizeof(double), c.stream));
    CK(launch_bin_ranges(c, x, y, ranges, c.stream));
    CK(cudaMemcpyAsync(c.acc_host, c.acc, kAccDoubles * sizeof(double), cudaMemcpyDeviceToHost,
                       c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (pairs) *pairs = (int64_t)llround(acc_total(c.acc_host, ACC_CHARGE));
    return FFTPL_OK;
}

// ------------------------------------------------------------ placement loop
fftpl_status fftpl_place_init(fftpl_t h, const float* x0, const float* y0) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (c.m_mov <= 0) return set_err(c, FFTPL_EINVAL, "no movable cells to place");
    if (!x0 || !y0) return set_err(c, FFTPL_EINVAL, "null positions");
    size_t m2 = 2 * (size_t)c.m_mov;
    if (!c.u) {
        TRY(dalloc(c, &c.u, m2));
        TRY(dalloc(c, &c.v, m2));
        TRY(dalloc(c, &c.vprev, m2));
        TRY(dalloc(c, &c.g, m2));
        TRY(dalloc(c, &c.gprev, m2));
        TRY(dalloc(c, &c.ctrl, C_COUNT + kCounters));
    }
    std::vector<double> ctrl(C_COUNT + kCounters, 0.0);
    ctrl[C_LAMBDA] = c.opt.lambda0;
    ctrl[C_GAMMA] = c.opt.gamma_fixed;
    ctrl[C_ALPHA_MAX0] = c.opt.alpha_max0_bins * c.wb;
    ctrl[C_ALPHA_MAX] = ctrl[C_ALPHA_MAX0];
    ctrl[C_A] = 1.0;
    ctrl[C_DW_REF] = c.opt.dw_ref;
    ctrl[C_GAMMA_FIXED] = c.opt.gamma_fixed;
    ctrl[C_LAMBDA0_OPT] = c.opt.lambda0;
    ctrl[C_STOP_ON_TAU] = c.opt.stop_on_tau ? 1.0 : 0.0;
    ctrl[C_TAU_STOP] = c.opt.tau_stop;
    ctrl[C_WB] = c.wb;
    ctrl[C_HALF_AB] = 0.5 * c.Ab;
    ctrl[C_MOV_AREA] = c.mov_area > 0 ? c.mov_area : 1.0;
    ctrl[C_ALPHA_CAP] = c.opt.alpha_max_cap_bins * c.wb;
    cudaStream_t s = c.stream;
    ctrl_mirror(ctrl.data());
    CK(cudaMemcpyAsync(c.ctrl, ctrl.data(), ctrl.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(launch_place_init(c, x0, y0, s));
    if (c.opt.gamma_fixed <= 0.0) {
        // gamma_0 from the overflow at the start
        size_t nn = (size_t)c.n * c.n;
        CK(cudaMemsetAsync(c.acc, 0, kAccDoubles * sizeof(double), s));
        if (c.opt.deterministic) CK(cudaMemsetAsync(c.Dq, 0, nn * sizeof(long long), s));
        else CK(cudaMemsetAsync(c.D, 0, nn * sizeof(float), s));
        CK(launch_scatter_mov(c, c.v, c.v + c.m_mov, false, nullptr, s));
        CK(launch_tau(c, s));
        CK(launch_gamma0(c, s));
    }
    CK(cudaStreamSynchronize(s));
    c.placing = true;
    return FFTPL_OK;
}

extern "C++" {
// One evaluation of the loop at the positions in c.v (gamma from the
// control scalars): zero the sums, density chain, WA branch, join; with
// `cells` also the per-cell gradients and lambda_k.
static fftpl_status loop_eval(Ctx& c, bool cells) {
    cudaStream_t s = c.stream;
    size_t nn = (size_t)c.n * c.n;
    const float* vx = c.v;
    const float* vy = c.v + c.m_mov;
    CK(cudaMemsetAsync(c.acc, 0, kAccDoubles * sizeof(double), s));
    {
        Stage st(c, 0, s);
        if (c.opt.deterministic) CK(cudaMemsetAsync(c.Dq, 0, nn * sizeof(long long), s));
        else CK(cudaMemsetAsync(c.D, 0, nn * sizeof(float), s));
        CK(launch_scatter_mov(c, vx, vy, true, nullptr, s));
    }
    // the WA branch forks after the scatter, which wrote its positions
    CK(cudaEventRecord(c.ev_fork, s));
    CK(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
    {
        Stage st(c, 4, c.side);
        if (!c.opt.deterministic)
            CK(cudaMemsetAsync(c.gW2, 0, (size_t)c.m_mov * sizeof(float2), c.side));
        CK(launch_wa_impl(c, vx, vy, 1.0f, ctrl_f(c.ctrl) + F_INV_G, ctrl_f(c.ctrl) + F_DONE,
                          false, c.side));
    }
    CK(cudaEventRecord(c.ev_join, c.side));
    TRY(enqueue_solve(c, s));
    CK(cudaStreamWaitEvent(s, c.ev_join, 0));
    if (cells) {
        Stage st(c, 5, s);
        CK(launch_loop_cells(c, s));
    }
    return FFTPL_OK;
}

fftpl_status fftpl::loop_enqueue(Ctx& c) {
    cudaStream_t s = c.stream;
    TRY(loop_eval(c, true));
    if (c.opt.optimizer == FFTPL_OPT_CG) {
        {
            Stage st(c, 6, s);
            CK(launch_cg_g(c, s));
            CK(launch_cg_dir(c, s));
            CK(launch_cg_trial(c, s));
        }
        TRY(loop_eval(c, false));   // f at the trial point
        Stage st(c, 6, s);
        CK(launch_cg_alpha(c, s));
        CK(launch_cg_update(c, s));
        return FFTPL_OK;
    }
    Stage st(c, 6, s);
    CK(launch_loop_g(c, s));
    CK(launch_loop_update(c, s));
    return FFTPL_OK;
}

// One loop iteration: replayed from a graph captured on first use when
// use_graphs is set (every other input of the iteration lives on the device:
// the control scalars, positions and the record counter).
fftpl_status fftpl::loop_iter(Ctx& c, bool launch) {
    if (!c.opt.use_graphs || c.profiling) return launch ? loop_enqueue(c) : FFTPL_OK;
    const void* key[3] = {c.recs, c.gN, c.gW};
    if (!c.loop_graph || memcmp(key, c.loop_key, sizeof(key)) != 0) {
        if (c.loop_graph) {
            cudaGraphExecDestroy(c.loop_graph);
            c.loop_graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        int64_t before = c.launches;
        fftpl_status st = loop_enqueue(c);
        cudaError_t ee = cudaStreamEndCapture(c.stream, &g);
        if (st != FFTPL_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        CK(ee);
        cudaError_t ie = cudaGraphInstantiate(&c.loop_graph, g, 0);
        cudaGraphDestroy(g);
        CK(ie);
        memcpy(c.loop_key, key, sizeof(key));
        c.loop_graph_nkernels = c.launches - before;
        c.launches = before;  // counted at replay
    }
    if (!launch) return FFTPL_OK;
    CK(cudaGraphLaunch(c.loop_graph, c.stream));
    c.launches += c.loop_graph_nkernels;
    return FFTPL_OK;
}

fftpl_status fftpl::serve_prepare(Ctx& c, const float* x0, const float* y0, int iters) {
    const size_t m = (size_t)c.m_mov;
    if (!c.hx) {
        TRY(dalloc(c, &c.hx, 2 * m));
        c.hy = c.hx + m;
    }
    if (m) {
        CK(cudaMemcpyAsync(c.hx, x0, m * sizeof(float), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(c.hy, y0, m * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    }
    TRY(fftpl_place_init(&static_cast<fftpl_ctx&>(c), c.hx, c.hy));
    TRY(loop_records(c, iters, 0.0));
    TRY(loop_iter(c, false));
    CK(cudaStreamSynchronize(c.stream));
    return FFTPL_OK;
}

fftpl_status fftpl::loop_records(Ctx& c, int cap, double base_k) {
    if (c.recs_cap < std::max(cap, 1)) {
        if (c.recs) {
            cudaFreeAsync(c.recs, c.stream);
            c.dev_allocs.erase(std::find(c.dev_allocs.begin(), c.dev_allocs.end(), (void*)c.recs));
            c.dev_bytes -= (size_t)c.recs_cap * kRecFields * sizeof(double);
            c.recs = nullptr;
        }
        TRY(dalloc(c, &c.recs, (size_t)std::max(cap, 1) * kRecFields));
        c.recs_cap = std::max(cap, 1);
    }
    double hdr[2] = {(double)cap, base_k};
    CK(cudaMemcpyAsync(c.ctrl + C_REC_CAP, hdr, sizeof(hdr), cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return FFTPL_OK;
}

}  // extern "C++"

fftpl_status fftpl_step(fftpl_t h, int32_t iters, fftpl_iter_record* recs, int32_t* ran) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (!c.placing) return set_err(c, FFTPL_ESTATE, "call fftpl_place_init first");
    if (iters < 0) return set_err(c, FFTPL_EINVAL, "iters must be >= 0");
    double k0 = 0.0;
    CK(cudaMemcpyAsync(&k0, c.ctrl + C_K, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    TRY(loop_records(c, iters, k0));
    // with the stop test on, enqueue in chunks and look at the device's
    // stop flag between them, so that a run that stops early does not keep
    // its remaining iterations' kernels in the queue
    constexpr int kChunk = 16;
    for (int it = 0; it < iters; it += kChunk) {
        for (int j = it; j < std::min(iters, it + kChunk); ++j) TRY(loop_iter(c, true));
        if (c.opt.stop_on_tau && it + kChunk < iters) {
            double done = 0.0;
            CK(cudaMemcpyAsync(&done, c.ctrl + C_DONE, sizeof(double), cudaMemcpyDeviceToHost,
                               c.stream));
            CK(cudaStreamSynchronize(c.stream));
            if (done != 0.0) break;
        }
    }
    double k1 = 0.0;
    CK(cudaMemcpyAsync(&k1, c.ctrl + C_K, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    int done = (int)(k1 - k0);
    if (ran) *ran = done;
    if (recs && done > 0) {
        std::vector<double> tmp((size_t)done * kRecFields);
        CK(cudaMemcpy(tmp.data(), c.recs, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int k = 0; k < done; ++k) {
            const double* r = tmp.data() + (size_t)k * kRecFields;
            recs[k].W = r[0]; recs[k].hpwl = r[1]; recs[k].N = r[2]; recs[k].tau = r[3];
            recs[k].lambda = r[4]; recs[k].gamma = r[5]; recs[k].alpha = r[6];
            recs[k].step_max = r[7];
        }
    }
    c.fields_valid = true;
    c.rho_valid = false;
    c.split_valid = false;
    c.psi_valid = c.tc != nullptr;
    return FFTPL_OK;
}

fftpl_status fftpl_place_positions(fftpl_t h, float* x, float* y) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (!c.placing) return set_err(c, FFTPL_ESTATE, "no placement run");
    size_t m = (size_t)c.m_mov;
    CK(cudaMemcpyAsync(x, c.u, m * sizeof(float), cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaMemcpyAsync(y, c.u + m, m * sizeof(float), cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return FFTPL_OK;
}

// state layout: magic, m, then u, v, vprev, g, gprev (2m float each), ctrl
static const uint64_t kStateMagic = 0x4646545053544154ULL;  // "FFTPSTAT"

fftpl_status fftpl_state_save(fftpl_t h, void* buf, size_t* bytes) {
    if (!h || !bytes) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (!c.placing) return set_err(c, FFTPL_ESTATE, "no placement run");
    size_t m2 = 2 * (size_t)c.m_mov;
    size_t need = 2 * sizeof(uint64_t) + 5 * m2 * sizeof(float) + C_COUNT * sizeof(double);
    if (!buf) {
        *bytes = need;
        return FFTPL_OK;
    }
    if (*bytes < need) return set_err(c, FFTPL_EINVAL, "state buffer too small");
    char* p = (char*)buf;
    uint64_t hdr[2] = {kStateMagic, (uint64_t)c.m_mov};
    memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    CK(cudaStreamSynchronize(c.stream));
    float* vecs[5] = {c.u, c.v, c.vprev, c.g, c.gprev};
    for (float* v : vecs) {
        CK(cudaMemcpy(p, v, m2 * sizeof(float), cudaMemcpyDeviceToHost));
        p += m2 * sizeof(float);
    }
    CK(cudaMemcpy(p, c.ctrl, C_COUNT * sizeof(double), cudaMemcpyDeviceToHost));
    *bytes = need;
    return FFTPL_OK;
}

fftpl_status fftpl_state_load(fftpl_t h, const void* buf, size_t bytes) {
    if (!h || !buf) return FFTPL_EINVAL;
    Ctx& c = *h;
    size_t m2 = 2 * (size_t)c.m_mov;
    size_t need = 2 * sizeof(uint64_t) + 5 * m2 * sizeof(float) + C_COUNT * sizeof(double);
    if (bytes < need) return set_err(c, FFTPL_EINVAL, "state buffer too small");
    const char* p = (const char*)buf;
    uint64_t hdr[2];
    memcpy(hdr, p, sizeof(hdr));
    if (hdr[0] != kStateMagic || hdr[1] != (uint64_t)c.m_mov)
        return set_err(c, FFTPL_EINVAL, "state does not match this instance");
    p += sizeof(hdr);
    if (!c.u) {
        TRY(dalloc(c, &c.u, m2));
        TRY(dalloc(c, &c.v, m2));
        TRY(dalloc(c, &c.vprev, m2));
        TRY(dalloc(c, &c.g, m2));
        TRY(dalloc(c, &c.gprev, m2));
        TRY(dalloc(c, &c.ctrl, C_COUNT + kCounters));
    }
    CK(cudaStreamSynchronize(c.stream));
    float* vecs[5] = {c.u, c.v, c.vprev, c.g, c.gprev};
    for (float* v : vecs) {
        CK(cudaMemcpy(v, p, m2 * sizeof(float), cudaMemcpyHostToDevice));
        p += m2 * sizeof(float);
    }
    CK(cudaMemcpy(c.ctrl, p, C_COUNT * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemset(c.ctrl + C_COUNT, 0, kCounters * sizeof(double)));
    c.placing = true;
    return FFTPL_OK;
}

// ------------------------------------------------------------ measurement
fftpl_status fftpl_set_profiling(fftpl_t h, int32_t on) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    if (on && c.prof_ev.empty()) {
        const int pairs = 4096;
        c.prof_ev.resize(2 * pairs);
        c.prof_stage.resize(pairs);
        for (auto& e : c.prof_ev) CK(cudaEventCreate(&e));
    }
    c.profiling = on != 0;
    return FFTPL_OK;
}

fftpl_status fftpl_stage_times(fftpl_t h, double* ms, int64_t* launches, int32_t reset) {
    if (!h) return FFTPL_EINVAL;
    Ctx& c = *h;
    CK(cudaStreamSynchronize(c.stream));
    CK(cudaStreamSynchronize(c.side));
    for (int i = 0; i + 1 < c.prof_used; i += 2) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, c.prof_ev[i], c.prof_ev[i + 1]));
        c.stage_ms[c.prof_stage[i / 2]] += t;
    }
    c.prof_used = 0;
    for (int k = 0; k < FFTPL_NUM_STAGES; ++k) {
        if (ms) ms[k] = c.stage_ms[k];
        if (launches) launches[k] = c.stage_launches[k];
        if (reset) {
            c.stage_ms[k] = 0.0;
            c.stage_launches[k] = 0;
        }
    }
    return FFTPL_OK;
}

int64_t fftpl_launch_count(fftpl_t h) { return h ? h->launches : 0; }

}  // extern "C"
