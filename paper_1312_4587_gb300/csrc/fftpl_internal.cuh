// Internal declarations shared by the libfftpl translation units.
//
// Layout in device memory (all float32 unless noted, row-major [n][n] maps
// with x fastest):
//   movable cells   w, h                       (m_mov)
//   fixed cells     fix_x, fix_y (m_fix)       macro map M = rho_t F  [n][n]
//   density         D (movable overlap area, float) or Dq (int64, 2^-32 units)
//   spectral        T1 [u][y]  (rows transformed along x, stored transposed)
//                   PT [y][u], RT [y][u]  (columns transformed and inverted)
//                   psi, ex, ey [y][x], rho [y][x] (formed on demand)
//   nets/pins       slabs of nets of equal degree; pin_cell, pin_dx, pin_dy,
//                   pin_slot in slab order (slot base + 32 k + lane);
//                   cell_pin_ptr (m_mov+1), gpin (float2 per pin) for the
//                   deterministic pin-to-cell reduction; gW2 (float2, m_mov)
//                   the atomic one
//   accumulators    acc[ACC_*] doubles, err word
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fftpl.h"

namespace fftpl {

// ------------------------------------------------------------------ sizes
constexpr int kSpecThreads = 256;   // threads of the transform kernels
constexpr int kSpecBuffers = 4;     // complex length-n buffers per CTA
constexpr int kCellThreads = 256;
constexpr int kWaThreads = 256;
// Nets of degree kBigMin..kBigMax go to the WA kernel with several lanes per
// net (k_wa_grp, grp_lanes(d) lanes each, at most 4 pins per lane); the rest
// to k_wa (one lane per net).
constexpr int kBigMin = 7;
constexpr int kBigMax = 64;
__host__ __device__ constexpr int grp_lanes(int d) {
    return d <= 8 ? 2 : (d <= 16 ? 4 : (d <= 32 ? 8 : 16));
}

// accumulator slots (FP64 sums written by the kernels)
enum {
    ACC_N = 0,      // sum B * Psi (times A_b/2 on the host)
    ACC_W,          // WA wirelength
    ACC_HPWL,
    ACC_TAU,        // overflow numerator
    ACC_GN_L1,
    ACC_GW_L1,
    ACC_CHARGE,     // sum (D + M) (times A_b... area units already)
    ACC_DV2,        // ||v_k - v_{k-1}||^2
    ACC_DG2,        // ||g_k - g_{k-1}||^2
    ACC_GINF,       // ||g_k||_inf (as ordered bits of a non-negative double)
    ACC_STEPMAX,    // max |u_{k+1} - v_k|
    ACC_GD,         // g_k . d_k (conjugate-gradient loop)
    ACC_DINF,       // ||d_k||_inf (conjugate-gradient loop)
    ACC_COUNT
};

// The FP64 sums are striped: a block adds its total to stripe
// (blockIdx & 31), one 128-byte line of kAccStride doubles per stripe, so no
// single address takes every block's atomic; readers add the stripes.
constexpr int kAccStripes = 32;
constexpr int kAccStride = 16;
constexpr int kAccDoubles = kAccStripes * kAccStride;
static_assert(ACC_COUNT <= kAccStride, "accumulator stripe too small");

// device error word bits
enum { ERR_TIMEOUT = 1, ERR_BOUNDS = 2 };

// Bin grid along both axes.  Edges e_k = x0 + k * wb are exact in float32
// (checked at create), so comparisons against them decide indices exactly.
// guard: see last_edge (1 = always take the exact comparisons).
struct Grid {
    int n;
    float x0, y0, wb, hb, inv_wb, inv_hb;
    float guard = 1.0f;
};

__device__ __forceinline__ float edge_at(float lo, float step, int k) {
    return __fadd_rn(lo, __fmul_rn((float)k, step));
}

// Largest k in [-1, n] with e_k <= t (strict: e_k < t).  The float estimate
// q = (t - x0) * (1/w_b) is within one of the answer (its relative error is a
// few 2^-24 and the quotient is at most n + 1 after clamping), so one
// comparison against the exact edges in each direction settles the index.
// Fast path: where 0 <= floor(q) < n and q lies at least `guard` bins from
// both neighbouring integers, floor(q) is the answer without comparisons:
// the edges are exact and q differs from (t - x0) / w_b by at most
// n 2^-22 bins there, below guard = (n + 1) 2^-20 (q - floor(q) is exact).
template <bool STRICT>
__device__ __forceinline__ int last_edge(float lo, float step, float inv, float guard, int n,
                                         float t) {
    const float q = __fmul_rn(__fsub_rn(t, lo), inv);
    float kf = floorf(q);
    const float fr = q - kf;
    if (kf >= 0.0f && kf < (float)n && fr >= guard && fr <= 1.0f - guard) return (int)kf;
    int k;
    if (!(kf >= -1.0f)) k = -1;          // also catches NaN
    else if (kf > (float)n) k = n;
    else k = (int)kf;
    if (k < n) {
        float e = edge_at(lo, step, k + 1);
        if (STRICT ? (e < t) : (e <= t)) return k + 1;
    }
    if (k >= 0) {
        float e = edge_at(lo, step, k);
        if (!(STRICT ? (e < t) : (e <= t))) return k - 1;
    }
    return k;
}

struct Span {
    float xl, xh, yl, yh;   // float32 cell edges
    int ilo, ihi, jlo, jhi; // clamped bin span (empty if ilo > ihi or jlo > jhi)
};

__device__ __forceinline__ Span cell_span(const Grid& g, float x, float y, float w, float h) {
    Span s;
    float hw = __fmul_rn(0.5f, w), hh = __fmul_rn(0.5f, h);
    s.xl = __fsub_rn(x, hw);
    s.xh = __fadd_rn(x, hw);
    s.yl = __fsub_rn(y, hh);
    s.yh = __fadd_rn(y, hh);
    s.ilo = max(last_edge<false>(g.x0, g.wb, g.inv_wb, g.guard, g.n, s.xl), 0);
    s.ihi = min(last_edge<true>(g.x0, g.wb, g.inv_wb, g.guard, g.n, s.xh), g.n - 1);
    s.jlo = max(last_edge<false>(g.y0, g.hb, g.inv_hb, g.guard, g.n, s.yl), 0);
    s.jhi = min(last_edge<true>(g.y0, g.hb, g.inv_hb, g.guard, g.n, s.yh), g.n - 1);
    return s;
}

// Overlap length of [a, b) with bin k (float32 arithmetic, no contraction).
__device__ __forceinline__ float ov_len(float lo, float step, int k, float a, float b) {
    float e0 = edge_at(lo, step, k), e1 = edge_at(lo, step, k + 1);
    float v = __fsub_rn(fminf(b, e1), fmaxf(a, e0));
    return fmaxf(v, 0.0f);
}

// Overlap lengths of a span [lo, hi] along one axis: the end bins take the
// generic formula; every bin strictly inside is covered whole, and
// e_{k+1} - e_k is exactly the bin size in float32, so "step" is the same
// value the generic formula gives there.
struct AxisOv {
    int lo, hi;
    float first, last, step;
};

__device__ __forceinline__ AxisOv axis_ov(float e0, float step, int lo, int hi, float a, float b) {
    AxisOv r;
    r.lo = lo;
    r.hi = hi;
    r.step = step;
    r.first = ov_len(e0, step, lo, a, b);
    r.last = ov_len(e0, step, hi, a, b);
    return r;
}

__device__ __forceinline__ float ov_at(const AxisOv& r, int k) {
    return k == r.lo ? r.first : (k == r.hi ? r.last : r.step);
}

// Field gather of one cell: sum_b ov(i,b) E2[b] over its bin span, E2 the
// interleaved (E_x, E_y) map, in chunks of 2 rows x 4 columns whose loads
// are all issued (predicated) before any use.  Nearly every cell is one
// chunk; a wider cell only adds chunks, so a warp's lanes run the same body.
__device__ __forceinline__ float2 gather_span(const Grid& g, const Span& s,
                                              const float2* __restrict__ E2) {
    float sx = 0.0f, sy = 0.0f;
    if (s.jlo > s.jhi || s.ilo > s.ihi) return make_float2(0.0f, 0.0f);
    const AxisOv ax = axis_ov(g.x0, g.wb, s.ilo, s.ihi, s.xl, s.xh);
    const AxisOv ay = axis_ov(g.y0, g.hb, s.jlo, s.jhi, s.yl, s.yh);
    for (int j0 = s.jlo; j0 <= s.jhi; j0 += 2) {
        for (int k0 = s.ilo; k0 <= s.ihi; k0 += 4) {
            float2 e[2][4];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int j = min(j0 + a, s.jhi);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int k = min(k0 + b, s.ihi);
                    e[a][b] = (j0 + a <= s.jhi && k0 + b <= s.ihi)
                                  ? __ldg(E2 + (size_t)j * g.n + k)
                                  : make_float2(0.0f, 0.0f);
                }
            }
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (j0 + a > s.jhi) break;
                const float oy = ov_at(ay, j0 + a);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    if (k0 + b > s.ihi) break;
                    const float o = __fmul_rn(ov_at(ax, k0 + b), oy);
                    sx = fmaf(o, e[a][b].x, sx);
                    sy = fmaf(o, e[a][b].y, sy);
                }
            }
        }
    }
    return make_float2(sx, sy);
}

// --------------------------------------------------- double-float sums
// An unevaluated sum hi + lo of two floats (error-free transformations:
// Knuth's TwoSum and Dekker's Fast2Sum).  Used to keep the grid-wide FP64
// reductions accurate without FP64 arithmetic in the inner loops.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_zero() { return {0.0f, 0.0f}; }

__device__ __forceinline__ dfloat df_add(dfloat a, float b) {
    float s = __fadd_rn(a.hi, b);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    float lo = __fadd_rn(a.lo, e);
    float hi = __fadd_rn(s, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    dfloat r = df_add(a, b.hi);
    return df_add(r, b.lo);
}

__device__ __forceinline__ dfloat warp_df_sum(dfloat v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfloat w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

__device__ __forceinline__ double* acc_stripe(double* acc, int q) {
    return acc + (blockIdx.x & (kAccStripes - 1)) * kAccStride + q;
}

// Max of non-negative doubles through their ordered bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(double* dst, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(dst),
              (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// *p += (a, b) as one relaxed, device-scope 8-byte vector reduction with no
// return value (the same operation as atomicAdd on a float2, which is issued
// as a returning atomic and so holds its destination registers until the
// answer comes back).
__device__ __forceinline__ void red_add_f2(float2* p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// *p += v as a relaxed, device-scope reduction with no return value.
__device__ __forceinline__ void red_add_f64(double* p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Sums of non-negative per-thread values a and b over each warp (a float32
// tree: relative error at most 5 units in the last place for non-negative
// terms); lane 0 adds each nonzero warp total in FP64 to the stripe of
// quantity qa / qb (qb < 0: none) chosen by the warp's global index.  No
// block-wide barrier, and the atomics spread over 32 lines.
__device__ __forceinline__ void block_acc2(float a, float b, double* acc, int qa, int qb) {
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        unsigned gw = (blockIdx.x * ((blockDim.x + 31) >> 5)) + (threadIdx.x >> 5);
        double* st = acc + (gw & (kAccStripes - 1)) * kAccStride;
        if (qa >= 0 && a != 0.0f) red_add_f64(st + qa, (double)a);
        if (qb >= 0 && b != 0.0f) red_add_f64(st + qb, (double)b);
    }
}

__device__ __forceinline__ void block_acc1(float a, double* acc, int qa) {
    block_acc2(a, 0.0f, acc, qa, -1);
}

// Deterministic (order-free) reduction for the deterministic mode: each
// block sums its threads in a fixed tree and stores its totals in its own
// slot of part[]; the block that draws the last ticket (after a fence) adds
// all slots in index order and stores the totals in stripe 0.  Nothing
// waits.  part == nullptr selects the striped atomics of block_acc2.
struct DetRed {
    double* part;       // [2][cap] block totals
    unsigned* ticket;   // zero between launches (the last block resets it)
    int cap;            // capacity in blocks
};

// add: the deterministic total is added to acc[q] instead of stored there
// (for a second kernel on the same stream that reduces into the same
// quantities after the first).
__device__ __forceinline__ void reduce2(float a, float b, double* acc, int qa, int qb,
                                        const DetRed& dr, bool add = false) {
    if (!dr.part) {
        block_acc2(a, b, acc, qa, qb);
        return;
    }
    __shared__ double s_a[32], s_b[32];
    __shared__ bool s_last;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    __syncthreads();
    if (l == 0) { s_a[w] = (double)a; s_b[w] = (double)b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int k = 0; k < nw; ++k) { ta += s_a[k]; tb += s_b[k]; }
        dr.part[blockIdx.x] = ta;
        dr.part[dr.cap + blockIdx.x] = tb;
        __threadfence();
        unsigned t = atomicAdd(dr.ticket, 1u);
        s_last = (t == gridDim.x - 1);
        if (s_last) *dr.ticket = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double ta = 0.0, tb = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        ta += __ldcg(dr.part + k);
        tb += __ldcg(dr.part + dr.cap + k);
    }
    __syncthreads();
    // fixed-order tree over the block (warps, then warp totals in order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ta += __shfl_down_sync(0xffffffffu, ta, o);
        tb += __shfl_down_sync(0xffffffffu, tb, o);
    }
    if (l == 0) { s_a[w] = ta; s_b[w] = tb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double fa = 0.0, fb = 0.0;
        for (int k = 0; k < nw; ++k) { fa += s_a[k]; fb += s_b[k]; }
        if (qa >= 0) acc[qa] = add ? acc[qa] + fa : fa;
        if (qb >= 0) acc[qb] = add ? acc[qb] + fb : fb;
        __threadfence();
    }
}

// a dfloat collapsed to the nearest float
__device__ __forceinline__ float df_val(dfloat d) { return d.hi + d.lo; }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Max of non-negative v over each warp into the stripe of quantity q.
__device__ __forceinline__ void block_max(float v, double* acc, int q) {
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) {
        unsigned gw = (blockIdx.x * ((blockDim.x + 31) >> 5)) + (threadIdx.x >> 5);
        atomic_max_nonneg(acc + (gw & (kAccStripes - 1)) * kAccStride + q, (double)v);
    }
}

// ------------------------------------------------------------ complex
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// WA smoothing factors of gamma in float32: 1/gamma and log2(e)/gamma (the
// exponentials are exp2(t log2(e) / gamma)), the same on host and device.
__host__ __device__ inline void wa_scale(float gamma, float* inv_g, float* l2g) {
    *inv_g = 1.0f / gamma;
    *l2g = (float)(1.4426950408889634 / (double)gamma);
}

// -------------------------------------------------------- the context
struct Ctx {
    // problem
    int n = 0, logn = 0, m_mov = 0, m_fix = 0, E = 0;
    int64_t P = 0;
    double x0 = 0, y0 = 0, x1 = 0, y1 = 0, Lx = 0, Ly = 0, wb = 0, hb = 0, Ab = 0;
    double mov_area = 0;
    Grid grid{};
    fftpl_options opt{};
    int wa_max_degree = 0;

    // streams and events
    cudaStream_t stream = nullptr, side = nullptr, own_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool profiling = false;
    double stage_ms[FFTPL_NUM_STAGES] = {};
    int64_t stage_launches[FFTPL_NUM_STAGES] = {};
    int64_t launches = 0;

    // device buffers
    float *w = nullptr, *h = nullptr, *fix_x = nullptr, *fix_y = nullptr;
    float *M = nullptr, *D = nullptr;
    long long* Dq = nullptr;
    float *T1 = nullptr, *PT = nullptr, *RT = nullptr;
    // tensor maps of T1 (boxes of 8 columns), PT and RT (boxes of 4 columns),
    // 256 rows (n if smaller): the transposed tiles of the row and column
    // passes leave shared memory through the tensor-memory-access unit
    CUtensorMap map_t1{}, map_pt{}, map_rt{};
    bool spec_tma = false;      // the transposed stores go through the maps
    bool spec_maps_ok = false;  // the maps could be encoded
    float *psi = nullptr, *ex = nullptr, *ey = nullptr, *rho = nullptr;
    float2* E2 = nullptr;       // interleaved field (E_x, E_y) [n][n]
    float2 *tw = nullptr, *ph = nullptr;
    // pins re-laid into degree slabs (see k_wire.cu): slot base + 32 k + lane
    int4* slabs = nullptr;      // {base slot, degree, net count, lanes per net (0: one
                                // net per lane)}
    int nslabs = 0;
    int nbig = 0;               // the first nbig slabs: degree kBigMin..kBigMax (k_wa_grp)
    int num_sms = 1;            // of the handle's device
    int64_t slab_slots = 0;
    int32_t *pin_cell = nullptr, *pin_slot = nullptr, *cell_pin_ptr = nullptr;
    float *pin_dx = nullptr, *pin_dy = nullptr;
    float2* gpin = nullptr;
    float2* gW2 = nullptr;      // interleaved wirelength gradient accumulator (m_mov),
                                // by internal number
    float2* pxy = nullptr;      // pin coordinates by slot, for the slabs of degree
                                // above kBigMax (their slots come first)
    float2* pos2 = nullptr;     // interleaved cell centres (m_mov), by internal number
    int32_t* cell_rank = nullptr;  // internal number of each movable cell (m_mov)
    // deterministic reductions: region 0 for the main stream, 1 for WA
    double* det_part = nullptr;
    unsigned* det_ticket = nullptr;
    int det_cap[2] = {0, 0};
    double* acc = nullptr;
    int* err = nullptr;
    double* acc_host = nullptr;   // pinned mirror

    // placement loop state (2 m_mov each: x then y)
    float *u = nullptr, *v = nullptr, *vprev = nullptr, *g = nullptr, *gprev = nullptr;
    float *gN = nullptr, *gW = nullptr;   // 2 m_mov each, loop scratch
    double* ctrl = nullptr;              // device control scalars
    double* recs = nullptr;              // device iteration records
    int recs_cap = 0;
    bool placing = false;
    int iter = 0;

    // host-side staging for fftpl_eval_host
    float *hx = nullptr, *hy = nullptr, *hg = nullptr;  // device staging (2m, 4m)

    // tensor-core solve path (solve_path FFTPL_SOLVE_TC_BF16X3), k_tc.cu
    struct TcPlan* tc = nullptr;
    // radix tensor-core path (solve_path FFTPL_SOLVE_TC_RADIX), k_tc.cu
    struct TcrPlan* tcr = nullptr;

    // captured CUDA graph of fftpl_eval for one set of buffers
    cudaGraphExec_t eval_graph = nullptr;
    // captured CUDA graph of one placement-loop iteration (fftpl_step), keyed
    // by the buffers its kernels take that can be reallocated
    cudaGraphExec_t loop_graph = nullptr;
    const void* loop_key[3] = {};
    int64_t loop_graph_nkernels = 0;
    const void* graph_key[8] = {};
    int64_t graph_nkernels = 0;
    // profiling ring of (stage, begin, end) event records
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_stage;
    int prof_used = 0;

    bool rho_valid = false, fields_valid = false, split_valid = false;
    bool psi_valid = false;     // psi matches the current fields (the transform
                                // path forms it on demand)
    std::string last_error;
    std::vector<void*> dev_allocs;
    size_t dev_bytes = 0;
};

// Reduction descriptor of region r (0: main stream, 1: WA stream); atomics
// unless the handle is deterministic.
inline DetRed det_red(const Ctx& c, int r) {
    if (!c.det_part) return DetRed{nullptr, nullptr, 0};
    double* base = c.det_part + (r == 0 ? 0 : 2 * (size_t)c.det_cap[0]);
    return DetRed{base, c.det_ticket + r, c.det_cap[r]};
}

// Enqueues one placement-loop iteration on the handle's streams (no sync).
fftpl_status loop_enqueue(Ctx& c);
// One iteration replayed from the handle's loop graph (captured on first use
// when use_graphs is set); launch = false only captures it.
fftpl_status loop_iter(Ctx& c, bool launch);
// For the server (on a worker thread): start positions from host memory,
// loop initialisation, room for iters records and the loop graph; returns
// with the handle's stream idle.
fftpl_status serve_prepare(Ctx& c, const float* x0, const float* y0, int iters);
// Makes room for cap iteration records and numbers them from base_k.
fftpl_status loop_records(Ctx& c, int cap, double base_k);

// Sets the text fftpl_last_error(NULL) returns on this thread.
void set_global_error(const std::string& msg);

// ------------------------------------------------------------ launchers
// (each returns the CUDA error of the launch)
void prepare_spectral(int logn);
cudaError_t launch_scatter(Ctx& c, const float* x, const float* y, const float* w,
                           const float* h, int m, float* D, long long* Dq, cudaStream_t s);
// movable cells into the handle's D / Dq; write_pos: also the interleaved
// centres pos2 (by internal cell number) for the WA kernel; stage (2 m_mov
// floats or null): also a device copy of (x, y)
cudaError_t launch_scatter_mov(Ctx& c, const float* x, const float* y, bool write_pos,
                               float* stage, cudaStream_t s);
cudaError_t launch_bin_ranges(Ctx& c, const float* x, const float* y, int32_t* ranges,
                              cudaStream_t s);
cudaError_t launch_rows_fwd(Ctx& c, cudaStream_t s);
cudaError_t launch_cols_spectral(Ctx& c, cudaStream_t s);
cudaError_t launch_rows_inv(Ctx& c, cudaStream_t s);
// psi rows from PT (transform path; formed on demand, not in the evaluation)
cudaError_t launch_rows_psi(Ctx& c, cudaStream_t s);
// Tensor maps for the transposed stores of the transform passes (host only,
// no allocation); clears c.spec_tma if the driver cannot encode them.
void spec_maps_init(Ctx& c);
// 2-D float32 tensor [rows][cols] in boxes of box_inner columns x box_outer rows.
bool make_map_f32(CUtensorMap* map, const float* base, int rows, int cols, int box_inner,
                  int box_outer);
cudaError_t launch_rho(Ctx& c, cudaStream_t s);
cudaError_t launch_split_field(Ctx& c, cudaStream_t s);
cudaError_t launch_q_to_f(const long long* q, float scale, float* out, int count, cudaStream_t s);
cudaError_t launch_gather(Ctx& c, const float* x, const float* y, float* gx, float* gy,
                          bool adjoint, cudaStream_t s);
cudaError_t launch_wa(Ctx& c, const float* x, const float* y, float gamma, cudaStream_t s);
// interleave = false: pos2 already written (by launch_scatter_mov)
cudaError_t launch_wa_impl(Ctx& c, const float* x, const float* y, float gamma,
                           const float* scale_dev, const float* done, bool interleave,
                           cudaStream_t s);
cudaError_t launch_pin_sum(Ctx& c, float* gx, float* gy, cudaStream_t s);
// 1 when the WA kernel runs slab pairs per warp (large instances)
int wa_pairs(const Ctx& c);

// create-time netlist layout (k_setup.cu): label rounds for the internal
// cell numbers (seeds every kSeedStride cells, kLabelRounds rounds, nets of
// more than kRankMaxDegree pins not followed), each net's lowest cell
// number, and the pin records in slab layout
constexpr int kSeedStride = 64;
constexpr int kLabelRounds = 6;
constexpr int kRankMaxDegree = 64;
cudaError_t launch_label_rounds(int m, int E, const int* np, const int* pc, int* lab, int* next,
                                int* dist, int* netlab, cudaStream_t s);
cudaError_t launch_net_key(int m, int E, const int* np, const int* pc, const int* rank, int* key,
                           cudaStream_t s);
cudaError_t launch_fill_slabs(int m, int E, const int* np, const int* pc, const float* dx,
                              const float* dy, const int* rank, const float* fix_x,
                              const float* fix_y, const int* net_slot, const int* net_lanes,
                              const int* cslot, int* spc, float* sdx, float* sdy, int* sslot,
                              cudaStream_t s);

// tensor-core solve path (k_tc.cu): tc_setup lays the plan out in a device
// block of tc_elems(n) bf16 elements owned by the handle and fills its
// cosine/sine tables on stream s; launch_tc part 0 splits rho (with the
// overflow and charge sums), 1 and 2 the forward contractions (2 with the
// spectral divide and the energy), 3 the inverse ones (psi, E_x, E_y).
size_t tc_elems(int n);
cudaError_t tc_setup(Ctx& c, uint16_t* block, cudaStream_t s);
void tc_free(Ctx& c);
cudaError_t launch_tc(Ctx& c, int part, cudaStream_t s);
cudaError_t tc_debug_gemm(const void* ah, const void* al, const void* bh, const void* bl, int M,
                          int N, int K, float* d, int nsplit, int no_loads, int* err,
                          cudaStream_t s);
// radix tensor-core path (k_tc.cu): tcr_setup lays the plan out in a device
// block of tcr_elems(n) bf16 elements and 2 n^2 float2 (Z, V) owned by the
// handle; launch_tcr part 0 the row pass, 1 the column pass, 2 the inverse
// row pass, 3 the overflow and charge sums alone.  launch_tcr_stage
// (k_spectral.cu): the pre- and post-processing kernels between its DFTs.
size_t tcr_elems(int n);
cudaError_t tcr_setup(Ctx& c, uint16_t* block, float2* zv, cudaStream_t s);
void tcr_free(Ctx& c);
cudaError_t launch_tcr(Ctx& c, int part, cudaStream_t s);
cudaError_t launch_tcr_stage(Ctx& c, int which, const float2* V, float2* Z, cudaStream_t s);
cudaError_t launch_cells(Ctx& c, const float* x, const float* y, float* gNx, float* gNy,
                         float* gWx, float* gWy, cudaStream_t s);
// placement loop
cudaError_t launch_loop_cells(Ctx& c, cudaStream_t s);
cudaError_t launch_loop_g(Ctx& c, cudaStream_t s);
cudaError_t launch_loop_update(Ctx& c, cudaStream_t s);
cudaError_t launch_place_init(Ctx& c, const float* x0, const float* y0, cudaStream_t s);
cudaError_t launch_gamma0(Ctx& c, cudaStream_t s);
// conjugate-gradient loop (k_step.cu)
cudaError_t launch_cg_g(Ctx& c, cudaStream_t s);
cudaError_t launch_cg_dir(Ctx& c, cudaStream_t s);
cudaError_t launch_cg_trial(Ctx& c, cudaStream_t s);
cudaError_t launch_cg_alpha(Ctx& c, cudaStream_t s);
cudaError_t launch_cg_update(Ctx& c, cudaStream_t s);

}  // namespace fftpl

// The opaque handle of the C ABI is the context.
struct fftpl_ctx : public fftpl::Ctx {};
