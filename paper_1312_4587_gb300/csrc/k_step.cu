// Placement loop kernels: the per-cell gradient with the lambda update, the
// combined gradient g = grad W~ + lambda grad N with the step-size sums, and
// the position update, either Nesterov's method or Algorithm 1's
// conjugate-gradient step (control of Section IV-A in loop_ctrl.cuh).
//
// Vectors hold x coordinates in [0, m) and y coordinates in [m, 2m).
#include <algorithm>

#include "loop_ctrl.cuh"

namespace fftpl {

struct LoopBufs {
    float *u, *v, *vprev, *g, *gprev, *gN, *gW;
    const float *w, *h;
    double *ctrl, *acc, *recs;
    unsigned int* counters;
    DetRed dr;
};

// gather + pin sums at v (like k_cells, 48 warps per SM); k_ctrl_lambda
// then forms lambda_k.
template <bool CSR>
__global__ void __launch_bounds__(kCellThreads, 6)
k_loop_cells(Grid gr, int m, LoopBufs b, const float2* __restrict__ E2,
             const int* __restrict__ rank, const int* __restrict__ cell_pin_ptr,
             const float2* __restrict__ gpin, const float2* __restrict__ gW2) {
    const float* cf = ctrl_f(b.ctrl);
    if (cf[F_DONE] != 0.0f) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float nx = 0.0f, ny = 0.0f, wx = 0.0f, wy = 0.0f;
    if (i < m) {
        // the wirelength gradient's loads go out before the field gather's
        const int r = rank[i];
        Span s = cell_span(gr, b.v[i], b.v[m + i], b.w[i], b.h[i]);
        if (CSR) {
            for (int q = cell_pin_ptr[r]; q < cell_pin_ptr[r + 1]; ++q) {
                float2 p = gpin[q];
                wx += p.x;
                wy += p.y;
            }
        } else {
            float2 v = gW2[r];
            wx = v.x;
            wy = v.y;
        }
        float2 e = gather_span(gr, s, E2);
        nx = -e.x;
        ny = -e.y;
        b.gN[i] = nx;
        b.gN[m + i] = ny;
        b.gW[i] = wx;
        b.gW[m + i] = wy;
    }
    reduce2(fabsf(nx) + fabsf(ny), fabsf(wx) + fabsf(wy), b.acc, ACC_GN_L1, ACC_GW_L1, b.dr);
}

// lambda_k from the cell kernel's sums (one thread, launched after it: a
// ticket at the end of each of the cell kernel's 8.6K blocks cost more)
__global__ void k_ctrl_lambda(double* ctrl, const double* acc) {
    if (ctrl_f(ctrl)[F_DONE] != 0.0f) return;
    ctrl_lambda(ctrl, acc);
}

// The vector kernels of the loop (2m coordinates) run on a fixed grid of
// kVecBlocksPerSm blocks per SM, each thread striding over the coordinates
// in batches of four (all loads of a batch before its stores, through
// restrict-qualified pointers, so that they are in flight together) with
// its sums kept as double-float pairs: each block ends with block
// reductions and a ticket (an atomic round trip) that a block per 256
// coordinates paid 17K times per kernel at 2.2M cells.
constexpr int kVecBlocksPerSm = 6;

// g = gW + lambda gN; sums for alpha_k; last CTA: alpha_k and beta_k.
__global__ void __launch_bounds__(kCellThreads, kVecBlocksPerSm) k_loop_g(int m2, LoopBufs b) {
    const float* cf = ctrl_f(b.ctrl);
    if (cf[F_DONE] != 0.0f) return;
    const float lam = cf[F_LAMBDA];
    const bool first = cf[F_FIRST] != 0.0f;
    dfloat dg = df_zero(), dv = df_zero();
    float gi = 0.0f;
    const int stride = gridDim.x * blockDim.x;
    const float* __restrict__ GN = b.gN;
    const float* __restrict__ GW = b.gW;
    const float* __restrict__ GP = b.gprev;
    const float* __restrict__ V = b.v;
    const float* __restrict__ VP = b.vprev;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < m2; i0 += 4 * stride) {
        float gn[4], gw[4], gp[4], v[4], vp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < m2) {
                gn[k] = GN[i];
                gw[k] = GW[i];
                if (!first) {
                    gp[k] = GP[i];
                    v[k] = V[i];
                    vp[k] = VP[i];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < m2) {
                const float gg = fmaf(lam, gn[k], gw[k]);
                b.g[i] = gg;
                gi = fmaxf(gi, fabsf(gg));
                if (!first) {
                    const float a = gg - gp[k], c = v[k] - vp[k];
                    dg = df_add(dg, a * a);
                    dv = df_add(dv, c * c);
                }
            }
        }
    }
    reduce2(df_val(dg), df_val(dv), b.acc, ACC_DG2, ACC_DV2, b.dr);
    block_max(gi, b.acc, ACC_GINF);
    if (last_cta(b.counters + 1) && threadIdx.x == 0) ctrl_alpha(b.ctrl, b.acc);
}

// u_{k+1} = clamp(v_k - alpha g_k); v_{k+1} = clamp(u_{k+1} + beta (u_{k+1} - u_k));
// clamp keeps the cell inside the region.  Last CTA: record and advance.
__global__ void __launch_bounds__(kCellThreads, kVecBlocksPerSm)
k_loop_update(int m, Grid gr, float x1, float y1, LoopBufs b) {
    const float* cf = ctrl_f(b.ctrl);
    if (cf[F_DONE] != 0.0f) return;
    const float alpha = cf[F_ALPHA], beta = cf[F_BETA];
    float step = 0.0f;
    dfloat uphill = df_zero();
    const int stride = gridDim.x * blockDim.x, n2 = 2 * m;
    const float* __restrict__ V = b.v;
    const float* __restrict__ G = b.g;
    const float* __restrict__ U = b.u;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n2; i0 += 4 * stride) {
        float vv[4], gg[4], uu[4], hw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < n2) {
                const bool isx = i < m;
                hw[k] = isx ? b.w[i] : b.h[i - m];
                vv[k] = V[i];
                gg[k] = G[i];
                uu[k] = U[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < n2) {
                const bool isx = i < m;
                float half = __fmul_rn(0.5f, hw[k]);
                float lo = __fadd_rn(isx ? gr.x0 : gr.y0, half), hi = __fsub_rn(isx ? x1 : y1, half);
                float un = fminf(hi, fmaxf(lo, vv[k] - alpha * gg[k]));
                step = fmaxf(step, fabsf(un - vv[k]));
                uphill = df_add(uphill, gg[k] * (un - uu[k]));
                float vn = fminf(hi, fmaxf(lo, un + beta * (un - uu[k])));
                b.vprev[i] = vv[k];
                b.gprev[i] = gg[k];
                b.u[i] = un;
                b.v[i] = vn;
            }
        }
    }
    block_max(step, b.acc, ACC_STEPMAX);
    reduce2(df_val(uphill), 0.0f, b.acc, ACC_GD, -1, b.dr);
    if (last_cta(b.counters + 2) && threadIdx.x == 0) ctrl_record(b.ctrl, b.acc, b.recs);
}

// ------------------------------------------------ conjugate-gradient loop
// The direction d_k lives in the Nesterov loop's vprev buffer (unused here);
// u holds x_k and v the point being evaluated (x_k, then the trial point).

// g = gW + lambda gN; sums |g|^2 and g . g_prev, max |g|; last CTA: beta,
// f_k and the values recorded for iteration k.
__global__ void __launch_bounds__(kCellThreads, kVecBlocksPerSm) k_cg_g(int m2, LoopBufs b) {
    const float* cf = ctrl_f(b.ctrl);
    if (cf[F_DONE] != 0.0f) return;
    const float lam = cf[F_LAMBDA];
    const bool first = cf[F_FIRST] != 0.0f;
    dfloat sq = df_zero(), gp = df_zero();
    float gi = 0.0f;
    const int stride = gridDim.x * blockDim.x;
    const float* __restrict__ GN = b.gN;
    const float* __restrict__ GW = b.gW;
    const float* __restrict__ GP = b.gprev;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < m2; i0 += 4 * stride) {
        float gn[4], gw[4], pr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < m2) {
                gn[k] = GN[i];
                gw[k] = GW[i];
                pr[k] = first ? 0.0f : GP[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < m2) {
                const float gg = fmaf(lam, gn[k], gw[k]);
                b.g[i] = gg;
                sq = df_add(sq, gg * gg);
                if (!first) gp = df_add(gp, gg * pr[k]);
                gi = fmaxf(gi, fabsf(gg));
            }
        }
    }
    reduce2(df_val(sq), df_val(gp), b.acc, ACC_DG2, ACC_DV2, b.dr);
    block_max(gi, b.acc, ACC_GINF);
    if (last_cta(b.counters + 3) && threadIdx.x == 0) ctrl_cg_g(b.ctrl, b.acc);
}

// d = -g + beta d; sum g . d and max |d|; last CTA: restart test, |d|_inf
// and the slope.
__global__ void __launch_bounds__(kCellThreads, kVecBlocksPerSm) k_cg_dir(int m2, LoopBufs b) {
    const float* cf = ctrl_f(b.ctrl);
    if (cf[F_DONE] != 0.0f) return;
    const float beta = cf[F_BETA];
    const bool first = cf[F_FIRST] != 0.0f;
    dfloat gd = df_zero();
    float da = 0.0f;
    const int stride = gridDim.x * blockDim.x;
    const float* __restrict__ G = b.g;
    const float* __restrict__ D = b.vprev;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < m2; i0 += 4 * stride) {
        float g[4], d[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < m2) {
                g[k] = G[i];
                d[k] = first ? 0.0f : D[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < m2) {
                const float dn = first ? -g[k] : fmaf(beta, d[k], -g[k]);
                b.vprev[i] = dn;
                gd = df_add(gd, g[k] * dn);
                da = fmaxf(da, fabsf(dn));
            }
        }
    }
    reduce2(df_val(gd), 0.0f, b.acc, ACC_GD, -1, b.dr);
    block_max(da, b.acc, ACC_DINF);
    if (last_cta(b.counters + 4) && threadIdx.x == 0) ctrl_cg_dir(b.ctrl, b.acc);
}

// per coordinate i < 2m: the direction (d, or -g after a restart) and the
// clamp bounds of the cell inside the region
__device__ __forceinline__ void cg_coord(int i, int m, const Grid& gr, float x1, float y1,
                                         const LoopBufs& b, float& dir, float& lo, float& hi) {
    const bool isx = i < m;
    const int c = isx ? i : i - m;
    const float half = __fmul_rn(0.5f, isx ? b.w[c] : b.h[c]);
    lo = __fadd_rn(isx ? gr.x0 : gr.y0, half);
    hi = __fsub_rn(isx ? x1 : y1, half);
    dir = ctrl_f(b.ctrl)[F_RESTART] != 0.0f ? -b.g[i] : b.vprev[i];
}

// trial point v = clamp(u + a_max dir / |d|_inf)
__global__ void __launch_bounds__(kCellThreads)
k_cg_trial(int m, Grid gr, float x1, float y1, LoopBufs b) {
    const float* cf = ctrl_f(b.ctrl);
    if (cf[F_DONE] != 0.0f) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * m) return;
    const float scale = cf[F_SCALE_TRIAL];
    float dir, lo, hi;
    cg_coord(i, m, gr, x1, y1, b, dir, lo, hi);
    b.v[i] = fminf(hi, fmaxf(lo, fmaf(scale, dir, b.u[i])));
}

// the step from the trial evaluation (one thread)
__global__ void k_cg_alpha(double* ctrl, const double* acc) {
    if (ctrl[C_DONE] != 0.0) return;
    ctrl_cg_alpha(ctrl, acc);
}

// u = v = clamp(u + a_k dir / |d|_inf); d = dir; g_prev = g.  Last CTA:
// record and advance.
__global__ void __launch_bounds__(kCellThreads, kVecBlocksPerSm)
k_cg_update(int m, Grid gr, float x1, float y1, LoopBufs b) {
    const float* cf = ctrl_f(b.ctrl);
    if (cf[F_DONE] != 0.0f) return;
    const float scale = cf[F_SCALE_UPDATE];
    const bool restart = cf[F_RESTART] != 0.0f;
    const int stride = gridDim.x * blockDim.x, n2 = 2 * m;
    const float* __restrict__ G = b.g;
    const float* __restrict__ D = b.vprev;
    const float* __restrict__ U = b.u;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n2; i0 += 4 * stride) {
        float g[4], dir[4], u[4], hw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < n2) {
                hw[k] = i < m ? b.w[i] : b.h[i - m];
                g[k] = G[i];
                dir[k] = restart ? -g[k] : D[i];
                u[k] = U[i];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * stride;
            if (i < n2) {
                const bool isx = i < m;
                const float half = __fmul_rn(0.5f, hw[k]);
                const float lo = __fadd_rn(isx ? gr.x0 : gr.y0, half);
                const float hi = __fsub_rn(isx ? x1 : y1, half);
                const float un = fminf(hi, fmaxf(lo, fmaf(scale, dir[k], u[k])));
                b.u[i] = un;
                b.v[i] = un;
                b.vprev[i] = dir[k];
                b.gprev[i] = g[k];
            }
        }
    }
    if (last_cta(b.counters + 5) && threadIdx.x == 0) ctrl_record_cg(b.ctrl, b.recs);
}

// u = v = clamp(x0, y0); previous vectors zeroed.
__global__ void k_place_init(int m, Grid gr, float x1, float y1, const float* __restrict__ x0,
                             const float* __restrict__ y0, LoopBufs b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * m) return;
    bool isx = i < m;
    int c = isx ? i : i - m;
    float half = __fmul_rn(0.5f, isx ? b.w[c] : b.h[c]);
    float lo = __fadd_rn(isx ? gr.x0 : gr.y0, half), hi = __fsub_rn(isx ? x1 : y1, half);
    float p = isx ? x0[c] : y0[c];
    p = fminf(hi, fmaxf(lo, p));
    b.u[i] = p;
    b.v[i] = p;
    b.vprev[i] = p;
    b.g[i] = 0.0f;
    b.gprev[i] = 0.0f;
}

// gamma_0 from the overflow at the start (schedule mode).
__global__ void k_gamma0(double* ctrl, const double* acc) {
    double tau = acc_sum(acc, ACC_TAU) / ctrl[C_MOV_AREA];
    ctrl[C_GAMMA] = gamma_schedule(tau, ctrl[C_WB]);
    ctrl_mirror(ctrl);
}

static inline int nblk(long long m, int t) { return (int)((m + t - 1) / t); }

// blocks of a vector kernel over n coordinates (grid-stride)
static inline int vec_blocks(const Ctx& c, long long n) {
    return std::max(1, std::min(nblk(n, kCellThreads), c.num_sms * kVecBlocksPerSm));
}

LoopBufs loop_bufs(Ctx& c) {
    LoopBufs b;
    b.u = c.u; b.v = c.v; b.vprev = c.vprev; b.g = c.g; b.gprev = c.gprev;
    b.gN = c.gN; b.gW = c.gW; b.w = c.w; b.h = c.h;
    b.ctrl = c.ctrl; b.acc = c.acc; b.recs = c.recs;
    b.counters = reinterpret_cast<unsigned int*>(c.ctrl + C_COUNT);
    b.dr = det_red(c, 0);
    return b;
}

cudaError_t launch_loop_cells(Ctx& c, cudaStream_t s) {
    LoopBufs b = loop_bufs(c);
    int nb = nblk(c.m_mov, kCellThreads);
    if (c.opt.deterministic)
        k_loop_cells<true><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, b, c.E2, c.cell_rank,
                                                       c.cell_pin_ptr, c.gpin, nullptr);
    else
        k_loop_cells<false><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, b, c.E2, c.cell_rank,
                                                        nullptr, nullptr, c.gW2);
    k_ctrl_lambda<<<1, 1, 0, s>>>(c.ctrl, c.acc);
    c.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_loop_g(Ctx& c, cudaStream_t s) {
    k_loop_g<<<vec_blocks(c, 2LL * c.m_mov), kCellThreads, 0, s>>>(2 * c.m_mov, loop_bufs(c));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_loop_update(Ctx& c, cudaStream_t s) {
    k_loop_update<<<vec_blocks(c, 2LL * c.m_mov), kCellThreads, 0, s>>>(
        c.m_mov, c.grid, (float)c.x1, (float)c.y1, loop_bufs(c));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_place_init(Ctx& c, const float* x0, const float* y0, cudaStream_t s) {
    k_place_init<<<nblk(2LL * c.m_mov, 256), 256, 0, s>>>(c.m_mov, c.grid, (float)c.x1,
                                                         (float)c.y1, x0, y0, loop_bufs(c));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cg_g(Ctx& c, cudaStream_t s) {
    k_cg_g<<<vec_blocks(c, 2LL * c.m_mov), kCellThreads, 0, s>>>(2 * c.m_mov, loop_bufs(c));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cg_dir(Ctx& c, cudaStream_t s) {
    k_cg_dir<<<vec_blocks(c, 2LL * c.m_mov), kCellThreads, 0, s>>>(2 * c.m_mov, loop_bufs(c));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cg_trial(Ctx& c, cudaStream_t s) {
    k_cg_trial<<<nblk(2LL * c.m_mov, kCellThreads), kCellThreads, 0, s>>>(
        c.m_mov, c.grid, (float)c.x1, (float)c.y1, loop_bufs(c));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cg_alpha(Ctx& c, cudaStream_t s) {
    k_cg_alpha<<<1, 1, 0, s>>>(c.ctrl, c.acc);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cg_update(Ctx& c, cudaStream_t s) {
    k_cg_update<<<vec_blocks(c, 2LL * c.m_mov), kCellThreads, 0, s>>>(
        c.m_mov, c.grid, (float)c.x1, (float)c.y1, loop_bufs(c));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_gamma0(Ctx& c, cudaStream_t s) {
    k_gamma0<<<1, 1, 0, s>>>(c.ctrl, c.acc);
    c.launches++;
    return cudaGetLastError();
}

}  // namespace fftpl
