// Density scatter, field gather and bookkeeping kernels.
//
// Scatter (Section II bin density, Section III charges q_i = A_i): every cell
// adds its exact rectangle-bin overlap areas to the movable area map D; the
// transform pass later forms rho = (D + rho_t F) / A_b.  Gather (the q.E of
// Eq. 7): dN/dx_i = -sum_b ov(i,b) E_x[b], the exact transpose of the
// scatter weights.  Adjoint: the exact derivative of the binned energy,
// sum over rows of the row overlap times (psi at the right-edge bin - psi at
// the left-edge bin), and likewise in y.
#include "fftpl_internal.cuh"

namespace fftpl {

// One thread per cell.  FP32 mode: ov added into D with 16-byte vector
// atomics over the aligned groups of 4 bins a row span touches (zeros for
// the bins of a group outside the span), which cuts the atomic count about
// in half for cells spanning 2-4 bins.
// Deterministic mode: ov is formed in float32 (x and y lengths, then their
// product), scaled by 2^32 (exact) and rounded to the nearest integer (ties to
// even); int64 atomics make the bin sums independent of order.
// pos, if given, receives the interleaved centre at the cell's internal
// number for the WA kernel (so that it needs no pass of its own); stage, if
// given, a device copy of (x, y) for the later kernels (x, y may then be
// pinned host memory read over the host link once).
template <bool QUANT>
__global__ void __launch_bounds__(kCellThreads)
k_scatter(Grid g, int m, const float* __restrict__ x, const float* __restrict__ y,
          const float* __restrict__ w, const float* __restrict__ h, const int* __restrict__ rank,
          float2* __restrict__ pos, float* __restrict__ stage, float* __restrict__ D,
          unsigned long long* __restrict__ Dq) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float xi = x[i], yi = y[i];
    if (pos) pos[rank[i]] = make_float2(xi, yi);
    if (stage) {
        stage[i] = xi;
        stage[m + i] = yi;
    }
    Span s = cell_span(g, xi, yi, w[i], h[i]);
    if (s.ilo > s.ihi || s.jlo > s.jhi) return;
    const AxisOv ax = axis_ov(g.x0, g.wb, s.ilo, s.ihi, s.xl, s.xh);
    const AxisOv ay = axis_ov(g.y0, g.hb, s.jlo, s.jhi, s.yl, s.yh);
    if (QUANT) {
        for (int j = s.jlo; j <= s.jhi; ++j) {
            float oy = ov_at(ay, j);
            for (int k = s.ilo; k <= s.ihi; ++k) {
                float a = __fmul_rn(ov_at(ax, k), oy);
                long long q = __float2ll_rn(__fmul_rn(a, 4294967296.0f));
                atomicAdd(Dq + (size_t)j * g.n + k, (unsigned long long)q);
            }
        }
    } else {
        // quads outer, rows inner: a quad's four x overlaps serve every row
        for (int q = s.ilo >> 2; q <= (s.ihi >> 2); ++q) {
            float ox[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                int k = 4 * q + t;
                ox[t] = (k >= s.ilo && k <= s.ihi) ? ov_at(ax, k) : 0.0f;
            }
            float* col = D + 4 * q;
            for (int j = s.jlo; j <= s.jhi; ++j) {
                const float oy = ov_at(ay, j);
                atomicAdd(reinterpret_cast<float4*>(col + (size_t)j * g.n),
                          make_float4(__fmul_rn(ox[0], oy), __fmul_rn(ox[1], oy),
                                      __fmul_rn(ox[2], oy), __fmul_rn(ox[3], oy)));
            }
        }
    }
}

__global__ void __launch_bounds__(kCellThreads)
k_bin_ranges(Grid g, int m, const float* __restrict__ x, const float* __restrict__ y,
             const float* __restrict__ w, const float* __restrict__ h, int4* __restrict__ out,
             double* __restrict__ acc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float cnt = 0.0f;
    if (i < m) {
        Span s = cell_span(g, x[i], y[i], w[i], h[i]);
        bool empty = s.ilo > s.ihi || s.jlo > s.jhi;
        if (empty) {
            out[i] = make_int4(0, -1, 0, -1);
        } else {
            out[i] = make_int4(s.ilo, s.ihi, s.jlo, s.jhi);
            cnt = (float)((s.ihi - s.ilo + 1) * (s.jhi - s.jlo + 1));
        }
    }
    block_acc1(cnt, acc, ACC_CHARGE);
}

// Field gather (ADJ = false) or exact edge-difference adjoint (ADJ = true,
// field = psi in fx).  Writes gx, gy and adds ||g||_1 to *l1.
template <bool ADJ>
__global__ void __launch_bounds__(kCellThreads, 6)
k_gather(Grid g, int m, const float* __restrict__ x, const float* __restrict__ y,
         const float* __restrict__ w, const float* __restrict__ h, const float* __restrict__ fx,
         const float2* __restrict__ E2, float* __restrict__ gx, float* __restrict__ gy,
         double* __restrict__ acc, DetRed dr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float sx = 0.0f, sy = 0.0f;
    if (i < m) {
        Span s = cell_span(g, x[i], y[i], w[i], h[i]);
        if (!ADJ) {
            float2 e = gather_span(g, s, E2);
            sx = -e.x;
            sy = -e.y;
        } else if (s.ilo <= s.ihi && s.jlo <= s.jhi) {
            int n = g.n;
            int kl = last_edge<false>(g.x0, g.wb, g.inv_wb, g.guard, n, s.xl);
            int kr = last_edge<false>(g.x0, g.wb, g.inv_wb, g.guard, n, s.xh);
            int jl = last_edge<false>(g.y0, g.hb, g.inv_hb, g.guard, n, s.yl);
            int jr = last_edge<false>(g.y0, g.hb, g.inv_hb, g.guard, n, s.yh);
            bool kr_in = kr >= 0 && kr < n, kl_in = kl >= 0 && kl < n;
            bool jr_in = jr >= 0 && jr < n, jl_in = jl >= 0 && jl < n;
            for (int j = s.jlo; j <= s.jhi; ++j) {
                float oy = ov_len(g.y0, g.hb, j, s.yl, s.yh);
                const float* r = fx + (size_t)j * n;
                float d = (kr_in ? __ldg(r + kr) : 0.0f) - (kl_in ? __ldg(r + kl) : 0.0f);
                sx = fmaf(oy, d, sx);
            }
            const float* rt = fx + (size_t)(jr_in ? jr : 0) * n;
            const float* rb = fx + (size_t)(jl_in ? jl : 0) * n;
            for (int k = s.ilo; k <= s.ihi; ++k) {
                float ox = ov_len(g.x0, g.wb, k, s.xl, s.xh);
                float d = (jr_in ? __ldg(rt + k) : 0.0f) - (jl_in ? __ldg(rb + k) : 0.0f);
                sy = fmaf(ox, d, sy);
            }
        }
        gx[i] = sx;
        gy[i] = sy;
    }
    reduce2(fabsf(sx) + fabsf(sy), 0.0f, acc, ACC_GN_L1, -1, dr);
}

// rho = (D + M) / A_b (formed on demand for fftpl_fields).
template <bool QUANT>
__global__ void k_rho(int count, const float* __restrict__ D, const long long* __restrict__ Dq,
                      const float* __restrict__ M, float inv_ab, float* __restrict__ rho) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float d = QUANT ? (float)Dq[i] * 2.3283064365386963e-10f : D[i];
    rho[i] = (d + M[i]) * inv_ab;
}

__global__ void k_split_field(int count, const float2* __restrict__ E2, float* __restrict__ ex,
                              float* __restrict__ ey) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        float2 e = E2[i];
        ex[i] = e.x;
        ey[i] = e.y;
    }
}

__global__ void k_q_to_f(const long long* __restrict__ q, float scale, float* __restrict__ out,
                         int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (float)q[i] * 2.3283064365386963e-10f * scale;
}

static inline int blocks_for(long long m, int t) { return (int)((m + t - 1) / t); }

cudaError_t launch_scatter(Ctx& c, const float* x, const float* y, const float* w, const float* h,
                           int m, float* D, long long* Dq, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    int nb = blocks_for(m, kCellThreads);
    if (Dq)
        k_scatter<true><<<nb, kCellThreads, 0, s>>>(c.grid, m, x, y, w, h, nullptr, nullptr,
                                                   nullptr, nullptr,
                                                   reinterpret_cast<unsigned long long*>(Dq));
    else
        k_scatter<false><<<nb, kCellThreads, 0, s>>>(c.grid, m, x, y, w, h, nullptr, nullptr,
                                                    nullptr, D, nullptr);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_scatter_mov(Ctx& c, const float* x, const float* y, bool write_pos,
                               float* stage, cudaStream_t s) {
    const int m = c.m_mov;
    if (m <= 0) return cudaSuccess;
    float2* pos = write_pos ? c.pos2 : nullptr;
    int nb = blocks_for(m, kCellThreads);
    if (c.opt.deterministic)
        k_scatter<true><<<nb, kCellThreads, 0, s>>>(c.grid, m, x, y, c.w, c.h, c.cell_rank, pos,
                                                   stage, nullptr,
                                                   reinterpret_cast<unsigned long long*>(c.Dq));
    else
        k_scatter<false><<<nb, kCellThreads, 0, s>>>(c.grid, m, x, y, c.w, c.h, c.cell_rank, pos,
                                                    stage, c.D, nullptr);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_bin_ranges(Ctx& c, const float* x, const float* y, int32_t* ranges,
                              cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    k_bin_ranges<<<blocks_for(c.m_mov, kCellThreads), kCellThreads, 0, s>>>(
        c.grid, c.m_mov, x, y, c.w, c.h, reinterpret_cast<int4*>(ranges), c.acc);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_gather(Ctx& c, const float* x, const float* y, float* gx, float* gy,
                          bool adjoint, cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    int nb = blocks_for(c.m_mov, kCellThreads);
    if (adjoint)
        k_gather<true><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, c.psi, nullptr,
                                                  gx, gy, c.acc, det_red(c, 0));
    else
        k_gather<false><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, nullptr, c.E2,
                                                   gx, gy, c.acc, det_red(c, 0));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_rho(Ctx& c, cudaStream_t s) {
    int count = c.n * c.n;
    float inv_ab = (float)(1.0 / c.Ab);
    if (c.opt.deterministic)
        k_rho<true><<<blocks_for(count, 256), 256, 0, s>>>(count, nullptr, c.Dq, c.M, inv_ab, c.rho);
    else
        k_rho<false><<<blocks_for(count, 256), 256, 0, s>>>(count, c.D, nullptr, c.M, inv_ab, c.rho);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_split_field(Ctx& c, cudaStream_t s) {
    int count = c.n * c.n;
    k_split_field<<<blocks_for(count, 256), 256, 0, s>>>(count, c.E2, c.ex, c.ey);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_q_to_f(const long long* q, float scale, float* out, int count,
                          cudaStream_t st) {
    k_q_to_f<<<blocks_for(count, 256), 256, 0, st>>>(q, scale, out, count);
    return cudaGetLastError();
}

}  // namespace fftpl
