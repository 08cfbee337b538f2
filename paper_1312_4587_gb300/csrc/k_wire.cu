// Weighted-average wirelength (Eq. 3) and the per-cell gradient kernel.
//
// WA, per net and axis, with pins p_j, M = max p, mu = min p, local
// coordinates t+_j = p_j - M <= 0 and t-_j = p_j - mu >= 0:
//   a+_j = exp(t+_j / g), a-_j = exp(-t-_j / g)
//   W~ = (M - mu) + sum t+ a+ / sum a+ - sum t- a- / sum a-
//   dW~/dp_j = (a+_j/S+)(1 + (t+_j - T+/S+)/g) - (a-_j/S-)(1 - (t-_j - T-/S-)/g)
// which is Eq. 3 with the exponentials shifted by M (resp. mu); working in
// the local coordinates keeps float32 accurate when coordinates are large
// compared with the net's span.  Pin coordinate = fl32(cell centre + offset).
//
// One CTA handles 256 consecutive nets; their pins (contiguous in the net
// order) are staged into shared memory with coalesced loads, the cell
// positions gathered once per pin; each thread then walks one net.
#include "fftpl_internal.cuh"

namespace fftpl {

template <bool CSR>
__global__ void __launch_bounds__(kWaThreads)
k_wa(int E, const int* __restrict__ net_ptr, const int* __restrict__ pin_cell,
     const float* __restrict__ pdx, const float* __restrict__ pdy, int m_mov,
     const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ fx,
     const float* __restrict__ fy, float gamma, const double* __restrict__ gamma_dev,
     float* __restrict__ gx, float* __restrict__ gy, const int* __restrict__ pin_slot,
     float2* __restrict__ gpin, double* __restrict__ acc, const double* __restrict__ done) {
    __shared__ float spx[kWaPinCap], spy[kWaPinCap];
    __shared__ int scell[kWaPinCap];
    if (done && *done != 0.0) return;
    if (gamma_dev) gamma = (float)*gamma_dev;
    const float inv_g = 1.0f / gamma;
    const int e0 = blockIdx.x * kWaThreads;
    const int e1 = min(e0 + kWaThreads, E);
    const int p0 = net_ptr[e0], p1 = net_ptr[e1];
    const bool staged = (p1 - p0) <= kWaPinCap;
    if (staged) {
        for (int p = p0 + threadIdx.x; p < p1; p += kWaThreads) {
            int c = pin_cell[p];
            float cx, cy;
            if (c < m_mov) { cx = x[c]; cy = y[c]; }
            else { cx = fx[c - m_mov]; cy = fy[c - m_mov]; }
            spx[p - p0] = __fadd_rn(cx, pdx[p]);
            spy[p - p0] = __fadd_rn(cy, pdy[p]);
            scell[p - p0] = c;
        }
    }
    __syncthreads();
    auto pin = [&](int p, float& px, float& py, int& c) {
        if (staged) {
            px = spx[p - p0]; py = spy[p - p0]; c = scell[p - p0];
        } else {
            c = pin_cell[p];
            float cx, cy;
            if (c < m_mov) { cx = x[c]; cy = y[c]; }
            else { cx = fx[c - m_mov]; cy = fy[c - m_mov]; }
            px = __fadd_rn(cx, pdx[p]);
            py = __fadd_rn(cy, pdy[p]);
        }
    };
    dfloat wsum = df_zero(), hsum = df_zero();
    const int e = e0 + threadIdx.x;
    if (e < E) {
        const int a = net_ptr[e], b = net_ptr[e + 1];
        if (b - a >= 2) {
            float Mx = -INFINITY, My = -INFINITY, mx = INFINITY, my = INFINITY;
            for (int p = a; p < b; ++p) {
                float px, py; int c;
                pin(p, px, py, c);
                Mx = fmaxf(Mx, px); mx = fminf(mx, px);
                My = fmaxf(My, py); my = fminf(my, py);
            }
            float Spx = 0, Tpx = 0, Smx = 0, Tmx = 0, Spy = 0, Tpy = 0, Smy = 0, Tmy = 0;
            for (int p = a; p < b; ++p) {
                float px, py; int c;
                pin(p, px, py, c);
                float tpx = px - Mx, tmx = px - mx, tpy = py - My, tmy = py - my;
                float apx = expf(tpx * inv_g), amx = expf(-tmx * inv_g);
                float apy = expf(tpy * inv_g), amy = expf(-tmy * inv_g);
                Spx += apx; Tpx = fmaf(tpx, apx, Tpx); Smx += amx; Tmx = fmaf(tmx, amx, Tmx);
                Spy += apy; Tpy = fmaf(tpy, apy, Tpy); Smy += amy; Tmy = fmaf(tmy, amy, Tmy);
            }
            const float Wpx = Tpx / Spx, Wmx = Tmx / Smx, Wpy = Tpy / Spy, Wmy = Tmy / Smy;
            const float isx = 1.0f / Spx, imx = 1.0f / Smx, isy = 1.0f / Spy, imy = 1.0f / Smy;
            dfloat spanx = df_add({Mx, 0.0f}, -mx);
            dfloat spany = df_add({My, 0.0f}, -my);
            hsum = df_add(spanx, spany);
            wsum = df_add(df_add(spanx, spany), (Wpx - Wmx) + (Wpy - Wmy));
            for (int p = a; p < b; ++p) {
                float px, py; int c;
                pin(p, px, py, c);
                float tpx = px - Mx, tmx = px - mx, tpy = py - My, tmy = py - my;
                float apx = expf(tpx * inv_g), amx = expf(-tmx * inv_g);
                float apy = expf(tpy * inv_g), amy = expf(-tmy * inv_g);
                float gxj = apx * isx * (1.0f + (tpx - Wpx) * inv_g) -
                            amx * imx * (1.0f - (tmx - Wmx) * inv_g);
                float gyj = apy * isy * (1.0f + (tpy - Wpy) * inv_g) -
                            amy * imy * (1.0f - (tmy - Wmy) * inv_g);
                if (CSR) {
                    int sl = pin_slot[p];
                    if (sl >= 0) gpin[sl] = make_float2(gxj, gyj);
                } else if (c < m_mov) {
                    atomicAdd(gx + c, gxj);
                    atomicAdd(gy + c, gyj);
                }
            }
        } else if (CSR) {
            for (int p = a; p < b; ++p) {
                int sl = pin_slot[p];
                if (sl >= 0) gpin[sl] = make_float2(0.0f, 0.0f);
            }
        }
    }
    df_warp_atomic(wsum, acc + ACC_W);
    df_warp_atomic(hsum, acc + ACC_HPWL);
}

// Per-cell kernel: density gradient by the field gather (q.E of Eq. 7),
// wirelength gradient by summing the cell's pin gradients (CSR mode) or
// reading the atomically accumulated sums, and the L1 norms of both.
template <bool CSR>
__global__ void __launch_bounds__(kCellThreads)
k_cells(Grid g, int m, const float* __restrict__ x, const float* __restrict__ y,
        const float* __restrict__ w, const float* __restrict__ h, const float* __restrict__ ex,
        const float* __restrict__ ey, float* __restrict__ gNx, float* __restrict__ gNy,
        float* __restrict__ gWx, float* __restrict__ gWy, const int* __restrict__ cell_pin_ptr,
        const float2* __restrict__ gpin, double* __restrict__ acc,
        const double* __restrict__ done) {
    if (done && *done != 0.0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float nx = 0.0f, ny = 0.0f, wx = 0.0f, wy = 0.0f;
    if (i < m) {
        Span s = cell_span(g, x[i], y[i], w[i], h[i]);
        for (int j = s.jlo; j <= s.jhi; ++j) {
            float oy = ov_len(g.y0, g.hb, j, s.yl, s.yh);
            const float* rx = ex + (size_t)j * g.n;
            const float* ry = ey + (size_t)j * g.n;
            for (int k = s.ilo; k <= s.ihi; ++k) {
                float o = __fmul_rn(ov_len(g.x0, g.wb, k, s.xl, s.xh), oy);
                nx = fmaf(o, __ldg(rx + k), nx);
                ny = fmaf(o, __ldg(ry + k), ny);
            }
        }
        nx = -nx;
        ny = -ny;
        gNx[i] = nx;
        gNy[i] = ny;
        if (CSR) {
            int q0 = cell_pin_ptr[i], q1 = cell_pin_ptr[i + 1];
            for (int q = q0; q < q1; ++q) {
                float2 v = gpin[q];
                wx += v.x;
                wy += v.y;
            }
            gWx[i] = wx;
            gWy[i] = wy;
        } else {
            wx = gWx[i];
            wy = gWy[i];
        }
    }
    df_warp_atomic(df_add(df_zero(), fabsf(nx) + fabsf(ny)), acc + ACC_GN_L1);
    df_warp_atomic(df_add(df_zero(), fabsf(wx) + fabsf(wy)), acc + ACC_GW_L1);
}

// Deterministic pin-to-cell sum on its own (fftpl_wa in CSR mode).
__global__ void __launch_bounds__(kCellThreads)
k_pin_sum(int m, const int* __restrict__ cell_pin_ptr, const float2* __restrict__ gpin,
          float* __restrict__ gx, float* __restrict__ gy, double* __restrict__ l1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float wx = 0.0f, wy = 0.0f;
    if (i < m) {
        for (int q = cell_pin_ptr[i]; q < cell_pin_ptr[i + 1]; ++q) {
            float2 v = gpin[q];
            wx += v.x;
            wy += v.y;
        }
        gx[i] = wx;
        gy[i] = wy;
    }
    df_warp_atomic(df_add(df_zero(), fabsf(wx) + fabsf(wy)), l1);
}

__global__ void __launch_bounds__(kCellThreads)
k_l1(int m, const float* __restrict__ gx, const float* __restrict__ gy, double* __restrict__ l1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float v = 0.0f;
    if (i < m) v = fabsf(gx[i]) + fabsf(gy[i]);
    df_warp_atomic(df_add(df_zero(), v), l1);
}

static inline int nblk(long long m, int t) { return (int)((m + t - 1) / t); }

cudaError_t launch_wa_impl(Ctx& c, const float* x, const float* y, float gamma,
                           const double* gamma_dev, float* gx, float* gy, const double* done,
                           cudaStream_t s) {
    if (c.E <= 0) return cudaSuccess;
    int nb = nblk(c.E, kWaThreads);
    if (c.opt.deterministic)
        k_wa<true><<<nb, kWaThreads, 0, s>>>(c.E, c.net_ptr, c.pin_cell, c.pin_dx, c.pin_dy,
                                             c.m_mov, x, y, c.fix_x, c.fix_y, gamma, gamma_dev,
                                             nullptr, nullptr, c.pin_slot, c.gpin, c.acc, done);
    else
        k_wa<false><<<nb, kWaThreads, 0, s>>>(c.E, c.net_ptr, c.pin_cell, c.pin_dx, c.pin_dy,
                                              c.m_mov, x, y, c.fix_x, c.fix_y, gamma, gamma_dev,
                                              gx, gy, nullptr, nullptr, c.acc, done);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_wa(Ctx& c, const float* x, const float* y, float gamma, float* gx, float* gy,
                      cudaStream_t s) {
    return launch_wa_impl(c, x, y, gamma, nullptr, gx, gy, nullptr, s);
}

cudaError_t launch_pin_sum(Ctx& c, float* gx, float* gy, cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    if (c.opt.deterministic)
        k_pin_sum<<<nblk(c.m_mov, kCellThreads), kCellThreads, 0, s>>>(c.m_mov, c.cell_pin_ptr,
                                                                      c.gpin, gx, gy,
                                                                      c.acc + ACC_GW_L1);
    else
        k_l1<<<nblk(c.m_mov, kCellThreads), kCellThreads, 0, s>>>(c.m_mov, gx, gy,
                                                                 c.acc + ACC_GW_L1);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cells_impl(Ctx& c, const float* x, const float* y, float* gNx, float* gNy,
                              float* gWx, float* gWy, const double* done, cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    int nb = nblk(c.m_mov, kCellThreads);
    if (c.opt.deterministic)
        k_cells<true><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, c.ex, c.ey, gNx,
                                                  gNy, gWx, gWy, c.cell_pin_ptr, c.gpin, c.acc,
                                                  done);
    else
        k_cells<false><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, c.ex, c.ey,
                                                   gNx, gNy, gWx, gWy, nullptr, nullptr, c.acc,
                                                   done);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cells(Ctx& c, const float* x, const float* y, float* gNx, float* gNy,
                         float* gWx, float* gWy, cudaStream_t s) {
    return launch_cells_impl(c, x, y, gNx, gNy, gWx, gWy, nullptr, s);
}

}  // namespace fftpl
