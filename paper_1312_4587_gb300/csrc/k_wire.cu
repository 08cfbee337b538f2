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
// The wirelength gradient of a pin goes to its cell with one 8-byte vector
// atomic into an interleaved (x, y) accumulator, or, in deterministic mode,
// to the pin's slot in a cell-ordered array that the cell kernel sums.
#include "fftpl_internal.cuh"

namespace fftpl {

// Nets are re-laid at create time into slabs of up to 32 nets of one degree
// d (slab = {first pin slot, d, net count}); pin k of the slab's net j sits
// at slot base + 32 k + j.  One warp takes one slab, one lane one net: every
// lane walks the same d pins (no divergence) and each pin load of the warp is
// one contiguous 128-byte access.  The first kWaRegPins pins stay in registers
// across the three passes; further pins are reloaded (L1 hits).
constexpr int kWaRegPins = 8;

template <bool CSR>
__global__ void __launch_bounds__(kWaThreads)
k_wa(int nslabs, const int4* __restrict__ slabs, const int* __restrict__ pin_cell,
     const float* __restrict__ pdx, const float* __restrict__ pdy, int m_mov,
     const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ fx,
     const float* __restrict__ fy, float gamma, const double* __restrict__ gamma_dev,
     float2* __restrict__ gW, const int* __restrict__ pin_slot, float2* __restrict__ gpin,
     double* __restrict__ acc, const double* __restrict__ done) {
    if (done && *done != 0.0) return;
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (gamma_dev) gamma = (float)*gamma_dev;
    const float inv_g = 1.0f / gamma;
    const int4 sl = warp < nslabs ? slabs[warp] : make_int4(0, 0, 0, 0);
    const int base = sl.x + lane, d = sl.y;
    const bool act = lane < sl.z;
    auto load = [&](int k, float& px, float& py, int& c) {
        int i = base + 32 * k;
        c = pin_cell[i];
        float cx, cy;
        if (c < m_mov) { cx = x[c]; cy = y[c]; }
        else { cx = fx[c - m_mov]; cy = fy[c - m_mov]; }
        px = __fadd_rn(cx, pdx[i]);
        py = __fadd_rn(cy, pdy[i]);
    };
    float rx[kWaRegPins], ry[kWaRegPins];
    int rc[kWaRegPins];
    float Mx = -INFINITY, My = -INFINITY, mx = INFINITY, my = INFINITY;
    dfloat wsum = df_zero(), hsum = df_zero();
    if (act) {
#pragma unroll
        for (int k = 0; k < kWaRegPins; ++k) {
            if (k < d) {
                load(k, rx[k], ry[k], rc[k]);
                Mx = fmaxf(Mx, rx[k]); mx = fminf(mx, rx[k]);
                My = fmaxf(My, ry[k]); my = fminf(my, ry[k]);
            }
        }
        for (int k = kWaRegPins; k < d; ++k) {
            float px, py; int c;
            load(k, px, py, c);
            Mx = fmaxf(Mx, px); mx = fminf(mx, px);
            My = fmaxf(My, py); my = fminf(my, py);
        }
        float Spx = 0, Tpx = 0, Smx = 0, Tmx = 0, Spy = 0, Tpy = 0, Smy = 0, Tmy = 0;
        auto accum = [&](float px, float py) {
            float tpx = px - Mx, tmx = px - mx, tpy = py - My, tmy = py - my;
            float apx = expf(tpx * inv_g), amx = expf(-tmx * inv_g);
            float apy = expf(tpy * inv_g), amy = expf(-tmy * inv_g);
            Spx += apx; Tpx = fmaf(tpx, apx, Tpx); Smx += amx; Tmx = fmaf(tmx, amx, Tmx);
            Spy += apy; Tpy = fmaf(tpy, apy, Tpy); Smy += amy; Tmy = fmaf(tmy, amy, Tmy);
        };
#pragma unroll
        for (int k = 0; k < kWaRegPins; ++k)
            if (k < d) accum(rx[k], ry[k]);
        for (int k = kWaRegPins; k < d; ++k) {
            float px, py; int c;
            load(k, px, py, c);
            accum(px, py);
        }
        const float Wpx = Tpx / Spx, Wmx = Tmx / Smx, Wpy = Tpy / Spy, Wmy = Tmy / Smy;
        const float isx = 1.0f / Spx, imx = 1.0f / Smx, isy = 1.0f / Spy, imy = 1.0f / Smy;
        dfloat spanx = df_add({Mx, 0.0f}, -mx);
        dfloat spany = df_add({My, 0.0f}, -my);
        hsum = df_add(spanx, spany);
        wsum = df_add(hsum, (Wpx - Wmx) + (Wpy - Wmy));
        auto emit = [&](int k, float px, float py, int c) {
            float tpx = px - Mx, tmx = px - mx, tpy = py - My, tmy = py - my;
            float apx = expf(tpx * inv_g), amx = expf(-tmx * inv_g);
            float apy = expf(tpy * inv_g), amy = expf(-tmy * inv_g);
            float gxj = apx * isx * (1.0f + (tpx - Wpx) * inv_g) -
                        amx * imx * (1.0f - (tmx - Wmx) * inv_g);
            float gyj = apy * isy * (1.0f + (tpy - Wpy) * inv_g) -
                        amy * imy * (1.0f - (tmy - Wmy) * inv_g);
            if (CSR) {
                int sl2 = pin_slot[base + 32 * k];
                if (sl2 >= 0) gpin[sl2] = make_float2(gxj, gyj);
            } else if (c < m_mov) {
                atomicAdd(gW + c, make_float2(gxj, gyj));
            }
        };
#pragma unroll
        for (int k = 0; k < kWaRegPins; ++k)
            if (k < d) emit(k, rx[k], ry[k], rc[k]);
        for (int k = kWaRegPins; k < d; ++k) {
            float px, py; int c;
            load(k, px, py, c);
            emit(k, px, py, c);
        }
    }
    block_acc2(wsum, hsum, acc, ACC_W, ACC_HPWL);
}

// Per-cell kernel: density gradient by the field gather (q.E of Eq. 7),
// wirelength gradient by summing the cell's pin gradients (CSR mode) or
// reading the atomically accumulated sums, and the L1 norms of both.
template <bool CSR>
__global__ void __launch_bounds__(kCellThreads)
k_cells(Grid g, int m, const float* __restrict__ x, const float* __restrict__ y,
        const float* __restrict__ w, const float* __restrict__ h, const float2* __restrict__ E2,
        float* __restrict__ gNx, float* __restrict__ gNy,
        float* __restrict__ gWx, float* __restrict__ gWy, const int* __restrict__ cell_pin_ptr,
        const float2* __restrict__ gpin, const float2* __restrict__ gW2, double* __restrict__ acc,
        const double* __restrict__ done) {
    if (done && *done != 0.0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float nx = 0.0f, ny = 0.0f, wx = 0.0f, wy = 0.0f;
    if (i < m) {
        Span s = cell_span(g, x[i], y[i], w[i], h[i]);
        float2 e = gather_span(g, s, E2);
        nx = -e.x;
        ny = -e.y;
        gNx[i] = nx;
        gNy[i] = ny;
        if (CSR) {
            int q0 = cell_pin_ptr[i], q1 = cell_pin_ptr[i + 1];
            for (int q = q0; q < q1; ++q) {
                float2 v = gpin[q];
                wx += v.x;
                wy += v.y;
            }
        } else {
            float2 v = gW2[i];
            wx = v.x;
            wy = v.y;
        }
        gWx[i] = wx;
        gWy[i] = wy;
    }
    block_acc2(dfloat{fabsf(nx) + fabsf(ny), 0.0f}, dfloat{fabsf(wx) + fabsf(wy), 0.0f}, acc,
               ACC_GN_L1, ACC_GW_L1);
}

// Deterministic pin-to-cell sum on its own (fftpl_wa in CSR mode).
__global__ void __launch_bounds__(kCellThreads)
k_pin_sum(int m, const int* __restrict__ cell_pin_ptr, const float2* __restrict__ gpin,
          float* __restrict__ gx, float* __restrict__ gy, double* __restrict__ acc) {
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
    block_acc1(dfloat{fabsf(wx) + fabsf(wy), 0.0f}, acc, ACC_GW_L1);
}

// Splits the interleaved atomic accumulator into gx, gy and adds ||g||_1.
__global__ void __launch_bounds__(kCellThreads)
k_split(int m, const float2* __restrict__ gW2, float* __restrict__ gx, float* __restrict__ gy,
        double* __restrict__ acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float v = 0.0f;
    if (i < m) {
        float2 g = gW2[i];
        gx[i] = g.x;
        gy[i] = g.y;
        v = fabsf(g.x) + fabsf(g.y);
    }
    block_acc1(dfloat{v, 0.0f}, acc, ACC_GW_L1);
}

static inline int nblk(long long m, int t) { return (int)((m + t - 1) / t); }

cudaError_t launch_wa_impl(Ctx& c, const float* x, const float* y, float gamma,
                           const double* gamma_dev, const double* done, cudaStream_t s) {
    if (c.nslabs <= 0) return cudaSuccess;
    const int wpb = kWaThreads / 32;
    int nb = nblk(c.nslabs, wpb);
    if (c.opt.deterministic)
        k_wa<true><<<nb, kWaThreads, 0, s>>>(c.nslabs, c.slabs, c.pin_cell, c.pin_dx, c.pin_dy,
                                             c.m_mov, x, y, c.fix_x, c.fix_y, gamma, gamma_dev,
                                             nullptr, c.pin_slot, c.gpin, c.acc, done);
    else
        k_wa<false><<<nb, kWaThreads, 0, s>>>(c.nslabs, c.slabs, c.pin_cell, c.pin_dx, c.pin_dy,
                                              c.m_mov, x, y, c.fix_x, c.fix_y, gamma, gamma_dev,
                                              c.gW2, nullptr, nullptr, c.acc, done);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_wa(Ctx& c, const float* x, const float* y, float gamma, cudaStream_t s) {
    return launch_wa_impl(c, x, y, gamma, nullptr, nullptr, s);
}

cudaError_t launch_pin_sum(Ctx& c, float* gx, float* gy, cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    if (c.opt.deterministic)
        k_pin_sum<<<nblk(c.m_mov, kCellThreads), kCellThreads, 0, s>>>(c.m_mov, c.cell_pin_ptr,
                                                                      c.gpin, gx, gy,
                                                                      c.acc);
    else
        k_split<<<nblk(c.m_mov, kCellThreads), kCellThreads, 0, s>>>(c.m_mov, c.gW2, gx, gy,
                                                                    c.acc);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cells_impl(Ctx& c, const float* x, const float* y, float* gNx, float* gNy,
                              float* gWx, float* gWy, const double* done, cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    int nb = nblk(c.m_mov, kCellThreads);
    if (c.opt.deterministic)
        k_cells<true><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, c.E2, gNx,
                                                  gNy, gWx, gWy, c.cell_pin_ptr, c.gpin, nullptr,
                                                  c.acc, done);
    else
        k_cells<false><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, c.E2,
                                                   gNx, gNy, gWx, gWy, nullptr, nullptr, c.gW2,
                                                   c.acc, done);
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cells(Ctx& c, const float* x, const float* y, float* gNx, float* gNy,
                         float* gWx, float* gWy, cudaStream_t s) {
    return launch_cells_impl(c, x, y, gNx, gNy, gWx, gWy, nullptr, s);
}

}  // namespace fftpl
