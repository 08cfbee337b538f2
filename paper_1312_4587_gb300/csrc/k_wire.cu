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
// reduction (red, no return value) into an interleaved (x, y) accumulator,
// or, in deterministic mode, to the pin's slot in a cell-ordered array that
// the cell kernel sums.
#include "fftpl_internal.cuh"

namespace fftpl {

// Nets are re-laid at create time into slabs of nets of one degree d (slab
// = {first pin slot, d, net count, lanes per net}).  Below kBigMin and
// above kBigMax a slab holds up to 32 nets, pin k of its net j at slot
// base + 32 k + j: one warp per slab, one lane per net, every lane walks the
// same d pins (no divergence), each pin-record read of the warp is one
// contiguous access, and the cell-centre gathers of a slab touch nearby
// lines (cells are numbered by regions of the netlist).  k_wa takes these
// (degree 2..6: the bulk of the nets, a body specialised for the degree,
// pin coordinates in registers, two slabs per warp for degree 2..4 on large
// instances; above kBigMax: runtime degree, coordinates staged in pxy).
// k_wa_grp takes the slabs of degree kBigMin..kBigMax, several lanes per net
// with shuffle reductions (see wa_group).

// (x, y) -> interleaved positions at each cell's internal number, so that
// one 8-byte load (one sector) fetches a pin's cell centre and the pins of a
// slab read nearby sectors.
__global__ void __launch_bounds__(256)
k_interleave(int m, const float* __restrict__ x, const float* __restrict__ y,
             const int* __restrict__ rank, float2* __restrict__ pos,
             const float* __restrict__ done) {
    if (done && *done != 0.0f) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) pos[rank[i]] = make_float2(x[i], y[i]);
}

// Per-net WA of one lane's net, D known at compile time (D > 0) or not
// (D == 0: runtime degree d).  Pin coordinate = fl32(cell centre + offset),
// the centre gathered from pos by the pin's internal cell number (a pin on a
// fixed cell carries -1 and its absolute coordinate as the offset).  For
// D > 0 the pins live in registers; for D == 0 the first pass stores the pin
// coordinates in the pin's own slot of pxy and the later passes re-read them.
// Adds W~ and the HPWL term to wsum/hsum and sends each pin's gradient out.
struct WaIo {
    const int* pin_cell;
    const float* pin_dx;
    const float* pin_dy;
    const float2* pos;
    float2* pxy;
    float2* gW;
    const int* pin_slot;
    float2* gpin;
};

__device__ __forceinline__ float2 pin_xy(const WaIo& io, int c, float ox, float oy) {
    const float2 p = c >= 0 ? io.pos[c] : make_float2(0.0f, 0.0f);
    return make_float2(__fadd_rn(p.x, ox), __fadd_rn(p.y, oy));
}

// One axis of a two-pin net, with d = |p1 - p2| and e = exp(-d/g) (the
// per-net shift of Eq. 3 leaves the terms 1 and e): W~ = d (1 - e)/(1 + e)
// = d tanh(d / 2g), and the pin at the maximum moves W~ by
// dW~/dd = tanh(d/2g) + (d/2g) sech^2(d/2g) = (1 - e)/(1 + e) + 2 (d/g) e/(1 + e)^2
// (the pin at the minimum by its negative).  LSE: W = d + 2 g ln(1 + e),
// dW/dd = (1 - e)/(1 + e).  Returns W~ (or W - d for LSE); *g1 = gradient
// of pin 1.
template <bool LSE>
__device__ __forceinline__ float wa_axis2(float p1, float p2, float l2g, float inv_g, float* g1) {
    const float d = fabsf(p1 - p2);
    const float e = exp2f(-d * l2g);
    const float r = __fdividef(1.0f, 1.0f + e);   // 1 + e in [1, 2]
    const float th = (1.0f - e) * r;
    float gd, w;
    if (LSE) {
        gd = th;
        w = __fdividef(2.0f, inv_g) * log1pf(e);
    } else {
        gd = fmaf(2.0f * d * inv_g * e, r * r, th);
        w = d * th;
    }
    *g1 = p1 >= p2 ? gd : -gd;
    return w;
}

template <bool CSR, bool LSE>
__device__ __forceinline__ void wa_core2(const float (&rx)[2], const float (&ry)[2], int base,
                                         const WaIo& io, float l2g, float inv_g, float& wsum,
                                         float& hsum) {
    float gx, gy;
    const float wx = wa_axis2<LSE>(rx[0], rx[1], l2g, inv_g, &gx);
    const float wy = wa_axis2<LSE>(ry[0], ry[1], l2g, inv_g, &gy);
    const float span = fabsf(rx[0] - rx[1]) + fabsf(ry[0] - ry[1]);
    hsum += span;
    wsum += LSE ? span + (wx + wy) : wx + wy;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float sg = k == 0 ? 1.0f : -1.0f;
        if (CSR) {
            int sl = io.pin_slot[base + 32 * k];
            if (sl >= 0) io.gpin[sl] = make_float2(sg * gx, sg * gy);
        } else {
            int c = io.pin_cell[base + 32 * k];
            if (c >= 0) red_add_f2(io.gW + c, sg * gx, sg * gy);
        }
    }
}

// WA of one net whose D pin coordinates are in registers: max/min, the
// exponential sums, W~ and HPWL into wsum/hsum, and the pin gradients out
// (the pin's cell number, or its deterministic slot, is re-read at the pin's
// slot base + 32 k: an L1 hit, cheaper than holding it in registers).
// Two-pin nets (D = 2) take the closed form above.
template <int D, bool CSR, bool LSE>
__device__ __forceinline__ void wa_core(const float (&rx)[D], const float (&ry)[D], int base,
                                        const WaIo& io, float l2g, float inv_g, float& wsum,
                                        float& hsum) {
    if constexpr (D == 2) {
        wa_core2<CSR, LSE>(rx, ry, base, io, l2g, inv_g, wsum, hsum);
        return;
    }
    // the exponentials are recomputed in the gradient loop (the same
    // operations, so the same values) rather than held in 4 D registers
    float Mx = -INFINITY, My = -INFINITY, mx = INFINITY, my = INFINITY;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        Mx = fmaxf(Mx, rx[k]); mx = fminf(mx, rx[k]);
        My = fmaxf(My, ry[k]); my = fminf(my, ry[k]);
    }
    float Spx = 0, Tpx = 0, Smx = 0, Tmx = 0, Spy = 0, Tpy = 0, Smy = 0, Tmy = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float tpx = rx[k] - Mx, tmx = rx[k] - mx, tpy = ry[k] - My, tmy = ry[k] - my;
        const float apx = exp2f(tpx * l2g), amx = exp2f(-tmx * l2g);
        const float apy = exp2f(tpy * l2g), amy = exp2f(-tmy * l2g);
        Spx += apx; Tpx = fmaf(tpx, apx, Tpx); Smx += amx; Tmx = fmaf(tmx, amx, Tmx);
        Spy += apy; Tpy = fmaf(tpy, apy, Tpy); Smy += amy; Tmy = fmaf(tmy, amy, Tmy);
    }
    // every S is in [1, d] (its largest term is exp(0) = 1): the fast
    // reciprocal (2 ulp) is accurate over that whole range
    const float isx = __fdividef(1.0f, Spx), imx = __fdividef(1.0f, Smx);
    const float isy = __fdividef(1.0f, Spy), imy = __fdividef(1.0f, Smy);
    const float Wpx = Tpx * isx, Wmx = Tmx * imx, Wpy = Tpy * isy, Wmy = Tmy * imy;
    // one net per lane: its span and W~ in float32 (the FP64 sums start at
    // the warp totals)
    const float span = (Mx - mx) + (My - my);
    hsum += span;
    if (LSE) {
        // g (ln S+ + ln S-) per axis on top of the span; gradient
        // a+/S+ - a-/S- (softmax difference)
        wsum += span + __fdividef(1.0f, inv_g) * ((logf(Spx) + logf(Smx)) +
                                                  (logf(Spy) + logf(Smy)));
#pragma unroll
        for (int k = 0; k < D; ++k) {
            float tpx = rx[k] - Mx, tmx = rx[k] - mx, tpy = ry[k] - My, tmy = ry[k] - my;
            float gxj = exp2f(tpx * l2g) * isx - exp2f(-tmx * l2g) * imx;
            float gyj = exp2f(tpy * l2g) * isy - exp2f(-tmy * l2g) * imy;
            if (CSR) {
                int sl = io.pin_slot[base + 32 * k];
                if (sl >= 0) io.gpin[sl] = make_float2(gxj, gyj);
            } else {
                int c = io.pin_cell[base + 32 * k];
                if (c >= 0) red_add_f2(io.gW + c, gxj, gyj);
            }
        }
        return;
    }
    wsum += span + ((Wpx - Wmx) + (Wpy - Wmy));
    // dW~/dp = a+ (P0 + t+ P1) - a- (Q0 - t- Q1) per axis, with
    // P0 = (1 - W+/g)/S+, P1 = 1/(g S+), Q0 = (1 + W-/g)/S-, Q1 = 1/(g S-)
    const float P0x = isx * fmaf(-Wpx, inv_g, 1.0f), P1x = isx * inv_g;
    const float Q0x = imx * fmaf(Wmx, inv_g, 1.0f), Q1x = imx * inv_g;
    const float P0y = isy * fmaf(-Wpy, inv_g, 1.0f), P1y = isy * inv_g;
    const float Q0y = imy * fmaf(Wmy, inv_g, 1.0f), Q1y = imy * inv_g;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float tpx = rx[k] - Mx, tmx = rx[k] - mx, tpy = ry[k] - My, tmy = ry[k] - my;
        float gxj = exp2f(tpx * l2g) * fmaf(tpx, P1x, P0x) - exp2f(-tmx * l2g) * fmaf(-tmx, Q1x, Q0x);
        float gyj = exp2f(tpy * l2g) * fmaf(tpy, P1y, P0y) - exp2f(-tmy * l2g) * fmaf(-tmy, Q1y, Q0y);
        if (CSR) {
            int sl = io.pin_slot[base + 32 * k];
            if (sl >= 0) io.gpin[sl] = make_float2(gxj, gyj);
        } else {
            int c = io.pin_cell[base + 32 * k];
            if (c >= 0) red_add_f2(io.gW + c, gxj, gyj);
        }
    }
}

// Pin coordinates of a net of degree D at slot base: all record loads
// first, then all centre gathers.
template <int D>
__device__ __forceinline__ void wa_load(const WaIo& io, int base, float (&rx)[D], float (&ry)[D]) {
    int cr[D];
    float ox[D], oy[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        cr[k] = io.pin_cell[base + 32 * k];
        ox[k] = io.pin_dx[base + 32 * k];
        oy[k] = io.pin_dy[base + 32 * k];
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float2 p = pin_xy(io, cr[k], ox[k], oy[k]);
        rx[k] = p.x;
        ry[k] = p.y;
    }
}

template <int D, bool CSR, bool LSE>
__device__ __forceinline__ void wa_net(const WaIo& io, int base, float l2g, float inv_g,
                                       float& wsum, float& hsum) {
    float rx[D], ry[D];
    wa_load<D>(io, base, rx, ry);
    wa_core<D, CSR, LSE>(rx, ry, base, io, l2g, inv_g, wsum, hsum);
}

// Two nets of the same degree per lane (from two slabs): both nets' loads
// are in flight together.  A lane outside a slab's net count reads that
// slab's padding slots (cell -1) and skips the net.
template <int D, bool CSR, bool LSE>
__device__ __forceinline__ void wa_pair(const WaIo& io, int base_a, bool live_a, int base_b,
                                        bool live_b, float l2g, float inv_g, float& wsum,
                                        float& hsum) {
    float ax[D], ay[D], bx[D], by[D];
    wa_load<D>(io, base_a, ax, ay);
    wa_load<D>(io, base_b, bx, by);
    if (live_a) wa_core<D, CSR, LSE>(ax, ay, base_a, io, l2g, inv_g, wsum, hsum);
    if (live_b) wa_core<D, CSR, LSE>(bx, by, base_b, io, l2g, inv_g, wsum, hsum);
}

// Runtime degree d (slabs of degree > 6): the first pass stores the pin
// coordinates in the pins' own slots of pxy, the later passes re-read them.
template <bool CSR, bool LSE>
__device__ __forceinline__ void wa_net_any(const WaIo& io, int base, int d, float l2g,
                                           float inv_g, float& wsum, float& hsum) {
    float Mx = -INFINITY, My = -INFINITY, mx = INFINITY, my = INFINITY;
#pragma unroll 4
    for (int k = 0; k < d; ++k) {
        const int sl = base + 32 * k;
        float2 p = pin_xy(io, io.pin_cell[sl], io.pin_dx[sl], io.pin_dy[sl]);
        io.pxy[sl] = p;
        Mx = fmaxf(Mx, p.x); mx = fminf(mx, p.x);
        My = fmaxf(My, p.y); my = fminf(my, p.y);
    }
    float Spx = 0, Tpx = 0, Smx = 0, Tmx = 0, Spy = 0, Tpy = 0, Smy = 0, Tmy = 0;
#pragma unroll 4
    for (int k = 0; k < d; ++k) {
        float2 p = io.pxy[base + 32 * k];
        float tpx = p.x - Mx, tmx = p.x - mx, tpy = p.y - My, tmy = p.y - my;
        float apx = exp2f(tpx * l2g), amx = exp2f(-tmx * l2g);
        float apy = exp2f(tpy * l2g), amy = exp2f(-tmy * l2g);
        Spx += apx; Tpx = fmaf(tpx, apx, Tpx); Smx += amx; Tmx = fmaf(tmx, amx, Tmx);
        Spy += apy; Tpy = fmaf(tpy, apy, Tpy); Smy += amy; Tmy = fmaf(tmy, amy, Tmy);
    }
    const float isx = __fdividef(1.0f, Spx), imx = __fdividef(1.0f, Smx);
    const float isy = __fdividef(1.0f, Spy), imy = __fdividef(1.0f, Smy);
    const float Wpx = Tpx * isx, Wmx = Tmx * imx, Wpy = Tpy * isy, Wmy = Tmy * imy;
    const float span = (Mx - mx) + (My - my);
    hsum += span;
    if (LSE)
        wsum += span + __fdividef(1.0f, inv_g) * ((logf(Spx) + logf(Smx)) +
                                                  (logf(Spy) + logf(Smy)));
    else
        wsum += span + ((Wpx - Wmx) + (Wpy - Wmy));
    const float P0x = isx * fmaf(-Wpx, inv_g, 1.0f), P1x = isx * inv_g;
    const float Q0x = imx * fmaf(Wmx, inv_g, 1.0f), Q1x = imx * inv_g;
    const float P0y = isy * fmaf(-Wpy, inv_g, 1.0f), P1y = isy * inv_g;
    const float Q0y = imy * fmaf(Wmy, inv_g, 1.0f), Q1y = imy * inv_g;
#pragma unroll 4
    for (int k = 0; k < d; ++k) {
        const int sl = base + 32 * k;
        float2 p = io.pxy[sl];
        float tpx = p.x - Mx, tmx = p.x - mx, tpy = p.y - My, tmy = p.y - my;
        float gxj, gyj;
        if (LSE) {
            gxj = exp2f(tpx * l2g) * isx - exp2f(-tmx * l2g) * imx;
            gyj = exp2f(tpy * l2g) * isy - exp2f(-tmy * l2g) * imy;
        } else {
            gxj = exp2f(tpx * l2g) * fmaf(tpx, P1x, P0x) - exp2f(-tmx * l2g) * fmaf(-tmx, Q1x, Q0x);
            gyj = exp2f(tpy * l2g) * fmaf(tpy, P1y, P0y) - exp2f(-tmy * l2g) * fmaf(-tmy, Q1y, Q0y);
        }
        if (CSR) {
            int q = io.pin_slot[sl];
            if (q >= 0) io.gpin[q] = make_float2(gxj, gyj);
        } else {
            int c = io.pin_cell[sl];
            if (c >= 0) red_add_f2(io.gW + c, gxj, gyj);
        }
    }
}

template <bool CSR, bool LSE>
__device__ __forceinline__ void wa_slab(const WaIo& io, const int4& sl, int lane, float l2g,
                                        float inv_g, float& wsum, float& hsum) {
    if (lane >= sl.z) return;
    const int base = sl.x + lane;
    // the degree is the same for the whole warp, so this switch does not diverge
    switch (sl.y) {
        case 2: wa_net<2, CSR, LSE>(io, base, l2g, inv_g, wsum, hsum); break;
        case 3: wa_net<3, CSR, LSE>(io, base, l2g, inv_g, wsum, hsum); break;
        case 4: wa_net<4, CSR, LSE>(io, base, l2g, inv_g, wsum, hsum); break;
        case 5: wa_net<5, CSR, LSE>(io, base, l2g, inv_g, wsum, hsum); break;
        case 6: wa_net<6, CSR, LSE>(io, base, l2g, inv_g, wsum, hsum); break;
        default: wa_net_any<CSR, LSE>(io, base, sl.y, l2g, inv_g, wsum, hsum); break;
    }
}

// pairs != 0: one warp per pair of consecutive slabs (2w, 2w+1); when both
// have the same degree 2..4 (most nets) each lane runs its two nets with
// their loads in flight together, otherwise the slabs go one after the
// other.  pairs == 0: one warp per slab (small instances, where the GPU has
// room for a warp per slab and latency matters more).
template <bool CSR, bool LSE>
__global__ void __launch_bounds__(kWaThreads, 4)
k_wa(int nslabs, int pairs, const int4* __restrict__ slabs, WaIo io, float inv_g, float l2g,
     const float* __restrict__ scale_dev, double* __restrict__ acc,
     const float* __restrict__ done, DetRed dr) {
    if (done && *done != 0.0f) return;
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    // 1/gamma and log2(e)/gamma: from the loop's control mirror, or computed
    // on the host (exp(t / g) = exp2(t * log2(e) / g))
    if (scale_dev) {
        const float2 sc = *reinterpret_cast<const float2*>(scale_dev);
        inv_g = sc.x;
        l2g = sc.y;
    }
    const int4 zero = make_int4(0, 0, 0, 0);
    float wsum = 0.0f, hsum = 0.0f;
    if (!pairs) {
        const int4 sl = warp < nslabs ? slabs[warp] : zero;
        wa_slab<CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum);
        reduce2(wsum, hsum, acc, ACC_W, ACC_HPWL, dr);
        return;
    }
    const int4 sa = 2 * warp < nslabs ? slabs[2 * warp] : zero;
    const int4 sb = 2 * warp + 1 < nslabs ? slabs[2 * warp + 1] : zero;
    if (sa.y == sb.y && sa.y >= 2 && sa.y <= 4) {
        const bool la = lane < sa.z, lb = lane < sb.z;
        switch (sa.y) {
            case 2: wa_pair<2, CSR, LSE>(io, sa.x + lane, la, sb.x + lane, lb, l2g, inv_g, wsum, hsum); break;
            case 3: wa_pair<3, CSR, LSE>(io, sa.x + lane, la, sb.x + lane, lb, l2g, inv_g, wsum, hsum); break;
            default: wa_pair<4, CSR, LSE>(io, sa.x + lane, la, sb.x + lane, lb, l2g, inv_g, wsum, hsum); break;
        }
    } else {
        wa_slab<CSR, LSE>(io, sa, lane, l2g, inv_g, wsum, hsum);
        wa_slab<CSR, LSE>(io, sb, lane, l2g, inv_g, wsum, hsum);
    }
    reduce2(wsum, hsum, acc, ACC_W, ACC_HPWL, dr);
}

// ------------------------------------------------ slabs of degree 7..64
// L = grp_lanes(d) lanes per net (2 up to degree 8, 4 up to 16, 8 up to 32,
// 16 up to 64), 32 / L nets per warp, R = ceil(d / L) <= 4 pins per lane: lane
// g L + j of the slab holds pins j, j + L, ... of net g (slots base + 32 r +
// lane), so all of a net's record loads and centre gathers are in flight at
// once.  Each lane reduces its pins, then the L lanes of a net combine the
// maxima, minima and the exponential sums with xor shuffles (lanes of other
// nets are never mixed: the groups are aligned).  Lanes past the net's
// degree or past the slab's net count hold padding and take no part.
template <int L, int R, bool CSR, bool LSE>
__device__ __forceinline__ void wa_group(const WaIo& io, const int4& sl, int lane, float l2g,
                                         float inv_g, float& wsum, float& hsum) {
    const int j = lane % L;
    const bool live = lane / L < sl.z;
    const int d = sl.y;
    int cr[R];
    float ox[R], oy[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int slot = sl.x + 32 * r + lane;
        cr[r] = io.pin_cell[slot];
        ox[r] = io.pin_dx[slot];
        oy[r] = io.pin_dy[slot];
    }
    float px[R], py[R];
    bool ok[R];
    float Mx = -INFINITY, My = -INFINITY, mx = INFINITY, my = INFINITY;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ok[r] = live && r * L + j < d;
        const float2 p = pin_xy(io, cr[r], ox[r], oy[r]);
        px[r] = p.x;
        py[r] = p.y;
        if (ok[r]) {
            Mx = fmaxf(Mx, px[r]); mx = fminf(mx, px[r]);
            My = fmaxf(My, py[r]); my = fminf(my, py[r]);
        }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        Mx = fmaxf(Mx, __shfl_xor_sync(0xffffffffu, Mx, o));
        mx = fminf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        My = fmaxf(My, __shfl_xor_sync(0xffffffffu, My, o));
        my = fminf(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    float apx[R], amx[R], apy[R], amy[R];
    float Spx = 0, Tpx = 0, Smx = 0, Tmx = 0, Spy = 0, Tpy = 0, Smy = 0, Tmy = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float tpx = px[r] - Mx, tmx = px[r] - mx, tpy = py[r] - My, tmy = py[r] - my;
        apx[r] = ok[r] ? exp2f(tpx * l2g) : 0.0f;
        amx[r] = ok[r] ? exp2f(-tmx * l2g) : 0.0f;
        apy[r] = ok[r] ? exp2f(tpy * l2g) : 0.0f;
        amy[r] = ok[r] ? exp2f(-tmy * l2g) : 0.0f;
        Spx += apx[r]; Tpx = fmaf(tpx, apx[r], Tpx); Smx += amx[r]; Tmx = fmaf(tmx, amx[r], Tmx);
        Spy += apy[r]; Tpy = fmaf(tpy, apy[r], Tpy); Smy += amy[r]; Tmy = fmaf(tmy, amy[r], Tmy);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        Spx += __shfl_xor_sync(0xffffffffu, Spx, o);
        Tpx += __shfl_xor_sync(0xffffffffu, Tpx, o);
        Smx += __shfl_xor_sync(0xffffffffu, Smx, o);
        Tmx += __shfl_xor_sync(0xffffffffu, Tmx, o);
        Spy += __shfl_xor_sync(0xffffffffu, Spy, o);
        Tpy += __shfl_xor_sync(0xffffffffu, Tpy, o);
        Smy += __shfl_xor_sync(0xffffffffu, Smy, o);
        Tmy += __shfl_xor_sync(0xffffffffu, Tmy, o);
    }
    if (!live) return;
    // every S is in [1, d] (its largest term is exp(0) = 1)
    const float isx = __fdividef(1.0f, Spx), imx = __fdividef(1.0f, Smx);
    const float isy = __fdividef(1.0f, Spy), imy = __fdividef(1.0f, Smy);
    const float Wpx = Tpx * isx, Wmx = Tmx * imx, Wpy = Tpy * isy, Wmy = Tmy * imy;
    if (j == 0) {
        const float span = (Mx - mx) + (My - my);
        hsum += span;
        if (LSE)
            wsum += span + __fdividef(1.0f, inv_g) * ((logf(Spx) + logf(Smx)) +
                                                      (logf(Spy) + logf(Smy)));
        else
            wsum += span + ((Wpx - Wmx) + (Wpy - Wmy));
    }
    const float P0x = isx * fmaf(-Wpx, inv_g, 1.0f), P1x = isx * inv_g;
    const float Q0x = imx * fmaf(Wmx, inv_g, 1.0f), Q1x = imx * inv_g;
    const float P0y = isy * fmaf(-Wpy, inv_g, 1.0f), P1y = isy * inv_g;
    const float Q0y = imy * fmaf(Wmy, inv_g, 1.0f), Q1y = imy * inv_g;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!ok[r]) continue;
        const float tpx = px[r] - Mx, tmx = px[r] - mx, tpy = py[r] - My, tmy = py[r] - my;
        float gxj, gyj;
        if (LSE) {
            gxj = apx[r] * isx - amx[r] * imx;
            gyj = apy[r] * isy - amy[r] * imy;
        } else {
            gxj = apx[r] * fmaf(tpx, P1x, P0x) - amx[r] * fmaf(-tmx, Q1x, Q0x);
            gyj = apy[r] * fmaf(tpy, P1y, P0y) - amy[r] * fmaf(-tmy, Q1y, Q0y);
        }
        const int slot = sl.x + 32 * r + lane;
        if (CSR) {
            const int q = io.pin_slot[slot];
            if (q >= 0) io.gpin[q] = make_float2(gxj, gyj);
        } else if (cr[r] >= 0) {
            red_add_f2(io.gW + cr[r], gxj, gyj);
        }
    }
}

// One warp per slab of degree kBigMin..kBigMax.  Runs after k_wa on the same
// stream and adds to its totals.
template <bool CSR, bool LSE>
__global__ void __launch_bounds__(kWaThreads)
k_wa_grp(int nbig, const int4* __restrict__ slabs, WaIo io, float inv_g, float l2g,
         const float* __restrict__ scale_dev, double* __restrict__ acc,
         const float* __restrict__ done, DetRed dr, int* __restrict__ err) {
    if (done && *done != 0.0f) return;
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    // 1/gamma and log2(e)/gamma: from the loop's control mirror, or computed
    // on the host (exp(t / g) = exp2(t * log2(e) / g))
    if (scale_dev) {
        const float2 sc = *reinterpret_cast<const float2*>(scale_dev);
        inv_g = sc.x;
        l2g = sc.y;
    }
    float wsum = 0.0f, hsum = 0.0f;
    if (warp < nbig) {
        const int4 sl = slabs[warp];
        // (L, R) is the same for the whole warp: no divergence
        switch (sl.w * 8 + (sl.y + sl.w - 1) / sl.w) {
            case 2 * 8 + 4: wa_group<2, 4, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            case 4 * 8 + 2: wa_group<4, 2, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            case 4 * 8 + 3: wa_group<4, 3, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            case 4 * 8 + 4: wa_group<4, 4, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            case 8 * 8 + 3: wa_group<8, 3, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            case 8 * 8 + 4: wa_group<8, 4, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            case 16 * 8 + 3: wa_group<16, 3, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            case 16 * 8 + 4: wa_group<16, 4, CSR, LSE>(io, sl, lane, l2g, inv_g, wsum, hsum); break;
            default: if (lane == 0) atomicOr(err, ERR_BOUNDS); break;   // no such layout
        }
    }
    reduce2(wsum, hsum, acc, ACC_W, ACC_HPWL, dr, true);
}

// Per-cell kernel: density gradient by the field gather (q.E of Eq. 7),
// wirelength gradient by summing the cell's pin gradients (CSR mode) or
// reading the atomically accumulated sums, and the L1 norms of both.
// (6 blocks per SM: at most 40 registers, 48 warps to hide the gathers'
// latency; it runs alone after the join)
template <bool CSR>
__global__ void __launch_bounds__(kCellThreads, 6)
k_cells(Grid g, int m, const float* __restrict__ x, const float* __restrict__ y,
        const float* __restrict__ w, const float* __restrict__ h, const float2* __restrict__ E2,
        float* __restrict__ gNx, float* __restrict__ gNy,
        float* __restrict__ gWx, float* __restrict__ gWy, const int* __restrict__ rank,
        const int* __restrict__ cell_pin_ptr, const float2* __restrict__ gpin,
        const float2* __restrict__ gW2, double* __restrict__ acc,
        const float* __restrict__ done, DetRed dr) {
    if (done && *done != 0.0f) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float nx = 0.0f, ny = 0.0f, wx = 0.0f, wy = 0.0f;
    if (i < m) {
        // the wirelength gradient's loads go out before the field gather's
        const int r = rank[i];
        Span s = cell_span(g, x[i], y[i], w[i], h[i]);
        if (CSR) {
            int q0 = cell_pin_ptr[r], q1 = cell_pin_ptr[r + 1];
            for (int q = q0; q < q1; ++q) {
                float2 v = gpin[q];
                wx += v.x;
                wy += v.y;
            }
        } else {
            float2 v = gW2[r];
            wx = v.x;
            wy = v.y;
        }
        float2 e = gather_span(g, s, E2);
        nx = -e.x;
        ny = -e.y;
        gNx[i] = nx;
        gNy[i] = ny;
        gWx[i] = wx;
        gWy[i] = wy;
    }
    reduce2(fabsf(nx) + fabsf(ny), fabsf(wx) + fabsf(wy), acc, ACC_GN_L1, ACC_GW_L1, dr);
}

// Deterministic pin-to-cell sum on its own (fftpl_wa in CSR mode).
__global__ void __launch_bounds__(kCellThreads)
k_pin_sum(int m, const int* __restrict__ rank, const int* __restrict__ cell_pin_ptr,
          const float2* __restrict__ gpin, float* __restrict__ gx, float* __restrict__ gy,
          double* __restrict__ acc, DetRed dr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float wx = 0.0f, wy = 0.0f;
    if (i < m) {
        const int r = rank[i];
        for (int q = cell_pin_ptr[r]; q < cell_pin_ptr[r + 1]; ++q) {
            float2 v = gpin[q];
            wx += v.x;
            wy += v.y;
        }
        gx[i] = wx;
        gy[i] = wy;
    }
    reduce2(fabsf(wx) + fabsf(wy), 0.0f, acc, ACC_GW_L1, -1, dr);
}

// Splits the interleaved atomic accumulator into gx, gy and adds ||g||_1.
__global__ void __launch_bounds__(kCellThreads)
k_split(int m, const int* __restrict__ rank, const float2* __restrict__ gW2,
        float* __restrict__ gx, float* __restrict__ gy, double* __restrict__ acc, DetRed dr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float v = 0.0f;
    if (i < m) {
        float2 g = gW2[rank[i]];
        gx[i] = g.x;
        gy[i] = g.y;
        v = fabsf(g.x) + fabsf(g.y);
    }
    reduce2(v, 0.0f, acc, ACC_GW_L1, -1, dr);
}

static inline int nblk(long long m, int t) { return (int)((m + t - 1) / t); }

// Slab pairs per warp once a warp per slab would fill the GPU about twice
// over (4 CTAs of 8 warps per SM); below that, one slab per warp.
int wa_pairs(const Ctx& c) {
    return (c.nslabs - c.nbig) >= 2LL * c.num_sms * 4 * (kWaThreads / 32) ? 1 : 0;
}

cudaError_t launch_wa_impl(Ctx& c, const float* x, const float* y, float gamma,
                           const float* scale_dev, const float* done, bool interleave,
                           cudaStream_t s) {
    if (c.nslabs <= 0) return cudaSuccess;
    if (c.m_mov > 0 && interleave) {
        k_interleave<<<nblk(c.m_mov, 256), 256, 0, s>>>(c.m_mov, x, y, c.cell_rank, c.pos2,
                                                         done);
        c.launches++;
    }
    const WaIo io{c.pin_cell, c.pin_dx, c.pin_dy, c.pos2, c.pxy,
                  c.opt.deterministic ? nullptr : c.gW2, c.pin_slot, c.gpin};
    const bool lse = c.opt.wirelength == FFTPL_WL_LSE;
    const bool det = c.opt.deterministic != 0;
    float inv_g = 0.0f, l2g = 0.0f;
    if (!scale_dev) wa_scale(gamma, &inv_g, &l2g);
    // k_wa: the slabs after the first nbig (degree 2..6 and above kBigMax);
    // it stores the deterministic totals, k_wa_grp (next, same stream) adds
    const int nsmall = c.nslabs - c.nbig;
    if (nsmall > 0) {
        const int wpb = kWaThreads / 32;
        const int pairs = wa_pairs(c);
        const int nb = std::max(1, nblk(pairs ? (nsmall + 1) / 2 : nsmall, wpb));
        auto go = [&](auto kern) {
            kern<<<nb, kWaThreads, 0, s>>>(nsmall, pairs, c.slabs + c.nbig, io, inv_g, l2g,
                                           scale_dev, c.acc, done, det_red(c, 1));
        };
        if (det) {
            if (lse) go(k_wa<true, true>);
            else go(k_wa<true, false>);
        } else {
            if (lse) go(k_wa<false, true>);
            else go(k_wa<false, false>);
        }
        c.launches++;
    }
    if (c.nbig > 0) {
        const int nb = nblk(c.nbig, kWaThreads / 32);
        auto go = [&](auto kern) {
            kern<<<nb, kWaThreads, 0, s>>>(c.nbig, c.slabs, io, inv_g, l2g, scale_dev, c.acc,
                                           done, det_red(c, 1), c.err);
        };
        if (det) {
            if (lse) go(k_wa_grp<true, true>);
            else go(k_wa_grp<true, false>);
        } else {
            if (lse) go(k_wa_grp<false, true>);
            else go(k_wa_grp<false, false>);
        }
        c.launches++;
    }
    return cudaGetLastError();
}

cudaError_t launch_wa(Ctx& c, const float* x, const float* y, float gamma, cudaStream_t s) {
    return launch_wa_impl(c, x, y, gamma, nullptr, nullptr, true, s);
}

cudaError_t launch_pin_sum(Ctx& c, float* gx, float* gy, cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    // region 1: this pass follows the WA kernels on their stream
    if (c.opt.deterministic)
        k_pin_sum<<<nblk(c.m_mov, kCellThreads), kCellThreads, 0, s>>>(
            c.m_mov, c.cell_rank, c.cell_pin_ptr, c.gpin, gx, gy, c.acc, det_red(c, 1));
    else
        k_split<<<nblk(c.m_mov, kCellThreads), kCellThreads, 0, s>>>(
            c.m_mov, c.cell_rank, c.gW2, gx, gy, c.acc, det_red(c, 1));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cells_impl(Ctx& c, const float* x, const float* y, float* gNx, float* gNy,
                              float* gWx, float* gWy, const float* done, cudaStream_t s) {
    if (c.m_mov <= 0) return cudaSuccess;
    int nb = nblk(c.m_mov, kCellThreads);
    if (c.opt.deterministic)
        k_cells<true><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, c.E2, gNx,
                                                  gNy, gWx, gWy, c.cell_rank, c.cell_pin_ptr,
                                                  c.gpin, nullptr,
                                                  c.acc, done, det_red(c, 0));
    else
        k_cells<false><<<nb, kCellThreads, 0, s>>>(c.grid, c.m_mov, x, y, c.w, c.h, c.E2,
                                                   gNx, gNy, gWx, gWy, c.cell_rank, nullptr,
                                                   nullptr, c.gW2,
                                                   c.acc, done, det_red(c, 0));
    c.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cells(Ctx& c, const float* x, const float* y, float* gNx, float* gNy,
                         float* gWx, float* gWy, cudaStream_t s) {
    return launch_cells_impl(c, x, y, gNx, gNy, gWx, gWy, nullptr, s);
}

}  // namespace fftpl
