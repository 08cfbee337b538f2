// Spectral solution of Poisson's equation (Section III-E, Eqs. 8-12) on FP32
// fast Fourier transforms.
//
// With C(u,x) = cos(pi u (2x+1) / 2n) and S(u,x) = sin(...):
//   a[v][u] = eps_u eps_v / n^2  sum_y sum_x rho[y][x] C(u,x) C(v,y)   (Eq. 10)
//   Psi = a / (w_u^2 + w_v^2), Psi_00 = 0
//   psi[y][x] = sum_u C(u,x) P[u][y],        P[u][y] = sum_v Psi[v][u] C(v,y)
//   E_x[y][x] = sum_u w_u S(u,x) P[u][y]
//   E_y[y][x] = sum_u C(u,x) R[u][y],        R[u][y] = sum_v w_v Psi[v][u] S(v,y)
//
// Three passes, each over whole rows held in shared memory:
//   rows_fwd  : rho rows -> DCT-II along x -> T1[u][y] (written transposed)
//   cols      : T1 rows  -> DCT-II along y -> divide -> inverse along y for P
//               and R -> PT[y][u], RT[y][u] (written transposed); the energy
//               N = 1/2 A_b sum B Psi (Parseval) is reduced here
//   rows_inv  : PT, RT rows -> E_x, E_y rows (psi from PT on demand)
//
// Each 1-D cosine transform of length n is one complex FFT of length n
// (Makhoul's reordering: v[k] = r[2k], v[n-1-k] = r[2k+1]; A[u] =
// Re(exp(-i pi u / 2n) V[u])), two real rows packed into one complex FFT.
// The inverse cosine sum y[x] = sum_u c[u] C(u,x) is the inverse of that map;
// a sine sum is a cosine sum of the reversed coefficients times (-1)^x.
// The FFTs are radix-4 Stockham (plus one radix-2 stage for odd log2 n) in
// shared memory with twiddles from a float32 table computed in FP64: a
// radix-R butterfly loads W^(b st) for b = 1, 2, 4, 8 and forms the other
// R - 1 - log2 R by products, at most three deep (about 3 ulp; each table
// load costs more than the multiplies: 4 instead of 15 loads per radix-16
// butterfly took the three passes from 124 to 114 us).
#include "fftpl_internal.cuh"

namespace fftpl {

// ------------------------------------------------------------ FFT core
// Buffers are padded by one element every 16 (index i lives at i + i/16) so
// that the strided Stockham writes spread over the shared-memory banks.
__host__ __device__ constexpr int padded(int n) { return n + n / 16; }
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// ------------------------------------- stores through the TMA unit
// A pass that writes its output transposed first lays the tile out in shared
// memory in the output's order, then one thread stores it box by box with
// cp.async.bulk.tensor: the tile leaves the SM as whole rows of the box
// instead of one 16- or 32-byte piece per thread and store instruction.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Every thread that wrote part of a tile: its shared-memory writes become
// visible to the asynchronous proxy (before the barrier that precedes the
// store).
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The box at (c0, c1) (c0 innermost) of a 2-D tensor map from shared memory.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int c0,
                                             int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
            (unsigned long long)(uintptr_t)map),
        "r"(c0), "r"(c1), "r"(smem_addr(src))
        : "memory");
}

// Commit the stores issued so far and wait until they are complete (the
// hardware wait of the bulk-copy group: it ends when the copies have been
// written, not a spin loop).
__device__ __forceinline__ void tma_store_drain() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Twiddle exp(-+2 pi i k / 16) for the small exponents a radix-16 butterfly
// uses (cos and sin of multiples of pi/8).
__device__ __forceinline__ float2 w16(int e, bool inv) {
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
    float2 w;
    switch (e & 15) {
        case 0: w = make_float2(1.0f, 0.0f); break;
        case 1: w = make_float2(c1, -s1); break;
        case 2: w = make_float2(h, -h); break;
        case 3: w = make_float2(s1, -c1); break;
        case 4: w = make_float2(0.0f, -1.0f); break;
        case 6: w = make_float2(-h, -h); break;
        case 9: w = make_float2(-c1, s1); break;
        default: w = make_float2(1.0f, 0.0f); break;  // not used
    }
    if (inv) w.y = -w.y;
    return w;
}

// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ float2 rot(float2 a, bool inv) {
    return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

__device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

// in-place 4-point DFT of (a0, a1, a2, a3)
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3, bool inv) {
    float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
    float2 s13 = cadd(a1, a3), d13 = rot(csub(a1, a3), inv);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

// R-point DFT in registers, natural order in and out.
template <int R>
__device__ __forceinline__ void dft(float2 (&v)[R], bool inv);

template <>
__device__ __forceinline__ void dft<2>(float2 (&v)[2], bool) { dft2(v[0], v[1]); }

template <>
__device__ __forceinline__ void dft<4>(float2 (&v)[4], bool inv) { dft4(v[0], v[1], v[2], v[3], inv); }

template <>
__device__ __forceinline__ void dft<8>(float2 (&v)[8], bool inv) {
    // 8 = 2 x 4: DFT4 of even and odd samples, twiddle W8^k, combine
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3, inv);
    dft4(o0, o1, o2, o3, inv);
    o1 = cmul(o1, w16(2, inv));
    o2 = cmul(o2, w16(4, inv));
    o3 = cmul(o3, w16(6, inv));
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <>
__device__ __forceinline__ void dft<16>(float2 (&v)[16], bool inv) {
    // 16 = 4 x 4: X[k1 + 4 k2] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 x[4 n1 + n2] W4^(n1 k1)
    float2 y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        y[n2][0] = v[n2]; y[n2][1] = v[n2 + 4]; y[n2][2] = v[n2 + 8]; y[n2][3] = v[n2 + 12];
        dft4(y[n2][0], y[n2][1], y[n2][2], y[n2][3], inv);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1)
            if (n2 > 0) y[n2][k1] = cmul(y[n2][k1], w16(n2 * k1, inv));
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
        dft4(a0, a1, a2, a3, inv);
        v[k1] = a0; v[k1 + 4] = a1; v[k1 + 8] = a2; v[k1 + 12] = a3;
    }
}

// One Stockham stage of radix R over NB padded buffers of length N, with Ns
// the product of the radices already applied.  Reads everything it needs
// into registers, synchronises, then writes.
template <int LOGN, int NB, int R>
__device__ __forceinline__ void stockham_stage(float2* __restrict__ buf, const float2* __restrict__ tw,
                                               int Ns, bool inv) {
    constexpr int N = 1 << LOGN;
    constexpr int NP = padded(N);
    constexpr int T = kSpecThreads;
    constexpr int NR = N / R;
    constexpr int ITEMS = NB * NR;
    constexpr int PER = (ITEMS + T - 1) / T;
    float2 v[PER][R];
    int dst[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        int gi = threadIdx.x + i * T;
        dst[i] = -1;
        if (ITEMS % T == 0 || gi < ITEMS) {
            int f = gi / NR, j = gi % NR;
            int k = j & (Ns - 1);
            const float2* src = buf + f * NP;
            int st = (N / (R * Ns)) * k;   // twiddle index step: W_N^(r st)
            v[i][0] = src[pidx(j)];
            if (Ns == 1) {
                // first stage: every twiddle is exp(0) = 1
#pragma unroll
                for (int r = 1; r < R; ++r) v[i][r] = src[pidx(j + r * NR)];
            } else {
                // W^(r st) for r < R from the table's W^(st), W^(2 st),
                // W^(4 st), W^(8 st) by products (at most three deep)
                float2 w[R];
                w[0] = make_float2(1.0f, 0.0f);
#pragma unroll
                for (int b = 1; b < R; b <<= 1) w[b] = tw[b * st];
#pragma unroll
                for (int r = 3; r < R; ++r)
                    if (r & (r - 1)) w[r] = cmul(w[r & (r - 1)], w[r & -r]);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 ww = w[r];
                    if (inv) ww.y = -ww.y;
                    v[i][r] = cmul(src[pidx(j + r * NR)], ww);
                }
            }
            dst[i] = (f << 24) | ((j - k) * R + k);   // buffer and element index
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        if (dst[i] < 0) continue;
        dft<R>(v[i], inv);
        float2* out = buf + (dst[i] >> 24) * NP;
        int o = dst[i] & 0xffffff;
#pragma unroll
        for (int r = 0; r < R; ++r) out[pidx(o + r * Ns)] = v[i][r];
    }
    __syncthreads();
}

// NB complex FFTs of length N = 2^LOGN in the padded buffers.  Forward:
// X[k] = sum x[j] exp(-2 pi i jk / N); inverse: + sign, no 1/N.  Radix-16
// stages first, then one radix-2/4/8 stage for the remaining factor.
template <int LOGN, int NB>
__device__ __forceinline__ void fft_block(float2* __restrict__ buf, const float2* __restrict__ tw,
                                          bool inv) {
    int Ns = 1;
#pragma unroll
    for (int s = 0; s + 4 <= LOGN; s += 4) {
        stockham_stage<LOGN, NB, 16>(buf, tw, Ns, inv);
        Ns <<= 4;
    }
    constexpr int REM = LOGN & 3;
    if (REM == 1) stockham_stage<LOGN, NB, 2>(buf, tw, Ns, inv);
    if (REM == 2) stockham_stage<LOGN, NB, 4>(buf, tw, Ns, inv);
    if (REM == 3) stockham_stage<LOGN, NB, 8>(buf, tw, Ns, inv);
}

// Position of sample x in Makhoul's reordering.
__device__ __forceinline__ int mk_pos(int x, int N) { return (x & 1) ? (N - 1 - (x >> 1)) : (x >> 1); }
// Sample of the natural order held at position k of the reordering.
__device__ __forceinline__ int mk_src(int y, int N) { return (y & 1) ? (N - 1 - (y >> 1)) : (y >> 1); }

// Spectrum of an inverse-cosine pair packed for one complex IFFT.  For the
// sums y1 = sum c1[u] C(u,.), y2 = sum c2[u] C(u,.), with ct[0] = c[0],
// ct[u] = c[u]/2 (u >= 1), ct[N] = 0:
//   Z[u] = exp(i pi u / 2N) * ((ct1[u] + ct2[N-u]) + i (ct2[u] - ct1[N-u]))
// and then y1 + i y2 = unshuffle(IFFT(Z)).
__device__ __forceinline__ float2 pack_inv(float c1u, float c1nu, float c2u, float c2nu, float2 ph) {
    float re = c1u + c2nu, im = c2u - c1nu;
    // multiply by conj(ph) = exp(+i pi u / 2N)
    return make_float2(re * ph.x + im * ph.y, im * ph.x - re * ph.y);
}

// -------------------------------------------------------- pass 1: rows
// CTA: 8 rows of rho (2 per complex buffer).  Writes T1[u][y0..y0+7].
// At most 96 registers below n = 4096 (it needs no more): two blocks leave
// room on the SM for a block of the concurrent WA kernel (measured 2 %
// faster steps than with 128).  At n = 4096 the four buffers (139 KB) allow
// one block per SM in every pass, which may then use all its registers
// instead of spilling.
template <int LOGN, bool QUANT>
__global__ void __maxnreg__(LOGN >= 12 ? 255 : 96)
k_rows_fwd(const float* __restrict__ D, const long long* __restrict__ Dq,
           const float* __restrict__ M, float inv_ab, float cap, float* __restrict__ T1,
           const float2* __restrict__ tw, const float2* __restrict__ ph, double* __restrict__ acc,
           DetRed dr, const __grid_constant__ CUtensorMap mT1, int tma) {
    constexpr int N = 1 << LOGN;
    constexpr int NB = kSpecBuffers;
    constexpr int ROWS = 2 * NB;
    constexpr int T = kSpecThreads;
    constexpr int NP = padded(N);
    extern __shared__ __align__(128) float2 sm[];
    const int y0 = blockIdx.x * ROWS;
    // per-thread sums of at most 8 n / 256 non-negative terms in float32
    float tau = 0.0f, charge = 0.0f;
    // Buffer f packs rows 2f (real part) and 2f+1 (imaginary part) in
    // Makhoul's order: item p reads samples 2p and 2p+1 of both rows
    // (8-byte loads, a warp reads 256 contiguous bytes of each row) and
    // writes positions p and N-1-p (consecutive across the warp: no bank
    // conflicts)
    constexpr int ITEMS_IN = NB * (N / 2);
#pragma unroll 4
    for (int it = 0; it < (ITEMS_IN + T - 1) / T; ++it) {
        const int q = threadIdx.x + it * T;
        if (ITEMS_IN % T != 0 && q >= ITEMS_IN) break;
        const int f = q / (N / 2), pp = q % (N / 2);
        const size_t b0 = (size_t)(y0 + 2 * f) * N + 2 * pp, b1 = b0 + N;
        float d[4], mm[4];
        const float2 m0 = *reinterpret_cast<const float2*>(M + b0);
        const float2 m1 = *reinterpret_cast<const float2*>(M + b1);
        mm[0] = m0.x; mm[1] = m0.y; mm[2] = m1.x; mm[3] = m1.y;
        if (QUANT) {
            const longlong2 q0 = *reinterpret_cast<const longlong2*>(Dq + b0);
            const longlong2 q1 = *reinterpret_cast<const longlong2*>(Dq + b1);
            d[0] = (float)q0.x * 2.3283064365386963e-10f;
            d[1] = (float)q0.y * 2.3283064365386963e-10f;
            d[2] = (float)q1.x * 2.3283064365386963e-10f;
            d[3] = (float)q1.y * 2.3283064365386963e-10f;
        } else {
            const float2 v0 = *reinterpret_cast<const float2*>(D + b0);
            const float2 v1 = *reinterpret_cast<const float2*>(D + b1);
            d[0] = v0.x; d[1] = v0.y; d[2] = v1.x; d[3] = v1.y;
        }
        float rv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            tau += fmaxf(0.0f, d[t] - (cap - mm[t]));
            charge += d[t] + mm[t];
            rv[t] = (d[t] + mm[t]) * inv_ab;
        }
        float2* buf = sm + f * NP;
        buf[pidx(pp)] = make_float2(rv[0], rv[2]);
        buf[pidx(N - 1 - pp)] = make_float2(rv[1], rv[3]);
    }
    reduce2(tau, charge, acc, ACC_TAU, ACC_CHARGE, dr);
    __syncthreads();
    fft_block<LOGN, NB>(sm, tw, false);
    // split the packed spectra and apply the post-twiddle:
    // A_j[u] = Re(ph[u] V_j[u]), V_1 = (Z[u] + conj Z[N-u]) / 2,
    // V_2 = (Z[u] - conj Z[N-u]) / 2i.
    constexpr int HALF = N / 2 + 1;
    constexpr int ITEMS = NB * HALF;
    constexpr int PI = (ITEMS + T - 1) / T;
    float out[PI][4];
    int where[PI];
#pragma unroll
    for (int i = 0; i < PI; ++i) {
        int gi = threadIdx.x + i * T;
        where[i] = -1;
        if (gi < ITEMS) {
            int f = gi / HALF, u = gi % HALF;
            float2 zu = sm[f * NP + pidx(u)];
            float2 zn = sm[f * NP + pidx((N - u) & (N - 1))];
            float2 v1 = make_float2(0.5f * (zu.x + zn.x), 0.5f * (zu.y - zn.y));
            float2 v2 = make_float2(0.5f * (zu.y + zn.y), 0.5f * (zn.x - zu.x));
            float2 p = ph[u];
            out[i][0] = v1.x * p.x - v1.y * p.y;   // A1[u]
            out[i][1] = v2.x * p.x - v2.y * p.y;   // A2[u]
            // at N-u the spectra are conjugated
            float2 q = ph[N - u];
            out[i][2] = v1.x * q.x + v1.y * q.y;   // A1[N-u]
            out[i][3] = v2.x * q.x + v2.y * q.y;   // A2[N-u]
            where[i] = f * HALF + u;
        }
    }
    __syncthreads();
    float* sf = reinterpret_cast<float*>(sm);
#pragma unroll
    for (int i = 0; i < PI; ++i) {
        if (where[i] < 0) continue;
        int f = where[i] / HALF, u = where[i] % HALF;
        float* r1 = sf + (2 * f) * N;
        float* r2 = sf + (2 * f + 1) * N;
        r1[u & (N - 1)] = out[i][0];
        r2[u & (N - 1)] = out[i][1];
        if (u > 0 && u < N / 2) {
            r1[N - u] = out[i][2];
            r2[N - u] = out[i][3];
        }
    }
    __syncthreads();
    // transposed write: T1[u][y0 .. y0+7]
    if (tma && (smem_addr(sm) & 127u) == 0) {
        // the eight values of each u go through registers into the tile
        // [u][8] (which replaces the rows), stored in boxes of BOX values of u
        constexpr int CNT = (N + T - 1) / T;
        constexpr int BOX = N < 256 ? N : 256;
        float4 va[CNT], vb[CNT];
#pragma unroll
        for (int k = 0; k < CNT; ++k) {
            const int u = threadIdx.x + k * T;
            if (N % T == 0 || u < N) {
                va[k] = make_float4(sf[0 * N + u], sf[1 * N + u], sf[2 * N + u], sf[3 * N + u]);
                vb[k] = make_float4(sf[4 * N + u], sf[5 * N + u], sf[6 * N + u], sf[7 * N + u]);
            }
        }
        __syncthreads();
        float4* tile = reinterpret_cast<float4*>(sm);
#pragma unroll
        for (int k = 0; k < CNT; ++k) {
            const int u = threadIdx.x + k * T;
            if (N % T == 0 || u < N) {
                tile[2 * u] = va[k];
                tile[2 * u + 1] = vb[k];
            }
        }
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int b = 0; b < N / BOX; ++b) tma_store_2d(&mT1, tile + 2 * b * BOX, y0, b * BOX);
            tma_store_drain();
        }
        return;
    }
    for (int u = threadIdx.x; u < N; u += T) {
        float4 a = make_float4(sf[0 * N + u], sf[1 * N + u], sf[2 * N + u], sf[3 * N + u]);
        float4 b = make_float4(sf[4 * N + u], sf[5 * N + u], sf[6 * N + u], sf[7 * N + u]);
        float4* dst = reinterpret_cast<float4*>(T1 + (size_t)u * N + y0);
        dst[0] = a;
        dst[1] = b;
    }
}

// ------------------------------------------------- pass 2: columns
// CTA: 4 rows u of T1.  Forward DCT-II along y, spectral divide, energy,
// then the inverse sums along y: P (cosine sum of Psi) and R (sine sum of
// w_v Psi, via reversed coefficients).  Each complex IFFT carries the same
// quantity for two rows (P with P, R with R), so both parts share a scale.
template <int LOGN>
__global__ void __launch_bounds__(kSpecThreads, LOGN >= 12 ? 1 : 2)
k_cols(const float* __restrict__ T1, float* __restrict__ PT, float* __restrict__ RT,
       const float2* __restrict__ tw, const float2* __restrict__ ph, float pi_lx, float pi_ly,
       float eps, double* __restrict__ acc, DetRed dr, const __grid_constant__ CUtensorMap mPT,
       const __grid_constant__ CUtensorMap mRT, int tma) {
    constexpr int N = 1 << LOGN;
    constexpr int NB = kSpecBuffers;
    constexpr int ROWS = NB;
    constexpr int T = kSpecThreads;
    constexpr int NP = padded(N);
    extern __shared__ __align__(128) float2 sm[];
    const int u0 = blockIdx.x * ROWS;
    // buffer f packs rows 2f, 2f+1 in Makhoul's order (as in k_rows_fwd)
    constexpr int ITEMS_IN = (ROWS / 2) * (N / 2);
#pragma unroll 4
    for (int it = 0; it < (ITEMS_IN + T - 1) / T; ++it) {
        const int q = threadIdx.x + it * T;
        if (ITEMS_IN % T != 0 && q >= ITEMS_IN) break;
        const int f = q / (N / 2), pp = q % (N / 2);
        const size_t b0 = (size_t)(u0 + 2 * f) * N + 2 * pp;
        const float2 a = *reinterpret_cast<const float2*>(T1 + b0);
        const float2 c = *reinterpret_cast<const float2*>(T1 + b0 + N);
        float2* buf = sm + f * NP;
        buf[pidx(pp)] = make_float2(a.x, c.x);
        buf[pidx(N - 1 - pp)] = make_float2(a.y, c.y);
    }
    __syncthreads();
    fft_block<LOGN, NB / 2>(sm, tw, false);
    constexpr int HALF = N / 2 + 1;
    constexpr int ITEMS = (NB / 2) * HALF;
    constexpr int PI = (ITEMS + T - 1) / T;
    float2 zo[PI][4];   // [P at v, P at N-v, R at v, R at N-v], rows packed re/im
    int where[PI];
    const float invn2 = 1.0f / ((float)N * (float)N);
    dfloat energy = df_zero();
#pragma unroll
    for (int i = 0; i < PI; ++i) {
        int gi = threadIdx.x + i * T;
        where[i] = -1;
        if (gi < ITEMS) {
            int f = gi / HALF, v = gi % HALF;
            int vn = (N - v) & (N - 1);
            float2 zu = sm[f * NP + pidx(v)];
            float2 zn = sm[f * NP + pidx(vn)];
            float2 v1 = make_float2(0.5f * (zu.x + zn.x), 0.5f * (zu.y - zn.y));
            float2 v2 = make_float2(0.5f * (zu.y + zn.y), 0.5f * (zn.x - zu.x));
            float2 p = ph[v], q = ph[N - v];
            // B[row][v], B[row][N-v] (unnormalised DCT-II along y)
            float B[2][2];
            B[0][0] = v1.x * p.x - v1.y * p.y;
            B[1][0] = v2.x * p.x - v2.y * p.y;
            B[0][1] = v1.x * q.x + v1.y * q.y;
            B[1][1] = v2.x * q.x + v2.y * q.y;
            float wv = pi_ly * (float)v, wvn = pi_ly * (float)(N - v);
            float ev = (v == 0) ? 1.0f : 2.0f;
            bool has_n = (v > 0 && v < N / 2);
            // halved inverse coefficients per row: c1 (P) and c2 (R) at v and N-v
            float c1v[2], c1n[2], c2v[2], c2n[2];
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                int u = u0 + 2 * f + rr;
                float wu = pi_lx * (float)u;
                float eu = (u == 0) ? 1.0f : 2.0f;
                float a0 = eu * ev * invn2 * B[rr][0];
                // Poisson: (0,0) mode dropped; Helmholtz (eps > 0): divisor
                // w^2 + eps and the (0,0) mode kept
                // the divisor is at least (pi/L)^2 > 0 (or eps): the fast
                // divide (2 ulp) stays far inside the transform's bound
                float psi0 = (u == 0 && v == 0 && !(eps > 0.0f))
                                 ? 0.0f
                                 : __fdividef(a0, wu * wu + wv * wv + eps);
                float psin = 0.0f;
                if (has_n) {
                    float an = eu * 2.0f * invn2 * B[rr][1];
                    psin = __fdividef(an, wu * wu + wvn * wvn + eps);
                    energy = df_add(energy, B[rr][1] * psin);
                }
                energy = df_add(energy, B[rr][0] * psi0);
                // P: cosine sum of Psi.  R: cosine sum of c2[v'] = s[N-v'],
                // s[v] = w_v Psi[v], c2[0] = 0; then R = (-1)^y * that.
                c1v[rr] = (v == 0) ? psi0 : 0.5f * psi0;
                c1n[rr] = 0.5f * psin;
                c2v[rr] = (v == 0) ? 0.0f : 0.5f * wvn * psin;
                c2n[rr] = (v == 0) ? 0.0f : 0.5f * wv * psi0;
                if (v == N / 2) {
                    c1n[rr] = c1v[rr];
                    c2v[rr] = 0.5f * wv * psi0;
                    c2n[rr] = c2v[rr];
                }
            }
            zo[i][0] = pack_inv(c1v[0], c1n[0], c1v[1], c1n[1], p);
            zo[i][1] = pack_inv(c1n[0], c1v[0], c1n[1], c1v[1], q);
            zo[i][2] = pack_inv(c2v[0], c2n[0], c2v[1], c2n[1], p);
            zo[i][3] = pack_inv(c2n[0], c2v[0], c2n[1], c2v[1], q);
            where[i] = f * HALF + v;
        }
    }
    reduce2(df_val(energy), 0.0f, acc, ACC_N, -1, dr);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PI; ++i) {
        if (where[i] < 0) continue;
        int f = where[i] / HALF, v = where[i] % HALF;
        float2* rowP = sm + (2 * f) * NP;
        float2* rowR = sm + (2 * f + 1) * NP;
        rowP[pidx(v & (N - 1))] = zo[i][0];
        rowR[pidx(v & (N - 1))] = zo[i][2];
        if (v > 0 && v < N / 2) {
            rowP[pidx(N - v)] = zo[i][1];
            rowR[pidx(N - v)] = zo[i][3];
        }
    }
    __syncthreads();
    fft_block<LOGN, NB>(sm, tw, true);
    // unshuffle: y even <- k = y/2, y odd <- k = N-1-(y-1)/2
    if (tma && (smem_addr(sm) & 127u) == 0) {
        // through registers into the tiles PT[y][u0..u0+3] and RT[y][...]
        // (16 bytes per y, in place of the buffers), stored in boxes of BOX y
        constexpr int CNT = (N + T - 1) / T;
        constexpr int BOX = N < 256 ? N : 256;
        float4 pv[CNT], rv[CNT];
#pragma unroll
        for (int k = 0; k < CNT; ++k) {
            const int y = threadIdx.x + k * T;
            if (N % T == 0 || y < N) {
                const int q = pidx(mk_src(y, N));
                const float sgn = (y & 1) ? -1.0f : 1.0f;
                const float2 p0 = sm[0 * NP + q], r0 = sm[1 * NP + q];
                const float2 p1 = sm[2 * NP + q], r1 = sm[3 * NP + q];
                pv[k] = make_float4(p0.x, p0.y, p1.x, p1.y);
                rv[k] = make_float4(sgn * r0.x, sgn * r0.y, sgn * r1.x, sgn * r1.y);
            }
        }
        __syncthreads();
        float4* tP = reinterpret_cast<float4*>(sm);
        float4* tR = tP + N;
#pragma unroll
        for (int k = 0; k < CNT; ++k) {
            const int y = threadIdx.x + k * T;
            if (N % T == 0 || y < N) {
                tP[y] = pv[k];
                tR[y] = rv[k];
            }
        }
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int b = 0; b < N / BOX; ++b) {
                tma_store_2d(&mPT, tP + b * BOX, u0, b * BOX);
                tma_store_2d(&mRT, tR + b * BOX, u0, b * BOX);
            }
            tma_store_drain();
        }
        return;
    }
    for (int y = threadIdx.x; y < N; y += T) {
        int k = pidx(mk_src(y, N));
        float sgn = (y & 1) ? -1.0f : 1.0f;
        float2 p0 = sm[0 * NP + k], r0 = sm[1 * NP + k], p1 = sm[2 * NP + k], r1 = sm[3 * NP + k];
        *reinterpret_cast<float4*>(PT + (size_t)y * N + u0) = make_float4(p0.x, p0.y, p1.x, p1.y);
        *reinterpret_cast<float4*>(RT + (size_t)y * N + u0) =
            make_float4(sgn * r0.x, sgn * r0.y, sgn * r1.x, sgn * r1.y);
    }
}

// ------------------------------------------------- pass 3: inverse rows
// CTA: 4 rows y, one round of four inverse FFTs: buffers 0 and 1 hold E_x
// (the sine sum of w_u P, via reversed coefficients: c[u'] = s[N-u'],
// u' >= 1, c[0] = 0, s[u] = w_u P[u]; E_x[x] = (-1)^x cosine-sum(c)[x]) for
// rows (0, 1) and (2, 3); buffers 2 and 3 hold E_y (the cosine sum of R).
// Written as the interleaved field map E2[y][x] = (E_x, E_y).  The potential
// psi (the cosine sum of P) is not needed by the evaluation (the energy comes
// from the column pass by Parseval) and is formed on demand by k_rows_psi.
template <int LOGN>
__global__ void __launch_bounds__(kSpecThreads, LOGN >= 12 ? 1 : 2)
k_rows_inv(const float* __restrict__ PT, const float* __restrict__ RT, float2* __restrict__ E2,
           const float2* __restrict__ tw, const float2* __restrict__ ph, float pi_lx) {
    constexpr int N = 1 << LOGN;
    constexpr int NB = kSpecBuffers;
    constexpr int ROWS = NB;
    constexpr int T = kSpecThreads;
    constexpr int HALF = N / 2 + 1;
    constexpr int NP = padded(N);
    extern __shared__ __align__(128) float2 sm[];
    const int y0 = blockIdx.x * ROWS;
#pragma unroll 2
    for (int idx = threadIdx.x; idx < (ROWS / 2) * HALF; idx += T) {
        int f = idx / HALF, u = idx % HALF;
        int un = (N - u) & (N - 1);
        // E_y: cosine sums of the R rows (2f, 2f+1)
        {
            const float* A = RT + (size_t)(y0 + 2 * f) * N;
            const float* Bq = A + N;
            float au = A[u & (N - 1)], bu = Bq[u & (N - 1)];
            float an = (u > 0) ? A[un] : 0.0f, bn = (u > 0) ? Bq[un] : 0.0f;
            float cau = (u == 0) ? au : 0.5f * au, cbu = (u == 0) ? bu : 0.5f * bu;
            float can = 0.5f * an, cbn = 0.5f * bn;
            if (u == N / 2) { can = cau; cbn = cbu; }
            float2* row = sm + (2 + f) * NP;
            row[pidx(u & (N - 1))] = pack_inv(cau, can, cbu, cbn, ph[u]);
            if (u > 0 && u < N / 2) row[pidx(N - u)] = pack_inv(can, cau, cbn, cbu, ph[N - u]);
        }
        // E_x: reversed sine coefficients of the P rows (2f, 2f+1)
        {
            const float* Pa = PT + (size_t)(y0 + 2 * f) * N;
            const float* Pb = Pa + N;
            float wu = pi_lx * (float)u, wn = pi_lx * (float)(N - u);
            // c[u] = s[N-u] = w_{N-u} P[N-u]  (u >= 1);  c[N-u] = s[u] = w_u P[u]
            float ca_u = (u == 0) ? 0.0f : 0.5f * wn * Pa[N - u];
            float cb_u = (u == 0) ? 0.0f : 0.5f * wn * Pb[N - u];
            float ca_n = (u == 0) ? 0.0f : 0.5f * wu * Pa[u];
            float cb_n = (u == 0) ? 0.0f : 0.5f * wu * Pb[u];
            if (u == N / 2) { ca_n = ca_u; cb_n = cb_u; }
            float2* row = sm + f * NP;
            row[pidx(u & (N - 1))] = pack_inv(ca_u, ca_n, cb_u, cb_n, ph[u]);
            if (u > 0 && u < N / 2) row[pidx(N - u)] = pack_inv(ca_n, ca_u, cb_n, cb_u, ph[N - u]);
        }
    }
    __syncthreads();
    fft_block<LOGN, NB>(sm, tw, true);
    for (int idx = threadIdx.x; idx < ROWS * N; idx += T) {
        int r = idx >> LOGN, x = idx & (N - 1);
        int k = pidx(mk_src(x, N));
        float2 zx = sm[(r >> 1) * NP + k], zy = sm[(2 + (r >> 1)) * NP + k];
        float vx = (r & 1) ? zx.y : zx.x, vy = (r & 1) ? zy.y : zy.x;
        E2[(size_t)(y0 + r) * N + x] = make_float2((x & 1) ? -vx : vx, vy);
    }
}

// psi on demand: CTA of 4 rows y, the cosine sums of the P rows (2f, 2f+1)
// in buffer f.
template <int LOGN>
__global__ void __launch_bounds__(kSpecThreads, LOGN >= 12 ? 1 : 2)
k_rows_psi(const float* __restrict__ PT, float* __restrict__ psi, const float2* __restrict__ tw,
           const float2* __restrict__ ph) {
    constexpr int N = 1 << LOGN;
    constexpr int ROWS = kSpecBuffers;
    constexpr int NB = ROWS / 2;
    constexpr int T = kSpecThreads;
    constexpr int HALF = N / 2 + 1;
    constexpr int NP = padded(N);
    extern __shared__ __align__(128) float2 sm[];
    const int y0 = blockIdx.x * ROWS;
    for (int idx = threadIdx.x; idx < NB * HALF; idx += T) {
        int f = idx / HALF, u = idx % HALF;
        int un = (N - u) & (N - 1);
        const float* A = PT + (size_t)(y0 + 2 * f) * N;
        const float* Bq = A + N;
        float au = A[u & (N - 1)], bu = Bq[u & (N - 1)];
        float an = (u > 0) ? A[un] : 0.0f, bn = (u > 0) ? Bq[un] : 0.0f;
        float cau = (u == 0) ? au : 0.5f * au, cbu = (u == 0) ? bu : 0.5f * bu;
        float can = 0.5f * an, cbn = 0.5f * bn;
        if (u == N / 2) { can = cau; cbn = cbu; }
        float2* row = sm + f * NP;
        row[pidx(u & (N - 1))] = pack_inv(cau, can, cbu, cbn, ph[u]);
        if (u > 0 && u < N / 2) row[pidx(N - u)] = pack_inv(can, cau, cbn, cbu, ph[N - u]);
    }
    __syncthreads();
    fft_block<LOGN, NB>(sm, tw, true);
    for (int idx = threadIdx.x; idx < ROWS * N; idx += T) {
        int r = idx >> LOGN, x = idx & (N - 1);
        float2 z = sm[(r >> 1) * NP + pidx(mk_src(x, N))];
        psi[(size_t)(y0 + r) * N + x] = (r & 1) ? z.y : z.x;
    }
}

// ------------------------------------- tensor-core radix path: the rows
// The solve path FFTPL_SOLVE_TC_RADIX (k_tc.cu) computes every complex DFT
// of length n as two small dense products on the tensor cores.  These
// kernels do the same pre- and post-processing as the three passes above,
// row by row in global memory: Z holds complex rows of length n (Makhoul's
// packing of two real rows, or the packed spectrum of an inverse pair) that
// go into the DFT, V the complex rows that come out.

// rho rows (2r, 2r+1) packed: Z[r][k] = rho_2r[2k] + i rho_2r+1[2k] (k < n/2),
// Z[r][n-1-k] = rho_2r[2k+1] + i rho_2r+1[2k+1]; with the overflow and charge
// sums of k_rows_fwd.
template <bool QUANT>
__global__ void __launch_bounds__(256)
k_tcr_pack_rho(int n, int rows2, const float* __restrict__ D, const long long* __restrict__ Dq,
               const float* __restrict__ M, float inv_ab, float cap, float2* __restrict__ Z,
               double* __restrict__ acc, DetRed dr) {
    const int half = n >> 1;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float tau = 0.0f, charge = 0.0f;
    if (q < (long long)rows2 * half) {
        const int r = (int)(q / half), k = (int)(q % half);
        const size_t b0 = (size_t)(2 * r) * n + 2 * k, b1 = b0 + n;
        float d[4], mm[4];
        const float2 m0 = *reinterpret_cast<const float2*>(M + b0);
        const float2 m1 = *reinterpret_cast<const float2*>(M + b1);
        mm[0] = m0.x; mm[1] = m0.y; mm[2] = m1.x; mm[3] = m1.y;
        if (QUANT) {
            const longlong2 q0 = *reinterpret_cast<const longlong2*>(Dq + b0);
            const longlong2 q1 = *reinterpret_cast<const longlong2*>(Dq + b1);
            d[0] = (float)q0.x * 2.3283064365386963e-10f;
            d[1] = (float)q0.y * 2.3283064365386963e-10f;
            d[2] = (float)q1.x * 2.3283064365386963e-10f;
            d[3] = (float)q1.y * 2.3283064365386963e-10f;
        } else {
            const float2 v0 = *reinterpret_cast<const float2*>(D + b0);
            const float2 v1 = *reinterpret_cast<const float2*>(D + b1);
            d[0] = v0.x; d[1] = v0.y; d[2] = v1.x; d[3] = v1.y;
        }
        float rv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            tau += fmaxf(0.0f, d[t] - (cap - mm[t]));
            charge += d[t] + mm[t];
            rv[t] = (d[t] + mm[t]) * inv_ab;
        }
        float2* zr = Z + (size_t)r * n;
        zr[k] = make_float2(rv[0], rv[2]);
        zr[n - 1 - k] = make_float2(rv[1], rv[3]);
    }
    reduce2(tau, charge, acc, ACC_TAU, ACC_CHARGE, dr);
}

// Rows (2r, 2r+1) of a real map packed the same way (no sums).
__global__ void __launch_bounds__(256)
k_tcr_pack_rows(int n, int rows2, const float* __restrict__ A, float2* __restrict__ Z) {
    const int half = n >> 1;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)rows2 * half) return;
    const int r = (int)(q / half), k = (int)(q % half);
    const size_t b0 = (size_t)(2 * r) * n + 2 * k;
    const float2 a = *reinterpret_cast<const float2*>(A + b0);
    const float2 c = *reinterpret_cast<const float2*>(A + b0 + n);
    float2* zr = Z + (size_t)r * n;
    zr[k] = make_float2(a.x, c.x);
    zr[n - 1 - k] = make_float2(a.y, c.y);
}

// DCT-II spectra of packed pairs: A_j[u] = Re(ph[u] V_j[u]) with
// V_1 = (Z[u] + conj Z[n-u]) / 2, V_2 = (Z[u] - conj Z[n-u]) / 2i, the two
// rows of pair r; written transposed, T[u][8 g .. 8 g + 7] for the 4 pairs
// of group g (as k_rows_fwd writes T1).
__global__ void __launch_bounds__(256)
k_tcr_post_fwd(int n, int groups, const float2* __restrict__ V, const float2* __restrict__ ph,
               float* __restrict__ T) {
    const int half = n / 2 + 1;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)groups * half) return;
    const int g = (int)(q / half), u = (int)(q % half);
    float a[8], an[8];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float2* vr = V + (size_t)(4 * g + t) * n;
        const float2 zu = vr[u & (n - 1)], zn = vr[(n - u) & (n - 1)];
        const float2 v1 = make_float2(0.5f * (zu.x + zn.x), 0.5f * (zu.y - zn.y));
        const float2 v2 = make_float2(0.5f * (zu.y + zn.y), 0.5f * (zn.x - zu.x));
        const float2 p = ph[u], pn = ph[n - u];
        a[2 * t] = v1.x * p.x - v1.y * p.y;
        a[2 * t + 1] = v2.x * p.x - v2.y * p.y;
        an[2 * t] = v1.x * pn.x + v1.y * pn.y;
        an[2 * t + 1] = v2.x * pn.x + v2.y * pn.y;
    }
    float4* dst = reinterpret_cast<float4*>(T + (size_t)(u & (n - 1)) * n + 8 * g);
    dst[0] = make_float4(a[0], a[1], a[2], a[3]);
    dst[1] = make_float4(a[4], a[5], a[6], a[7]);
    if (u > 0 && u < n / 2) {
        float4* dn = reinterpret_cast<float4*>(T + (size_t)(n - u) * n + 8 * g);
        dn[0] = make_float4(an[0], an[1], an[2], an[3]);
        dn[1] = make_float4(an[4], an[5], an[6], an[7]);
    }
}

// Column spectra of u-row pairs r (V, as in k_cols): divide by
// w_u^2 + w_v^2 (+ eps), drop the (0,0) mode, the energy, and the packed
// inverse inputs: Z[r] for P (cosine sums of Psi), Z[rows2 + r] for R
// (cosine sums of the reversed w_v Psi).
__global__ void __launch_bounds__(256)
k_tcr_spectral(int n, int rows2, const float2* __restrict__ V, const float2* __restrict__ ph,
               float pi_lx, float pi_ly, float eps, float2* __restrict__ Z,
               double* __restrict__ acc, DetRed dr) {
    const int half = n / 2 + 1;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    dfloat energy = df_zero();
    if (q < (long long)rows2 * half) {
        const int r = (int)(q / half), v = (int)(q % half);
        const float2* vr = V + (size_t)r * n;
        const float2 zu = vr[v & (n - 1)], zn = vr[(n - v) & (n - 1)];
        const float2 v1 = make_float2(0.5f * (zu.x + zn.x), 0.5f * (zu.y - zn.y));
        const float2 v2 = make_float2(0.5f * (zu.y + zn.y), 0.5f * (zn.x - zu.x));
        const float2 p = ph[v], qq = ph[n - v];
        float B[2][2];
        B[0][0] = v1.x * p.x - v1.y * p.y;
        B[1][0] = v2.x * p.x - v2.y * p.y;
        B[0][1] = v1.x * qq.x + v1.y * qq.y;
        B[1][1] = v2.x * qq.x + v2.y * qq.y;
        const float invn2 = 1.0f / ((float)n * (float)n);
        const float wv = pi_ly * (float)v, wvn = pi_ly * (float)(n - v);
        const float ev = (v == 0) ? 1.0f : 2.0f;
        const bool has_n = (v > 0 && v < n / 2);
        float c1v[2], c1n[2], c2v[2], c2n[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int u = 2 * r + rr;
            const float wu = pi_lx * (float)u;
            const float eu = (u == 0) ? 1.0f : 2.0f;
            const float a0 = eu * ev * invn2 * B[rr][0];
            const float psi0 = (u == 0 && v == 0 && !(eps > 0.0f))
                                   ? 0.0f
                                   : __fdividef(a0, wu * wu + wv * wv + eps);
            float psin = 0.0f;
            if (has_n) {
                const float an = eu * 2.0f * invn2 * B[rr][1];
                psin = __fdividef(an, wu * wu + wvn * wvn + eps);
                energy = df_add(energy, B[rr][1] * psin);
            }
            energy = df_add(energy, B[rr][0] * psi0);
            c1v[rr] = (v == 0) ? psi0 : 0.5f * psi0;
            c1n[rr] = 0.5f * psin;
            c2v[rr] = (v == 0) ? 0.0f : 0.5f * wvn * psin;
            c2n[rr] = (v == 0) ? 0.0f : 0.5f * wv * psi0;
            if (v == n / 2) {
                c1n[rr] = c1v[rr];
                c2v[rr] = 0.5f * wv * psi0;
                c2n[rr] = c2v[rr];
            }
        }
        float2* zp = Z + (size_t)r * n;
        float2* zr = Z + (size_t)(rows2 + r) * n;
        zp[v & (n - 1)] = pack_inv(c1v[0], c1n[0], c1v[1], c1n[1], p);
        zr[v & (n - 1)] = pack_inv(c2v[0], c2n[0], c2v[1], c2n[1], p);
        if (has_n) {
            zp[n - v] = pack_inv(c1n[0], c1v[0], c1n[1], c1v[1], qq);
            zr[n - v] = pack_inv(c2n[0], c2v[0], c2n[1], c2v[1], qq);
        }
    }
    reduce2(df_val(energy), 0.0f, acc, ACC_N, -1, dr);
}

// Inverse outputs of the column pass: pair r of P (V[r]) and of R
// (V[rows2 + r]) unshuffled (y <- position mk_src(y); R times (-1)^y) and
// written transposed, PT[y][8 g .. 8 g + 7], RT likewise.
__global__ void __launch_bounds__(256)
k_tcr_post_cols(int n, int rows2, const float2* __restrict__ V, float* __restrict__ PT,
                float* __restrict__ RT) {
    const int groups = rows2 / 4;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)groups * n) return;
    const int g = (int)(q / n), y = (int)(q % n);
    const int k = mk_src(y, n);
    const float sgn = (y & 1) ? -1.0f : 1.0f;
    float p[8], rr[8];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float2 zp = V[(size_t)(4 * g + t) * n + k];
        const float2 zr = V[(size_t)(rows2 + 4 * g + t) * n + k];
        p[2 * t] = zp.x; p[2 * t + 1] = zp.y;
        rr[2 * t] = sgn * zr.x; rr[2 * t + 1] = sgn * zr.y;
    }
    float4* dp = reinterpret_cast<float4*>(PT + (size_t)y * n + 8 * g);
    float4* dr4 = reinterpret_cast<float4*>(RT + (size_t)y * n + 8 * g);
    dp[0] = make_float4(p[0], p[1], p[2], p[3]);
    dp[1] = make_float4(p[4], p[5], p[6], p[7]);
    dr4[0] = make_float4(rr[0], rr[1], rr[2], rr[3]);
    dr4[1] = make_float4(rr[4], rr[5], rr[6], rr[7]);
}

// Inverse inputs of the row pass for y-row pairs r: Z[r] E_x (reversed sine
// coefficients of w_u P), Z[rows2 + r] E_y (cosine sums of R), as the fill
// of k_rows_inv.
__global__ void __launch_bounds__(256)
k_tcr_pack_inv(int n, int rows2, const float* __restrict__ PT, const float* __restrict__ RT,
               const float2* __restrict__ ph, float pi_lx, float2* __restrict__ Z) {
    const int half = n / 2 + 1;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)rows2 * half) return;
    const int r = (int)(q / half), u = (int)(q % half);
    const int un = (n - u) & (n - 1);
    {
        const float* A = RT + (size_t)(2 * r) * n;
        const float* Bq = A + n;
        const float au = A[u & (n - 1)], bu = Bq[u & (n - 1)];
        const float an = (u > 0) ? A[un] : 0.0f, bn = (u > 0) ? Bq[un] : 0.0f;
        const float cau = (u == 0) ? au : 0.5f * au, cbu = (u == 0) ? bu : 0.5f * bu;
        float can = 0.5f * an, cbn = 0.5f * bn;
        if (u == n / 2) { can = cau; cbn = cbu; }
        float2* row = Z + (size_t)(rows2 + r) * n;
        row[u & (n - 1)] = pack_inv(cau, can, cbu, cbn, ph[u]);
        if (u > 0 && u < n / 2) row[n - u] = pack_inv(can, cau, cbn, cbu, ph[n - u]);
    }
    {
        const float* Pa = PT + (size_t)(2 * r) * n;
        const float* Pb = Pa + n;
        const float wu = pi_lx * (float)u, wn = pi_lx * (float)(n - u);
        const float ca_u = (u == 0) ? 0.0f : 0.5f * wn * Pa[n - u];
        const float cb_u = (u == 0) ? 0.0f : 0.5f * wn * Pb[n - u];
        float ca_n = (u == 0) ? 0.0f : 0.5f * wu * Pa[u];
        float cb_n = (u == 0) ? 0.0f : 0.5f * wu * Pb[u];
        if (u == n / 2) { ca_n = ca_u; cb_n = cb_u; }
        float2* row = Z + (size_t)r * n;
        row[u & (n - 1)] = pack_inv(ca_u, ca_n, cb_u, cb_n, ph[u]);
        if (u > 0 && u < n / 2) row[n - u] = pack_inv(ca_n, ca_u, cb_n, cb_u, ph[n - u]);
    }
}

// Inverse outputs of the row pass: E2[y][x] = ((-1)^x E_x, E_y) for the rows
// of pair r, unshuffled.
__global__ void __launch_bounds__(256)
k_tcr_post_rows(int n, int rows2, const float2* __restrict__ V, float2* __restrict__ E2) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)rows2 * n) return;
    const int r = (int)(q / n), x = (int)(q % n);
    const int k = mk_src(x, n);
    const float2 zx = V[(size_t)r * n + k], zy = V[(size_t)(rows2 + r) * n + k];
    const float s = (x & 1) ? -1.0f : 1.0f;
    E2[(size_t)(2 * r) * n + x] = make_float2(s * zx.x, zy.x);
    E2[(size_t)(2 * r + 1) * n + x] = make_float2(s * zx.y, zy.y);
}

static inline unsigned tcr_blocks(long long items) { return (unsigned)((items + 255) / 256); }

cudaError_t launch_tcr_stage(Ctx& c, int which, const float2* V, float2* Z, cudaStream_t s) {
    const int n = c.n, rows2 = n / 2;
    const float pi_lx = (float)(M_PI / c.Lx), pi_ly = (float)(M_PI / c.Ly);
    switch (which) {
        case 0: {   // rho rows -> Z (with the overflow and charge sums)
            const float inv_ab = (float)(1.0 / c.Ab);
            const float cap = (float)(c.opt.target_density * c.Ab);
            const unsigned nb = tcr_blocks((long long)rows2 * (n / 2));
            if (c.opt.deterministic)
                k_tcr_pack_rho<true><<<nb, 256, 0, s>>>(n, rows2, nullptr, c.Dq, c.M, inv_ab, cap,
                                                        Z, c.acc, det_red(c, 0));
            else
                k_tcr_pack_rho<false><<<nb, 256, 0, s>>>(n, rows2, c.D, nullptr, c.M, inv_ab, cap,
                                                         Z, c.acc, det_red(c, 0));
            break;
        }
        case 1:     // row spectra -> T1 (transposed)
            k_tcr_post_fwd<<<tcr_blocks((long long)(rows2 / 4) * (n / 2 + 1)), 256, 0, s>>>(
                n, rows2 / 4, V, c.ph, c.T1);
            break;
        case 2:     // T1 rows -> Z
            k_tcr_pack_rows<<<tcr_blocks((long long)rows2 * (n / 2)), 256, 0, s>>>(n, rows2, c.T1, Z);
            break;
        case 3:     // column spectra -> divide, energy -> Z (P rows, then R rows)
            k_tcr_spectral<<<tcr_blocks((long long)rows2 * (n / 2 + 1)), 256, 0, s>>>(
                n, rows2, V, c.ph, pi_lx, pi_ly, (float)c.opt.helmholtz_eps, Z, c.acc,
                det_red(c, 0));
            break;
        case 4:     // P, R sums -> PT, RT (transposed)
            k_tcr_post_cols<<<tcr_blocks((long long)(rows2 / 4) * n), 256, 0, s>>>(n, rows2, V,
                                                                                  c.PT, c.RT);
            break;
        case 5:     // PT, RT rows -> Z (E_x rows, then E_y rows)
            k_tcr_pack_inv<<<tcr_blocks((long long)rows2 * (n / 2 + 1)), 256, 0, s>>>(
                n, rows2, c.PT, c.RT, c.ph, pi_lx, Z);
            break;
        default:    // E_x, E_y sums -> E2
            k_tcr_post_rows<<<tcr_blocks((long long)rows2 * n), 256, 0, s>>>(n, rows2, V, c.E2);
            break;
    }
    c.launches++;
    return cudaGetLastError();
}

// ------------------------------------------------------------ launch
template <int LOGN>
static cudaError_t launch_all_logn(Ctx& c, int which, cudaStream_t s) {
    constexpr int N = 1 << LOGN;
    size_t smem = (size_t)kSpecBuffers * padded(N) * sizeof(float2);
    float inv_ab = (float)(1.0 / c.Ab);
    float cap = (float)(c.opt.target_density * c.Ab);
    float pi_lx = (float)(M_PI / c.Lx), pi_ly = (float)(M_PI / c.Ly);
    cudaError_t e = cudaSuccess;
    if (which == 0) {
        if (c.opt.deterministic) {
            auto kf = k_rows_fwd<LOGN, true>;
            kf<<<N / (2 * kSpecBuffers), kSpecThreads, smem, s>>>(nullptr, c.Dq, c.M, inv_ab, cap,
                                                                   c.T1, c.tw, c.ph, c.acc,
                                                                   det_red(c, 0), c.map_t1,
                                                                   c.spec_tma ? 1 : 0);
        } else {
            auto kf = k_rows_fwd<LOGN, false>;
            kf<<<N / (2 * kSpecBuffers), kSpecThreads, smem, s>>>(c.D, nullptr, c.M, inv_ab, cap,
                                                                   c.T1, c.tw, c.ph, c.acc,
                                                                   det_red(c, 0), c.map_t1,
                                                                   c.spec_tma ? 1 : 0);
        }
    } else if (which == 1) {
        auto kf = k_cols<LOGN>;
        kf<<<N / kSpecBuffers, kSpecThreads, smem, s>>>(c.T1, c.PT, c.RT, c.tw, c.ph, pi_lx, pi_ly,
                                                        (float)c.opt.helmholtz_eps, c.acc,
                                                        det_red(c, 0), c.map_pt, c.map_rt,
                                                        c.spec_tma ? 1 : 0);
    } else if (which == 2) {
        auto kf = k_rows_inv<LOGN>;
        kf<<<N / kSpecBuffers, kSpecThreads, smem, s>>>(c.PT, c.RT, c.E2, c.tw, c.ph, pi_lx);
    } else {
        auto kf = k_rows_psi<LOGN>;
        kf<<<N / kSpecBuffers, kSpecThreads, smem / 2, s>>>(c.PT, c.psi, c.tw, c.ph);
    }
    c.launches++;
    e = cudaGetLastError();
    return e;
}

// Shared-memory opt-in for every kernel of one transform size (done at create,
// outside any stream capture).
template <int LOGN>
static void prepare_logn() {
    int smem = (int)((size_t)kSpecBuffers * padded(1 << LOGN) * sizeof(float2));
    cudaFuncSetAttribute(k_rows_fwd<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_rows_fwd<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_cols<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_rows_inv<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_rows_psi<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem / 2);
}

void prepare_spectral(int logn) {
    switch (logn) {
        case 4: prepare_logn<4>(); break;
        case 5: prepare_logn<5>(); break;
        case 6: prepare_logn<6>(); break;
        case 7: prepare_logn<7>(); break;
        case 8: prepare_logn<8>(); break;
        case 9: prepare_logn<9>(); break;
        case 10: prepare_logn<10>(); break;
        case 11: prepare_logn<11>(); break;
        case 12: prepare_logn<12>(); break;
        default: break;
    }
}

static cudaError_t dispatch(Ctx& c, int which, cudaStream_t s) {
    switch (c.logn) {
        case 4: return launch_all_logn<4>(c, which, s);
        case 5: return launch_all_logn<5>(c, which, s);
        case 6: return launch_all_logn<6>(c, which, s);
        case 7: return launch_all_logn<7>(c, which, s);
        case 8: return launch_all_logn<8>(c, which, s);
        case 9: return launch_all_logn<9>(c, which, s);
        case 10: return launch_all_logn<10>(c, which, s);
        case 11: return launch_all_logn<11>(c, which, s);
        case 12: return launch_all_logn<12>(c, which, s);
        default: return cudaErrorInvalidValue;
    }
}

void spec_maps_init(Ctx& c) {
    const int n = c.n, box = n < 256 ? n : 256;
    c.spec_maps_ok = c.T1 && c.PT && c.RT && n >= 16 &&
                     make_map_f32(&c.map_t1, c.T1, n, n, 8, box) &&
                     make_map_f32(&c.map_pt, c.PT, n, n, 4, box) &&
                     make_map_f32(&c.map_rt, c.RT, n, n, 4, box);
    c.spec_tma = c.spec_maps_ok;
}

cudaError_t launch_rows_fwd(Ctx& c, cudaStream_t s) { return dispatch(c, 0, s); }
cudaError_t launch_cols_spectral(Ctx& c, cudaStream_t s) { return dispatch(c, 1, s); }
cudaError_t launch_rows_inv(Ctx& c, cudaStream_t s) { return dispatch(c, 2, s); }
cudaError_t launch_rows_psi(Ctx& c, cudaStream_t s) { return dispatch(c, 3, s); }

}  // namespace fftpl
