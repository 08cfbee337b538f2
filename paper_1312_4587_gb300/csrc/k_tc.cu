// Spectral solve as dense cosine/sine-matrix contractions on the tcgen05
// tensor cores (solve path FFTPL_SOLVE_TC_BF16X3).
//
// With C[u][x] = cos(pi u (2x+1) / 2n), Ct = C^T, Sx[x][u] = w_u sin(...),
// Sy[y][v] = w_v sin(...), every product below is D[M][N] = sum_k A[M][k] B[N][k]
// (both operands K-major, row-major in memory):
//   G1   A1t[u][y]  = sum_x C[u][x]   rho[y][x]
//   G2   B[v][u]    = sum_y C[v][y]   A1t[u][y]  -> Psi = a / (w_u^2+w_v^2), a = eps eps B / n^2
//   G35  [Ut;Xt][x][v] = sum_u [Ct;Sx][x][u] Psi[v][u]
//   G46  [psi|E_x][y][x] = sum_v Ct[y][v] [Ut;Xt][x][v]
//   G7   E_y[y][x]  = sum_v Sy[y][v]  Ut[x][v]
// (Eqs. 10-12 at the bin centres; the energy N = 1/2 A_b sum B Psi is
// reduced in the G2 epilogue.)  Operands are float32 values split into two
// bf16 halves, x = hi + lo; each product accumulates hi*hi + hi*lo + lo*hi in
// float32 in tensor memory (the lo*lo term, 2^-16 relative, is dropped), in
// four chains over consecutive quarters of K summed in the epilogue.
//
// Kernel: one CTA per 128 x 128 output tile, 4 warps.  Warp 0 (one thread)
// loads 128 x 64 operand tiles with TMA (128-byte swizzle) into a 3-stage
// ring; warp 1 (one thread) issues tcgen05.mma (M = N = 128, K = 16) and
// commits each stage back to the producer; all four warps read the
// accumulator with tcgen05.ld (warp w owns lanes 32w..32w+31) for the
// epilogue.  Every mbarrier wait is bounded in time: on expiry the kernel
// records ERR_TIMEOUT in the handle's error word, skips its stores, waits
// (bounded) for its own operations and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "fftpl_internal.cuh"

namespace fftpl {
namespace tc {

// k-step of 64 bf16 (one 128-byte swizzle row), a 3-stage ring of 192 KiB,
// one CTA per SM.  (BK = 32 runs two 96 KiB CTAs per SM with the 64-byte
// swizzle: measured no faster at 2048^3 and slower at 4096^3.)
constexpr int BM = 128, BN = 128, BK = 64;
constexpr int kSwz = BK * 2;                   // swizzle span in bytes (64 or 128)
constexpr int kMinBlocks = BK == 32 ? 2 : 1;   // CTAs per SM the launch bounds ask for
constexpr int kStages = 3;
constexpr int kTileBytes = BM * BK * 2;        // bf16 tile of one operand half
constexpr int kStageBytes = 4 * kTileBytes;    // A hi, A lo, B hi, B lo
constexpr int kThreads = 128;
constexpr int kSmemBytes = kStages * kStageBytes + 1024;
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s per wait
// Accumulators per tile: the k-tiles are cut into kAcc consecutive chunks,
// each accumulated in its own 128-column region of tensor memory and the
// chunks summed in float32 in the epilogue.  The error of the tensor cores'
// float32 accumulation grows with the chain length: one chain over K = 4096
// left psi 3.7e-4 (relative L2) from the transform path at n = 4096, four
// chains of K/4 stay within 2e-4.  kAcc * BN = 512 columns is all of an SM's
// tensor memory, which the one CTA per SM owns.
constexpr int kAcc = 4;
// Row pitch of the radix path's staged epilogue tile (256 bytes of data plus
// 8, so that the 32 lanes' 8-byte stores of one row each fall on distinct
// banks two lanes at a time).
constexpr int kStgRow = 264;
static_assert(2 * 128 * kStgRow <= kStages * kStageBytes, "staging tile exceeds the ring");
static_assert(2 * 128 * 128 * 4 <= kStages * kStageBytes, "staging rows exceed the ring");

enum Epi { EPI_F32 = 0, EPI_SPLIT = 1, EPI_SPECTRAL = 2, EPI_PSI_EX = 3, EPI_EY = 4,
           EPI_TWIDDLE = 5, EPI_CPLX = 6 };

struct EpiArgs {
    __nv_bfloat16* hi;   // EPI_SPLIT / EPI_SPECTRAL outputs [row][ld]
    __nv_bfloat16* lo;
    int ld;
    float* f32;          // EPI_F32 [row][ld]; EPI_PSI_EX: psi [row][n]
    float2* E2;          // EPI_PSI_EX (.x) and EPI_EY (.y), [row][n]
    int n;
    float pi_lx, pi_ly, invn2;
    float eps;           // EPI_SPECTRAL: Helmholtz term (0: Poisson)
    double* acc;
    DetRed dr;
    int* err;
    int no_loads;        // test hook: issue no TMA loads (the waits then expire)
    // radix path (EPI_TWIDDLE, EPI_CPLX): DFT length n = 64 n2, g = 64 / n2
    // rows per second-stage tile, twiddles tw[k] = exp(-2 pi i k / n),
    // inv: conjugate twiddles, V: complex output rows [r][n]
    int n2, g, inv;
    int ln2, lg;         // log2 n2, log2 g (n2 and g are powers of two)
    const float2* tw;
    float2* V;
};

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase,
                                          unsigned long long limit_ns) {
    if (mbar_try(bar, phase)) return true;
    unsigned long long t0 = global_ns();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 256; ++i)
            if (mbar_try(bar, phase)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)(uintptr_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand in swizzled atoms of
// 8 rows x kSwz bytes, atoms 8 kSwz bytes apart (layout 2: 128-byte
// swizzle, 4: 64-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused here)
    d |= (uint64_t)((8 * kSwz) >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)(kSwz == 128 ? 2 : 4) << 61;     // swizzle mode
    return d;
}

// Instruction descriptor, kind::f16: bf16 A and B, f32 accumulator, both
// K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// ------------------------------------------------------------------ kernel
template <int EPI>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
k_tc_gemm(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
          const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
          int K, int ntn, int nsplit, EpiArgs ep) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages];
    __shared__ __align__(8) uint64_t empty_bar[kStages];
    __shared__ __align__(8) uint64_t accum_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // one 1-D grid of tiles, column tiles fastest (CTAs in flight share A rows)
    const int m0 = (blockIdx.x / ntn) * BM, n0 = (blockIdx.x % ntn) * BN;
    const int ktiles = K / BK;
    const int nacc = ktiles < kAcc ? ktiles : kAcc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&accum_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(kAcc * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the operand tiles into the stage ring
        const uint32_t bytes = (nsplit == 3 ? 4u : 2u) * kTileBytes;
        int issued = 0;
        for (int kt = 0; kt < ktiles && !ep.no_loads; ++kt) {
            const int s = kt % kStages;
            const uint32_t ph = (uint32_t)(kt / kStages) & 1u;
            if (*(volatile int*)&s_abort) break;
            if (kt >= kStages && !mbar_wait(&empty_bar[s], ph ^ 1u, kWaitNs)) {
                atomicOr(ep.err, ERR_TIMEOUT);
                s_abort = 1;
                break;
            }
            uint8_t* st = smem + (size_t)s * kStageBytes;
            mbar_expect_tx(&full_bar[s], bytes);
            tma_load_2d(st, &tAh, kt * BK, m0, &full_bar[s]);
            tma_load_2d(st + 2 * kTileBytes, &tBh, kt * BK, n0, &full_bar[s]);
            if (nsplit == 3) {
                tma_load_2d(st + kTileBytes, &tAl, kt * BK, m0, &full_bar[s]);
                tma_load_2d(st + 3 * kTileBytes, &tBl, kt * BK, n0, &full_bar[s]);
            }
            ++issued;
        }
        // loads still in flight must land before the CTA can exit
        for (int kt = (issued > kStages ? issued - kStages : 0); kt < issued; ++kt)
            mbar_wait(&full_bar[kt % kStages], (uint32_t)(kt / kStages) & 1u, kWaitNs);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer; chunk c holds k-tiles [ceil(c K' / nacc), ceil((c+1) K' / nacc))
        int chunk = 0, next_start = (ktiles + nacc - 1) / nacc;
        const uint64_t d_ring = smem_desc(smem_u32(smem));
        for (int kt = 0; kt < ktiles; ++kt) {
            bool first = kt == 0;
            if (kt == next_start) {
                ++chunk;
                first = true;
                next_start = ((chunk + 1) * ktiles + nacc - 1) / nacc;
            }
            const int s = kt % kStages;
            const uint32_t ph = (uint32_t)(kt / kStages) & 1u;
            if (!mbar_wait(&full_bar[s], ph, kWaitNs)) {
                atomicOr(ep.err, ERR_TIMEOUT);
                s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // descriptors of this stage: the start-address field (bits 0-13,
            // address >> 4) of the ring's base descriptor advanced by the
            // stage, operand and k offsets (the whole ring lies below 256 KiB,
            // so the field cannot carry into the next one)
            const uint64_t ds = d_ring + (uint64_t)((s * kStageBytes) >> 4);
            const uint32_t d = tmem + (uint32_t)(chunk * BN);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                // 16 bf16 along K inside the swizzle atom: 32 bytes
                const uint64_t a_hi = ds + (uint64_t)((kk * 32) >> 4);
                const uint64_t a_lo = a_hi + (uint64_t)(kTileBytes >> 4);
                const uint64_t b_hi = a_hi + (uint64_t)((2 * kTileBytes) >> 4);
                const uint64_t b_lo = a_hi + (uint64_t)((3 * kTileBytes) >> 4);
                const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
                mma_bf16(d, a_hi, b_hi, acc);
                if (nsplit == 3) {
                    mma_bf16(d, a_hi, b_lo, 1u);
                    mma_bf16(d, a_lo, b_hi, 1u);
                }
            }
            mma_commit(&empty_bar[s]);
        }
        mma_commit(&accum_bar);   // arrives once every issued MMA has completed
    }
    __syncthreads();
    // epilogue: accumulator rows 32 w .. 32 w + 31 belong to warp w
    const bool ok = mbar_wait(&accum_bar, 0, 2 * kWaitNs);
    if (!ok && lane == 0) atomicOr(ep.err, ERR_TIMEOUT);
    // block-uniform decision: tcgen05.ld is warp-collective
    const bool store = __syncthreads_and(ok && !s_abort) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    dfloat energy = df_zero();
    const int row = m0 + warp * 32 + lane;
    if (store) {
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            float v[32], t[32];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32);
            tmem_ld32(ta, v);
            // chunks summed in a fixed order
            for (int a = 1; a < nacc; ++a) {
                tmem_ld32(ta + (uint32_t)(a * BN), t);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] += t[j];
            }
            const int col0 = n0 + c * 32;
            if (EPI == EPI_F32) {
                float4* dst = reinterpret_cast<float4*>(ep.f32 + (size_t)row * ep.ld + col0);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else if (EPI == EPI_SPLIT || EPI == EPI_SPECTRAL) {
                if (EPI == EPI_SPECTRAL) {
                    // row = v, column = u; v[] holds B[v][u] (unnormalised)
                    const int vv = row;
                    const float wv = ep.pi_ly * (float)vv;
                    const float ev = vv == 0 ? 1.0f : 2.0f;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int u = col0 + j;
                        const float wu = ep.pi_lx * (float)u;
                        const float eu = u == 0 ? 1.0f : 2.0f;
                        const float a = eu * ev * ep.invn2 * v[j];
                        const float p = (u == 0 && vv == 0 && !(ep.eps > 0.0f))
                                            ? 0.0f
                                            : a / (wu * wu + wv * wv + ep.eps);
                        energy = df_add(energy, v[j] * p);
                        v[j] = p;
                    }
                }
                __align__(16) __nv_bfloat16 h[32], l[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) split_bf16(v[j], h[j], l[j]);
                uint4* dh = reinterpret_cast<uint4*>(ep.hi + (size_t)row * ep.ld + col0);
                uint4* dl = reinterpret_cast<uint4*>(ep.lo + (size_t)row * ep.ld + col0);
                const uint4* sh = reinterpret_cast<const uint4*>(h);
                const uint4* sl = reinterpret_cast<const uint4*>(l);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    dh[q] = sh[q];
                    dl[q] = sl[q];
                }
            } else if (EPI == EPI_TWIDDLE) {
                // row = 2 k1 + c (c: real / imaginary part), column = r n2 + j2:
                // Y[r][k1][j2] times exp(-+2 pi i j2 k1 / n), written as the
                // second stage's operand A2[(r / g) 64 + k1][(r % g) 2 n2 + c n2 + j2]
                const int k1 = row >> 1, cc = row & 1;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float other = __shfl_xor_sync(0xffffffffu, v[j], 1);
                    const int col = col0 + j;
                    const int j2 = col & (ep.n2 - 1);
                    const float2 w = ep.tw[j2 * k1];
                    const float wi = ep.inv ? -w.y : w.y;
                    const float re = cc ? other : v[j], im = cc ? v[j] : other;
                    v[j] = cc ? fmaf(re, wi, im * w.x) : fmaf(re, w.x, -im * wi);
                }
                __align__(16) __nv_bfloat16 h[32], l[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) split_bf16(v[j], h[j], l[j]);
                // the tile's output is rows [n0, n0 + 128) of A2, whole: staged
                // in the (now idle) operand ring, rows kStgRow bytes apart, hi
                // then lo; 4 consecutive j2 of one r per store (n2 is a
                // multiple of 4)
                for (int j = 0; j < 32; j += 4) {
                    const int col = col0 + j;
                    const int r = col >> ep.ln2, j2 = col & (ep.n2 - 1);
                    const int lr = ((r >> ep.lg) << 6) + k1 - n0;
                    const int kk = (((r & (ep.g - 1)) << 1) + cc) * ep.n2 + j2;
                    uint8_t* at = smem + (size_t)lr * kStgRow + 2 * kk;
                    *reinterpret_cast<uint2*>(at) = *reinterpret_cast<const uint2*>(h + j);
                    *reinterpret_cast<uint2*>(at + 128 * kStgRow) =
                        *reinterpret_cast<const uint2*>(l + j);
                }
            } else if (EPI == EPI_CPLX) {
                // row = (G, k1), column = q 2 n2 + c n2 + k2: component c of
                // V[G g + q][k1 + 64 k2].  The tile's output is the 2 g whole
                // rows from V[(m0 / 64) g]: staged in the idle operand ring
                const int lg = (row >> 6) - (m0 >> 6), k1 = row & 63;
                float* stg = reinterpret_cast<float*>(smem);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = col0 + j;
                    const int q = col >> (ep.ln2 + 1), cc = (col >> ep.ln2) & 1;
                    const int k2 = col & (ep.n2 - 1);
                    stg[((size_t)(lg * ep.g + q) * ep.n + k1 + 64 * k2) * 2 + cc] = v[j];
                }
            } else if (EPI == EPI_PSI_EX) {
                if (col0 < ep.n) {
                    float4* dst = reinterpret_cast<float4*>(ep.f32 + (size_t)row * ep.n + col0);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
                    float* dst = reinterpret_cast<float*>(ep.E2 + (size_t)row * ep.n + (col0 - ep.n));
#pragma unroll
                    for (int j = 0; j < 32; ++j) dst[2 * j] = v[j];
                }
            } else {   // EPI_EY
                float* dst = reinterpret_cast<float*>(ep.E2 + (size_t)row * ep.n + col0) + 1;
#pragma unroll
                for (int j = 0; j < 32; ++j) dst[2 * j] = v[j];
            }
        }
    }
    if (EPI == EPI_TWIDDLE && store) {
        // rows [n0, n0 + 128) of A2 (hi, lo): 256 bytes each, 8 bytes a
        // thread (the staged rows are kStgRow = 8 mod 16 bytes apart)
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * 128 * 32; i += kThreads) {
            const int half = i >> 12, lr = (i >> 5) & 127, q = i & 31;
            const uint2 val = *reinterpret_cast<const uint2*>(
                smem + (size_t)(half * 128 + lr) * kStgRow + 8 * q);
            __nv_bfloat16* dst = (half ? ep.lo : ep.hi) + (size_t)(n0 + lr) * 128;
            reinterpret_cast<uint2*>(dst)[q] = val;
        }
    }
    if (EPI == EPI_CPLX && store) {
        // 2 g rows of n complex values from V[(m0 / 64) g]: 64 KiB, contiguous
        __syncthreads();
        const size_t count4 = (size_t)2 * ep.g * ep.n * 2 / 4;
        const float4* src = reinterpret_cast<const float4*>(smem);
        float4* dst = reinterpret_cast<float4*>(ep.V + (size_t)(m0 >> 6) * ep.g * ep.n);
        for (size_t i = threadIdx.x; i < count4; i += kThreads) dst[i] = src[i];
    }
    if (EPI == EPI_SPECTRAL) reduce2(df_val(energy), 0.0f, ep.acc, ACC_N, -1, ep.dr);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAcc * BN));
}

// Tables: C[u][x], the stacked [Ct; Sx] (Ct[x][u] = C[u][x]) and Sy[y][v],
// each split into bf16 hi and lo.  Arguments reduced exactly:
// cos(pi u (2x+1) / 2n) = cospi(k / 2n), k = u (2x+1) mod 4n.
__global__ void k_tc_tables(int n, double pi_lx, double pi_ly, __nv_bfloat16* C_hi,
                            __nv_bfloat16* C_lo, __nv_bfloat16* CS_hi, __nv_bfloat16* CS_lo,
                            __nv_bfloat16* Sy_hi, __nv_bfloat16* Sy_lo) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    int r = (int)(idx / n), k = (int)(idx % n);     // row, column
    // C[u = r][x = k]
    long long a = ((long long)r * (2LL * k + 1)) % (4LL * n);
    double s, cc;
    sincospi((double)a / (2.0 * n), &s, &cc);
    split_bf16((float)cc, C_hi[idx], C_lo[idx]);
    // Ct[x = r][u = k] and Sx[x = r][u = k]
    long long b = ((long long)k * (2LL * r + 1)) % (4LL * n);
    sincospi((double)b / (2.0 * n), &s, &cc);
    split_bf16((float)cc, CS_hi[idx], CS_lo[idx]);
    split_bf16((float)(pi_lx * k * s), CS_hi[(size_t)n * n + idx], CS_lo[(size_t)n * n + idx]);
    // Sy[y = r][v = k]
    split_bf16((float)(pi_ly * k * s), Sy_hi[idx], Sy_lo[idx]);
}


// Radix path tables: the 64-point DFT as a real 128 x 128 block
// F1[2 k1 + c'][c 64 + j1] and the n2-point DFT block-diagonal over g rows,
// F2[q 2 n2 + c' n2 + k2][q' 2 n2 + c n2 + j2] (0 for q != q'), for the
// forward (exp(-i theta)) and inverse (exp(+i theta)) directions, split into
// bf16 hi and lo.  Entry (c' <- c): cos for c = c', +sin (re <- im) and
// -sin (im <- re) forward, the opposite signs inverse.  Arguments reduced
// exactly: theta = 2 pi (j k mod L) / L.
__global__ void k_tcr_tables(int n2, int g, __nv_bfloat16* F1, __nv_bfloat16* F2) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 128 * 128) return;
    const int m = idx / 128, kk = idx % 128;
    for (int dir = 0; dir < 2; ++dir) {
        const double sg = dir == 0 ? 1.0 : -1.0;
        {
            const int k1 = m >> 1, co = m & 1, ci = kk >> 6, j1 = kk & 63;
            double sn, cs;
            sincospi(2.0 * (double)((j1 * k1) % 64) / 64.0, &sn, &cs);
            const double val = co == ci ? cs : (co == 0 ? sg * sn : -sg * sn);
            __nv_bfloat16* base = F1 + (size_t)dir * 2 * 128 * 128;
            split_bf16((float)val, base[idx], base[128 * 128 + idx]);
        }
        {
            const int qo = m / (2 * n2), co = (m % (2 * n2)) / n2, k2 = m % n2;
            const int qi = kk / (2 * n2), ci = (kk % (2 * n2)) / n2, j2 = kk % n2;
            double val = 0.0;
            if (qo == qi && qo < g) {
                double sn, cs;
                sincospi(2.0 * (double)((j2 * k2) % n2) / (double)n2, &sn, &cs);
                val = co == ci ? cs : (co == 0 ? sg * sn : -sg * sn);
            }
            __nv_bfloat16* base = F2 + (size_t)dir * 2 * 128 * 128;
            split_bf16((float)val, base[idx], base[128 * 128 + idx]);
        }
    }
}

// Complex rows Z[r][0..n) into the first stage's operand, bf16 hi/lo:
// Xt[r n2 + j2][c 64 + j1] = component c of Z[r][n2 j1 + j2] (one CTA per
// row, staged in shared memory, padded one element in 32).
__global__ void __launch_bounds__(128)
k_tcr_split(int n, int n2, const float2* __restrict__ Z, __nv_bfloat16* __restrict__ xh,
            __nv_bfloat16* __restrict__ xl) {
    extern __shared__ float2 zs[];
    const int r = blockIdx.x;
    const float2* zr = Z + (size_t)r * n;
    for (int i = threadIdx.x; i < n; i += 128) zs[i + (i >> 5)] = zr[i];
    __syncthreads();
    const int t = threadIdx.x, c = t >> 6, j1 = t & 63;
    for (int j2 = 0; j2 < n2; ++j2) {
        const int i = n2 * j1 + j2;
        const float2 z = zs[i + (i >> 5)];
        __nv_bfloat16 h, l;
        split_bf16(c ? z.y : z.x, h, l);
        const size_t at = ((size_t)r * n2 + j2) * 128 + t;
        xh[at] = h;
        xl[at] = l;
    }
}

// rho = (D + M) / A_b split into bf16 hi/lo, four bins per thread, with the
// overflow and charge sums of the transform path's row pass.
template <bool QUANT>
__global__ void __launch_bounds__(256)
k_tc_rho(int count4, const float* __restrict__ D, const long long* __restrict__ Dq,
         const float* __restrict__ M, float inv_ab, float cap, __nv_bfloat16* __restrict__ hi,
         __nv_bfloat16* __restrict__ lo, double* __restrict__ acc, DetRed dr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    dfloat tau = df_zero(), charge = df_zero();
    if (i < count4) {
        size_t b = (size_t)i * 4;
        float4 mv = *reinterpret_cast<const float4*>(M + b);
        float m4[4] = {mv.x, mv.y, mv.z, mv.w}, d4[4];
        if (QUANT) {
            longlong2 q0 = *reinterpret_cast<const longlong2*>(Dq + b);
            longlong2 q1 = *reinterpret_cast<const longlong2*>(Dq + b + 2);
            d4[0] = (float)q0.x * 2.3283064365386963e-10f;
            d4[1] = (float)q0.y * 2.3283064365386963e-10f;
            d4[2] = (float)q1.x * 2.3283064365386963e-10f;
            d4[3] = (float)q1.y * 2.3283064365386963e-10f;
        } else {
            float4 dv = *reinterpret_cast<const float4*>(D + b);
            d4[0] = dv.x; d4[1] = dv.y; d4[2] = dv.z; d4[3] = dv.w;
        }
        __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            tau = df_add(tau, fmaxf(0.0f, d4[t] - (cap - m4[t])));
            charge = df_add(charge, d4[t] + m4[t]);
            split_bf16((d4[t] + m4[t]) * inv_ab, h[t], l[t]);
        }
        *reinterpret_cast<uint2*>(hi + b) = *reinterpret_cast<const uint2*>(h);
        *reinterpret_cast<uint2*>(lo + b) = *reinterpret_cast<const uint2*>(l);
    }
    reduce2(df_val(tau), df_val(charge), acc, ACC_TAU, ACC_CHARGE, dr);
}

}  // namespace tc

// ------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D bf16 tensor [rows][cols] (cols contiguous) read in 128-row x BK-column
// boxes with the kSwz-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int rows, int cols) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)tc::BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    tc::kSwz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool make_map_f32(CUtensorMap* map, const float* base, int rows, int cols, int box_inner,
                  int box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

template <int EPI>
void set_smem_attr() {
    cudaFuncSetAttribute(tc::k_tc_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::kSmemBytes);
}

void prepare_gemm() {
    static std::once_flag once;
    std::call_once(once, [] {
        set_smem_attr<tc::EPI_F32>();
        set_smem_attr<tc::EPI_SPLIT>();
        set_smem_attr<tc::EPI_SPECTRAL>();
        set_smem_attr<tc::EPI_PSI_EX>();
        set_smem_attr<tc::EPI_EY>();
        set_smem_attr<tc::EPI_TWIDDLE>();
        set_smem_attr<tc::EPI_CPLX>();
        cudaFuncSetAttribute(tc::k_tcr_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((4096 + 4096 / 32) * sizeof(float2)));
    });
}

// D[M][N] = sum_k A[M][k] B[N][k]; M, N multiples of 128, K of 64.
template <int EPI>
cudaError_t gemm(const CUtensorMap* a, const CUtensorMap* b, int M, int N, int K, int nsplit,
                 const tc::EpiArgs& ep, cudaStream_t s) {
    const int ntn = N / tc::BN;
    tc::k_tc_gemm<EPI><<<(M / tc::BM) * ntn, tc::kThreads, tc::kSmemBytes, s>>>(
        a[0], a[1], b[0], b[1], K, ntn, nsplit, ep);
    return cudaGetLastError();
}

}  // namespace

// Device operands of the tensor-core solve: one block of 18 n^2 bf16.
struct TcPlan {
    int n = 0;
    __nv_bfloat16 *C[2], *CS[2], *Sy[2], *R[2], *A1[2], *P[2], *UX[2];
    CUtensorMap mC[2], mCS[2], mSy[2], mR[2], mA1[2], mP[2], mUX[2];
    // G7 runs on its own stream beside G46 (both only read G35's output)
    cudaStream_t s2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~TcPlan() {
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (s2) cudaStreamDestroy(s2);
    }
};

size_t tc_elems(int n) { return 18 * (size_t)n * n; }

cudaError_t tc_setup(Ctx& c, uint16_t* block, cudaStream_t s) {
    const int n = c.n;
    const size_t nn = (size_t)n * n;
    TcPlan* p = new (std::nothrow) TcPlan();
    if (!p) return cudaErrorMemoryAllocation;
    p->n = n;
    __nv_bfloat16* q = reinterpret_cast<__nv_bfloat16*>(block);
    auto take = [&](size_t count) { __nv_bfloat16* r = q; q += count; return r; };
    for (int h = 0; h < 2; ++h) {
        p->C[h] = take(nn);
        p->CS[h] = take(2 * nn);
        p->Sy[h] = take(nn);
        p->R[h] = take(nn);
        p->A1[h] = take(nn);
        p->P[h] = take(nn);
        p->UX[h] = take(2 * nn);
    }
    bool ok = true;
    for (int h = 0; h < 2; ++h) {
        ok = ok && make_map(&p->mC[h], p->C[h], n, n) && make_map(&p->mCS[h], p->CS[h], 2 * n, n) &&
             make_map(&p->mSy[h], p->Sy[h], n, n) && make_map(&p->mR[h], p->R[h], n, n) &&
             make_map(&p->mA1[h], p->A1[h], n, n) && make_map(&p->mP[h], p->P[h], n, n) &&
             make_map(&p->mUX[h], p->UX[h], 2 * n, n);
    }
    if (!ok) {
        delete p;
        return cudaErrorInvalidValue;
    }
    if (ok)
        ok = cudaStreamCreateWithFlags(&p->s2, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        delete p;
        return cudaErrorInvalidValue;
    }
    prepare_gemm();
    c.tc = p;
    tc::k_tc_tables<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(
        n, M_PI / c.Lx, M_PI / c.Ly, p->C[0], p->C[1], p->CS[0], p->CS[1], p->Sy[0], p->Sy[1]);
    return cudaGetLastError();
}

void tc_free(Ctx& c) {
    delete c.tc;
    c.tc = nullptr;
}

// part 0: rho split (with the overflow and charge sums); 1: G1; 2: G2 with
// the spectral divide and the energy; 3: G35, G46 and G7 (psi, E_x, E_y).
cudaError_t launch_tc(Ctx& c, int part, cudaStream_t s) {
    TcPlan& p = *c.tc;
    const int n = c.n;
    tc::EpiArgs ep{};
    ep.n = n;
    ep.ld = n;
    ep.err = c.err;
    ep.acc = c.acc;
    ep.dr = det_red(c, 0);
    cudaError_t e = cudaSuccess;
    if (part == 0) {
        const int count4 = n * n / 4;
        const float inv_ab = (float)(1.0 / c.Ab);
        const float cap = (float)(c.opt.target_density * c.Ab);
        const unsigned blocks = (unsigned)((count4 + 255) / 256);
        if (c.opt.deterministic)
            tc::k_tc_rho<true><<<blocks, 256, 0, s>>>(count4, nullptr, c.Dq, c.M, inv_ab, cap,
                                                      p.R[0], p.R[1], c.acc, ep.dr);
        else
            tc::k_tc_rho<false><<<blocks, 256, 0, s>>>(count4, c.D, nullptr, c.M, inv_ab, cap,
                                                       p.R[0], p.R[1], c.acc, ep.dr);
        e = cudaGetLastError();
        c.launches++;
    } else if (part == 1) {
        ep.hi = p.A1[0];
        ep.lo = p.A1[1];
        e = gemm<tc::EPI_SPLIT>(p.mC, p.mR, n, n, n, 3, ep, s);
        c.launches++;
    } else if (part == 2) {
        ep.hi = p.P[0];
        ep.lo = p.P[1];
        ep.pi_lx = (float)(M_PI / c.Lx);
        ep.pi_ly = (float)(M_PI / c.Ly);
        ep.invn2 = 1.0f / ((float)n * (float)n);
        ep.eps = (float)c.opt.helmholtz_eps;
        e = gemm<tc::EPI_SPECTRAL>(p.mC, p.mA1, n, n, n, 3, ep, s);
        c.launches++;
    } else {
        ep.hi = p.UX[0];
        ep.lo = p.UX[1];
        e = gemm<tc::EPI_SPLIT>(p.mCS, p.mP, 2 * n, n, n, 3, ep, s);
        c.launches++;
        if (e != cudaSuccess) return e;
        // G46 (512 tiles at the launch's own stream) and G7 (256 tiles on
        // s2) together: their 768 tiles fill about 5 waves of SMs instead of
        // 4 + 2 one after the other; they write disjoint halves of E2
        ep.f32 = c.psi;
        ep.E2 = c.E2;
        e = cudaEventRecord(p.fork, s);
        if (e != cudaSuccess) return e;
        e = cudaStreamWaitEvent(p.s2, p.fork, 0);
        if (e != cudaSuccess) return e;
        e = gemm<tc::EPI_PSI_EX>(p.mCS, p.mUX, n, 2 * n, n, 3, ep, s);
        c.launches++;
        const cudaError_t e7 = gemm<tc::EPI_EY>(p.mSy, p.mUX, n, n, n, 3, ep, p.s2);
        c.launches++;
        // join in every case, so that a capture stays well formed
        const cudaError_t ej = cudaEventRecord(p.join, p.s2);
        const cudaError_t ew = ej == cudaSuccess ? cudaStreamWaitEvent(s, p.join, 0) : ej;
        if (e == cudaSuccess) e = e7;
        if (e == cudaSuccess) e = ew;
    }
    return e;
}

// ----------------------------------------------- radix path (f3)
// Every complex DFT of length n = 64 n2 on R rows as two products on the
// tensor cores (a four-step factorisation): stage 1, the 64-point DFTs
// over j1 for every (row, j2), D1 = F1 Xt^T (M = 128, N = R n2, K = 128),
// with the twiddles exp(-+2 pi i j2 k1 / n) in its epilogue; stage 2, the
// n2-point DFTs over j2, D2 = A2 F2^T (M = R n2, N = 128, K = 128), g rows
// side by side in one tile (F2 block-diagonal), written as complex rows.
struct TcrPlan {
    int n = 0, n2 = 0, g = 0;
    __nv_bfloat16 *F1 = nullptr, *F2 = nullptr, *X[2] = {}, *A2[2] = {};
    CUtensorMap mF1[2][2], mF2[2][2], mX[2], mA2[2];
    float2 *Z = nullptr, *V = nullptr;
};

size_t tcr_elems(int n) {
    // bf16: F1, F2 (2 directions x hi/lo x 128^2), X and A2 (hi/lo x 2 n^2 each)
    return 8 * 128 * 128 + 8 * (size_t)n * n;
}

cudaError_t tcr_setup(Ctx& c, uint16_t* block, float2* zv, cudaStream_t s) {
    const int n = c.n;
    TcrPlan* p = new (std::nothrow) TcrPlan();
    if (!p) return cudaErrorMemoryAllocation;
    p->n = n;
    p->n2 = n / 64;
    p->g = 64 / p->n2 > 0 ? 64 / p->n2 : 1;
    __nv_bfloat16* q = reinterpret_cast<__nv_bfloat16*>(block);
    auto take = [&](size_t count) { __nv_bfloat16* r = q; q += count; return r; };
    p->F1 = take(4 * 128 * 128);
    p->F2 = take(4 * 128 * 128);
    const size_t rows = (size_t)n * p->n2;   // R_max n2 with R_max = n rows
    for (int h = 0; h < 2; ++h) {
        p->X[h] = take(rows * 128);
        p->A2[h] = take(rows * 128);
    }
    p->Z = zv;
    p->V = zv + (size_t)n * n;
    bool ok = true;
    for (int dir = 0; dir < 2; ++dir)
        for (int h = 0; h < 2; ++h) {
            ok = ok && make_map(&p->mF1[dir][h], p->F1 + (size_t)(2 * dir + h) * 128 * 128, 128, 128);
            ok = ok && make_map(&p->mF2[dir][h], p->F2 + (size_t)(2 * dir + h) * 128 * 128, 128, 128);
        }
    for (int h = 0; h < 2; ++h)
        ok = ok && make_map(&p->mX[h], p->X[h], (int)rows, 128) &&
             make_map(&p->mA2[h], p->A2[h], (int)rows, 128);
    if (!ok) {
        delete p;
        return cudaErrorInvalidValue;
    }
    prepare_gemm();
    c.tcr = p;
    tc::k_tcr_tables<<<(128 * 128 + 255) / 256, 256, 0, s>>>(p->n2, p->g, p->F1, p->F2);
    return cudaGetLastError();
}

void tcr_free(Ctx& c) {
    delete c.tcr;
    c.tcr = nullptr;
}

// DFT of rows Z[0..R) into V[0..R): forward (exp(-i ...)) or inverse
// (exp(+i ...), no 1/n), as the transform path's FFTs.
static cudaError_t tcr_dft(Ctx& c, int R, int inv, cudaStream_t s) {
    TcrPlan& p = *c.tcr;
    const int n = p.n;
    tc::k_tcr_split<<<R, 128, (size_t)(n + n / 32) * sizeof(float2), s>>>(n, p.n2, p.Z, p.X[0],
                                                                          p.X[1]);
    cudaError_t e = cudaGetLastError();
    c.launches++;
    if (e != cudaSuccess) return e;
    tc::EpiArgs ep{};
    ep.n = n;
    ep.n2 = p.n2;
    ep.g = p.g;
    ep.ln2 = 0;
    while ((1 << ep.ln2) < p.n2) ep.ln2++;
    ep.lg = 0;
    while ((1 << ep.lg) < p.g) ep.lg++;
    ep.inv = inv;
    ep.tw = c.tw;
    ep.err = c.err;
    ep.dr = det_red(c, 0);
    ep.hi = p.A2[0];
    ep.lo = p.A2[1];
    const int cols = R * p.n2;
    e = gemm<tc::EPI_TWIDDLE>(p.mF1[inv], p.mX, 128, cols, 128, 3, ep, s);
    c.launches++;
    if (e != cudaSuccess) return e;
    ep.V = p.V;
    e = gemm<tc::EPI_CPLX>(p.mA2, p.mF2[inv], cols, 128, 128, 3, ep, s);
    c.launches++;
    return e;
}

// part 0: the row pass (rho -> T1, with the overflow and charge sums);
// 1: the column pass (T1 -> spectra, divide, energy -> PT, RT); 2: the
// inverse row pass (PT, RT -> E2); 3: the overflow and charge sums alone.
cudaError_t launch_tcr(Ctx& c, int part, cudaStream_t s) {
    TcrPlan& p = *c.tcr;
    const int n = p.n;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (part == 0) {
        step(launch_tcr_stage(c, 0, p.V, p.Z, s));
        step(tcr_dft(c, n / 2, 0, s));
        step(launch_tcr_stage(c, 1, p.V, p.Z, s));
    } else if (part == 1) {
        step(launch_tcr_stage(c, 2, p.V, p.Z, s));
        step(tcr_dft(c, n / 2, 0, s));
        step(launch_tcr_stage(c, 3, p.V, p.Z, s));
        step(tcr_dft(c, n, 1, s));
        step(launch_tcr_stage(c, 4, p.V, p.Z, s));
    } else if (part == 2) {
        step(launch_tcr_stage(c, 5, p.V, p.Z, s));
        step(tcr_dft(c, n, 1, s));
        step(launch_tcr_stage(c, 6, p.V, p.Z, s));
    } else {
        step(launch_tcr_stage(c, 0, p.V, p.Z, s));
    }
    return e;
}

// Test entry of the GEMM core (see fftpl_debug_tc_gemm).
cudaError_t tc_debug_gemm(const void* ah, const void* al, const void* bh, const void* bl, int M,
                          int N, int K, float* d, int nsplit, int no_loads, int* err,
                          cudaStream_t s) {
    CUtensorMap ma[2], mb[2];
    if (!make_map(&ma[0], ah, M, K) || !make_map(&ma[1], al, M, K) || !make_map(&mb[0], bh, N, K) ||
        !make_map(&mb[1], bl, N, K))
        return cudaErrorInvalidValue;
    prepare_gemm();
    tc::EpiArgs ep{};
    ep.f32 = d;
    ep.ld = N;
    ep.err = err;
    ep.no_loads = no_loads;
    ep.dr = DetRed{nullptr, nullptr, 0};
    return gemm<tc::EPI_F32>(ma, mb, M, N, K, nsplit, ep, s);
}

}  // namespace fftpl
