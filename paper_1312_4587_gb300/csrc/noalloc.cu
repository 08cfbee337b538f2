// fftpl_solve_noalloc: the spectral Poisson solve of a caller-supplied
// density map without any device allocation, for callers that cannot
// allocate (see include/fftpl.h).  The three transform passes and the field
// split are the library's own kernels; their intermediates (the transposed
// row transforms, the column results, the interleaved field), the transform
// tables and the FP64 sums live in one file-scope device array.
#include <math.h>

#include <mutex>

#include "fftpl_internal.cuh"

namespace fftpl {

namespace {

constexpr int kMaxN = FFTPL_NOALLOC_MAX_N;
constexpr size_t kMap = (size_t)kMaxN * kMaxN;   // floats per map
// layout in bytes (all offsets multiples of 256)
constexpr size_t kOffT1 = 0;
constexpr size_t kOffPT = kOffT1 + kMap * sizeof(float);
constexpr size_t kOffRT = kOffPT + kMap * sizeof(float);
constexpr size_t kOffE2 = kOffRT + kMap * sizeof(float);
constexpr size_t kOffTw = kOffE2 + kMap * sizeof(float2);
constexpr size_t kOffPh = kOffTw + (size_t)kMaxN * sizeof(float2);
constexpr size_t kOffAcc = kOffPh + ((size_t)kMaxN + 256 / sizeof(float2)) * sizeof(float2);
constexpr size_t kScratchBytes = kOffAcc + (size_t)kAccDoubles * sizeof(double);
static_assert(kOffAcc % 256 == 0, "scratch layout alignment");

// The scratch array.  In host code this name is a host-side stand-in; its
// device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {};

// FFT twiddles exp(-2 pi i k / n) and cosine-transform twiddles
// exp(-i pi u / 2n), from sincospi in FP64.
__global__ void k_tables(int n, float2* __restrict__ tw, float2* __restrict__ ph) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double s, c;
        sincospi(2.0 * i / n, &s, &c);
        tw[i] = make_float2((float)c, (float)-s);
    }
    if (i <= n) {
        double s, c;
        sincospi((double)i / (2.0 * n), &s, &c);
        ph[i] = make_float2((float)c, (float)-s);
    }
}

// Per-device set-up: the array's device address (with the device current),
// and the kernels' shared-memory limits for every grid size.
fftpl_status scratch_for_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_global_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return FFTPL_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_global_error("device index out of range for the allocation-free path");
        return FFTPL_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_global_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return FFTPL_ECUDA;
        }
        for (int logn = 4; (1 << logn) <= kMaxN; ++logn) prepare_spectral(logn);
        g_dev_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_dev_ptr[dev];
    return FFTPL_OK;
}

}  // namespace

}  // namespace fftpl

using namespace fftpl;

extern "C" fftpl_status fftpl_solve_noalloc(const float* rho, int32_t n, double Lx, double Ly,
                                            float* psi, float* ex, float* ey, double* N,
                                            void* stream) {
    if (n < FFTPL_MIN_N || n > kMaxN || (n & (n - 1)) != 0) {
        set_global_error("fftpl_solve_noalloc: n must be a power of two in [16, " +
                         std::to_string(kMaxN) + "]");
        return FFTPL_EINVAL;
    }
    if (!rho || !psi || !ex || !ey) {
        set_global_error("fftpl_solve_noalloc: null map pointer");
        return FFTPL_EINVAL;
    }
    if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(psi) |
         reinterpret_cast<uintptr_t>(ex) | reinterpret_cast<uintptr_t>(ey)) & 15u) {
        set_global_error("fftpl_solve_noalloc: rho, psi, ex and ey must be 16-byte aligned");
        return FFTPL_EINVAL;
    }
    if (!(Lx > 0.0) || !(Ly > 0.0) || !isfinite(Lx) || !isfinite(Ly)) {
        set_global_error("fftpl_solve_noalloc: region sizes must be finite and > 0");
        return FFTPL_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (N) {
        // N is read back with a synchronisation, which a capture cannot hold
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing(s, &cap);
        if (ce != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
            set_global_error("fftpl_solve_noalloc: N must be NULL while the stream is captured");
            return FFTPL_EINVAL;
        }
    }
    unsigned char* base = nullptr;
    fftpl_status st = scratch_for_device(&base);
    if (st != FFTPL_OK) return st;

    // A context on the stack pointing into the scratch array.  The row pass
    // forms (D + M) / A_b; with D = M = rho and 1/A_b = 0.5 that is rho
    // exactly.  The target density 0 makes its overflow sum unused.
    Ctx c;
    c.n = n;
    c.logn = 0;
    while ((1 << c.logn) < n) c.logn++;
    c.Lx = Lx;
    c.Ly = Ly;
    c.Ab = 2.0;
    c.opt.target_density = 0.0;
    c.opt.deterministic = 0;
    c.D = const_cast<float*>(rho);
    c.M = const_cast<float*>(rho);
    c.T1 = reinterpret_cast<float*>(base + kOffT1);
    c.PT = reinterpret_cast<float*>(base + kOffPT);
    c.RT = reinterpret_cast<float*>(base + kOffRT);
    spec_maps_init(c);
    c.E2 = reinterpret_cast<float2*>(base + kOffE2);
    c.tw = reinterpret_cast<float2*>(base + kOffTw);
    c.ph = reinterpret_cast<float2*>(base + kOffPh);
    c.acc = reinterpret_cast<double*>(base + kOffAcc);
    c.psi = psi;
    c.ex = ex;
    c.ey = ey;

    cudaError_t e = cudaMemsetAsync(c.acc, 0, (size_t)kAccDoubles * sizeof(double), s);
    if (e == cudaSuccess) {
        k_tables<<<(n + 1 + 255) / 256, 256, 0, s>>>(n, c.tw, c.ph);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_rows_fwd(c, s);
    if (e == cudaSuccess) e = launch_cols_spectral(c, s);
    if (e == cudaSuccess) e = launch_rows_inv(c, s);
    if (e == cudaSuccess) e = launch_rows_psi(c, s);
    if (e == cudaSuccess) e = launch_split_field(c, s);
    if (e == cudaSuccess && N) {
        double acc[kAccDoubles];
        e = cudaMemcpyAsync(acc, c.acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            double t = 0.0;
            for (int k = 0; k < kAccStripes; ++k) t += acc[k * kAccStride + ACC_N];
            *N = 0.5 * (Lx / n) * (Ly / n) * t;
        }
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("fftpl_solve_noalloc: ") + cudaGetErrorString(e));
        return FFTPL_ECUDA;
    }
    return FFTPL_OK;
}
