// Placement-loop control scalars (Algorithm 1 with a Nesterov step; the
// parameter control of Section IV-A), kept in FP64 in device memory and
// updated by the last CTA of the kernel that produces their inputs (a CTA
// learns it is last from an atomic ticket after a memory fence; nothing
// waits, so no kernel can hang on it).
#pragma once

#include "fftpl_internal.cuh"

namespace fftpl {

enum {
    C_LAMBDA = 0, C_GAMMA, C_ALPHA, C_ALPHA_MAX, C_A, C_BETA, C_HP_PREV, C_K, C_DONE, C_A_NEXT,
    C_ALPHA_MAX0, C_DW_REF, C_GAMMA_FIXED, C_LAMBDA0_OPT, C_STOP_ON_TAU, C_TAU_STOP, C_WB,
    C_HALF_AB, C_MOV_AREA, C_REC_CAP, C_REC_BASE,
    // conjugate-gradient loop: |g_{k-1}|^2, f_k, slope along d/|d|_inf,
    // |d|_inf, restart flag, and the values recorded for iteration k
    C_GG_PREV, C_FK, C_SLOPE, C_DINF, C_RESTART, C_W_K, C_HP_K, C_N_K, C_TAU_K,
    C_ALPHA_CAP,   // ceiling of alpha_max in the Nesterov loop (0: none)
    // float32 copies of the values the per-element kernels read (F_*),
    // packed two to a slot
    C_FMIRROR, C_FMIRROR_LAST = C_FMIRROR + 4,
    C_COUNT
};

// The per-element kernels read their control values as float32 from this
// mirror, written by whichever thread last changed the FP64 scalars (the
// FP64 pipe of the GPU is narrow: a double compare, conversion or division
// per thread costs more than the kernel's own arithmetic).  The values are
// those the kernels computed before from the FP64 scalars.
enum {
    F_DONE = 0, F_FIRST, F_LAMBDA, F_ALPHA, F_BETA, F_RESTART, F_SCALE_TRIAL, F_SCALE_UPDATE,
    F_INV_G, F_L2G,   // 1/gamma and log2(e)/gamma (adjacent: one 8-byte load)
    F_COUNT
};
static_assert(F_COUNT <= 2 * (C_FMIRROR_LAST - C_FMIRROR + 1), "control mirror too small");
static_assert(F_INV_G % 2 == 0, "1/gamma and log2(e)/gamma share an 8-byte word");

__host__ __device__ inline float* ctrl_f(double* ctrl) {
    return reinterpret_cast<float*>(ctrl + C_FMIRROR);
}
__host__ __device__ inline const float* ctrl_f(const double* ctrl) {
    return reinterpret_cast<const float*>(ctrl + C_FMIRROR);
}

__host__ __device__ inline void ctrl_mirror(double* ctrl) {
    float* f = ctrl_f(ctrl);
    f[F_DONE] = ctrl[C_DONE] != 0.0 ? 1.0f : 0.0f;
    f[F_FIRST] = ctrl[C_K] == 0.0 ? 1.0f : 0.0f;
    f[F_LAMBDA] = (float)ctrl[C_LAMBDA];
    f[F_ALPHA] = (float)ctrl[C_ALPHA];
    f[F_BETA] = (float)ctrl[C_BETA];
    f[F_RESTART] = ctrl[C_RESTART] != 0.0 ? 1.0f : 0.0f;
    const double dinf = ctrl[C_DINF];
    f[F_SCALE_TRIAL] = dinf > 0.0 ? (float)(ctrl[C_ALPHA_MAX] / dinf) : 0.0f;
    f[F_SCALE_UPDATE] = dinf > 0.0 ? (float)(ctrl[C_ALPHA] / dinf) : 0.0f;
    const float g = (float)ctrl[C_GAMMA];
    if (g > 0.0f) wa_scale(g, &f[F_INV_G], &f[F_L2G]);
}
constexpr int kRecFields = 8;
constexpr int kCounters = 4;   // one ticket counter per loop kernel kind

// After a block barrier (which orders every thread's earlier reductions
// before thread 0's next operations), thread 0 fences at device scope and
// takes a ticket; the CTA that draws the last ticket resets the counter,
// fences again (its later reads see every CTA's reductions) and returns
// true.  One fence per block: a fence in every thread held each thread
// until its own stores had completed, which doubled the loop's vector
// kernels.
__device__ __forceinline__ bool last_cta(unsigned int* counter) {
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) {
            *counter = 0u;
            __threadfence();
        }
    }
    __syncthreads();
    return is_last;
}

// totals of the striped accumulators (read past L1)
__device__ __forceinline__ double acc_sum(const double* acc, int q) {
    double s = 0.0;
    for (int k = 0; k < kAccStripes; ++k) s += __ldcg(acc + k * kAccStride + q);
    return s;
}
__device__ __forceinline__ double acc_max(const double* acc, int q) {
    double s = 0.0;
    for (int k = 0; k < kAccStripes; ++k) s = fmax(s, __ldcg(acc + k * kAccStride + q));
    return s;
}

// After the cell kernel: lambda_k.  lambda_0 = ||grad W~||_1 / ||grad N||_1
// unless given; for k >= 1 lambda_k = mu_k lambda_{k-1} with
// mu_k = 1.1^(-dW/dW_ref + 1) bounded to [0.75, 1.1], dW the HPWL change.
__device__ __forceinline__ void ctrl_lambda(double* ctrl, const double* acc) {
    int k = (int)ctrl[C_K];
    double hp = acc_sum(acc, ACC_HPWL);
    double lam = ctrl[C_LAMBDA];
    if (k == 0 && ctrl[C_LAMBDA0_OPT] <= 0.0) {
        double gn = acc_sum(acc, ACC_GN_L1), gw = acc_sum(acc, ACC_GW_L1);
        lam = gn > 0.0 ? gw / gn : 1.0;
    }
    if (k >= 1) {
        double mu = pow(1.1, -(hp - ctrl[C_HP_PREV]) / ctrl[C_DW_REF] + 1.0);
        lam *= fmin(1.1, fmax(0.75, mu));
    }
    ctrl[C_HP_PREV] = hp;
    ctrl[C_LAMBDA] = lam;
    ctrl_mirror(ctrl);
}

// After the combined gradient: the step alpha_k and the momentum weight.
// alpha_0 = alpha_max_0 / ||g||_inf; alpha_k = ||v_k - v_{k-1}|| / ||g_k - g_{k-1}||;
// alpha_k ||g||_inf is then kept within [0.01 alpha_max_k, alpha_max_k].
__device__ __forceinline__ void ctrl_alpha(double* ctrl, const double* acc) {
    int k = (int)ctrl[C_K];
    double ginf = acc_max(acc, ACC_GINF);
    double alpha = ctrl[C_ALPHA], amax = ctrl[C_ALPHA_MAX];
    if (k == 0) {
        alpha = ginf > 0.0 ? ctrl[C_ALPHA_MAX0] / ginf : 0.0;
    } else {
        double dg2 = acc_sum(acc, ACC_DG2), dv2 = acc_sum(acc, ACC_DV2);
        if (dg2 > 0.0) alpha = sqrt(dv2) / sqrt(dg2);
    }
    if (ginf > 0.0) {
        if (alpha * ginf > amax) alpha = amax / ginf;
        if (alpha * ginf < 0.01 * amax) alpha = 0.01 * amax / ginf;
    }
    double a = ctrl[C_A];
    double an = 0.5 * (1.0 + sqrt(1.0 + 4.0 * a * a));
    ctrl[C_ALPHA] = alpha;
    ctrl[C_A_NEXT] = an;
    ctrl[C_BETA] = (a - 1.0) / an;
    ctrl_mirror(ctrl);
}

// gamma = 8.0 w_b 10^((20/9)(tau - 0.1) - 1) (Section IV-A).
__device__ __forceinline__ double gamma_schedule(double tau, double wb) {
    return 8.0 * wb * pow(10.0, (20.0 / 9.0) * (tau - 0.1) - 1.0);
}

// After the position update: record iteration k, then alpha_max_{k+1},
// gamma_{k+1}, k+1 and the stop test tau <= tau_stop.  Adaptive restart
// (the gradient test of O'Donoghue and Candes, 2015), one iteration late:
// when g_k . (u_{k+1} - u_k) > 0 the momentum sequence starts over,
// a_{k+1} = 1, so that the next momentum weight is 0.  alpha_max_{k+1} is
// kept at or below the handle's ceiling (alpha_max_cap_bins bin widths).
__device__ __forceinline__ void ctrl_record(double* ctrl, const double* acc, double* recs) {
    int k = (int)ctrl[C_K];
    double tau = acc_sum(acc, ACC_TAU) / ctrl[C_MOV_AREA];
    double step_max = acc_max(acc, ACC_STEPMAX);
    int slot = k - (int)ctrl[C_REC_BASE];
    if (slot >= 0 && slot < (int)ctrl[C_REC_CAP]) {
        double* r = recs + (size_t)slot * kRecFields;
        r[0] = acc_sum(acc, ACC_W);
        r[1] = acc_sum(acc, ACC_HPWL);
        r[2] = acc_sum(acc, ACC_N) * ctrl[C_HALF_AB];
        r[3] = tau;
        r[4] = ctrl[C_LAMBDA];
        r[5] = ctrl[C_GAMMA];
        r[6] = ctrl[C_ALPHA];
        r[7] = step_max;
    }
    ctrl[C_A] = acc_sum(acc, ACC_GD) > 0.0 ? 1.0 : ctrl[C_A_NEXT];
    double amax = fmax(ctrl[C_ALPHA_MAX0], 2.0 * step_max);
    if (ctrl[C_ALPHA_CAP] > 0.0) amax = fmin(amax, fmax(ctrl[C_ALPHA_CAP], ctrl[C_ALPHA_MAX0]));
    ctrl[C_ALPHA_MAX] = amax;
    if (ctrl[C_GAMMA_FIXED] <= 0.0) ctrl[C_GAMMA] = gamma_schedule(tau, ctrl[C_WB]);
    ctrl[C_K] = (double)(k + 1);
    if (ctrl[C_STOP_ON_TAU] != 0.0 && tau <= ctrl[C_TAU_STOP]) ctrl[C_DONE] = 1.0;
    ctrl_mirror(ctrl);
}

// ------------------------------------------------ conjugate-gradient loop
// Algorithm 1's CGsolver with the search interval [0.01 a_max, a_max] of
// Section IV-A: Polak-Ribiere+ directions, the step measured as the farthest
// cell move (direction scaled by 1/|d|_inf), one quadratic-fit line search
// from f_k, the slope and one trial evaluation at a_max.

// After g_k: beta_k (PR+), f_k and the values recorded for iteration k.
__device__ __forceinline__ void ctrl_cg_g(double* ctrl, const double* acc) {
    int k = (int)ctrl[C_K];
    double gg = acc_sum(acc, ACC_DG2), ggp = acc_sum(acc, ACC_DV2);
    double prev = ctrl[C_GG_PREV];
    ctrl[C_BETA] = (k > 0 && prev > 0.0) ? fmax(0.0, (gg - ggp) / prev) : 0.0;
    ctrl[C_GG_PREV] = gg;
    double W = acc_sum(acc, ACC_W), N = acc_sum(acc, ACC_N) * ctrl[C_HALF_AB];
    ctrl[C_FK] = W + ctrl[C_LAMBDA] * N;
    ctrl[C_W_K] = W;
    ctrl[C_HP_K] = acc_sum(acc, ACC_HPWL);
    ctrl[C_N_K] = N;
    ctrl[C_TAU_K] = acc_sum(acc, ACC_TAU) / ctrl[C_MOV_AREA];
    ctrl_mirror(ctrl);
}

// After d_k: restart to -g_k unless g_k . d_k < 0; |d|_inf and the slope.
__device__ __forceinline__ void ctrl_cg_dir(double* ctrl, const double* acc) {
    double gd = acc_sum(acc, ACC_GD), dinf = acc_max(acc, ACC_DINF);
    bool restart = !(gd < 0.0);
    if (restart) {
        dinf = acc_max(acc, ACC_GINF);
        gd = -ctrl[C_GG_PREV];
    }
    ctrl[C_RESTART] = restart ? 1.0 : 0.0;
    ctrl[C_DINF] = dinf;
    ctrl[C_SLOPE] = dinf > 0.0 ? gd / dinf : 0.0;
    ctrl_mirror(ctrl);
}

// After the trial evaluation at a_max: the step a_k from the parabola
// through f_k (slope s) and f_t, kept in [0.01 a_max, a_max].
__device__ __forceinline__ void ctrl_cg_alpha(double* ctrl, const double* acc) {
    double amax = ctrl[C_ALPHA_MAX], alpha = 0.0;
    if (ctrl[C_DINF] > 0.0) {
        double ft = acc_sum(acc, ACC_W) + ctrl[C_LAMBDA] * acc_sum(acc, ACC_N) * ctrl[C_HALF_AB];
        double s = ctrl[C_SLOPE];
        double c = (ft - ctrl[C_FK] - s * amax) / (amax * amax);
        double as = c > 0.0 ? -s / (2.0 * c) : amax;
        alpha = fmin(amax, fmax(0.01 * amax, as));
    }
    ctrl[C_ALPHA] = alpha;
    ctrl_mirror(ctrl);
}

// After the position update: record iteration k, then a_max_{k+1} =
// max(a_max_0, 2 a_k), gamma_{k+1}, k+1 and the stop test.
__device__ __forceinline__ void ctrl_record_cg(double* ctrl, double* recs) {
    int k = (int)ctrl[C_K];
    double tau = ctrl[C_TAU_K], alpha = ctrl[C_ALPHA];
    int slot = k - (int)ctrl[C_REC_BASE];
    if (slot >= 0 && slot < (int)ctrl[C_REC_CAP]) {
        double* r = recs + (size_t)slot * kRecFields;
        r[0] = ctrl[C_W_K];
        r[1] = ctrl[C_HP_K];
        r[2] = ctrl[C_N_K];
        r[3] = tau;
        r[4] = ctrl[C_LAMBDA];
        r[5] = ctrl[C_GAMMA];
        r[6] = alpha;
        r[7] = alpha;
    }
    ctrl[C_ALPHA_MAX] = fmax(ctrl[C_ALPHA_MAX0], 2.0 * alpha);
    if (ctrl[C_GAMMA_FIXED] <= 0.0) ctrl[C_GAMMA] = gamma_schedule(tau, ctrl[C_WB]);
    ctrl[C_K] = (double)(k + 1);
    if (ctrl[C_STOP_ON_TAU] != 0.0 && tau <= ctrl[C_TAU_STOP]) ctrl[C_DONE] = 1.0;
    ctrl_mirror(ctrl);
}

}  // namespace fftpl
