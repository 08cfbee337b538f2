/*
 * fftpl.h -- C ABI of the GB300 FFTPL objective-gradient library (libfftpl.so).
 *
 * The library evaluates, on one GPU, the per-iteration objective and gradient
 * of the FFTPL electrostatic placement method (Lu et al., "FFTPL: An Analytic
 * Placement Algorithm Using Fast Fourier Transform for Density Equalization"):
 *
 *   f(v) = W~(v) + lambda N(v)                                   (Eq. 7)
 *
 * with W~ the weighted-average wirelength (Eq. 3) and N the electrostatic
 * potential energy (Eq. 6) of the bin density rho.  The potential psi and the
 * field E solve Poisson's equation with Neumann boundary (Eq. 8) through the
 * cosine/sine series of Eqs. 9-12.  fftpl_step runs Algorithm 1's loop with
 * the parameter control of Section IV-A and either the paper's
 * conjugate-gradient step or Nesterov's method (fftpl_options.optimizer);
 * LSE wirelength and the Helmholtz smoothing of Eq. 4 are model options.
 *
 * Conventions (they define the results; the oracle used by the tests states
 * the same):
 *   - Region R = [x0, x1] x [y0, y1] split into n x n bins (Section II);
 *     bin (j, k) is row j (y) and column k (x); all maps are float32 row-major
 *     [n][n] with x fastest.  Bins are half-open [e_k, e_k+1) with
 *     e_k = x0 + k (x1 - x0) / n; every edge must be exact in float32.
 *   - Cells are given by centre (x, y) and size (w, h); the edges used are
 *     fl32(x -/+ w/2).  Charge q_i = w_i h_i (Section III).  Fixed cells
 *     (macros) enter rho scaled by the target density (Section III-B).
 *   - rho_b = (rho_t F_b + D_b) / A_b with D_b, F_b the movable and fixed
 *     overlap areas.  Coefficients a_vu = eps_u eps_v / n^2 sum rho cos cos
 *     (bin-centre DCT-II), w_u = pi u / (x1 - x0), w_v = pi v / (y1 - y0),
 *     the (0,0) mode dropped (DC removal, Section III-A).
 *   - N = 1/2 sum_b A_b rho_b psi_b; the density gradient is
 *     dN/dx_i = -sum_b ov(i,b) E_x[b] (the q.E of Eq. 7).
 *   - Pin coordinate = fl32(cell centre + pin offset); W~ is Eq. 3 per net and
 *     axis, summed over nets (weight 1); degree-1 nets contribute 0.
 *   - HPWL is Eq. 1 on pin coordinates.  Overflow
 *     tau = sum_b max(0, D_b - rho_t (A_b - F_b)) / sum_i q_i.
 *
 * Memory and ownership: fftpl_create deep-copies every host array it is given
 * into device memory owned by the handle.  Position and gradient arguments of
 * the evaluation calls are caller-owned DEVICE pointers (float32, contiguous,
 * m_mov entries) unless the name ends in _host.  Returned map views are
 * borrowed device pointers, valid until the next call on the handle.
 *
 * Streams: every call enqueues its work on the stream given to fftpl_create
 * and, where it says so, synchronises it.  With NULL the handle creates a
 * blocking stream of its own, which the legacy default stream orders with
 * implicitly.  A handle is not thread-safe; use one handle per host thread.
 *
 * Errors: every call returns fftpl_status and never throws.  FFTPL_EINVAL
 * comes from host-side validation before any device work is queued.  The
 * text of the last error is fftpl_last_error(handle) (or
 * fftpl_last_error(NULL) for a failed fftpl_create).  Kernels that wait
 * (bounded spin-waits only) record a device error word instead of trapping;
 * fftpl_check reads it as FFTPL_ETIMEOUT / FFTPL_ECUDA.
 */
#ifndef FFTPL_H
#define FFTPL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FFTPL_VERSION 100
#define FFTPL_MIN_N 16
#define FFTPL_MAX_N 4096

typedef struct fftpl_ctx* fftpl_t; /* opaque, library-owned */

typedef enum {
    FFTPL_OK = 0,
    FFTPL_EINVAL = 1,      /* invalid argument (host-side validation) */
    FFTPL_ENOMEM = 2,      /* device or host allocation failed */
    FFTPL_ECUDA = 3,       /* CUDA runtime or kernel error */
    FFTPL_ETIMEOUT = 4,    /* a bounded device wait gave up */
    FFTPL_ESTATE = 5,      /* call not valid in the handle's state */
    FFTPL_EUNSUPPORTED = 6 /* option not available in this build */
} fftpl_status;

/* Placement region R (Section II); bounding box of the placeable area. */
typedef struct { double x0, y0, x1, y1; } fftpl_region;

/* Cells (Section II: movable V_m first, then fixed V_f).  Host arrays.
 *   w, h:          m_mov + m_fix sizes (> 0, finite)
 *   fix_x, fix_y:  m_fix centres of the fixed cells (may be NULL if m_fix 0) */
typedef struct {
    int32_t m_mov, m_fix;
    const float* w;
    const float* h;
    const float* fix_x;
    const float* fix_y;
} fftpl_cells;

/* Nets as CSR over pins: net e owns pins [net_ptr[e], net_ptr[e+1]).
 * Host array of E + 1 non-decreasing entries, net_ptr[0] = 0. */
typedef struct {
    int32_t E;
    const int32_t* net_ptr;
} fftpl_nets;

/* Pins (host arrays of P entries): pin_cell in [0, m_mov + m_fix) (an index
 * >= m_mov names fixed cell pin_cell - m_mov); dx, dy offsets from the cell
 * centre. */
typedef struct {
    int64_t P;
    const int32_t* pin_cell;
    const float* dx;
    const float* dy;
} fftpl_pins;

/* Spectral solve paths for Eqs. 9-12 (Section III-E names the transform;
 * both paths compute the same bin-centre cosine/sine sums).
 * FFTPL_SOLVE_TC_BF16X3 evaluates them as five dense products with the n x n
 * cosine and sine matrices on the tcgen05 tensor cores: every float32
 * operand x is split into bf16 x_hi + x_lo and each product sums
 * hi*hi + hi*lo + lo*hi in float32 (relative error about 1e-5 per product,
 * against 1e-7 for the FFT path).  It costs 42 n^3 flops per solve (the FFT
 * path O(n^2 log n)), needs n >= FFTPL_TC_MIN_N, and holds 36 n^2 extra
 * bytes of device memory (bf16 tables and intermediates).
 * FFTPL_SOLVE_TC_RADIX keeps the transform path's passes (Makhoul's
 * reordering of each cosine or sine transform into a complex DFT of length
 * n, two real rows per DFT) and computes every DFT on the tensor cores as two
 * small dense products of a four-step factorisation n = 64 n2: 64-point
 * DFTs (a 128 x 128 real block), twiddles exp(-+2 pi i j2 k1 / n) in that
 * product's epilogue, then n2-point DFTs (block-diagonal over 64 / n2 rows),
 * with the same bf16 x 3 split and FP32 accumulation: 3072 R n flops for
 * the DFTs of R rows (6.4 GFLOP for the n / 2 rows of one pass at n = 2048)
 * instead of the dense form's O(n^3).  Needs n >= 256 and
 * holds 48 n^2 extra bytes of device memory. */
enum {
    FFTPL_SOLVE_FFT = 0,       /* real-to-real transforms built on FP32 FFTs */
    FFTPL_SOLVE_TC_BF16X3 = 1, /* dense DCT matrices on tcgen05 tensor cores,
                                  operands split into bf16 hi+lo, 3 products,
                                  FP32 accumulation */
    FFTPL_SOLVE_TC_RADIX = 2   /* the transform path's DFTs as radix-64 x n/64
                                  products on tcgen05 tensor cores, bf16 x 3 */
};
#define FFTPL_TC_MIN_N 128
#define FFTPL_TCR_MIN_N 256

/* Wirelength models.  FFTPL_WL_WA: the weighted average of Eq. 3.
 * FFTPL_WL_LSE: the log-sum-exp model Section II names, per net and axis
 * g ln sum exp(p/g) + g ln sum exp(-p/g), with gradient
 * softmax(p/g) - softmax(-p/g). */
enum { FFTPL_WL_WA = 0, FFTPL_WL_LSE = 1 };

/* Placement-loop step (fftpl_step).  FFTPL_OPT_NESTEROV: Nesterov's method
 * with the step alpha_k = |v_k - v_{k-1}| / |g_k - g_{k-1}| kept in the
 * interval [0.01 alpha_max, alpha_max] of Section IV-A.  FFTPL_OPT_CG: the
 * nonlinear conjugate-gradient step of Algorithm 1 (Polak-Ribiere+
 * direction d, restarted to -g when not a descent direction; the step a is
 * the farthest cell move, x + a d / |d|_inf, chosen in the same interval by
 * one quadratic fit through f(x), the slope and a trial evaluation at
 * alpha_max; then alpha_max = max(alpha_max_0, 2 a)).  One CG iteration
 * costs two evaluations. */
enum { FFTPL_OPT_NESTEROV = 0, FFTPL_OPT_CG = 1 };

typedef struct {
    double target_density;  /* rho_t (Section III-B, Section V: 1.0) */
    int32_t solve_path;     /* FFTPL_SOLVE_* */
    int32_t deterministic;  /* 1: int64 fixed-point density (ov rounded to
                               float32 then to units of 2^-32) and an
                               atomic-free pin-to-cell reduction, so results
                               do not depend on scheduling */
    /* placement loop (Section IV-A constants) */
    double lambda0;         /* <= 0: ||grad W~||_1 / ||grad N||_1 at start */
    double gamma_fixed;     /* > 0: fixed WA gamma; <= 0: gamma(tau) schedule */
    double dw_ref;          /* reference HPWL variation, 3.5e5 */
    double alpha_max0_bins; /* initial step bound in bin widths, 0.044 */
    double tau_stop;        /* stop threshold for the overflow, 0.1 */
    int32_t stop_on_tau;    /* 1: fftpl_step stops when tau <= tau_stop */
    int32_t use_graphs;     /* 1: replay captured CUDA graphs for repeated
                               evaluations with the same buffers and for
                               the iterations of fftpl_step */
    int32_t wirelength;     /* FFTPL_WL_WA (default) or FFTPL_WL_LSE */
    int32_t optimizer;      /* FFTPL_OPT_NESTEROV (default) or FFTPL_OPT_CG */
    double helmholtz_eps;   /* 0: the Poisson equation of Eq. 8 (the (0,0)
                               mode dropped); > 0: the Helmholtz smoothing of
                               Eq. 4, laplacian psi - eps psi = -rho: every
                               mode divided by w_u^2 + w_v^2 + eps and the
                               (0,0) mode kept as a_00 / eps (placement
                               units^-2; finite, >= 0, else FFTPL_EINVAL) */
    double alpha_max_cap_bins; /* Nesterov loop: the step bound alpha_max never
                               exceeds this many bin widths (> 0; 0: no
                               bound; default 16).  The rule alpha_max =
                               max(alpha_max_0, 2 a) of Section IV-A was
                               made for the paper's line search; the
                               Barzilai-Borwein steps have none, and without
                               a ceiling their largest moves doubled up to
                               the region's size on the 210K- and 2.2M-cell
                               instances */
} fftpl_options;

/* FP64 scalars of one evaluation. */
typedef struct {
    double N;              /* energy, 1/2 sum A_b rho_b psi_b (Eq. 6) */
    double W;              /* weighted-average wirelength (Eq. 3) */
    double hpwl;           /* Eq. 1 */
    double tau;            /* density overflow */
    double gN_l1, gW_l1;   /* ||grad N||_1, ||grad W~||_1 over movable cells */
    double charge;         /* sum_b A_b rho_b (in-region charge incl. rho_t F) */
    double mov_area;       /* sum_i q_i of movable cells */
} fftpl_eval_report;

/* One iteration of fftpl_step (values at the evaluated point v_k). */
typedef struct {
    double W, hpwl, N, tau, lambda, gamma, alpha, step_max;
} fftpl_iter_record;

/* ---------------------------------------------------------------- setup */

int32_t fftpl_version(void);
void fftpl_default_options(fftpl_options* opt);

/* Creates a handle for one placement instance (Section II: G = (V, E, R),
 * n x n bins).  n is a power of two in [FFTPL_MIN_N, FFTPL_MAX_N]; every bin
 * edge must be exact in float32; all sizes > 0 and finite; pin_cell in range;
 * net_ptr valid CSR.  Builds on the device: the fixed-cell map rho_t F
 * (Section III-B), transform tables, and the pin layouts.  cuda_stream is a
 * cudaStream_t (NULL: default stream).  On failure *out is NULL and nothing
 * is leaked. */
fftpl_status fftpl_create(const fftpl_region* region, int32_t n, const fftpl_cells* cells,
                          const fftpl_nets* nets, const fftpl_pins* pins,
                          const fftpl_options* opt, void* cuda_stream, fftpl_t* out);

/* Frees every device and host resource of the handle (NULL is a no-op). */
void fftpl_destroy(fftpl_t h);

/* Text of the last error on the handle (NULL: of the last failed create on
 * this thread).  Owned by the library. */
const char* fftpl_last_error(fftpl_t h);

/* Synchronises the handle's stream and reads the device error word. */
fftpl_status fftpl_check(fftpl_t h);

/* Device memory the handle holds, in bytes. */
size_t fftpl_device_bytes(fftpl_t h);

/* ----------------------------------------------------- evaluation calls */

/* Density energy and gradient (Section III; Algorithm 1 "compute density",
 * "FFTsolver" and the density part of the gradient): scatter, spectral
 * solve, gather.  x, y: device positions (m_mov).  gx, gy: device outputs
 * dN/dx, dN/dy (m_mov), may be NULL.  N: host output; if non-NULL the call
 * synchronises, otherwise it stays asynchronous (read with fftpl_report). */
fftpl_status fftpl_density(fftpl_t h, const float* x, const float* y, double* N,
                           float* gx, float* gy);

/* As fftpl_density, but the gradient is the exact derivative of the binned
 * energy (edge difference of psi: d ov(i,b)/dx is +1 at the bin holding the
 * right edge and -1 at the bin holding the left edge, times the row overlap)
 * instead of the paper's q.E gather. */
fftpl_status fftpl_density_adjoint(fftpl_t h, const float* x, const float* y, double* N,
                                   float* gx, float* gy);

/* The two halves of fftpl_density, for callers that differentiate N
 * themselves (an autograd backward).  fftpl_energy: scatter and spectral
 * solve only (Section III: density, Eqs. 9-12), energy N to *N (host; the
 * call synchronises when N is non-NULL).  fftpl_gather: the density
 * gradient at (x, y) from the maps of the last density evaluation on this
 * handle (FFTPL_ESTATE if there is none): mode 0 the field gather
 * -sum_b ov(i,b) E_b (q.E of Eq. 7), mode 1 the exact derivative of the
 * binned N (as fftpl_density_adjoint).  x, y must be the positions that
 * evaluation used. */
fftpl_status fftpl_energy(fftpl_t h, const float* x, const float* y, double* N);
fftpl_status fftpl_gather(fftpl_t h, const float* x, const float* y, int32_t mode, float* gx,
                          float* gy);

/* Weighted-average wirelength (Eq. 3) and its gradient; HPWL (Eq. 1) as a
 * by-product.  gx, gy device outputs (m_mov), may be NULL.  W host output:
 * non-NULL synchronises. */
fftpl_status fftpl_wa(fftpl_t h, const float* x, const float* y, float gamma, double* W,
                      float* gx, float* gy);

/* One full objective-gradient evaluation: density energy and gradient, WA
 * wirelength and gradient (the two run concurrently on the device), and the
 * FP64 sums of fftpl_eval_report.  Outputs are device arrays (any may be
 * NULL).  rep: host; non-NULL synchronises. */
fftpl_status fftpl_eval(fftpl_t h, const float* x, const float* y, float gamma,
                        float* gNx, float* gNy, float* gWx, float* gWy,
                        fftpl_eval_report* rep);

/* fftpl_eval on HOST buffers (m_mov floats each; gradient outputs may be
 * NULL), synchronising before it returns.  When all six are pinned
 * (page-locked, device-mapped) host memory the kernels read x, y and write
 * the gradients over the host link themselves, overlapping the transfers
 * with the computation (the scatter reads the positions once and keeps a
 * device copy for the later kernels; the wirelength gradient is written
 * while the transforms still run); otherwise the call copies x, y in,
 * evaluates and copies the gradients out.  Results are the same either way
 * (bit-identical in deterministic mode). */
fftpl_status fftpl_eval_host(fftpl_t h, const float* x_host, const float* y_host, float gamma,
                             float* gNx_host, float* gNy_host, float* gWx_host,
                             float* gWy_host, fftpl_eval_report* rep);

/* Synchronises and returns the scalars of the last evaluation call. */
fftpl_status fftpl_report(fftpl_t h, fftpl_eval_report* rep);

/* Borrowed device views of the maps of the last density evaluation: bin
 * density rho, potential psi (Eq. 11), field E_x, E_y (Eq. 12).  Any pointer
 * may be NULL.  rho is formed on demand. */
fftpl_status fftpl_fields(fftpl_t h, const float** rho, const float** psi,
                          const float** ex, const float** ey);

/* Movable-cell area map of the last density call in deterministic mode, in
 * int64 units of 2^-32 (borrowed device view); FFTPL_ESTATE otherwise. */
fftpl_status fftpl_fields_q(fftpl_t h, const int64_t** movable_area_q);

/* Bin bookkeeping: for each movable cell the clamped bin range
 * (ilo, ihi, jlo, jhi) into ranges (device, 4 m_mov int32; empty: ilo > ihi)
 * and the total number of (cell, bin) pairs into *pairs (host; syncs). */
fftpl_status fftpl_bin_ranges(fftpl_t h, const float* x, const float* y, int32_t* ranges,
                              int64_t* pairs);

/* Filler cells (Section III-B: disconnected movable cells that take up the
 * free area).  The paper gives no count or size; this library's rule: the
 * fillers' total area is target_density times the free area of the region
 * (its area minus the fixed cells' overlap with it) minus the movable area;
 * each filler has the mean movable width and height (float32); *count is
 * that area over one filler's, rounded down, 0 when the movable cells
 * already fill it.  Host only (no device work, no handle): the caller
 * appends the fillers as pin-less movable cells (any start positions) to the
 * cells it passes to fftpl_create.  Dark nodes (non-placeable rectangles)
 * are fixed cells.  cells: as for fftpl_create (host arrays).  FFTPL_EINVAL
 * for null arguments or sizes that are not finite and > 0. */
fftpl_status fftpl_fillers(const fftpl_region* region, const fftpl_cells* cells,
                           double target_density, int64_t* count, float* filler_w,
                           float* filler_h);

/* ------------------------------------------------------ placement loop */

/* Starts a placement run at (x0, y0) (device, m_mov): u = v = clamp(x0),
 * Nesterov a = 1 / no CG direction yet, lambda, gamma and alpha_max from the
 * options.  FFTPL_EINVAL when the instance has no movable cells. */
fftpl_status fftpl_place_init(fftpl_t h, const float* x0, const float* y0);

/* Runs up to iters iterations of the loop (Algorithm 1 with the step of
 * fftpl_options.optimizer; Section IV-A control).  recs: host array of iters
 * records (may be NULL).  *ran: iterations done (host).  Synchronises at the
 * end, and with stop_on_tau also every 16 iterations to stop enqueuing once
 * the device has met the stop test. */
fftpl_status fftpl_step(fftpl_t h, int32_t iters, fftpl_iter_record* recs, int32_t* ran);

/* Copies the current major iterate u to device arrays x, y (m_mov). */
fftpl_status fftpl_place_positions(fftpl_t h, float* x, float* y);

/* Serialises the loop state (positions, Nesterov state, lambda, gamma,
 * alpha_max, k) to host memory.  With buf NULL, *bytes receives the size. */
fftpl_status fftpl_state_save(fftpl_t h, void* buf, size_t* bytes);
fftpl_status fftpl_state_load(fftpl_t h, const void* buf, size_t bytes);

/* --------------------------------------------------------- measurement */

/* Stage timing with CUDA events on the stream each stage runs on.  Stages:
 * 0 scatter, 1 forward rows, 2 spectral columns, 3 inverse rows, 4 WA,
 * 5 cells (gather + pin sums), 6 step.  Times accumulate (ms) until reset. */
#define FFTPL_NUM_STAGES 8
fftpl_status fftpl_set_profiling(fftpl_t h, int32_t on);
fftpl_status fftpl_stage_times(fftpl_t h, double* ms, int64_t* launches, int32_t reset);

/* Number of kernels this handle has launched (all stages). */
int64_t fftpl_launch_count(fftpl_t h);

/* ------------------------------------------------------------ serving */

/* A stream of placement jobs served with continuous batching (build system
 * pattern; the paper places one design at a time).  Each job is one
 * instance plus start positions and an iteration count; it runs Algorithm 1
 * with the Nesterov step (as fftpl_step), each iteration replayed from the
 * job's captured loop graph on the job's own stream, so that jobs of
 * different sizes run concurrently on the device.  fftpl_server_tick never
 * waits for the device: it admits queued jobs in arrival order while their
 * estimated device memory fits the budget and a slot is free (their handles
 * are then created by worker threads), launches the next iters_per_tick
 * iterations of every active job whose previous ones have completed (polled
 * with events: no job waits for another), and hands finished jobs to the
 * workers, which copy the final positions to the host and return the
 * device memory to the library's stream-ordered pool without synchronising
 * the device.  Jobs that arrive while others run join at the next tick.
 * With dry_run the server executes nothing on a GPU: each launch completes
 * at once and only advances the job's count (admission, budget and latency
 * bookkeeping can be exercised on any host, with fftpl_server_set_clock). */

typedef struct fftpl_server* fftpl_server_t;

typedef struct {
    size_t hbm_budget_bytes;  /* device memory all active jobs may hold */
    int32_t max_active;       /* at most this many jobs on the device */
    int32_t iters_per_tick;   /* loop iterations per job and tick (>= 1) */
    int32_t deterministic;    /* run every job in deterministic mode */
    int32_t dry_run;          /* bookkeeping only, no device work */
    int32_t workers;          /* threads that create and retire handles (0: 4) */
    int32_t reserved[3];
} fftpl_server_options;

enum { FFTPL_JOB_QUEUED = 0, FFTPL_JOB_ACTIVE = 1, FFTPL_JOB_DONE = 2, FFTPL_JOB_FAILED = 3 };

typedef struct {
    int64_t id;
    int32_t state;           /* FFTPL_JOB_* */
    int32_t iters_done;
    int32_t m_mov, n;
    double t_submit, t_admit, t_done;   /* seconds on the server's clock */
    double hpwl, tau;        /* at the job's last iteration (0 in dry runs) */
    size_t device_bytes;     /* held while active */
} fftpl_job_info;

typedef struct {
    int64_t submitted, completed, failed;
    int32_t active, queued, peak_active;
    size_t peak_device_bytes;
    double wall_s;                       /* first submit to last completion */
    double jobs_per_s;                   /* completed / wall_s */
    double iter_p50_ms, iter_p99_ms;     /* per-iteration latency seen by a job:
                                            time since its previous iterations
                                            completed, per iteration */
    double job_p50_ms, job_p99_ms;       /* submit to completion */
} fftpl_server_stats;

void fftpl_server_default_options(fftpl_server_options* opt);
/* Device-memory estimate of one job, used for admission. */
size_t fftpl_estimate_bytes(int32_t n, int32_t m_mov, int32_t m_fix, int32_t E, int64_t P,
                            int32_t iters, int32_t deterministic);
fftpl_status fftpl_server_create(const fftpl_server_options* opt, fftpl_server_t* out);
void fftpl_server_destroy(fftpl_server_t s);
/* Queues a job; all host arrays are deep-copied (as fftpl_create); x0, y0
 * are host start positions (m_mov).  *id receives the job id. */
fftpl_status fftpl_server_submit(fftpl_server_t s, const fftpl_region* region, int32_t n,
                                 const fftpl_cells* cells, const fftpl_nets* nets,
                                 const fftpl_pins* pins, const fftpl_options* opt,
                                 const float* x0, const float* y0, int32_t iters, int64_t* id);
/* One round of admit / launch / retire; returns without waiting for the
 * device.  *active counts the jobs being created, running or retired. */
fftpl_status fftpl_server_tick(fftpl_server_t s, int32_t* active, int32_t* queued);
/* Job state; x, y (host, m_mov, may be NULL) receive the final positions
 * once the job is done. */
fftpl_status fftpl_server_job(fftpl_server_t s, int64_t id, fftpl_job_info* info, float* x,
                              float* y);
fftpl_status fftpl_server_report(fftpl_server_t s, fftpl_server_stats* out);
/* Uses now_s as the clock from here on (now_s < 0: back to the steady
 * clock). */
fftpl_status fftpl_server_set_clock(fftpl_server_t s, double now_s);

/* --------------------------------------------- allocation-free solve */

/* Largest grid fftpl_solve_noalloc accepts. */
#define FFTPL_NOALLOC_MAX_N 1024

/* Poisson solve of a caller-supplied density map, for callers that cannot
 * allocate device memory themselves: code running where cudaMalloc is not
 * allowed or not wanted (inside a host callback, a real-time or
 * preallocated-memory service, an allocator-less plugin host), or where an
 * allocation could fail or stall mid-run.  The paper has no counterpart: it
 * is the same spectral solve as the density path, offered without a handle.
 *
 * rho: device, n*n float32 bin densities, row-major [y][x].  psi, ex, ey:
 * device outputs of the same layout: the potential psi and the field E_x,
 * E_y of the Poisson solve for a region of size Lx x Ly (the mean of rho is
 * dropped).  All four pointers must be 16-byte aligned (the kernels move
 * rows in 16-byte vectors); a misaligned one returns FFTPL_EINVAL.  N: host,
 * may be NULL; if given, the call synchronises the stream and stores
 * 1/2 (Lx Ly / n^2) sum rho psi there, so N must be NULL while the stream
 * is being captured (FFTPL_EINVAL otherwise).  n: power of two in [16,
 * FFTPL_NOALLOC_MAX_N]; any other n returns FFTPL_EINVAL.  stream: a
 * cudaStream_t (NULL: legacy default stream).
 *
 * Memory: the intermediate transforms live in one fixed array in the
 * library's device image (about 20 MiB), which every GPU that loads the
 * library keeps until the process exits; the call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  The first call on a
 * device looks up that array's device address and sets up the kernels for
 * it, so make the first call on each device before any stream capture.
 * Every call shares the array: calls that may overlap on the GPU (different
 * streams, different host threads) race; serialise them, e.g. on one
 * stream. */
fftpl_status fftpl_solve_noalloc(const float* rho, int32_t n, double Lx, double Ly, float* psi,
                                 float* ex, float* ey, double* N, void* stream);

/* ------------------------------------------------------- test hooks */

/* Host-side fault injection: the k-th device allocation from now fails with
 * FFTPL_ENOMEM (k <= 0 disables). */
void fftpl_debug_fail_alloc_after(int32_t k);

/* The tensor-core product behind FFTPL_SOLVE_TC_BF16X3, on its own:
 * d[i][j] = sum_k A[i][k] B[j][k] (float32, row-major [M][N]) where
 * A = a_hi + a_lo ([M][K] bf16 each) and B = b_hi + b_lo ([N][K] bf16 each),
 * all row-major device arrays with 16-byte aligned bases.  nsplit 3 sums
 * hi*hi + hi*lo + lo*hi, nsplit 1 hi*hi only (the lo arrays are then not
 * read but must still be valid).  M and N positive multiples of 128, K of
 * 64; otherwise FFTPL_EINVAL.  err: device int32 that receives bit 1 when a
 * wait inside the kernel gives up (after about one second); no_loads != 0
 * issues no operand loads, so that the kernel's first wait expires and it
 * returns with err set and d unwritten (the timeout path, exercised without
 * any fault).  Asynchronous on stream (a cudaStream_t; NULL: the legacy
 * default stream); allocates no device memory. */
fftpl_status fftpl_debug_tc_gemm(const void* a_hi, const void* a_lo, const void* b_hi,
                                 const void* b_lo, int32_t M, int32_t N, int32_t K, float* d,
                                 int32_t nsplit, int32_t no_loads, int32_t* err, void* stream);

/* Selects how the transform path's row and column passes write their
 * transposed outputs: tma != 0 through the tensor-memory-access unit (the
 * default, when the driver could encode the tensor maps at create), 0 with
 * plain per-thread stores.  Both write the same values; the captured
 * graphs of the handle are dropped so that the next call takes the choice.
 * Returns FFTPL_EINVAL for a null handle, FFTPL_ESTATE if tma != 0 was asked
 * for and the tensor maps are not available. */
fftpl_status fftpl_debug_transpose_stores(fftpl_t h, int32_t tma);

#ifdef __cplusplus
}
#endif

#endif /* FFTPL_H */
