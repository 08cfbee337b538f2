/*
 * FP64 CPU oracle for the FFTPL objective-gradient evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  It shares no code, header,
 * table or helper with the CUDA path; only the tests, the smoke check and the
 * CPU baseline leg of the benchmark may load it.
 *
 * Paper: Lu et al., "FFTPL: An Analytic Placement Algorithm Using Fast Fourier
 * Transform for Density Equalization".  Every function names the section or
 * equation it follows.  Readings of passages that are silent or garbled:
 *   - bins are sampled at their centres, so the cosine basis of Eq. 9 is
 *     cos(pi u (2x+1) / 2n) and the mirror of Section III-E sits on the region
 *     edge (Neumann condition of Eq. 8 holds exactly for the sine field);
 *   - frequencies are in placement units: w_u = pi u / Lx, w_v = pi v / Ly;
 *   - the coefficients of Eq. 10 carry eps_u eps_v / n^2 (eps_0 = 1, else 2),
 *     which makes Eq. 9 reproduce rho exactly; the (0,0) mode is dropped
 *     (DC removal of Section III-A, zero-integral potential of Eq. 8);
 *   - N = 1/2 sum_b A_b rho_b psi_b (Eq. 6 with the pair double count removed),
 *     and the density gradient is -sum_b ov(i,b) E_b (the q.E of Eq. 7 with the
 *     field averaged over the cell's overlap);
 *   - cell edges and pin coordinates are rounded to float32 before use, as the
 *     inputs are float32 arrays: xl = fl32(x - w/2), xh = fl32(x + w/2),
 *     px = fl32(x + dx).  Bins are half-open [e_k, e_k+1).
 *   - the LSE wirelength that Section II names (without a formula) is the
 *     usual g ln sum exp(p/g) + g ln sum exp(-p/g) per axis;
 *   - the Helmholtz smoothing of Eq. 4 is taken with the right-hand side of
 *     Eq. 8 (laplacian psi - eps psi = -rho), so each mode is divided by
 *     w_u^2 + w_v^2 + eps and, for eps > 0, the (0,0) mode is kept (a_00/eps:
 *     the unique solution).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double x0, y0, x1, y1; } orc_region;

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Bin bookkeeping (Section II: region R split into n x n uniform bins)      */
/* ------------------------------------------------------------------------ */

/* Edge k of the grid along one axis: lo + k * (hi - lo) / n, in FP64. */
static double edge(double lo, double hi, int n, int k) {
    return lo + (double)k * ((hi - lo) / (double)n);
}

/* Largest k in [-1, n] with e_k <= t (strict: e_k < t), found by bisection
 * over the exact FP64 edges, so that no division or rounding decides an
 * index.  e_{-1} is taken as -inf. */
static int last_edge_le(double lo, double hi, int n, double t, int strict) {
    int a = -1, b = n; /* invariant: e_a satisfies (or a == -1), answer in [a, b] */
    if (strict ? (edge(lo, hi, n, n) < t) : (edge(lo, hi, n, n) <= t)) return n;
    while (b - a > 1) {
        int c = a + (b - a) / 2;
        double e = edge(lo, hi, n, c);
        if (strict ? (e < t) : (e <= t)) a = c; else b = c;
    }
    return a;
}

/* First bin touched by [a, b): the largest k with e_k <= a; last bin: the
 * largest k with e_k < b.  Returns the unclamped pair. */
static void bin_span(double lo, double hi, int n, double a, double b, int* klo, int* khi) {
    *klo = last_edge_le(lo, hi, n, a, 0);
    *khi = last_edge_le(lo, hi, n, b, 1);
}

/* Clamp a span to the grid [0, n-1].  An empty result has klo > khi. */
static void clamp_span(int n, int* klo, int* khi) {
    if (*klo < 0) *klo = 0;
    if (*khi > n - 1) *khi = n - 1;
}

static void cell_edges(float x, float w, double* lo, double* hi) {
    float h = 0.5f * w;
    volatile float l = x - h;   /* fl32(x - w/2) */
    volatile float r = x + h;   /* fl32(x + w/2) */
    *lo = (double)l;
    *hi = (double)r;
}

/* Bin ranges touched by each cell: out[4i..4i+3] = (ilo, ihi, jlo, jhi),
 * clamped to the grid; a cell that misses the region has ilo > ihi or
 * jlo > jhi.  Returns the number of (cell, bin) pairs. */
int64_t orc_bin_ranges(const orc_region* R, int n, int m, const float* x, const float* y,
                       const float* w, const float* h, int32_t* out) {
    int64_t pairs = 0;
    for (int i = 0; i < m; ++i) {
        double xl, xh, yl, yh;
        int ilo, ihi, jlo, jhi;
        cell_edges(x[i], w[i], &xl, &xh);
        cell_edges(y[i], h[i], &yl, &yh);
        bin_span(R->x0, R->x1, n, xl, xh, &ilo, &ihi);
        bin_span(R->y0, R->y1, n, yl, yh, &jlo, &jhi);
        clamp_span(n, &ilo, &ihi);
        clamp_span(n, &jlo, &jhi);
        if (ilo > ihi || jlo > jhi) { ilo = 0; ihi = -1; jlo = 0; jhi = -1; }
        out[4 * i + 0] = ilo; out[4 * i + 1] = ihi;
        out[4 * i + 2] = jlo; out[4 * i + 3] = jhi;
        if (ilo <= ihi && jlo <= jhi) pairs += (int64_t)(ihi - ilo + 1) * (jhi - jlo + 1);
    }
    return pairs;
}

/* Overlap length of [a, b) with bin k along one axis (FP64, exact for the
 * float32 inputs used here). */
static double ov1(double lo, double hi, int n, int k, double a, double b) {
    double e0 = edge(lo, hi, n, k), e1 = edge(lo, hi, n, k + 1);
    return dmax(0.0, dmin(b, e1) - dmax(a, e0));
}

/* Adds the exact rectangle-bin overlap area of every cell to area[n*n]
 * (row-major, y rows, x fastest).  Section II bin density, Section III cell
 * charge q_i = A_i. */
void orc_overlap_map(const orc_region* R, int n, int m, const float* x, const float* y,
                     const float* w, const float* h, double* area) {
    for (int i = 0; i < m; ++i) {
        double xl, xh, yl, yh;
        int ilo, ihi, jlo, jhi;
        cell_edges(x[i], w[i], &xl, &xh);
        cell_edges(y[i], h[i], &yl, &yh);
        bin_span(R->x0, R->x1, n, xl, xh, &ilo, &ihi);
        bin_span(R->y0, R->y1, n, yl, yh, &jlo, &jhi);
        clamp_span(n, &ilo, &ihi);
        clamp_span(n, &jlo, &jhi);
        for (int j = jlo; j <= jhi; ++j) {
            double oy = ov1(R->y0, R->y1, n, j, yl, yh);
            for (int k = ilo; k <= ihi; ++k) {
                double ox = ov1(R->x0, R->x1, n, k, xl, xh);
                area[(size_t)j * n + k] += ox * oy;
            }
        }
    }
}

/* Deterministic (fixed-point) form of the same map: each pair's overlap is
 * formed in float32 (x and y lengths rounded to float32, then their product
 * rounded to float32) and quantised to round-to-nearest-even units of 2^-32;
 * the bin sums are exact int64.  Fixed-point accumulation is order-free, so
 * any summation order gives the same integers. */
void orc_overlap_map_q(const orc_region* R, int n, int m, const float* x, const float* y,
                       const float* w, const float* h, int64_t* q) {
    for (int i = 0; i < m; ++i) {
        double xl, xh, yl, yh;
        int ilo, ihi, jlo, jhi;
        cell_edges(x[i], w[i], &xl, &xh);
        cell_edges(y[i], h[i], &yl, &yh);
        bin_span(R->x0, R->x1, n, xl, xh, &ilo, &ihi);
        bin_span(R->y0, R->y1, n, yl, yh, &jlo, &jhi);
        clamp_span(n, &ilo, &ihi);
        clamp_span(n, &jlo, &jhi);
        for (int j = jlo; j <= jhi; ++j) {
            float e0 = (float)edge(R->y0, R->y1, n, j), e1 = (float)edge(R->y0, R->y1, n, j + 1);
            volatile float oy = fminf((float)yh, e1) - fmaxf((float)yl, e0);
            if (oy < 0.0f) oy = 0.0f;
            for (int k = ilo; k <= ihi; ++k) {
                float f0 = (float)edge(R->x0, R->x1, n, k), f1 = (float)edge(R->x0, R->x1, n, k + 1);
                volatile float ox = fminf((float)xh, f1) - fmaxf((float)xl, f0);
                if (ox < 0.0f) ox = 0.0f;
                volatile float a = ox * oy;
                double s = (double)a * 4294967296.0; /* exact scaling by 2^32 */
                q[(size_t)j * n + k] += (int64_t)nearbyint(s);
            }
        }
    }
}

/* Bin density (Section II; fixed area scaled by the target density as in
 * Section III-B):  rho_b = (rho_t * F_b + D_b) / A_b  with D_b the movable
 * overlap area and F_b the fixed (macro) overlap area.  mov_area and fix_area
 * (n*n, may be NULL) receive D and F. */
void orc_density(const orc_region* R, int n, double rho_t,
                 int m_mov, const float* x, const float* y, const float* w, const float* h,
                 int m_fix, const float* fx, const float* fy, const float* fw, const float* fh,
                 double* rho, double* mov_area, double* fix_area) {
    size_t nn = (size_t)n * n;
    double* D = (double*)calloc(nn, sizeof(double));
    double* F = (double*)calloc(nn, sizeof(double));
    orc_overlap_map(R, n, m_mov, x, y, w, h, D);
    if (m_fix > 0) orc_overlap_map(R, n, m_fix, fx, fy, fw, fh, F);
    double Ab = ((R->x1 - R->x0) / n) * ((R->y1 - R->y0) / n);
    for (size_t b = 0; b < nn; ++b) rho[b] = (rho_t * F[b] + D[b]) / Ab;
    if (mov_area) memcpy(mov_area, D, nn * sizeof(double));
    if (fix_area) memcpy(fix_area, F, nn * sizeof(double));
    free(D);
    free(F);
}

/* ------------------------------------------------------------------------ */
/* Spectral solution of Poisson's equation (Section III-E, Eqs. 8-12)        */
/* ------------------------------------------------------------------------ */

/* cos(pi * u * (2x+1) / (2n)) with the integer argument reduced mod 4n first. */
static double cos_b(int u, int x, int n) {
    long long k = ((long long)u * (2LL * x + 1)) % (4LL * n);
    return cos(M_PI * (double)k / (2.0 * n));
}
static double sin_b(int u, int x, int n) {
    long long k = ((long long)u * (2LL * x + 1)) % (4LL * n);
    return sin(M_PI * (double)k / (2.0 * n));
}

/* cs[u*n + x] = cos(pi u (2x+1)/2n); the same table transposed is cs_t. */
static double* cos_table(int n, int transposed) {
    double* t = (double*)malloc((size_t)n * n * sizeof(double));
    for (int u = 0; u < n; ++u)
        for (int x = 0; x < n; ++x) {
            if (transposed) t[(size_t)x * n + u] = cos_b(u, x, n);
            else t[(size_t)u * n + x] = cos_b(u, x, n);
        }
    return t;
}
static double* sin_table_t(int n) {
    double* t = (double*)malloc((size_t)n * n * sizeof(double));
    for (int u = 0; u < n; ++u)
        for (int x = 0; x < n; ++x) t[(size_t)x * n + u] = sin_b(u, x, n);
    return t;
}

static double eps(int u) { return u == 0 ? 1.0 : 2.0; }

/* Eq. 10 (normalised so that Eq. 9 is its inverse):
 *   a[v][u] = (eps_u eps_v / n^2) sum_y sum_x rho[y][x] cos(w_u x) cos(w_v y)
 * The double sum is taken one index at a time (the sum of products factors).
 * All coefficients, the (0,0) one included. */
void orc_dct_coeffs_dc(int n, const double* rho, double* a) {
    double* C = cos_table(n, 0);                   /* C[u][x] */
    double* t = (double*)malloc((size_t)n * n * sizeof(double)); /* t[u][y] */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int u = 0; u < n; ++u) {
            double s = 0.0;
            for (int x = 0; x < n; ++x) s += rho[(size_t)y * n + x] * C[(size_t)u * n + x];
            t[(size_t)u * n + y] = s;
        }
#pragma omp parallel for schedule(static)
    for (int v = 0; v < n; ++v)
        for (int u = 0; u < n; ++u) {
            double s = 0.0;
            for (int y = 0; y < n; ++y) s += C[(size_t)v * n + y] * t[(size_t)u * n + y];
            a[(size_t)v * n + u] = eps(u) * eps(v) / ((double)n * n) * s;
        }
    free(C);
    free(t);
}

/* Eq. 10 with the (0,0) coefficient set to zero (DC removal, Section III-A). */
void orc_dct_coeffs(int n, const double* rho, double* a) {
    orc_dct_coeffs_dc(n, rho, a);
    a[0] = 0.0;
}

/* Spectral divide: a/(w_u^2 + w_v^2 + eps); the (0,0) mode is a_00/eps for
 * eps > 0 (Helmholtz, Eq. 4) and left out for eps = 0 (Poisson, Eq. 8). */
static double spectral_hat(double a, int u, int v, double Lx, double Ly, double eps_h) {
    double wu = M_PI * u / Lx, wv = M_PI * v / Ly;
    if (u == 0 && v == 0) return eps_h > 0.0 ? a / eps_h : 0.0;
    return a / (wu * wu + wv * wv + eps_h);
}

/* Eqs. 11 and 12 at the bin centres:
 *   psi = sum_{u,v} a/(w_u^2+w_v^2) cos(w_u x) cos(w_v y)
 *   E_x = sum_{u,v} a w_u/(w_u^2+w_v^2) sin(w_u x) cos(w_v y)
 *   E_y = sum_{u,v} a w_v/(w_u^2+w_v^2) cos(w_u x) sin(w_v y)
 * with w_u = pi u / Lx, w_v = pi v / Ly and the (0,0) term left out; with
 * eps_h > 0 the divisor is w_u^2 + w_v^2 + eps_h and the (0,0) term is kept
 * (Helmholtz, Eq. 4).  a is indexed a[v][u]; outputs are [y][x].  Any output
 * may be NULL. */
void orc_potential_field_eps(int n, double Lx, double Ly, const double* a, double eps_h,
                             double* psi, double* ex, double* ey) {
    size_t nn = (size_t)n * n;
    double* hat = (double*)malloc(nn * sizeof(double));  /* hat[u][v] = a/(w^2) */
    for (int v = 0; v < n; ++v)
        for (int u = 0; u < n; ++u)
            hat[(size_t)u * n + v] = spectral_hat(a[(size_t)v * n + u], u, v, Lx, Ly, eps_h);
    double* Ct = cos_table(n, 1);  /* Ct[x][u] = cos(w_u x) */
    double* St = sin_table_t(n);   /* St[x][u] = sin(w_u x) */
    /* inner sums over v for each (u, y) */
    double* pc = (double*)malloc(nn * sizeof(double)); /* pc[u][y] = sum_v hat cos(w_v y) */
    double* ps = (double*)malloc(nn * sizeof(double)); /* ps[u][y] = sum_v hat w_v sin(w_v y) */
#pragma omp parallel for schedule(static)
    for (int u = 0; u < n; ++u)
        for (int y = 0; y < n; ++y) {
            double s1 = 0.0, s2 = 0.0;
            for (int v = 0; v < n; ++v) {
                double hv = hat[(size_t)u * n + v];
                s1 += hv * Ct[(size_t)y * n + v];
                s2 += hv * (M_PI * v / Ly) * St[(size_t)y * n + v];
            }
            pc[(size_t)u * n + y] = s1;
            ps[(size_t)u * n + y] = s2;
        }
    /* transpose so the outer sums over u run along contiguous memory */
    double* pcT = (double*)malloc(nn * sizeof(double));
    double* psT = (double*)malloc(nn * sizeof(double));
    for (int u = 0; u < n; ++u)
        for (int y = 0; y < n; ++y) {
            pcT[(size_t)y * n + u] = pc[(size_t)u * n + y];
            psT[(size_t)y * n + u] = ps[(size_t)u * n + y];
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double s_psi = 0.0, s_ex = 0.0, s_ey = 0.0;
            for (int u = 0; u < n; ++u) {
                double c = Ct[(size_t)x * n + u];
                double p = pcT[(size_t)y * n + u];
                s_psi += p * c;
                s_ex += p * (M_PI * u / Lx) * St[(size_t)x * n + u];
                s_ey += psT[(size_t)y * n + u] * c;
            }
            if (psi) psi[(size_t)y * n + x] = s_psi;
            if (ex) ex[(size_t)y * n + x] = s_ex;
            if (ey) ey[(size_t)y * n + x] = s_ey;
        }
    free(hat); free(Ct); free(St); free(pc); free(ps); free(pcT); free(psT);
}

void orc_potential_field(int n, double Lx, double Ly, const double* a,
                         double* psi, double* ex, double* ey) {
    orc_potential_field_eps(n, Lx, Ly, a, 0.0, psi, ex, ey);
}

/* Eqs. 11 and 12 at chosen bin centres only: for each k < count the sums
 * over all (u, v) at bin (ys[k], xs[k]).  Same definition as
 * orc_potential_field, O(n^2) per point, for spot checks of large grids. */
void orc_potential_at(int n, double Lx, double Ly, const double* a, int count,
                      const int32_t* xs, const int32_t* ys, double* psi, double* ex, double* ey) {
#pragma omp parallel
    {
        double* cu = (double*)malloc((size_t)n * sizeof(double));
        double* su = (double*)malloc((size_t)n * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < count; ++k) {
            int x = xs[k], y = ys[k];
            for (int u = 0; u < n; ++u) { cu[u] = cos_b(u, x, n); su[u] = sin_b(u, x, n); }
            double s_psi = 0.0, s_ex = 0.0, s_ey = 0.0;
            for (int v = 0; v < n; ++v) {
                double cv = cos_b(v, y, n), sv = sin_b(v, y, n), wv = M_PI * v / Ly;
                for (int u = 0; u < n; ++u) {
                    if (u == 0 && v == 0) continue;
                    double wu = M_PI * u / Lx;
                    double hat = a[(size_t)v * n + u] / (wu * wu + wv * wv);
                    s_psi += hat * cu[u] * cv;
                    s_ex += hat * wu * su[u] * cv;
                    s_ey += hat * wv * cu[u] * sv;
                }
            }
            psi[k] = s_psi;
            ex[k] = s_ex;
            ey[k] = s_ey;
        }
        free(cu);
        free(su);
    }
}

/* Potential energy, Eq. 6 over all charges (movable and fixed) with the factor
 * 1/2:  N = 1/2 sum_b A_b rho_b psi_b. */
double orc_energy(int n, double Ab, const double* rho, const double* psi) {
    double s = 0.0;
    for (size_t b = 0; b < (size_t)n * n; ++b) s += rho[b] * psi[b];
    return 0.5 * Ab * s;
}

/* Density gradient (Eq. 7, q.E):  dN/dx_i = -sum_b ov(i,b) E_x[b],
 * dN/dy_i = -sum_b ov(i,b) E_y[b]. */
void orc_gather(const orc_region* R, int n, int m, const float* x, const float* y,
                const float* w, const float* h, const double* ex, const double* ey,
                double* gx, double* gy) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        double xl, xh, yl, yh;
        int ilo, ihi, jlo, jhi;
        cell_edges(x[i], w[i], &xl, &xh);
        cell_edges(y[i], h[i], &yl, &yh);
        bin_span(R->x0, R->x1, n, xl, xh, &ilo, &ihi);
        bin_span(R->y0, R->y1, n, yl, yh, &jlo, &jhi);
        clamp_span(n, &ilo, &ihi);
        clamp_span(n, &jlo, &jhi);
        double sx = 0.0, sy = 0.0;
        for (int j = jlo; j <= jhi; ++j) {
            double oy = ov1(R->y0, R->y1, n, j, yl, yh);
            for (int k = ilo; k <= ihi; ++k) {
                double o = ov1(R->x0, R->x1, n, k, xl, xh) * oy;
                sx += o * ex[(size_t)j * n + k];
                sy += o * ey[(size_t)j * n + k];
            }
        }
        gx[i] = -sx;
        gy[i] = -sy;
    }
}

/* Exact derivative of the binned energy N = 1/2 A_b rho^T psi with respect to
 * the cell centre.  N is a symmetric quadratic form in rho, so
 * dN/drho_b = A_b psi_b and dN/dx_i = sum_b psi_b d ov(i,b)/dx_i.  Moving the
 * cell right by dx grows its overlap with the bin holding the right edge and
 * shrinks it with the bin holding the left edge, each by dx times the y
 * overlap of that row.  "Holding" uses the half-open bins [e_k, e_k+1), which
 * makes this the right derivative where an edge sits exactly on a bin edge;
 * an edge outside the grid contributes nothing.  Likewise in y. */
void orc_adjoint(const orc_region* R, int n, int m, const float* x, const float* y,
                 const float* w, const float* h, const double* psi, double* gx, double* gy) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        double xl, xh, yl, yh;
        int ilo, ihi, jlo, jhi;
        cell_edges(x[i], w[i], &xl, &xh);
        cell_edges(y[i], h[i], &yl, &yh);
        bin_span(R->x0, R->x1, n, xl, xh, &ilo, &ihi);
        bin_span(R->y0, R->y1, n, yl, yh, &jlo, &jhi);
        clamp_span(n, &ilo, &ihi);
        clamp_span(n, &jlo, &jhi);
        double sx = 0.0, sy = 0.0;
        if (ilo <= ihi && jlo <= jhi) {
            int kl = last_edge_le(R->x0, R->x1, n, xl, 0);
            int kr = last_edge_le(R->x0, R->x1, n, xh, 0);
            int jl = last_edge_le(R->y0, R->y1, n, yl, 0);
            int jr = last_edge_le(R->y0, R->y1, n, yh, 0);
            for (int j = jlo; j <= jhi; ++j) {
                double oy = ov1(R->y0, R->y1, n, j, yl, yh);
                if (kr >= 0 && kr <= n - 1) sx += oy * psi[(size_t)j * n + kr];
                if (kl >= 0 && kl <= n - 1) sx -= oy * psi[(size_t)j * n + kl];
            }
            for (int k = ilo; k <= ihi; ++k) {
                double ox = ov1(R->x0, R->x1, n, k, xl, xh);
                if (jr >= 0 && jr <= n - 1) sy += ox * psi[(size_t)jr * n + k];
                if (jl >= 0 && jl <= n - 1) sy -= ox * psi[(size_t)jl * n + k];
            }
        }
        gx[i] = sx;
        gy[i] = sy;
    }
}

/* Density overflow (Section IV-A, read as the total overflow ratio):
 *   tau = sum_b max(0, D_b - rho_t (A_b - F_b)) / sum_{i in V_m} q_i */
double orc_overflow(int n, double Ab, double rho_t, const double* mov_area,
                    const double* fix_area, double total_mov_area) {
    double s = 0.0;
    for (size_t b = 0; b < (size_t)n * n; ++b) {
        double cap = rho_t * (Ab - (fix_area ? fix_area[b] : 0.0));
        s += dmax(0.0, mov_area[b] - cap);
    }
    /* no movable cells: nothing can overflow (the ratio is read as 0) */
    return total_mov_area > 0.0 ? s / total_mov_area : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Wirelength (Eq. 1 HPWL and Eq. 3 weighted-average model)                  */
/* ------------------------------------------------------------------------ */

static double pin_coord(float c, float d) {
    volatile float p = c + d;   /* fl32(cell centre + offset) */
    return (double)p;
}

/* Weighted-average wirelength of one net along one axis (Eq. 3), with the
 * exponentials shifted by the max (resp. min) pin coordinate, which leaves the
 * ratios unchanged.  For pins p_j, M = max p, mu = min p:
 *   a+_j = exp((p_j - M)/g),  a-_j = exp((mu - p_j)/g)
 *   W+ = sum p a+ / sum a+,   W- = sum p a- / sum a-,   W~ = W+ - W-
 *   dW~/dp_j = (a+_j/S+)(1 + (p_j - W+)/g) - (a-_j/S-)(1 - (p_j - W-)/g)
 * Returns W~; grad (deg entries, may be NULL) receives dW~/dp_j; *span gets
 * max - min (the net's HPWL term, Eq. 1). */
static double wa_axis(int deg, const double* p, double g, double* grad, double* span) {
    double M = p[0], mu = p[0];
    for (int j = 1; j < deg; ++j) { M = dmax(M, p[j]); mu = dmin(mu, p[j]); }
    *span = M - mu;
    double Sp = 0, Tp = 0, Sm = 0, Tm = 0;
    for (int j = 0; j < deg; ++j) {
        double ap = exp((p[j] - M) / g), am = exp((mu - p[j]) / g);
        Sp += ap; Tp += p[j] * ap;
        Sm += am; Tm += p[j] * am;
    }
    double Wp = Tp / Sp, Wm = Tm / Sm;
    if (grad) {
        for (int j = 0; j < deg; ++j) {
            double ap = exp((p[j] - M) / g), am = exp((mu - p[j]) / g);
            grad[j] = ap / Sp * (1.0 + (p[j] - Wp) / g) - am / Sm * (1.0 - (p[j] - Wm) / g);
        }
    }
    return Wp - Wm;
}

/* Log-sum-exp wirelength of one net along one axis (the LSE model Section II
 * names): g ln sum_j exp(p_j/g) + g ln sum_j exp(-p_j/g), evaluated with the
 * exponentials shifted by the max (resp. min):
 *   = (M - mu) + g (ln S+ + ln S-),  S+ = sum exp((p_j - M)/g),
 *                                    S- = sum exp((mu - p_j)/g)
 *   d/dp_j = exp((p_j - M)/g)/S+ - exp((mu - p_j)/g)/S-
 * Same interface as wa_axis. */
static double lse_axis(int deg, const double* p, double g, double* grad, double* span) {
    double M = p[0], mu = p[0];
    for (int j = 1; j < deg; ++j) { M = dmax(M, p[j]); mu = dmin(mu, p[j]); }
    *span = M - mu;
    double Sp = 0, Sm = 0;
    for (int j = 0; j < deg; ++j) {
        Sp += exp((p[j] - M) / g);
        Sm += exp((mu - p[j]) / g);
    }
    if (grad)
        for (int j = 0; j < deg; ++j)
            grad[j] = exp((p[j] - M) / g) / Sp - exp((mu - p[j]) / g) / Sm;
    return (M - mu) + g * (log(Sp) + log(Sm));
}

/* Smoothed wirelength of all nets and its gradient.  Pin j of net e sits on
 * cell pin_cell[j] (movable if < m_mov, else macro pin_cell[j]-m_mov) at offset
 * (dx, dy) from the centre.  Degree-1 nets contribute nothing (W~ = 0, zero
 * gradient).  Outputs (each may be NULL):
 *   net_w[E]      W~_e (x plus y)
 *   gpx/gpy[P]    dW~/d(pin coordinate)
 *   gcx/gcy[m]    dW~/d(cell centre) = sum over that cell's pins
 * Returns sum_e W~_e; *hpwl receives the HPWL of Eq. 1 on pin coordinates. */
double orc_wl(int model, int E, const int32_t* net_ptr, const int32_t* pin_cell,
              const float* dx, const float* dy, int m_mov,
              const float* x, const float* y, const float* fx, const float* fy,
              double gamma, double* net_w, double* gpx, double* gpy,
              double* gcx, double* gcy, double* hpwl) {
    double (*axis)(int, const double*, double, double*, double*) = model ? lse_axis : wa_axis;
    double total = 0.0, hp = 0.0;
    if (gcx) memset(gcx, 0, (size_t)m_mov * sizeof(double));
    if (gcy) memset(gcy, 0, (size_t)m_mov * sizeof(double));
    int maxdeg = 1;
    for (int e = 0; e < E; ++e) {
        int d = net_ptr[e + 1] - net_ptr[e];
        if (d > maxdeg) maxdeg = d;
    }
    double* px = (double*)malloc((size_t)maxdeg * sizeof(double));
    double* py = (double*)malloc((size_t)maxdeg * sizeof(double));
    double* gx = (double*)malloc((size_t)maxdeg * sizeof(double));
    double* gy = (double*)malloc((size_t)maxdeg * sizeof(double));
    for (int e = 0; e < E; ++e) {
        int b = net_ptr[e], d = net_ptr[e + 1] - b;
        for (int j = 0; j < d; ++j) {
            int c = pin_cell[b + j];
            float cx = c < m_mov ? x[c] : fx[c - m_mov];
            float cy = c < m_mov ? y[c] : fy[c - m_mov];
            px[j] = pin_coord(cx, dx[b + j]);
            py[j] = pin_coord(cy, dy[b + j]);
        }
        double we = 0.0;
        if (d >= 2) {
            double sx, sy;
            we = axis(d, px, gamma, gx, &sx) + axis(d, py, gamma, gy, &sy);
            hp += sx + sy;
        } else {
            for (int j = 0; j < d; ++j) { gx[j] = 0.0; gy[j] = 0.0; }
        }
        total += we;
        if (net_w) net_w[e] = we;
        for (int j = 0; j < d; ++j) {
            if (gpx) gpx[b + j] = gx[j];
            if (gpy) gpy[b + j] = gy[j];
            int c = pin_cell[b + j];
            if (c < m_mov) {
                if (gcx) gcx[c] += gx[j];
                if (gcy) gcy[c] += gy[j];
            }
        }
    }
    free(px); free(py); free(gx); free(gy);
    if (hpwl) *hpwl = hp;
    return total;
}

/* The weighted-average model (Eq. 3) of orc_wl. */
double orc_wa(int E, const int32_t* net_ptr, const int32_t* pin_cell,
              const float* dx, const float* dy, int m_mov,
              const float* x, const float* y, const float* fx, const float* fy,
              double gamma, double* net_w, double* gpx, double* gpy,
              double* gcx, double* gcy, double* hpwl) {
    return orc_wl(0, E, net_ptr, pin_cell, dx, dy, m_mov, x, y, fx, fy, gamma, net_w, gpx, gpy,
                  gcx, gcy, hpwl);
}

/* ------------------------------------------------------------------------ */
/* One full objective-gradient evaluation (Algorithm 1, steps f, rho, FFT    */
/* solve and gradient).                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double N, W, hpwl, tau, total_mov_area;
    double gN_l1, gW_l1;
} orc_eval_out;

/* Evaluates density energy + gradient and the wirelength + gradient at
 * (x, y): model 0 weighted average (Eq. 3), 1 log-sum-exp; eps_h 0 the
 * Poisson solve (Eq. 8), > 0 the Helmholtz solve (Eq. 4).  Any of the map
 * outputs (rho, psi, ex, ey) may be NULL. */
void orc_eval2(const orc_region* R, int n, double rho_t,
               int m_mov, const float* x, const float* y, const float* w, const float* h,
               int m_fix, const float* fx, const float* fy, const float* fw, const float* fh,
               int E, const int32_t* net_ptr, const int32_t* pin_cell,
               const float* pdx, const float* pdy, double gamma, int model, double eps_h,
               double* gNx, double* gNy, double* gWx, double* gWy,
               double* rho_o, double* psi_o, double* ex_o, double* ey_o, orc_eval_out* out) {
    size_t nn = (size_t)n * n;
    double Lx = R->x1 - R->x0, Ly = R->y1 - R->y0;
    double Ab = (Lx / n) * (Ly / n);
    double* rho = (double*)malloc(nn * sizeof(double));
    double* D = (double*)malloc(nn * sizeof(double));
    double* F = (double*)malloc(nn * sizeof(double));
    double* a = (double*)malloc(nn * sizeof(double));
    double* psi = (double*)malloc(nn * sizeof(double));
    double* ex = (double*)malloc(nn * sizeof(double));
    double* ey = (double*)malloc(nn * sizeof(double));
    orc_density(R, n, rho_t, m_mov, x, y, w, h, m_fix, fx, fy, fw, fh, rho, D, F);
    if (eps_h > 0.0) orc_dct_coeffs_dc(n, rho, a);
    else orc_dct_coeffs(n, rho, a);
    orc_potential_field_eps(n, Lx, Ly, a, eps_h, psi, ex, ey);
    double q = 0.0;
    for (int i = 0; i < m_mov; ++i) q += (double)w[i] * (double)h[i];
    out->total_mov_area = q;
    out->N = orc_energy(n, Ab, rho, psi);
    out->tau = orc_overflow(n, Ab, rho_t, D, F, q);
    orc_gather(R, n, m_mov, x, y, w, h, ex, ey, gNx, gNy);
    out->W = orc_wl(model, E, net_ptr, pin_cell, pdx, pdy, m_mov, x, y, fx, fy, gamma,
                    NULL, NULL, NULL, gWx, gWy, &out->hpwl);
    double l1n = 0.0, l1w = 0.0;
    for (int i = 0; i < m_mov; ++i) {
        l1n += fabs(gNx[i]) + fabs(gNy[i]);
        l1w += fabs(gWx[i]) + fabs(gWy[i]);
    }
    out->gN_l1 = l1n;
    out->gW_l1 = l1w;
    if (rho_o) memcpy(rho_o, rho, nn * sizeof(double));
    if (psi_o) memcpy(psi_o, psi, nn * sizeof(double));
    if (ex_o) memcpy(ex_o, ex, nn * sizeof(double));
    if (ey_o) memcpy(ey_o, ey, nn * sizeof(double));
    free(rho); free(D); free(F); free(a); free(psi); free(ex); free(ey);
}

/* orc_eval2 with the weighted-average model and the Poisson solve. */
void orc_eval(const orc_region* R, int n, double rho_t,
              int m_mov, const float* x, const float* y, const float* w, const float* h,
              int m_fix, const float* fx, const float* fy, const float* fw, const float* fh,
              int E, const int32_t* net_ptr, const int32_t* pin_cell,
              const float* pdx, const float* pdy, double gamma,
              double* gNx, double* gNy, double* gWx, double* gWy,
              double* rho_o, double* psi_o, double* ex_o, double* ey_o, orc_eval_out* out) {
    orc_eval2(R, n, rho_t, m_mov, x, y, w, h, m_fix, fx, fy, fw, fh, E, net_ptr, pin_cell, pdx,
              pdy, gamma, 0, 0.0, gNx, gNy, gWx, gWy, rho_o, psi_o, ex_o, ey_o, out);
}

/* ------------------------------------------------------------------------ */
/* Parameter control (Section IV-A) and the Nesterov loop that stands in for */
/* the conjugate-gradient solver of Algorithm 1.                            */
/* ------------------------------------------------------------------------ */

/* mu_k = 1.1^(-dW/dW_ref + 1), bounded to [0.75, 1.1]. */
double orc_mu(double dW, double dW_ref) {
    double mu = pow(1.1, -dW / dW_ref + 1.0);
    return dmin(1.1, dmax(0.75, mu));
}

/* gamma = 8.0 w_b * 10^((20/9)(tau - 0.1) - 1). */
double orc_gamma(double tau, double wb) {
    return 8.0 * wb * pow(10.0, (20.0 / 9.0) * (tau - 0.1) - 1.0);
}

/* Nesterov momentum sequence: a_{k+1} = (1 + sqrt(1 + 4 a_k^2)) / 2. */
double orc_nesterov_a(double a) { return 0.5 * (1.0 + sqrt(1.0 + 4.0 * a * a)); }

typedef struct {
    double W, hpwl, N, tau, lambda, gamma, alpha, step_max;
} orc_iter_rec;

typedef struct {
    double lambda0;      /* <= 0: ||grad W~||_1 / ||grad N||_1 at the start */
    double gamma_fixed;  /* > 0: fixed gamma; else the schedule of tau */
    double dw_ref;       /* reference HPWL variation (3.5e5 in the paper) */
    double alpha_max0_bins; /* 0.044 */
    int stop_on_tau;     /* stop when tau <= tau_stop */
    double tau_stop;     /* 0.1 */
    int wirelength;      /* 0 weighted average (Eq. 3), 1 log-sum-exp */
    double helmholtz_eps; /* 0 Poisson (Eq. 8), > 0 Helmholtz (Eq. 4) */
    double alpha_max_cap_bins; /* Nesterov loop: alpha_max <= this many bins (0: none) */
} orc_loop_opts;

/* The objective as the loop sees it: at the point v (nvar doubles, all x
 * then all y for a placement) and smoothing gamma, the wirelength gradient gW,
 * the density gradient gN (nvar each) and the scalars of out.  With
 * gW == NULL only out->tau is wanted (the gamma schedule's start). */
typedef struct {
    double W, hpwl, N, tau, gN_l1, gW_l1;
} orc_point_out;

typedef void (*orc_objective_fn)(void* ctx, const double* v, double gamma, double* gW,
                                 double* gN, orc_point_out* out);

/* Nesterov's method in place of the conjugate-gradient solver of Algorithm 1,
 * with the parameter control of Section IV-A, on any objective f of the form
 * W~ + lambda N given by its callback.  x (nvar) holds the start and receives
 * the final major iterate u; lo, hi bound each variable (the projection Pi);
 * wb is the bin width (alpha_max_0 = alpha_max0_bins wb and the gamma
 * schedule).  recs (iters entries) receive per-iteration metrics.  Returns
 * the number of iterations run.
 *
 * u_0 = v_0 = Pi(x), a_0 = 1.  Iteration k, at the look-ahead point v_k:
 *   g_k = grad W~(v_k; gamma_k) + lambda_k grad N(v_k)
 *   lambda_0 = ||grad W~||_1 / ||grad N||_1 at v_0 unless given;
 *   lambda_k = mu_k lambda_{k-1} (k >= 1), mu from dW = HPWL(v_k) - HPWL(v_{k-1})
 *   alpha_0 = alpha_max_0 / ||g_0||_inf,
 *   alpha_k = ||v_k - v_{k-1}||_2 / ||g_k - g_{k-1}||_2 (k >= 1),
 *   then alpha_k ||g_k||_inf is clamped to [0.01 alpha_max_k, alpha_max_k]
 *   u_{k+1} = Pi(v_k - alpha_k g_k)
 *   a_{k+1} = (1 + sqrt(1 + 4 a_k^2))/2, beta = (a_k - 1)/a_{k+1}
 *   v_{k+1} = Pi(u_{k+1} + beta (u_{k+1} - u_k))
 *   alpha_max_{k+1} = max(alpha_max_0, 2 max_i |u_{k+1} - v_k|), kept at
 *   or below max(alpha_max_0, cap wb) when the option's cap (bins) is > 0:
 *   the doubling rule of Section IV-A was made for the paper's line search,
 *   and with Barzilai-Borwein steps alone the largest move can double every
 *   iteration up to the size of the region
 *   gamma_{k+1} = gamma(tau_k) unless fixed.
 * Adaptive restart (the gradient test of O'Donoghue and Candes, "Adaptive
 * restart for accelerated gradient schemes", 2015), taken one iteration
 * late: when g_k . (u_{k+1} - u_k) > 0 the step went uphill for the
 * gradient at v_k, and the sequence starts over, a_{k+1} := 1, so that the
 * next momentum weight is 0. */
int orc_nesterov_run(int nvar, double* x, const double* lo, const double* hi, double wb,
                     orc_objective_fn f, void* ctx, const orc_loop_opts* o, int iters,
                     orc_iter_rec* recs) {
    size_t m2 = (size_t)nvar;
    double* u = (double*)malloc(m2 * sizeof(double));
    double* v = (double*)malloc(m2 * sizeof(double));
    double* vp = (double*)malloc(m2 * sizeof(double));
    double* g = (double*)malloc(m2 * sizeof(double));
    double* gp = (double*)malloc(m2 * sizeof(double));
    double* gN = (double*)malloc(m2 * sizeof(double));
    double* gW = (double*)malloc(m2 * sizeof(double));
    for (size_t i = 0; i < m2; ++i) {
        u[i] = dmin(hi[i], dmax(lo[i], x[i]));
        v[i] = u[i];
    }
    double a_k = 1.0, lambda = o->lambda0, alpha_max0 = o->alpha_max0_bins * wb;
    double alpha_max = alpha_max0, alpha = 0.0, hp_prev = 0.0;
    double gamma = o->gamma_fixed;
    int k;
    for (k = 0; k < iters; ++k) {
        orc_point_out ev;
        if (k == 0 && gamma <= 0.0) {
            /* the schedule needs tau at the start */
            f(ctx, v, 0.0, NULL, NULL, &ev);
            gamma = orc_gamma(ev.tau, wb);
        }
        f(ctx, v, gamma, gW, gN, &ev);
        if (k == 0 && lambda <= 0.0) lambda = ev.gN_l1 > 0 ? ev.gW_l1 / ev.gN_l1 : 1.0;
        if (k >= 1) lambda *= orc_mu(ev.hpwl - hp_prev, o->dw_ref);
        hp_prev = ev.hpwl;
        double ginf = 0.0;
        for (size_t i = 0; i < m2; ++i) {
            g[i] = gW[i] + lambda * gN[i];
            ginf = dmax(ginf, fabs(g[i]));
        }
        if (k == 0) {
            alpha = ginf > 0 ? alpha_max0 / ginf : 0.0;
        } else {
            double dv = 0.0, dg = 0.0;
            for (size_t i = 0; i < m2; ++i) {
                dv += (v[i] - vp[i]) * (v[i] - vp[i]);
                dg += (g[i] - gp[i]) * (g[i] - gp[i]);
            }
            if (dg > 0.0) alpha = sqrt(dv) / sqrt(dg);
        }
        if (ginf > 0.0) {
            if (alpha * ginf > alpha_max) alpha = alpha_max / ginf;
            if (alpha * ginf < 0.01 * alpha_max) alpha = 0.01 * alpha_max / ginf;
        }
        double a_next = orc_nesterov_a(a_k);
        double beta = (a_k - 1.0) / a_next;
        double step_max = 0.0, uphill = 0.0;
        for (size_t i = 0; i < m2; ++i) {
            double un = dmin(hi[i], dmax(lo[i], v[i] - alpha * g[i]));
            step_max = dmax(step_max, fabs(un - v[i]));
            uphill += g[i] * (un - u[i]);
            double vn = dmin(hi[i], dmax(lo[i], un + beta * (un - u[i])));
            vp[i] = v[i];
            gp[i] = g[i];
            u[i] = un;
            v[i] = vn;
        }
        if (uphill > 0.0) a_next = 1.0;
        if (recs) {
            recs[k].W = ev.W; recs[k].hpwl = ev.hpwl; recs[k].N = ev.N; recs[k].tau = ev.tau;
            recs[k].lambda = lambda; recs[k].gamma = gamma; recs[k].alpha = alpha;
            recs[k].step_max = step_max;
        }
        a_k = a_next;
        alpha_max = dmax(alpha_max0, 2.0 * step_max);
        if (o->alpha_max_cap_bins > 0.0)
            alpha_max = dmin(alpha_max, dmax(alpha_max0, o->alpha_max_cap_bins * wb));
        if (o->gamma_fixed <= 0.0) gamma = orc_gamma(ev.tau, wb);
        if (o->stop_on_tau && ev.tau <= o->tau_stop) { ++k; break; }
    }
    for (size_t i = 0; i < m2; ++i) x[i] = u[i];
    free(u); free(v); free(vp); free(g); free(gp); free(gN); free(gW);
    return k;
}

/* A placement instance as the loop's objective: positions rounded to
 * float32 for each evaluation (the library's inputs), then orc_eval2. */
typedef struct {
    const orc_region* R;
    int n;
    double rho_t;
    int m_mov;
    const float *w, *h;
    int m_fix;
    const float *fx, *fy, *fw, *fh;
    int E;
    const int32_t *net_ptr, *pin_cell;
    const float *pdx, *pdy;
    int wirelength;
    double helmholtz_eps;
    float *xf, *yf;
} orc_place_ctx;

static void place_objective(void* vctx, const double* v, double gamma, double* gW, double* gN,
                            orc_point_out* out) {
    orc_place_ctx* c = (orc_place_ctx*)vctx;
    int m = c->m_mov;
    for (int i = 0; i < m; ++i) { c->xf[i] = (float)v[i]; c->yf[i] = (float)v[m + i]; }
    if (!gW) {
        size_t nn = (size_t)c->n * c->n;
        double* rho = (double*)malloc(nn * sizeof(double));
        double* D = (double*)malloc(nn * sizeof(double));
        double* F = (double*)malloc(nn * sizeof(double));
        orc_density(c->R, c->n, c->rho_t, m, c->xf, c->yf, c->w, c->h, c->m_fix, c->fx, c->fy,
                    c->fw, c->fh, rho, D, F);
        double q = 0.0;
        for (int i = 0; i < m; ++i) q += (double)c->w[i] * (double)c->h[i];
        double Ab = ((c->R->x1 - c->R->x0) / c->n) * ((c->R->y1 - c->R->y0) / c->n);
        out->tau = orc_overflow(c->n, Ab, c->rho_t, D, F, q);
        free(rho); free(D); free(F);
        return;
    }
    orc_eval_out ev;
    orc_eval2(c->R, c->n, c->rho_t, m, c->xf, c->yf, c->w, c->h, c->m_fix, c->fx, c->fy, c->fw,
              c->fh, c->E, c->net_ptr, c->pin_cell, c->pdx, c->pdy, gamma, c->wirelength,
              c->helmholtz_eps, gN, gN + m, gW, gW + m, NULL, NULL, NULL, NULL, &ev);
    out->W = ev.W; out->hpwl = ev.hpwl; out->N = ev.N; out->tau = ev.tau;
    out->gN_l1 = ev.gN_l1; out->gW_l1 = ev.gW_l1;
}

/* Global placement loop (Algorithm 1 with the CG step replaced by Nesterov's
 * method, orc_nesterov_run) on a placement instance.  Positions are kept in
 * FP64 and rounded to float32 for each evaluation.  x, y (m_mov) are updated
 * in place with the final major iterate u.  The projection keeps each cell
 * inside the region: [x0 + w/2, x1 - w/2]. */
int orc_nesterov(const orc_region* R, int n, double rho_t,
                 int m_mov, float* x, float* y, const float* w, const float* h,
                 int m_fix, const float* fx, const float* fy, const float* fw, const float* fh,
                 int E, const int32_t* net_ptr, const int32_t* pin_cell,
                 const float* pdx, const float* pdy, const orc_loop_opts* o,
                 int iters, orc_iter_rec* recs) {
    size_t m2 = (size_t)2 * m_mov;
    double wb = (R->x1 - R->x0) / n;
    double* u = (double*)malloc(m2 * sizeof(double));
    double* lo = (double*)malloc(m2 * sizeof(double));
    double* hi = (double*)malloc(m2 * sizeof(double));
    orc_place_ctx c = {R, n, rho_t, m_mov, w, h, m_fix, fx, fy, fw, fh, E, net_ptr, pin_cell,
                       pdx, pdy, o->wirelength, o->helmholtz_eps,
                       (float*)malloc((size_t)m_mov * sizeof(float)),
                       (float*)malloc((size_t)m_mov * sizeof(float))};
    for (int i = 0; i < m_mov; ++i) {
        lo[i] = R->x0 + 0.5 * w[i]; hi[i] = R->x1 - 0.5 * w[i];
        lo[m_mov + i] = R->y0 + 0.5 * h[i]; hi[m_mov + i] = R->y1 - 0.5 * h[i];
        u[i] = (double)x[i];
        u[m_mov + i] = (double)y[i];
    }
    int k = orc_nesterov_run((int)m2, u, lo, hi, wb, place_objective, &c, o, iters, recs);
    for (int i = 0; i < m_mov; ++i) { x[i] = (float)u[i]; y[i] = (float)u[m_mov + i]; }
    free(u); free(lo); free(hi); free(c.xf); free(c.yf);
    return k;
}

/* Global placement loop with the nonlinear conjugate-gradient step of
 * Algorithm 1 ("CGsolver" with the search interval [0.01 a_max, a_max] of
 * Section IV-A).  Same options, records and clamping as orc_nesterov.
 * The paper does not spell the CG step out; this is the reading:
 *   g_k = grad W~(x_k; gamma_k) + lambda_k grad N(x_k),
 *   f_k = W~(x_k) + lambda_k N(x_k)
 *   d_k = -g_k + beta_k d_{k-1},  beta_k = max(0, g_k.(g_k - g_{k-1}) / |g_{k-1}|^2)
 *         (Polak-Ribiere+; d_0 = -g_0; restart d_k = -g_k if g_k.d_k >= 0)
 *   dh = d_k / |d_k|_inf  (so a step a moves the farthest cell by a)
 *   slope s = g_k.dh;  trial f_t = f(clamp(x_k + a_max dh)) with the same
 *   lambda_k, gamma_k;  quadratic fit c = (f_t - f_k - s a_max) / a_max^2,
 *   a* = -s / (2c) if c > 0 else a_max;  a_k = min(a_max, max(0.01 a_max, a*))
 *   x_{k+1} = clamp(x_k + a_k dh)
 *   a_max_{k+1} = max(a_max_0, 2 a_k)  (Section IV-A)
 *   lambda, gamma and the stop test as in orc_nesterov (HPWL at the x_k).
 * recs[k].alpha = a_k; recs[k].step_max = a_k (the farthest move). */
int orc_cg(const orc_region* R, int n, double rho_t,
           int m_mov, float* x, float* y, const float* w, const float* h,
           int m_fix, const float* fx, const float* fy, const float* fw, const float* fh,
           int E, const int32_t* net_ptr, const int32_t* pin_cell,
           const float* pdx, const float* pdy, const orc_loop_opts* o,
           int iters, orc_iter_rec* recs) {
    size_t m2 = (size_t)2 * m_mov;
    double wb = (R->x1 - R->x0) / n;
    double* u = (double*)malloc(m2 * sizeof(double));
    double* d = (double*)malloc(m2 * sizeof(double));
    double* g = (double*)malloc(m2 * sizeof(double));
    double* gp = (double*)malloc(m2 * sizeof(double));
    double* gN = (double*)malloc(m2 * sizeof(double));
    double* gW = (double*)malloc(m2 * sizeof(double));
    double* lo = (double*)malloc(m2 * sizeof(double));
    double* hi = (double*)malloc(m2 * sizeof(double));
    float* xf = (float*)malloc((size_t)m_mov * sizeof(float));
    float* yf = (float*)malloc((size_t)m_mov * sizeof(float));
    for (int i = 0; i < m_mov; ++i) {
        lo[i] = R->x0 + 0.5 * w[i]; hi[i] = R->x1 - 0.5 * w[i];
        lo[m_mov + i] = R->y0 + 0.5 * h[i]; hi[m_mov + i] = R->y1 - 0.5 * h[i];
        u[i] = dmin(hi[i], dmax(lo[i], (double)x[i]));
        u[m_mov + i] = dmin(hi[m_mov + i], dmax(lo[m_mov + i], (double)y[i]));
    }
    double lambda = o->lambda0, alpha_max0 = o->alpha_max0_bins * wb;
    double alpha_max = alpha_max0, hp_prev = 0.0, gg_prev = 0.0;
    double gamma = o->gamma_fixed;
    int k;
    for (k = 0; k < iters; ++k) {
        for (int i = 0; i < m_mov; ++i) { xf[i] = (float)u[i]; yf[i] = (float)u[m_mov + i]; }
        orc_eval_out ev;
        if (k == 0 && gamma <= 0.0) {
            size_t nn = (size_t)n * n;
            double* rho = (double*)malloc(nn * sizeof(double));
            double* D = (double*)malloc(nn * sizeof(double));
            double* F = (double*)malloc(nn * sizeof(double));
            orc_density(R, n, rho_t, m_mov, xf, yf, w, h, m_fix, fx, fy, fw, fh, rho, D, F);
            double q = 0.0;
            for (int i = 0; i < m_mov; ++i) q += (double)w[i] * (double)h[i];
            gamma = orc_gamma(orc_overflow(n, wb * ((R->y1 - R->y0) / n), rho_t, D, F, q), wb);
            free(rho); free(D); free(F);
        }
        orc_eval2(R, n, rho_t, m_mov, xf, yf, w, h, m_fix, fx, fy, fw, fh, E, net_ptr, pin_cell,
                  pdx, pdy, gamma, o->wirelength, o->helmholtz_eps, gN, gN + m_mov, gW,
                  gW + m_mov, NULL, NULL, NULL, NULL, &ev);
        if (k == 0 && lambda <= 0.0) lambda = ev.gN_l1 > 0 ? ev.gW_l1 / ev.gN_l1 : 1.0;
        if (k >= 1) lambda *= orc_mu(ev.hpwl - hp_prev, o->dw_ref);
        hp_prev = ev.hpwl;
        double fk = ev.W + lambda * ev.N;
        double gg = 0.0, ggp = 0.0;
        for (size_t i = 0; i < m2; ++i) {
            g[i] = gW[i] + lambda * gN[i];
            gg += g[i] * g[i];
            if (k > 0) ggp += g[i] * gp[i];
        }
        double beta = (k > 0 && gg_prev > 0.0) ? dmax(0.0, (gg - ggp) / gg_prev) : 0.0;
        double gd = 0.0, dinf = 0.0;
        for (size_t i = 0; i < m2; ++i) {
            d[i] = -g[i] + beta * (k > 0 ? d[i] : 0.0);
            gd += g[i] * d[i];
        }
        if (!(gd < 0.0)) {   /* not a descent direction: restart */
            gd = 0.0;
            for (size_t i = 0; i < m2; ++i) { d[i] = -g[i]; gd -= g[i] * g[i]; }
        }
        for (size_t i = 0; i < m2; ++i) dinf = dmax(dinf, fabs(d[i]));
        double alpha = 0.0;
        if (dinf > 0.0) {
            double slope = gd / dinf;
            for (int i = 0; i < m_mov; ++i) {
                xf[i] = (float)dmin(hi[i], dmax(lo[i], u[i] + alpha_max * d[i] / dinf));
                yf[i] = (float)dmin(hi[m_mov + i],
                                    dmax(lo[m_mov + i], u[m_mov + i] + alpha_max * d[m_mov + i] / dinf));
            }
            orc_eval_out et;
            orc_eval2(R, n, rho_t, m_mov, xf, yf, w, h, m_fix, fx, fy, fw, fh, E, net_ptr,
                      pin_cell, pdx, pdy, gamma, o->wirelength, o->helmholtz_eps, gp, gp + m_mov,
                      gp, gp + m_mov, NULL, NULL, NULL, NULL, &et);
            double ft = et.W + lambda * et.N;
            double c = (ft - fk - slope * alpha_max) / (alpha_max * alpha_max);
            double as = c > 0.0 ? -slope / (2.0 * c) : alpha_max;
            alpha = dmin(alpha_max, dmax(0.01 * alpha_max, as));
            for (size_t i = 0; i < m2; ++i)
                u[i] = dmin(hi[i], dmax(lo[i], u[i] + alpha * d[i] / dinf));
        }
        for (size_t i = 0; i < m2; ++i) gp[i] = g[i];
        gg_prev = gg;
        if (recs) {
            recs[k].W = ev.W; recs[k].hpwl = ev.hpwl; recs[k].N = ev.N; recs[k].tau = ev.tau;
            recs[k].lambda = lambda; recs[k].gamma = gamma; recs[k].alpha = alpha;
            recs[k].step_max = alpha;
        }
        alpha_max = dmax(alpha_max0, 2.0 * alpha);
        if (o->gamma_fixed <= 0.0) gamma = orc_gamma(ev.tau, wb);
        if (o->stop_on_tau && ev.tau <= o->tau_stop) { ++k; break; }
    }
    for (int i = 0; i < m_mov; ++i) { x[i] = (float)u[i]; y[i] = (float)u[m_mov + i]; }
    free(u); free(d); free(g); free(gp); free(gN); free(gW); free(lo); free(hi);
    free(xf); free(yf);
    return k;
}

/* Filler cells (Section III-B: disconnected movable cells that take up the
 * free area the movable cells leave).  The paper gives no count or size;
 * the reading: the fillers' total area is rho_t times the free area of the
 * region (its area minus the fixed cells' overlap with it) minus the movable
 * area, each filler has the mean movable width and height, and the count is
 * that area over one filler's, rounded down (0 if the movable cells already
 * fill rho_t of the free area).  Sizes are returned in float32, as the
 * library stores them. */
void orc_fillers(const orc_region* R, int m_mov, const float* w, const float* h,
                 int m_fix, const float* fx, const float* fy, const float* fw, const float* fh,
                 double rho_t, int64_t* count, float* filler_w, float* filler_h) {
    double area = (R->x1 - R->x0) * (R->y1 - R->y0), fixed = 0.0, mov = 0.0, sw = 0.0, sh = 0.0;
    for (int f = 0; f < m_fix; ++f) {
        double ox = dmin(R->x1, (double)fx[f] + 0.5 * fw[f]) - dmax(R->x0, (double)fx[f] - 0.5 * fw[f]);
        double oy = dmin(R->y1, (double)fy[f] + 0.5 * fh[f]) - dmax(R->y0, (double)fy[f] - 0.5 * fh[f]);
        if (ox > 0.0 && oy > 0.0) fixed += ox * oy;
    }
    for (int i = 0; i < m_mov; ++i) {
        mov += (double)w[i] * (double)h[i];
        sw += w[i];
        sh += h[i];
    }
    *count = 0;
    *filler_w = 0.0f;
    *filler_h = 0.0f;
    if (m_mov <= 0) return;
    float mw = (float)(sw / m_mov), mh = (float)(sh / m_mov);
    double fill = rho_t * (area - fixed) - mov;
    *filler_w = mw;
    *filler_h = mh;
    if (fill > 0.0) *count = (int64_t)floor(fill / ((double)mw * (double)mh));
}
