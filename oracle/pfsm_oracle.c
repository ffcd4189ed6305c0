/*
 * PFSM oracle: a plain, slow, FP64 CPU restatement of the partitioned folded spectrum method
 * (Briggs, Kelley, Bernholc, "Parallel implementation of electronic structure eigensolver using
 * a partitioned folded spectrum method", arXiv:1502.07806).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. The GPU library shares no code with it: no headers, no helpers, no
 * constants. Everything here is straight loops over row-major arrays; OpenMP is used only over
 * independent units (blocks, vectors, output rows), each of which is computed by one fixed
 * sequential loop, so results do not depend on the thread count.
 *
 * Readings where the paper is silent (each one also documented with the GPU library):
 *   R1  slices are contiguous in ascending previous-eigenvalue order; sizes floor(N/P), the first
 *       N mod P slices one larger (Section II, Fig. 1 assigns m = N/P eigenvectors per node).
 *   R2  each window is the slice plus `halo` indices on both sides, clamped to [0, N)
 *       (Section II: overlapping diagonal submatrices of order M = gamma N containing the slice);
 *       default halo = ceil(0.1 N), giving gamma ~ 0.3 at m ~ 0.1 N (Section II, last paragraph).
 *   R3  cluster snap: an interior slice boundary that falls inside a near-degenerate cluster
 *       (previous-eigenvalue gap < cluster_tol) moves to the nearest gap >= cluster_tol within a
 *       quarter of the neighbouring nominal slices, trying "down" before "up" at each distance.
 *   R4  a slice keeps the window eigenpairs whose ascending positions match the slice's own
 *       indices (Section II: submatrix eigenvectors start the iteration, eigenvalues are shifts).
 *   R5  sign of a start vector: its component at its own (home) index is made positive when its
 *       magnitude is >= 0.1, else its largest-magnitude component (lowest index on ties).
 *   R6  alpha_k = min(theta / d_k^2, 1 - 2^-20) with d_k = max(hi - eps_k, eps_k - lo) and
 *       [lo, hi] the Gershgorin interval of A: every factor 1 - alpha (lambda - eps)^2 then lies
 *       in [0, 1) (Eq. 7-11; the conditions printed as Eq. 8-9 lose their squares).
 *   R7  exactly K iterations of Eq. 11 with fixed shifts and no normalisation in between, each
 *       done as two matrix-vector products (Section II: no explicit square of A - eps I).
 *   R8  Gram-Schmidt: modified Gram-Schmidt in ascending index order (Section II); a vector whose
 *       norm after projection is < 1e-8 of its norm before stops the solve with NOT_SPD.
 *   R9  outputs: lambda_k = v_k^T A v_k (Rayleigh quotient), r_k = ||A v_k - lambda_k v_k||_2;
 *       index k stays tied to previous eigenpair k (no re-sorting).
 *
 * Status codes mirror the library's numbering but are defined here independently.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define OR_OK 0
#define OR_INVALID_ARG 1
#define OR_NOT_SPD 3
#define OR_NAN_INPUT 4
#define OR_NOT_CONVERGED 5

/* ------------------------------------------------------------------------------------------ */
/* Partition plan: slices and windows (Section II, Fig. 1; readings R1-R3).                    */
/* ------------------------------------------------------------------------------------------ */
int oracle_plan(int64_t n, int32_t nb, int32_t halo, double cluster_tol, const double *prev,
                const int32_t *slice_sizes, int32_t *k0, int32_t *m, int32_t *s, int32_t *w)
{
    if (n < 1 || nb < 1 || nb > n || n > 2147483647LL) return OR_INVALID_ARG;
    for (int64_t i = 0; i < n; i++) {
        if (isnan(prev[i]) || isinf(prev[i])) return OR_NAN_INPUT;
        if (i > 0 && prev[i] < prev[i - 1]) return OR_INVALID_ARG;   /* must be ascending */
    }
    int32_t *nom = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int64_t total = 0;
    for (int32_t b = 0; b < nb; b++) {
        if (slice_sizes) {
            nom[b] = slice_sizes[b];
            if (nom[b] < 1) { free(nom); return OR_INVALID_ARG; }
        } else {
            nom[b] = (int32_t)(n / nb) + (b < (int32_t)(n % nb) ? 1 : 0);
        }
        total += nom[b];
    }
    if (total != n) { free(nom); return OR_INVALID_ARG; }
    /* nominal starts */
    int32_t start = 0;
    for (int32_t b = 0; b < nb; b++) { k0[b] = start; start += nom[b]; }
    /* R3: snap interior boundaries, each decided from the nominal layout alone */
    for (int32_t b = 1; b < nb; b++) {
        int32_t k = k0[b];
        if (prev[k] - prev[k - 1] >= cluster_tol) continue;
        int32_t reach = (nom[b - 1] < nom[b] ? nom[b - 1] : nom[b]) / 4;
        for (int32_t d = 1; d <= reach; d++) {
            int32_t dn = k - d, up = k + d;
            if (dn >= 1 && prev[dn] - prev[dn - 1] >= cluster_tol) { k0[b] = dn; break; }
            if (up <= n - 1 && prev[up] - prev[up - 1] >= cluster_tol) { k0[b] = up; break; }
        }
    }
    int32_t h = halo < 0 ? (int32_t)((n + 9) / 10) : halo;
    for (int32_t b = 0; b < nb; b++) {
        int32_t end = (b + 1 < nb) ? k0[b + 1] : (int32_t)n;
        m[b] = end - k0[b];
        int64_t width = (int64_t)m[b] + 2 * (int64_t)h;
        w[b] = (int32_t)(width < n ? width : n);
        int64_t lo = (int64_t)k0[b] - h;
        if (lo < 0) lo = 0;
        if (lo > n - w[b]) lo = n - w[b];
        s[b] = (int32_t)lo;
    }
    free(nom);
    return OR_OK;
}

/* Gershgorin interval [lo, hi] containing every eigenvalue of A (used by reading R6). */
int oracle_gershgorin(int64_t n, const double *A, double *lo, double *hi)
{
    double l = INFINITY, u = -INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double r = 0.0;
        for (int64_t j = 0; j < n; j++) {
            double a = A[i * n + j];
            if (isnan(a) || isinf(a)) return OR_NAN_INPUT;
            if (j != i) r += fabs(a);
        }
        double d = A[i * n + i];
        if (d - r < l) l = d - r;
        if (d + r > u) u = d + r;
    }
    *lo = l;
    *hi = u;
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Dense symmetric eigensolver for one submatrix (the per-node LAPACK/MAGMA solve, Section II). */
/* Householder reduction to tridiagonal form, then the implicit symmetric QR iteration with a  */
/* Wilkinson shift (Golub & Van Loan, Matrix Computations, Sections 8.3.1-8.3.3), written out. */
/* w: eigenvalues ascending; Z: n x n row-major, column j the unit eigenvector of w[j].        */
/* ------------------------------------------------------------------------------------------ */
int oracle_symeig(int64_t n, const double *B, double *wout, double *Zout)
{
    if (n < 1) return OR_INVALID_ARG;
    double *a = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *q = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int status = OR_OK;
    memcpy(a, B, sizeof(double) * (size_t)(n * n));
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) q[i * n + j] = (i == j) ? 1.0 : 0.0;

    /* Householder tridiagonalisation: for column k, reflect a[k+1:, k] onto a multiple of e1. */
    for (int64_t k = 0; k + 2 < n; k++) {
        int64_t len = n - k - 1;
        double xnorm2 = 0.0;
        for (int64_t i = 0; i < len; i++) {
            double x = a[(k + 1 + i) * n + k];
            v[i] = x;
            xnorm2 += x * x;
        }
        double tail2 = xnorm2 - v[0] * v[0];
        if (tail2 == 0.0) continue;                       /* column already tridiagonal */
        double xnorm = sqrt(xnorm2);
        double alpha = (v[0] >= 0.0) ? -xnorm : xnorm;    /* avoid cancellation in v0 - alpha */
        v[0] -= alpha;
        double vtv = v[0] * v[0] + tail2;
        double beta = 2.0 / vtv;
        /* p = beta * A22 v */
        for (int64_t i = 0; i < len; i++) {
            double acc = 0.0;
            for (int64_t j = 0; j < len; j++) acc += a[(k + 1 + i) * n + (k + 1 + j)] * v[j];
            p[i] = beta * acc;
        }
        /* w = p - (beta p^T v / 2) v, stored back in p */
        double ptv = 0.0;
        for (int64_t i = 0; i < len; i++) ptv += p[i] * v[i];
        double kk = 0.5 * beta * ptv;
        for (int64_t i = 0; i < len; i++) p[i] -= kk * v[i];
        /* A22 <- A22 - v w^T - w v^T */
        for (int64_t i = 0; i < len; i++)
            for (int64_t j = 0; j < len; j++)
                a[(k + 1 + i) * n + (k + 1 + j)] -= v[i] * p[j] + p[i] * v[j];
        a[(k + 1) * n + k] = alpha;
        a[k * n + (k + 1)] = alpha;
        for (int64_t i = 1; i < len; i++) {
            a[(k + 1 + i) * n + k] = 0.0;
            a[k * n + (k + 1 + i)] = 0.0;
        }
        /* Q <- Q H, H = I - beta v v^T acting on columns k+1 .. n-1 */
        for (int64_t r = 0; r < n; r++) {
            double acc = 0.0;
            for (int64_t j = 0; j < len; j++) acc += q[r * n + (k + 1 + j)] * v[j];
            acc *= beta;
            for (int64_t j = 0; j < len; j++) q[r * n + (k + 1 + j)] -= acc * v[j];
        }
    }
    for (int64_t i = 0; i < n; i++) d[i] = a[i * n + i];
    for (int64_t i = 0; i + 1 < n; i++) e[i] = a[(i + 1) * n + i];
    if (n > 0) e[n - 1] = 0.0;

    /* Implicit QR on (d, e): chase a bulge down the unreduced block [lo, hi] after a Wilkinson
     * shift; rotations R (row_k' = c row_k + s row_k+1, row_k+1' = -s row_k + c row_k+1) are
     * applied as T <- R T R^T and accumulated as Q <- Q R^T. */
    int64_t hi = n - 1;
    int64_t iter = 0, max_iter = 60 * (n > 1 ? n : 1);
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= DBL_EPSILON * (fabs(d[hi - 1]) + fabs(d[hi])) ||
            fabs(e[hi - 1]) < DBL_MIN) {
            e[hi - 1] = 0.0;
            hi--;
            continue;
        }
        int64_t lo = hi - 1;
        while (lo > 0) {
            if (fabs(e[lo - 1]) <= DBL_EPSILON * (fabs(d[lo - 1]) + fabs(d[lo])) ||
                fabs(e[lo - 1]) < DBL_MIN) {
                e[lo - 1] = 0.0;
                break;
            }
            lo--;
        }
        if (++iter > max_iter) { status = OR_NOT_CONVERGED; break; }
        /* Wilkinson shift from the trailing 2x2 of the block */
        double delta = 0.5 * (d[hi - 1] - d[hi]);
        double eb = e[hi - 1];
        double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * hypot(delta, eb);
        double mu = d[hi] - eb * eb / den;
        double x = d[lo] - mu, z = e[lo];
        for (int64_t k = lo; k < hi; k++) {
            double r = hypot(x, z);
            double c = 1.0, s = 0.0;
            if (r != 0.0) { c = x / r; s = z / r; }
            if (k > lo) e[k - 1] = r;
            double dk = d[k], dk1 = d[k + 1], f = e[k];
            d[k] = c * c * dk + 2.0 * c * s * f + s * s * dk1;
            d[k + 1] = s * s * dk - 2.0 * c * s * f + c * c * dk1;
            e[k] = c * s * (dk1 - dk) + (c * c - s * s) * f;
            if (k + 1 < hi) {
                double bulge = s * e[k + 1];
                e[k + 1] = c * e[k + 1];
                x = e[k];
                z = bulge;
            }
            for (int64_t row = 0; row < n; row++) {
                double qk = q[row * n + k], qk1 = q[row * n + k + 1];
                q[row * n + k] = c * qk + s * qk1;
                q[row * n + k + 1] = -s * qk + c * qk1;
            }
        }
    }
    /* ascending order, stable (lower original index first on exact ties) */
    for (int64_t i = 0; i < n; i++) ord[i] = i;
    for (int64_t i = 1; i < n; i++) {
        int64_t t = ord[i];
        int64_t j = i - 1;
        while (j >= 0 && d[ord[j]] > d[t]) { ord[j + 1] = ord[j]; j--; }
        ord[j + 1] = t;
    }
    for (int64_t j = 0; j < n; j++) {
        wout[j] = d[ord[j]];
        for (int64_t i = 0; i < n; i++) Zout[i * n + j] = q[i * n + ord[j]];
    }
    free(a); free(q); free(v); free(p); free(d); free(e); free(ord);
    return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Folded-spectrum iteration, Eq. 11 (reading R7). X holds `cnt` vectors as rows (cnt x n);    */
/* vector k uses shift eps[k] and step alpha[k]. Each iteration is two products with A.        */
/* ------------------------------------------------------------------------------------------ */
void oracle_fs_iterate(int64_t n, int64_t cnt, const double *A, double *X, const double *eps,
                       const double *alpha, int32_t iters)
{
#pragma omp parallel
    {
        double *y = (double *)malloc(sizeof(double) * (size_t)n);
        double *z = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < cnt; k++) {
            double *x = X + k * n;
            for (int32_t it = 0; it < iters; it++) {
                for (int64_t i = 0; i < n; i++) {            /* y = (A - eps I) x */
                    double acc = 0.0;
                    for (int64_t j = 0; j < n; j++) acc += A[i * n + j] * x[j];
                    y[i] = acc - eps[k] * x[i];
                }
                for (int64_t i = 0; i < n; i++) {            /* z = (A - eps I) y */
                    double acc = 0.0;
                    for (int64_t j = 0; j < n; j++) acc += A[i * n + j] * y[j];
                    z[i] = acc - eps[k] * y[i];
                }
                for (int64_t i = 0; i < n; i++) x[i] -= alpha[k] * z[i];
            }
        }
        free(y);
        free(z);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Adaptive variant of Eq. 11 (not in the paper, which fixes the shift and the count): each    */
/* iteration first moves every shift to the Rayleigh quotient of its vector and measures the   */
/* residual, then takes the Eq. 11 step with the new shift:                                     */
/*   y = (A - eps I) x;  delta = x.y / x.x;  eps += delta;  y -= delta x   (y = (A - eps I) x); */
/*   alpha = min(theta / d^2, 1 - 2^-20), d = max(ghi - eps, eps - glo);  r = ||y|| / ||x||;   */
/*   stop when max_k r_k <= tol_abs (before the step) or after max_iters steps;                */
/*   x -= alpha (A - eps I) y.                                                                  */
/* X: cnt x n rows; eps, alpha updated in place. *iters = steps done, *resid = the last        */
/* max_k r_k. Returns OR_OK (tolerance met) or OR_NOT_CONVERGED (max_iters reached).          */
/* ------------------------------------------------------------------------------------------ */
int oracle_fs_iterate_adaptive(int64_t n, int64_t cnt, const double *A, double *X, double *eps, double *alpha,
                               int32_t max_iters, double tol_abs, double theta, double glo, double ghi,
                               int32_t *iters, double *resid)
{
    double *Y = (double *)malloc(sizeof(double) * (size_t)(cnt * n));
    double *r = (double *)malloc(sizeof(double) * (size_t)cnt);
    int status = OR_NOT_CONVERGED;
    int32_t it = 0;
    double rmax = 0.0;
    for (;;) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t k = 0; k < cnt; k++) {
            const double *xr = X + k * n;
            double *yr = Y + k * n;
            for (int64_t i = 0; i < n; i++) {                /* y = (A - eps I) x */
                double acc = 0.0;
                for (int64_t c = 0; c < n; c++) acc += A[i * n + c] * xr[c];
                yr[i] = acc - eps[k] * xr[i];
            }
            double xy = 0.0, xx = 0.0;
            for (int64_t i = 0; i < n; i++) { xy += xr[i] * yr[i]; xx += xr[i] * xr[i]; }
            const double delta = xy / xx;                    /* Rayleigh quotient - eps */
            eps[k] += delta;
            double dmax = ghi - eps[k];                      /* the step size follows the shift */
            if (eps[k] - glo > dmax) dmax = eps[k] - glo;
            const double a = theta / (dmax * dmax), cap = 1.0 - ldexp(1.0, -20);
            alpha[k] = (a < cap) ? a : cap;
            double yy = 0.0;
            for (int64_t i = 0; i < n; i++) { yr[i] -= delta * xr[i]; yy += yr[i] * yr[i]; }
            r[k] = sqrt(yy / xx);
        }
        rmax = 0.0;
        for (int64_t k = 0; k < cnt; k++) rmax = fmax(rmax, r[k]);
        if (rmax <= tol_abs) { status = OR_OK; break; }
        if (it >= max_iters) break;
#pragma omp parallel
        {
            double *z = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
            for (int64_t k = 0; k < cnt; k++) {
                double *xr = X + k * n;
                const double *yr = Y + k * n;
                for (int64_t i = 0; i < n; i++) {            /* z = (A - eps I) y */
                    double acc = 0.0;
                    for (int64_t c = 0; c < n; c++) acc += A[i * n + c] * yr[c];
                    z[i] = acc - eps[k] * yr[i];
                }
                for (int64_t i = 0; i < n; i++) xr[i] -= alpha[k] * z[i];
            }
            free(z);
        }
        it++;
    }
    free(Y);
    free(r);
    *iters = it;
    *resid = rmax;
    return status;
}

/* Modified Gram-Schmidt over the rows of X (cnt x n), ascending index order (reading R8).     */
/* The right-looking form below performs, for every vector, the same ordered sequence of       */
/* projections as the textbook left-looking loop, so it is the same arithmetic.               */
int oracle_mgs(int64_t n, int64_t cnt, double *X, double *rdiag)
{
    double *norm0 = (double *)malloc(sizeof(double) * (size_t)cnt);
    int status = OR_OK;
    for (int64_t k = 0; k < cnt; k++) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; i++) acc += X[k * n + i] * X[k * n + i];
        norm0[k] = sqrt(acc);
    }
    for (int64_t k = 0; k < cnt; k++) {
        double *qk = X + k * n;
        double acc = 0.0;
        for (int64_t i = 0; i < n; i++) acc += qk[i] * qk[i];
        double r = sqrt(acc);
        if (rdiag) rdiag[k] = r;
        if (!(r >= 1e-8 * norm0[k]) || r == 0.0) { status = OR_NOT_SPD; break; }
        for (int64_t i = 0; i < n; i++) qk[i] /= r;
#pragma omp parallel for schedule(static)
        for (int64_t j = k + 1; j < cnt; j++) {
            double *xj = X + j * n;
            double c = 0.0;
            for (int64_t i = 0; i < n; i++) c += qk[i] * xj[i];
            for (int64_t i = 0; i < n; i++) xj[i] -= c * qk[i];
        }
    }
    free(norm0);
    return status;
}

/* Rayleigh quotients and residual norms of unit vectors held as rows of Q (reading R9). */
void oracle_rayleigh(int64_t n, int64_t cnt, const double *A, const double *Q, double *lam,
                     double *res)
{
#pragma omp parallel
    {
        double *wv = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < cnt; k++) {
            const double *q = Q + k * n;
            for (int64_t i = 0; i < n; i++) {
                double acc = 0.0;
                for (int64_t j = 0; j < n; j++) acc += A[i * n + j] * q[j];
                wv[i] = acc;
            }
            double l = 0.0;
            for (int64_t i = 0; i < n; i++) l += q[i] * wv[i];
            double r = 0.0;
            for (int64_t i = 0; i < n; i++) {
                double t = wv[i] - l * q[i];
                r += t * t;
            }
            lam[k] = l;
            if (res) res[k] = sqrt(r);
        }
        free(wv);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Whole PFSM solve (Section II).                                                             */
/* Outputs (all optional except lam/V): lam[N]; V N x N row-major with V[:, k] vector k;       */
/* res[N]; xfs N x N in V's layout holding the vectors after the FS iterations and before      */
/* Gram-Schmidt; eps[N], alpha[N]; plan[4*nb] = (k0, m, s, M) per block.                      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t halo;
    int32_t fs_iters;            /* Eq. 11 iterations (the cap with fs_adaptive) */
    double alpha_theta;
    double cluster_tol;
    const int32_t *slice_sizes;
    int32_t fs_adaptive;         /* 0: Eq. 11 as printed; 1: oracle_fs_iterate_adaptive */
    double fs_tol;               /* its residual tolerance, relative to max(|glo|, |ghi|) */
} oracle_params_t;

int oracle_pfsm(int64_t n, int32_t nb, const oracle_params_t *prm, const double *A,
                const double *prev, double *lam, double *V, double *res, double *xfs,
                double *eps_out, double *alpha_out, int32_t *plan_out)
{
    int32_t *k0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb * 4);
    int32_t *m = k0 + nb, *s = k0 + 2 * nb, *w = k0 + 3 * nb;
    int st = oracle_plan(n, nb, prm->halo, prm->cluster_tol, prev, prm->slice_sizes, k0, m, s, w);
    if (st != OR_OK) { free(k0); return st; }
    if (prm->fs_iters < 0 || !(prm->alpha_theta > 0.0)) { free(k0); return OR_INVALID_ARG; }
    if (plan_out) memcpy(plan_out, k0, sizeof(int32_t) * (size_t)nb * 4);
    double glo, ghi;
    st = oracle_gershgorin(n, A, &glo, &ghi);
    if (st != OR_OK) { free(k0); return st; }

    double *X = (double *)calloc((size_t)(n * n), sizeof(double));   /* rows = vectors */
    double *ep = (double *)malloc(sizeof(double) * (size_t)n);
    double *al = (double *)malloc(sizeof(double) * (size_t)n);
    int bad = OR_OK;

    /* Submatrix solves, start vectors, shifts (Section II; readings R4-R6) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t b = 0; b < nb; b++) {
        int64_t M = w[b];
        double *sub = (double *)malloc(sizeof(double) * (size_t)(M * M));
        double *mu = (double *)malloc(sizeof(double) * (size_t)M);
        double *Y = (double *)malloc(sizeof(double) * (size_t)(M * M));
        for (int64_t i = 0; i < M; i++)
            for (int64_t j = 0; j < M; j++) sub[i * M + j] = A[(s[b] + i) * n + (s[b] + j)];
        int rs = oracle_symeig(M, sub, mu, Y);
        if (rs != OR_OK) {
#pragma omp critical
            bad = rs;
        }
        for (int32_t t = 0; t < m[b]; t++) {
            int64_t k = k0[b] + t;            /* global eigen-index */
            int64_t col = k - s[b];           /* its ascending position inside the window */
            int64_t home = k - s[b];          /* its own row inside the window */
            double flip = 1.0;
            double yh = Y[home * M + col];
            if (fabs(yh) >= 0.1) {
                flip = (yh < 0.0) ? -1.0 : 1.0;
            } else {
                int64_t arg = 0;
                double best = -1.0;
                for (int64_t i = 0; i < M; i++) {
                    double av = fabs(Y[i * M + col]);
                    if (av > best) { best = av; arg = i; }
                }
                flip = (Y[arg * M + col] < 0.0) ? -1.0 : 1.0;
            }
            for (int64_t i = 0; i < M; i++) X[k * n + s[b] + i] = flip * Y[i * M + col];
            ep[k] = mu[col];
            double dmax = ghi - ep[k];
            if (ep[k] - glo > dmax) dmax = ep[k] - glo;
            double a = prm->alpha_theta / (dmax * dmax);
            double cap = 1.0 - ldexp(1.0, -20);
            al[k] = (a < cap) ? a : cap;
        }
        free(sub); free(mu); free(Y);
    }
    if (bad != OR_OK) { st = bad; goto done; }

    /* Eq. 11, K times (or the adaptive variant, at most K steps) */
    if (prm->fs_adaptive) {
        int32_t fit;
        double fres;
        oracle_fs_iterate_adaptive(n, n, A, X, ep, al, prm->fs_iters, prm->fs_tol * fmax(fabs(glo), fabs(ghi)),
                                   prm->alpha_theta, glo, ghi, &fit, &fres);
    } else {
        oracle_fs_iterate(n, n, A, X, ep, al, prm->fs_iters);
    }
    if (eps_out) memcpy(eps_out, ep, sizeof(double) * (size_t)n);
    if (alpha_out) memcpy(alpha_out, al, sizeof(double) * (size_t)n);
    if (xfs)
        for (int64_t i = 0; i < n; i++)
            for (int64_t k = 0; k < n; k++) xfs[i * n + k] = X[k * n + i];

    /* Gram-Schmidt over all N vectors */
    st = oracle_mgs(n, n, X, NULL);
    if (st != OR_OK) goto done;

    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_rayleigh(n, n, A, X, lam, r);
    if (res) memcpy(res, r, sizeof(double) * (size_t)n);
    free(r);
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = 0; k < n; k++) V[i * n + k] = X[k * n + i];
done:
    free(X); free(ep); free(al); free(k0);
    return st;
}

/* ------------------------------------------------------------------------------------------ */
/* Eigen-adjoint (not in the paper): dA = sym( V (diag(dLam) + F o (V^T dV)) V^T ),            */
/* F_ij = 1/(lam_j - lam_i) for i != j and |lam_i - lam_j| >= tau, else 0.                    */
/* V, dV, dA: n x n row-major; V[:, k] = vector k.                                            */
/* ------------------------------------------------------------------------------------------ */
void oracle_backward(int64_t n, const double *V, const double *lam, const double *dlam,
                     const double *dV, double tau, double *dA)
{
    double *G = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *T = (double *)malloc(sizeof(double) * (size_t)(n * n));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)              /* G = V^T dV, then the masked Hadamard */
        for (int64_t j = 0; j < n; j++) {
            double acc = 0.0;
            for (int64_t r = 0; r < n; r++) acc += V[r * n + i] * dV[r * n + j];
            double g;
            if (i == j) {
                g = dlam ? dlam[i] : 0.0;
            } else {
                double gap = lam[j] - lam[i];
                g = (fabs(gap) >= tau) ? acc / gap : 0.0;
            }
            G[i * n + j] = g;
        }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)              /* T = V G */
        for (int64_t j = 0; j < n; j++) {
            double acc = 0.0;
            for (int64_t r = 0; r < n; r++) acc += V[i * n + r] * G[r * n + j];
            T[i * n + j] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)              /* dA = T V^T */
        for (int64_t j = 0; j < n; j++) {
            double acc = 0.0;
            for (int64_t r = 0; r < n; r++) acc += T[i * n + r] * V[j * n + r];
            dA[i * n + j] = acc;
        }
    for (int64_t i = 0; i < n; i++)              /* symmetric part */
        for (int64_t j = i + 1; j < n; j++) {
            double sym = 0.5 * (dA[i * n + j] + dA[j * n + i]);
            dA[i * n + j] = sym;
            dA[j * n + i] = sym;
        }
    free(G);
    free(T);
}

/* ------------------------------------------------------------------------------------------ */
/* Generalized -> standard conversion, Eq. 14-15 (not on the eigensolver's hot path: the step */
/* before it). A x = lambda B x with B diagonally dominant; Z = B^{-1} A by the Jacobi        */
/* iteration of Eq. 14,  Z_{n+1} = (I - D^{-1} B) Z_n + D^{-1} A,  D = diag(B), written as     */
/* Z_{n+1} = Z_n + D^{-1} (A - B Z_n), from Z_0 = 0 (so Z_1 = D^{-1} A: the identity-like     */
/* first approximation of B^{-1} the paper describes). Before each update the residual        */
/* R_n = A - B Z_n is measured; the iteration stops when max|R_n| <= tol max|A| or after       */
/* max_iters updates. A, B, Z: n x n row-major. *iters = updates done, *resid = max|R| /       */
/* max|A| of the returned Z. Returns OR_OK, OR_NOT_CONVERGED (Z = last iterate) or             */
/* OR_INVALID_ARG (a zero diagonal entry of B).                                               */
/* ------------------------------------------------------------------------------------------ */
int oracle_gen_to_std(int64_t n, const double *A, const double *B, double *Z, int32_t max_iters,
                      double tol, int32_t *iters, double *resid)
{
    for (int64_t i = 0; i < n; i++)
        if (B[i * n + i] == 0.0) return OR_INVALID_ARG;
    double amax = 0.0;
    for (int64_t i = 0; i < n * n; i++) amax = fmax(amax, fabs(A[i]));
    if (amax == 0.0) amax = 1.0;
    double *R = (double *)malloc(sizeof(double) * (size_t)(n * n));
    for (int64_t i = 0; i < n * n; i++) Z[i] = 0.0;
    int status = OR_NOT_CONVERGED;
    int32_t it = 0;
    double r = 0.0;
    for (;;) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)              /* R = A - B Z */
            for (int64_t j = 0; j < n; j++) {
                double acc = 0.0;
                for (int64_t k = 0; k < n; k++) acc += B[i * n + k] * Z[k * n + j];
                R[i * n + j] = A[i * n + j] - acc;
            }
        r = 0.0;
        for (int64_t i = 0; i < n * n; i++) r = fmax(r, fabs(R[i]));
        r /= amax;
        if (r <= tol) { status = OR_OK; break; }
        if (it >= max_iters) break;
        for (int64_t i = 0; i < n; i++)              /* Z += D^{-1} R */
            for (int64_t j = 0; j < n; j++) Z[i * n + j] += R[i * n + j] / B[i * n + i];
        it++;
    }
    free(R);
    *iters = it;
    *resid = r;
    return status;
}

/* C = X Y for n x n row-major matrices (plain loops). */
static void or_matmul(int64_t n, const double *X, const double *Y, double *C)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) {
            double acc = 0.0;
            for (int64_t k = 0; k < n; k++) acc += X[i * n + k] * Y[k * n + j];
            C[i * n + j] = acc;
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Symmetric form of the conversion (a deviation from Eq. 14-15: the eigensolver needs a      */
/* symmetric matrix and B^{-1} A is not one): C = B^{-1/2} A B^{-1/2}, whose eigenvalues are   */
/* those of B^{-1} A and whose eigenvectors y give the generalized ones as x = B^{-1/2} y      */
/* (B-orthonormal). S = B^{-1/2} by the coupled Newton-Schulz iteration for the matrix square */
/* root and its inverse (Higham, Functions of Matrices, 2008): with c = the largest Gershgorin */
/* row bound of B (so the eigenvalues of B / c lie in (0, 1]),                               */
/*   Y_0 = B / c, Q_0 = I;  P_k = Q_k Y_k;  T_k = (3 I - P_k) / 2;  Y_{k+1} = Y_k T_k;          */
/*   Q_{k+1} = T_k Q_k,                                                                        */
/* Y_k -> (B/c)^{1/2}, Q_k -> (B/c)^{-1/2}; it stops when max|I - P_k| <= tol (checked before  */
/* each update) or after max_iters updates; then S = Q / sqrt(c) and C = S A S. A, B, C, S:    */
/* n x n row-major. *iters = updates done, *resid = max|I - P| at the stop. Returns OR_OK,     */
/* OR_NOT_CONVERGED or OR_NOT_SPD (a row bound c <= 0).                                       */
/* ------------------------------------------------------------------------------------------ */
int oracle_gen_to_std_sym(int64_t n, const double *A, const double *B, double *C, double *S,
                          int32_t max_iters, double tol, int32_t *iters, double *resid)
{
    double c = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double row = 0.0;
        for (int64_t j = 0; j < n; j++) row += fabs(B[i * n + j]);
        c = fmax(c, row);
    }
    if (!(c > 0.0)) return OR_NOT_SPD;
    const size_t sz = sizeof(double) * (size_t)(n * n);
    double *Y = (double *)malloc(sz), *Q = (double *)malloc(sz), *P = (double *)malloc(sz);
    double *T = (double *)malloc(sz), *W = (double *)malloc(sz);
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) {
            Y[i * n + j] = B[i * n + j] / c;
            Q[i * n + j] = (i == j) ? 1.0 : 0.0;
        }
    int status = OR_NOT_CONVERGED;
    int32_t it = 0;
    double r = 0.0;
    for (;;) {
        or_matmul(n, Q, Y, P);                       /* P = Q Y */
        r = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++) r = fmax(r, fabs(((i == j) ? 1.0 : 0.0) - P[i * n + j]));
        if (r <= tol) { status = OR_OK; break; }
        if (it >= max_iters) break;
        for (int64_t i = 0; i < n; i++)              /* T = (3 I - P) / 2 */
            for (int64_t j = 0; j < n; j++) T[i * n + j] = 0.5 * (((i == j) ? 3.0 : 0.0) - P[i * n + j]);
        or_matmul(n, Y, T, W);                       /* Y = Y T */
        memcpy(Y, W, sz);
        or_matmul(n, T, Q, W);                       /* Q = T Q */
        memcpy(Q, W, sz);
        it++;
    }
    const double isc = 1.0 / sqrt(c);
    for (int64_t i = 0; i < n * n; i++) S[i] = Q[i] * isc;
    or_matmul(n, S, A, W);                           /* C = S A S */
    or_matmul(n, W, S, C);
    free(Y); free(Q); free(P); free(T); free(W);
    *iters = it;
    *resid = r;
    return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Diagonal-dominance guard (Section II: the method needs A diagonally dominant, and the      */
/* paper diagonalizes conventionally for the first SCF steps). The paper gives no formula;    */
/* the reading used here: g = max_i sqrt(sum_{j != i} A_ij^2) / (max_i A_ii - min_i A_ii),    */
/* the largest l2 coupling of a basis state relative to the spread of the diagonal (zero      */
/* spread: g = 0 if A is diagonal, else +inf).                                                */
/* ------------------------------------------------------------------------------------------ */
void oracle_guard(int64_t n, const double *A, double *g)
{
    double cmax = 0.0, dmin = INFINITY, dmax = -INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < n; j++)
            if (j != i) s += A[i * n + j] * A[i * n + j];
        cmax = fmax(cmax, sqrt(s));
        dmin = fmin(dmin, A[i * n + i]);
        dmax = fmax(dmax, A[i * n + i]);
    }
    const double spread = dmax - dmin;
    *g = (spread > 0.0) ? cmax / spread : ((cmax > 0.0) ? INFINITY : 0.0);
}

/* ------------------------------------------------------------------------------------------ */
/* Full diagonalization, the conventional step the paper uses instead of the method for the   */
/* first SCF steps: every eigenpair of A (oracle_symeig), each vector signed by the start-     */
/* vector rule with the whole matrix as its window (home component k positive when            */
/* |y_k| >= 0.1, else the largest component positive), then the Rayleigh quotients and        */
/* residuals of oracle_rayleigh. Outputs as oracle_pfsm: lam[N], V N x N with V[:, k] vector  */
/* k, res[N]. Equivalent to the method with one block covering A and no Eq. 11 iterations.    */
/* ------------------------------------------------------------------------------------------ */
int oracle_full(int64_t n, const double *A, double *lam, double *V, double *res)
{
    double *mu = (double *)malloc(sizeof(double) * (size_t)n);
    double *Y = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *X = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    int st = oracle_symeig(n, A, mu, Y);
    if (st == OR_OK) {
        for (int64_t k = 0; k < n; k++) {
            double flip, yh = Y[k * n + k];
            if (fabs(yh) >= 0.1) {
                flip = (yh >= 0.0) ? 1.0 : -1.0;
            } else {
                int64_t arg = 0;
                double best = -1.0;
                for (int64_t i = 0; i < n; i++) {
                    double av = fabs(Y[i * n + k]);
                    if (av > best) { best = av; arg = i; }
                }
                flip = (Y[arg * n + k] < 0.0) ? -1.0 : 1.0;
            }
            for (int64_t i = 0; i < n; i++) X[k * n + i] = flip * Y[i * n + k];
        }
        oracle_rayleigh(n, n, A, X, lam, r);
        if (res) memcpy(res, r, sizeof(double) * (size_t)n);
        for (int64_t i = 0; i < n; i++)
            for (int64_t k = 0; k < n; k++) V[i * n + k] = X[k * n + i];
    }
    free(mu); free(Y); free(X); free(r);
    return st;
}
