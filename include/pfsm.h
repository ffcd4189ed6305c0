/*
 * pfsm.h -- C ABI of the B300 (sm_103a) partitioned folded spectrum method (PFSM) library.
 *
 * The method (Briggs, Kelley, Bernholc, arXiv:1502.07806, Section II) finds all N eigenpairs
 * of a real symmetric N x N matrix A that is nearly diagonal in the previous SCF step's
 * eigenbasis (the reduced subspace Hamiltonian of Eq. 3):
 *   1. split the eigen-indices into contiguous slices (Fig. 1, m = N/P per slice);
 *   2. for each slice, solve the overlapping diagonal submatrix B = A[s:s+M, s:s+M] that
 *      contains it (M = gamma N);
 *   3. zero-pad the slice's submatrix eigenvectors to length N; they start Eq. 11 with the
 *      submatrix eigenvalues as shifts eps;
 *   4. iterate Eq. 11, x <- x - alpha (A - eps I)^2 x, as two matrix products per iteration;
 *   5. orthonormalise all N vectors (Gram-Schmidt, ascending index order).
 * Outputs are Rayleigh quotients lambda_k = v_k^T A v_k and unit vectors v_k.
 *
 * Conventions for every call:
 *   - All matrix/vector pointers are DEVICE pointers to FP64 data unless stated otherwise.
 *     Matrices are dense, row-major, N x N, leading dimension N. V_out[i*N + k] is component i
 *     of eigenvector k (column k is vector k, as in torch.linalg.eigh).
 *   - The caller owns every buffer it passes. The handle owns its workspace (allocated once in
 *     pfsm_init with cudaMalloc, freed in pfsm_destroy) and keeps the last solve's (lambda, V)
 *     for pfsm_backward.
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream). Every kernel of a
 *     call is enqueued on that stream; calls return without synchronising, except
 *     pfsm_get_status.
 *   - Return value: PFSM_OK or a pfsm_status_t error. Argument errors and launch errors are
 *     reported synchronously; conditions the GPU detects while running (NaN input, an
 *     unsorted prev_eigvals, a Gram-Schmidt breakdown, ...) are recorded in a device status
 *     word that pfsm_get_status reads. No call exits, traps or waits without bound.
 *   - pfsm_last_error() returns a thread-local message describing the most recent failure.
 *
 * Readings of the paper fixed by this library (identical in the test oracle):
 *   slices: sizes floor(N/P), the first N mod P one larger, unless slice_sizes is given;
 *   windows: slice plus `halo` rows each side, clamped to [0, N) (Section II; default halo
 *     ceil(0.1 N) gives gamma ~ 0.3 at m ~ 0.1 N, the working rule at the end of Section II);
 *   cluster snap: an interior slice boundary inside a near-degenerate cluster of
 *     prev_eigvals (gap < cluster_tol) moves to the nearest gap >= cluster_tol within a quarter
 *     of the neighbouring nominal slices ("down" before "up" at each distance);
 *   start vectors: the window eigenpairs at the slice indices' own ascending positions; sign
 *     chosen so the home component is positive (largest component if the home one is < 0.1);
 *   alpha_k = min(alpha_theta / d_k^2, 1 - 2^-20), d_k = max(hi - eps_k, eps_k - lo), [lo, hi]
 *     the Gershgorin interval of A (keeps 1 - alpha (lambda - eps)^2 in [0, 1], Eq. 7-11);
 *   exactly fs_iters iterations of Eq. 11, fixed shifts, no normalisation in between;
 *   Gram-Schmidt done as Cholesky-QR (S = X^T X = R^T R, V = X R^-1), equal in exact arithmetic
 *     to Gram-Schmidt in ascending index order; a vector whose norm after projection falls
 *     below 1e-8 of its norm before is a breakdown (PFSM_ERR_NOT_SPD);
 *   eigenvalue k stays tied to previous index k: outputs are not re-sorted.
 */
#ifndef PFSM_H
#define PFSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfsm_handle_s *pfsm_handle_t;

typedef enum {
    PFSM_OK = 0,
    PFSM_ERR_INVALID_ARG = 1,   /* bad size, null pointer, parameter out of range, prev_eigvals
                                   not ascending (device-detected) */
    PFSM_ERR_CUDA = 2,          /* a CUDA runtime call failed; see pfsm_last_error() */
    PFSM_ERR_NOT_SPD = 3,       /* Gram-Schmidt breakdown: overlap matrix not positive definite */
    PFSM_ERR_NAN_INPUT = 4,     /* A or prev_eigvals holds NaN or Inf */
    PFSM_ERR_NOT_CONVERGED = 5, /* a submatrix eigensolve did not converge, or an iterative
                                   conversion missed its tolerance */
    PFSM_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    PFSM_ERR_NO_SOLVE = 7,      /* pfsm_backward called before any pfsm_solve on the handle */
    PFSM_ERR_OUT_OF_MEMORY = 8  /* workspace allocation failed in pfsm_init */
} pfsm_status_t;

typedef enum {
    PFSM_FP64 = 0,        /* every product in FP64 (DFMA) */
    PFSM_TF32_SPLIT = 1,  /* Eq. 11 products on tcgen05 tensor cores in split TF32, FP32
                             accumulation, FP64 diagonal part and FP64 residual correction */
    PFSM_BF16_SPLIT = 2   /* as PFSM_TF32_SPLIT with three-way BF16 splitting */
} pfsm_precision_t;

typedef struct {
    int32_t halo;          /* rows added on each side of a slice; < 0 selects ceil(0.1 N) */
    int32_t fs_iters;      /* K >= 0 iterations of Eq. 11 (default 3) */
    double alpha_theta;    /* theta > 0 in alpha_k = min(theta / d_k^2, 1 - 2^-20) (default 1) */
    double cluster_tol;    /* slice-boundary snap gap, absolute (default 1e-5; 0 disables) */
    double degen_tol;      /* backward: pairs with |lambda_i - lambda_j| < degen_tol get no
                              eigenvector coupling term (default 1e-8) */
    int32_t precision;     /* pfsm_precision_t (default PFSM_FP64) */
    int32_t recompute_v;   /* backward recomputes (lambda, V) from the last A instead of
                              using the kept copy (default 0) */
    const int32_t *slice_sizes; /* HOST array of nblocks sizes summing to N, or NULL */
    double guard_max;      /* diagonal-dominance guard (Section II: the method needs A
                              diagonally dominant): a solve whose A has
                              g = max_i ||A_{i,:} without A_ii||_2 / (max_i A_ii - min_i A_ii)
                              above guard_max is a full diagonalization instead; <= 0 disables
                              (default 0). Measuring g synchronises the solve's stream. */
    int32_t full_steps;    /* the first full_steps solves on the handle are full
                              diagonalizations (the paper's conventional first SCF steps;
                              default 0). A full diagonalization (cuSOLVER syevd) gives the same
                              outputs as the method: vectors signed by the start-vector rule,
                              Rayleigh quotients, residuals, V; pfsm_backward works after it. */
    int32_t fs_adaptive;   /* not in the paper: 1 replaces the fixed Eq. 11 count by steps that
                              first move every shift to its vector's Rayleigh quotient (and the
                              step size alpha with it) and stop once max_k ||(A - eps_k) x_k|| /
                              ||x_k|| <= fs_tol * ||A||_Gershgorin, fs_iters steps at most; runs
                              its products in FP64 in every precision; one residual read-back (a
                              stream synchronisation) per step (default 0) */
    double fs_tol;         /* its tolerance (default 0: the cap decides) */
    int32_t reduction;     /* how the mixed forms reduce each window to tridiagonal form before
                              its eigenpairs (Section II's submatrix eigensolves; same result up
                              to rounding): 0 automatic (two-stage for windows of 1024 rows or
                              more), 1 one-stage Householder on the FP64 pipe, 2 two-stage: dense
                              to band (half-width 32) with FP64-accurate digit products on the
                              tensor cores, band to tridiagonal by FP64 bulge chasing. The FP64
                              form always reduces in one stage (default 0) */
} pfsm_params_t;

/* Fills *p with the defaults listed above. */
void pfsm_default_params(pfsm_params_t *p);

/* Creates a handle for N x N problems split into nblocks slices (1 <= nblocks <= N).
 * p may be NULL (defaults). Allocates all device workspace on the current device. A handle of
 * the mixed forms also creates one internal stream: a solve forks work that needs only A or only
 * the window reduction onto it and joins it back before the call's later work, so callers see
 * ordinary stream order (and a solve captured into a CUDA graph captures both streams).
 * Returns PFSM_ERR_INVALID_ARG for bad sizes/params, PFSM_ERR_OUT_OF_MEMORY or PFSM_ERR_CUDA. */
int pfsm_init(int64_t N, int32_t nblocks, const pfsm_params_t *p, pfsm_handle_t *out);

/* One PFSM solve (Section II, steps 1-5).
 *   A            device, N x N FP64, symmetric (the full matrix is read, not symmetrised)
 *   prev_eigvals device, N FP64, ascending: the previous step's eigenvalues; they order the
 *                eigen-indices and place the slice boundaries
 *   eigvals_out  device, N FP64: Rayleigh quotient of vector k at index k (not re-sorted)
 *   V_out        device, N x N FP64: V_out[i*N + k] = component i of vector k
 * A and prev_eigvals must stay valid until the stream reaches the end of the call. In the mixed
 * forms an eager solve (not being captured into a CUDA graph) reads one 8-byte value back in its
 * Gram-Schmidt phase (a stream synchronisation) to choose the preconditioner's path. */
int pfsm_solve(pfsm_handle_t h, const double *A, const double *prev_eigvals,
               double *eigvals_out, double *V_out, void *stream);

/* Eigen-adjoint of the last solve on h (not in the paper): for a loss L(lambda, V),
 *   dA = sym( V (diag(dLambda) + F o (V^T dV)) V^T ),  F_ij = 1/(lambda_j - lambda_i)
 * for i != j with |lambda_i - lambda_j| >= degen_tol, else 0; sym(X) = (X + X^T)/2.
 *   dLambda  device, N FP64, or NULL (treated as zeros)
 *   dV       device, N x N FP64 in V_out's layout, or NULL (treated as zeros)
 *   dA_out   device, N x N FP64, written in full (symmetric)
 * With recompute_v set, (lambda, V) are recomputed from the A of the last solve, which must
 * still be valid. The FP64 form computes the three N x N products on the FP64 pipe; the mixed
 * forms (PFSM_TF32_SPLIT, PFSM_BF16_SPLIT) compute them as FP64-accurate digit products on the
 * tensor cores (each about sqrt(N) 2^-49 of its operand rows' largest entries, the rounding of
 * an FP64 product). Returns PFSM_ERR_NO_SOLVE if h has not solved yet. */
int pfsm_backward(pfsm_handle_t h, const double *dLambda, const double *dV, double *dA_out,
                  void *stream);

/* Synchronises the stream of the last call on h and returns the device status word of that
 * call (PFSM_OK or a device-detected pfsm_status_t) in *device_status (host pointer).
 * The status word is cleared at the start of every solve. */
int pfsm_get_status(pfsm_handle_t h, int32_t *device_status);

/* One step of the SCF loop the method assumes (its input "similar to the previous iteration",
 * Sec. I): the Hamiltonian H (N x N symmetric, any fixed basis) is rotated into the previous
 * eigenbasis, A = sym(Vb^T H Vb) with Vb (N x N row-major, columns = basis vectors), A is solved
 * on h exactly as pfsm_solve does (its precision, first-steps rule and guard apply; lam_prev is
 * prev_eigvals, ascending), and then Vb <- Vb V (in place) and lam_out <- the eigenvalues, so
 * Vb's columns are the eigenvector estimates of H in its own basis. The rotation and update are
 * FP64-accurate digit products; temporaries come from cudaMallocAsync on `stream`. Start a loop
 * with Vb = I, lam_prev = 0 and full_steps >= 1 (H_0 is generally not diagonally dominant).
 * Diagnostics afterwards describe the solve of A; pfsm_backward needs recompute_v = 0 after it. */
int pfsm_scf_step(pfsm_handle_t h, const double *H, double *Vb, const double *lam_prev, double *lam_out,
                  void *stream);

/* Diagnostics of the last solve, copied on `stream` into caller device buffers:
 *   which = 0: residual norms r_k = ||A v_k - lambda_k v_k||_2          (N doubles)
 *   which = 1: vectors after the Eq. 11 iterations, before Gram-Schmidt (N x N, V layout)
 *   which = 2: shifts eps_k                                             (N doubles)
 *   which = 3: step sizes alpha_k                                       (N doubles)
 *   which = 4: the partition plan as 4*nblocks int32 (k0[], m[], s[], M[]) reinterpreted
 *              into the first 2*nblocks doubles' bytes
 * Returns PFSM_ERR_INVALID_ARG for an unknown `which`, PFSM_ERR_NO_SOLVE before a solve. */
int pfsm_get_diagnostic(pfsm_handle_t h, int32_t which, void *out, void *stream);

/* ---- batches of independent problems (k-points / spin channels of one SCF step) ---------
 * Not in the paper. A batch owns one workspace per problem and a set of internal streams;
 * problems are assigned longest first (N^3) to the least-loaded stream so small problems run
 * beside large ones. The first pfsm_solve_batched call with a given set of buffers and stream
 * captures the fork / per-problem solves / join into a CUDA graph; later calls with the same
 * buffers replay it with one graph launch (new buffers trigger a new capture). */
typedef struct pfsm_batch_s *pfsm_batch_t;

/* count problems; N[i], nblocks[i] (HOST arrays) as for pfsm_init; p shared by all problems
 * (p->slice_sizes is ignored). Allocates every problem's workspace. */
int pfsm_batch_init(int32_t count, const int64_t *N, const int32_t *nblocks, const pfsm_params_t *p,
                    pfsm_batch_t *out);

/* A, prev, eigvals_out, V_out: HOST arrays of `count` DEVICE pointers, each laid out as in
 * pfsm_solve for its own N[i]. Ordered on `stream` (any stream, including the legacy default):
 * the graph runs on a private stream of the batch after the caller's earlier work on `stream`,
 * and later work on `stream` waits for it. Not synchronised. The buffers must stay valid until
 * the stream reaches the end of the call. */
int pfsm_solve_batched(pfsm_batch_t b, const double *const *A, const double *const *prev,
                       double *const *eigvals_out, double *const *V_out, void *stream);

/* Synchronises the batch's last stream and writes each problem's device status word to
 * statuses[i] (HOST array of count int32). */
int pfsm_batch_get_status(pfsm_batch_t b, int32_t *statuses);

/* Frees the batch (synchronises the device first). NULL is allowed. */
int pfsm_batch_destroy(pfsm_batch_t b);

/* Split-precision product on the tcgen05 tensor cores, the building block of the mixed forms
 * (Eq. 11 products). C[r, c] = sum_k P[r, k] Q[c, k] for FP64 row-major P (rows x K), Q
 * (cols x K) and C (rows x cols), all device pointers. Each operand is split into BF16 (3
 * pieces, precision PFSM_BF16_SPLIT) or TF32 (2 pieces, PFSM_TF32_SPLIT) and the cross products
 * of total order below the piece count are accumulated in FP32 in tensor memory: relative
 * accuracy about 2^-22 (TF32) or 2^-24 (BF16) of sum_k |P[r,k] Q[c,k]|. With precision
 * PFSM_FP64 the product is FP64-accurate: each row is scaled by a power of two and cut into seven
 * base-128 digits held exactly in BF16, digit products of equal level are summed exactly in FP32
 * tensor memory (K chunks of 512) and levels 0..6 are combined in float-float, then FP64 (error
 * about sqrt(K) 2^-49 max|P[r,:]| max|Q[c,:]| for random-sign terms, at most K 2^-46 of it;
 * Ozaki, Ogita, Oishi, Rump 2012). Allocates its slices
 * with cudaMallocAsync on `stream`, frees them, and synchronises the stream before returning;
 * returns PFSM_ERR_TIMEOUT if a bounded device wait gave up. rows, cols <= 65535. */
int pfsm_split_gemm(int64_t rows, int64_t cols, int64_t K, const double *P, const double *Q,
                    double *C, int32_t precision, void *stream);

/* pfsm_split_gemm with the split products' output-tile width given: tile_n = 64, 96 or 128
 * columns (rows are always 128), or 0 for the autotuned width (every candidate timed once per
 * device, slice kind and shape class, the fastest kept; the same tuner picks the width of a
 * handle's Eq. 11 products at pfsm_init). Ignored for PFSM_FP64. Returns PFSM_ERR_INVALID_ARG
 * for any other tile_n. */
int pfsm_split_gemm_ex(int64_t rows, int64_t cols, int64_t K, const double *P, const double *Q,
                       double *C, int32_t precision, int32_t tile_n, void *stream);

/* Eq. 11 on caller vectors WITHOUT ANY DEVICE ALLOCATION. The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory when they call the
 * library, e.g. codes that reserve all device memory up front for their own pool, or
 * latency-critical loops where the device-wide synchronisation of cudaMalloc/cudaFree would
 * stall other streams.
 *   N       order of A
 *   count   number of vectors; count * N must not exceed 1048576 (8 MiB of FP64 scratch),
 *           otherwise the call returns PFSM_ERR_INVALID_ARG without touching the GPU
 *   A       device, N x N FP64, symmetric
 *   X       device, count x N FP64, ROW k = vector k (note: rows, unlike V_out); updated in
 *           place with `iters` iterations x <- x - alpha_k (A - eps_k I)^2 x
 *   eps, alpha  device, count FP64 shifts and steps
 * The only scratch, (A - eps I) X between the two products of each iteration, lives in one
 * fixed 8 MiB device array of the library. CUDA loads the array's module into a context
 * lazily (the default module loading since CUDA 12.2), so the FIRST call on each device (and
 * the first in any new context, e.g. after cudaDeviceReset) loads it and allocates those
 * 8 MiB, then looks up the array's device address (cudaGetSymbolAddress) and caches it for
 * that context. Make that first call before reserving the device's memory for a pool, and
 * outside any stream capture; from then on the device holds the array until the process exits
 * (or the context is destroyed) and no call allocates. All calls share the array: calls that
 * may overlap on the GPU (different streams, or several host threads) race on it and must be
 * serialised by the caller. Nothing in it needs clearing between calls. */
int pfsm_fs_iterate_noalloc(int64_t N, int64_t count, const double *A, double *X,
                            const double *eps, const double *alpha, int32_t iters, void *stream);

/* ---- generalized -> standard conversion (Eq. 14-15), the step before the eigensolve ----------
 * A x = lambda B x with A symmetric and B the symmetric, diagonally dominant overlap matrix; all
 * matrices N x N row-major FP64 on the device (N <= 65535), A and B read only. Both run on
 * `stream`, allocate their temporaries with cudaMallocAsync, read one residual per iteration back
 * to the host (so they synchronise the stream) and write *iters_out (updates done) and
 * *resid_out (the stopping residual) when those host pointers are non-null. Products are the
 * FP64-accurate digit products of pfsm_split_gemm(..., PFSM_FP64); the residuals they measure
 * have a floor of a few sqrt(N) 2^-46 (6.5e-13 for the Jacobi residual at N = 1280, 1.6e-12
 * for max|I - Q Y| at N = 200), so tol should stay above it (1e-12 and 1e-11).
 *
 * pfsm_gen_to_std: Z = B^{-1} A by the Jacobi iteration of Eq. 14,
 *   Z_{n+1} = (I - D^{-1} B) Z_n + D^{-1} A,  D = diag(B),  Z_0 = 0,
 * stopped before an update when max|A - B Z_n| <= tol max|A| or after max_iters updates.
 * Returns PFSM_OK, PFSM_ERR_NOT_CONVERGED (Z holds the last iterate), PFSM_ERR_INVALID_ARG
 * (bad arguments, or a zero diagonal entry of B: Z untouched), PFSM_ERR_CUDA. */
int pfsm_gen_to_std(int64_t N, const double *A, const double *B, double *Z, int32_t max_iters, double tol,
                    int32_t *iters_out, double *resid_out, void *stream);

/* Symmetric form of the conversion (not in the paper, which leaves B^{-1} A non-symmetric; the
 * eigensolver needs a symmetric matrix): C = B^{-1/2} A B^{-1/2} and S = B^{-1/2}, so that C has
 * the eigenvalues of A x = lambda B x and its eigenvectors y give x = S y (B-orthonormal).
 * S by the coupled Newton-Schulz iteration for the inverse square root (c = the largest
 * Gershgorin row bound of B; Y_0 = B / c, Q_0 = I; T = (3 I - Q Y) / 2; Y <- Y T; Q <- T Q),
 * stopped before an update when max|I - Q Y| <= tol or after max_iters updates; S = Q / sqrt(c),
 * C = S A S. Returns PFSM_OK, PFSM_ERR_NOT_CONVERGED (C, S from the last iterate),
 * PFSM_ERR_NOT_SPD (no positive row bound), PFSM_ERR_INVALID_ARG, PFSM_ERR_CUDA. */
int pfsm_gen_to_std_sym(int64_t N, const double *A, const double *B, double *C, double *S, int32_t max_iters,
                        double tol, int32_t *iters_out, double *resid_out, void *stream);

/* Per-call instrumentation, for benchmarks and profiling. */
typedef struct {
    int32_t launches;     /* kernels enqueued by the last pfsm_solve / pfsm_backward on h */
    int32_t timed;        /* 1 when phase_ms holds measurements (timing enabled on h) */
    float phase_ms[12];   /* CUDA-event times on the call's stream, in milliseconds:
                             0 validation + partition plan, 1 submatrix solves + start vectors,
                             2 Eq. 11 iterations, 3 Gram-Schmidt (overlap, Cholesky, solve),
                             4 Rayleigh quotients, residuals and outputs, 5 backward;
                             inside 1: 6 tridiagonalisation, 7 bisection, 8 inverse iteration,
                             9 back-transformation + start vectors; inside 3: 10 overlap,
                             11 Cholesky or, in the mixed forms, the preconditioner; the
                             triangular solve is phase 3 minus 10 and 11 */
    int32_t gemm_tile_n;  /* output-tile width (64, 96 or 128 columns) of the handle's split
                             products, measured at pfsm_init; 0 for PFSM_FP64 handles */
    int32_t path;         /* last pfsm_solve: 0 the method, 1 full diagonalization by the
                             first-steps rule, 2 full diagonalization by the guard */
    double guard_value;   /* its guard value g (0 when not measured) */
    int32_t fs_steps;     /* Eq. 11 steps taken by the last solve */
    double fs_residual;   /* with fs_adaptive: the last max_k residual measured (else 0) */
    int32_t gs_precond;   /* mixed forms, last pfsm_solve by the method: Gram-Schmidt
                             preconditioner 2 second-order series, 3 the series followed by the
                             FP32 Cholesky factorisation (series residual too large; eager solves
                             only); 0 otherwise */
    double gs_precond_residual; /* max |M S M^T - I| after the series, measured by eager solves
                                   (0 for solves captured into a CUDA graph) */
    float band_ms[4];     /* two-stage reduction (mixed forms, wide windows), with timing: inside
                             phase 6, 0 dense to band (panels), 1 band to tridiagonal (bulge
                             chasing); inside phase 9, 2 the bulge reflectors applied to the
                             eigenvectors, 3 the panel reflectors and the start vectors; zeros
                             otherwise */
} pfsm_profile_t;

/* Enables (enable != 0) or disables CUDA-event phase timing on h. Timing adds one event record
 * per phase boundary to the stream and nothing else. */
int pfsm_set_timing(pfsm_handle_t h, int32_t enable);

/* Synchronises the stream of the last call on h and fills *out (host pointer). */
int pfsm_get_profile(pfsm_handle_t h, pfsm_profile_t *out);

/* ---- test entry points: the hand-written FP64 helpers ------------------------------------------
 * The serial FP64 paths (window eigensolves, bulge chasing, panel QR) avoid the IEEE FP64 divide
 * and square-root sequences, and the digit products' epilogues avoid FP64 conversions: reciprocals
 * and inverse square roots are FP32 seeds refined by two Newton steps, and an exact 64-bit integer
 * sum is rounded to FP64 by integer operations. These calls evaluate those helpers elementwise on
 * caller-given device arrays so that tests can compare them with CUDA's correctly rounded 1/x,
 * 1/sqrt(x) and integer conversion. They have no counterpart in the paper and play no part in a
 * solve. All pointers are device pointers; launches go to `stream`; nothing is synchronised.
 *
 * pfsm_selftest_fp64_helpers: for i < n, rcp_scaled[i] = 1/x[i] and rsqrt_scaled[i] = 1/sqrt(x[i])
 * by the exponent-splitting Newton helpers (0 where x[i] <= 0, outside their domain), rcp_fast[i]
 * = 1/x[i] by the bit-pattern Newton helper (either sign; |x| outside [2^-125, 2^126) takes
 * CUDA's division), rsqrt_fast[i] = 1/sqrt(x[i]) by the bit-pattern Newton helper (0 where
 * x[i] <= 0; x outside [2^-125, 2^124) takes the exponent-splitting helper).
 * pfsm_selftest_i64_to_f64: out[i] = t[i] * 2^e[i] rounded to nearest, ties to even (the digit
 * products' exact level-sum conversion).
 * Both return PFSM_ERR_INVALID_ARG for n < 0 or a null pointer with n > 0, PFSM_ERR_CUDA if the
 * launch fails. */
int pfsm_selftest_fp64_helpers(const double *x, int64_t n, double *rcp_scaled, double *rsqrt_scaled,
                               double *rcp_fast, double *rsqrt_fast, void *stream);
int pfsm_selftest_i64_to_f64(const int64_t *t, const int32_t *e, int64_t n, double *out, void *stream);

/* Thread-local text of the last error raised on this thread ("" if none). */
const char *pfsm_last_error(void);

/* Frees the handle and its workspace (synchronises the device first). NULL is allowed. */
int pfsm_destroy(pfsm_handle_t h);

#ifdef __cplusplus
}
#endif

#endif /* PFSM_H */
