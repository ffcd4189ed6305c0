// Internal declarations shared by the PFSM CUDA sources (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/pfsm.h"

namespace pfsm {

// Device status word: the first error recorded wins (atomicCAS from 0).
__device__ __forceinline__ void set_status(int32_t *status, int32_t code)
{
    atomicCAS(status, 0, code);
}

// Plan layout in device memory: int32 arrays k0[nb], m[nb], s[nb], M[nb], then per-row-tile
// K-ranges for the block-sparse first product of Eq. 11 (pairs kbeg, kend).
struct PlanView {
    int32_t *k0, *m, *s, *M;
};

// Workspace owned by a handle. Row-major N x N buffers hold vectors as ROWS ("Xt" layout):
// row k is eigenvector k, so every product of Eq. 11 reads both operands along rows.
struct Workspace {
    int32_t *plan = nullptr;       // 4*nb
    int32_t *tile_krange = nullptr; // 2 * ceil(N / kFsTileRows)
    int32_t *status = nullptr;     // 1
    double *gersh = nullptr;       // 2*N row bounds, then [lo, hi] at 2*N, 2*N+1
    double *X = nullptr;           // N*N vectors (rows); becomes V (rows) after Gram-Schmidt
    double *Xfs = nullptr;         // N*N copy of X after the Eq. 11 iterations (diagnostics)
    double *Y = nullptr;           // N*N (A - eps I) X
    double *S = nullptr;           // N*N overlap / Cholesky factor L (lower)
    double *W = nullptr;           // N*N A V (rows), backward scratch
    double *Vrm = nullptr;         // N*N V in output layout (kept for backward)
    double *sdiag = nullptr;       // N diag(S) before factorisation
    double *Linv = nullptr;        // N x 64 inverses of the 64 x 64 diagonal blocks of L
    double *eps = nullptr, *alpha = nullptr, *lam = nullptr, *res = nullptr; // N each
    // submatrix eigensolver
    double *refl = nullptr;        // nb * Mmax * Mmax Householder vectors (row k = v_k)
    double *tau = nullptr;         // nb * Mmax reflector scalars beta_k
    double *td = nullptr, *te = nullptr; // nb * Mmax tridiagonal diagonal / off-diagonal
    double *sel_val = nullptr;     // nb * mmax selected eigenvalues
    double *sel_vec = nullptr;     // nb * mmax * Mmax selected eigenvectors of T (rows)
    double *iiwork = nullptr;      // nb * mmax * 5 * Mmax inverse-iteration LU storage (also
                                   // the window rows when they do not fit in shared memory)
    int32_t *slices = nullptr;     // nb explicit slice sizes, or null
    // mixed forms: BF16/TF32 slices of E = A - diag(A), X, Y, Z (rows x ld, ns per operand)
    void *slE = nullptr, *slX = nullptr, *slY = nullptr, *slZ = nullptr;
    double *Z = nullptr;           // N*N (A - eps I) Y
    double *dA = nullptr;          // N diag(A)
    void *ozP = nullptr, *ozQ = nullptr;   // OZ_SLICES digit matrices (BF16) of two operands
    int32_t *ozeP = nullptr, *ozeQ = nullptr;   // their row exponents
    // mixed-form Gram-Schmidt: FP32 Cholesky working matrix, augmented right-hand side and the
    // preconditioner M = L~^-1 (zero above the diagonal), and the FP64 correction factor F
    float *L32 = nullptr, *R32 = nullptr, *M32 = nullptr;
    double *F = nullptr;
    // mixed-form blocked tridiagonalisation: per window rows of [V W] and [W V] (nb * Mmax x
    // 2 * 32), their digit matrices and row exponents
    double *VW = nullptr, *WV = nullptr;
    void *tdP = nullptr, *tdQ = nullptr;
    int32_t *tdeP = nullptr, *tdeQ = nullptr;
    // mixed-form back-transformation in compact-WY form (k_bt_wy.cu), per window: G = V^T V
    // (Mmax x Mmax, lower), V^T (Mmax x Mmax), W1 = V^T Z (Mmax x mmax), W2^T (mmax x Mmax), Y
    // (mmax x Mmax); the digit matrices of the Mmax-row and the mmax-row operands and their row
    // exponents; per-window extents (reflectors, vectors, rows)
    // mixed forms: digits of A' = A - diag(A) for the Rayleigh product, split on the side stream
    void *ozA = nullptr;
    int32_t *ozeA = nullptr;
    double *btG = nullptr, *btRT = nullptr, *btW1 = nullptr, *btW2T = nullptr, *btY = nullptr;
    void *btDA = nullptr, *btDB = nullptr;
    int32_t *btEA = nullptr, *btEB = nullptr, *btExt = nullptr;
    // mixed-form two-stage reduction (k_band.cu): digits of the trailing matrices and of the
    // panel reflectors with their row exponents, Y = A22 V (then W = Y T; nb * Mmax x 32), T and
    // U (nb x 32 x 32), the chunk partials of V^T W, the per-panel window extents, the band
    // storage of stage 2 and its reflectors (per window, sweep and task: 32 entries and beta)
    void *bdA = nullptr, *bdV = nullptr;
    int32_t *bdeA = nullptr, *bdeV = nullptr, *bExt = nullptr, *bKB = nullptr;
    double *bV = nullptr;          // every panel's reflectors as rows j (panels x nb * Mmax x 32)
    double *bY = nullptr, *bT = nullptr, *bU = nullptr, *bXp = nullptr, *bBw = nullptr, *bR2 = nullptr,
           *bT2 = nullptr, *bD = nullptr;   // bD: the trailing matrices' diagonals (nb * Mmax)
};

}  // namespace pfsm

struct pfsm_handle_s {
    int64_t N = 0;
    int32_t nb = 0;
    pfsm_params_t prm{};
    int32_t halo = 0;
    int32_t mmax = 0;    // largest slice after cluster snap
    int32_t Mmax = 0;    // largest window
    int32_t cl = 8;      // CTAs per submatrix cluster
    int32_t tc_bn = 128; // tile width of the split products (tuned at init for the handle's N)
    // conventional path (k_fallback.cu): first-steps rule and diagonal-dominance guard
    int64_t nsolves = 0;           // solves done on the handle
    int32_t last_path = 0;         // 0 the method, 1 first-steps rule, 2 guard
    double last_guard = 0.0;       // guard value of the last solve (0 when not measured)
    void *cusolver = nullptr;      // cusolverDnHandle_t, created when the path can be taken
    double *syevd_work = nullptr;
    int syevd_lwork = 0;
    int *syevd_info = nullptr;
    unsigned long long *guard_buf = nullptr;
    int32_t last_fs_steps = 0;     // Eq. 11 steps of the last solve
    double last_fs_resid = 0.0;    // adaptive variant: its last measured residual
    unsigned long long *fs_rmax = nullptr;   // 8-byte read-back word (device): the adaptive
                                             // variant's residual, the mixed Gram-Schmidt's
                                             // preconditioner residual
    int32_t gs_precond = 0;        // mixed Gram-Schmidt preconditioner of the last solve (profile)
    double gs_precond_resid = 0.0; // its measured residual
    bool rows_in_smem = true;
    bool tri_blocked = false;      // mixed forms: blocked reduction (k_tridiag_panel)
    int32_t tri_rpw = 8;           // its rows-per-warp register capacity (8 or 24)
    int32_t tri_mcap = 0;          // largest window kept in shared memory by it
    bool tri_two_stage = false;    // mixed forms: two-stage reduction (k_band.cu)
    int32_t *h_slices = nullptr;   // host copy of explicit slice sizes (or null)
    pfsm::Workspace ws;
    cudaStream_t last_stream = nullptr;
    bool solved = false;
    const double *last_A = nullptr;
    const double *last_prev = nullptr;
    // instrumentation
    bool timing = false;
    cudaEvent_t ev[8] = {};
    cudaEvent_t sub_ev[4] = {};   // inside the submatrix phase (timing only)
    cudaEvent_t gs_ev[2] = {};    // inside Gram-Schmidt: after the overlap, after Cholesky
    cudaEvent_t band_ev[3] = {};  // two-stage reduction: after the panels, after the bulge chase,
                                  // after the bulge reflectors' back-transformation
    // mixed forms: a second stream for work that depends only on A or on the window reduction
    // (the Eq. 11 operand split of A, the back-transform's reflector preparation and V^T V), run
    // beside the window kernels that leave SMs idle; forked and joined through events
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool side_pending = false;     // side work enqueued and not yet waited for on the solve stream
    bool a_split = false;          // this solve split A' into ws.ozA on the side stream
    int32_t last_launches = 0;
    bool last_was_backward = false;
};

namespace pfsm {

constexpr int kFsTileRows = 64;     // row tile of the FP64 GEMM (also the K-range granularity)

// Kernels enqueued by this host thread since the counter was last reset (instrumentation).
inline thread_local int64_t g_launches = 0;
inline cudaError_t counted(cudaError_t e) { if (e == cudaSuccess) g_launches++; return e; }

// Records the thread-local message returned by pfsm_last_error().
void set_last_error(const char *msg);

// ---- launchers (each enqueues on `st`; returns cudaGetLastError()) ----
cudaError_t launch_validate_gersh(const double *A, const double *prev, int64_t N, double *gersh,
                                  int32_t *status, cudaStream_t st);
cudaError_t launch_plan(const double *prev, int64_t N, int32_t nb, int32_t halo, double cluster_tol,
                        const int32_t *slice_sizes_dev, int32_t *plan, int32_t *tile_krange,
                        double *gersh, int32_t *status, cudaStream_t st);

cudaError_t launch_subeig(pfsm_handle_s *h, const double *A, cudaStream_t st);
// mixed forms: y = H_0 ... H_{M-3} z and the start vectors by the compact-WY form (k_bt_wy.cu);
// false when the solve's shared memory cannot hold a column chunk (the FP64 kernel is used).
// reflectors_done: launch_backtransform_wy_reflectors already ran on the side stream.
bool backtransform_wy_fits(int Mmax);
cudaError_t launch_backtransform_wy(pfsm_handle_s *h, cudaStream_t st, bool reflectors_done);
// the part of it that needs only the reduction's reflectors (on the handle's side stream)
cudaError_t launch_backtransform_wy_reflectors(pfsm_handle_s *h, cudaStream_t st);
// the solve stream waits for the side stream's work, if any is pending
cudaError_t join_side(pfsm_handle_s *h, cudaStream_t st);
cudaError_t configure_bt_wy_kernels();
cudaError_t configure_kernels(pfsm_handle_s *h);   // shared-memory / cluster attributes

enum Epi : int { EPI_STORE = 0, EPI_SUB = 1, EPI_FS1 = 2, EPI_FS2 = 3 };
enum QLayout : int { Q_KMAJOR = 0, Q_NMAJOR = 1 };

struct GemmArgs {
    int64_t rows, cols, K;
    const double *P; int64_t ldp;        // rows x K, row-major (K contiguous)
    const double *Q; int64_t ldq;        // K_MAJOR: cols x K row-major; N_MAJOR: K x cols row-major
    double *C; int64_t ldc;              // rows x cols
    const double *aux_x;                 // FS1: X (rows x cols, ld ldc); FS2: X updated in place = C
    const double *aux_y;                 // FS2: Y
    const double *eps, *alpha;           // per row
    const int32_t *krange;               // per row tile (kbeg, kend) or null
    int lower_only;                      // skip tiles strictly above the diagonal
};
cudaError_t launch_gemm_f64(const GemmArgs &a, int epi, int qlayout, cudaStream_t st);

// ---- tensor-core split-precision GEMM (k_gemm_tc.cu) ----
enum TcEpi : int { TC_EPI_STORE = 0, TC_EPI_Y0 = 1, TC_EPI_Z = 2, TC_EPI_YN = 3, TC_EPI_RSUB = 4 };

// A matrix held as `ns` slices (kind 0: BF16, kind 1: TF32 in FP32 containers), each rows x ld,
// ld a multiple of 64 elements with zero padding columns.
struct SliceBuf {
    void *ptr;
    int64_t rows, ld;
    int ns, kind;
};

struct TcParams {
    int rows, cols;                 // output extent
    int kblocks, bk, npairs;        // filled by launch_gemm_tc
    const int32_t *krange;          // per 64-row tile K range, or null
    int nrowtiles64;
    int epi;
    double *out; int64_t ldo;
    void *out_slices; int64_t sl_ld, sl_stride; int out_ns;
    double *X;                      // TC_EPI_Z: x <- x - alpha z
    const double *V;                // operand in FP64 (Y for TC_EPI_Z, Z for TC_EPI_YN, the
                                    // minuend of TC_EPI_RSUB: out = V - P Q^T, may alias out)
    const double *Yold;             // TC_EPI_YN
    const double *d, *eps, *alpha;
    const int32_t *plan; int nb;    // TC_EPI_Y0 window mask
    int lower_only;                 // skip output tiles strictly above the diagonal
    int bn;                         // tile width 64, 96 or 128 (0: 128; lower-only products: 128)
    int32_t *status;
};
cudaError_t configure_tc_kernels();
int tune_tc_tile(const SliceBuf &P, const SliceBuf &Q, int rows, int cols, double *scratch);
cudaError_t launch_split(const double *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                         bool zero_diag, double *d, cudaStream_t st);
cudaError_t launch_gemm_tc(const SliceBuf &P, const SliceBuf &Q, TcParams prm, SliceBuf *out_sl,
                           cudaStream_t st);
// ---- FP64-accurate products on the BF16 tensor cores (k_gemm_oz.cu) ----
#define OZ_SLICES 7                 // base-128 digits per entry (2^-49 of the row's largest)
#define OZ_LEVELS 7                 // digit levels s + t kept by default (see k_gemm_oz.cu)
struct OzParams {
    int rows, cols;                 // output extent
    int kblocks;                    // 32-element K blocks (filled by launch_gemm_oz)
    const int32_t *ep, *eq;         // row exponents of P and Q (filled by launch_gemm_oz)
    double *C; int64_t ldc;
    int sub;                        // C -= P Q^T instead of C = P Q^T
    int lower_only;                 // only entries with c <= r
    int p_lower;                    // P is lower triangular: skip K blocks beyond the tile's rows
    int levels;                     // digit levels L = s + t kept (0: OZ_LEVELS)
    // batched windows (blockIdx.z = window z): operand rows z * zrow + i, C + z * zc, output
    // entries (i, j) for row_base <= i, j < ext[z] (ext null: one product, row_base 0)
    int64_t zrow, zc;
    int row_base;
    const int32_t *ext;
    int cols_from_zero;             // output columns start at 0 instead of row_base
    int col_off;                    // ... and col_off further on
    const int32_t *krange64;        // per 64-row tile K range (kbeg, kend) of P's rows, or null
    int nrowtiles64;
    const int32_t *win_plan;        // with win_nb: output (r, c) zero for c inside the window of
    int win_nb;                     // the slice owning row r (the first Eq. 11 product)
    int64_t zrow_q;                 // Q's operand rows per window (0: zrow)
    const int32_t *ext_c;           // output column extents per window (null: ext)
    const double *Vp; int64_t ldv;  // with dcol: C[r, c] += Vp[r, c] dcol[c] (exact diagonal term)
    const double *dcol;
    const double *drow;             // with drow instead: C[r, c] += Vp[r, c] drow[r]
    int64_t vcs;                    // column stride of Vp (0: 1); Vp[r, c] = Vp[r ldv + c vcs]
    int64_t zv, zd;                 // batched: window z's Vp and dcol / drow start z zv and z zd further
    int32_t *status;
};
cudaError_t configure_oz_kernels();
int sm_count();                     // multiprocessors of the current device (cached)
// ---- conventional path: guard and full diagonalization (k_fallback.cu) ----
cudaError_t fallback_init(pfsm_handle_s *h);
void fallback_free(pfsm_handle_s *h);
cudaError_t measure_guard(pfsm_handle_s *h, const double *A, cudaStream_t st, double &g);
cudaError_t run_full_diag(pfsm_handle_s *h, const double *A, cudaStream_t st);
// ---- dense FP64-accurate N x N products with scratch digits (k_gen2std.cu) ----
struct Digits {                     // digit operand of an N x N product, allocated on a stream
    void *sl = nullptr;
    int32_t *ex = nullptr;
    SliceBuf buf{};
};
cudaError_t make_digits(Digits &d, int64_t N, cudaStream_t st);
void free_digits(Digits &d, cudaStream_t st);
cudaError_t digit_product(const Digits &dx, const Digits &dy, double *C, int64_t N, bool sub, int32_t *status,
                          cudaStream_t st);
// C = X Yrows^T (split both, then the digit product)
cudaError_t dense_product(const double *X, const double *Yrows, double *C, int64_t N, Digits &dx, Digits &dy,
                          int32_t *status, cudaStream_t st);
cudaError_t launch_symmetrize(const double *T, double *S, int64_t N, cudaStream_t st);   // S = (T + T^T) / 2
// adaptive Eq. 11 (k_dense.cu): per row k, eps_k += x.y / x.x, y -= that x, alpha_k from the new
// shift, *rmax (bits, zeroed by the caller) = max_k ||y_k|| / ||x_k||
cudaError_t launch_rq_shift(double *X, double *Y, double *eps, double *alpha, const double *gersh, double theta,
                            int64_t N, unsigned long long *rmax, cudaStream_t st);
// ---- generalized -> standard conversion (k_gen2std.cu) ----
struct Gen2StdResult {
    int iters = 0;                  // updates done
    double resid = 0.0;             // stopping residual of the returned result
    int status = 0;                 // PFSM_OK, PFSM_ERR_NOT_CONVERGED, PFSM_ERR_INVALID_ARG (zero
                                    // diagonal of B), PFSM_ERR_NOT_SPD, or a device status
};
cudaError_t run_gen_to_std(int64_t N, const double *A, const double *B, double *Z, int max_iters, double tol,
                           cudaStream_t st, Gen2StdResult &res);
cudaError_t run_gen_to_std_sym(int64_t N, const double *A, const double *B, double *C, double *S, int max_iters,
                               double tol, cudaStream_t st, Gen2StdResult &res);
cudaError_t launch_oz_split(const double *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                            int32_t *exps, cudaStream_t st, bool zero_diag = false, double *d = nullptr);
// batched over nb windows: ext[z] - ext_off rows (or rows_fixed rows) x (ext[z] - ext_off) columns
// of the block at src + z * src_z + row0 * ld + col0, digits zero-filled to dst.ld (see k_gemm_oz.cu);
// with diag_out, the block's diagonal is split off (digits of zero) and stored there
cudaError_t launch_oz_split_win(const double *src, int64_t src_z, int64_t ld, int64_t row0, int64_t col0,
                                const int32_t *ext, int ext_off, int rows_fixed, const int32_t *rext, int max_rows,
                                int nb, const SliceBuf &dst, int64_t dst_zrow, int64_t dst_row0, int32_t *exps,
                                cudaStream_t st, double *diag_out = nullptr);
cudaError_t launch_oz_split_f32(const float *src, int64_t rows, int64_t cols, int64_t ld, const SliceBuf &dst,
                                int32_t *exps, cudaStream_t st);
cudaError_t launch_gemm_oz(const SliceBuf &P, const int32_t *ep, const SliceBuf &Q, const int32_t *eq,
                           OzParams prm, cudaStream_t st, int batch = 1);
// the same for K <= 64 (P.ld <= 64), a CTA per 128-row tile and strip of `strip` column tiles
// (no lower_only / p_lower / diagonal terms / window mask / K ranges)
cudaError_t launch_gemm_oz_strip(const SliceBuf &P, const int32_t *ep, const SliceBuf &Q, const int32_t *eq,
                                 OzParams prm, cudaStream_t st, int batch, int strip);

inline int slices_for(int precision) { return precision == PFSM_BF16_SPLIT ? 3 : 2; }
inline int slice_kind(int precision) { return precision == PFSM_BF16_SPLIT ? 0 : 1; }
inline int64_t padded_ld(int64_t n) { return (n + 63) / 64 * 64; }

// cluster size and row placement of the window reduction (k_subeig.cu)
cudaError_t select_tridiag_cluster(pfsm_handle_s *h, size_t smem_cap);

// blocked tridiagonalisation of the mixed forms (k_subeig.cu): panel width and the panel
// kernel's dynamic shared memory (window rows for windows up to Mcap, or none)
constexpr int kPanel = 32;
inline size_t tri_panel_smem(int Mmax, int CL, int Mcap)
{
    size_t b = (size_t)(3 * Mmax + 64) * sizeof(double);                       // vbuf, pbuf, hv, red
    b += 2 * (size_t)(kPanel + 2) * kPanel * sizeof(double);                    // panel rows of V, W
    b += (size_t)(CL + 1 + 8) * 2 * kPanel * sizeof(double);                    // dots, ab, per-warp dots
    if (Mcap > 0) b += (size_t)((Mcap + CL - 1) / CL) * Mcap * sizeof(double);
    return b;
}

// two-stage reduction of the mixed forms (k_band.cu): band half-width, CTAs per window of the
// panel and bulge-chasing kernels, warps per bulge-chasing CTA
constexpr int kBand = 32;
constexpr int kPanelCL = 8;
constexpr int kChaseCL = 3;
constexpr int kChaseWarps = 8;
__host__ __device__ int band_panels(int M);
size_t band_panel_smem(int Mmax);
bool band_reduction_fits(int Mmax, size_t smem_cap);
int band_tasks_per_sweep(int Mmax);
cudaError_t configure_band_kernels();
cudaError_t launch_band_reduction(pfsm_handle_s *h, const double *A, cudaStream_t st);
cudaError_t launch_band_backtransform(pfsm_handle_s *h, cudaStream_t st);
// the start-vector rules on back-transformed window eigenvectors Y (rows t, entries j; k_bt_wy.cu)
cudaError_t launch_bt_finish(pfsm_handle_s *h, const double *Y, cudaStream_t st);

cudaError_t configure_dense_kernels();   // shared-memory attributes of k_dense.cu
cudaError_t launch_gram_schmidt_f64(pfsm_handle_s *h, cudaStream_t st);
cudaError_t launch_rayleigh_f64(pfsm_handle_s *h, const double *A, double *eigvals_out,
                                double *V_out, cudaStream_t st);
cudaError_t launch_transpose(const double *in, double *out, int64_t N, cudaStream_t st);
cudaError_t launch_copy_diag(const double *S, int64_t N, double *d, cudaStream_t st);
// mixed-form Gram-Schmidt (k_gs_mixed.cu)
cudaError_t configure_gs_mixed_kernels();
cudaError_t launch_gram_schmidt_mixed(pfsm_handle_s *h, cudaStream_t st);
cudaError_t launch_backward_f64(pfsm_handle_s *h, const double *dLambda, const double *dV,
                                double *dA_out, cudaStream_t st);
cudaError_t launch_backward_mixed(pfsm_handle_s *h, const double *dLambda, const double *dV,
                                  double *dA_out, cudaStream_t st);

}  // namespace pfsm
