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
    bool rows_in_smem = true;
    int32_t *h_slices = nullptr;   // host copy of explicit slice sizes (or null)
    pfsm::Workspace ws;
    cudaStream_t last_stream = nullptr;
    bool solved = false;
    const double *last_A = nullptr;
    const double *last_prev = nullptr;
    // instrumentation
    bool timing = false;
    cudaEvent_t ev[8] = {};
    int32_t last_launches = 0;
    bool last_was_backward = false;
};

namespace pfsm {

constexpr int kFsTileRows = 64;     // row tile of the FP64 GEMM (also the K-range granularity)

// Kernels enqueued by this host thread since the counter was last reset (instrumentation).
inline thread_local int64_t g_launches = 0;
inline cudaError_t counted(cudaError_t e) { if (e == cudaSuccess) g_launches++; return e; }

// ---- launchers (each enqueues on `st`; returns cudaGetLastError()) ----
cudaError_t launch_validate_gersh(const double *A, const double *prev, int64_t N, double *gersh,
                                  int32_t *status, cudaStream_t st);
cudaError_t launch_plan(const double *prev, int64_t N, int32_t nb, int32_t halo, double cluster_tol,
                        const int32_t *slice_sizes_dev, int32_t *plan, int32_t *tile_krange,
                        double *gersh, int32_t *status, cudaStream_t st);

cudaError_t launch_subeig(pfsm_handle_s *h, const double *A, cudaStream_t st);
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

cudaError_t launch_gram_schmidt_f64(pfsm_handle_s *h, cudaStream_t st);
cudaError_t launch_rayleigh_f64(pfsm_handle_s *h, const double *A, double *eigvals_out,
                                double *V_out, cudaStream_t st);
cudaError_t launch_transpose(const double *in, double *out, int64_t N, cudaStream_t st);
cudaError_t launch_backward_f64(pfsm_handle_s *h, const double *dLambda, const double *dV,
                                double *dA_out, cudaStream_t st);

}  // namespace pfsm
