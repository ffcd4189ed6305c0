// C ABI of the PFSM library: argument checks, workspace ownership, and the order of kernels for
// one solve (Section II: partition, submatrix solves, Eq. 11 iterations, Gram-Schmidt).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pfsm_internal.cuh"

using namespace pfsm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(PFSM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PFSM_CUDA(expr)                                        \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr);    \
    } while (0)

template <typename T>
cudaError_t alloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, count * sizeof(T) + 256);
}

void free_ws(pfsm_handle_s *h)
{
    Workspace &w = h->ws;
    void *ptrs[] = {w.plan, w.tile_krange, w.status, w.gersh, w.X, w.Xfs, w.Y, w.S, w.W, w.Vrm,
                    w.sdiag, w.eps, w.alpha, w.lam, w.res, w.refl, w.tau, w.td, w.te,
                    w.sel_val, w.sel_vec, w.iiwork, w.slices, w.slE, w.slX, w.slY, w.slZ,
                    w.Z, w.dA, w.Linv, w.ozP, w.ozQ, w.ozeP, w.ozeQ, w.L32, w.R32, w.M32, w.F, w.VW, w.WV, w.tdP, w.tdQ, w.tdeP, w.tdeQ,
                    w.btG, w.btRT, w.btW1, w.btW2T, w.btY, w.btDA, w.btDB, w.btEA, w.btEB, w.btExt,
                    w.ozA, w.ozeA, w.bdA, w.bdV, w.bdeA, w.bdeV, w.bExt, w.bKB, w.bV, w.bY, w.bT, w.bU, w.bXp,
                    w.bBw, w.bR2, w.bT2, w.bD};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    w = Workspace{};
}

// Largest dynamic shared memory a CTA may use on this part.
constexpr size_t kSmemCap = 227 * 1024;
// The blocked reduction (k_tridiag_panel) issues more FP64 instructions per step than the
// unblocked one saves (B300 spends ~64 cycles of an SMSP's FP64 pipe on every FP64 warp
// instruction, shuffle reductions and redundant scalar work included); off until that changes.
constexpr bool kUseBlockedReduction = false;
// Window width from which the mixed forms reduce in two stages by default (the one-stage
// reduction keeps windows up to a few hundred rows in a cluster's shared memory).
constexpr int kTwoStageMinWidth = 1024;

}  // namespace

void pfsm::set_last_error(const char *msg) { g_last_error = msg; }

extern "C" {

void pfsm_default_params(pfsm_params_t *p)
{
    if (!p) return;
    p->halo = -1;
    p->fs_iters = 3;
    p->alpha_theta = 1.0;
    p->cluster_tol = 1e-5;
    p->degen_tol = 1e-8;
    p->precision = PFSM_FP64;
    p->recompute_v = 0;
    p->slice_sizes = nullptr;
    p->guard_max = 0.0;
    p->full_steps = 0;
    p->fs_adaptive = 0;
    p->fs_tol = 0.0;
    p->reduction = 0;
}

const char *pfsm_last_error(void) { return g_last_error.c_str(); }

int pfsm_init(int64_t N, int32_t nblocks, const pfsm_params_t *p, pfsm_handle_t *out)
{
    if (!out) return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: out is NULL");
    *out = nullptr;
    if (N < 1 || N > 65535) return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: N=%lld outside [1, 65535]", (long long)N);
    if (nblocks < 1 || nblocks > N)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: nblocks=%d outside [1, N]", nblocks);
    pfsm_params_t prm;
    pfsm_default_params(&prm);
    if (p) prm = *p;
    if (prm.fs_iters < 0 || prm.fs_iters > 1000) return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: fs_iters=%d", prm.fs_iters);
    if (!(prm.fs_tol >= 0.0) || (prm.fs_adaptive != 0 && prm.fs_adaptive != 1))
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: fs_adaptive must be 0 or 1 and fs_tol >= 0");
    if (prm.full_steps < 0 || prm.guard_max != prm.guard_max)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: full_steps must be >= 0 and guard_max a number");
    if (!(prm.alpha_theta > 0.0) || !(prm.cluster_tol >= 0.0) || !(prm.degen_tol >= 0.0))
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: alpha_theta must be > 0, tolerances >= 0");
    if (prm.precision != PFSM_FP64 && prm.precision != PFSM_TF32_SPLIT && prm.precision != PFSM_BF16_SPLIT)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: unknown precision %d", prm.precision);
    if (prm.reduction < 0 || prm.reduction > 2)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: reduction must be 0, 1 or 2");
    int32_t mnom = (int32_t)((N + nblocks - 1) / nblocks);
    if (prm.slice_sizes) {
        int64_t tot = 0;
        mnom = 0;
        for (int32_t b = 0; b < nblocks; b++) {
            if (prm.slice_sizes[b] < 1) return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: slice %d has size %d", b, prm.slice_sizes[b]);
            tot += prm.slice_sizes[b];
            mnom = prm.slice_sizes[b] > mnom ? prm.slice_sizes[b] : mnom;
        }
        if (tot != N) return fail(PFSM_ERR_INVALID_ARG, "pfsm_init: slice sizes sum to %lld, not N", (long long)tot);
    }
    pfsm_handle_s *h = new pfsm_handle_s();
    h->N = N;
    h->nb = nblocks;
    h->prm = prm;
    h->halo = prm.halo < 0 ? (int32_t)((N + 9) / 10) : prm.halo;
    // the cluster snap moves each boundary by at most a quarter of a nominal slice
    int64_t mmax = (int64_t)mnom + 2 * (mnom / 4);
    h->mmax = (int32_t)(mmax < N ? mmax : N);
    int64_t Mmax = (int64_t)h->mmax + 2 * (int64_t)h->halo;
    h->Mmax = (int32_t)(Mmax < N ? Mmax : N);
    // cluster shape of the tridiagonalisation
    const int Mx = h->Mmax;
    {
        cudaError_t ce = configure_kernels(h);
        if (ce == cudaSuccess) ce = select_tridiag_cluster(h, kSmemCap);
        if (ce != cudaSuccess) {
            delete h;
            cudaGetLastError();
            return fail(PFSM_ERR_CUDA, "pfsm_init: %s", cudaGetErrorString(ce));
        }
    }
    // the mixed forms' blocked reduction keeps each warp's rows of V and W in registers (up to
    // 24 rows a warp) and the window rows in shared memory for windows up to tri_mcap
    if (prm.precision != PFSM_FP64 && kUseBlockedReduction) {
        const int cl = Mx <= 128 ? 4 : (Mx <= 512 ? 8 : 16);
        const int rpw = ((Mx + cl - 1) / cl + 7) / 8;
        if (rpw <= 24) {
            h->tri_blocked = true;
            h->cl = cl;
            h->tri_rpw = rpw <= 8 ? 8 : 24;
            int mc = Mx;
            while (mc > 0 && tri_panel_smem(Mx, cl, mc) > kSmemCap) mc -= 8;
            h->tri_mcap = mc < 0 ? 0 : mc;
        }
    }

    // the mixed forms' two-stage reduction: chosen for wide windows (automatic) or on request,
    // when its kernels' shared memory and schedule allow the window width
    if (prm.precision != PFSM_FP64 && prm.reduction != 1 && band_reduction_fits(Mx, kSmemCap) &&
        (prm.reduction == 2 || Mx >= kTwoStageMinWidth)) {
        h->tri_two_stage = true;
        h->tri_blocked = false;
    }

    Workspace &w = h->ws;
    const size_t NN = (size_t)N * N;
    const int64_t ntiles = (N + kFsTileRows - 1) / kFsTileRows;
    const size_t nbM = (size_t)nblocks * h->Mmax;
    size_t ii = (size_t)nblocks * h->mmax * 5 * h->Mmax;
    // the window matrices in global memory: for rows that do not fit in shared memory, and for the
    // blocked reduction of the mixed forms, whose trailing updates run between panel launches
    if ((!h->rows_in_smem || prm.precision != PFSM_FP64) && nbM * h->Mmax > ii) ii = nbM * h->Mmax;
    cudaError_t e = cudaSuccess;
#define PFSM_ALLOC(ptr, cnt) if (e == cudaSuccess) e = alloc(&(ptr), (cnt))
    PFSM_ALLOC(w.plan, 4 * (size_t)nblocks);
    PFSM_ALLOC(w.tile_krange, 2 * (size_t)ntiles);
    PFSM_ALLOC(w.status, 1);
    PFSM_ALLOC(w.gersh, 2 * (size_t)N + 2);
    PFSM_ALLOC(w.X, NN);
    PFSM_ALLOC(w.Xfs, NN);
    PFSM_ALLOC(w.Y, NN);
    PFSM_ALLOC(w.S, NN);
    PFSM_ALLOC(w.W, NN);
    PFSM_ALLOC(w.Vrm, NN);
    PFSM_ALLOC(w.sdiag, (size_t)N);
    PFSM_ALLOC(w.Linv, (size_t)(N + 64) * 64);
    PFSM_ALLOC(w.eps, (size_t)N);
    PFSM_ALLOC(w.alpha, (size_t)N);
    PFSM_ALLOC(w.lam, (size_t)N);
    PFSM_ALLOC(w.res, (size_t)N);
    PFSM_ALLOC(w.refl, nbM * h->Mmax);
    PFSM_ALLOC(w.tau, nbM);
    PFSM_ALLOC(w.td, nbM);
    PFSM_ALLOC(w.te, nbM);
    PFSM_ALLOC(w.sel_val, (size_t)nblocks * h->mmax);
    PFSM_ALLOC(w.sel_vec, (size_t)nblocks * h->mmax * h->Mmax);
    PFSM_ALLOC(w.iiwork, ii);
    if (prm.slice_sizes) PFSM_ALLOC(w.slices, (size_t)nblocks);
    if (prm.precision != PFSM_FP64) {
        const size_t esz = slice_kind(prm.precision) == 0 ? 2 : 4;
        const size_t sl_bytes = (size_t)slices_for(prm.precision) * N * padded_ld(N) * esz;
        uint8_t *tmp[4] = {};
        for (int i = 0; i < 4; i++) {
            PFSM_ALLOC(tmp[i], sl_bytes);
            if (e == cudaSuccess) e = cudaMemset(tmp[i], 0, sl_bytes);   // zero padding columns
        }
        w.slE = tmp[0]; w.slX = tmp[1]; w.slY = tmp[2]; w.slZ = tmp[3];
        PFSM_ALLOC(w.Z, NN);
        PFSM_ALLOC(w.dA, (size_t)N);
        const size_t oz_bytes = (size_t)OZ_SLICES * N * padded_ld(N) * 2;
        uint8_t *o1 = nullptr, *o2 = nullptr;
        PFSM_ALLOC(o1, oz_bytes);
        PFSM_ALLOC(o2, oz_bytes);
        if (e == cudaSuccess) e = cudaMemset(o1, 0, oz_bytes);      // zero padding columns
        if (e == cudaSuccess) e = cudaMemset(o2, 0, oz_bytes);
        w.ozP = o1; w.ozQ = o2;
        uint8_t *o3 = nullptr;
        PFSM_ALLOC(o3, oz_bytes);
        if (e == cudaSuccess) e = cudaMemset(o3, 0, oz_bytes);
        w.ozA = o3;
        PFSM_ALLOC(w.ozeA, (size_t)N);
        PFSM_ALLOC(w.ozeP, (size_t)N);
        PFSM_ALLOC(w.ozeQ, (size_t)N);
        PFSM_ALLOC(w.L32, NN);
        PFSM_ALLOC(w.R32, NN);
        PFSM_ALLOC(w.M32, NN);
        if (e == cudaSuccess) e = cudaMemset(w.M32, 0, NN * sizeof(float));   // stays zero above the diagonal
        PFSM_ALLOC(w.F, NN);
        {
            const size_t vw = nbM * 2 * kPanel;                  // nb * Mmax rows x 2 * kPanel
            PFSM_ALLOC(w.VW, vw);
            PFSM_ALLOC(w.WV, vw);
            if (e == cudaSuccess) e = cudaMemset(w.VW, 0, vw * sizeof(double));
            if (e == cudaSuccess) e = cudaMemset(w.WV, 0, vw * sizeof(double));
            uint8_t *t1 = nullptr, *t2 = nullptr;
            PFSM_ALLOC(t1, (size_t)OZ_SLICES * vw * 2);
            PFSM_ALLOC(t2, (size_t)OZ_SLICES * vw * 2);
            w.tdP = t1; w.tdQ = t2;
            PFSM_ALLOC(w.tdeP, nbM);
            PFSM_ALLOC(w.tdeQ, nbM);
        }
        if (backtransform_wy_fits(h->Mmax) && !h->tri_two_stage) {
            const size_t Mx = (size_t)h->Mmax, mx = (size_t)h->mmax, nbx = (size_t)nblocks;
            const size_t ldk = (size_t)padded_ld(h->Mmax);
            PFSM_ALLOC(w.btG, nbx * Mx * Mx);
            PFSM_ALLOC(w.btRT, nbx * Mx * Mx);
            PFSM_ALLOC(w.btW1, nbx * Mx * mx);
            PFSM_ALLOC(w.btW2T, nbx * mx * Mx);
            PFSM_ALLOC(w.btY, nbx * mx * Mx);
            uint8_t *da = nullptr, *db = nullptr;
            PFSM_ALLOC(da, (size_t)OZ_SLICES * nbx * Mx * ldk * 2);
            PFSM_ALLOC(db, (size_t)OZ_SLICES * nbx * mx * ldk * 2);
            if (e == cudaSuccess) e = cudaMemset(da, 0, (size_t)OZ_SLICES * nbx * Mx * ldk * 2);   // padding
            if (e == cudaSuccess) e = cudaMemset(db, 0, (size_t)OZ_SLICES * nbx * mx * ldk * 2);
            w.btDA = da; w.btDB = db;
            PFSM_ALLOC(w.btEA, nbx * Mx);
            PFSM_ALLOC(w.btEB, nbx * mx);
            PFSM_ALLOC(w.btExt, 3 * nbx);
            if (e == cudaSuccess) e = configure_bt_wy_kernels();
        }
        if (h->tri_two_stage) {
            const size_t Mx = (size_t)h->Mmax, nbx = (size_t)nblocks, KBx = (size_t)kBand;
            const size_t ldk = (size_t)padded_ld(h->Mmax);
            const size_t nt = (size_t)band_tasks_per_sweep(h->Mmax), nch = (Mx + 63) / 64;
            const size_t np = (size_t)std::max(1, band_panels(h->Mmax));
            uint8_t *d1 = nullptr, *d2 = nullptr;
            PFSM_ALLOC(d1, (size_t)OZ_SLICES * nbx * Mx * ldk * 2);
            PFSM_ALLOC(d2, (size_t)OZ_SLICES * nbx * KBx * ldk * 2);
            w.bdA = d1; w.bdV = d2;
            PFSM_ALLOC(w.bdeA, nbx * Mx);
            PFSM_ALLOC(w.bdeV, nbx * KBx);
            PFSM_ALLOC(w.bExt, np * nbx);
            PFSM_ALLOC(w.bKB, nbx);
            PFSM_ALLOC(w.bY, nbx * Mx * KBx);
            PFSM_ALLOC(w.bT, np * nbx * KBx * KBx);
            PFSM_ALLOC(w.bV, np * nbx * Mx * KBx);
            // a window without some panel keeps that panel's T and reflector rows zero
            if (e == cudaSuccess) e = cudaMemset(w.bT, 0, np * nbx * KBx * KBx * sizeof(double));
            if (e == cudaSuccess) e = cudaMemset(w.bV, 0, np * nbx * Mx * KBx * sizeof(double));
            if (e == cudaSuccess) {
                std::vector<int32_t> kbv(nbx, kBand);
                e = cudaMemcpy(w.bKB, kbv.data(), nbx * sizeof(int32_t), cudaMemcpyHostToDevice);
            }
            PFSM_ALLOC(w.bU, nbx * KBx * KBx);
            PFSM_ALLOC(w.bXp, nbx * nch * KBx * KBx);
            PFSM_ALLOC(w.bBw, nbx * (Mx + 2 * KBx) * 2 * KBx);
            PFSM_ALLOC(w.bR2, nbx * Mx * nt * KBx);
            PFSM_ALLOC(w.bD, nbx * Mx);
            PFSM_ALLOC(w.bT2, nbx * Mx * nt);
            if (e == cudaSuccess) e = configure_band_kernels();
        }
        if (e == cudaSuccess) e = configure_gs_mixed_kernels();
        if (e == cudaSuccess) e = configure_tc_kernels();
        if (e == cudaSuccess) e = configure_oz_kernels();
    }
#undef PFSM_ALLOC
    if (e == cudaSuccess && prm.slice_sizes)
        e = cudaMemcpy(w.slices, prm.slice_sizes, sizeof(int32_t) * nblocks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = configure_kernels(h);
    if (e == cudaSuccess) e = configure_dense_kernels();
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? PFSM_ERR_OUT_OF_MEMORY : PFSM_ERR_CUDA;
        free_ws(h);
        delete h;
        cudaGetLastError();
        return fail(code, "pfsm_init: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < 8 && e == cudaSuccess; i++) e = cudaEventCreate(&h->ev[i]);
    for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaEventCreate(&h->sub_ev[i]);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaEventCreate(&h->gs_ev[i]);
    for (int i = 0; i < 3 && e == cudaSuccess; i++) e = cudaEventCreate(&h->band_ev[i]);
    if (prm.precision != PFSM_FP64) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_ws(h);
        delete h;
        cudaGetLastError();
        return fail(PFSM_ERR_CUDA, "pfsm_init: %s", cudaGetErrorString(e));
    }
    h->prm.slice_sizes = nullptr;   // the host array is not kept
    if ((prm.fs_adaptive || prm.precision != PFSM_FP64) &&
        cudaMalloc((void **)&h->fs_rmax, sizeof(unsigned long long)) != cudaSuccess) {
        free_ws(h);
        delete h;
        cudaGetLastError();
        return fail(PFSM_ERR_OUT_OF_MEMORY, "pfsm_init: residual buffer");
    }
    if (prm.full_steps > 0 || prm.guard_max > 0.0) {
        const cudaError_t fe = fallback_init(h);
        if (fe != cudaSuccess) {
            fallback_free(h);
            free_ws(h);
            delete h;
            cudaGetLastError();
            return fail(PFSM_ERR_CUDA, "pfsm_init: full-diagonalization setup: %s", cudaGetErrorString(fe));
        }
    }
    if (prm.precision != PFSM_FP64) {
        // tile width of the Eq. 11 products: measured on this shape (cached per shape class)
        SliceBuf sE{w.slE, N, padded_ld(N), slices_for(prm.precision), slice_kind(prm.precision)};
        h->tc_bn = tune_tc_tile(sE, sE, (int)N, (int)N, w.Z);
    }
    *out = h;
    return PFSM_OK;
}

// Eq. 11 in the mixed forms. With A = D + E (D = diag A) the iteration runs on the residual
// vectors, the same recurrence as Eq. 11:
//   Y_0 = (A - eps I) X_0 ;  Z_j = (A - eps I) Y_j ;  X_{j+1} = X_j - alpha Z_j ;
//   Y_{j+1} = Y_j - alpha (A - eps I) Z_j.
// Every tensor-core product is E times a small operand; the diagonal part is applied exactly in
// FP64 in the epilogue. Y_0 vanishes inside each start vector's window (there the start vector is
// an eigenvector of the window with eigenvalue eps), so the first product keeps only the entries
// outside the window, where no cancellation occurs.
static cudaError_t fs_mixed(pfsm_handle_s *h, const double *A, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    const int K = h->prm.fs_iters;
    if (K == 0) return cudaSuccess;
    const int ns = slices_for(h->prm.precision), kind = slice_kind(h->prm.precision);
    const int64_t ld = padded_ld(N);
    SliceBuf sE{w.slE, N, ld, ns, kind}, sY{w.slY, N, ld, ns, kind}, sZ{w.slZ, N, ld, ns, kind};
    cudaError_t e;
    // the slices of E = A - diag(A) (and diag(A)) were split on the side stream during the window
    // eigensolves when the handle has one (launch_subeig)
    if (!h->side && (e = launch_split(A, N, N, N, sE, true, w.dA, st)) != cudaSuccess) return e;
    if ((e = join_side(h, st)) != cudaSuccess) return e;
    // Y_0 = (A - eps I) X_0 is the window eigenvectors' residual E x outside each window (zero
    // inside). It is the largest operand of the recurrence (the method's residual, 5e-3 on the
    // vacancy-like matrix) and a split product loses about sqrt(N) 2^-24 of it to cancellation in
    // dense couplings, so this one product is the FP64-accurate digit product (rows of X_0 against
    // the digits of E split beside the window eigensolves), then split for the next products.
    {
        const SliceBuf dX{w.ozP, N, ld, OZ_SLICES, 0};
        const bool presplit = h->a_split;
        const SliceBuf dE{presplit ? w.ozA : w.ozQ, N, ld, OZ_SLICES, 0};
        int32_t *eE = presplit ? w.ozeA : w.ozeQ;
        if (!presplit && (e = launch_oz_split(A, N, N, N, dE, eE, st, true, w.dA)) != cudaSuccess) return e;
        if ((e = launch_oz_split(w.X, N, N, N, dX, w.ozeP, st)) != cudaSuccess) return e;
        OzParams o{};
        o.rows = (int)N; o.cols = (int)N; o.C = w.Y; o.ldc = N; o.status = w.status;
        o.krange64 = w.tile_krange; o.nrowtiles64 = (int)((N + kFsTileRows - 1) / kFsTileRows);
        o.win_plan = w.plan; o.win_nb = h->nb;
        if ((e = launch_gemm_oz(dX, w.ozeP, dE, eE, o, st)) != cudaSuccess) return e;
        if ((e = launch_split(w.Y, N, N, N, sY, false, nullptr, st)) != cudaSuccess) return e;
    }
    TcParams p{};
    p.rows = (int)N; p.cols = (int)N; p.ldo = N; p.bn = h->tc_bn;
    p.d = w.dA; p.eps = w.eps; p.alpha = w.alpha; p.status = w.status;
    p.plan = w.plan; p.nb = h->nb;
    for (int j = 0; j < K; j++) {
        TcParams z = p;
        z.epi = TC_EPI_Z; z.out = w.Z; z.V = w.Y; z.X = w.X;
        if ((e = launch_gemm_tc(sY, sE, z, j + 1 < K ? &sZ : nullptr, st)) != cudaSuccess) return e;
        if (j + 1 < K) {
            TcParams y = p;
            y.epi = TC_EPI_YN; y.out = w.Y; y.V = w.Z; y.Yold = w.Y;
            if ((e = launch_gemm_tc(sZ, sE, y, &sY, st)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

static int solve_impl(pfsm_handle_s *h, const double *A, const double *prev, double *eigvals_out,
                      double *V_out, cudaStream_t st)
{
    Workspace &w = h->ws;
    const int64_t N = h->N;
    auto mark = [&](int i) -> cudaError_t { return h->timing ? cudaEventRecord(h->ev[i], st) : cudaSuccess; };
    PFSM_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int32_t), st));
    h->a_split = false;
    PFSM_CUDA(mark(0));
    PFSM_CUDA(launch_validate_gersh(A, prev, N, w.gersh, w.status, st));
    // the conventional path: first-steps rule, then the guard (Section II)
    int path = 0;
    double g = 0.0;
    if (h->nsolves < h->prm.full_steps) {
        path = 1;
    } else if (h->prm.guard_max > 0.0) {
        PFSM_CUDA(measure_guard(h, A, st, g));
        if (!(g <= h->prm.guard_max)) path = 2;
    }
    h->nsolves++;
    h->last_path = path;
    h->last_guard = g;
    if (path != 0) {
        PFSM_CUDA(mark(1));
        PFSM_CUDA(run_full_diag(h, A, st));
        for (int i = 2; i <= 4; i++) PFSM_CUDA(mark(i));
        if (h->timing)
            for (int i = 0; i < 3; i++) PFSM_CUDA(cudaEventRecord(h->sub_ev[i], st));
        if (h->timing)
            for (int i = 0; i < 2; i++) PFSM_CUDA(cudaEventRecord(h->gs_ev[i], st));
        PFSM_CUDA(launch_rayleigh_f64(h, A, eigvals_out, V_out, st));
        PFSM_CUDA(mark(5));
        h->solved = true;
        h->last_A = A;
        h->last_prev = prev;
        h->last_stream = st;
        return PFSM_OK;
    }
    PFSM_CUDA(launch_plan(prev, N, h->nb, h->halo, h->prm.cluster_tol, w.slices, w.plan,
                          w.tile_krange, w.gersh, w.status, st));
    PFSM_CUDA(mark(1));
    PFSM_CUDA(launch_subeig(h, A, st));
    PFSM_CUDA(join_side(h, st));
    PFSM_CUDA(mark(2));
    h->last_fs_steps = h->prm.fs_iters;
    h->last_fs_resid = 0.0;
    if (h->prm.fs_adaptive) {
        // Rayleigh-quotient shifts and residual stopping (FP64 products in every precision); the
        // Gershgorin ends (for the tolerance) come back with the first residual
        double gb[2] = {0.0, 0.0};
        PFSM_CUDA(cudaMemcpyAsync(gb, w.gersh + 2 * N, sizeof(gb), cudaMemcpyDeviceToHost, st));
        unsigned long long *rmax = h->fs_rmax;
        int steps = 0;
        double r = 0.0;
        for (;;) {
            GemmArgs g{};
            g.rows = N; g.cols = N; g.K = N;
            g.P = w.X; g.ldp = N; g.Q = A; g.ldq = N; g.C = w.Y; g.ldc = N;
            g.aux_x = w.X; g.eps = w.eps;
            g.krange = (steps == 0) ? w.tile_krange : nullptr;   // start vectors vanish outside windows
            PFSM_CUDA(launch_gemm_f64(g, EPI_FS1, Q_KMAJOR, st));
            PFSM_CUDA(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), st));
            PFSM_CUDA(launch_rq_shift(w.X, w.Y, w.eps, w.alpha, w.gersh, h->prm.alpha_theta, N, rmax, st));
            unsigned long long rb = 0;
            PFSM_CUDA(cudaMemcpyAsync(&rb, rmax, sizeof(rb), cudaMemcpyDeviceToHost, st));
            PFSM_CUDA(cudaStreamSynchronize(st));
            std::memcpy(&r, &rb, sizeof(r));
            const double tol_abs = h->prm.fs_tol * std::max(std::fabs(gb[0]), std::fabs(gb[1]));
            if (r <= tol_abs || steps >= h->prm.fs_iters) break;
            GemmArgs u{};
            u.rows = N; u.cols = N; u.K = N;
            u.P = w.Y; u.ldp = N; u.Q = A; u.ldq = N; u.C = w.X; u.ldc = N;
            u.aux_y = w.Y; u.eps = w.eps; u.alpha = w.alpha;
            PFSM_CUDA(launch_gemm_f64(u, EPI_FS2, Q_KMAJOR, st));
            steps++;
        }
        h->last_fs_steps = steps;
        h->last_fs_resid = r;
    } else if (h->prm.precision != PFSM_FP64) {
        PFSM_CUDA(fs_mixed(h, A, st));
    } else
    // Eq. 11, fs_iters times: Y = (A - eps I) X ; X <- X - alpha (A - eps I) Y
    for (int it = 0; it < h->prm.fs_iters; it++) {
        GemmArgs g{};
        g.rows = N; g.cols = N; g.K = N;
        g.P = w.X; g.ldp = N; g.Q = A; g.ldq = N; g.C = w.Y; g.ldc = N;
        g.aux_x = w.X; g.eps = w.eps;
        g.krange = (it == 0) ? w.tile_krange : nullptr;   // start vectors vanish outside windows
        PFSM_CUDA(launch_gemm_f64(g, EPI_FS1, Q_KMAJOR, st));
        GemmArgs u{};
        u.rows = N; u.cols = N; u.K = N;
        u.P = w.Y; u.ldp = N; u.Q = A; u.ldq = N; u.C = w.X; u.ldc = N;
        u.aux_y = w.Y; u.eps = w.eps; u.alpha = w.alpha;
        PFSM_CUDA(launch_gemm_f64(u, EPI_FS2, Q_KMAJOR, st));
    }
    PFSM_CUDA(mark(3));
    PFSM_CUDA(cudaMemcpyAsync(w.Xfs, w.X, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    PFSM_CUDA(h->prm.precision == PFSM_FP64 ? launch_gram_schmidt_f64(h, st) : launch_gram_schmidt_mixed(h, st));
    PFSM_CUDA(mark(4));
    PFSM_CUDA(launch_rayleigh_f64(h, A, eigvals_out, V_out, st));
    PFSM_CUDA(mark(5));
    h->solved = true;
    h->last_A = A;
    h->last_prev = prev;
    h->last_stream = st;
    return PFSM_OK;
}

int pfsm_solve(pfsm_handle_t h, const double *A, const double *prev_eigvals, double *eigvals_out,
               double *V_out, void *stream)
{
    if (!h) return fail(PFSM_ERR_INVALID_ARG, "pfsm_solve: null handle");
    if (!A || !prev_eigvals || !eigvals_out || !V_out)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_solve: null buffer");
    g_launches = 0;
    int rc = solve_impl(h, A, prev_eigvals, eigvals_out, V_out, (cudaStream_t)stream);
    h->last_launches = (int32_t)g_launches;
    h->last_was_backward = false;
    return rc;
}

int pfsm_scf_step(pfsm_handle_t h, const double *H, double *Vb, const double *lam_prev, double *lam_out,
                  void *stream)
{
    if (!h) return fail(PFSM_ERR_INVALID_ARG, "pfsm_scf_step: null handle");
    if (!H || !Vb || !lam_prev || !lam_out) return fail(PFSM_ERR_INVALID_ARG, "pfsm_scf_step: null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = h->N;
    const size_t n2b = (size_t)N * N * sizeof(double);
    PFSM_CUDA(configure_oz_kernels());
    g_launches = 0;
    double *VbT = nullptr, *T = nullptr, *A = nullptr, *Vp = nullptr;
    Digits d1, d2;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };
    for (double **p : {&VbT, &T, &A, &Vp}) step(cudaMallocAsync((void **)p, n2b, st));
    step(make_digits(d1, N, st));
    step(make_digits(d2, N, st));
    int rc = PFSM_OK;
    if (e == cudaSuccess) {
        // A = sym(Vb^T H Vb): T = Vb^T H (H symmetric: its rows are its columns), A = T Vb
        step(launch_transpose(Vb, VbT, N, st));
        step(dense_product(VbT, H, T, N, d1, d2, h->ws.status, st));
        step(dense_product(T, VbT, A, N, d1, d2, h->ws.status, st));
        step(launch_symmetrize(A, T, N, st));
    }
    if (e == cudaSuccess) {
        const int launches_rot = (int)g_launches;
        rc = solve_impl(h, T, lam_prev, lam_out, Vp, st);
        if (rc == PFSM_OK) {
            // Vb <- Vb V: the solve leaves V's columns as the rows of its vector matrix X
            step(dense_product(Vb, h->ws.X, A, N, d1, d2, h->ws.status, st));
            step(cudaMemcpyAsync(Vb, A, n2b, cudaMemcpyDeviceToDevice, st));
        }
        (void)launches_rot;
    }
    free_digits(d1, st);
    free_digits(d2, st);
    for (double *p : {VbT, T, A, Vp})
        if (p) cudaFreeAsync(p, st);
    h->last_launches = (int32_t)g_launches;
    h->last_was_backward = false;
    if (e != cudaSuccess) return cuda_fail(e, "pfsm_scf_step");
    // the solve kept pointers to its inputs for pfsm_backward with recompute_v; they were temporaries
    h->last_A = nullptr;
    h->last_prev = nullptr;
    return rc;
}

int pfsm_backward(pfsm_handle_t h, const double *dLambda, const double *dV, double *dA_out,
                  void *stream)
{
    if (!h) return fail(PFSM_ERR_INVALID_ARG, "pfsm_backward: null handle");
    if (!dA_out) return fail(PFSM_ERR_INVALID_ARG, "pfsm_backward: null dA_out");
    if (!h->solved) return fail(PFSM_ERR_NO_SOLVE, "pfsm_backward: no solve on this handle yet");
    if (h->prm.recompute_v && !h->last_A)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_backward: recompute_v needs the last solve's input (none after "
                                          "pfsm_scf_step)");
    cudaStream_t st = (cudaStream_t)stream;
    g_launches = 0;
    if (h->prm.recompute_v) {
        // rebuild (lambda, V) from the last inputs; outputs land in the handle's own buffers
        int rc = solve_impl(h, h->last_A, h->last_prev, h->ws.lam, h->ws.Vrm, st);
        if (rc != PFSM_OK) return rc;
    }
    if (h->timing) PFSM_CUDA(cudaEventRecord(h->ev[6], st));
    // FP64 form: the products on the FP64 pipe; mixed forms: FP64-accurate digit products
    if (h->prm.precision == PFSM_FP64)
        PFSM_CUDA(launch_backward_f64(h, dLambda, dV, dA_out, st));
    else
        PFSM_CUDA(launch_backward_mixed(h, dLambda, dV, dA_out, st));
    if (h->timing) PFSM_CUDA(cudaEventRecord(h->ev[7], st));
    h->last_stream = st;
    h->last_launches = (int32_t)g_launches;
    h->last_was_backward = true;
    return PFSM_OK;
}

int pfsm_get_status(pfsm_handle_t h, int32_t *device_status)
{
    if (!h || !device_status) return fail(PFSM_ERR_INVALID_ARG, "pfsm_get_status: null argument");
    PFSM_CUDA(cudaStreamSynchronize(h->last_stream));
    PFSM_CUDA(cudaMemcpy(device_status, h->ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return PFSM_OK;
}

int pfsm_get_diagnostic(pfsm_handle_t h, int32_t which, void *out, void *stream)
{
    if (!h || !out) return fail(PFSM_ERR_INVALID_ARG, "pfsm_get_diagnostic: null argument");
    if (!h->solved) return fail(PFSM_ERR_NO_SOLVE, "pfsm_get_diagnostic: no solve yet");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)h->N;
    const void *src = nullptr;
    size_t bytes = 0;
    switch (which) {
    case 0: src = h->ws.res; bytes = n * 8; break;
    case 1: {
        cudaError_t e = launch_transpose(h->ws.Xfs, (double *)out, h->N, st);
        if (e != cudaSuccess) return cuda_fail(e, "transpose");
        return PFSM_OK;
    }
    case 2: src = h->ws.eps; bytes = n * 8; break;
    case 3: src = h->ws.alpha; bytes = n * 8; break;
    case 4: src = h->ws.plan; bytes = (size_t)4 * h->nb * sizeof(int32_t); break;
    default: return fail(PFSM_ERR_INVALID_ARG, "pfsm_get_diagnostic: unknown which=%d", which);
    }
    PFSM_CUDA(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, st));
    return PFSM_OK;
}

int pfsm_split_gemm(int64_t rows, int64_t cols, int64_t K, const double *P, const double *Q,
                    double *C, int32_t precision, void *stream)
{
    return pfsm_split_gemm_ex(rows, cols, K, P, Q, C, precision, 0, stream);
}

int pfsm_split_gemm_ex(int64_t rows, int64_t cols, int64_t K, const double *P, const double *Q,
                       double *C, int32_t precision, int32_t tile_n, void *stream)
{
    if (tile_n != 0 && tile_n != 64 && tile_n != 96 && tile_n != 128)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_split_gemm_ex: tile_n must be 0, 64, 96 or 128");
    if (rows < 1 || cols < 1 || K < 1 || rows > 65535 || cols > 65535 || K > (1 << 24) || !P || !Q || !C)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_split_gemm: bad size or null pointer");
    if (precision != PFSM_TF32_SPLIT && precision != PFSM_BF16_SPLIT && precision != PFSM_FP64)
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_split_gemm: unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    PFSM_CUDA(configure_tc_kernels());
    if (precision == PFSM_FP64) {       // FP64-accurate: base-128 digits, exact level sums
        PFSM_CUDA(configure_oz_kernels());
        const int64_t ld = padded_ld(K);
        void *sp = nullptr, *sq = nullptr;
        int32_t *ep = nullptr, *eq = nullptr, *status = nullptr;
        const size_t bp = (size_t)OZ_SLICES * rows * ld * 2, bq = (size_t)OZ_SLICES * cols * ld * 2;
        PFSM_CUDA(cudaMallocAsync(&sp, bp, st));
        PFSM_CUDA(cudaMallocAsync(&sq, bq, st));
        PFSM_CUDA(cudaMallocAsync((void **)&ep, rows * sizeof(int32_t), st));
        PFSM_CUDA(cudaMallocAsync((void **)&eq, cols * sizeof(int32_t), st));
        PFSM_CUDA(cudaMallocAsync((void **)&status, sizeof(int32_t), st));
        PFSM_CUDA(cudaMemsetAsync(sp, 0, bp, st));
        PFSM_CUDA(cudaMemsetAsync(sq, 0, bq, st));
        PFSM_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
        SliceBuf dp{sp, rows, ld, OZ_SLICES, 0}, dq{sq, cols, ld, OZ_SLICES, 0};
        PFSM_CUDA(launch_oz_split(P, rows, K, K, dp, ep, st));
        PFSM_CUDA(launch_oz_split(Q, cols, K, K, dq, eq, st));
        OzParams o{};
        o.rows = (int)rows; o.cols = (int)cols; o.C = C; o.ldc = cols; o.status = status;
        PFSM_CUDA(launch_gemm_oz(dp, ep, dq, eq, o, st));
        int32_t hs = 0;
        PFSM_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PFSM_CUDA(cudaFreeAsync(sp, st));
        PFSM_CUDA(cudaFreeAsync(sq, st));
        PFSM_CUDA(cudaFreeAsync(ep, st));
        PFSM_CUDA(cudaFreeAsync(eq, st));
        PFSM_CUDA(cudaFreeAsync(status, st));
        PFSM_CUDA(cudaStreamSynchronize(st));
        if (hs != 0) return fail(hs, "pfsm_split_gemm: device status %d", hs);
        return PFSM_OK;
    }
    const int ns = slices_for(precision), kind = slice_kind(precision);
    const int64_t ld = padded_ld(K);
    const size_t esz = kind == 0 ? 2 : 4;
    void *sp = nullptr, *sq = nullptr;
    int32_t *status = nullptr;
    PFSM_CUDA(cudaMallocAsync(&sp, (size_t)ns * rows * ld * esz, st));
    PFSM_CUDA(cudaMallocAsync(&sq, (size_t)ns * cols * ld * esz, st));
    PFSM_CUDA(cudaMallocAsync((void **)&status, sizeof(int32_t), st));
    PFSM_CUDA(cudaMemsetAsync(sp, 0, (size_t)ns * rows * ld * esz, st));
    PFSM_CUDA(cudaMemsetAsync(sq, 0, (size_t)ns * cols * ld * esz, st));
    PFSM_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    SliceBuf bp{sp, rows, ld, ns, kind}, bq{sq, cols, ld, ns, kind};
    PFSM_CUDA(launch_split(P, rows, K, K, bp, false, nullptr, st));
    PFSM_CUDA(launch_split(Q, cols, K, K, bq, false, nullptr, st));
    TcParams p{};
    p.rows = (int)rows; p.cols = (int)cols; p.epi = TC_EPI_STORE; p.out = C; p.ldo = cols;
    p.status = status; p.bn = tile_n;
    if (tile_n == 0) {                  // tuned (C serves as the tuner's scratch output)
        PFSM_CUDA(cudaStreamSynchronize(st));
        p.bn = tune_tc_tile(bp, bq, (int)rows, (int)cols, C);
    }
    PFSM_CUDA(launch_gemm_tc(bp, bq, p, nullptr, st));
    int32_t hs = 0;
    PFSM_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PFSM_CUDA(cudaFreeAsync(sp, st));
    PFSM_CUDA(cudaFreeAsync(sq, st));
    PFSM_CUDA(cudaFreeAsync(status, st));
    PFSM_CUDA(cudaStreamSynchronize(st));
    if (hs != 0) return fail(hs, "pfsm_split_gemm: device status %d", hs);
    return PFSM_OK;
}

static int gen2std_result(const Gen2StdResult &r, int32_t *iters_out, double *resid_out, const char *who)
{
    if (iters_out) *iters_out = r.iters;
    if (resid_out) *resid_out = r.resid;
    switch (r.status) {
    case PFSM_OK: return PFSM_OK;
    case PFSM_ERR_INVALID_ARG: return fail(PFSM_ERR_INVALID_ARG, "%s: B has a zero diagonal entry", who);
    case PFSM_ERR_NOT_SPD: return fail(PFSM_ERR_NOT_SPD, "%s: B has no positive row bound", who);
    case PFSM_ERR_NOT_CONVERGED:
        return fail(PFSM_ERR_NOT_CONVERGED, "%s: residual %.3e after %d updates", who, r.resid, r.iters);
    default: return fail(r.status, "%s: device status %d", who, r.status);
    }
}

int pfsm_gen_to_std(int64_t N, const double *A, const double *B, double *Z, int32_t max_iters, double tol,
                    int32_t *iters_out, double *resid_out, void *stream)
{
    if (N < 1 || N > 65535 || !A || !B || !Z || max_iters < 0 || !(tol >= 0.0))
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_gen_to_std: bad size, pointer, max_iters or tol");
    PFSM_CUDA(configure_oz_kernels());
    Gen2StdResult r;
    PFSM_CUDA(run_gen_to_std(N, A, B, Z, max_iters, tol, (cudaStream_t)stream, r));
    return gen2std_result(r, iters_out, resid_out, "pfsm_gen_to_std");
}

int pfsm_gen_to_std_sym(int64_t N, const double *A, const double *B, double *C, double *S, int32_t max_iters,
                        double tol, int32_t *iters_out, double *resid_out, void *stream)
{
    if (N < 1 || N > 65535 || !A || !B || !C || !S || max_iters < 0 || !(tol >= 0.0))
        return fail(PFSM_ERR_INVALID_ARG, "pfsm_gen_to_std_sym: bad size, pointer, max_iters or tol");
    PFSM_CUDA(configure_oz_kernels());
    Gen2StdResult r;
    PFSM_CUDA(run_gen_to_std_sym(N, A, B, C, S, max_iters, tol, (cudaStream_t)stream, r));
    return gen2std_result(r, iters_out, resid_out, "pfsm_gen_to_std_sym");
}

int pfsm_set_timing(pfsm_handle_t h, int32_t enable)
{
    if (!h) return fail(PFSM_ERR_INVALID_ARG, "pfsm_set_timing: null handle");
    h->timing = enable != 0;
    return PFSM_OK;
}

int pfsm_get_profile(pfsm_handle_t h, pfsm_profile_t *out)
{
    if (!h || !out) return fail(PFSM_ERR_INVALID_ARG, "pfsm_get_profile: null argument");
    std::memset(out, 0, sizeof(*out));
    out->launches = h->last_launches;
    out->gemm_tile_n = h->prm.precision != PFSM_FP64 ? h->tc_bn : 0;
    out->path = h->last_path;
    out->guard_value = h->last_guard;
    out->fs_steps = h->last_path ? 0 : h->last_fs_steps;
    out->fs_residual = h->last_path ? 0.0 : h->last_fs_resid;
    const bool gs_mixed = !h->last_path && h->prm.precision != PFSM_FP64;
    out->gs_precond = gs_mixed ? h->gs_precond : 0;
    out->gs_precond_residual = gs_mixed ? h->gs_precond_resid : 0.0;
    if (!h->timing || !h->solved) return PFSM_OK;
    PFSM_CUDA(cudaStreamSynchronize(h->last_stream));
    auto span = [&](int a, int b, float *dst) -> cudaError_t { return cudaEventElapsedTime(dst, h->ev[a], h->ev[b]); };
    const bool fwd = !h->last_was_backward || h->prm.recompute_v;
    if (fwd) {
        for (int i = 0; i < 5; i++) PFSM_CUDA(span(i, i + 1, &out->phase_ms[i]));
        // submatrix sub-phases: ev[1] | tridiag | sub_ev[0] | bisect | sub_ev[1] | inverse
        // iteration | sub_ev[2] | back-transform | ev[2]
        cudaEvent_t seq[5] = {h->ev[1], h->sub_ev[0], h->sub_ev[1], h->sub_ev[2], h->ev[2]};
        for (int i = 0; i < 4; i++) PFSM_CUDA(cudaEventElapsedTime(&out->phase_ms[6 + i], seq[i], seq[i + 1]));
        PFSM_CUDA(cudaEventElapsedTime(&out->phase_ms[10], h->ev[3], h->gs_ev[0]));
        PFSM_CUDA(cudaEventElapsedTime(&out->phase_ms[11], h->gs_ev[0], h->gs_ev[1]));
        if (h->tri_two_stage && h->last_path == 0 && !h->last_was_backward) {
            PFSM_CUDA(cudaEventElapsedTime(&out->band_ms[0], h->ev[1], h->band_ev[0]));
            PFSM_CUDA(cudaEventElapsedTime(&out->band_ms[1], h->band_ev[0], h->band_ev[1]));
            PFSM_CUDA(cudaEventElapsedTime(&out->band_ms[2], h->sub_ev[2], h->band_ev[2]));
            PFSM_CUDA(cudaEventElapsedTime(&out->band_ms[3], h->band_ev[2], h->ev[2]));
        }
    }
    if (h->last_was_backward) PFSM_CUDA(span(6, 7, &out->phase_ms[5]));
    out->timed = 1;
    return PFSM_OK;
}

int pfsm_destroy(pfsm_handle_t h)
{
    if (!h) return PFSM_OK;
    cudaDeviceSynchronize();
    for (int i = 0; i < 8; i++)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (int i = 0; i < 4; i++)
        if (h->sub_ev[i]) cudaEventDestroy(h->sub_ev[i]);
    for (int i = 0; i < 2; i++)
        if (h->gs_ev[i]) cudaEventDestroy(h->gs_ev[i]);
    for (int i = 0; i < 3; i++)
        if (h->band_ev[i]) cudaEventDestroy(h->band_ev[i]);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    fallback_free(h);
    if (h->fs_rmax) cudaFree(h->fs_rmax);
    free_ws(h);
    delete h;
    return PFSM_OK;
}

}  // extern "C"
