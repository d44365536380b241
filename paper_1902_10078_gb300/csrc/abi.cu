// extern "C" entry points of the banded operator library (include/banded.h).
#include <cstdint>

#include "common.cuh"
#include "products.cuh"
#include "sweep_cta.cuh"
#include "sweep_impl.cuh"

using namespace bnd;

namespace {

inline cudaStream_t S(void *stream) { return (cudaStream_t)stream; }

inline bnd_status ok_or(cudaError_t e) { return e == cudaSuccess ? BND_OK : BND_ECUDA; }

// Right-hand sides one sweep carries: 4 in the register-window kernels; 16 when
// every instance is of the wide class (l = 0 or l above the register-window
// limit), whose kernels take the column count at run time.
int rhs_block(const bnd_plan *p) { return p->class_task0[1] == p->ntasks ? kCtaMaxK : kMaxK; }

bnd_status check_plan(const bnd_plan *p) {
    if (!p || !p->bound) return BND_EINVAL;
    return BND_OK;
}

bnd_status check_ptr(const bnd_plan *p, const void *ptr, bool required = true) {
    if (!ptr) return required ? BND_EINVAL : BND_OK;
    const size_t esz = p->dtype == BND_F32 ? 4 : 8;
    if (((uintptr_t)ptr % esz) != 0) return BND_EALIGN;
    return BND_OK;
}

#define BND_TRY(x)                      \
    do {                                \
        bnd_status _st = (x);           \
        if (_st != BND_OK) return _st;  \
    } while (0)
#define BND_CUDA(x)                                  \
    do {                                             \
        cudaError_t _e = (x);                        \
        if (_e != cudaSuccess) return BND_ECUDA;     \
    } while (0)

template <typename T>
SweepArgs<T> blank_args(const bnd_plan *p) {
    SweepArgs<T> A{};
    A.scratch = (T *)p->dev.band_tmp2;
    A.scratch2 = (T *)p->dev.band_tmp3;
    A.kk = 0;
    return A;
}

// Zero the generic-path scratch pools when the plan has wide-band instances.
template <typename T>
cudaError_t zero_generic_scratch(const bnd_plan *p, cudaStream_t s) {
    if (!p->has_generic) return cudaSuccess;
    const size_t bytes = sizeof(T) * (size_t)p->band_pool_elems;
    cudaError_t e = cudaMemsetAsync(p->dev.band_tmp2, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->dev.band_tmp3, 0, bytes, s);
    return e;
}

inline void fixcount_reset(const bnd_plan *p, int kind, cudaStream_t s) {
    cudaMemsetAsync(p->dev.counters + kNumSweepKinds + kind, 0, sizeof(unsigned int), s);
}

template <typename T>
cudaError_t fwd(const bnd_plan *p, int fl, SweepArgs<T> A, cudaStream_t s) {
    fixcount_reset(p, A.kind, s);
    if (fl & (F_ALG4)) { cudaError_t e = zero_generic_scratch<T>(p, s); if (e != cudaSuccess) return e; }
    const int K = A.kk <= 0 ? 0 : (A.kk == 1 ? 1 : 4);
    return launch_fwd<T>(p, fl, K, A, s);
}

template <typename T>
cudaError_t bwd(const bnd_plan *p, int fl, SweepArgs<T> A, cudaStream_t s) {
    fixcount_reset(p, A.kind, s);
    if (fl & (B_ALG2)) { cudaError_t e = zero_generic_scratch<T>(p, s); if (e != cudaSuccess) return e; }
    const int K = A.kk <= 0 ? 0 : (A.kk == 1 ? 1 : 4);
    return launch_bwd<T>(p, fl, K, A, s);
}

// ---------------------------------------------------------------------------
template <typename T>
bnd_status cholesky_t(const bnd_plan *p, const void *Q, void *L, double *logdet, int32_t *info, cudaStream_t s) {
    SweepArgs<T> A = blank_args<T>(p);
    A.Q = (const T *)Q; A.L = (T *)L; A.logdet = logdet; A.info = info;
    A.kind = kSweepChol;
    return ok_or(fwd<T>(p, F_CHOL, A, s));
}

template <typename T>
bnd_status solve_t(const bnd_plan *p, const void *L, const void *B, void *X, int mode, cudaStream_t s) {
    const int kb = rhs_block(p);
    for (int r0 = 0; r0 < p->k; r0 += kb) {
        const int kk = (p->k - r0) < kb ? (p->k - r0) : kb;
        SweepArgs<T> A = blank_args<T>(p);
        A.Lin = (const T *)L; A.rhs0 = r0; A.kk = kk;
        if (mode == 0 || mode == 1) {
            A.Bin = (const T *)B; A.Xout = (T *)X;
            A.kind = mode == 0 ? kSweepFSolve : kSweepBSolve;
            cudaError_t e = mode == 0 ? fwd<T>(p, F_SOLVE, A, s) : bwd<T>(p, B_SOLVE, A, s);
            if (e != cudaSuccess) return BND_ECUDA;
        } else {
            A.Bin = (const T *)B; A.Xout = (T *)p->dev.rhs_tmp; A.kind = kSweepFSolve;
            BND_CUDA(fwd<T>(p, F_SOLVE, A, s));
            A.Bin = (const T *)p->dev.rhs_tmp; A.Xout = (T *)X; A.kind = kSweepBSolve;
            BND_CUDA(bwd<T>(p, B_SOLVE, A, s));
        }
    }
    return BND_OK;
}

template <typename T>
bnd_status outer_t(const bnd_plan *p, const void *M, const void *V, void *C, int clo, int cup, int acc, T alpha,
                   cudaStream_t s) {
    OuterArgs<T> A{};
    A.M = (const T *)M; A.V = (const T *)V; A.C = (T *)C;
    A.clo = clo; A.cup = cup; A.k = p->k; A.acc = acc; A.alpha = alpha;
    return ok_or(launch_outer<T>(p, A, s));
}

template <typename T>
bnd_status matvec_t(const bnd_plan *p, const void *Am, int alo, int aup, int transA, const void *V, void *P, int acc,
                    T alpha, cudaStream_t s) {
    MatvecArgs<T> A{};
    A.A = (const T *)Am; A.V = (const T *)V; A.P = (T *)P;
    A.alo = alo; A.aup = aup; A.transA = transA; A.k = p->k; A.acc = acc; A.alpha = alpha;
    return ok_or(launch_matvec<T>(p, A, s));
}

template <typename T>
bnd_status product_t(const bnd_plan *p, const void *Am, int alo, int aup, int ta, const void *Bm, int blo, int bup,
                     int tb, void *Cm, int clo, int cup, int acc, T alpha, cudaStream_t s) {
    ProdArgs<T> A{};
    A.A = (const T *)Am; A.B = (const T *)Bm; A.C = (T *)Cm;
    A.alo = alo; A.aup = aup; A.blo = blo; A.bup = bup; A.clo = clo; A.cup = cup;
    A.transA = ta; A.transB = tb; A.acc = acc; A.alpha = alpha;
    return ok_or(launch_product<T>(p, A, s));
}

// Table 1, solve: Lbar (+)= -band(vbar s^T) (mode 0) or -band(s vbar^T) (mode 1)
template <typename T>
bnd_status solve_vjp_t(const bnd_plan *p, const void *L, const void *X, const void *Xbar, int mode, void *Bbar,
                       void *Lbar, int acc, cudaStream_t s) {
    if (mode == 0 || mode == 1) {
        void *vbar = Bbar ? Bbar : p->dev.rhs_tmp;
        BND_TRY(solve_t<T>(p, L, Xbar, vbar, mode == 0 ? 1 : 0, s));
        if (Lbar) {
            // lower band of the outer product: rows j..j+l of column j
            if (mode == 0) BND_TRY(outer_t<T>(p, vbar, X, Lbar, -1, 0, acc, T(-1), s));
            else BND_TRY(outer_t<T>(p, X, vbar, Lbar, -1, 0, acc, T(-1), s));
        }
        return BND_OK;
    }
    // mode 2: X = L^{-T} Y, Y = L^{-1} B
    void *ybar = p->dev.rhs_tmp;
    void *y = p->dev.rhs_tmp2;
    BND_TRY(solve_t<T>(p, L, Xbar, ybar, 0, s));                       // Ybar = L^{-1} Xbar
    void *bbar = Bbar;
    if (!bbar) return BND_EINVAL;                                      // needs a buffer for Bbar
    BND_TRY(solve_t<T>(p, L, ybar, bbar, 1, s));                       // Bbar = L^{-T} Ybar
    if (Lbar) {
        BND_TRY(matvec_t<T>(p, L, -1, 0, 1, X, y, 0, T(1), s));  // Y = L^T X
        BND_TRY(outer_t<T>(p, X, ybar, Lbar, -1, 0, acc, T(-1), s));
        BND_TRY(outer_t<T>(p, bbar, y, Lbar, -1, 0, 1, T(-1), s));
    }
    return BND_OK;
}

template <typename T>
bnd_status subinv_t(const bnd_plan *p, const void *L, void *Sout, cudaStream_t s) {
    SweepArgs<T> A = blank_args<T>(p);
    A.Lin = (const T *)L; A.Sout = (T *)Sout; A.kind = kSweepTaka;
    return ok_or(bwd<T>(p, B_TAKA, A, s));
}

template <typename T>
bnd_status subinv_vjp_t(const bnd_plan *p, const void *L, const void *Sm, const void *Sbar, void *Lbar, int acc,
                        cudaStream_t s) {
    SweepArgs<T> A = blank_args<T>(p);
    A.Lin = (const T *)L; A.S = (const T *)Sm; A.Sbar = (const T *)Sbar; A.Lbar = (T *)Lbar; A.acc = acc;
    A.kind = kSweepTakaBar;
    // a segment rerun by the verify pass rewrites its columns; to accumulate exactly once,
    // segmented plans write to scratch and add it afterwards
    const bool via_tmp = acc && p->nsegs > p->count;
    if (via_tmp) { A.Lbar = (T *)p->dev.band_tmp; A.acc = 0; }
    BND_CUDA(fwd<T>(p, F_ALG4, A, s));
    if (via_tmp) BND_CUDA(launch_band_add<T>(p, (const T *)p->dev.band_tmp, (T *)Lbar, s));
    return BND_OK;
}

template <typename T>
bnd_status chol_vjp_t(const bnd_plan *p, const void *L, const void *Lbar, const double *ldbar, void *Qbar, int acc,
                      cudaStream_t s) {
    SweepArgs<T> A = blank_args<T>(p);
    A.Lin = (const T *)L; A.Lbar_in = (const T *)Lbar; A.Qbar = (T *)Qbar; A.acc = acc; A.ldbar = ldbar;
    A.kind = kSweepCholBar;
    const bool via_tmp = acc && p->nsegs > p->count;     // see subinv_vjp_t
    if (via_tmp) { A.Qbar = (T *)p->dev.band_tmp; A.acc = 0; }
    BND_CUDA(bwd<T>(p, B_ALG2, A, s));
    if (via_tmp) BND_CUDA(launch_band_add<T>(p, (const T *)p->dev.band_tmp, (T *)Qbar, s));
    return BND_OK;
}

template <typename T>
bnd_status gmm_forward_t(const bnd_plan *p, const void *Q, const void *B, void *L, void *X, void *Sout,
                         double *logdet, int32_t *info, cudaStream_t s) {
    SweepArgs<T> A = blank_args<T>(p);
    A.Q = (const T *)Q; A.L = (T *)L; A.logdet = logdet; A.info = info;
    A.Bin = (const T *)B; A.Xout = (T *)p->dev.rhs_tmp; A.rhs0 = 0; A.kk = p->k;
    A.kind = kSweepChol;
    BND_CUDA(fwd<T>(p, F_CHOL | F_SOLVE, A, s));
    SweepArgs<T> Bw = blank_args<T>(p);
    Bw.Lin = (const T *)L; Bw.Sout = (T *)Sout;
    Bw.Bin = (const T *)p->dev.rhs_tmp; Bw.Xout = (T *)X; Bw.rhs0 = 0; Bw.kk = p->k;
    Bw.kind = kSweepTaka;
    BND_CUDA(bwd<T>(p, B_TAKA | B_SOLVE, Bw, s));
    return BND_OK;
}

template <typename T>
bnd_status gmm_backward_t(const bnd_plan *p, const void *L, const void *X, const void *Sm, const void *Xbar,
                          const void *Sbar, const double *ldbar, void *Qbar, void *Bbar, cudaStream_t s) {
    // forward sweep: Ybar = L^{-1} Xbar and Lbar_partial = Ibar(L, S, Sbar)
    SweepArgs<T> A = blank_args<T>(p);
    A.Lin = (const T *)L; A.S = (const T *)Sm; A.Sbar = (const T *)Sbar; A.Lbar = (T *)p->dev.band_tmp; A.acc = 0;
    A.Bin = (const T *)Xbar; A.Xout = (T *)p->dev.rhs_tmp; A.rhs0 = 0; A.kk = p->k;
    A.kind = kSweepTakaBar;
    BND_CUDA(fwd<T>(p, F_ALG4 | F_SOLVE, A, s));
    // backward sweep: Bbar = L^{-T} Ybar, Lbar += outer terms + log-det term, Qbar = Cbar(L, Lbar)
    SweepArgs<T> Bw = blank_args<T>(p);
    Bw.Lin = (const T *)L; Bw.Lbar_in = (const T *)p->dev.band_tmp; Bw.Qbar = (T *)Qbar; Bw.acc = 0;
    Bw.Bin = (const T *)p->dev.rhs_tmp; Bw.Ybar = (const T *)p->dev.rhs_tmp;
    Bw.Xout = (T *)(Bbar ? Bbar : p->dev.rhs_tmp2); Bw.Xin = (const T *)X; Bw.rhs0 = 0; Bw.kk = p->k;
    Bw.ldbar = ldbar;
    Bw.kind = kSweepCholBar;
    BND_CUDA(bwd<T>(p, B_ALG2 | B_SOLVE | B_OUTER, Bw, s));
    return BND_OK;
}

}  // namespace

// ===========================================================================
// extern "C"
// ===========================================================================
#define BND_DISPATCH(call_f32, call_f64) ((p->dtype == BND_F32) ? (call_f32) : (call_f64))

extern "C" bnd_status banded_cholesky(const bnd_plan *p, const void *Q, void *L, double *logdet, int32_t *info,
                                      void *stream) {
    BND_TRY(check_plan(p));
    BND_TRY(check_ptr(p, Q)); BND_TRY(check_ptr(p, L));
    if (!info) return BND_EINVAL;
    return BND_DISPATCH(cholesky_t<float>(p, Q, L, logdet, info, S(stream)),
                        cholesky_t<double>(p, Q, L, logdet, info, S(stream)));
}

extern "C" bnd_status banded_cholesky_vjp(const bnd_plan *p, const void *L, const void *Lbar, const double *ldbar,
                                          void *Qbar, int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, Lbar)); BND_TRY(check_ptr(p, Qbar));
    return BND_DISPATCH(chol_vjp_t<float>(p, L, Lbar, ldbar, Qbar, accumulate != 0, S(stream)),
                        chol_vjp_t<double>(p, L, Lbar, ldbar, Qbar, accumulate != 0, S(stream)));
}

extern "C" bnd_status banded_solve(const bnd_plan *p, const void *L, const void *B, void *X, int32_t mode,
                                   void *stream) {
    BND_TRY(check_plan(p));
    if (mode < 0 || mode > 2 || p->k < 1) return BND_EINVAL;
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, B)); BND_TRY(check_ptr(p, X));
    if (B == X) return BND_EINVAL;
    return BND_DISPATCH(solve_t<float>(p, L, B, X, mode, S(stream)), solve_t<double>(p, L, B, X, mode, S(stream)));
}

extern "C" bnd_status banded_solve_vjp(const bnd_plan *p, const void *L, const void *X, const void *Xbar,
                                       int32_t mode, void *Bbar, void *Lbar, int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    if (mode < 0 || mode > 2 || p->k < 1) return BND_EINVAL;
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, X)); BND_TRY(check_ptr(p, Xbar));
    BND_TRY(check_ptr(p, Bbar, false)); BND_TRY(check_ptr(p, Lbar, false));
    if (mode == 2 && !Bbar) return BND_EINVAL;
    return BND_DISPATCH(solve_vjp_t<float>(p, L, X, Xbar, mode, Bbar, Lbar, accumulate != 0, S(stream)),
                        solve_vjp_t<double>(p, L, X, Xbar, mode, Bbar, Lbar, accumulate != 0, S(stream)));
}

extern "C" bnd_status banded_subset_inverse(const bnd_plan *p, const void *L, void *Sout, void *stream) {
    BND_TRY(check_plan(p));
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, Sout));
    return BND_DISPATCH(subinv_t<float>(p, L, Sout, S(stream)), subinv_t<double>(p, L, Sout, S(stream)));
}

extern "C" bnd_status banded_subset_inverse_vjp(const bnd_plan *p, const void *L, const void *Sm, const void *Sbar,
                                                void *Lbar, int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, Sm)); BND_TRY(check_ptr(p, Sbar)); BND_TRY(check_ptr(p, Lbar));
    return BND_DISPATCH(subinv_vjp_t<float>(p, L, Sm, Sbar, Lbar, accumulate != 0, S(stream)),
                        subinv_vjp_t<double>(p, L, Sm, Sbar, Lbar, accumulate != 0, S(stream)));
}

extern "C" bnd_status banded_gmm_forward(const bnd_plan *p, const void *Q, const void *B, void *L, void *X,
                                         void *Sout, double *logdet, int32_t *info, void *stream) {
    BND_TRY(check_plan(p));
    if (p->k < 1 || p->k > rhs_block(p) || !info) return BND_EINVAL;
    BND_TRY(check_ptr(p, Q)); BND_TRY(check_ptr(p, B)); BND_TRY(check_ptr(p, L));
    BND_TRY(check_ptr(p, X)); BND_TRY(check_ptr(p, Sout));
    return BND_DISPATCH(gmm_forward_t<float>(p, Q, B, L, X, Sout, logdet, info, S(stream)),
                        gmm_forward_t<double>(p, Q, B, L, X, Sout, logdet, info, S(stream)));
}

extern "C" bnd_status banded_gmm_backward(const bnd_plan *p, const void *L, const void *X, const void *Sm,
                                          const void *Xbar, const void *Sbar, const double *ldbar, void *Qbar,
                                          void *Bbar, void *stream) {
    BND_TRY(check_plan(p));
    if (p->k < 1 || p->k > rhs_block(p)) return BND_EINVAL;
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, X)); BND_TRY(check_ptr(p, Sm));
    BND_TRY(check_ptr(p, Xbar)); BND_TRY(check_ptr(p, Sbar)); BND_TRY(check_ptr(p, Qbar));
    BND_TRY(check_ptr(p, Bbar, false));
    return BND_DISPATCH(gmm_backward_t<float>(p, L, X, Sm, Xbar, Sbar, ldbar, Qbar, Bbar, S(stream)),
                        gmm_backward_t<double>(p, L, X, Sm, Xbar, Sbar, ldbar, Qbar, Bbar, S(stream)));
}

// lo < 0 selects each instance's own bandwidth l (mixed-l batches)
static bool band_ok(int lo, int up) { return lo >= -1 && up >= 0 && lo <= 2048 && up <= 2048; }

extern "C" bnd_status banded_product(const bnd_plan *p, const void *Am, int32_t alo, int32_t aup, int32_t transA,
                                     const void *Bm, int32_t blo, int32_t bup, int32_t transB, void *Cm, int32_t clo,
                                     int32_t cup, int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    if (!band_ok(alo, aup) || !band_ok(blo, bup) || !band_ok(clo, cup)) return BND_EINVAL;
    BND_TRY(check_ptr(p, Am)); BND_TRY(check_ptr(p, Bm)); BND_TRY(check_ptr(p, Cm));
    if (Cm == Am || Cm == Bm) return BND_EINVAL;
    return BND_DISPATCH(
        product_t<float>(p, Am, alo, aup, transA != 0, Bm, blo, bup, transB != 0, Cm, clo, cup, accumulate != 0, 1.0f, S(stream)),
        product_t<double>(p, Am, alo, aup, transA != 0, Bm, blo, bup, transB != 0, Cm, clo, cup, accumulate != 0, 1.0, S(stream)));
}

extern "C" bnd_status banded_outer(const bnd_plan *p, const void *M, const void *V, void *Cm, int32_t clo,
                                   int32_t cup, int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    if (!band_ok(clo, cup) || p->k < 1) return BND_EINVAL;
    BND_TRY(check_ptr(p, M)); BND_TRY(check_ptr(p, V)); BND_TRY(check_ptr(p, Cm));
    return BND_DISPATCH(outer_t<float>(p, M, V, Cm, clo, cup, accumulate != 0, 1.0f, S(stream)),
                        outer_t<double>(p, M, V, Cm, clo, cup, accumulate != 0, 1.0, S(stream)));
}

extern "C" bnd_status banded_matvec(const bnd_plan *p, const void *Am, int32_t alo, int32_t aup, int32_t transA,
                                    const void *V, void *P, int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    if (!band_ok(alo, aup) || p->k < 1) return BND_EINVAL;
    BND_TRY(check_ptr(p, Am)); BND_TRY(check_ptr(p, V)); BND_TRY(check_ptr(p, P));
    if (P == V) return BND_EINVAL;
    return BND_DISPATCH(matvec_t<float>(p, Am, alo, aup, transA != 0, V, P, accumulate != 0, 1.0f, S(stream)),
                        matvec_t<double>(p, Am, alo, aup, transA != 0, V, P, accumulate != 0, 1.0, S(stream)));
}

// Table 1, product matrix-matrix (band-projected adjoints)
template <typename T>
static bnd_status product_vjp_t(const bnd_plan *p, const void *Am, int alo, int aup, int ta, const void *Bm, int blo,
                                int bup, int tb, const void *Cbar, int clo, int cup, void *Abar, void *Bbar, int acc,
                                cudaStream_t s) {
    if (Abar) {
        if (!ta) BND_TRY(product_t<T>(p, Cbar, clo, cup, 0, Bm, blo, bup, !tb, Abar, alo, aup, acc, T(1), s));
        else BND_TRY(product_t<T>(p, Bm, blo, bup, tb, Cbar, clo, cup, 1, Abar, alo, aup, acc, T(1), s));
    }
    if (Bbar) {
        if (!tb) BND_TRY(product_t<T>(p, Am, alo, aup, !ta, Cbar, clo, cup, 0, Bbar, blo, bup, acc, T(1), s));
        else BND_TRY(product_t<T>(p, Cbar, clo, cup, 1, Am, alo, aup, ta, Bbar, blo, bup, acc, T(1), s));
    }
    return BND_OK;
}

extern "C" bnd_status banded_product_vjp(const bnd_plan *p, const void *Am, int32_t alo, int32_t aup,
                                         int32_t transA, const void *Bm, int32_t blo, int32_t bup, int32_t transB,
                                         const void *Cbar, int32_t clo, int32_t cup, void *Abar, void *Bbar,
                                         int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    if (!band_ok(alo, aup) || !band_ok(blo, bup) || !band_ok(clo, cup)) return BND_EINVAL;
    BND_TRY(check_ptr(p, Am)); BND_TRY(check_ptr(p, Bm)); BND_TRY(check_ptr(p, Cbar));
    BND_TRY(check_ptr(p, Abar, false)); BND_TRY(check_ptr(p, Bbar, false));
    return BND_DISPATCH(
        product_vjp_t<float>(p, Am, alo, aup, transA != 0, Bm, blo, bup, transB != 0, Cbar, clo, cup, Abar, Bbar, accumulate != 0, S(stream)),
        product_vjp_t<double>(p, Am, alo, aup, transA != 0, Bm, blo, bup, transB != 0, Cbar, clo, cup, Abar, Bbar, accumulate != 0, S(stream)));
}

// Alg. 5 and its Table 1 adjoint ("solve matrix-matrix")
template <typename T>
static bnd_status solve_band_t(const bnd_plan *p, const void *L, const void *R, int rlo, int rup, void *O, int olo,
                               int oup, int trans, cudaStream_t s) {
    SolveBandArgs<T> A{};
    A.L = (const T *)L; A.R = (const T *)R; A.O = (T *)O;
    A.rlo = rlo; A.rup = rup; A.olo = olo; A.oup = oup; A.trans = trans;
    return ok_or(launch_solve_band<T>(p, A, s));
}

template <typename T>
static bnd_status solve_band_vjp_t(const bnd_plan *p, const void *L, const void *O, int olo, int oup, const void *Obar,
                                   int trans, int rlo, int rup, void *G, void *Rbar, void *Lbar, int acc,
                                   cudaStream_t s) {
    BND_TRY(solve_band_t<T>(p, L, Obar, olo, oup, G, olo, oup, !trans, s));       // G = op(L)^{-T} Obar
    if (Rbar) {
        BandCopyArgs<T> A{};
        A.src = (const T *)G; A.dst = (T *)Rbar; A.slo = olo; A.sup = oup; A.dlo = rlo; A.dup = rup; A.acc = acc;
        BND_CUDA(launch_band_copy<T>(p, A, s));
    }
    if (Lbar) {            // Lbar -= band_l(G O^T)  (or band_l(O G^T) for the transposed solve)
        if (!trans) BND_TRY(product_t<T>(p, G, olo, oup, 0, O, olo, oup, 1, Lbar, -1, 0, acc, T(-1), s));
        else BND_TRY(product_t<T>(p, O, olo, oup, 0, G, olo, oup, 1, Lbar, -1, 0, acc, T(-1), s));
    }
    return BND_OK;
}

static bool solve_band_shape_ok(int rlo, int rup, int olo, int oup, int trans) {
    if (!band_ok(rlo, rup) || !band_ok(olo, oup) || rlo < 0 || olo < 0) return false;
    return trans ? olo >= rlo : oup >= rup;           // the computed band holds every nonzero it needs
}

extern "C" bnd_status banded_solve_band(const bnd_plan *p, const void *L, const void *R, int32_t rlo, int32_t rup,
                                        void *O, int32_t olo, int32_t oup, int32_t trans, void *stream) {
    BND_TRY(check_plan(p));
    if (!solve_band_shape_ok(rlo, rup, olo, oup, trans != 0)) return BND_EINVAL;
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, R)); BND_TRY(check_ptr(p, O));
    if (O == R || O == L) return BND_EINVAL;
    return BND_DISPATCH(solve_band_t<float>(p, L, R, rlo, rup, O, olo, oup, trans != 0, S(stream)),
                        solve_band_t<double>(p, L, R, rlo, rup, O, olo, oup, trans != 0, S(stream)));
}

extern "C" bnd_status banded_solve_band_vjp(const bnd_plan *p, const void *L, const void *O, int32_t olo, int32_t oup,
                                            const void *Obar, int32_t trans, int32_t rlo, int32_t rup, void *G,
                                            void *Rbar, void *Lbar, int32_t accumulate, void *stream) {
    BND_TRY(check_plan(p));
    if (!solve_band_shape_ok(rlo, rup, olo, oup, trans != 0)) return BND_EINVAL;
    BND_TRY(check_ptr(p, L)); BND_TRY(check_ptr(p, O)); BND_TRY(check_ptr(p, Obar)); BND_TRY(check_ptr(p, G));
    BND_TRY(check_ptr(p, Rbar, false)); BND_TRY(check_ptr(p, Lbar, false));
    if (G == O || G == Obar || G == L || (Rbar && (Rbar == G || Rbar == Obar)) || (Lbar && Lbar == G))
        return BND_EINVAL;
    return BND_DISPATCH(
        solve_band_vjp_t<float>(p, L, O, olo, oup, Obar, trans != 0, rlo, rup, G, Rbar, Lbar, accumulate != 0, S(stream)),
        solve_band_vjp_t<double>(p, L, O, olo, oup, Obar, trans != 0, rlo, rup, G, Rbar, Lbar, accumulate != 0, S(stream)));
}

extern "C" const char *bnd_version(void) { return "banded-gb300 0.1 (sm_103a)"; }
