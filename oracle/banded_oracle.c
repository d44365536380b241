/*
 * Plain FP64 CPU oracle for the banded operators of Durrande et al.,
 * "Banded Matrix Operators for Gaussian Markov Models in the Automatic
 * Differentiation Era" (arXiv 1902.10078).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code with the CUDA library (paper_1902_10078_gb300/csrc), and the CUDA
 * library never calls it.
 *
 * Every function works on ONE instance, written with the paper's dense (i, j)
 * indexing over band storage (App. B: the algorithms are stated densely but
 * touch only the band).  Loops follow the paper's order; there is no blocking,
 * no fusion and no reordering.  Floating-point contraction is disabled at
 * build time (-ffp-contract=off) so x86 and Arm builds give identical bits.
 *
 * Storage (Sec. 4.3): a band matrix with lower/upper bandwidths (lo, up) is an
 * (lo+up+1) x n array B' with  B[i, j] = B'[up + i - j][j]  (0-based reading
 * of the paper's index formula; row stride ld >= n).  For lower-banded
 * matrices (up = 0) this is B'[i - j][j].  Corner entries whose row i falls
 * outside [0, n) are never read; outputs write 0 there.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *  - Alg. 1: the inner loop "j in max(i-l,0) to i+1" has an exclusive upper
 *    bound, so j runs up to and including i.
 *  - Alg. 2: the innermost loop "for l in j-1, in j_stop" re-uses the symbol
 *    l; it is read as k = j-1 down to j_stop inclusive.  The result Q_b is the
 *    gradient with respect to the LOWER stored entries of Q (each
 *    off-diagonal stored entry stands for Q_ij and Q_ji).
 *  - Alg. 3 and Alg. 4: the symbol l (and the undefined k of Alg. 4) in the
 *    slices U[i, i+1:i+l] and the loop bounds denote the band HEIGHT l+1,
 *    with exclusive slice ends; so m runs over i+1 .. i+l and i over
 *    j .. max(j-l, 0).
 *  - Alg. 4: "bS treated as symmetric" means the lower triangle starts with
 *    the upstream gradient of the stored entries and the upper triangle
 *    starts at zero; the algorithm itself moves gradient between the two.
 *  - Table 1, solve with a vector: Lbar = -band_l(vbar s^T) where
 *    s = L^{-1} v and vbar = L^{-T} sbar (the appendix derivation drops the
 *    minus sign and writes u for ubar).
 *  - Product and outer-product adjoints are projected onto the band of the
 *    operand they are the gradient of (Sec. 4.2, point (2) after Table 1).
 *  - Cholesky of a non-SPD input: the paper is silent.  The first row r whose
 *    pivot is not > 0 is reported as info = r + 1 (LAPACK pbtrf style); rows
 *    r .. n-1 of L are then filled with NaN.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

static i64 imax(i64 a, i64 b) { return a > b ? a : b; }
static i64 imin(i64 a, i64 b) { return a < b ? a : b; }

/* Lower-band accessor, Sec. 4.3 with up = 0: M[i, j] at m[(i - j) * ld + j]. */
#define LB(m, ld, i, j) ((m)[(size_t)((i) - (j)) * (size_t)(ld) + (size_t)(j)])

/* General band accessor with upper bandwidth up: M[i, j] at m[(up + i - j) * ld + j]. */
#define GB(m, ld, up, i, j) ((m)[(size_t)((up) + (i) - (j)) * (size_t)(ld) + (size_t)(j)])

/* Zero a lower band array including its corners. */
static void lb_zero(i64 n, int l, double *m, i64 ld)
{
    for (int d = 0; d <= l; ++d)
        for (i64 j = 0; j < n; ++j) m[(size_t)d * ld + j] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (App. B): Cholesky of a banded SPD matrix, row by row.             */
/* ------------------------------------------------------------------------ */
int orc_cholesky(i64 n, int l, const double *Q, i64 ldq, double *L, i64 ldl)
{
    lb_zero(n, l, L, ldl);                       /* "Initialize L with zeros" */
    for (i64 i = 0; i < n; ++i) {
        for (i64 j = imax(i - l, 0); j <= i; ++j) {
            i64 m = imax(imax(i - l, j - l), 0);
            double s = 0.0;                      /* s = sum(L[i, m:j] * L[j, m:j]) */
            for (i64 t = m; t < j; ++t) s += LB(L, ldl, i, t) * LB(L, ldl, j, t);
            if (i == j) {
                double piv = LB(Q, ldq, i, i) - s;
                if (!(piv > 0.0)) {              /* not SPD: report row i, NaN the rest */
                    for (i64 r = i; r < n; ++r)
                        for (i64 c = imax(r - l, 0); c <= r; ++c) LB(L, ldl, r, c) = NAN;
                    return (int)(i + 1);
                }
                LB(L, ldl, i, j) = sqrt(piv);
            } else {
                LB(L, ldl, i, j) = (LB(Q, ldq, i, j) - s) / LB(L, ldl, j, j);
            }
        }
    }
    return 0;
}

/* log det Q = 2 * sum_i log L_ii  (Sec. 3.1 and App. C.5: log|Lambda| = 2 sum log C_ii). */
double orc_logdet(i64 n, const double *L)
{
    double s = 0.0;
    for (i64 i = 0; i < n; ++i) s += log(L[i]);
    return 2.0 * s;
}

/* ------------------------------------------------------------------------ */
/* Triangular solves S (Sec. 4.1): trans = 0 gives L^{-1} B (forward        */
/* substitution), trans = 1 gives L^{-T} B (back substitution).  The inner  */
/* loop starts at the beginning of the band.  B and X hold k columns, column */
/* r at offset r * ldb (resp. r * ldx); X may alias B.                       */
/* ------------------------------------------------------------------------ */
void orc_solve(i64 n, int l, const double *L, i64 ldl, int trans, int k,
               const double *B, i64 ldb, double *X, i64 ldx)
{
    for (int r = 0; r < k; ++r) {
        const double *b = B + (size_t)r * ldb;
        double *x = X + (size_t)r * ldx;
        if (!trans) {
            for (i64 i = 0; i < n; ++i) {
                double s = b[i];
                for (i64 m = imax(i - l, 0); m < i; ++m) s -= LB(L, ldl, i, m) * x[m];
                x[i] = s / LB(L, ldl, i, i);
            }
        } else {
            for (i64 i = n - 1; i >= 0; --i) {
                double s = b[i];
                for (i64 m = i + 1; m <= imin(i + l, n - 1); ++m) s -= LB(L, ldl, m, i) * x[m];
                x[i] = s / LB(L, ldl, i, i);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 (App. B): lower band of (L L^T)^{-1} from L (Takahashi).           */
/* Sym is a symmetric band with both bandwidths l: general storage, up = l.  */
/* ------------------------------------------------------------------------ */
void orc_subset_inverse(i64 n, int l, const double *L, i64 ldl, double *S, i64 lds)
{
    i64 ldw = n;
    double *Sym = (double *)calloc((size_t)(2 * l + 1) * (size_t)ldw, sizeof(double));
    double *vec = (double *)malloc((size_t)n * sizeof(double));
    double *U = (double *)calloc((size_t)(l + 1) * (size_t)ldw, sizeof(double)); /* U[i, i+e] at U[e*ldw + i] */
    for (i64 i = 0; i < n; ++i) vec[i] = LB(L, ldl, i, i);          /* vec = diag(L) */
    for (i64 i = 0; i < n; ++i)                                       /* U = transpose(L / vec) */
        for (i64 m = i; m <= imin(i + l, n - 1); ++m)
            U[(size_t)(m - i) * ldw + i] = LB(L, ldl, m, i) / vec[i];
#define UU(i, m) U[(size_t)((m) - (i)) * ldw + (i)]
#define SY(i, j) GB(Sym, ldw, l, i, j)
    for (i64 j = n - 1; j >= 0; --j) {
        for (i64 i = j; i >= imax(j - l, 0); --i) {
            double s = 0.0;                   /* sum(U[i, i+1:i+k] Sym[i+1:i+k, j]), k = l+1 */
            for (i64 m = i + 1; m <= imin(i + l, n - 1); ++m) s += UU(i, m) * SY(m, j);
            SY(i, j) = -s;
            SY(j, i) = SY(i, j);
            if (i == j) SY(i, i) += 1.0 / (vec[i] * vec[i]);
        }
    }
    lb_zero(n, l, S, lds);                    /* S = lower_band(Sym) */
    for (i64 j = 0; j < n; ++j)
        for (i64 i = j; i <= imin(j + l, n - 1); ++i) LB(S, lds, i, j) = SY(i, j);
#undef UU
#undef SY
    free(Sym); free(vec); free(U);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 (App. B): reverse mode of Alg. 1.  Lbar is copied (the algorithm   */
/* updates it in place); Qbar is the gradient w.r.t. the lower stored        */
/* entries of Q.                                                             */
/* ------------------------------------------------------------------------ */
void orc_cholesky_vjp(i64 n, int l, const double *L, i64 ldl, const double *Lbar, i64 ldlb,
                      double *Qbar, i64 ldqb)
{
    double *Lb = (double *)malloc((size_t)(l + 1) * (size_t)n * sizeof(double));
    for (int d = 0; d <= l; ++d)
        for (i64 j = 0; j < n; ++j) Lb[(size_t)d * n + j] = (j + d < n) ? Lbar[(size_t)d * ldlb + j] : 0.0;
    lb_zero(n, l, Qbar, ldqb);                       /* "Initialize Q_b with zeros" */
    for (i64 i = n - 1; i >= 0; --i) {
        i64 jstop = imax(i - l, 0);
        for (i64 j = i; j >= jstop; --j) {
            if (j == i) {
                LB(Qbar, ldqb, i, i) = 0.5 * LB(Lb, n, i, i) / LB(L, ldl, i, i);
            } else {
                LB(Qbar, ldqb, i, j) = LB(Lb, n, i, j) / LB(L, ldl, j, j);
                LB(Lb, n, j, j) -= LB(Lb, n, i, j) * LB(L, ldl, i, j) / LB(L, ldl, j, j);
            }
            for (i64 k = j - 1; k >= jstop; --k) {
                LB(Lb, n, i, k) -= LB(Qbar, ldqb, i, j) * LB(L, ldl, j, k);
                LB(Lb, n, j, k) -= LB(Qbar, ldqb, i, j) * LB(L, ldl, i, k);
            }
        }
    }
    free(Lb);
}

/* ------------------------------------------------------------------------ */
/* Alg. 4 (App. B): reverse mode of Alg. 3.  Output Lbar (lower band) is the  */
/* gradient w.r.t. the stored entries of L; accumulate = 1 adds into Lbar.   */
/* ------------------------------------------------------------------------ */
void orc_subset_inverse_vjp(i64 n, int l, const double *L, i64 ldl, const double *S, i64 lds,
                            const double *Sbar, i64 ldsb, double *Lbar, i64 ldlb, int accumulate)
{
    i64 ldw = n;
    double *bS = (double *)calloc((size_t)(2 * l + 1) * (size_t)ldw, sizeof(double));
    double *bU = (double *)calloc((size_t)(l + 1) * (size_t)ldw, sizeof(double)); /* bU[i, i+e] at e*ldw+i */
    double *U = (double *)calloc((size_t)(l + 1) * (size_t)ldw, sizeof(double));
    double *vec = (double *)malloc((size_t)n * sizeof(double));
    double *bvec_inv_2 = (double *)calloc((size_t)n, sizeof(double));
    double *bvec = (double *)malloc((size_t)n * sizeof(double));
#define SYM(i, j) ((i) >= (j) ? LB(S, lds, i, j) : LB(S, lds, j, i))
#define BS(i, j) GB(bS, ldw, l, i, j)
#define UU(i, m) U[(size_t)((m) - (i)) * ldw + (i)]
#define BU(i, m) bU[(size_t)((m) - (i)) * ldw + (i)]
    /* bS: lower triangle holds Sbar on the stored entries, upper starts at 0. */
    for (i64 j = 0; j < n; ++j)
        for (i64 i = j; i <= imin(j + l, n - 1); ++i) BS(i, j) = LB(Sbar, ldsb, i, j);
    for (i64 i = 0; i < n; ++i) vec[i] = LB(L, ldl, i, i);          /* vec = diag(L) */
    for (i64 i = 0; i < n; ++i)                                       /* U = transpose(L / vec) */
        for (i64 m = i; m <= imin(i + l, n - 1); ++m) UU(i, m) = LB(L, ldl, m, i) / vec[i];

    for (i64 j = 0; j < n; ++j) {
        for (i64 i = imax(0, j - l); i <= j; ++i) {
            if (i == j) bvec_inv_2[i] += BS(i, i);
            /* grad of Sym[j, i] = Sym[i, j] */
            double tmp = BS(j, i);
            BS(j, i) = 0.0;
            BS(i, j) += tmp;
            /* grad of Sym[i, j] = -sum(U[i, i+1:i+k] Sym[i+1:i+k, j]) */
            for (i64 m = i + 1; m <= imin(i + l, n - 1); ++m) {
                BU(i, m) -= SYM(m, j) * BS(i, j);
                BS(m, j) -= UU(i, m) * BS(i, j);
            }
            BS(i, j) = 0.0;
        }
    }
    /* grad of U = transpose(L / vec):  bL = transpose(bU) / vec */
    if (!accumulate) lb_zero(n, l, Lbar, ldlb);
    for (i64 i = 0; i < n; ++i)
        for (i64 m = i + 1; m <= imin(i + l, n - 1); ++m) LB(Lbar, ldlb, m, i) += BU(i, m) / vec[i];
    /* grad of 1 / vec^2 */
    for (i64 i = 0; i < n; ++i) bvec[i] = -2.0 * bvec_inv_2[i] / (vec[i] * vec[i] * vec[i]);
    /* grad of 1 / vec:  bvec -= sum(transpose(bU) * L, 0) / vec^2 */
    for (i64 i = 0; i < n; ++i) {
        double s = 0.0;
        for (i64 m = i; m <= imin(i + l, n - 1); ++m) s += BU(i, m) * LB(L, ldl, m, i);
        bvec[i] -= s / (vec[i] * vec[i]);
    }
    /* grad of vec = diag(L) */
    for (i64 i = 0; i < n; ++i) LB(Lbar, ldlb, i, i) += bvec[i];
#undef SYM
#undef BS
#undef UU
#undef BU
    free(bS); free(bU); free(U); free(vec); free(bvec_inv_2); free(bvec);
}

/* ------------------------------------------------------------------------ */
/* Products P (Sec. 4.1).  C = op(A) op(B) projected onto C's band           */
/* (clo, cup); op(X) = X or X^T.  Every operand uses general band storage.   */
/* ------------------------------------------------------------------------ */
static double gb_get(const double *m, i64 ld, int lo, int up, int trans, i64 n, i64 i, i64 j)
{
    if (trans) { i64 t = i; i = j; j = t; }
    if (i < 0 || j < 0 || i >= n || j >= n) return 0.0;
    if (i - j > lo || j - i > up) return 0.0;
    return GB(m, ld, up, i, j);
}

void orc_product(i64 n, const double *A, i64 lda, int alo, int aup, int transA,
                 const double *B, i64 ldb, int blo, int bup, int transB,
                 double *C, i64 ldc, int clo, int cup)
{
    int alo_op = transA ? aup : alo, aup_op = transA ? alo : aup;
    for (int r = 0; r < clo + cup + 1; ++r)
        for (i64 j = 0; j < n; ++j) C[(size_t)r * ldc + j] = 0.0;
    for (i64 j = 0; j < n; ++j) {
        for (i64 i = imax(j - cup, 0); i <= imin(j + clo, n - 1); ++i) {
            double s = 0.0;
            for (i64 t = imax(i - alo_op, 0); t <= imin(i + aup_op, n - 1); ++t)
                s += gb_get(A, lda, alo, aup, transA, n, i, t) * gb_get(B, ldb, blo, bup, transB, n, t, j);
            GB(C, ldc, cup, i, j) = s;
        }
    }
}

/* Band matrix times k vectors: P = op(A) V (Sec. 4.1, "product between a banded
 * matrix and a vector").  Column r of V at V + r*ldv. */
void orc_band_matvec(i64 n, const double *A, i64 lda, int alo, int aup, int transA,
                     int k, const double *V, i64 ldv, double *P, i64 ldp)
{
    int alo_op = transA ? aup : alo, aup_op = transA ? alo : aup;
    for (int r = 0; r < k; ++r)
        for (i64 i = 0; i < n; ++i) {
            double s = 0.0;
            for (i64 t = imax(i - alo_op, 0); t <= imin(i + aup_op, n - 1); ++t)
                s += gb_get(A, lda, alo, aup, transA, n, i, t) * V[(size_t)r * ldv + t];
            P[(size_t)r * ldp + i] = s;
        }
}

/* Band-projected outer product O (Sec. 4.1): C = band_{clo,cup}(sum_r m_r v_r^T). */
void orc_outer(i64 n, int k, const double *M, i64 ldm, const double *V, i64 ldv,
               double *C, i64 ldc, int clo, int cup)
{
    for (int r = 0; r < clo + cup + 1; ++r)
        for (i64 j = 0; j < n; ++j) C[(size_t)r * ldc + j] = 0.0;
    for (i64 j = 0; j < n; ++j)
        for (i64 i = imax(j - cup, 0); i <= imin(j + clo, n - 1); ++i) {
            double s = 0.0;
            for (int r = 0; r < k; ++r) s += M[(size_t)r * ldm + i] * V[(size_t)r * ldv + j];
            GB(C, ldc, cup, i, j) = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Table 1 compositions.                                                     */
/* ------------------------------------------------------------------------ */

/* Solve with k vectors, s = L^{-1} v (trans = 0) or s = L^{-T} v (trans = 1).
 * Given s (the forward output) and sbar:
 *   vbar = S(L^T, sbar)                 (trans = 0)   or S(L, sbar) (trans = 1)
 *   Lbar += -band_l(vbar s^T)           (trans = 0)
 *   Lbar += -band_l(s vbar^T)           (trans = 1: the transposed solve)
 * vbar is written to Vbar (k columns); Lbar is accumulated (lower band). */
void orc_solve_vjp(i64 n, int l, const double *L, i64 ldl, int trans, int k,
                   const double *S, i64 lds, const double *Sbar, i64 ldsb,
                   double *Vbar, i64 ldvb, double *Lbar, i64 ldlb)
{
    orc_solve(n, l, L, ldl, !trans, k, Sbar, ldsb, Vbar, ldvb);
    double *O = (double *)malloc((size_t)(l + 1) * (size_t)n * sizeof(double));
    if (!trans) orc_outer(n, k, Vbar, ldvb, S, lds, O, n, l, 0);
    else        orc_outer(n, k, S, lds, Vbar, ldvb, O, n, l, 0);
    for (int d = 0; d <= l; ++d)
        for (i64 j = 0; j + d < n; ++j) Lbar[(size_t)d * ldlb + j] -= O[(size_t)d * n + j];
    free(O);
}

/* Matrix-matrix product C = op(A) op(B) (Table 1, first row), projected:
 *   G_A = Cbar op(B)^T,  Abar = band_A(G_A) or band_A(G_A^T) when transA
 *   G_B = op(A)^T Cbar,  Bbar = band_B(G_B) or band_B(G_B^T) when transB */
void orc_product_vjp(i64 n, const double *A, i64 lda, int alo, int aup, int transA,
                     const double *B, i64 ldb, int blo, int bup, int transB,
                     const double *Cbar, i64 ldcb, int clo, int cup,
                     double *Abar, i64 ldab, double *Bbar, i64 ldbb)
{
    if (Abar) {
        if (!transA) /* Abar = Cbar op(B)^T */
            orc_product(n, Cbar, ldcb, clo, cup, 0, B, ldb, blo, bup, !transB, Abar, ldab, alo, aup);
        else         /* Abar = op(B) Cbar^T */
            orc_product(n, B, ldb, blo, bup, transB, Cbar, ldcb, clo, cup, 1, Abar, ldab, alo, aup);
    }
    if (Bbar) {
        if (!transB) /* Bbar = op(A)^T Cbar */
            orc_product(n, A, lda, alo, aup, !transA, Cbar, ldcb, clo, cup, 0, Bbar, ldbb, blo, bup);
        else         /* Bbar = Cbar^T op(A) */
            orc_product(n, Cbar, ldcb, clo, cup, 1, A, lda, alo, aup, transA, Bbar, ldbb, blo, bup);
    }
}

/* Band-times-vector product p = op(A) v (Table 1, second row):
 *   Abar = O(pbar, v) projected (or O(v, pbar) when transA),  vbar = op(A)^T pbar */
void orc_band_matvec_vjp(i64 n, const double *A, i64 lda, int alo, int aup, int transA,
                         int k, const double *V, i64 ldv, const double *Pbar, i64 ldpb,
                         double *Abar, i64 ldab, double *Vbar, i64 ldvb)
{
    if (Abar) {
        if (!transA) orc_outer(n, k, Pbar, ldpb, V, ldv, Abar, ldab, alo, aup);
        else         orc_outer(n, k, V, ldv, Pbar, ldpb, Abar, ldab, alo, aup);
    }
    if (Vbar) orc_band_matvec(n, A, lda, alo, aup, !transA, k, Pbar, ldpb, Vbar, ldvb);
}

/* Outer product O = band(sum_r m_r v_r^T) (Table 1, third row):
 *   mbar = P(Obar, v),  vbar = P(Obar^T, m) */
void orc_outer_vjp(i64 n, int k, const double *M, i64 ldm, const double *V, i64 ldv,
                   const double *Obar, i64 ldob, int olo, int oup,
                   double *Mbar, i64 ldmb, double *Vbar, i64 ldvb)
{
    if (Mbar) orc_band_matvec(n, Obar, ldob, olo, oup, 0, k, V, ldv, Mbar, ldmb);
    if (Vbar) orc_band_matvec(n, Obar, ldob, olo, oup, 1, k, M, ldm, Vbar, ldvb);
}

/* ------------------------------------------------------------------------ */
/* The uneven-batch step: for each instance                                  */
/*   forward : L = C(Q), ld = log det Q, X = Q^{-1} B = S(L^T, S(L, B)),     */
/*             S = I(L)                                                      */
/*   backward: given Xbar, Sbar and ldbar                                    */
/*             Lbar  = Ibar(L, S, Sbar)                        (Alg. 4)      */
/*             Ybar, Lbar += S-bar of X = L^{-T} Y             (Table 1)     */
/*             Bbar, Lbar += S-bar of Y = L^{-1} B             (Table 1)     */
/*             Lbar_ii += 2 ldbar / L_ii                       (log det)     */
/*             Qbar = Cbar(L, Lbar)                            (Alg. 2)      */
/* Instances are independent; OpenMP distributes whole instances over host   */
/* threads and each instance runs the steps above in order.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    i64 n; int l; int k;
    const double *Q; const double *B; const double *Xbar; const double *Sbar; double ldbar;
    double *L; double *X; double *S; double *Qbar; double *Bbar; double *logdet; int *info;
} orc_step_io;

static void step_one(const orc_step_io *io)
{
    i64 n = io->n; int l = io->l, k = io->k;
    *io->info = orc_cholesky(n, l, io->Q, n, io->L, n);
    *io->logdet = *io->info ? NAN : orc_logdet(n, io->L);
    double *Y = (double *)malloc((size_t)k * (size_t)n * sizeof(double));
    double *Ybar = (double *)malloc((size_t)k * (size_t)n * sizeof(double));
    double *Lbar = (double *)calloc((size_t)(l + 1) * (size_t)n, sizeof(double));
    orc_solve(n, l, io->L, n, 0, k, io->B, n, Y, n);
    orc_solve(n, l, io->L, n, 1, k, Y, n, io->X, n);
    orc_subset_inverse(n, l, io->L, n, io->S, n);
    orc_subset_inverse_vjp(n, l, io->L, n, io->S, n, io->Sbar, n, Lbar, n, 0);
    orc_solve_vjp(n, l, io->L, n, 1, k, io->X, n, io->Xbar, n, Ybar, n, Lbar, n);
    orc_solve_vjp(n, l, io->L, n, 0, k, Y, n, Ybar, n, io->Bbar, n, Lbar, n);
    for (i64 i = 0; i < n; ++i) Lbar[i] += 2.0 * io->ldbar / io->L[i];
    orc_cholesky_vjp(n, l, io->L, n, Lbar, n, io->Qbar, n);
    free(Y); free(Ybar); free(Lbar);
}

/* Runs `count` instances; returns the number of host threads used. */
int orc_batch_step(int count, const orc_step_io *io)
{
    int threads = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        threads = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < count; ++c) step_one(&io[c]);
    return threads;
}
