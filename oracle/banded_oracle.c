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
 * Every function works on ONE instance, written with dense (i, j) indexing
 * over band storage (the operators touch only the band).  The Cholesky and
 * the solves follow the paper's row-by-row recurrences (Alg. 1, Sec. 4.1);
 * the subset inverse is derived from the identity L^T Sigma = L^{-1}, and the
 * two adjoints are the reverse mode of those recurrences, each written out
 * with its derivation above the function.  There is no blocking and no
 * fusion.  Floating-point contraction is disabled at build time
 * (-ffp-contract=off) so x86 and Arm builds give identical bits.
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
 *  - Cholesky adjoint (Alg. 2): Qbar is the gradient with respect to the
 *    LOWER stored entries of Q (each off-diagonal stored entry stands for
 *    Q_ij and Q_ji), because the factorisation reads only those.
 *  - Subset-inverse adjoint (Alg. 4): Sbar is the gradient with respect to
 *    the stored (lower) entries of S; each unordered pair {i, j} of the
 *    symmetric Sigma is one variable whose adjoint starts at Sbar.
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
/* Cholesky C (Sec. 4.1, Alg. 1) of a banded SPD matrix, row by row.         */
/* ------------------------------------------------------------------------ */
int orc_cholesky(i64 n, int l, const double *Q, i64 ldq, double *L, i64 ldl)
{
    lb_zero(n, l, L, ldl);
    for (i64 i = 0; i < n; ++i) {
        for (i64 j = imax(i - l, 0); j <= i; ++j) {
            i64 m = imax(imax(i - l, j - l), 0);
            double s = 0.0;                      /* inner product of rows i and j of L left of column j */
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
/* Subset inverse I (Sec. 4.1, Alg. 3): S = lower band of Sigma = (L L^T)^-1. */
/*                                                                           */
/* Derived from Sigma = L^{-T} L^{-1}, i.e. L^T Sigma = L^{-1}.  L^{-1} is   */
/* lower triangular with diagonal 1 / L_ii, so entry (i, j), j >= i, of      */
/* L^T Sigma = L^{-1} reads                                                  */
/*     L_ii Sigma_ij + sum_{k=i+1}^{i+l} L_ki Sigma_kj = [i == j] / L_ii,     */
/* which gives Sigma_ij from entries of rows below i.  Rows are taken from   */
/* the last one up; inside row i the off-diagonal entries j = i+l .. i+1     */
/* first (they use only rows below i), then the diagonal (it uses them).    */
/* Every Sigma_kj referenced has |k - j| <= l, so only the band is needed;   */
/* the symmetric entry (k, j) with k < j is read as (j, k).                  */
/* ------------------------------------------------------------------------ */
void orc_subset_inverse(i64 n, int l, const double *L, i64 ldl, double *S, i64 lds)
{
#define SIG(a, b) ((a) >= (b) ? LB(S, lds, a, b) : LB(S, lds, b, a))
    lb_zero(n, l, S, lds);
    for (i64 i = n - 1; i >= 0; --i) {
        i64 last = imin(i + l, n - 1);
        double lii = LB(L, ldl, i, i);
        for (i64 j = last; j >= i; --j) {
            double acc = (j == i) ? 1.0 / lii : 0.0;
            for (i64 k = i + 1; k <= last; ++k) acc -= LB(L, ldl, k, i) * SIG(k, j);
            LB(S, lds, j, i) = acc / lii;
        }
    }
#undef SIG
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the Cholesky (Alg. 2), derived by differentiating the     */
/* entries of L as functions of Q.  Forward, column by column:               */
/*     a_ij = Q_ij - sum_{k=max(i-l,0)}^{j-1} L_ik L_jk      (j <= i <= j+l)   */
/*     L_jj = sqrt(a_jj),   L_ij = a_ij / L_jj  (i > j).                     */
/* The adjoints are taken in the exact reverse order: columns from the last  */
/* one down, inside a column the off-diagonal entries from the bottom up,    */
/* then the diagonal (which every off-diagonal entry of its column uses):    */
/*     abar_ij = Lbar_ij / L_jj;  Lbar_jj -= abar_ij L_ij          (i > j)   */
/*     abar_jj = Lbar_jj / (2 L_jj)                                          */
/*     Qbar_ij = abar_ij;  for each k in the sum:                            */
/*         Lbar_ik -= abar_ij L_jk,  Lbar_jk -= abar_ij L_ik                  */
/* (for i = j both updates hit Lbar_jk).  The forward reads only the lower   */
/* entries of Q, so Qbar is the gradient w.r.t. the LOWER stored entries     */
/* (an off-diagonal stored entry stands for Q_ij and Q_ji).  Lbar is copied. */
/* ------------------------------------------------------------------------ */
void orc_cholesky_vjp(i64 n, int l, const double *L, i64 ldl, const double *Lbar, i64 ldlb,
                      double *Qbar, i64 ldqb)
{
    double *G = (double *)malloc((size_t)(l + 1) * (size_t)n * sizeof(double));   /* running Lbar */
    for (int d = 0; d <= l; ++d)
        for (i64 j = 0; j < n; ++j) G[(size_t)d * n + j] = (j + d < n) ? Lbar[(size_t)d * ldlb + j] : 0.0;
    lb_zero(n, l, Qbar, ldqb);
    for (i64 j = n - 1; j >= 0; --j) {
        double ljj = LB(L, ldl, j, j);
        for (i64 i = imin(j + l, n - 1); i >= j; --i) {
            double abar;
            if (i > j) {
                abar = LB(G, n, i, j) / ljj;
                LB(G, n, j, j) -= abar * LB(L, ldl, i, j);
            } else {
                abar = LB(G, n, j, j) / (2.0 * ljj);
            }
            LB(Qbar, ldqb, i, j) = abar;
            for (i64 k = imax(i - l, 0); k < j; ++k) {
                LB(G, n, i, k) -= abar * LB(L, ldl, j, k);
                LB(G, n, j, k) -= abar * LB(L, ldl, i, k);
            }
        }
    }
    free(G);
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the subset inverse (Alg. 4), derived by differentiating   */
/* the recursion of orc_subset_inverse above.  Each unordered pair {i, j}    */
/* of Sigma is one variable, so its adjoint sits on the stored entry (the    */
/* lower one) and starts as Sbar.  With t_ij = sum_{k=i+1}^{i+l} L_ki Sigma_kj: */
/*     Sigma_ij = -t_ij / L_ii                         (j > i)                */
/*     Sigma_ii = 1 / L_ii^2 - t_ii / L_ii                                   */
/* so, for g = Sigma-bar_ij:                                                 */
/*     Lbar_ii += g (t_ij / L_ii^2)            (j > i)                       */
/*     Lbar_ii += g (-2 / L_ii^3 + t_ii / L_ii^2)   (j = i)                   */
/*     Lbar_ki -= g Sigma_kj / L_ii,   Sigma-bar_kj -= g L_ki / L_ii          */
/* The forward takes rows from the last up and, in a row, the diagonal       */
/* last; the reverse takes rows from the first down and, in a row, the       */
/* diagonal first.  Row i only feeds adjoints of pairs whose smaller index  */
/* is > i, or of its own off-diagonal pairs (through the diagonal), so every */
/* adjoint is complete when it is consumed.  Sigma is read from S (the       */
/* forward output).  accumulate = 1 adds into Lbar.                          */
/* ------------------------------------------------------------------------ */
void orc_subset_inverse_vjp(i64 n, int l, const double *L, i64 ldl, const double *S, i64 lds,
                            const double *Sbar, i64 ldsb, double *Lbar, i64 ldlb, int accumulate)
{
    double *G = (double *)calloc((size_t)(l + 1) * (size_t)n, sizeof(double));   /* pair adjoints */
#define SIG(a, b) ((a) >= (b) ? LB(S, lds, a, b) : LB(S, lds, b, a))
#define GP(a, b) (*((a) >= (b) ? &LB(G, n, a, b) : &LB(G, n, b, a)))
    for (int d = 0; d <= l; ++d)
        for (i64 j = 0; j + d < n; ++j) G[(size_t)d * n + j] = Sbar[(size_t)d * ldsb + j];
    if (!accumulate) lb_zero(n, l, Lbar, ldlb);
    for (i64 i = 0; i < n; ++i) {
        i64 last = imin(i + l, n - 1);
        double lii = LB(L, ldl, i, i);
        for (i64 j = i; j <= last; ++j) {
            double g = GP(j, i);
            double t = 0.0;
            for (i64 k = i + 1; k <= last; ++k) t += LB(L, ldl, k, i) * SIG(k, j);
            if (j == i) LB(Lbar, ldlb, i, i) += g * (-2.0 / (lii * lii * lii) + t / (lii * lii));
            else        LB(Lbar, ldlb, i, i) += g * t / (lii * lii);
            for (i64 k = i + 1; k <= last; ++k) {
                LB(Lbar, ldlb, k, i) -= g * SIG(k, j) / lii;
                GP(k, j) -= g * LB(L, ldl, k, i) / lii;
            }
        }
    }
#undef SIG
#undef GP
    free(G);
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
/* Solve with a banded right-hand side (Alg. 5): O = band_{olo,oup}(L^{-1} R) */
/* (trans = 0) or band_{olo,oup}(L^{-T} R) (trans = 1), R a general band     */
/* (rlo, rup).  Diagonal by diagonal, in the order Alg. 5 gives for the      */
/* lower solve: offset k = row - column from -oup up to olo (trans = 0; each */
/* entry uses only entries of its column on smaller offsets), or from olo    */
/* down to -oup (trans = 1, the mirror order of the upper solve).  Entries   */
/* outside the computed band are taken as 0; they are exactly 0 when         */
/* oup >= rup (trans = 0: L^{-1} R has upper bandwidth rup) or olo >= rlo    */
/* (trans = 1: L^{-T} R has lower bandwidth rlo), which callers must ensure  */
/* for an exact band.                                                        */
/* ------------------------------------------------------------------------ */
void orc_solve_band(i64 n, int l, const double *L, i64 ldl, int trans,
                    const double *R, i64 ldr, int rlo, int rup,
                    double *O, i64 ldo, int olo, int oup)
{
    for (int r = 0; r < olo + oup + 1; ++r)
        for (i64 j = 0; j < n; ++j) O[(size_t)r * ldo + j] = 0.0;
    for (int kk = 0; kk <= olo + oup; ++kk) {
        int k = trans ? olo - kk : kk - oup;                 /* diagonal offset i - c */
        for (i64 i = imax(0, k); i <= imin(n - 1, n - 1 + k); ++i) {
            i64 c = i - k;
            double rv = (k <= rlo && -k <= rup) ? GB(R, ldr, rup, i, c) : 0.0;
            double s = 0.0;
            if (!trans) {                                    /* sum_m L[i, m] O[m, c], m < i */
                for (i64 m = imax(i - l, 0); m < i; ++m)
                    if (m - c >= -oup && m - c <= olo) s += LB(L, ldl, i, m) * GB(O, ldo, oup, m, c);
            } else {                                         /* sum_m L[m, i] O[m, c], m > i */
                for (i64 m = i + 1; m <= imin(i + l, n - 1); ++m)
                    if (m - c >= -oup && m - c <= olo) s += LB(L, ldl, m, i) * GB(O, ldo, oup, m, c);
            }
            GB(O, ldo, oup, i, c) = (rv - s) / LB(L, ldl, i, i);
        }
    }
}

/* Reverse mode of orc_solve_band (Table 1, "solve matrix-matrix"): for
 * O = band(L^{-1} R) and its cotangent Obar (both on O's band (olo, oup)):
 *   G = band_{olo,oup}(L^{-T} Obar),  Rbar = band_R(G),  Lbar -= band_l(G O^T);
 * for O = band(L^{-T} R):
 *   G = band_{olo,oup}(L^{-1} Obar),  Rbar = band_R(G),  Lbar -= band_l(O G^T).
 * Lbar is accumulated (lower band l); Rbar is written on R's band (rlo, rup). */
void orc_solve_band_vjp(i64 n, int l, const double *L, i64 ldl, int trans,
                        const double *O, i64 ldo, int olo, int oup, const double *Obar, i64 ldob,
                        int rlo, int rup, double *Rbar, i64 ldrb, double *Lbar, i64 ldlb)
{
    double *G = (double *)malloc((size_t)(olo + oup + 1) * (size_t)n * sizeof(double));
    double *P = (double *)malloc((size_t)(l + 1) * (size_t)n * sizeof(double));
    orc_solve_band(n, l, L, ldl, !trans, Obar, ldob, olo, oup, G, n, olo, oup);
    if (Rbar) {
        for (int r = 0; r < rlo + rup + 1; ++r)
            for (i64 j = 0; j < n; ++j) Rbar[(size_t)r * ldrb + j] = 0.0;
        for (i64 c = 0; c < n; ++c)
            for (i64 i = imax(c - rup, 0); i <= imin(c + rlo, n - 1); ++i)
                if (i - c <= olo && c - i <= oup) GB(Rbar, ldrb, rup, i, c) = GB(G, n, oup, i, c);
    }
    if (Lbar) {
        if (!trans) orc_product(n, G, n, olo, oup, 0, O, ldo, olo, oup, 1, P, n, l, 0);
        else        orc_product(n, O, ldo, olo, oup, 0, G, n, olo, oup, 1, P, n, l, 0);
        for (int d = 0; d <= l; ++d)
            for (i64 j = 0; j + d < n; ++j) Lbar[(size_t)d * ldlb + j] -= P[(size_t)d * n + j];
    }
    free(G); free(P);
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
