/*
 * banded.h -- C ABI of the GB300 banded SPD operator library.
 *
 * The library implements the banded linear-algebra operators of Durrande et
 * al., "Banded Matrix Operators for Gaussian Markov Models in the Automatic
 * Differentiation Era" (arXiv 1902.10078), and their reverse-mode adjoints,
 * as CUDA kernels for sm_103a.  Every entry point is batched: one call runs
 * `count` independent instances of uneven order n and lower bandwidth l.
 *
 * ---------------------------------------------------------------------------
 * Storage (Sec. 4.3).  A band matrix with lower/upper bandwidths (lo, up) is
 * an (lo+up+1) x n array B' with  B[i, j] = B'[up + i - j][j]  (0-based
 * reading of the paper's index formula).  Lower-banded operands (L, and the
 * symmetric Q, S, Qbar, Sbar stored by their lower half) use up = 0:
 *     B'[d][j] = B[j + d, j],   d = 0..l.
 * Element (d, j) of instance i lives at
 *     pool[inst[i].band + d * inst[i].ld + j * cs_i],   cs_i = inst[i].cs (0 means 1).
 * Corner entries (j + d >= n for lower bands) are never read; outputs write 0
 * there.  Every band operand of one call uses the same per-instance offset
 * `band`, row stride `ld` and column stride `cs`; the caller sizes each
 * instance's region for the tallest operand of the call (e.g. lo+up+1 rows
 * for products).
 *
 * Right-hand sides are n x k column blocks: element (j, r) of instance i at
 *     pool[inst[i].rhs + r * inst[i].ldr + j * cs_i].
 *
 * Two arrangements of a batch in a pool have fast paths:
 *  - rows (cs = 1): each row of B' (and each RHS column) is contiguous.  The
 *    sweeps stage every instance's rows through shared memory lane by lane.
 *    Offsets band, rhs and strides ld, ldr that are multiples of 16 bytes
 *    keep the staged kernels; other values run the direct kernels.
 *  - panels (cs = 32): instances come in groups.  A group is a run of at
 *    most 32 consecutive descriptors whose offsets step by one -- the p-th
 *    descriptor of the run ("lane" p) has band = band_g + p and
 *    rhs = rhs_g + p -- and which share l, ld and ldr; ld and ldr are
 *    multiples of 32, (l+1) ld and k ldr below 2^31 elements, and band_g,
 *    rhs_g multiples of 16 bytes.  A descriptor
 *    that does not continue the previous run starts a new group.  Row d,
 *    column j of the 32 lanes are then 32 adjacent elements, so one warp
 *    moves whole 128-byte (FP32) lines: this is the layout that reaches HBM
 *    bandwidth.  The kernels read all 32 lanes of a group row even where a
 *    lane is absent or shorter, so each group's pool region must span
 *    (rows) x ld elements from band_g (k x ldr from rhs_g).  Descriptors
 *    should be ordered so that a group's orders n are close (e.g. sorted)
 *    and groups are full; a group advances at the pace of its longest
 *    member.
 * Any other column stride is accepted and runs the direct kernels.
 *
 * Symmetric matrices (Q, S = band(Q^{-1})) are stored by their lower band;
 * their gradients (Qbar, Sbar) are gradients with respect to these STORED
 * entries, so an off-diagonal stored entry carries the derivative of both
 * (i, j) and (j, i).
 *
 * ---------------------------------------------------------------------------
 * Conventions.
 *  - Memory: the caller owns every device buffer.  The library never
 *    allocates device memory and never synchronises the stream; each call
 *    only enqueues kernels (and small memsets) on `stream`.
 *  - Pointers: `inst` passed to bnd_plan_create is HOST memory; every data
 *    pointer passed to an operator (pools, workspace, logdet, info) is DEVICE
 *    memory.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *  - Inputs are never written.  Outputs must not alias inputs unless stated.
 *  - Errors: host-side validation failures return BND_EINVAL / BND_EALIGN
 *    before anything is enqueued; a failed launch returns BND_ECUDA.
 *    Numerical failure of the Cholesky (a pivot that is not > 0) is reported
 *    per instance in `info` (LAPACK pbtrf style), never by the return code.
 *  - dtype: BND_F32 or BND_F64 for all floating-point pools of a plan; the
 *    log-determinant is always returned in double precision.
 *  - Thread safety: a plan may be used from one stream at a time (it owns the
 *    workspace bound to it); distinct plans are independent.
 */
#ifndef BANDED_H
#define BANDED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BND_OK = 0,
    BND_EINVAL = 1,      /* invalid argument (sizes, strides, mode, unbound plan) */
    BND_ENOTSPD = 2,     /* reserved: a host-visible summary of info != 0 */
    BND_ECUDA = 3,       /* a CUDA launch or memset failed */
    BND_ETIMEOUT = 4,    /* reserved: a bounded device wait gave up */
    BND_EALIGN = 5       /* a pointer or stride violates the stated alignment */
} bnd_status;

typedef enum { BND_F32 = 0, BND_F64 = 1 } bnd_dtype;

/* One instance of a batch (host array given to bnd_plan_create). */
typedef struct {
    int64_t n;      /* order of the matrix, n >= 1 */
    int64_t band;   /* element offset of B'[0][0] in every band pool of a call */
    int64_t ld;     /* row stride of B' in elements, ld >= n * cs */
    int64_t rhs;    /* element offset of the first RHS column in every RHS pool */
    int64_t ldr;    /* stride between RHS columns in elements, ldr >= n * cs (ignored if k = 0) */
    int32_t l;      /* lower bandwidth, 0 <= l <= 1024 */
    int32_t cs;     /* column stride in elements of the band and the RHS block
                       (0 or 1: contiguous rows; 32: panel lanes, see Storage) */
} bnd_inst;

/* Scheduling knobs (all optional; zero fields take the library defaults). */
typedef struct {
    int64_t seg_len;     /* rows per chain segment; long instances are split into segments
                            run in parallel (0 = default: 2048 for rows, 384 for panels;
                            bandwidths above 8: about 152 segments over the plan's wide
                            instances, each at least one warm-up long; < 0 = never split) */
    int32_t warmup;      /* warm-up rows of a speculative segment start (0 = default:
                            16 l + 32 rows in FP32, 48 l + 64 in FP64; bandwidths above 8:
                            8 l + 32 and 16 l + 64) */
    int32_t blocks_per_sm; /* persistent-grid occupancy (0 = default) */
    int32_t flags;       /* bit 0: never use the shared-memory staged kernels;
                            bit 1: segment length seg_len * warmup / 128 (the same share of
                            warm-up rows for every bandwidth);
                            bit 2: no staged reruns (mismatching segments are only rerun
                            serially by the verify pass) */
    int32_t warm_per_l;  /* > 0: warm-up rows = warm_per_l * l + warm_base for bandwidth l
                            (overrides the defaults; `warmup` > 0 overrides both) */
    int32_t warm_base;
} bnd_tuning;

typedef struct bnd_plan bnd_plan;

/* ---------------------------------------------------------------------------
 * Plans.  A plan fixes the batch (instances, dtype, number of right-hand
 * sides k) and precomputes the schedule on the host: every instance is cut
 * into row segments ("chains") that run as independent lanes of the GPU;
 * chains of equal bandwidth are grouped 32 to a warp; warp tasks are ordered
 * longest first for the persistent kernels.  Segments of one instance start
 * from a speculative warm-up and are checked against their neighbour
 * afterwards; a mismatch reruns that segment from its exact start state.  For
 * bandwidths up to 8 the check is bit for bit, so results do not depend on the
 * segmentation.  Above 8 (one thread block per segment) a start passes when
 * its state agrees with the exact one within 2^-16 (FP32) / 2^-44 (FP64) of
 * the largest entry of each part of the state (band window; each RHS row):
 * there a converged cold start stays about one ulp from the exact state
 * instead of meeting it, so results agree with an unsplit run to rounding
 * noise (deterministically for a given plan).
 *
 * bnd_plan_create copies `inst` (HOST) and returns BND_EINVAL on a bad
 * descriptor (n < 1, l < 0 or > 1024, cs < 0, ld < n cs, ldr < n cs when
 * k > 0, k < 0 or k > 64, count < 0).  A batch whose column strides are not
 * all 1 is planned as panels when every descriptor has cs = 32 and ld, ldr
 * multiples of 32 (groups as in Storage), else as a general strided batch
 * (direct kernels).  bnd_plan_workspace_bytes gives the device workspace the
 * plan needs; bnd_plan_bind uploads the plan's tables into that caller-owned
 * workspace on `stream` and returns once the copies are complete (it
 * synchronises `stream`; it is a set-up call, not an operator); `ws` must be
 * 256-byte aligned and stay allocated while the plan is used.  The workspace
 * holds the schedule tables, per-segment state snapshots and scratch pools
 * shaped like the band and RHS pools of the plan.  bnd_plan_destroy frees
 * host memory only.
 * ------------------------------------------------------------------------- */
bnd_status bnd_plan_create(bnd_plan **plan, bnd_dtype dtype, int32_t count, const bnd_inst *inst,
                           int32_t k, const bnd_tuning *tuning);
size_t bnd_plan_workspace_bytes(const bnd_plan *plan);
bnd_status bnd_plan_bind(bnd_plan *plan, void *ws, size_t ws_bytes, void *stream);
void bnd_plan_destroy(bnd_plan *plan);
/* Number of chains (lanes of work) and warp tasks of the plan (for reporting). */
int64_t bnd_plan_chains(const bnd_plan *plan);
int64_t bnd_plan_tasks(const bnd_plan *plan);
/* Arrangement the plan recognised: 0 = rows (cs = 1), 1 = panels (cs = 32
 * groups), 2 = general strides; -1 for a NULL plan. */
int32_t bnd_plan_layout(const bnd_plan *plan);
/* Number of segments rerun by the verify pass of the last launch of the given
 * sweep kind (0 = Cholesky forward sweep, 1 = subset-inverse sweep,
 * 2 = subset-inverse adjoint sweep, 3 = Cholesky adjoint sweep, 4 = forward
 * solve sweep, 5 = backward solve sweep).  kind = 6 returns instead the number
 * of bounded device waits (on the shared-memory barriers of the bulk tile
 * copies, a build option) that gave up since the plan was bound: it must be 0;
 * any other value means the results of the plan's calls are invalid.  Copies
 * the counter into the HOST int64 *out and synchronises `stream`. */
bnd_status bnd_plan_fixups(const bnd_plan *plan, int32_t kind, int64_t *out, void *stream);

/* ---------------------------------------------------------------------------
 * C: banded Cholesky, Alg. 1 (App. B) and Sec. 4.1.  Q (lower band, SPD) ->
 * L with L L^T = Q, lower bandwidth l.  logdet[i] = log det Q_i =
 * 2 sum_j log L_jj in double precision (nullable).  info[i] = 0 on success,
 * else r+1 where r is the first row whose pivot is not > 0; rows >= r of L
 * are then unspecified (NaN in practice).  info is required.
 * ------------------------------------------------------------------------- */
bnd_status banded_cholesky(const bnd_plan *plan, const void *Q, void *L, double *logdet,
                           int32_t *info, void *stream);

/* Cbar: reverse mode of C, Alg. 2 (App. B).  L, Lbar -> Qbar, the gradient
 * with respect to the lower stored entries of Q.  ldbar (DEVICE, one double
 * per instance, nullable) is the cotangent of logdet; it adds 2 ldbar / L_jj
 * to the diagonal of Lbar before the sweep (d log det Q / d L_jj = 2 / L_jj).
 * accumulate = 1 adds into Qbar instead of overwriting it. */
bnd_status banded_cholesky_vjp(const bnd_plan *plan, const void *L, const void *Lbar, const double *ldbar,
                               void *Qbar, int32_t accumulate, void *stream);

/* S: triangular solve with the plan's k right-hand sides, Sec. 4.1.
 * mode 0: X = L^{-1} B;  mode 1: X = L^{-T} B;  mode 2: X = (L L^T)^{-1} B.
 * X must not alias B. */
bnd_status banded_solve(const bnd_plan *plan, const void *L, const void *B, void *X, int32_t mode,
                        void *stream);

/* Sbar: reverse mode of S, Table 1 ("solve matrix-vector").  Given the forward
 * output X and its cotangent Xbar:
 *   mode 0 (X = L^{-1} B):  Bbar = L^{-T} Xbar,  Lbar -= band_l(Bbar X^T)
 *   mode 1 (X = L^{-T} B):  Bbar = L^{-1} Xbar,  Lbar -= band_l(X Bbar^T)
 *   mode 2 (X = Q^{-1} B):  the composition of the two with Y = L^T X.
 * Bbar is written (nullable); Lbar is overwritten, or added to when
 * accumulate = 1 (nullable). */
bnd_status banded_solve_vjp(const bnd_plan *plan, const void *L, const void *X, const void *Xbar,
                            int32_t mode, void *Bbar, void *Lbar, int32_t accumulate, void *stream);

/* I: subset inverse, Alg. 3 (App. B) and Sec. 4.1 (Takahashi).  L -> S, the
 * lower band of (L L^T)^{-1}. */
bnd_status banded_subset_inverse(const bnd_plan *plan, const void *L, void *S, void *stream);

/* Ibar: reverse mode of I, Alg. 4 (App. B).  L, S, Sbar -> Lbar, the gradient
 * with respect to the stored entries of L; Sbar is the gradient with respect
 * to the stored (lower) entries of S.  accumulate = 1 adds into Lbar. */
bnd_status banded_subset_inverse_vjp(const bnd_plan *plan, const void *L, const void *S,
                                     const void *Sbar, void *Lbar, int32_t accumulate, void *stream);

/* ---------------------------------------------------------------------------
 * Fused step of the precision-parameterised Gaussian models (Sec. 3): one
 * forward sweep pair and one backward sweep pair over every instance.
 *   forward : L = C(Q), logdet = log det Q, X = Q^{-1} B, S = I(L)
 *   backward: given Xbar, Sbar (stored entries) and ldbar (DEVICE, one double
 *             per instance, nullable = 0), the gradients Qbar (stored entries
 *             of Q) and Bbar (nullable) of
 *             <Xbar, X> + <Sbar, S> + sum_i ldbar_i * logdet_i,
 *             composed per Table 1, Alg. 2 and Alg. 4.
 * Needs a plan with 1 <= k <= 4, or 1 <= k <= 16 when every instance has
 * l = 0 or l > 8 (the wide-band kernels take the column count at run time);
 * BND_EINVAL otherwise.  Plans with more columns use the separate operators.  The forward writes L, X, S (and keeps L^{-1} B in the
 * workspace); the backward reads L, X, S.
 * ------------------------------------------------------------------------- */
bnd_status banded_gmm_forward(const bnd_plan *plan, const void *Q, const void *B, void *L, void *X,
                              void *S, double *logdet, int32_t *info, void *stream);
bnd_status banded_gmm_backward(const bnd_plan *plan, const void *L, const void *X, const void *S,
                               const void *Xbar, const void *Sbar, const double *ldbar, void *Qbar,
                               void *Bbar, void *stream);

/* ---------------------------------------------------------------------------
 * P and O: products (Sec. 4.1).  These take the same plan (for n, offsets and
 * strides); operand shapes are per call.
 *
 * banded_product: C = op(A) op(B) projected onto C's band (clo, cup), with
 *   op(X) = X or X^T (transX = 0 / 1).  A has bandwidths (alo, aup), B has
 *   (blo, bup).  C must not alias A or B.
 * banded_outer:   C = band_{clo,cup}(M V^T) = band(sum_r m_r v_r^T) over the
 *   plan's k right-hand-side columns of M and V.
 * banded_matvec:  P = op(A) V for the plan's k columns.
 * accumulate = 1 adds into the output.
 * ------------------------------------------------------------------------- */
bnd_status banded_product(const bnd_plan *plan, const void *A, int32_t alo, int32_t aup,
                          int32_t transA, const void *B, int32_t blo, int32_t bup, int32_t transB,
                          void *C, int32_t clo, int32_t cup, int32_t accumulate, void *stream);
bnd_status banded_outer(const bnd_plan *plan, const void *M, const void *V, void *C, int32_t clo,
                        int32_t cup, int32_t accumulate, void *stream);
bnd_status banded_matvec(const bnd_plan *plan, const void *A, int32_t alo, int32_t aup,
                         int32_t transA, const void *V, void *P, int32_t accumulate, void *stream);

/* Pbar: Table 1 ("product matrix-matrix"), band-projected (Sec. 4.2):
 *   Abar = band_A(Cbar op(B)^T)  (or its transpose when transA),
 *   Bbar = band_B(op(A)^T Cbar)  (or its transpose when transB).
 * Either output may be NULL.  accumulate = 1 adds into the outputs. */
bnd_status banded_product_vjp(const bnd_plan *plan, const void *A, int32_t alo, int32_t aup,
                              int32_t transA, const void *B, int32_t blo, int32_t bup,
                              int32_t transB, const void *Cbar, int32_t clo, int32_t cup,
                              void *Abar, void *Bbar, int32_t accumulate, void *stream);

/* ---------------------------------------------------------------------------
 * S with a banded right-hand side, Alg. 5 (App. B): O = band_{olo,oup}(L^{-1} R)
 * (trans = 0) or band_{olo,oup}(L^{-T} R) (trans = 1), for a general band R
 * with bandwidths (rlo, rup); L is lower band l (the plan's per-instance l).
 * Every band is exact: trans = 0 needs oup >= rup (L^{-1} R has no entries
 * above that), trans = 1 needs olo >= rlo; BND_EINVAL otherwise.  Each
 * column of O is an independent triangular solve restricted to the band (the
 * dependency Alg. 5 walks diagonal by diagonal).  O must not alias L or R.
 *
 * Reverse mode, Table 1 ("solve matrix-matrix"): given the forward output O
 * and its cotangent Obar (on O's band),
 *   G    = band_{olo,oup}(L^{-T} Obar)   (trans = 0; L^{-1} Obar for trans = 1)
 *   Rbar = band_{rlo,rup}(G)             (nullable)
 *   Lbar -= band_l(G O^T)  (trans = 0)   or  band_l(O G^T)  (trans = 1)   (nullable)
 * G is a caller band pool shaped like O (written; it is also the unprojected
 * R-bar).  accumulate = 1 adds into Rbar and Lbar.
 * ------------------------------------------------------------------------- */
bnd_status banded_solve_band(const bnd_plan *plan, const void *L, const void *R, int32_t rlo, int32_t rup, void *O,
                             int32_t olo, int32_t oup, int32_t trans, void *stream);
bnd_status banded_solve_band_vjp(const bnd_plan *plan, const void *L, const void *O, int32_t olo, int32_t oup,
                                 const void *Obar, int32_t trans, int32_t rlo, int32_t rup, void *G, void *Rbar,
                                 void *Lbar, int32_t accumulate, void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free precision solve (the paper has no counterpart; it exists for
 * callers that cannot allocate device memory at all, not even a workspace to
 * hand over -- e.g. code inside a framework hook that forbids allocation, or a
 * process whose device memory is reserved up front by another component).
 *
 *   x = (L L^T)^{-1} b   for ONE instance (order n, lower bandwidth l) and one
 *   right-hand side; L (lower band, row stride ld >= n), b and x are DEVICE
 *   pointers, b and x hold n elements.  x may share no byte with b or with
 *   L's (l ld + n)-element region (BND_EINVAL otherwise).
 *
 * No plan and no workspace: the intermediate y = L^{-1} b lives in a fixed
 * 16 MiB device array inside the library (n <= 4,194,304 in FP32,
 * n <= 2,097,152 in FP64; larger n returns BND_EINVAL).  Every GPU that loads
 * the library keeps that array until the process exits.  The call allocates
 * nothing (no cudaMalloc / cudaFree, no allocating library routine).
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.  The address is kept for the life of the process: after
 *    cudaDeviceReset the library has to be reloaded before this call is used
 *    again.
 *  - All calls on a device share that device's array, which keeps the last
 *    call's contents (nothing in it needs to start at zero).  Calls that
 *    overlap on the same GPU (e.g. issued on two streams) race on it: order
 *    them on one stream.
 *  - It runs one thread per sweep: meant for availability, not throughput.
 * ------------------------------------------------------------------------- */
bnd_status banded_solve_precision_noalloc(bnd_dtype dtype, int64_t n, int32_t l, const void *L, int64_t ld,
                                          const void *b, void *x, void *stream);

/* Library version string (static storage). */
const char *bnd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BANDED_H */
