/*
 * scqr3.h -- C ABI of the GB300 (sm_103a) shifted CholeskyQR3 library.
 *
 * Computes the QR factorization X = QR of a tall-skinny m x n matrix
 * (m >= n), with Q^T Q = I (or Q^T B Q = I for an oblique inner product) and
 * R upper triangular with positive diagonal, by shifted CholeskyQR3
 * (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa: Sec. 2 Alg. 1,
 * Sec. 4 Alg. 3, Sec. 5 Alg. 4 and Alg. 5), with the breakdown rule of Alg. 2.
 *
 * Conventions shared by every entry point
 *  - Matrices are row-major FP64: element (i, j) of X is X[i*ldx + j].
 *    Row-major keeps each row x_i^T contiguous, which is what the row-wise
 *    substitution Q = X R^{-1} (Eq. backward2) works on.
 *  - Every pointer argument is DEVICE memory owned by the caller, except
 *    the scqr3_B / scqr3_opts descriptors themselves, which are host structs
 *    (their `blocks` pointer is device memory).
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream). No call synchronizes the host on the
 *    compute path. The return value reports only errors detectable on the
 *    host before any work is queued; everything found while computing is
 *    written to the device-side scqr3_info and is valid once the stream has
 *    been synchronized.
 *  - No entry point allocates device memory: scratch comes from the
 *    caller's `workspace` of at least scqr3_workspace_bytes() bytes,
 *    256-byte aligned, not shared with a concurrent call.
 */
#ifndef SCQR3_H
#define SCQR3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCQR3_MAX_PASSES 8   /* upper limit of opts.max_passes            */
#define SCQR3_MAX_N 256      /* largest n (FP64 and SCQR3_PREC_TC, B = I);
                                the oblique, mixed, batched and adjoint
                                forms take n <= 128                        */

/* Status codes (return values and scqr3_info.status).
 *   > 0  : the SHIFTED Cholesky broke down at this 1-based column, i.e.
 *          chol(A + sI) of Alg. 1 failed (X numerically rank
 *          deficient beyond what the shift of Eq. (finds2) covers).
 *   -1..-20 : argument k (1-based, in the order of the prototype) invalid. */
#define SCQR3_OK 0
#define SCQR3_E_NONFINITE (-100)  /* the Gram matrix has a NaN/Inf entry   */
#define SCQR3_E_MAXPASS (-101)    /* max_passes reached before two plain
                                     CholeskyQR passes followed the last
                                     shifted one; Q, R are still X = QR   */
#define SCQR3_E_CUDA (-103)       /* a CUDA launch failed                  */
#define SCQR3_E_TIMEOUT (-102) /* a wait inside a tensor-core kernel ran out
                                     of time (see scqr3_debug_set)         */
#define SCQR3_E_WORKSPACE (-104)  /* workspace too small or misaligned     */
#define SCQR3_E_B_NOT_SPD (-105)  /* a diagonal block of B is not SPD      */
#define SCQR3_E_UNSUPPORTED (-106)/* size not supported by this build      */
#define SCQR3_E_B_INVALID (-108)  /* CSR form of B malformed: row_ptr not
                                     non-decreasing within [0, nnz], a column
                                     index outside [0, m), or a row without a
                                     positive diagonal entry                */
#define SCQR3_E_SCRATCH_LIMIT (-107) /* scqr3_factor_noalloc: the problem needs
                                        more scratch than its fixed array   */

#define SCQR3_PREC_FP64 0
/* Mixed form (B = I only): the bulk Gram and substitution of every pass run
 * on the FP32 pipe in pairs of floats (h, l), x ~ h + l, with error-free
 * products and TwoSum accumulation (about 48 significant bits); the Gram
 * partial sums are accumulated in FP64, and the shift of Eq. (finds2), the
 * Cholesky factorizations and R = R_k ... R_1 are FP64. Intermediate
 * iterates are held in Q as float pairs; Q and R are returned in FP64.
 * Inputs must lie within the float exponent range. Not in the paper (which
 * uses FP64 throughout, Sec. 6); expected orthogonality ~1e-14. */
#define SCQR3_PREC_MIXED 1
/* FP64-accurate form with the bulk of the arithmetic on the BF16 tensor cores
 * (tcgen05). Not in the paper. Every value a tensor core multiplies is
 * rounded to 2^-56 of a power-of-two scale (per Gram column; per row of Y and
 * per column of R_JK in the substitution) and cut into eight signed digits in
 * [-64, 64]: each digit is exactly a BF16 number, every digit product and
 * every tensor-core sum (at most 2^24 in magnitude) is exact in FP32, and the
 * digit-pair sums are combined in int64; the error is zero-mean.
 *  - Gram matrices: below about 8.5 m u ||q_j|| ||q_k|| per entry, within the
 *    norm-wise bound that the shift of Eq. (finds2) covers; the diagonal adds
 *    the digit squares the tiles leave out, so it is not biased low.
 *  - Substitution Q := X R^{-1}: the triangular diagonal blocks of R (16
 *    columns for n <= 64, 32 above) in FP64, the products with the
 *    off-diagonal blocks on the tensor cores, a perturbation of R of norm
 *    O(u ||R||) per row (the form of the row-wise backward error, Eq.
 *    backward2). For 16 < n <= 64 a pass reads each row once and writes it
 *    once (one sweep, see scqr3_debug_set).
 * Results match the FP64 form to rounding. m <= 2^31; n <= 256 with
 * B = NULL (for 128 < n <= 256 the Gram matrix is ten 64-column block pairs),
 * or n <= 128 with B block-diagonal with blocks of 1, 2, 4 or 8 rows (the
 * Gram matrix of Z = L^T Q, L_j^T applied to each 8-row unit before the
 * split); other shapes return SCQR3_E_UNSUPPORTED. */
#define SCQR3_PREC_TC 2
/* The mixed form's substitution (FP32 pairs) with the Gram matrices of
 * SCQR3_PREC_TC, read directly from the float-pair iterates. n <= 128,
 * m <= 2^31 and B = NULL. Not in the paper. */
#define SCQR3_PREC_MIXED_TC 3

/* Oblique inner product (x, y)_B = x^T B y of Sec. 5, for SPD B given
 * either block-diagonal, B = blockdiag(B_1, ..., B_{m/bs}) (bs > 0), or as a
 * general sparse matrix in CSR form (bs = 0; Sec. 7.2 uses sparse B and
 * forms B Q by a sparse product). The CSR form must be symmetric (the
 * library uses its rows as given and does not check symmetry), with int64
 * row offsets and int32 column indices, m < 2^31; n <= 128, FP64 only. */
typedef struct {
  int bs;               /* block size, m % bs == 0: 1, 2, 4, 8 or 16 (FP64;
                           the tensor-core form takes 1, 2, 4 or 8); 0 selects
                           the CSR fields below (FP64 only)                 */
  const double *blocks; /* device: (m/bs) blocks of bs*bs row-major FP64    */
  double norm2;         /* ||B||_2 if > 0; otherwise an upper bound is
                           computed on the device: max_j ||B_j||_F (blocks),
                           the largest absolute row sum (CSR)               */
  const int64_t *row_ptr; /* CSR: device, m + 1 offsets, row_ptr[0] = 0     */
  const int32_t *col_idx; /* CSR: device, nnz column indices                */
  const double *vals;     /* CSR: device, nnz values                        */
  int64_t nnz;            /* CSR: entries in col_idx / vals                 */
} scqr3_B;

typedef struct {
  int max_passes;  /* total CholeskyQR passes allowed, 3..SCQR3_MAX_PASSES;
                      0 selects 6                                          */
  int precision;   /* SCQR3_PREC_FP64 (0), SCQR3_PREC_MIXED,
                      SCQR3_PREC_TC or SCQR3_PREC_MIXED_TC (see above)    */
  double norm_x2;  /* > 0: value of ||X||_2^2 used in the pass-1 shift of
                      Eq. (finds2)/(finds2B); 0: ||Q||_F^2 of each shifted
                      pass's iterate (Sec. 4.1 allows this more conservative
                      substitute); SCQR3_NORM_X2_TWO_EST (B = NULL only):
                      ||Q||_2^2 of each shifted pass's iterate estimated as
                      lambda_max of its Gram matrix by the power method (the
                      normest of Sec. 4.1; iterated until the estimate changes
                      by at most 1e-12 of itself, at most 200 steps)         */
  double shift_scale; /* > 0: a shifted pass first tries the smaller shift
                      s = shift_scale * u * ||Q||^2 (times ||B|| for oblique
                      B) that the remark of Sec. 6.1 and Sec. 8 suggest
                      (shift_scale = 1 is the remark's u ||X||^2), and uses
                      Eq. (finds2)/(finds2B) only if that Cholesky breaks
                      down; <= 0: Eq. (finds2)/(finds2B) only. A smaller
                      shift leaves kappa(Q_1) smaller and can save a pass
                      for kappa(X) near 1/u, with no guarantee (Sec. 6.1)    */
  int algorithm;   /* SCQR3_ALG_SCQR3 (or 0): Alg. 3; SCQR3_ALG_ADAPTIVE:
                      Alg. 2                                               */
  double tol;      /* Alg. 2 only: stop once ||Q^T Q - I||_F <= tol
                      (||Q^T B Q - I||_F for oblique B), tested on the Gram
                      matrix of the current iterate; <= 0 selects
                      6 {mn + n(n+1)} u, the orthogonality bound of
                      Thm. (maincholqr3) (the printed sqrt(n) u is below the
                      rounding error of a computed Gram matrix)             */
} scqr3_opts;

#define SCQR3_NORM_X2_TWO_EST (-1.0)

/* scqr3_opts.algorithm. Alg. 3 shifts pass 1 unconditionally and ends after
 * two consecutive unshifted passes. Alg. 2 tries the plain Cholesky in every
 * pass (shifting only on breakdown) and ends on its orthogonality test, so a
 * well-conditioned X takes one or two passes; its test needs the Gram matrix
 * of every iterate, including the last. Both end with SCQR3_E_MAXPASS when
 * max_passes passes did not finish. */
#define SCQR3_ALG_ADAPTIVE 2
#define SCQR3_ALG_SCQR3 3

/* Per-call record, written on the device. */
typedef struct {
  int status;                            /* SCQR3_OK or a code above       */
  int passes;                            /* CholeskyQR passes executed     */
  int shifted[SCQR3_MAX_PASSES];         /* pass k used chol(A + sI)       */
  int unshifted_fail[SCQR3_MAX_PASSES];  /* column where the plain chol(A)
                                            of pass k broke down, else 0   */
  double s[SCQR3_MAX_PASSES];            /* shift of pass k, 0 if none     */
  double norm2[SCQR3_MAX_PASSES];        /* ||Q_{k-1}||^2 estimate used    */
  int more;                              /* 1: the device planned another
                                            pass after pass `passes` (its
                                            Gram matrix follows the last
                                            solve); 0 once the call is done */
} scqr3_info;

/* Bytes of device workspace that scqr3_factor needs for (m, n, B, opts).
 * Writes *bytes; returns SCQR3_OK or a negative argument code. */
int scqr3_workspace_bytes(int64_t m, int n, const scqr3_B *B,
                          const scqr3_opts *opts, size_t *bytes);

/* Shifted CholeskyQR3: X = QR (Alg. 3), or X = QR with Q^T B Q = I (Alg. 5).
 *
 *  X      m x n input, leading dimension ldx >= n. Read only.
 *  B      NULL for B = I, else the block-diagonal SPD descriptor above.
 *  Q      m x n output, ldq >= n. May alias X exactly (X == Q, ldx == ldq)
 *         for an in-place factorization; any other overlap is an error.
 *  R      n x n output, leading dimension n, upper triangular, positive
 *         diagonal, strictly lower part set to zero: R = R_k ... R_2 R_1.
 *  Rpass  NULL, or SCQR3_MAX_PASSES * n * n doubles receiving the per-pass
 *         factors R_k (pass k at Rpass + k*n*n, row-major, lower part zero),
 *         as the adjoint scqr3_backward needs them.
 *  info   device scqr3_info filled by the call (required).
 *
 * By default (opts->algorithm = SCQR3_ALG_SCQR3) pass 1 always adds the
 * shift s of Eq. (finds2) (Eq. finds2B if B != NULL) before its Cholesky
 * factorization (Alg. 3). A later pass whose plain Cholesky breaks down is
 * redone with the shift recomputed from that pass's ||Q||^2 (the breakdown
 * rule of Alg. 2). The call ends after two consecutive plain passes
 * (CholeskyQR2, the last two steps of Alg. 3) or at max_passes
 * (SCQR3_E_MAXPASS). SCQR3_ALG_ADAPTIVE runs Alg. 2 instead (see
 * scqr3_opts). Each pass's solve Q := Q R_k^{-1} is done row by row by
 * substitution, as the row-wise analysis (Eq. backward2) assumes. When a
 * pass fails (status > 0 or a negative code found on the device), Q holds
 * the last completed iterate in FP64, or is untouched if pass 1 failed. */
int scqr3_factor(const double *X, int64_t m, int n, int64_t ldx,
                 const scqr3_B *B, double *Q, int64_t ldq, double *R,
                 double *Rpass, void *workspace, size_t workspace_bytes,
                 const scqr3_opts *opts, scqr3_info *info, void *stream);

/* ---------------------------------------------------------------------------
 * Host-buffer form: the same factorization with X, Q, R and info in host
 * memory. Not in the paper; it exists so that a caller whose data lives on
 * the host pays for the transfers only once, overlapped with the work:
 *  - X goes to the device in row chunks on a second stream. With B = NULL,
 *    each chunk's share of the first Gram matrix X^T X starts as soon as the
 *    chunk has arrived; each chunk writes its own partial sums, so the
 *    first Gram matrix is summed in a different order than by scqr3_factor
 *    when m > 262,144 (same result up to rounding; bit for bit below that).
 *  - After each Cholesky the host reads the device's pass flags (about
 *    100 bytes), so it knows which solve is the last one. That solve runs in
 *    row chunks, and each chunk of Q is copied back while the next is solved.
 *
 *  X, Q   host, m x n row-major, leading dimensions ldx, ldq >= n. Q may be
 *         X (ldq == ldx). Pinned memory (cudaHostAlloc, cudaHostRegister)
 *         lets the copies overlap the work; pageable memory also works.
 *  R      host, n x n, as for scqr3_factor.
 *  Qdev   device scratch of m x n doubles (leading dimension n) holding the
 *         iterates; it is the caller's, like the workspace.
 *  workspace  device, scqr3_host_workspace_bytes() bytes, 256-byte aligned.
 *  info   host scqr3_info, filled before the call returns.
 *
 * The call is synchronous: it returns when Q, R and info are written (or
 * with a negative code before any work was queued, or SCQR3_E_CUDA). It
 * uses one internal copy stream per device, created by the first call, and
 * calls on the same device run one at a time. Failure: Q receives the last
 * completed iterate (X itself if pass 1 failed). Neither the batched form
 * nor Rpass is offered here. */
int scqr3_host_workspace_bytes(int64_t m, int n, const scqr3_B *B,
                               const scqr3_opts *opts, size_t *bytes);
int scqr3_factor_host(const double *X, int64_t m, int n, int64_t ldx,
                      const scqr3_B *B, double *Q, int64_t ldq, double *R,
                      double *Qdev, void *workspace, size_t workspace_bytes,
                      const scqr3_opts *opts, scqr3_info *info, void *stream);

/* ---------------------------------------------------------------------------
 * Row-partitioned form: the data-parallel structure of the method, for a
 * caller that holds X in row blocks X_r on several devices or processes. The
 * Gram matrix of X is the sum of its blocks' Gram matrices (Sec. 1: the
 * Gram matrix is formed "by addition", one reduction of n(n+1)/2 values per
 * pass; Sec. 7.1, Table 8); the shift, the Cholesky factorization and R are
 * then the same on every block's holder, and each solves its own rows. Per
 * rank, with G and G' device vectors of `gram_words` doubles:
 *
 *   scqr3_gram_partial(X_r, ..., G)          G = X_r's share of X^T X
 *   [caller: G := sum of G over the ranks, e.g. an allreduce]
 *   for pass = 0, 1, ..., max_passes - 1:
 *     scqr3_apply_pass(pass, G, m, X_r, ..., Q_r, R, G')
 *         the shift / Cholesky of this pass on G (shift from the global m),
 *         Q_r := (pass 0: X_r; later: Q_r) R_pass^{-1}, and, if the device
 *         planned another pass (info->more), G' = Q_r's share of Q^T Q
 *     [caller: G := sum of G' over the ranks]
 *
 * The pass decisions of Alg. 3 / Alg. 2 are taken on the device from G, so
 * every rank takes the same ones; once a factorization is done the remaining
 * calls return at once (a fixed sequence is correct; a caller may also stop
 * after the first call whose info->more is 0). G's entries are partial sums
 * in an internal packed order: the caller only adds them elementwise. The
 * workspace carries the state from call to call: one per rank, not shared.
 * Forms: SCQR3_PREC_FP64 or SCQR3_PREC_TC; B NULL or block-diagonal with
 * the caller's ||B||_2 in B->norm2 (> 0, the same on every rank) and each
 * rank's rows whole blocks (m_r % bs == 0); the mixed forms and a CSR B
 * (whose rows reach across the blocks) are SCQR3_E_UNSUPPORTED. Argument codes
 * -k name argument k of the function called. */
int scqr3_shard_sizes(int64_t m_local, int n, const scqr3_B *B,
                      const scqr3_opts *opts, size_t *workspace_bytes,
                      size_t *gram_words);
int scqr3_gram_partial(const double *X, int64_t m_local, int n, int64_t ldx,
                       const scqr3_B *B, double *G, void *workspace,
                       size_t workspace_bytes, const scqr3_opts *opts,
                       scqr3_info *info, void *stream);
int scqr3_apply_pass(int pass, const double *G, int64_t m_global,
                     const double *X, int64_t m_local, int n, int64_t ldx,
                     const scqr3_B *B, double *Q, int64_t ldq, double *R,
                     double *G_next, void *workspace, size_t workspace_bytes,
                     const scqr3_opts *opts, scqr3_info *info, void *stream);

/* ---------------------------------------------------------------------------
 * Batched form (FP64, B = I): many independent, uneven factorizations, each
 * exactly as scqr3_factor would compute it (Alg. 3 with the breakdown rule
 * of Alg. 2), in one fixed launch sequence. Not in the paper, whose
 * experiments factor one matrix at a time.
 *
 * Each phase is one persistent launch: every CTA takes tiles (a run of row
 * panels of one matrix) from an atomic queue, largest n first; each tile
 * writes its own partial Gram matrix, and each matrix's tiles are summed in
 * tile order, so results do not depend on scheduling. Shift, Cholesky and
 * pass bookkeeping run with one CTA per matrix.
 *
 * Use: scqr3_batch_plan_create (host only: validates the items, builds the
 * tile list, returns the workspace size); scqr3_batch_plan_upload (copies the
 * tables into the workspace and synchronizes `stream`; call before any
 * capture); then scqr3_factor_batched any number of times -- it only queues
 * memsets and kernels on `stream`, so it can be captured in a CUDA graph and
 * replayed; finally scqr3_batch_plan_destroy. The workspace and all item
 * buffers must stay valid and unmoved while the plan is used. opts: FP64
 * precision only; max_passes, shift_scale, algorithm and tol apply to every
 * matrix as in scqr3_factor (Alg. 2's default tol from each matrix's m, n). */
typedef struct {
  const double *X;    /* device, m x n row-major, ldx >= n                  */
  double *Q;          /* device, m x n, ldq >= n (may equal X, ldq == ldx)   */
  double *R;          /* device, n x n                                       */
  double *Rpass;      /* device, SCQR3_MAX_PASSES * n * n, or NULL           */
  scqr3_info *info;   /* device record of this matrix's call                 */
  int64_t m;
  int n;              /* 1 .. 128 (else SCQR3_E_UNSUPPORTED)                  */
  int64_t ldx, ldq;
} scqr3_batch_item;

typedef struct {
  int ctas_per_sm;     /* persistent CTAs per SM (0: 1)                      */
  int tile_panels[4];  /* row panels per tile for n padded to 16, 32, 64, 128
                          (0: 8); panels are 256 rows (128 for n > 64)      */
} scqr3_batch_tuning;

typedef struct scqr3_batch_plan scqr3_batch_plan;

int scqr3_batch_plan_create(const scqr3_batch_item *items, int count,
                            const scqr3_opts *opts,
                            const scqr3_batch_tuning *tuning,
                            scqr3_batch_plan **plan, size_t *workspace_bytes);
int scqr3_batch_plan_upload(scqr3_batch_plan *plan, void *workspace,
                            size_t workspace_bytes, void *stream);
int scqr3_factor_batched(const scqr3_batch_plan *plan, void *stream);
void scqr3_batch_plan_destroy(scqr3_batch_plan *plan);

/* ---------------------------------------------------------------------------
 * Adjoint (reverse mode) of scqr3_factor for B = I. Not in the paper; it is
 * the chain rule through the passes of Alg. 2/3 (Q_k = Q_{k-1} R_k^{-1},
 * R_k = chol(Q_{k-1}^T Q_{k-1} + s_k I), R = R_P ... R_1) with each shift s_k
 * held fixed: in exact arithmetic the factorization X -> (Q, R) does not
 * depend on s (R_2 R_1 is the R factor of X for any s), so the shift carries
 * no gradient. Per pass k, in reverse:
 *   M_k = Q_k^T Qbar_k,  Rbar_k = triu(L_k^T dR Racc_{k-1}^T - M_k R_k^{-T}),
 *   P_k = sym(Phi(Rbar_k R_k^T)),  Qbar_{k-1} = (Qbar_k + 2 Q_k P_k) R_k^{-T},
 *   Q_{k-1} = Q_k R_k  (recomputed; no intermediate Q is stored),
 * with L_k = R_P ... R_{k+1}, Racc_{k-1} = R_{k-1} ... R_1 and Phi the upper
 * triangle with its diagonal halved. dX = Qbar_0.
 *
 *  Q       m x n result of scqr3_factor (ldq >= n), read only.
 *  Rpass   per-pass factors as written by scqr3_factor (R_k at Rpass+(k-1)n^2).
 *  passes  scqr3_info.passes of that call (1..SCQR3_MAX_PASSES).
 *  dQ      m x n cotangent of Q (lddq >= n); dR: n x n cotangent of R or NULL.
 *  dX      m x n output (lddx >= n); may alias dQ exactly.
 * Device pointers; asynchronous on `stream`; n <= 128 (else
 * SCQR3_E_UNSUPPORTED). */
int scqr3_backward_workspace_bytes(int64_t m, int n, size_t *bytes);
int scqr3_backward(const double *Q, int64_t m, int n, int64_t ldq,
                   const double *Rpass, int passes, const double *dQ,
                   int64_t lddq, const double *dR, double *dX, int64_t lddx,
                   void *workspace, size_t workspace_bytes, void *stream);

/* The adjoint with options: opts->precision selects its form (opts NULL:
 * SCQR3_PREC_FP64).
 *  SCQR3_PREC_FP64  scqr3_backward (FP64 arithmetic throughout).
 *  SCQR3_PREC_TC    the same chain rule with the row work on the tensor
 *         cores: the iterate is held as Z = [Q_k | Qbar_k J] (J reverses the
 *         column order); Qbar_k + 2 Q_k P_k and Q_{k-1} = Q_k R_k are
 *         products with n x n matrices through the exact digit split (each
 *         product within 2^-56 of the scales of its row and column; within
 *         2^-49 at n = 64, where one kernel forms both products from seven
 *         digits per value, a perturbation of P_k and R_k of order
 *         2^-49 of their norms, far inside the adjoint's O(n kappa u) error);
 *         Qbar_{k-1} R_k^T = t is the row-wise substitution of Eq.
 *         (backward2) with U = J R_k^T J applied to t J (FP64 diagonal
 *         blocks, backward stable row by row);
 *         M_k J is the upper right block of the tensor-core Gram matrix of Z.
 *         n <= 128, m <= 2^31 (else SCQR3_E_UNSUPPORTED). The workspace
 *         holds two m x 2n iterates (16 m n doubles in all).
 *  other values: SCQR3_E_UNSUPPORTED.
 * The other arguments are scqr3_backward's (argument codes -1 .. -11 the
 * same; opts is argument 12). status: NULL or a device int that receives,
 * in stream order after the adjoint, SCQR3_OK or SCQR3_E_TIMEOUT (a
 * tensor-core kernel gave up a bounded wait; dX is then not valid).
 * scqr3_backward_workspace_bytes_ex: the workspace for (m, n, opts); the
 * tensor-core form needs the device (SCQR3_E_CUDA without one). */
int scqr3_backward_workspace_bytes_ex(int64_t m, int n, const scqr3_opts *opts,
                                      size_t *bytes);
int scqr3_backward_ex(const double *Q, int64_t m, int n, int64_t ldq,
                      const double *Rpass, int passes, const double *dQ,
                      int64_t lddq, const double *dR, double *dX, int64_t lddx,
                      const scqr3_opts *opts, void *workspace,
                      size_t workspace_bytes, int *status, void *stream);

/* ---------------------------------------------------------------------------
 * scqr3_factor_noalloc: the same factorization (B = I, default options)
 * without a workspace argument, for callers that cannot allocate device
 * memory -- e.g. a host application that owns all device memory through its
 * own pool and forbids allocation by plug-in code, a caller running so close
 * to the memory limit that a late cudaMalloc could fail, or a C/Fortran code
 * that receives device pointers but has no allocator. The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Scratch comes from a fixed array of SCQR3_NOALLOC_SCRATCH_BYTES inside the
 * library. A device reserves it when the library's module holding it is
 * loaded there, and holds it until the process exits: on the first call of
 * this entry point on that device under lazy module loading (CUDA's default),
 * or when the context is created under CUDA_MODULE_LOADING=EAGER (then every
 * process using the library reserves it). Problems whose scqr3_workspace_bytes()
 * exceeds it (the scratch grows with n and with the number of CTAs, which
 * is capped by the SM count) are rejected with SCQR3_E_SCRATCH_LIMIT, so
 * scqr3_workspace_bytes() tells in advance whether a problem fits. The first call
 * on a device looks up the array's device address; make it before any stream
 * capture. All calls share the array, so calls whose GPU work overlaps (other
 * streams or host threads) race; serialize them. The call allocates nothing
 * (no cudaMalloc/cudaFree, no allocating library routine). X, Q, R, info:
 * as for scqr3_factor. A negative argument code -k names argument k of THIS
 * prototype (X 1, m 2, n 3, ldx 4, Q 5, ldq 6, R 7, info 8). */
#define SCQR3_NOALLOC_SCRATCH_BYTES (16u << 20)
int scqr3_factor_noalloc(const double *X, int64_t m, int n, int64_t ldx,
                         double *Q, int64_t ldq, double *R, scqr3_info *info,
                         void *stream);

/* ---------------------------------------------------------------------------
 * Launch timing (tracing). The paper reports per-routine times of each pass
 * (Sec. 7, Table 7); this is the device counterpart. Between
 * scqr3_timing_begin and scqr3_timing_end, every kernel that scqr3_factor
 * queues (from any host thread) is bracketed by CUDA events recorded on the
 * call's stream, so each record's time is that launch's device duration.
 * Kernels of passes that the device decides to skip are still launched (they
 * return at once) and are recorded too.
 */
#define SCQR3_KERNEL_GRAM 0     /* pass kernel: Gram of X (pass 1)          */
#define SCQR3_KERNEL_PASS 1     /* pass kernel: Q := Q R_k^{-1} (+ Gram)    */
#define SCQR3_KERNEL_REDUCE 2   /* fixed-order sum of partial Grams         */
#define SCQR3_KERNEL_CHOL 3     /* shift, Cholesky, R := R_k R, bookkeeping */
#define SCQR3_KERNEL_BFACTOR 4  /* per-block Cholesky of the oblique B      */
#define SCQR3_KERNEL_TRSM 5     /* Q := Q R_k^{-1} alone (n > 128)          */
#define SCQR3_KERNEL_FINISH 6   /* mixed form: float-pair Q to FP64, if the
                                   last solve left it in pairs             */
#define SCQR3_KERNEL_TCUPDATE 7 /* tensor-core form: diagonal blocks of R_k,
                                   X_K -= Y_J R_JK on the tensor cores     */

typedef struct {
  int kernel;  /* SCQR3_KERNEL_*                                          */
  int pass;    /* 0-based pass index the launch belongs to                */
  float ms;    /* device time from this launch's start event to the next  */
} scqr3_launch_time;

/* Start recording up to `capacity` launches (host-side; creates events).
 * Returns SCQR3_OK, -1 for capacity < 1, or SCQR3_E_CUDA. */
int scqr3_timing_begin(int capacity);

/* Stop recording, wait for the recorded events, and copy up to `capacity`
 * records (in launch order) to the HOST array `out`; *count receives the
 * number of launches recorded (which may exceed capacity). */
int scqr3_timing_end(scqr3_launch_time *out, int capacity, int *count);

/* ---------------------------------------------------------------------------
 * Test and tuning hooks (process-wide; not part of the method, and not needed
 * for normal use). They affect calls queued after they are set.
 *   SCQR3_DEBUG_WAIT_NS      value: the time limit, in nanoseconds, of the
 *                            waits by which the warps of a tensor-core kernel
 *                            hand work to each other (default 2 s; value < 0
 *                            restores it). A wait that runs out records
 *                            SCQR3_E_TIMEOUT in scqr3_info; the kernel then
 *                            waits, always with the default limit, for its own
 *                            tensor-core operations and copies before it frees
 *                            its tensor memory, so a short limit is safe. A
 *                            limit of 0 gives up at the first such wait; tests
 *                            set it to drive that path.
 *   SCQR3_DEBUG_WAIT_SCOPE   value: which kernels the limit above applies to
 *                            (bit 0: the tensor-core Gram kernel, bit 1: the
 *                            tensor-core substitution kernels; default 3);
 *                            the others keep the default limit.
 *   SCQR3_DEBUG_FUSED_SOLVE  value 1 (default): SCQR3_PREC_TC with
 *                            16 < n <= 64 runs each pass's substitution in one
 *                            sweep; 0: in the separate diagonal-block and
 *                            update launches (for comparison).
 * Returns SCQR3_OK, -1 for an unknown key, -2 for an invalid value. */
#define SCQR3_DEBUG_WAIT_NS 1
#define SCQR3_DEBUG_FUSED_SOLVE 2
#define SCQR3_DEBUG_WAIT_SCOPE 3
int scqr3_debug_set(int key, long long value);

#ifdef __cplusplus
}
#endif
#endif /* SCQR3_H */
