/*
 * scqr3_oracle.h -- plain FP64 CPU reference of shifted CholeskyQR3.
 *
 * TEST INFRASTRUCTURE ONLY. This oracle exists to check the CUDA library
 * against the paper (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
 * "Shifted Cholesky QR for computing the QR factorization of ill-conditioned
 * matrices"). Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load it. The product path never calls it.
 *
 * Conventions: row-major storage, 0-based indices, X is m x n with leading
 * dimension ldx >= n, R is n x n upper triangular (row-major, lower part
 * zero). All arithmetic is binary64; the library is compiled with
 * -ffp-contract=off so that every a*b+c is two roundings, identical on
 * x86-64 and AArch64.
 */
#ifndef SCQR3_ORACLE_H
#define SCQR3_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_PASSES 16

/* Status values, same meaning as the CUDA library's. */
#define ORC_OK 0
#define ORC_E_ARG (-1)
#define ORC_E_NONFINITE (-100)
#define ORC_E_MAXPASS (-101)

/* Per-pass record of one factorization (Alg. 2 / Alg. 3). */
typedef struct {
  int passes;                         /* CholeskyQR passes executed        */
  int shifted[ORC_MAX_PASSES];        /* 1 if pass k used chol(A + sI)     */
  int unshifted_fail[ORC_MAX_PASSES]; /* column (1-based) where the plain
                                         chol(A) broke down, else 0        */
  double s[ORC_MAX_PASSES];           /* shift used in pass k (0 if none)  */
  double norm2[ORC_MAX_PASSES];       /* ||Q_{k-1}||^2 estimate used       */
} orc_trace;

/* Gram matrix A = X^T X (Eq. gram; the first step of Alg. 1). A is n x n full
 * symmetric; the upper triangle is computed, the lower mirrored. Each entry
 * is the sum over rows i = 0..m-1 in ascending order. */
void orc_gram(int64_t m, int n, const double *X, int64_t ldx, double *A);

/* Oblique Gram A = X^T (B X) (the first step of Alg. 4) for block-diagonal B made of
 * m/bs dense bs x bs blocks (row-major, block j at Bblk + j*bs*bs). Y = B X
 * is formed block by block, then the upper triangle of X^T Y, ascending
 * rows, mirrored. Also returns sum_ij x_ij^2 in *fro2 (may be NULL). */
void orc_gram_oblique(int64_t m, int n, const double *X, int64_t ldx, int bs,
                      const double *Bblk, double *A, double *fro2);

/* Shift s = 11 {mn + n(n+1)} u ||X||_2^2, Eq. (finds2); u = 2^-53. */
double orc_shift(int64_t m, int n, double normx2);

/* lambda_max(A) of an n x n symmetric positive semidefinite A (row-major) by
 * the power method: the estimate of ||Q||_2^2 = lambda_max(Q^T Q) that Sec. 4.1
 * allows in the shift (normest). */
double orc_normest2(int n, const double *A);

/* Oblique shift s = 11 {2 m sqrt(mn) + n(n+1)} u ||X||_2^2 ||B||_2,
 * Eq. (finds2B). */
double orc_shift_oblique(int64_t m, int n, double normx2, double normb);

/* Cholesky factor R (upper, R^T R = A + sI), column by column (the shifted
 * Cholesky of Alg. 1). Returns 0, or the 1-based column j at which the radicand
 * a_jj + s - sum_{k<j} r_kj^2 is not a positive finite number. */
int orc_chol(int n, const double *A, double s, double *R);

/* Q = X R^{-1} row by row: x_i^T = q_i^T R is solved by substitution
 * across the columns (Eq. backward2). Q may alias X. */
void orc_trsm(int64_t m, int n, const double *X, int64_t ldx, const double *R,
              double *Q, int64_t ldq);

/* R := Rt R for upper triangular Rt, R (the R update of Alg. 2). */
void orc_trmm(int n, const double *Rt, double *R);

/* Upper bound of ||B||_2 for block-diagonal B: max over blocks of the
 * block's Frobenius norm. */
double orc_normb_bound(int64_t m, int bs, const double *Bblk);

/* Oblique Gram A = X^T (B X) for a sparse symmetric B held in CSR form
 * (Sec. 7.2 forms Y := B X with a sparse product, then X^T Y). Row i of Y is
 * y_i = sum over the stored entries p = row_ptr[i] .. row_ptr[i+1]-1, in
 * storage order, of vals[p] x_{col_idx[p]}; then the upper triangle of X^T Y
 * by ascending rows, mirrored. Also sum_ij x_ij^2 in *fro2 (may be NULL). */
void orc_gram_csr(int64_t m, int n, const double *X, int64_t ldx, const int64_t *row_ptr,
                  const int32_t *col_idx, const double *vals, double *A, double *fro2);

/* Upper bound of ||B||_2 for symmetric B in CSR form: the largest absolute
 * row sum (||B||_2 = rho(B) <= ||B||_inf, Gershgorin). */
double orc_normb_csr(int64_t m, const int64_t *row_ptr, const double *vals);

/* Shifted CholeskyQR3 (Alg. 3; oblique: Alg. 5) with the breakdown rule of
 * Alg. 2: pass 1 is always shifted; a later pass whose plain Cholesky
 * breaks down is redone with the shift; the factorization ends after two
 * consecutive unshifted passes. bs == 0 means B = I. normx2 < 0 (B = I only)
 * estimates ||Q||_2^2 of every shifted pass by orc_normest2 of its Gram
 * matrix. normx2 > 0 replaces
 * ||X||_2^2 in the pass-1 shift (else ||X||_F^2 is used, see Sec. 4.1);
 * normb > 0 is ||B||_2 (else orc_normb_bound). Returns ORC_OK, a positive
 * breakdown column, or a negative ORC_E_* code. Q may alias X. */
int orc_scqr3(int64_t m, int n, const double *X, int64_t ldx, int bs,
              const double *Bblk, double normx2, double normb, int max_passes,
              double *Q, int64_t ldq, double *R, orc_trace *trace);

/* Options of the generalized driver below.
 *  shift_scale <= 0: the shift of Eq. (finds2)/(finds2B) (safe);
 *             c > 0: first the smaller shift c u ||X||^2 (c u ||X||^2 ||B|| in
 *                the oblique case) -- the remark of Sec. 6.1 and the conclusion
 *                suggest s = O(u ||X||^2), c = 1 being the remark's choice --
 *                then the safe shift if that Cholesky breaks down.
 *  algorithm  3: Alg. 3 -- pass 1 always shifted, end after two consecutive
 *                unshifted passes;
 *             2: Alg. 2 -- every pass first tries the plain Cholesky and
 *                shifts only on breakdown; the iteration ends as soon as
 *                ||Q^T Q - I||_F <= tol (||Q^T B Q - I||_F for oblique B),
 *                tested on the Gram matrix of the current iterate; tol <= 0
 *                selects 6 {mn + n(n+1)} u, the bound of Thm. (maincholqr3)
 *                (the printed sqrt(n) u is below the rounding error of the
 *                computed Gram matrix and is reached only by chance). */
int orc_scqr3_ex(int64_t m, int n, const double *X, int64_t ldx, int bs,
                 const double *Bblk, double normx2, double normb, int max_passes,
                 double shift_scale, int algorithm, double tol, double *Q,
                 int64_t ldq, double *R, orc_trace *trace);

/* orc_scqr3_ex with the oblique inner product of a sparse SPD B in CSR form
 * (Alg. 5, Gram by orc_gram_csr; normb <= 0 selects orc_normb_csr). */
int orc_scqr3_csr(int64_t m, int n, const double *X, int64_t ldx, const int64_t *row_ptr,
                  const int32_t *col_idx, const double *vals, double normx2, double normb,
                  int max_passes, double shift_scale, int algorithm, double tol, double *Q,
                  int64_t ldq, double *R, orc_trace *trace);

#ifdef __cplusplus
}
#endif
#endif
