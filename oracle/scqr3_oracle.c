/*
 * scqr3_oracle.c -- plain FP64 CPU reference of shifted CholeskyQR3.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU legs of bench.py to check and time the CUDA library; never by the
 * library itself. It shares no code with the CUDA path.
 *
 * Every routine is the textbook loop for the formula it cites, written for
 * a reader checking it against the paper: no blocking, no reordering, no
 * fused multiply-add (built with -ffp-contract=off).
 */
#include "scqr3_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Unit roundoff of IEEE binary64 (Sec. 6: u = 2^-53). */
static const double ORC_U = 1.1102230246251565e-16;

void orc_gram(int64_t m, int n, const double *X, int64_t ldx, double *A) {
  /* a_jk = sum_i x_ij x_ik (Eq. gram). Rows are visited in ascending i, so
   * every entry is the plain left-to-right sum of its m products. */
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) A[j * n + k] = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    const double *x = X + i * ldx;
    for (int j = 0; j < n; ++j)
      for (int k = j; k < n; ++k) A[j * n + k] = A[j * n + k] + x[j] * x[k];
  }
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < j; ++k) A[j * n + k] = A[k * n + j];
}

void orc_gram_oblique(int64_t m, int n, const double *X, int64_t ldx, int bs,
                      const double *Bblk, double *A, double *fro2) {
  /* A = X^T Y with Y = B X formed explicitly (Sec. 7.2 describes forming
   * Y := B X and then X^T Y). B is block diagonal: y_i = sum over the rows
   * l of i's block of b_il x_l. */
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double f = 0.0;
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) A[j * n + k] = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    const int64_t blk = i / bs;
    const int r = (int)(i - blk * bs);
    const double *b = Bblk + blk * (int64_t)bs * bs + (int64_t)r * bs;
    for (int k = 0; k < n; ++k) {
      double t = 0.0;
      for (int l = 0; l < bs; ++l) t = t + b[l] * X[(blk * bs + l) * ldx + k];
      y[k] = t;
    }
    const double *x = X + i * ldx;
    for (int j = 0; j < n; ++j) {
      f = f + x[j] * x[j];
      for (int k = j; k < n; ++k) A[j * n + k] = A[j * n + k] + x[j] * y[k];
    }
  }
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < j; ++k) A[j * n + k] = A[k * n + j];
  if (fro2) *fro2 = f;
  free(y);
}

double orc_shift(int64_t m, int n, double normx2) {
  /* Eq. (finds2). */
  const double mn = (double)m * (double)n;
  const double nn1 = (double)n * (double)(n + 1);
  return 11.0 * (mn + nn1) * ORC_U * normx2;
}

double orc_normest2(int n, const double *A) {
  /* Power method: v := A v / ||A v|| from v = (1, ..., 1) / sqrt(n); the
   * estimate is the Rayleigh quotient v^T A v (v of unit length), stopped once
   * it changes by at most 1e-12 of itself, or after 200 steps. */
  double *v = (double *)malloc(sizeof(double) * (size_t)n);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  for (int j = 0; j < n; ++j) v[j] = 1.0 / sqrt((double)n);
  double lam = 0.0;
  for (int it = 0; it < 200; ++it) {
    for (int j = 0; j < n; ++j) {
      double t = 0.0;
      for (int k = 0; k < n; ++k) t = t + A[j * n + k] * v[k];
      w[j] = t;
    }
    double q = 0.0, ww = 0.0;
    for (int j = 0; j < n; ++j) {
      q = q + v[j] * w[j];
      ww = ww + w[j] * w[j];
    }
    const double nw = sqrt(ww);
    const int done = it > 0 && fabs(q - lam) <= 1e-12 * q;
    lam = q;
    if (done || !(nw > 0.0)) break;
    for (int j = 0; j < n; ++j) v[j] = w[j] / nw;
  }
  free(v);
  free(w);
  return lam;
}

double orc_shift_oblique(int64_t m, int n, double normx2, double normb) {
  /* Eq. (finds2B). */
  const double dm = (double)m;
  const double t = 2.0 * dm * sqrt(dm * (double)n);
  const double nn1 = (double)n * (double)(n + 1);
  return 11.0 * (t + nn1) * ORC_U * normx2 * normb;
}

int orc_chol(int n, const double *A, double s, double *R) {
  /* R^T R = A + sI: for column j, r_jj = sqrt(a_jj + s - sum_{k<j} r_kj^2)
   * and r_jl = (a_jl - sum_{k<j} r_kj r_kl) / r_jj for l > j. */
  for (int j = 0; j < n * n; ++j) R[j] = 0.0;
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j] + s;
    for (int k = 0; k < j; ++k) d = d - R[k * n + j] * R[k * n + j];
    if (!(d > 0.0) || !isfinite(d)) return j + 1;
    const double rjj = sqrt(d);
    R[j * n + j] = rjj;
    for (int l = j + 1; l < n; ++l) {
      double t = A[j * n + l];
      for (int k = 0; k < j; ++k) t = t - R[k * n + j] * R[k * n + l];
      R[j * n + l] = t / rjj;
    }
  }
  return 0;
}

void orc_trsm(int64_t m, int n, const double *X, int64_t ldx, const double *R,
              double *Q, int64_t ldq) {
  /* q_i^T R = x_i^T, i.e. x_ij = sum_{k<=j} q_ik r_kj, solved for
   * j = 0, 1, ... in turn: q_ij = (x_ij - sum_{k<j} q_ik r_kj) / r_jj. */
  for (int64_t i = 0; i < m; ++i) {
    const double *x = X + i * ldx;
    double *q = Q + i * ldq;
    for (int j = 0; j < n; ++j) {
      double t = x[j];
      for (int k = 0; k < j; ++k) t = t - q[k] * R[k * n + j];
      q[j] = t / R[j * n + j];
    }
  }
}

void orc_trmm(int n, const double *Rt, double *R) {
  /* (Rt R)_ij = sum_{i<=k<=j} rt_ik r_kj for i <= j; the product of two
   * upper triangular matrices is upper triangular. */
  double *P = (double *)calloc((size_t)n * n, sizeof(double));
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      double t = 0.0;
      for (int k = i; k <= j; ++k) t = t + Rt[i * n + k] * R[k * n + j];
      P[i * n + j] = t;
    }
  memcpy(R, P, sizeof(double) * (size_t)n * n);
  free(P);
}

double orc_normb_bound(int64_t m, int bs, const double *Bblk) {
  /* ||B||_2 = max_j ||B_j||_2 <= max_j ||B_j||_F. */
  double best = 0.0;
  const int64_t nb = m / bs;
  for (int64_t j = 0; j < nb; ++j) {
    const double *b = Bblk + j * (int64_t)bs * bs;
    double f = 0.0;
    for (int l = 0; l < bs * bs; ++l) f = f + b[l] * b[l];
    f = sqrt(f);
    if (f > best) best = f;
  }
  return best;
}

void orc_gram_csr(int64_t m, int n, const double *X, int64_t ldx, const int64_t *row_ptr,
                  const int32_t *col_idx, const double *vals, double *A, double *fro2) {
  /* Y = B X with the sparse product of Sec. 7.2, then A = X^T Y. */
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double f = 0.0;
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) A[j * n + k] = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    for (int k = 0; k < n; ++k) y[k] = 0.0;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      const double *xl = X + (int64_t)col_idx[p] * ldx;
      for (int k = 0; k < n; ++k) y[k] = y[k] + vals[p] * xl[k];
    }
    const double *x = X + i * ldx;
    for (int j = 0; j < n; ++j) {
      f = f + x[j] * x[j];
      for (int k = j; k < n; ++k) A[j * n + k] = A[j * n + k] + x[j] * y[k];
    }
  }
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < j; ++k) A[j * n + k] = A[k * n + j];
  if (fro2) *fro2 = f;
  free(y);
}

double orc_normb_csr(int64_t m, const int64_t *row_ptr, const double *vals) {
  double best = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    double r = 0.0;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) r = r + fabs(vals[p]);
    if (r > best) best = r;
  }
  return best;
}

/* The inner product of one factorization: B = I, block-diagonal B or CSR B. */
typedef struct {
  int kind; /* 0: B = I; 1: block diagonal (bs, Bblk); 2: CSR */
  int bs;
  const double *Bblk;
  const int64_t *row_ptr;
  const int32_t *col_idx;
  const double *vals;
} orc_inner;

static int orc_drive(int64_t m, int n, const double *X, int64_t ldx, const orc_inner *B,
                     double normx2, double normb, int max_passes, double shift_scale,
                     int algorithm, double tol, double *Q, int64_t ldq, double *R,
                     orc_trace *trace);

int orc_scqr3(int64_t m, int n, const double *X, int64_t ldx, int bs,
              const double *Bblk, double normx2, double normb, int max_passes,
              double *Q, int64_t ldq, double *R, orc_trace *trace) {
  return orc_scqr3_ex(m, n, X, ldx, bs, Bblk, normx2, normb, max_passes, 0.0, 3, 0.0,
                      Q, ldq, R, trace);
}

int orc_scqr3_ex(int64_t m, int n, const double *X, int64_t ldx, int bs,
                 const double *Bblk, double normx2, double normb, int max_passes,
                 double shift_scale, int algorithm, double tol, double *Q,
                 int64_t ldq, double *R, orc_trace *trace) {
  if (bs > 0 && (m % bs) != 0) return ORC_E_ARG;
  orc_inner B = {bs > 0 ? 1 : 0, bs, Bblk, NULL, NULL, NULL};
  return orc_drive(m, n, X, ldx, &B, normx2, normb, max_passes, shift_scale, algorithm, tol, Q,
                   ldq, R, trace);
}

int orc_scqr3_csr(int64_t m, int n, const double *X, int64_t ldx, const int64_t *row_ptr,
                  const int32_t *col_idx, const double *vals, double normx2, double normb,
                  int max_passes, double shift_scale, int algorithm, double tol, double *Q,
                  int64_t ldq, double *R, orc_trace *trace) {
  if (!row_ptr || !col_idx || !vals) return ORC_E_ARG;
  orc_inner B = {2, 0, NULL, row_ptr, col_idx, vals};
  return orc_drive(m, n, X, ldx, &B, normx2, normb, max_passes, shift_scale, algorithm, tol, Q,
                   ldq, R, trace);
}

static int orc_drive(int64_t m, int n, const double *X, int64_t ldx, const orc_inner *B,
                     double normx2, double normb, int max_passes, double shift_scale,
                     int algorithm, double tol, double *Q, int64_t ldq, double *R,
                     orc_trace *trace) {
  if (m < n || n < 1 || ldx < n || ldq < n || max_passes < 3 ||
      max_passes > ORC_MAX_PASSES || (algorithm != 2 && algorithm != 3))
    return ORC_E_ARG;
  /* Alg. 2's printed tolerance sqrt(n) u lies below the rounding error of a
   * computed Gram matrix of orthonormal columns, so tol <= 0 selects the
   * orthogonality bound that Thm. (maincholqr3) proves for the final Q,
   * 6 {mn + n(n+1)} u. */
  if (!(tol > 0.0)) tol = 6.0 * ((double)m * (double)n + (double)n * (double)(n + 1)) * ORC_U;
  const int oblique = B->kind != 0;
  if (normx2 < 0.0 && oblique) return ORC_E_ARG;  /* the 2-norm estimate: B = I only */
  if (B->kind == 1 && !(normb > 0.0)) normb = orc_normb_bound(m, B->bs, B->Bblk);
  if (B->kind == 2 && !(normb > 0.0)) normb = orc_normb_csr(m, B->row_ptr, B->vals);

  double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
  double *Rt = (double *)malloc(sizeof(double) * (size_t)n * n);
  orc_trace tr;
  memset(&tr, 0, sizeof(tr));
  int status = ORC_E_MAXPASS;

  /* Alg. 2 and Alg. 3 start from Q := X, R := I. */
  if (Q != X)
    for (int64_t i = 0; i < m; ++i)
      memcpy(Q + i * ldq, X + i * ldx, sizeof(double) * (size_t)n);
  for (int i = 0; i < n * n; ++i) R[i] = 0.0;
  for (int i = 0; i < n; ++i) R[i * n + i] = 1.0;

  int plain_in_a_row = 0;
  for (int p = 0; p < max_passes; ++p) {
    /* A := Q^T Q (or Q^T B Q); ||Q||^2 is estimated by ||Q||_F^2, which
     * for B = I is the trace of the computed Gram matrix (Sec. 4.1). */
    double nrm2 = 0.0;
    if (B->kind == 1) {
      orc_gram_oblique(m, n, Q, ldq, B->bs, B->Bblk, A, &nrm2);
    } else if (B->kind == 2) {
      orc_gram_csr(m, n, Q, ldq, B->row_ptr, B->col_idx, B->vals, A, &nrm2);
    } else {
      orc_gram(m, n, Q, ldq, A);
      for (int j = 0; j < n; ++j) nrm2 = nrm2 + A[j * n + j];
    }
    if (!isfinite(nrm2)) {
      status = ORC_E_NONFINITE;
      break;
    }
    if (p == 0 && normx2 > 0.0) nrm2 = normx2;
    /* normx2 < 0: ||Q||_2^2 estimated by the power method (Sec. 4.1: normest) */
    if (normx2 < 0.0) nrm2 = orc_normest2(n, A);

    /* Alg. 2's loop test: stop when the current iterate is orthonormal enough
     * (its Gram matrix A is already at hand). */
    if (algorithm == 2 && p > 0) {
      double d2 = 0.0;
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          const double e = A[j * n + k] - (j == k ? 1.0 : 0.0);
          d2 = d2 + e * e;
        }
      if (sqrt(d2) <= tol) {
        status = ORC_OK;
        break;
      }
    }
    tr.norm2[p] = nrm2;

    /* Alg. 3: pass 1 always shifts. Alg. 2 and the later passes of
     * Alg. 3 try the plain Cholesky and shift only if it breaks down (Alg. 2
     * breakdown rule). */
    int shifted = (algorithm == 3 && p == 0);
    if (!shifted) {
      const int fail = orc_chol(n, A, 0.0, Rt);
      tr.unshifted_fail[p] = fail;
      shifted = (fail != 0);
    }
    double s = 0.0;
    if (shifted) {
      const double safe = oblique ? orc_shift_oblique(m, n, nrm2, normb) : orc_shift(m, n, nrm2);
      int fail = 1;
      if (shift_scale > 0.0) {
        /* the smaller shift c u ||X||^2 (x ||B||) of the remark in Sec. 6.1 */
        s = oblique ? shift_scale * ORC_U * nrm2 * normb : shift_scale * ORC_U * nrm2;
        fail = orc_chol(n, A, s, Rt);
      }
      if (fail) {
        s = safe;
        fail = orc_chol(n, A, s, Rt);
      }
      if (fail) {
        tr.passes = p + 1;
        tr.shifted[p] = 1;
        tr.s[p] = s;
        status = fail;
        break;
      }
    }
    tr.shifted[p] = shifted;
    tr.s[p] = s;
    tr.passes = p + 1;

    /* Q := Q Rt^{-1}, R := Rt R (the update of Alg. 2). */
    orc_trsm(m, n, Q, ldq, Rt, Q, ldq);
    orc_trmm(n, Rt, R);

    /* Alg. 3: two plain CholeskyQR passes after the last shifted one complete
     * CholeskyQR2 (the last two steps of Alg. 3). */
    plain_in_a_row = shifted ? 0 : plain_in_a_row + 1;
    if (algorithm == 3 && plain_in_a_row == 2) {
      status = ORC_OK;
      break;
    }
  }
  if (trace) *trace = tr;
  free(A);
  free(Rt);
  return status;
}
