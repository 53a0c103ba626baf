// adjoint.cu -- reverse mode of shifted CholeskyQR3 (B = I), FP64, sm_103a.
//
// Forward pass k (Alg. 2/3): A_k = Q_{k-1}^T Q_{k-1} + s_k I, R_k = chol(A_k),
// Q_k = Q_{k-1} R_k^{-1}; R = R_P ... R_1. With the shifts held fixed (in
// exact arithmetic the factorization does not depend on them), the chain rule
// through one pass, given Qbar_k and the cotangent Rbar of R, is
//
//   M_k        = Q_k^T Qbar_k                                   (cross Gram)
//   Rbar_k     = triu(L_k^T Rbar Racc_{k-1}^T - M_k R_k^{-T})    (TRSM + product)
//   P_k        = sym(Phi(Rbar_k R_k^T))                          (Cholesky)
//   Qbar_{k-1} = (Qbar_k + 2 Q_k P_k) R_k^{-T}                   (Gram + TRSM)
//   Q_{k-1}    = Q_k R_k                                         (recomputed)
//
// with L_k = R_P ... R_{k+1}, Racc_{k-1} = R_{k-1} ... R_1 and Phi(W) the
// upper triangle of W with its diagonal halved. Nothing from the forward
// pass but Q (= Q_P) and the factors R_k is kept: the intermediate Q_k are
// recomputed one pass at a time, walking back from Q_P.
//
//   bw_rows_kernel   one streaming pass over the rows: Qbar_{k-1}, Q_{k-1},
//                    and per-CTA partial sums of M_{k-1} = Q_{k-1}^T Qbar_{k-1}
//   bw_small_kernel  one CTA: the n x n algebra of Rbar_k and P_k
#include <cmath>

#include "scqr3_internal.cuh"

namespace scqr3 {

template <int NP> struct BwCfg;
template <> struct BwCfg<16>  { static constexpr int PR = 128, T = 16,  C = 16; };
template <> struct BwCfg<32>  { static constexpr int PR = 128, T = 32,  C = 32; };
template <> struct BwCfg<64>  { static constexpr int PR = 128, T = 64,  C = 64; };
template <> struct BwCfg<128> { static constexpr int PR = 32,  T = 256, C = 64; };

template <int NP> struct BwGeo {
  static constexpr int PR = BwCfg<NP>::PR, T = BwCfg<NP>::T, C = BwCfg<NP>::C;
  static constexpr int G = kThreads / T;   // cross-Gram groups per CTA
  static constexpr int RG = PR / G;        // panel rows per group
  static constexpr int LD = NP + 1;
  static constexpr int E = pk_size(NP);
  static constexpr int NN = NP * NP;
  // panels Q and Qbar, P_k (symmetric, packed upper), R_k (packed), 1/r_jj
  static constexpr size_t smem = sizeof(double) * ((size_t)2 * PR * LD + E + E + NP);
};

enum { BW_FIRST = 0, BW_PASS = 1 };

// mode BW_FIRST: copy Q -> Qw and dQ -> dX, and accumulate M_P = Q^T dQ.
// mode BW_PASS:  pass k (1-based): Qbar_{k-1} -> dX (in place), Q_{k-1} -> Qw
//                (in place) and, if k > 1, partial sums of M_{k-1}.
template <int NP>
__global__ void __launch_bounds__(kThreads, 1)
bw_rows_kernel(int mode, int k, int64_t m, int n, const double* qsrc, int64_t ldqs,
               const double* bsrc, int64_t ldbs, double* __restrict__ qw, double* dx, int64_t lddx,
               const double* __restrict__ Pk, const double* __restrict__ rk,
               double* __restrict__ partials) {
  using g = BwGeo<NP>;
  extern __shared__ __align__(16) double smem[];
  double* pq = smem;                       // PR x LD : rows of Q_k, then Q_{k-1}
  double* pb = pq + g::PR * g::LD;         // PR x LD : rows of Qbar_k, then Qbar_{k-1}
  double* P = pb + g::PR * g::LD;          // symmetric P_k, packed upper
  double* rp = P + g::E;                   // packed R_k
  double* rinv = rp + g::E;
  const int tid = threadIdx.x;
  const bool rows_work = (mode == BW_PASS);
  const bool want_m = (mode == BW_FIRST) || k > 1;

  if (rows_work) {
    for (int e = tid; e < g::E; e += kThreads) P[e] = Pk[e];
    for (int e = tid; e < g::E; e += kThreads) rp[e] = rk[e];
    __syncthreads();
    if (tid < NP) rinv[tid] = 1.0 / rp[pk_row(NP, tid)];
  }
  const int tt = tid % g::T, grp = tid / g::T;
  const int mj = tt % NP;                       // row j of M owned by this thread
  const int l0 = (tt / NP) * g::C;              // first column of its slice
  double acc[g::C];
#pragma unroll
  for (int l = 0; l < g::C; ++l) acc[l] = 0.0;

  const int64_t npanels = (m + g::PR - 1) / g::PR;
  for (int64_t pnl = blockIdx.x; pnl < npanels; pnl += gridDim.x) {
    const int64_t row0 = pnl * g::PR;
    const int rows = (int)((m - row0) < (int64_t)g::PR ? (m - row0) : (int64_t)g::PR);
    __syncthreads();
    const double* qs = (mode == BW_FIRST) ? qsrc : qw;
    const int64_t lq = (mode == BW_FIRST) ? ldqs : (int64_t)n;
    const double* bs = (mode == BW_FIRST) ? bsrc : dx;
    const int64_t lb = (mode == BW_FIRST) ? ldbs : lddx;
    for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
      const int r = idx / NP, c = idx % NP;
      double vq = 0.0, vb = 0.0;
      if (r < rows && c < n) {
        vq = qs[(row0 + r) * lq + c];
        vb = bs[(row0 + r) * lb + c];
      }
      pq[r * g::LD + c] = vq;
      pb[r * g::LD + c] = vb;
    }
    __syncthreads();

    if (rows_work && tid < rows) {
      double* q = pq + tid * g::LD;
      double* b = pb + tid * g::LD;
      // b := Qbar_k row + 2 q P_k   (n^2 FMAs, independent per column);
      // P_k(l, j) is P(min, max) of the packed upper triangle
      for (int l = 0; l < n; ++l) {
        const double c = 2.0 * q[l];
#pragma unroll 4
        for (int j = 0; j < l; ++j) b[j] = fma(c, P[pk_idx(NP, j, l)], b[j]);
        const double* Pl = P + pk_row(NP, l) - l;  // Pl[j] = P(l, j), j >= l
#pragma unroll 4
        for (int j = l; j < n; ++j) b[j] = fma(c, Pl[j], b[j]);
      }
      // y R_k^T = b, i.e. R_k y^T = b^T: back substitution, column oriented
      for (int j = n - 1; j >= 0; --j) {
        const double y = b[j] * rinv[j];
        b[j] = y;
#pragma unroll 4
        for (int l = 0; l < j; ++l) b[l] = fma(-y, rp[pk_idx(NP, l, j)], b[l]);
      }
      // Q_{k-1} row = q R_k  (x_j = sum_{l<=j} q_l r_lj), descending j in place
      if (k > 1) {
        for (int j = n - 1; j >= 0; --j) {
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int l = 0;
          for (; l + 3 <= j; l += 4) {
            s0 = fma(q[l], rp[pk_idx(NP, l, j)], s0);
            s1 = fma(q[l + 1], rp[pk_idx(NP, l + 1, j)], s1);
            s2 = fma(q[l + 2], rp[pk_idx(NP, l + 2, j)], s2);
            s3 = fma(q[l + 3], rp[pk_idx(NP, l + 3, j)], s3);
          }
          for (; l <= j; ++l) s0 = fma(q[l], rp[pk_idx(NP, l, j)], s0);
          q[j] = (s0 + s1) + (s2 + s3);
        }
      }
    }
    __syncthreads();
    // write back: Qbar (always), Q (pass k > 1, or the copy of the first mode)
    for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
      const int r = idx / NP, c = idx % NP;
      if (r < rows && c < n) {
        dx[(row0 + r) * lddx + c] = pb[r * g::LD + c];
        if (want_m) qw[(row0 + r) * n + c] = pq[r * g::LD + c];
      }
    }
    if (!want_m) continue;
    // cross Gram M += q^T b over this group's rows: thread owns M(mj, l0..l0+C)
    const int rbeg = grp * g::RG;
    const int rend = min(rbeg + g::RG, rows);
    for (int r = rbeg; r < rend; ++r) {
      const double a = pq[r * g::LD + mj];
      const double* brow = pb + r * g::LD + l0;
#pragma unroll
      for (int l = 0; l < g::C; ++l) acc[l] = fma(a, brow[l], acc[l]);
    }
  }
  if (!want_m) return;
  double* part = partials + ((int64_t)blockIdx.x * g::G + grp) * g::NN;
#pragma unroll
  for (int l = 0; l < g::C; ++l) part[mj * NP + l0 + l] = acc[l];
}

// -------------------------------------------------------------------------------------------
// n x n algebra of pass k (one CTA). Matrices are full NP x NP row-major in
// the scratch `w` (L2-resident); R_i are read from Rpass (n x n each).
//   T   = Rbar Racc_{k-1}^T,  Rb = L_k^T T              (cotangent of R_k via R)
//   Z   = M_k R_k^{-T}                                   (TRSM adjoint)
//   Rb  = triu(Rb - Z)
//   W   = Rb R_k^T,  P_k = sym(Phi(W))                   (Cholesky adjoint)
__device__ void mat_set_identity(double* A, int np) {
  for (int e = threadIdx.x; e < np * np; e += blockDim.x) A[e] = (e / np == e % np) ? 1.0 : 0.0;
}

// C = A * B (all np x np, full); C must not alias A or B
__device__ void mat_mul(const double* A, const double* B, double* C, int np, int n) {
  for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
    const int i = e / np, j = e % np;
    double s = 0.0;
    if (i < n && j < n)
      for (int l = 0; l < n; ++l) s = fma(A[i * np + l], B[l * np + j], s);
    C[e] = s;
  }
}

template <int NP>
__global__ void __launch_bounds__(1024, 1)
bw_small_kernel(int k, int P, int n, const double* __restrict__ Rpass, const double* __restrict__ dR,
                const double* __restrict__ M, double* __restrict__ w, double* __restrict__ Pk,
                double* __restrict__ rk) {
  constexpr int NN = NP * NP;
  double* Lk = w;            // R_P ... R_{k+1}
  double* Ra = w + NN;       // R_{k-1} ... R_1
  double* T = w + 2 * NN;
  double* Rb = w + 3 * NN;
  double* Tmp = w + 4 * NN;
  double* Rk = w + 5 * NN;   // R_k, full, padded with identity
  const int tid = threadIdx.x, nt = blockDim.x;
  auto Rof = [&](int i, int r, int c) -> double {  // entry (r, c) of R_i (1-based i)
    return (r < n && c < n) ? Rpass[(int64_t)(i - 1) * n * n + r * n + c] : (r == c ? 1.0 : 0.0);
  };
  // R_k (full + packed for the row kernel)
  for (int e = tid; e < NN; e += nt) Rk[e] = Rof(k, e / NP, e % NP);
  for (int e = tid; e < pk_size(NP); e += nt) {
    int j = 0;
    while (pk_row(NP, j + 1) <= e) ++j;
    rk[e] = Rof(k, j, j + (e - pk_row(NP, j)));
  }
  // Ra = R_{k-1} ... R_1 (left-multiplied in turn)
  mat_set_identity(Ra, NP);
  __syncthreads();
  for (int i = 1; i < k; ++i) {
    for (int e = tid; e < NN; e += nt) {
      const int r = e / NP, c = e % NP;
      double s = 0.0;
      for (int l = 0; l < NP; ++l) s = fma(Rof(i, r, l), Ra[l * NP + c], s);
      Tmp[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < NN; e += nt) Ra[e] = Tmp[e];
    __syncthreads();
  }
  // Lk = R_P ... R_{k+1}
  mat_set_identity(Lk, NP);
  __syncthreads();
  for (int i = k + 1; i <= P; ++i) {
    for (int e = tid; e < NN; e += nt) {
      const int r = e / NP, c = e % NP;
      double s = 0.0;
      for (int l = 0; l < NP; ++l) s = fma(Rof(i, r, l), Lk[l * NP + c], s);
      Tmp[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < NN; e += nt) Lk[e] = Tmp[e];
    __syncthreads();
  }
  // T = Rbar Ra^T ; Rb = Lk^T T
  for (int e = tid; e < NN; e += nt) {
    const int r = e / NP, c = e % NP;
    double s = 0.0;
    if (dR && r < n && c < n)
      for (int l = 0; l < n; ++l) s = fma(dR[r * n + l], Ra[c * NP + l], s);
    T[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < NN; e += nt) {
    const int r = e / NP, c = e % NP;
    double s = 0.0;
    if (r < n && c < n)
      for (int l = 0; l < n; ++l) s = fma(Lk[l * NP + r], T[l * NP + c], s);
    Rb[e] = s;
  }
  __syncthreads();
  // Z = M R_k^{-T}: each row z of Z solves R_k z^T = m^T (back substitution); Z -> T
  for (int r = tid; r < NP; r += nt) {
    double* z = T + r * NP;
    for (int j = 0; j < NP; ++j) z[j] = (r < n && j < n) ? M[r * NP + j] : 0.0;
    for (int j = n - 1; j >= 0; --j) {
      double t = z[j];
      for (int l = j + 1; l < n; ++l) t = fma(-Rk[j * NP + l], z[l], t);
      z[j] = t / Rk[j * NP + j];
    }
  }
  __syncthreads();
  // Rb = triu(Rb - Z)
  for (int e = tid; e < NN; e += nt) {
    const int r = e / NP, c = e % NP;
    Rb[e] = (c >= r) ? Rb[e] - T[e] : 0.0;
  }
  __syncthreads();
  // W = Rb R_k^T -> Tmp ; P_k = sym(Phi(W))
  for (int e = tid; e < NN; e += nt) {
    const int r = e / NP, c = e % NP;
    double s = 0.0;
    if (r < n && c < n)
      for (int l = (r > c ? r : c); l < n; ++l) s = fma(Rb[r * NP + l], Rk[c * NP + l], s);
    Tmp[e] = s;
  }
  __syncthreads();
  // packed upper: P(r, c) = W(r, c) / 2 for r <= c (the diagonal is halved once
  // by Phi and the off-diagonal once by the symmetrization)
  for (int e = tid; e < pk_size(NP); e += nt) {
    int r = 0;
    while (pk_row(NP, r + 1) <= e) ++r;
    const int c = r + (e - pk_row(NP, r));
    Pk[e] = 0.5 * Tmp[r * NP + c];
  }
}

// -------------------------------------------------------------------------------------------
// Host side.

template <int NP>
static cudaError_t bw_setup(int* ctas_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(bw_rows_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BwGeo<NP>::smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, bw_rows_kernel<NP>, kThreads,
                                                       BwGeo<NP>::smem);
}

struct BwPlan {
  int np, grid, groups, pr;
  size_t qw, partials, M, Pk, rk, w, total;
};

static int bw_padded(int n) { return n <= 16 ? 16 : n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 0; }
static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static int bw_plan(int64_t m, int n, BwPlan* p) {
  const int np = bw_padded(n);
  if (!np) return SCQR3_E_UNSUPPORTED;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCQR3_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SCQR3_E_CUDA;
  cudaError_t e;
  switch (np) {
    case 16: e = bw_setup<16>(&per); p->groups = BwGeo<16>::G; p->pr = BwGeo<16>::PR; break;
    case 32: e = bw_setup<32>(&per); p->groups = BwGeo<32>::G; p->pr = BwGeo<32>::PR; break;
    case 64: e = bw_setup<64>(&per); p->groups = BwGeo<64>::G; p->pr = BwGeo<64>::PR; break;
    default: e = bw_setup<128>(&per); p->groups = BwGeo<128>::G; p->pr = BwGeo<128>::PR; break;
  }
  if (e != cudaSuccess || per < 1) return SCQR3_E_CUDA;
  p->np = np;
  const int64_t npanels = (m + p->pr - 1) / p->pr;
  const int64_t gmax = (int64_t)sms * per;
  p->grid = (int)(npanels < gmax ? npanels : gmax);
  if (p->grid < 1) p->grid = 1;
  const size_t NN = (size_t)np * np;
  size_t off = 0;
  p->qw = off;       off = a256(off + sizeof(double) * (size_t)m * n);
  p->partials = off; off = a256(off + sizeof(double) * NN * (size_t)p->grid * p->groups);
  p->M = off;        off = a256(off + sizeof(double) * NN);
  p->Pk = off;       off = a256(off + sizeof(double) * pk_size(np));
  p->rk = off;       off = a256(off + sizeof(double) * pk_size(np));
  p->w = off;        off = a256(off + sizeof(double) * NN * 6);
  p->total = off;
  return SCQR3_OK;
}

void launch_reduce(cudaStream_t s, const double* partials, int n_partials, int stride, double* out,
                   const DevState* st, int pass);

template <int NP>
static void bw_rows_launch(const BwPlan& p, cudaStream_t s, int mode, int k, int64_t m, int n,
                           const double* q, int64_t ldq, const double* b, int64_t ldb, double* qw,
                           double* dx, int64_t lddx, const double* Pk, const double* rk,
                           double* partials) {
  bw_rows_kernel<NP><<<p.grid, kThreads, BwGeo<NP>::smem, s>>>(mode, k, m, n, q, ldq, b, ldb, qw, dx,
                                                               lddx, Pk, rk, partials);
}

static void bw_rows(const BwPlan& p, cudaStream_t s, int mode, int k, int64_t m, int n, const double* q,
                    int64_t ldq, const double* b, int64_t ldb, double* qw, double* dx, int64_t lddx,
                    const double* Pk, const double* rk, double* partials) {
  switch (p.np) {
    case 16: bw_rows_launch<16>(p, s, mode, k, m, n, q, ldq, b, ldb, qw, dx, lddx, Pk, rk, partials); break;
    case 32: bw_rows_launch<32>(p, s, mode, k, m, n, q, ldq, b, ldb, qw, dx, lddx, Pk, rk, partials); break;
    case 64: bw_rows_launch<64>(p, s, mode, k, m, n, q, ldq, b, ldb, qw, dx, lddx, Pk, rk, partials); break;
    default: bw_rows_launch<128>(p, s, mode, k, m, n, q, ldq, b, ldb, qw, dx, lddx, Pk, rk, partials); break;
  }
}

static void bw_small(int np, cudaStream_t s, int k, int P, int n, const double* Rpass, const double* dR,
                     const double* M, double* w, double* Pk, double* rk) {
  switch (np) {
    case 16: bw_small_kernel<16><<<1, 1024, 0, s>>>(k, P, n, Rpass, dR, M, w, Pk, rk); break;
    case 32: bw_small_kernel<32><<<1, 1024, 0, s>>>(k, P, n, Rpass, dR, M, w, Pk, rk); break;
    case 64: bw_small_kernel<64><<<1, 1024, 0, s>>>(k, P, n, Rpass, dR, M, w, Pk, rk); break;
    default: bw_small_kernel<128><<<1, 1024, 0, s>>>(k, P, n, Rpass, dR, M, w, Pk, rk); break;
  }
}

// -------------------------------------------------------------------------------------------
// The tensor-core form (opts.precision = SCQR3_PREC_TC): the same chain rule,
// with the row work run by the factorization's tensor-core kernels. The
// iterate of pass k is held as Z = [Q_k | Qbar_k J] (m x 2n, row-major; J
// reverses the order of the columns), and with t = Qbar_k + 2 Q_k P_k:
//  * t J = Qbar_k J - Q_k Bt with Bt = -2 P_k J: tc_update_kernel's x - Y B
//    with a dense B, each product exact to within 2^-56 of the scales of its
//    row and column (the digit split of the factorization's substitution);
//  * Qbar_{k-1} R_k^T = t is a back substitution; with U = J R_k^T J, upper
//    triangular with the entries of R_k, it reads (Qbar_{k-1} J) U = t J: the
//    row-wise substitution Q := X U^{-1} of Eq. (backward2) that the
//    factorization runs (FP64 diagonal blocks, off-diagonal products on the
//    tensor cores; one sweep for 16 < n <= 64), backward stable row by row;
//  * Q_{k-1} = Q_k R_k: x - Y B with x = 0 and B = -R_k;
//  * M_{k-1} J = Q_{k-1}^T (Qbar_{k-1} J) is the upper right block of the Gram
//    matrix of the new Z, which the tensor-core Gram forms (2n <= 256 columns).
// The n x n algebra is bw_small_kernel's. Pass k's kernels use pass slot 0 of
// their own DevState, with every solve enabled and no Gram fused into it.

void launch_pass(int np, int grid, cudaStream_t s, const double* src, int64_t lds, double* dst, int64_t ldd,
                 const Params& P, int pass, const double* rk, const double* lt, double* partials, int part_stride,
                 DevState* st);
int tc_grid(int64_t m, int np, int sms);
void launch_tc_split_r(cudaStream_t s, const double* rk, int np, int n, int w, int pass, const DevState* st,
                       double* rdiag);
void launch_tc_update(int sms, cudaStream_t s, int k, const double* y, int64_t ldy, const double* x1,
                      int64_t ldx, double* q1, int64_t ldq, int64_t m, int n1, int pass, const double* rk, int np,
                      int r0, int c0, int ldb, int ky, DevState* st, long long wait_ns);
void launch_tc_gram(int grid, int sms, cudaStream_t s, const double* src, int64_t lds, const Params& P, int pass,
                    unsigned long long* colmax, double* partials, int part_stride, DevState* st, int pairs,
                    const double* lt, int64_t blk0, int scan, int offd_only);
void launch_tc_fused(int sms, cudaStream_t s, const double* X, int64_t ldx, double* Q, int64_t ldq, const Params& P,
                     int pass, const double* rk, unsigned long long* colmax, DevState* st);
void set_options(Params* P, const scqr3_opts* opts);
bool tc_bwprod_supported(int n);
void launch_tc_bwprod(int sms, cudaStream_t s, double* z, double* zn, int64_t m, const double* bt,
                      const double* bq, int ldb, bool both, DevState* st, long long wait_ns);
int tc_kernels_ready(int* sms);
int pass_kernel_grid(int np, int64_t m);
bool fused_solve_selected(int n);

__global__ void bwt_init_kernel(DevState* st) {
  if (threadIdx.x != 0) return;
  st->status = SCQR3_OK;
  st->passes = 0;
  st->plain_in_a_row = 0;
  st->pad0 = 0;
  for (int i = 0; i < SCQR3_MAX_PASSES; ++i) {
    st->run_trsm[i] = 1;
    st->gram_after[i] = 0;
  }
  st->normb = 0.0;
  st->normb_bits_max = 0.0;
}

// mode 0: z = [a | b J] (a = Q, b = dQ); mode 1: dx = the right half of z in
// natural column order (dX = Qbar_0).
__global__ void bwt_pack_kernel(int mode, int64_t m, int n, const double* __restrict__ a, int64_t lda,
                                const double* b, int64_t ldb, double* z, double* dx, int64_t lddx) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n;
    const int c = (int)(e - i * n);
    double* zr = z + i * 2 * n;
    if (mode == 0) {
      zr[c] = a[i * lda + c];
      zr[2 * n - 1 - c] = b[i * ldb + c];
    } else {
      dx[i * lddx + c] = zr[2 * n - 1 - c];
    }
  }
}

// M (full np x np, zero padding) from the packed Gram matrix G (npz) of Z:
// M(r, j) = G(r, 2n - 1 - j).
__global__ void bwt_gram_to_m_kernel(const double* __restrict__ G, int npz, int n, int np, double* __restrict__ M) {
  for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
    const int r = e / np, j = e % np;
    M[e] = (r < n && j < n) ? G[pk_idx(npz, r, 2 * n - 1 - j)] : 0.0;
  }
}

// Pass k's matrices: Bt = -2 P_k J and Bq = -R_k (dense nb x nb, zero outside
// n x n; P_k packed np, symmetric) and U = J R_k^T J packed nps x nps, the
// identity in its padding: U(a, b) = R_k(n-1-b, n-1-a).
__global__ void bwt_mats_kernel(int k, int n, const double* __restrict__ Rpass, const double* __restrict__ Pk,
                                int np, int nb, double* __restrict__ Bt, double* __restrict__ Bq, int nps,
                                double* __restrict__ U) {
  const double* R = Rpass + (int64_t)(k - 1) * n * n;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int a = e / nb, b = e % nb;
    double t = 0.0, q = 0.0;
    if (a < n && b < n) {
      const int c = n - 1 - b;
      t = -2.0 * Pk[a <= c ? pk_idx(np, a, c) : pk_idx(np, c, a)];
      q = a <= b ? -R[a * n + b] : 0.0;
    }
    Bt[e] = t;
    Bq[e] = q;
  }
  for (int e = threadIdx.x; e < pk_size(nps); e += blockDim.x) {
    int a = 0;
    while (pk_row(nps, a + 1) <= e) ++a;
    const int b = a + (e - pk_row(nps, a));
    U[e] = b < n ? R[(n - 1 - b) * n + (n - 1 - a)] : (a == b ? 1.0 : 0.0);
  }
}

struct BwTcPlan {
  int np, nps, npz, nb, kw, sms, grid_g, stride_g;
  size_t st, z0, z1, partials, G, colmax, M, Pk, rk, w, Bt, Bq, U, tcr, total;
};

static int bwt_plan(int64_t m, int n, BwTcPlan* p) {
  p->np = bw_padded(n);
  if (!p->np || m > (int64_t)1 << 31) return SCQR3_E_UNSUPPORTED;  // n <= 128; the Gram's row limit
  if (tc_kernels_ready(&p->sms) != SCQR3_OK) return SCQR3_E_CUDA;
  p->nps = n <= 64 ? 64 : 128;
  p->npz = 2 * n <= 64 ? 64 : 2 * n <= 128 ? 128 : 256;
  p->nb = (n + 31) / 32 * 32;
  p->kw = n <= 16 ? 16 : 32;
  p->grid_g = tc_grid(m, p->npz, p->sms);
  p->stride_g = pk_size(p->npz) + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = a256(off + bytes);
    return o;
  };
  const size_t NN = (size_t)p->np * p->np;
  p->st = take(sizeof(DevState));
  p->z0 = take(sizeof(double) * (size_t)m * 2 * n);
  p->z1 = take(sizeof(double) * (size_t)m * 2 * n);
  p->partials = take(sizeof(double) * (size_t)p->grid_g * p->stride_g);
  p->G = take(sizeof(double) * p->stride_g);
  p->colmax = take(sizeof(unsigned long long) * 256);
  p->M = take(sizeof(double) * NN);
  p->Pk = take(sizeof(double) * pk_size(p->np));
  p->rk = take(sizeof(double) * pk_size(p->np));
  p->w = take(sizeof(double) * NN * 6);
  p->Bt = take(sizeof(double) * p->nb * p->nb);
  p->Bq = take(sizeof(double) * p->nb * p->nb);
  p->U = take(sizeof(double) * pk_size(p->nps));
  p->tcr = take(sizeof(double) * 8 * pk_size(32));
  p->total = off;
  return SCQR3_OK;
}

static Params bwt_params(int64_t m, int n, int np) {
  Params P{};
  P.m = m;
  P.n = n;
  P.np = np;
  P.max_passes = SCQR3_MAX_PASSES;
  P.tc = 1;
  P.solve_only = 1;
  set_options(&P, nullptr);
  return P;
}

// (Y J) U = T J row by row: src = T J, dst = Y J (Eq. (backward2) with U).
static void bwt_substitute(const BwTcPlan& p, cudaStream_t s, const Params& Ps, const double* src, int64_t lds,
                           double* dst, int64_t ldd, const double* U, double* tcr, double* partials, DevState* st) {
  const int n = Ps.n;
  if (fused_solve_selected(n)) {
    launch_tc_fused(p.sms, s, src, lds, dst, ldd, Ps, 0, U, nullptr, st);
    return;
  }
  const int w = n <= 64 ? 16 : 32, nblk = (n + w - 1) / w;
  launch_tc_split_r(s, U, p.nps, n, w, 0, st, tcr);
  for (int J = 0; J < nblk; ++J) {
    const int wj = n - w * J < w ? n - w * J : w;
    const int npj = wj <= 16 ? 16 : 32;
    Params PJ = Ps;
    PJ.n = wj;
    PJ.np = npj;
    const double* in = J == 0 ? src : dst + w * J;
    const int64_t ldin = J == 0 ? lds : ldd;
    launch_pass(npj, pass_kernel_grid(npj, Ps.m), s, in, ldin, dst + w * J, ldd, PJ, 0, tcr + J * pk_size(32),
                nullptr, partials, p.stride_g, st);
    for (int c0 = w * (J + 1); c0 < n; c0 += 32) {
      const int n1 = n - c0 < 32 ? n - c0 : 32;
      const double* x1 = J == 0 ? src + c0 : dst + c0;
      const int64_t ldx1 = J == 0 ? lds : ldd;
      launch_tc_update(p.sms, s, w, dst + w * J, ldd, x1, ldx1, dst + c0, ldd, Ps.m, n1, 0, U, p.nps, w * J, c0, 0,
                       w, st, Ps.wait_ns);
    }
  }
}

static void bwt_run(const BwTcPlan& p, cudaStream_t s, const double* Q, int64_t m, int n, int64_t ldq,
                    const double* Rpass, int passes, const double* dQ, int64_t lddq, const double* dR, double* dX,
                    int64_t lddx, char* ws, int* status) {
  DevState* st = (DevState*)(ws + p.st);
  double* Z[2] = {(double*)(ws + p.z0), (double*)(ws + p.z1)};
  double* partials = (double*)(ws + p.partials);
  double* G = (double*)(ws + p.G);
  unsigned long long* colmax = (unsigned long long*)(ws + p.colmax);
  double* M = (double*)(ws + p.M);
  double* Pk = (double*)(ws + p.Pk);
  double* rk = (double*)(ws + p.rk);
  double* w = (double*)(ws + p.w);
  double* Bt = (double*)(ws + p.Bt);
  double* Bq = (double*)(ws + p.Bq);
  double* U = (double*)(ws + p.U);
  double* tcr = (double*)(ws + p.tcr);
  const int64_t ldz = 2 * (int64_t)n;
  const Params Pg = bwt_params(m, 2 * n, p.npz);
  const Params Ps = bwt_params(m, n, p.nps);
  const int pg = p.sms * 8;
  // G = Z^T Z (packed npz) through the partial slots. The columns of Q_k fill
  // whole 64-column blocks of Z when 64 divides n: then M J lies in the
  // off-diagonal blocks alone, and only those are formed.
  const int offd_only = n % 64 == 0 ? 1 : 0;
  auto gram = [&](const double* z) {
    launch_tc_gram(p.grid_g, p.sms, s, z, ldz, Pg, -1, colmax, partials, p.stride_g, st, 0, nullptr, 0, 1,
                   offd_only);
    launch_reduce(s, partials, p.grid_g, p.stride_g, G, nullptr, -1);
  };
  bwt_init_kernel<<<1, 32, 0, s>>>(st);
  bwt_pack_kernel<<<pg, 256, 0, s>>>(0, m, n, Q, ldq, dQ, lddq, Z[0], nullptr, 0);
  gram(Z[0]);
  int cur = 0;
  for (int k = passes; k >= 1; --k) {
    double* A = Z[cur];
    double* B = Z[cur ^ 1];
    bwt_gram_to_m_kernel<<<1, 1024, 0, s>>>(G, p.npz, n, p.np, M);
    bw_small(p.np, s, k, passes, n, Rpass, dR, M, w, Pk, rk);
    bwt_mats_kernel<<<1, 1024, 0, s>>>(k, n, Rpass, Pk, p.np, p.nb, Bt, Bq, p.nps, U);
    if (tc_bwprod_supported(n)) {
      // both products from one cut of Q_k: t J in place, Q_{k-1} into the left half of B
      launch_tc_bwprod(p.sms, s, A, B, m, Bt, Bq, p.nb, k > 1, st, Ps.wait_ns);
    } else {
      // t J = Qbar_k J - Q_k Bt, in place in the right half of A
      for (int J = 0; J * p.kw < n; ++J) {
        const int ky = n - J * p.kw < p.kw ? n - J * p.kw : p.kw;
        for (int c0 = 0; c0 < n; c0 += 32) {
          const int n1 = n - c0 < 32 ? n - c0 : 32;
          launch_tc_update(p.sms, s, p.kw, A + J * p.kw, ldz, A + n + c0, ldz, A + n + c0, ldz, m, n1, 0, Bt, 0,
                           J * p.kw, c0, p.nb, ky, st, Ps.wait_ns);
        }
      }
      // Q_{k-1} = Q_k R_k into the left half of B (rows of R_k up to the block's last column)
      if (k > 1) {
        for (int c0 = 0; c0 < n; c0 += 32) {
          const int n1 = n - c0 < 32 ? n - c0 : 32;
          for (int J = 0; J * p.kw < c0 + n1; ++J) {
            const int ky = n - J * p.kw < p.kw ? n - J * p.kw : p.kw;
            launch_tc_update(p.sms, s, p.kw, A + J * p.kw, ldz, J == 0 ? nullptr : B + c0, ldz, B + c0, ldz, m, n1,
                             0, Bq, 0, J * p.kw, c0, p.nb, ky, st, Ps.wait_ns);
          }
        }
      }
    }
    // Qbar_{k-1} J = (t J) U^{-1} into the right half of B
    bwt_substitute(p, s, Ps, A + n, ldz, B + n, ldz, U, tcr, partials, st);
    if (k > 1) gram(B);
    cur ^= 1;
  }
  bwt_pack_kernel<<<pg, 256, 0, s>>>(1, m, n, nullptr, 0, nullptr, 0, Z[cur], dX, lddx);
  if (status) cudaMemcpyAsync(status, &st->status, sizeof(int), cudaMemcpyDeviceToDevice, s);
}

}  // namespace scqr3

using namespace scqr3;

extern "C" int scqr3_backward_workspace_bytes(int64_t m, int n, size_t* bytes) {
  if (!bytes) return -3;
  if (n < 1) return -2;
  if (m < n) return -1;
  BwPlan p;
  const int r = bw_plan(m, n, &p);
  if (r != SCQR3_OK) return r;
  *bytes = p.total;
  return SCQR3_OK;
}

static int bw_args(const double* Q, int64_t m, int n, int64_t ldq, const double* Rpass, int passes,
                   const double* dQ, int64_t lddq, const double* dX, int64_t lddx, const void* workspace) {
  if (!Q) return -1;
  if (m < n || m < 1) return -2;
  if (n < 1) return -3;
  if (ldq < n) return -4;
  if (!Rpass) return -5;
  if (passes < 1 || passes > SCQR3_MAX_PASSES) return -6;
  if (!dQ) return -7;
  if (lddq < n) return -8;
  if (!dX) return -10;
  if (lddx < n) return -11;
  if (!workspace || ((uintptr_t)workspace & 255) != 0) return SCQR3_E_WORKSPACE;
  return SCQR3_OK;
}

extern "C" int scqr3_backward(const double* Q, int64_t m, int n, int64_t ldq, const double* Rpass,
                              int passes, const double* dQ, int64_t lddq, const double* dR, double* dX,
                              int64_t lddx, void* workspace, size_t workspace_bytes, void* stream) {
  const int a = bw_args(Q, m, n, ldq, Rpass, passes, dQ, lddq, dX, lddx, workspace);
  if (a != SCQR3_OK) return a;
  BwPlan p;
  const int r = bw_plan(m, n, &p);
  if (r != SCQR3_OK) return r;
  if (workspace_bytes < p.total) return SCQR3_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  double* qw = (double*)(ws + p.qw);
  double* partials = (double*)(ws + p.partials);
  double* M = (double*)(ws + p.M);
  double* Pk = (double*)(ws + p.Pk);
  double* rk = (double*)(ws + p.rk);
  double* w = (double*)(ws + p.w);
  const int NN = p.np * p.np;
  const int nparts = p.grid * p.groups;

  // M_P = Q^T dQ ; Qw := Q, dX := dQ
  bw_rows(p, s, BW_FIRST, passes + 1, m, n, Q, ldq, dQ, lddq, qw, dX, lddx, nullptr, nullptr, partials);
  launch_reduce(s, partials, nparts, NN, M, nullptr, -1);
  for (int k = passes; k >= 1; --k) {
    bw_small(p.np, s, k, passes, n, Rpass, dR, M, w, Pk, rk);
    bw_rows(p, s, BW_PASS, k, m, n, nullptr, 0, nullptr, 0, qw, dX, lddx, Pk, rk, partials);
    if (k > 1) launch_reduce(s, partials, nparts, NN, M, nullptr, -1);
  }
  if (cudaGetLastError() != cudaSuccess) return SCQR3_E_CUDA;
  return SCQR3_OK;
}

extern "C" int scqr3_backward_workspace_bytes_ex(int64_t m, int n, const scqr3_opts* opts, size_t* bytes) {
  if (!bytes) return -4;
  if (n < 1) return -2;
  if (m < n) return -1;
  const int prec = opts ? opts->precision : SCQR3_PREC_FP64;
  if (prec == SCQR3_PREC_FP64) return scqr3_backward_workspace_bytes(m, n, bytes);
  if (prec != SCQR3_PREC_TC) return SCQR3_E_UNSUPPORTED;
  BwTcPlan p;
  const int r = bwt_plan(m, n, &p);
  if (r != SCQR3_OK) return r;
  *bytes = p.total;
  return SCQR3_OK;
}

extern "C" int scqr3_backward_ex(const double* Q, int64_t m, int n, int64_t ldq, const double* Rpass, int passes,
                                 const double* dQ, int64_t lddq, const double* dR, double* dX, int64_t lddx,
                                 const scqr3_opts* opts, void* workspace, size_t workspace_bytes, int* status,
                                 void* stream) {
  const int prec = opts ? opts->precision : SCQR3_PREC_FP64;
  if (prec != SCQR3_PREC_FP64 && prec != SCQR3_PREC_TC) return SCQR3_E_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == SCQR3_PREC_FP64) {
    const int r = scqr3_backward(Q, m, n, ldq, Rpass, passes, dQ, lddq, dR, dX, lddx, workspace, workspace_bytes,
                                 stream);
    if (r == SCQR3_OK && status && cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return SCQR3_E_CUDA;
    return r;
  }
  const int a = bw_args(Q, m, n, ldq, Rpass, passes, dQ, lddq, dX, lddx, workspace);
  if (a != SCQR3_OK) return a;
  BwTcPlan p;
  const int r = bwt_plan(m, n, &p);
  if (r != SCQR3_OK) return r;
  if (workspace_bytes < p.total) return SCQR3_E_WORKSPACE;
  bwt_run(p, s, Q, m, n, ldq, Rpass, passes, dQ, lddq, dR, dX, lddx, (char*)workspace, status);
  if (cudaGetLastError() != cudaSuccess) return SCQR3_E_CUDA;
  return SCQR3_OK;
}
