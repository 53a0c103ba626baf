// n256.cu -- FP64 kernels for 128 < n <= 256 (padded size 256).
//
// At this width neither R_k (263 KB packed) nor the n(n+1)/2 = 32,896 Gram
// accumulators fit in one CTA, so the pass is split in two kernels:
//
//   trsm256_kernel  the substitution Q_k = Q_{k-1} R_k^{-1} (Eq. backward2),
//                   one row per thread over panels of 256 rows, in 64-column
//                   blocks J: the block's 64 entries of t live in registers
//                   and take t -= q_i R_k(i, J) for every solved q_i of the
//                   earlier blocks (restaged from L2 through shared memory,
//                   with the 64 x 64 block of R_k beside it), then the 64 x 64
//                   diagonal block is solved in the staging row in shared
//                   memory. Summation order per entry is ascending i, as in the
//                   row-wise substitution.
//   gram256_kernel  Q_k^T Q_k: the folded upper triangle split between two
//                   CTA roles (each owns 64 of the 128 folded row pairs, 65
//                   accumulators per thread), each role reading every panel.
//
// The shift / Cholesky step runs on workspace buffers in global memory (L2)
// instead of shared memory.
#include "fp64_device.cuh"

namespace scqr3 {

constexpr int N256 = 256;
constexpr int T_PR = 256;         // rows per substitution panel
constexpr int T_BW = 64;          // column block
constexpr int T_LD = T_BW + 1;    // staging row stride (odd: conflict-free)
constexpr int G_PR = 64;          // rows per Gram panel
constexpr int G_LD = N256 + 1;
constexpr int G_C = 65;           // accumulators per thread (257 / 4, rounded up)
constexpr size_t TRSM256_SMEM = sizeof(double) * ((size_t)T_PR * T_LD + 2 * T_BW * T_BW + T_BW);
constexpr size_t GRAM256_SMEM = sizeof(double) * ((size_t)G_PR * G_LD + kThreads / 32);

__device__ __forceinline__ double r256(const double* rk, int i, int j) {
  return j >= i ? rk[pk_idx(N256, i, j)] : 0.0;
}

__global__ void __launch_bounds__(kThreads, 1)
trsm256_kernel(const double* src, int64_t lds, double* dst, int64_t ldd, Params P, int pass,
               const double* __restrict__ rk, const DevState* __restrict__ st) {
  if (!st->run_trsm[pass]) return;
  extern __shared__ __align__(16) double sm[];
  double* stage = sm;                       // T_PR x T_LD
  double* Rb = stage + T_PR * T_LD;         // 64 x 64, off-diagonal block R_k(I, J)
  double* Rd = Rb + T_BW * T_BW;            // 64 x 64, diagonal block R_k(J, J)
  double* rinv = Rd + T_BW * T_BW;          // 1 / r_jj of block J
  const int tid = threadIdx.x;
  const int n = P.n;
  const int64_t m = P.m;
  const int nbJ = (n + T_BW - 1) / T_BW;
  const int64_t npanels = (m + T_PR - 1) / T_PR;

  for (int64_t pnl = blockIdx.x; pnl < npanels; pnl += gridDim.x) {
    const int64_t row0 = pnl * T_PR;
    const int rows = (int)((m - row0) < (int64_t)T_PR ? (m - row0) : (int64_t)T_PR);
    for (int J = 0; J < nbJ; ++J) {
      const int c0 = J * T_BW;
      __syncthreads();
      for (int idx = tid; idx < T_PR * T_BW; idx += kThreads) {
        const int r = idx / T_BW, c = idx % T_BW;
        double v = 0.0;
        if (r < rows && c0 + c < n) v = src[(row0 + r) * lds + c0 + c];
        stage[r * T_LD + c] = v;
      }
      for (int idx = tid; idx < T_BW * T_BW; idx += kThreads) {
        const int i = idx / T_BW, c = idx % T_BW;
        Rd[idx] = r256(rk, c0 + i, c0 + c);
      }
      if (tid < T_BW) rinv[tid] = 1.0 / rk[pk_row(N256, c0 + tid)];
      __syncthreads();
      double t[T_BW];
#pragma unroll
      for (int c = 0; c < T_BW; ++c) t[c] = stage[tid * T_LD + c];
      for (int I = 0; I < J; ++I) {
        const int i0 = I * T_BW;
        __syncthreads();
        for (int idx = tid; idx < T_PR * T_BW; idx += kThreads) {
          const int r = idx / T_BW, c = idx % T_BW;
          stage[r * T_LD + c] = (r < rows) ? dst[(row0 + r) * ldd + i0 + c] : 0.0;
        }
        for (int idx = tid; idx < T_BW * T_BW; idx += kThreads) {
          const int i = idx / T_BW, c = idx % T_BW;
          Rb[idx] = r256(rk, i0 + i, c0 + c);
        }
        __syncthreads();
        for (int i = 0; i < T_BW; ++i) {
          const double q = stage[tid * T_LD + i];
          const double* ri = Rb + i * T_BW;
#pragma unroll
          for (int c = 0; c < T_BW; ++c) t[c] = fma(-q, ri[c], t[c]);
        }
      }
      // diagonal block: 6% of the work, solved in the staging row (rolled loops
      // keep t out of local memory)
      __syncthreads();
#pragma unroll
      for (int c = 0; c < T_BW; ++c) stage[tid * T_LD + c] = t[c];
      {
        double* row = stage + tid * T_LD;
        for (int c = 0; c < T_BW; ++c) {
          const double q = row[c] * rinv[c];
          row[c] = q;
          const double* rc = Rd + c * T_BW;
#pragma unroll 4
          for (int c2 = c + 1; c2 < T_BW; ++c2) row[c2] = fma(-q, rc[c2], row[c2]);
        }
      }
      __syncthreads();
      for (int idx = tid; idx < T_PR * T_BW; idx += kThreads) {
        const int r = idx / T_BW, c = idx % T_BW;
        if (r < rows && c0 + c < n) dst[(row0 + r) * ldd + c0 + c] = stage[r * T_LD + c];
      }
    }
  }
}

// Gram of the rows (pass < 0: X; else the Q written by pass `pass`), if needed.
__global__ void __launch_bounds__(kThreads, 1)
gram256_kernel(const double* src, int64_t lds, Params P, int pass, double* __restrict__ partials,
               int part_stride, const DevState* __restrict__ st) {
  if (pass >= 0 && !(st->run_trsm[pass] && st->gram_after[pass])) return;
  extern __shared__ __align__(16) double sm[];
  double* panel = sm;  // G_PR x G_LD, column N256 stays 0
  const int tid = threadIdx.x;
  const int n = P.n;
  const int64_t m = P.m;
  const int role = blockIdx.x & 1;
  const int nrole = gridDim.x / 2;
  const int me = blockIdx.x >> 1;
  const int pidx = 64 * role + (tid % 64);
  const int h = tid / 64;
  for (int r = tid; r < G_PR; r += kThreads) panel[r * G_LD + N256] = 0.0;
  double acc[G_C];
#pragma unroll
  for (int l = 0; l < G_C; ++l) acc[l] = 0.0;
  const int64_t npanels = (m + G_PR - 1) / G_PR;
  for (int64_t pnl = me; pnl < npanels; pnl += nrole) {
    const int64_t row0 = pnl * G_PR;
    const int rows = (int)((m - row0) < (int64_t)G_PR ? (m - row0) : (int64_t)G_PR);
    __syncthreads();
    for (int idx = tid; idx < G_PR * N256; idx += kThreads) {
      const int r = idx / N256, c = idx % N256;
      double v = 0.0;
      if (r < rows && c < n) v = src[(row0 + r) * lds + c];
      panel[r * G_LD + c] = v;
    }
    __syncthreads();
    for (int r = 0; r < rows; ++r) {
      const double* row = panel + r * G_LD;
      const double a = row[pidx], b = row[N256 - 1 - pidx];
#pragma unroll
      for (int l = 0; l < G_C; ++l) {
        const int L = h * G_C + l;
        const bool seg_a = L < N256 - pidx;
        int col = seg_a ? pidx + L : L - 1;
        col = col > N256 ? N256 : col;  // slots past the pair read the zero column
        acc[l] = fma(seg_a ? a : b, row[col], acc[l]);
      }
    }
  }
  double* part = partials + (int64_t)blockIdx.x * part_stride;
  // this CTA owns folded pairs [64 role, 64 role + 64); zero the other role's entries
  for (int e = tid; e < pk_size(N256); e += kThreads) {
    int j = 0;
    while (pk_row(N256, j + 1) <= e) ++j;
    const int pj = j < N256 / 2 ? j : N256 - 1 - j;
    if (pj / 64 != role) part[e] = 0.0;
  }
#pragma unroll
  for (int l = 0; l < G_C; ++l) {
    const int L = h * G_C + l;
    if (L > N256) continue;
    const bool seg_a = L < N256 - pidx;
    const int j = seg_a ? pidx : N256 - 1 - pidx;
    const int k = seg_a ? pidx + L : L - 1;
    part[pk_idx(N256, j, k)] = acc[l];
  }
  if (tid == 0) part[pk_size(N256)] = 0.0;
}

__global__ void __launch_bounds__(512, 1)
chol256_kernel(Params P, int pass, const double* __restrict__ gram, double* __restrict__ rstack,
               double* __restrict__ racc, double* __restrict__ Rout, double* __restrict__ Rpass,
               DevState* __restrict__ st, scqr3_info* __restrict__ info, double* __restrict__ S,
               double* __restrict__ Ra) {
  chol_body<N256>(P, pass, gram, rstack, racc, Rout, Rpass, st, info, S, Ra);
}

// ---- host side ----------------------------------------------------------------------------

cudaError_t n256_setup(int* trsm_per_sm, int* gram_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(trsm256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TRSM256_SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gram256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAM256_SMEM);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(trsm_per_sm, trsm256_kernel, kThreads, TRSM256_SMEM);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(gram_per_sm, gram256_kernel, kThreads, GRAM256_SMEM);
}

void launch_trsm256(int grid, cudaStream_t s, const double* src, int64_t lds, double* dst, int64_t ldd,
                    const Params& P, int pass, const double* rk, const DevState* st) {
  trsm256_kernel<<<grid, kThreads, TRSM256_SMEM, s>>>(src, lds, dst, ldd, P, pass, rk, st);
}

void launch_gram256(int grid, cudaStream_t s, const double* src, int64_t lds, const Params& P, int pass,
                    double* partials, int part_stride, const DevState* st) {
  gram256_kernel<<<grid, kThreads, GRAM256_SMEM, s>>>(src, lds, P, pass, partials, part_stride, st);
}

void launch_chol256(cudaStream_t s, const Params& P, int pass, const double* gram, double* rstack,
                    double* racc, double* Rout, double* Rpass, DevState* st, scqr3_info* info, double* S,
                    double* Ra) {
  chol256_kernel<<<1, 512, 0, s>>>(P, pass, gram, rstack, racc, Rout, Rpass, st, info, S, Ra);
}

int n256_rows_per_gram_panel() { return G_PR; }
int n256_rows_per_trsm_panel() { return T_PR; }

}  // namespace scqr3
