// csr.cu -- the oblique Gram matrix A = Q^T (B Q) for a sparse SPD B in CSR
// form (Alg. 4 / Alg. 5 with the sparse product of Sec. 7.2).
//
// Sec. 7.2 forms Y := B Q with a sparse product and then Q^T Y. Row i of Y
// needs the rows of Q that row i of B names, which lie outside the row panel
// being solved, so the product cannot be fused into the solve of the same
// pass: with a CSR B the pass kernel only solves (Params::csr), and
// csr_gram_kernel then sweeps Q once. Per panel of PR rows it stages Q(panel)
// in shared memory, forms Y(panel) = B(panel, :) Q by gathering the named rows
// (mostly L2 hits for banded B: a Laplacian reaches +-1, +-nx, +-nx*ny rows),
// and accumulates the panel's share of Q^T Y.
//
// Gram layout (cyclic): each group of NP threads owns every entry once;
// thread j holds the pairs {j, (j + d) mod NP}, d = 0 .. NP/2, accumulating
// q_j * y_{(j+d) mod NP}. For j + d < NP that is (Q^T Y)_{j, j+d}, an
// upper-triangle entry. For j + d >= NP it is (Q^T Y)_{j, k}, k = j + d - NP
// < j, which equals (Q^T Y)_{k, j} in exact arithmetic (Q^T B Q is symmetric)
// and is used for that entry. Y is stored twice per row ([y | y]) so every
// thread reads y at j + d without a wrap test: one shared load per FMA. At
// d = NP/2 the threads j and j + NP/2 reach the same pair; the lower keeps it.
//
// csr_check_kernel validates the CSR arrays on the device (no access outside
// them ever happens: csr_gram_kernel clamps every range and index it reads)
// and computes the bound max_i sum_j |b_ij| >= ||B||_2 for Eq. (finds2B).
#include "fp64_device.cuh"

namespace scqr3 {

template <int NP>
struct CsrGeo {
  static constexpr int PR = 4096 / NP;     // rows per panel
  static constexpr int G = kThreads / NP;  // groups of NP threads, each a partial slot
  static constexpr int C = NP / 2 + 1;     // accumulators per thread
  static constexpr int LDY = 2 * NP;       // [y | y]
  static constexpr int CPL = NP < 32 ? 1 : NP / 32;  // Y columns per lane
  static constexpr size_t smem = sizeof(double) * ((size_t)PR * NP + (size_t)PR * LDY + kThreads / 32);
  static constexpr int MINB = NP == 128 ? 1 : 2;  // 65 accumulators need > 128 registers
};

template <int NP>
__global__ void __launch_bounds__(kThreads, CsrGeo<NP>::MINB)
csr_gram_kernel(const double* src, int64_t lds, Params P, int pass, const int64_t* __restrict__ row_ptr,
                const int32_t* __restrict__ col_idx, const double* __restrict__ vals, int64_t nnz,
                double* __restrict__ partials, int part_stride, const DevState* __restrict__ st) {
  using g = CsrGeo<NP>;
  if (pass >= 0 && !(st->run_trsm[pass] && st->gram_after[pass])) return;
  extern __shared__ __align__(16) double sm[];
  double* sq = sm;                     // PR x NP: Q(panel), zero padded
  double* sy = sq + g::PR * NP;        // PR x LDY: [Y(panel) | Y(panel)]
  double* red = sy + g::PR * g::LDY;   // per-warp sums of squares
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid / NP, j = tid % NP;
  const int n = P.n;
  const int64_t m = P.m;

  double acc[g::C];
#pragma unroll
  for (int d = 0; d < g::C; ++d) acc[d] = 0.0;
  double f2 = 0.0;

  const int64_t npanels = (m + g::PR - 1) / g::PR;
  for (int64_t pnl = blockIdx.x; pnl < npanels; pnl += gridDim.x) {
    const int64_t row0 = pnl * g::PR;
    const int rows = (int)((m - row0) < (int64_t)g::PR ? (m - row0) : (int64_t)g::PR);
    __syncthreads();  // the previous panel is consumed
    for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
      const int r = idx / NP, c = idx % NP;
      double v = 0.0;
      if (r < rows && c < n) v = src[(row0 + r) * lds + c];
      sq[idx] = v;
      f2 = fma(v, v, f2);
    }
    // Y(panel) = B(panel, :) Q: one warp per row, lanes across the columns,
    // stored entries in storage order.
    for (int r = warp; r < g::PR; r += kThreads / 32) {
      double y[g::CPL];
#pragma unroll
      for (int t = 0; t < g::CPL; ++t) y[t] = 0.0;
      if (r < rows) {
        const int64_t i = row0 + r;
        int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
        p0 = p0 < 0 ? 0 : p0;
        p1 = p1 > nnz ? nnz : p1;
#pragma unroll 4
        for (int64_t p = p0; p < p1; ++p) {
          const int64_t c = col_idx[p];
          if (c < 0 || c >= m) continue;  // reported by csr_check_kernel
          const double v = vals[p];
          const double* qc = src + c * lds;
#pragma unroll
          for (int t = 0; t < g::CPL; ++t) {
            const int col = lane + 32 * t;
            if (col < n) y[t] = fma(v, qc[col], y[t]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < g::CPL; ++t) {
        const int col = lane + 32 * t;
        if (col < NP) {
          sy[r * g::LDY + col] = y[t];
          sy[r * g::LDY + NP + col] = y[t];
        }
      }
    }
    __syncthreads();
    for (int r = grp; r < rows; r += g::G) {
      const double qj = sq[r * NP + j];
      const double* yr = sy + r * g::LDY + j;
#pragma unroll
      for (int d = 0; d < g::C; ++d) acc[d] = fma(qj, yr[d], acc[d]);
    }
  }

  double* mine = partials + ((int64_t)blockIdx.x * g::G + grp) * part_stride;
#pragma unroll
  for (int d = 0; d < g::C; ++d) {
    if (d == NP / 2 && j >= NP / 2) continue;
    const int k = j + d;
    mine[k < NP ? pk_idx(NP, j, k) : pk_idx(NP, k - NP, j)] = acc[d];
  }
  // ||Q||_F^2 of the rows this CTA saw, in group 0's slot (the others get 0).
  for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
  if (lane == 0) red[warp] = f2;
  __syncthreads();
  if (tid < g::G) {
    double t = 0.0;
    if (tid == 0)
      for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    partials[((int64_t)blockIdx.x * g::G + tid) * part_stride + pk_size(NP)] = t;
  }
}

// Validation of the CSR arrays and the bound max_i sum_j |b_ij| of ||B||_2.
__global__ void __launch_bounds__(256)
csr_check_kernel(int64_t m, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                 const double* __restrict__ vals, int64_t nnz, DevState* __restrict__ st) {
  __shared__ double wmax[8];
  __shared__ int bad_sh;
  if (threadIdx.x == 0) bad_sh = 0;
  __syncthreads();
  double best = 0.0;
  int bad = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && row_ptr[0] != 0) bad = 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
    if (p0 < 0 || p1 < p0 || p1 > nnz) {
      bad = 1;
      continue;
    }
    double r = 0.0;
    bool diag = false;
    for (int64_t p = p0; p < p1; ++p) {
      const int64_t c = col_idx[p];
      const double v = vals[p];
      if (c < 0 || c >= m || !isfinite(v)) bad = 1;
      if (c == i && v > 0.0) diag = true;
      r += fabs(v);
    }
    if (!diag) bad = 1;
    best = fmax(best, r);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  if (bad) bad_sh = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, wmax[w]);
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long*)&st->normb_bits_max, (unsigned long long)__double_as_longlong(b));
    if (bad_sh) atomicCAS(&st->status, SCQR3_OK, SCQR3_E_B_INVALID);
  }
}

// ---- host side ----------------------------------------------------------------------------

template <int NP>
static cudaError_t csr_setup_one(int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(csr_gram_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)CsrGeo<NP>::smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, csr_gram_kernel<NP>, kThreads,
                                                       CsrGeo<NP>::smem);
}

// Resident CTAs per SM of csr_gram_kernel for the padded sizes 16, 32, 64, 128.
cudaError_t csr_setup(int per_sm[4]) {
  cudaError_t e;
  if ((e = csr_setup_one<16>(&per_sm[0])) != cudaSuccess) return e;
  if ((e = csr_setup_one<32>(&per_sm[1])) != cudaSuccess) return e;
  if ((e = csr_setup_one<64>(&per_sm[2])) != cudaSuccess) return e;
  return csr_setup_one<128>(&per_sm[3]);
}

int csr_rows_per_panel(int np) { return 4096 / np; }
int csr_groups(int np) { return kThreads / np; }

void launch_csr_check(int grid, cudaStream_t s, int64_t m, const scqr3_B* B, DevState* st) {
  csr_check_kernel<<<grid, 256, 0, s>>>(m, B->row_ptr, B->col_idx, B->vals, B->nnz, st);
}

void launch_csr_gram(int np, int grid, cudaStream_t s, const double* src, int64_t lds, const Params& P,
                     int pass, const scqr3_B* B, double* partials, int part_stride, const DevState* st) {
  switch (np) {
#define SCQR3_CSR(NPV)                                                                                \
  case NPV:                                                                                           \
    csr_gram_kernel<NPV><<<grid, kThreads, CsrGeo<NPV>::smem, s>>>(                                   \
        src, lds, P, pass, B->row_ptr, B->col_idx, B->vals, B->nnz, partials, part_stride, st);       \
    break;
    SCQR3_CSR(16)
    SCQR3_CSR(32)
    SCQR3_CSR(64)
    SCQR3_CSR(128)
#undef SCQR3_CSR
    default: break;
  }
}

}  // namespace scqr3
