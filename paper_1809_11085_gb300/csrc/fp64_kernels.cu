// fp64_kernels.cu -- FP64 kernels of shifted CholeskyQR3 for sm_103a.
//
// On GB300 the FP64 pipe retires 2 DFMA per clock per SM (about 1.2 TFLOP/s
// for the chip), 1/62 of the FP32 rate, while a pass over X moves only 8
// bytes per n(n+1) flops. Every kernel here is therefore built around one
// goal: issue no FP64 instruction that the method does not need, from warps
// whose 32 lanes all do useful work. Loads, index arithmetic and shared
// memory traffic are nearly free next to that.
//
//   pass_kernel   one streaming pass over the rows: the substitution
//                 Q_k = Q_{k-1} R_k^{-1} of pass k (Alg. 3) and,
//                 fused with it, the Gram matrix Q_k^T Q_k of pass k+1
//                 (or Q_k^T B Q_k, Alg. 5), as per-CTA partial sums.
//   reduce_kernel fixed-order sum of the partial Gram matrices.
//   chol_kernel   one CTA: the shift of Eq. (finds2)/(finds2B), the
//                 Cholesky factor R_k, the product R := R_k R, and the pass
//                 bookkeeping of Alg. 2 / Alg. 3, all on the device so that
//                 a whole factorization is one asynchronous launch sequence.
//   bfactor_kernel  per-block Cholesky B_j = L_j L_j^T of the oblique B.
#include "fp64_device.cuh"

namespace scqr3 {

template <int NP>
__global__ void __launch_bounds__(kThreads, Cfg<NP>::MINB)
pass_kernel(const double* src, int64_t lds, double* dst, int64_t ldd, Params P, int pass,
            const double* __restrict__ rk, const double* __restrict__ lt,
            double* __restrict__ partials, int part_stride, DevState* __restrict__ st) {
  using g = Geo<NP>;
  const int64_t npanels = (P.m + g::PR - 1) / g::PR;
  pass_segment<NP>(src, lds, dst, ldd, P, pass, rk, lt,
                   partials + (int64_t)blockIdx.x * g::G * part_stride, part_stride, st, blockIdx.x,
                   npanels, gridDim.x);
}

// -------------------------------------------------------------------------------------------
// Fixed-order sum of the partial Gram matrices: entry e of A is the sum of
// slot 0, 1, 2, ... in that order, so A is bitwise reproducible for a given
// grid.
__global__ void reduce_kernel(const double* __restrict__ partials, int n_partials, int stride,
                              double* __restrict__ out, const DevState* __restrict__ st, int pass) {
  if (pass >= 0 && !st->gram_after[pass]) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= stride) return;
  double s = 0.0;
  for (int p = 0; p < n_partials; ++p) s += partials[(int64_t)p * stride + e];
  out[e] = s;
}

template <int NP>
__global__ void __launch_bounds__(512, 1)
chol_kernel(Params P, int pass, const double* __restrict__ gram, double* __restrict__ rstack,
            double* __restrict__ racc, double* __restrict__ Rout, double* __restrict__ Rpass,
            DevState* __restrict__ st, scqr3_info* __restrict__ info) {
  extern __shared__ __align__(16) double sm[];
  chol_body<NP>(P, pass, gram, rstack, racc, Rout, Rpass, st, info, sm, sm + pk_size(NP));
}

// A failure recorded in the device state by a kernel that runs after the last
// Cholesky (a tensor-core wait that ran out) reaches the call's record.
__global__ void status_kernel(const DevState* __restrict__ st, scqr3_info* __restrict__ info) {
  if (threadIdx.x == 0 && st->status != SCQR3_OK && info->status == SCQR3_OK) info->status = st->status;
}

// -------------------------------------------------------------------------------------------
// B_j = L_j L_j^T for every diagonal block; stores L_j^T packed (upper, row-
// major) and the max over j of ||B_j||_F (for ||B||_2 in Eq. finds2B).
template <int BS>
__global__ void bfactor_kernel(const double* __restrict__ B, int64_t nblk, double* __restrict__ lt,
                               DevState* __restrict__ st) {
  constexpr int BSP = BS * (BS + 1) / 2;
  double fmax = 0.0;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
       b += (int64_t)gridDim.x * blockDim.x) {
    const double* Bb = B + b * BS * BS;
    double L[BS][BS];
    double f = 0.0;
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
      for (int k = 0; k < BS; ++k) {
        const double v = Bb[i * BS + k];
        f = fma(v, v, f);
        L[i][k] = v;
      }
    fmax = fmax > sqrt(f) ? fmax : sqrt(f);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < BS; ++j) {
      double d = L[j][j];
#pragma unroll
      for (int k = 0; k < j; ++k) d = fma(-L[j][k], L[j][k], d);
      ok = ok && (d > 0.0) && isfinite(d);
      const double ljj = sqrt(d);
      L[j][j] = ljj;
#pragma unroll
      for (int i = j + 1; i < BS; ++i) {
        double t = L[i][j];
#pragma unroll
        for (int k = 0; k < j; ++k) t = fma(-L[i][k], L[j][k], t);
        L[i][j] = t / ljj;
      }
    }
    if (!ok) atomicCAS(&st->status, SCQR3_OK, SCQR3_E_B_NOT_SPD);
    double* o = lt + b * BSP;
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
      for (int l = i; l < BS; ++l) o[pk_idx(BS, i, l)] = L[l][i];
  }
  // non-negative doubles order like their bit patterns
  atomicMax((unsigned long long*)&st->normb_bits_max, (unsigned long long)__double_as_longlong(fmax));
}

// -------------------------------------------------------------------------------------------
// Host launchers.

template <int NP>
static cudaError_t setup_pass(int* max_ctas_per_sm) {
  auto k = pass_kernel<NP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo<NP>::smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(chol_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(2 * sizeof(double) * pk_size(NP)));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_ctas_per_sm, k, kThreads, Geo<NP>::smem);
}

cudaError_t pass_setup(int np, int* ctas_per_sm, PassGeom* geo) {
  switch (np) {
    case 16: *geo = pass_geom<16>(); return setup_pass<16>(ctas_per_sm);
    case 32: *geo = pass_geom<32>(); return setup_pass<32>(ctas_per_sm);
    case 64: *geo = pass_geom<64>(); return setup_pass<64>(ctas_per_sm);
    case 128: *geo = pass_geom<128>(); return setup_pass<128>(ctas_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

void launch_pass(int np, int grid, cudaStream_t s, const double* src, int64_t lds, double* dst,
                 int64_t ldd, const Params& P, int pass, const double* rk, const double* lt,
                 double* partials, int part_stride, DevState* st) {
  switch (np) {
#define SCQR3_PASS(NPV)                                                                        \
  case NPV:                                                                                    \
    pass_kernel<NPV><<<grid, kThreads, Geo<NPV>::smem, s>>>(src, lds, dst, ldd, P, pass, rk, lt, \
                                                            partials, part_stride, st);        \
    break;
    SCQR3_PASS(16)
    SCQR3_PASS(32)
    SCQR3_PASS(64)
    SCQR3_PASS(128)
#undef SCQR3_PASS
    default: break;
  }
}

void launch_reduce(cudaStream_t s, const double* partials, int n_partials, int stride, double* out,
                   const DevState* st, int pass) {
  reduce_kernel<<<ceil_div(stride, 128), 128, 0, s>>>(partials, n_partials, stride, out, st, pass);
}

void launch_chol(int np, cudaStream_t s, const Params& P, int pass, const double* gram,
                 double* rstack, double* racc, double* Rout, double* Rpass, DevState* st,
                 scqr3_info* info) {
  const size_t sm = 2 * sizeof(double) * pk_size(np);
  switch (np) {
    case 16: chol_kernel<16><<<1, 256, sm, s>>>(P, pass, gram, rstack, racc, Rout, Rpass, st, info); break;
    case 32: chol_kernel<32><<<1, 256, sm, s>>>(P, pass, gram, rstack, racc, Rout, Rpass, st, info); break;
    case 64: chol_kernel<64><<<1, 512, sm, s>>>(P, pass, gram, rstack, racc, Rout, Rpass, st, info); break;
    case 128: chol_kernel<128><<<1, 512, sm, s>>>(P, pass, gram, rstack, racc, Rout, Rpass, st, info); break;
    default: break;
  }
}

void launch_status(cudaStream_t s, const DevState* st, scqr3_info* info) { status_kernel<<<1, 32, 0, s>>>(st, info); }

void launch_bfactor(cudaStream_t s, int bs, const double* B, int64_t nblk, double* lt, DevState* st,
                    int sms) {
  const int threads = 128;
  int64_t want = (nblk + threads - 1) / threads;
  const int grid = (int)(want < (int64_t)sms * 8 ? (want < 1 ? 1 : want) : (int64_t)sms * 8);
  switch (bs) {
    case 1: bfactor_kernel<1><<<grid, threads, 0, s>>>(B, nblk, lt, st); break;
    case 2: bfactor_kernel<2><<<grid, threads, 0, s>>>(B, nblk, lt, st); break;
    case 4: bfactor_kernel<4><<<grid, threads, 0, s>>>(B, nblk, lt, st); break;
    case 8: bfactor_kernel<8><<<grid, threads, 0, s>>>(B, nblk, lt, st); break;
    case 16: bfactor_kernel<16><<<grid, threads, 0, s>>>(B, nblk, lt, st); break;
    default: break;
  }
}

}  // namespace scqr3
