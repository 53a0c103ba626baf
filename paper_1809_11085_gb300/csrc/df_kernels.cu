// df_kernels.cu -- the mixed-precision pass kernel: FP32 pairs ("double-float")
// on the FP32 pipe, FP64 for the Gram accumulation, shift and Cholesky.
//
// GB300 retires 62x more FP32 than FP64 FMAs. Here each value of the bulk
// Gram and substitution is a pair (h, l) of floats with x ~ h + l (48
// significant bits), and every product and sum is done with error-free
// transformations:
//   product  x*y   = p + e with p = fl(xh*yh), e = fma(xh,yh,-p) + xh*yl + xl*yh
//   Gram sum S += p by TwoSum, its rounding error and e summed into C
//            (Ogita-Rump-Oishi Dot2), and (S, C) added into FP64 partials
//            every 256 rows of a group;
//   solve    t_l -= q_j r_jl with the same TwoSum, q_j = t_j * (1/r_jj).
// The worst-case Gram error is then below that of a plain FP64 sum over m
// rows (gamma_m of Eq. err_1), so the shift of Eq. (finds2), the FP64
// Cholesky and the pass control are used unchanged. Iterates Q_k are stored
// in HBM as float pairs in the same 8 bytes per element as FP64; X is split
// when read and the last solve writes FP64 Q.
#include <cmath>

#include "scqr3_internal.cuh"

namespace scqr3 {

template <int NP> struct DfCfg;
template <> struct DfCfg<16>  { static constexpr int PR = 256, T = 8,   H = 1; };
template <> struct DfCfg<32>  { static constexpr int PR = 256, T = 16,  H = 1; };
template <> struct DfCfg<64>  { static constexpr int PR = 256, T = 32,  H = 1; };
template <> struct DfCfg<128> { static constexpr int PR = 128, T = 128, H = 2; };

template <int NP> struct DfGeo {
  static constexpr int PR = DfCfg<NP>::PR, T = DfCfg<NP>::T, H = DfCfg<NP>::H;
  static constexpr int G = kThreads / T;
  static constexpr int RG = PR / G;
  static constexpr int C = (NP + 1 + H - 1) / H;
  static constexpr int LD = NP + 1;
  static constexpr int E = pk_size(NP);
  static constexpr int FLUSH = (256 / RG) > 0 ? (256 / RG) : 1;  // panels between FP64 flushes
  static constexpr size_t smem = sizeof(float2) * ((size_t)PR * LD + E + NP);
};

__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}

__device__ __forceinline__ double df_join(float2 v) { return (double)v.x + (double)v.y; }

// (S, C) += x * y   (Dot2 step with a pair-valued x and y)
__device__ __forceinline__ void df_acc(float& S, float& Cc, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  const float s = __fadd_rn(S, p);
  const float z = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, z)), __fsub_rn(p, z));
  S = s;
  Cc = __fadd_rn(Cc, __fadd_rn(err, e));
}

// (th, tl) -= q * r
__device__ __forceinline__ void df_sub(float& th, float& tl, float2 q, float2 r) {
  const float p = __fmul_rn(q.x, r.x);
  float e = __fmaf_rn(q.x, r.x, -p);
  e = __fmaf_rn(q.x, r.y, e);
  e = __fmaf_rn(q.y, r.x, e);
  const float s = __fsub_rn(th, p);
  const float z = __fsub_rn(s, th);
  const float err = __fadd_rn(__fsub_rn(th, __fsub_rn(s, z)), __fsub_rn(-p, z));
  th = s;
  tl = __fadd_rn(tl, __fsub_rn(err, e));
}

// normalized (t) * (r)
__device__ __forceinline__ float2 df_mul(float2 t, float2 r) {
  const float p = __fmul_rn(t.x, r.x);
  float e = __fmaf_rn(t.x, r.x, -p);
  e = __fmaf_rn(t.x, r.y, e);
  e = __fmaf_rn(t.y, r.x, e);
  const float h = __fadd_rn(p, e);
  const float l = __fsub_rn(e, __fsub_rn(h, p));
  return make_float2(h, l);
}

// pass < 0: Gram of X (FP64 input). pass >= 0: solve with R_pass; src is X
// (FP64) for pass 0, else the float-pair iterate; dst gets float pairs, or
// FP64 when this is the last solve (no Gram after it).
template <int NP>
__global__ void __launch_bounds__(kThreads, 1)
df_pass_kernel(const double* src, int64_t lds, double* dst, int64_t ldd, Params P, int pass,
               const double* __restrict__ rk, double* __restrict__ partials, int part_stride,
               DevState* __restrict__ st) {
  using g = DfGeo<NP>;
  extern __shared__ __align__(16) float2 fsm[];
  float2* panel = fsm;               // PR x LD pairs
  float2* rp = panel + g::PR * g::LD;  // packed R_k as pairs
  float2* rinv = rp + g::E;

  const int tid = threadIdx.x;
  const int n = P.n;
  const int64_t m = P.m;
  bool do_trsm = false, do_gram = true;
  if (pass >= 0) {
    if (!st->run_trsm[pass]) return;
    do_trsm = true;
    do_gram = st->gram_after[pass] != 0 && !P.solve_only;
  }
  const bool src_fp64 = pass <= 0;
  const bool dst_fp64 = pass >= 0 && !st->gram_after[pass];  // pairs while another pass follows
  const float2* srcf = reinterpret_cast<const float2*>(src);
  float2* dstf = reinterpret_cast<float2*>(dst);

  if (do_trsm) {
    for (int e = tid; e < g::E; e += kThreads) rp[e] = df_split(rk[e]);
    if (tid < NP) rinv[tid] = df_split(1.0 / rk[pk_row(NP, tid)]);
    __syncthreads();
  }
  for (int r = tid; r < g::PR; r += kThreads) panel[r * g::LD + NP] = make_float2(0.f, 0.f);

  const int tt = tid % g::T, grp = tid / g::T;
  const int pidx = tt % (NP / 2), h = tt / (NP / 2);
  float aS[g::C], aC[g::C];
#pragma unroll
  for (int l = 0; l < g::C; ++l) { aS[l] = 0.f; aC[l] = 0.f; }
  double* part = partials + ((int64_t)blockIdx.x * g::G + grp) * part_stride;
  bool first_flush = true;
  int since_flush = 0;

  const int64_t npanels = (m + g::PR - 1) / g::PR;
  for (int64_t pnl = blockIdx.x; pnl < npanels; pnl += gridDim.x) {
    const int64_t row0 = pnl * g::PR;
    const int rows = (int)((m - row0) < (int64_t)g::PR ? (m - row0) : (int64_t)g::PR);
    __syncthreads();
    for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
      const int r = idx / NP, c = idx % NP;
      float2 v = make_float2(0.f, 0.f);
      if (r < rows && c < n) {
        if (src_fp64)
          v = df_split(src[(row0 + r) * lds + c]);
        else
          v = srcf[(row0 + r) * lds + c];
      }
      panel[r * g::LD + c] = v;
    }
    __syncthreads();

    if (do_trsm) {
      if (tid < rows) {
        float2* row = panel + tid * g::LD;
        for (int j = 0; j < n; ++j) {
          const float2 q = df_mul(row[j], rinv[j]);
          row[j] = q;
          const float2* rj = rp + pk_row(NP, j) - j;
#pragma unroll 4
          for (int l = j + 1; l < n; ++l) {
            float2 t = row[l];
            df_sub(t.x, t.y, q, rj[l]);
            row[l] = t;
          }
        }
      }
      __syncthreads();
      for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
        const int r = idx / NP, c = idx % NP;
        if (r < rows && c < n) {
          const float2 v = panel[r * g::LD + c];
          if (dst_fp64)
            dst[(row0 + r) * ldd + c] = df_join(v);
          else
            dstf[(row0 + r) * ldd + c] = v;
        }
      }
    }
    if (!do_gram) continue;

    const int rbeg = grp * g::RG;
    const int rend = min(rbeg + g::RG, rows);
    for (int r = rbeg; r < rend; ++r) {
      const float2* row = panel + r * g::LD;
      const float2 a = row[pidx], b = row[NP - 1 - pidx];
#pragma unroll
      for (int l = 0; l < g::C; ++l) {
        const int L = h * g::C + l;
        const bool seg_a = L < NP - pidx;
        const int col = seg_a ? pidx + L : L - 1;
        df_acc(aS[l], aC[l], seg_a ? a : b, row[col]);
      }
    }
    if (++since_flush == g::FLUSH) {
      since_flush = 0;
#pragma unroll
      for (int l = 0; l < g::C; ++l) {
        const int L = h * g::C + l;
        if (L > NP) continue;
        const bool seg_a = L < NP - pidx;
        const int j = seg_a ? pidx : NP - 1 - pidx;
        const int k = seg_a ? pidx + L : L - 1;
        const double v = (double)aS[l] + (double)aC[l];
        double* d = part + pk_idx(NP, j, k);
        *d = first_flush ? v : *d + v;
        aS[l] = 0.f;
        aC[l] = 0.f;
      }
      first_flush = false;
    }
  }

  if (pass >= 0 && !do_gram) return;
#pragma unroll
  for (int l = 0; l < g::C; ++l) {
    const int L = h * g::C + l;
    if (L > NP) continue;
    const bool seg_a = L < NP - pidx;
    const int j = seg_a ? pidx : NP - 1 - pidx;
    const int k = seg_a ? pidx + L : L - 1;
    const double v = (double)aS[l] + (double)aC[l];
    double* d = part + pk_idx(NP, j, k);
    *d = first_flush ? v : *d + v;
  }
  if (tid < g::G) partials[((int64_t)blockIdx.x * g::G + tid) * part_stride + g::E] = 0.0;
}

// -------------------------------------------------------------------------------------------
// Version for NP <= 64, shaped for the FP32 pipe (every issue slot counts):
//  * cyclic Gram layout: thread j of a group owns the entries (j, j+d mod NP),
//    d = 0 .. NP/2 - 1, plus d = NP/2 for j < NP/2 (which covers every entry
//    of the upper triangle exactly once). Each panel row carries a copy of its
//    first NP/2 - 1 columns after column NP-1, so thread j reads the
//    consecutive words row[j], row[j+1], ... at compile-time offsets: no
//    index arithmetic or selects per product, no bank conflicts;
//  * left-looking, register-blocked substitution: one row per thread, eight
//    columns of t held in registers and updated by every solved q_i (ascending
//    i, the same order as the right-looking form), then solved in place: eight
//    independent chains per thread and no shared-memory store per update;
//  * every thread of the CTA solves a row (panel of 256 rows), R_k and 1/r_jj
//    as float pairs in shared memory.
template <int NP> struct Df2Cfg;
template <> struct Df2Cfg<16> { static constexpr int PR = 256, MINB = 2; };
template <> struct Df2Cfg<32> { static constexpr int PR = 256, MINB = 2; };
template <> struct Df2Cfg<64> { static constexpr int PR = 256, MINB = 1; };

template <int NP> struct Df2Geo {
  static constexpr int PR = Df2Cfg<NP>::PR, MINB = Df2Cfg<NP>::MINB;
  static constexpr int T = NP;                  // threads of a Gram group
  static constexpr int G = kThreads / T;
  static constexpr int RG = PR / G;
  static constexpr int HALF = NP / 2;
  static constexpr int C = HALF + 1;            // entries of threads j < NP/2
  static constexpr int LD = NP + HALF - 1;      // odd: conflict-free row-per-thread access
  static constexpr int E = pk_size(NP);
  static constexpr int FLUSH = (256 / RG) > 0 ? (256 / RG) : 1;
  static constexpr int NB = NP / 8;             // column blocks of the solve
  static constexpr size_t smem = sizeof(float2) * ((size_t)PR * LD + E + NP);
};

template <int NP>
__global__ void __launch_bounds__(kThreads, Df2Cfg<NP>::MINB)
df2_pass_kernel(const double* src, int64_t lds, double* dst, int64_t ldd, Params P, int pass,
                const double* __restrict__ rk, double* __restrict__ partials, int part_stride,
                DevState* __restrict__ st) {
  using g = Df2Geo<NP>;
  extern __shared__ __align__(16) float2 fsm[];
  float2* panel = fsm;                 // PR x LD pairs
  float2* rp = panel + g::PR * g::LD;  // packed R_k as pairs
  float2* rinv = rp + g::E;

  const int tid = threadIdx.x;
  const int n = P.n;
  const int64_t m = P.m;
  bool do_trsm = false, do_gram = true;
  if (pass >= 0) {
    if (!st->run_trsm[pass]) return;
    do_trsm = true;
    do_gram = st->gram_after[pass] != 0 && !P.solve_only;
  }
  const bool src_fp64 = pass <= 0;
  const bool dst_fp64 = pass >= 0 && !st->gram_after[pass];  // pairs while another pass follows
  const float2* srcf = reinterpret_cast<const float2*>(src);
  float2* dstf = reinterpret_cast<float2*>(dst);

  if (do_trsm) {
    for (int e = tid; e < g::E; e += kThreads) rp[e] = df_split(rk[e]);
    if (tid < NP) rinv[tid] = df_split(1.0 / rk[pk_row(NP, tid)]);
  }
  const int nb = (n + 7) / 8;  // column blocks that hold data (padding has R = I)

  const int j = tid % g::T, grp = tid / g::T;
  float aS[g::C], aC[g::C];
#pragma unroll
  for (int d = 0; d < g::C; ++d) { aS[d] = 0.f; aC[d] = 0.f; }
  double* part = partials + ((int64_t)blockIdx.x * g::G + grp) * part_stride;
  bool first_flush = true;
  int since_flush = 0;

  const int64_t npanels = (m + g::PR - 1) / g::PR;
  for (int64_t pnl = blockIdx.x; pnl < npanels; pnl += gridDim.x) {
    const int64_t row0 = pnl * g::PR;
    const int rows = (int)((m - row0) < (int64_t)g::PR ? (m - row0) : (int64_t)g::PR);
    __syncthreads();
    for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
      const int r = idx / NP, c = idx % NP;
      float2 v = make_float2(0.f, 0.f);
      if (r < rows && c < n) {
        if (src_fp64)
          v = df_split(src[(row0 + r) * lds + c]);
        else
          v = srcf[(row0 + r) * lds + c];
      }
      panel[r * g::LD + c] = v;
    }
    __syncthreads();

    if (do_trsm && tid < rows) {
      float2* row = panel + tid * g::LD;
      for (int J = 0; J < nb; ++J) {
        float th[8], tl[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) { const float2 v = row[8 * J + c]; th[c] = v.x; tl[c] = v.y; }
        for (int i = 0; i < 8 * J; ++i) {
          const float2 q = row[i];
          const float2* ri = rp + pk_row(NP, i) - i + 8 * J;  // R_k(i, 8J .. 8J+7)
#pragma unroll
          for (int c = 0; c < 8; ++c) df_sub(th[c], tl[c], q, ri[c]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float2 q = df_mul(make_float2(th[c], tl[c]), rinv[8 * J + c]);
          th[c] = q.x;
          tl[c] = q.y;
          const float2* rc = rp + pk_row(NP, 8 * J + c) - (8 * J + c) + 8 * J;  // R_k(8J+c, 8J..)
#pragma unroll
          for (int c2 = c + 1; c2 < 8; ++c2) df_sub(th[c2], tl[c2], q, rc[c2]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) row[8 * J + c] = make_float2(th[c], tl[c]);
      }
    }
    if (do_trsm) {
      __syncthreads();
      for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
        const int r = idx / NP, c = idx % NP;
        if (r < rows && c < n) {
          const float2 v = panel[r * g::LD + c];
          if (dst_fp64)
            dst[(row0 + r) * ldd + c] = df_join(v);
          else
            dstf[(row0 + r) * ldd + c] = v;
        }
      }
    }
    if (!do_gram) continue;
    // mirror columns 0 .. NP/2-2 after column NP-1
    for (int idx = tid; idx < g::PR * (g::HALF - 1); idx += kThreads) {
      const int r = idx / (g::HALF - 1), c = idx % (g::HALF - 1);
      panel[r * g::LD + NP + c] = panel[r * g::LD + c];
    }
    __syncthreads();

    const int rbeg = grp * g::RG;
    const int rend = min(rbeg + g::RG, rows);
    for (int r = rbeg; r < rend; ++r) {
      const float2* rb = panel + r * g::LD + j;
      const float2 a = rb[0];
#pragma unroll
      for (int d = 0; d < g::HALF; ++d) df_acc(aS[d], aC[d], a, rb[d]);
      if (j < g::HALF) df_acc(aS[g::HALF], aC[g::HALF], a, rb[g::HALF]);
    }
    if (++since_flush == g::FLUSH || pnl + gridDim.x >= npanels) {
      since_flush = 0;
#pragma unroll
      for (int d = 0; d < g::C; ++d) {
        if (d == g::HALF && j >= g::HALF) continue;
        int r = j, c = j + d;
        if (c >= NP) { c -= NP; const int t = r; r = c; c = t; }
        const double v = (double)aS[d] + (double)aC[d];
        double* p = part + pk_idx(NP, r, c);
        *p = first_flush ? v : *p + v;
        aS[d] = 0.f;
        aC[d] = 0.f;
      }
      first_flush = false;
    }
  }
  if (pass >= 0 && !do_gram) return;
  if (first_flush) {  // this CTA saw no panel: its slots still have to be written
#pragma unroll
    for (int d = 0; d < g::C; ++d) {
      if (d == g::HALF && j >= g::HALF) continue;
      int r = j, c = j + d;
      if (c >= NP) { c -= NP; const int t = r; r = c; c = t; }
      part[pk_idx(NP, r, c)] = 0.0;
    }
  }
  if (tid < g::G) partials[((int64_t)blockIdx.x * g::G + tid) * part_stride + g::E] = 0.0;
}

// -------------------------------------------------------------------------------------------
// Version for NP = 64 and 128: panels of 128 rows,
//  * two threads per row in the solve (adjacent lanes; each owns four of the
//    eight columns of a block, the first lane hands its four solved values to
//    the second by shuffle), so every thread of the CTA solves;
//  * R_k staged one 8-column block at a time (the panel with its mirrored
//    tail fills most of shared memory for NP = 128);
//  * cyclic Gram. NP = 128: the whole CTA is one group, thread (j, half) owns
//    the entries (j, j+d) for d in [33 half, 33 half + 33) (d <= 64; d = 64
//    only for j < 64). NP = 64: four groups of 64 threads, each over 32 rows
//    of the panel, thread j owning d = 0..31 plus d = 32 for j < 32;
//  * NP = 64 fits two CTAs per SM, so one CTA's loads overlap the other's
//    arithmetic.
template <int NP> struct DfpCfg;
template <> struct DfpCfg<64>  { static constexpr int GT = 64,  MINB = 2; };
template <> struct DfpCfg<128> { static constexpr int GT = 256, MINB = 1; };

template <int NP> struct DfpGeo {
  static constexpr int PR = 128, HALF = NP / 2;
  static constexpr int GT = DfpCfg<NP>::GT;       // threads of a Gram group
  static constexpr int G = kThreads / GT;         // groups
  static constexpr int RG = PR / G;               // panel rows per group
  static constexpr int C = NP == 128 ? 33 : HALF + 1;  // accumulator pairs per thread
  static constexpr int LD = NP + HALF - 1;        // odd
  static constexpr int E = pk_size(NP);
  static constexpr int FLUSH = 256 / RG;          // panels per FP64 flush (256 rows)
  static constexpr size_t smem = sizeof(float2) * ((size_t)PR * LD + NP * 8 + NP);
};

template <int NP>
__global__ void __launch_bounds__(kThreads, DfpCfg<NP>::MINB)
dfp_pass_kernel(const double* src, int64_t lds, double* dst, int64_t ldd, Params P, int pass,
                const double* __restrict__ rk, double* __restrict__ partials, int part_stride,
                DevState* __restrict__ st) {
  using g = DfpGeo<NP>;
  constexpr int PR = g::PR, HALF = g::HALF, C = g::C, LD = g::LD, E = g::E;
  extern __shared__ __align__(16) float2 fsm[];
  float2* panel = fsm;                // PR x LD
  float2* rb = panel + PR * LD;       // R_k(0 .. 8J+7, 8J .. 8J+7), row-major 8 wide
  float2* rinv = rb + NP * 8;

  const int tid = threadIdx.x;
  const int n = P.n;
  const int64_t m = P.m;
  bool do_trsm = false, do_gram = true;
  if (pass >= 0) {
    if (!st->run_trsm[pass]) return;
    do_trsm = true;
    do_gram = st->gram_after[pass] != 0 && !P.solve_only;
  }
  const bool src_fp64 = pass <= 0;
  const bool dst_fp64 = pass >= 0 && !st->gram_after[pass];  // pairs while another pass follows
  const float2* srcf = reinterpret_cast<const float2*>(src);
  float2* dstf = reinterpret_cast<float2*>(dst);
  if (do_trsm && tid < NP) rinv[tid] = df_split(1.0 / rk[pk_row(NP, tid)]);
  const int nb = (n + 7) / 8;

  const int srow = tid >> 1, sh = tid & 1;  // solve: row, and which four columns
  // Gram: row j of the entries, first d and count; group and its rows
  const int j = tid % NP;
  const int grp = tid / g::GT;
  int d0, dn;
  if (NP == 128) {
    const int gh = tid >> 7;
    d0 = gh * C;
    dn = gh == 0 ? C : (j < HALF ? C - 1 : C - 2);
  } else {
    d0 = 0;
    dn = j < HALF ? C : C - 1;
  }
  float aS[C], aC[C];
#pragma unroll
  for (int d = 0; d < C; ++d) { aS[d] = 0.f; aC[d] = 0.f; }
  double* part = partials + ((int64_t)blockIdx.x * g::G + grp) * part_stride;
  bool first_flush = true;
  int since_flush = 0;

  auto flush = [&]() {
#pragma unroll
    for (int dd = 0; dd < C; ++dd) {
      if (dd >= dn) continue;
      const int d = d0 + dd;
      int r = j, c = j + d;
      if (c >= NP) { c -= NP; const int t = r; r = c; c = t; }
      const double v = (double)aS[dd] + (double)aC[dd];
      double* p = part + pk_idx(NP, r, c);
      *p = first_flush ? v : *p + v;
      aS[dd] = 0.f;
      aC[dd] = 0.f;
    }
    first_flush = false;
  };

  const int64_t npanels = (m + PR - 1) / PR;
  for (int64_t pnl = blockIdx.x; pnl < npanels; pnl += gridDim.x) {
    const int64_t row0 = pnl * PR;
    const int rows = (int)((m - row0) < (int64_t)PR ? (m - row0) : (int64_t)PR);
    __syncthreads();
    for (int idx = tid; idx < PR * NP; idx += kThreads) {
      const int r = idx / NP, c = idx % NP;
      float2 v = make_float2(0.f, 0.f);
      if (r < rows && c < n) {
        if (src_fp64)
          v = df_split(src[(row0 + r) * lds + c]);
        else
          v = srcf[(row0 + r) * lds + c];
      }
      panel[r * LD + c] = v;
    }

    if (do_trsm) {
      float2* row = panel + srow * LD;
      for (int J = 0; J < nb; ++J) {
        __syncthreads();  // panel loaded / previous block of R_k consumed
        for (int idx = tid; idx < (8 * J + 8) * 8; idx += kThreads) {
          const int i = idx >> 3, c = idx & 7;
          const int col = 8 * J + c;
          rb[idx] = df_split(col >= i ? rk[pk_idx(NP, i, col)] : 0.0);
        }
        __syncthreads();
        float th[4], tl[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) { const float2 v = row[8 * J + 4 * sh + c]; th[c] = v.x; tl[c] = v.y; }
        for (int i = 0; i < 8 * J; ++i) {
          const float2 q = row[i];
          const float2* ri = rb + i * 8 + 4 * sh;
#pragma unroll
          for (int c = 0; c < 4; ++c) df_sub(th[c], tl[c], q, ri[c]);
        }
        // diagonal block: lane sh = 0 solves columns 0..3 and hands them to sh = 1
        float2 q4[4];
        if (sh == 0) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float2 q = df_mul(make_float2(th[c], tl[c]), rinv[8 * J + c]);
            q4[c] = q;
#pragma unroll
            for (int c2 = c + 1; c2 < 4; ++c2) df_sub(th[c2], tl[c2], q, rb[(8 * J + c) * 8 + c2]);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          q4[c].x = __shfl_sync(0xffffffffu, q4[c].x, tid & ~1);
          q4[c].y = __shfl_sync(0xffffffffu, q4[c].y, tid & ~1);
        }
        if (sh == 1) {
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) df_sub(th[c2], tl[c2], q4[c], rb[(8 * J + c) * 8 + 4 + c2]);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float2 q = df_mul(make_float2(th[c], tl[c]), rinv[8 * J + 4 + c]);
            th[c] = q.x;
            tl[c] = q.y;
#pragma unroll
            for (int c2 = c + 1; c2 < 4; ++c2) df_sub(th[c2], tl[c2], q, rb[(8 * J + 4 + c) * 8 + 4 + c2]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) { th[c] = q4[c].x; tl[c] = q4[c].y; }
        }
        if (srow < rows) {
#pragma unroll
          for (int c = 0; c < 4; ++c) row[8 * J + 4 * sh + c] = make_float2(th[c], tl[c]);
        }
      }
      __syncthreads();
      for (int idx = tid; idx < PR * NP; idx += kThreads) {
        const int r = idx / NP, c = idx % NP;
        if (r < rows && c < n) {
          const float2 v = panel[r * LD + c];
          if (dst_fp64)
            dst[(row0 + r) * ldd + c] = df_join(v);
          else
            dstf[(row0 + r) * ldd + c] = v;
        }
      }
    }
    if (!do_gram) continue;
    __syncthreads();
    for (int idx = tid; idx < PR * (HALF - 1); idx += kThreads) {
      const int r = idx / (HALF - 1), c = idx % (HALF - 1);
      panel[r * LD + NP + c] = panel[r * LD + c];
    }
    __syncthreads();
    const int rbeg = grp * g::RG;
    const int rend = min(rbeg + g::RG, rows);
    for (int r = rbeg; r < rend; ++r) {
      const float2* rbase = panel + r * LD + j;
      const float2 a = rbase[0];
      const float2* p2 = rbase + d0;
#pragma unroll
      for (int dd = 0; dd < C - 2; ++dd) df_acc(aS[dd], aC[dd], a, p2[dd]);
      if (dn > C - 2) df_acc(aS[C - 2], aC[C - 2], a, p2[C - 2]);
      if (dn > C - 1) df_acc(aS[C - 1], aC[C - 1], a, p2[C - 1]);
    }
    if (++since_flush == g::FLUSH || pnl + gridDim.x >= npanels) {
      since_flush = 0;
      flush();
    }
  }
  if (pass >= 0 && !do_gram) return;
  if (first_flush) {
#pragma unroll
    for (int dd = 0; dd < C; ++dd) {
      if (dd >= dn) continue;
      const int d = d0 + dd;
      int r = j, c = j + d;
      if (c >= NP) { c -= NP; const int t = r; r = c; c = t; }
      part[pk_idx(NP, r, c)] = 0.0;
    }
  }
  if (tid < g::G) partials[((int64_t)blockIdx.x * g::G + tid) * part_stride + E] = 0.0;
}

template <int NP>
static cudaError_t df_setup_one() {
  return cudaFuncSetAttribute(df_pass_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)DfGeo<NP>::smem);
}

template <int NP>
static cudaError_t df2_setup_one() {
  return cudaFuncSetAttribute(df2_pass_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Df2Geo<NP>::smem);
}

// After the last solve that ran: if it left Q as float pairs (a Gram step was
// still planned after it -- Alg. 2's stopping test, or a later pass that broke
// down), convert Q to FP64 in place, element by element.
__global__ void __launch_bounds__(kThreads)
df_finish_kernel(double* Q, int64_t ldq, int64_t m, int n, int max_passes, const DevState* st) {
  int last = -1;
  for (int k = max_passes - 1; k >= 0; --k)
    if (st->run_trsm[k]) {
      last = k;
      break;
    }
  if (last < 0 || !st->gram_after[last]) return;
  const int64_t total = m * (int64_t)n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / n;
    const int c = (int)(idx - r * n);
    double* e = Q + r * ldq + c;
    const float2 v = *reinterpret_cast<const float2*>(e);
    *e = df_join(v);
  }
}

void launch_df_finish(int grid, cudaStream_t s, double* Q, int64_t ldq, int64_t m, int n,
                      int max_passes, const DevState* st) {
  df_finish_kernel<<<grid, kThreads, 0, s>>>(Q, ldq, m, n, max_passes, st);
}

cudaError_t df_setup() {
  cudaError_t e;
  if ((e = df2_setup_one<16>()) != cudaSuccess) return e;
  if ((e = df2_setup_one<32>()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(dfp_pass_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)DfpGeo<64>::smem)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(dfp_pass_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)DfpGeo<128>::smem);
}

// Resident CTAs per SM of the df pass kernel for a padded size.
cudaError_t df_occupancy(int np, int* per_sm) {
  switch (np) {
    case 16: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, df2_pass_kernel<16>, kThreads, Df2Geo<16>::smem);
    case 32: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, df2_pass_kernel<32>, kThreads, Df2Geo<32>::smem);
    case 64: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, dfp_pass_kernel<64>, kThreads, DfpGeo<64>::smem);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, dfp_pass_kernel<128>, kThreads, DfpGeo<128>::smem);
  }
}

// Gram groups per CTA of the df pass kernel for a padded size (partial-slot count).
int df_groups(int np) {
  switch (np) {
    case 16: return Df2Geo<16>::G;
    case 32: return Df2Geo<32>::G;
    case 64: return DfpGeo<64>::G;
    default: return DfpGeo<128>::G;
  }
}

// Rows per panel of the df pass kernel (grid sizing).
int df_rows_per_panel(int np) {
  switch (np) {
    case 16: return Df2Geo<16>::PR;
    case 32: return Df2Geo<32>::PR;
    case 64: return DfpGeo<64>::PR;
    default: return DfpGeo<128>::PR;
  }
}

void launch_df_pass(int np, int grid, cudaStream_t s, const double* src, int64_t lds, double* dst,
                    int64_t ldd, const Params& P, int pass, const double* rk, double* partials,
                    int part_stride, DevState* st) {
  switch (np) {
#define SCQR3_DF2(NPV)                                                                            \
  case NPV:                                                                                       \
    df2_pass_kernel<NPV><<<grid, kThreads, Df2Geo<NPV>::smem, s>>>(src, lds, dst, ldd, P, pass, rk,  \
                                                                   partials, part_stride, st);    \
    break;
    SCQR3_DF2(16)
    SCQR3_DF2(32)
#undef SCQR3_DF2
    case 64:
      dfp_pass_kernel<64><<<grid, kThreads, DfpGeo<64>::smem, s>>>(src, lds, dst, ldd, P, pass, rk,
                                                                   partials, part_stride, st);
      break;
    case 128:
      dfp_pass_kernel<128><<<grid, kThreads, DfpGeo<128>::smem, s>>>(src, lds, dst, ldd, P, pass, rk,
                                                                     partials, part_stride, st);
      break;
    default: break;
  }
}

}  // namespace scqr3
