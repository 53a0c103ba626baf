// fp64_device.cuh -- device code of the FP64 path shared by the single-matrix
// and batched launches: the pass-kernel geometry, the per-CTA pass over a
// range of row panels (pass_segment) and the one-CTA shift / Cholesky /
// bookkeeping step (chol_body). Included by fp64_kernels.cu and batched.cu.
#pragma once
#include <cmath>

#include "scqr3_internal.cuh"

namespace scqr3 {


// -------------------------------------------------------------------------------------------
// Pass kernel configuration per padded size NP.
//   PR  rows per panel held in shared memory (one row per thread in the solve)
//   T   threads of one Gram group; a group owns all n(n+1)/2 entries
//   H   pieces each folded row pair is cut into (keeps accumulators in registers)
// A group's thread tt owns folded pair p = tt % (NP/2): Gram row p (entries
// (p, p..NP-1)) followed by Gram row NP-1-p (entries (NP-1-p, NP-1-p..NP-1)),
// NP+1 entries in all, so every thread of a group does the same work and the
// columns read by neighbouring lanes are neighbouring words of shared memory.
template <int NP> struct Cfg;
//   MINB  resident CTAs per SM the register budget is sized for (small n
//         needs few registers; more CTAs let one CTA's loads overlap another's
//         arithmetic)
template <> struct Cfg<16>  { static constexpr int PR = 256, T = 8,   H = 1, MINB = 3; };
template <> struct Cfg<32>  { static constexpr int PR = 256, T = 16,  H = 1, MINB = 2; };
template <> struct Cfg<64>  { static constexpr int PR = 256, T = 32,  H = 1, MINB = 1; };
template <> struct Cfg<128> { static constexpr int PR = 128, T = 128, H = 2, MINB = 1; };

template <int NP> struct Geo {
  static constexpr int PR = Cfg<NP>::PR, T = Cfg<NP>::T, H = Cfg<NP>::H;
  static constexpr int G = kThreads / T;          // Gram groups per CTA
  static constexpr int RG = PR / G;               // panel rows per group
  static constexpr int C = (NP + 1 + H - 1) / H;  // accumulators per thread
  static constexpr int LD = NP + 1;               // panel row stride (col NP stays 0)
  static constexpr int E = pk_size(NP);
  static constexpr size_t smem = sizeof(double) * ((size_t)PR * LD + E + NP + kThreads / 32);
};

template <int NP>
PassGeom pass_geom() {
  using g = Geo<NP>;
  return PassGeom{NP, g::PR, g::G, g::T, g::H, g::C, g::smem};
}

// In-place Z = L^T Q for each bs-row block of the panel (B = L L^T), so that
// Z^T Z = Q^T B Q is the oblique Gram matrix of Alg. 4.
template <int NP, int BS>
__device__ __forceinline__ void apply_lt(double* panel, int rows, int n, int64_t blk0,
                                         int64_t nblk_total, const double* __restrict__ lt) {
  using g = Geo<NP>;
  constexpr int BSP = BS * (BS + 1) / 2;
  const int nblk = rows / BS;  // rows is a multiple of BS (m % bs == 0, PR % bs == 0)
  for (int item = threadIdx.x; item < nblk * n; item += kThreads) {
    const int b = item / n, c = item - b * n;
    const int64_t gb = blk0 + b;
    if (gb >= nblk_total) continue;
    const double* L = lt + gb * BSP;
    double q[BS];
#pragma unroll
    for (int i = 0; i < BS; ++i) q[i] = panel[(b * BS + i) * g::LD + c];
#pragma unroll
    for (int i = 0; i < BS; ++i) {
      double z = 0.0;
#pragma unroll
      for (int l = i; l < BS; ++l) z = fma(L[pk_idx(BS, i, l)], q[l], z);
      panel[(b * BS + i) * g::LD + c] = z;
    }
  }
}

template <int NP>
__device__ __forceinline__ void apply_lt_bs(double* panel, int rows, int n, int bs, int64_t row0,
                                            int64_t m, const double* __restrict__ lt) {
  switch (bs) {
    case 1: apply_lt<NP, 1>(panel, rows, n, row0, m, lt); break;
    case 2: apply_lt<NP, 2>(panel, rows, n, row0 / 2, m / 2, lt); break;
    case 4: apply_lt<NP, 4>(panel, rows, n, row0 / 4, m / 4, lt); break;
    case 8: apply_lt<NP, 8>(panel, rows, n, row0 / 8, m / 8, lt); break;
    case 16: apply_lt<NP, 16>(panel, rows, n, row0 / 16, m / 16, lt); break;
    default: break;
  }
}

// One CTA's share of a pass over one matrix: panels p_begin, p_begin + p_step,
// ... < p_end. pass < 0: Gram of X only (the first Gram of Alg. 3). pass >= 0:
// solve with R_pass (packed) and, when the state asks for it, the next Gram
// matrix, whose partial sums go to part + group * part_stride (group 0's slot
// also receives the sum of squares used by the oblique shift).
template <int NP>
__device__ __forceinline__ void pass_segment(const double* src, int64_t lds, double* dst, int64_t ldd,
                                             const Params& P, int pass, const double* __restrict__ rk,
                                             const double* __restrict__ lt, double* __restrict__ part,
                                             int part_stride, const DevState* __restrict__ st,
                                             int64_t p_begin, int64_t p_end, int64_t p_step) {
  using g = Geo<NP>;
  extern __shared__ __align__(16) double smem[];
  __syncthreads();  // a previous segment of this CTA may still be reading shared memory
  double* panel = smem;                      // PR x LD
  double* rp = panel + g::PR * g::LD;        // packed R_k
  double* rinv = rp + g::E;                  // 1 / r_jj
  double* red = rinv + NP;                   // per-warp ||.||_F^2 partials

  const int tid = threadIdx.x;
  const int n = P.n;
  const int64_t m = P.m;
  const bool oblique = P.bs > 0;
  bool do_trsm = false, do_gram = true;
  if (pass >= 0) {
    if (!st->run_trsm[pass]) return;
    do_trsm = true;
    do_gram = st->gram_after[pass] != 0 && !P.solve_only;  // else the Gram has its own kernel
  }

  if (do_trsm) {
    for (int e = tid; e < g::E; e += kThreads) rp[e] = rk[e];
    __syncthreads();
    if (tid < NP) rinv[tid] = 1.0 / rp[pk_row(NP, tid)];
  }
  for (int r = tid; r < g::PR; r += kThreads) panel[r * g::LD + NP] = 0.0;  // zero pad column

  const int tt = tid % g::T, grp = tid / g::T;
  const int pidx = tt % (NP / 2), h = tt / (NP / 2);
  double acc[g::C];
#pragma unroll
  for (int l = 0; l < g::C; ++l) acc[l] = 0.0;
  double f2 = 0.0;  // sum of squares of this thread's rows (oblique shift)

  for (int64_t pnl = p_begin; pnl < p_end; pnl += p_step) {
    const int64_t row0 = pnl * g::PR;
    const int rows = (int)((m - row0) < (int64_t)g::PR ? (m - row0) : (int64_t)g::PR);
    __syncthreads();  // previous panel fully consumed
    for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
      const int r = idx / NP, c = idx % NP;
      double v = 0.0;
      if (r < rows && c < n) v = src[(row0 + r) * lds + c];
      panel[r * g::LD + c] = v;
    }
    __syncthreads();

    if (do_trsm) {
      // Row-wise substitution q_i^T R_k = x_i^T (Eq. backward2), one row per
      // thread, left-looking in blocks of eight columns held in registers:
      // t_c -= q_i r_ic for every solved q_i (ascending i, one load of q_i
      // and eight broadcast loads of R_k per eight independent FMAs, no
      // store in the loop), then the 8 x 8 diagonal block by substitution.
      if (NP == 128) {
        // 128-row panels: two threads per row (adjacent lanes, four of the
        // eight columns of each block each), so all eight warps solve
        const int srow = tid >> 1, sh = tid & 1;
        double* row = panel + srow * g::LD;
        const int nb = (n + 7) / 8;
        for (int J = 0; J < nb; ++J) {
          double t[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) t[c] = row[8 * J + 4 * sh + c];
          for (int i = 0; i < 8 * J; ++i) {
            const double q = row[i];
            const double* ri = rp + pk_row(NP, i) - i + 8 * J + 4 * sh;
#pragma unroll
            for (int c = 0; c < 4; ++c) t[c] = fma(-q, ri[c], t[c]);
          }
          double q4[4];
          if (sh == 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const double q = t[c] * rinv[8 * J + c];
              q4[c] = q;
              if (oblique && 8 * J + c < n) f2 = fma(q, q, f2);
              const double* rc = rp + pk_row(NP, 8 * J + c) - (8 * J + c) + 8 * J;
#pragma unroll
              for (int c2 = c + 1; c2 < 4; ++c2) t[c2] = fma(-q, rc[c2], t[c2]);
            }
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) q4[c] = __shfl_sync(0xffffffffu, q4[c], tid & ~1);
          if (sh == 1) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const double* rc = rp + pk_row(NP, 8 * J + c) - (8 * J + c) + 8 * J + 4;
#pragma unroll
              for (int c2 = 0; c2 < 4; ++c2) t[c2] = fma(-q4[c], rc[c2], t[c2]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const double q = t[c] * rinv[8 * J + 4 + c];
              t[c] = q;
              if (oblique && 8 * J + 4 + c < n) f2 = fma(q, q, f2);
              const double* rc = rp + pk_row(NP, 8 * J + 4 + c) - (8 * J + 4 + c) + 8 * J + 4;
#pragma unroll
              for (int c2 = c + 1; c2 < 4; ++c2) t[c2] = fma(-q, rc[c2], t[c2]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) t[c] = q4[c];
          }
          if (srow < rows) {
#pragma unroll
            for (int c = 0; c < 4; ++c) row[8 * J + 4 * sh + c] = t[c];
          }
          __syncwarp();  // the partner lane reads these solved values in the next block
        }
      } else if (tid < rows) {
        double* row = panel + tid * g::LD;
        const int nb = (n + 7) / 8;
        for (int J = 0; J < nb; ++J) {
          double t[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) t[c] = row[8 * J + c];
          for (int i = 0; i < 8 * J; ++i) {
            const double q = row[i];
            const double* ri = rp + pk_row(NP, i) - i + 8 * J;  // R_k(i, 8J .. 8J+7)
#pragma unroll
            for (int c = 0; c < 8; ++c) t[c] = fma(-q, ri[c], t[c]);
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const double q = t[c] * rinv[8 * J + c];
            t[c] = q;
            if (oblique && 8 * J + c < n) f2 = fma(q, q, f2);
            const double* rc = rp + pk_row(NP, 8 * J + c) - (8 * J + c) + 8 * J;  // R_k(8J+c, 8J..)
#pragma unroll
            for (int c2 = c + 1; c2 < 8; ++c2) t[c2] = fma(-q, rc[c2], t[c2]);
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) row[8 * J + c] = t[c];
        }
      }
      __syncthreads();
      for (int idx = tid; idx < g::PR * NP; idx += kThreads) {
        const int r = idx / NP, c = idx % NP;
        if (r < rows && c < n) dst[(row0 + r) * ldd + c] = panel[r * g::LD + c];
      }
    } else if (oblique && tid < rows) {
      const double* row = panel + tid * g::LD;
      for (int j = 0; j < n; ++j) f2 = fma(row[j], row[j], f2);
    }

    if (!do_gram) continue;
    if (oblique) {
      __syncthreads();  // Q rows written out before Z = L^T Q overwrites them
      apply_lt_bs<NP>(panel, rows, n, P.bs, row0, m, lt);
      __syncthreads();
    }

    // Folded SYRK: acc += (entries of this thread's folded pair) over the group's rows.
    const int rbeg = grp * g::RG;
    const int rend = min(rbeg + g::RG, rows);
    for (int r = rbeg; r < rend; ++r) {
      const double* row = panel + r * g::LD;
      const double a = row[pidx], b = row[NP - 1 - pidx];
#pragma unroll
      for (int l = 0; l < g::C; ++l) {
        const int L = h * g::C + l;
        const bool seg_a = L < NP - pidx;
        const int col = seg_a ? pidx + L : L - 1;  // L = NP+1 only when H > 1: pad column
        acc[l] = fma(seg_a ? a : b, row[col], acc[l]);
      }
    }
  }

  if (pass >= 0 && !do_gram) return;
  double* mine = part + (int64_t)grp * part_stride;
#pragma unroll
  for (int l = 0; l < g::C; ++l) {
    const int L = h * g::C + l;
    if (L > NP) continue;
    const bool seg_a = L < NP - pidx;
    const int j = seg_a ? pidx : NP - 1 - pidx;
    const int k = seg_a ? pidx + L : L - 1;
    mine[pk_idx(NP, j, k)] = acc[l];
  }
  // ||.||_F^2 of the rows this CTA saw, in the slot after the packed Gram of group 0.
  for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = f2;
  __syncthreads();
  if (tid < g::G) {
    double t = 0.0;
    if (tid == 0)
      for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    part[(int64_t)tid * part_stride + g::E] = t;
  }
}

// -------------------------------------------------------------------------------------------
// Shift of Eq. (finds2) and Eq. (finds2B); u = 2^-53. Written with explicit
// round-to-nearest operations so that the compiler cannot contract them.
__device__ __forceinline__ double shift_value(const Params& P, double nrm2, double normb) {
  const double u = 1.1102230246251565e-16;
  const double dm = (double)P.m, dn = (double)P.n;
  const double nn1 = __dmul_rn(dn, (double)(P.n + 1));
  double t;
  if (is_oblique(P)) {
    t = __dmul_rn(__dmul_rn(2.0, dm), sqrt(__dmul_rn(dm, dn)));
  } else {
    t = __dmul_rn(dm, dn);
  }
  double s = __dmul_rn(11.0, __dadd_rn(t, nn1));
  s = __dmul_rn(s, u);
  s = __dmul_rn(s, nrm2);
  if (is_oblique(P)) s = __dmul_rn(s, normb);
  return s;
}

// The smaller shift c u ||Q||^2 (times ||B||) of the remark in Sec. 6.1.
__device__ __forceinline__ double small_shift_value(const Params& P, double nrm2, double normb) {
  const double u = 1.1102230246251565e-16;
  double s = __dmul_rn(__dmul_rn(P.shift_scale, u), nrm2);
  if (is_oblique(P)) s = __dmul_rn(s, normb);
  return s;
}

// ||A - I||_F^2 of the packed symmetric A (off-diagonal entries count twice),
// summed over the whole block; the result is valid in every thread.
template <int NP>
__device__ double dev_from_identity2(const double* S, int n, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double d = 0.0;
  for (int j = warp; j < n; j += nw)
    for (int k = j + lane; k < n; k += 32) {
      const double v = S[pk_idx(NP, j, k)] - (k == j ? 1.0 : 0.0);
      d = fma(k == j ? v : 2.0 * v, v, d);
    }
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  __syncthreads();
  if (lane == 0) red[warp] = d;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// Sum of one value per thread over the block, in a fixed order, valid in
// every thread.
__device__ __forceinline__ double block_sum(double x, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// lambda_max of the packed symmetric positive semidefinite S (columns < n) by
// the power method: the estimate of ||Q||_2^2 = lambda_max(Q^T Q) that
// Sec. 4.1 allows in the shift (normest). v := S v / ||S v|| from
// v = (1, ..., 1) / sqrt(n); the estimate is the Rayleigh quotient, stopped
// once it changes by at most 1e-12 of itself, or after 200 steps. v and w hold
// n doubles each; the result is valid in every thread.
template <int NP>
__device__ double normest2(const double* S, int n, double* v, double* w, double* red) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) v[j] = 1.0 / sqrt((double)n);
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < 200; ++it) {
    double q = 0.0, ww = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double t = 0.0;
      for (int k = 0; k < n; ++k) t = fma(S[k <= j ? pk_idx(NP, k, j) : pk_idx(NP, j, k)], v[k], t);
      w[j] = t;
      q = fma(v[j], t, q);
      ww = fma(t, t, ww);
    }
    q = block_sum(q, red);
    ww = block_sum(ww, red);
    const double nw = sqrt(ww);
    const bool done = it > 0 && fabs(q - lam) <= 1e-12 * q;
    lam = q;
    if (done || !(nw > 0.0)) break;  // the same in every thread
    for (int j = threadIdx.x; j < n; j += blockDim.x) v[j] = w[j] / nw;
    __syncthreads();
  }
  return lam;
}

// Cholesky of the packed matrix S in place (upper factor), columns < n.
// Returns 0 or the 1-based breakdown column (radicand not positive/finite).
template <int NP>
__device__ int chol_packed(double* S, int n, int* fail_sh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  if (tid == 0) *fail_sh = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = S[pk_idx(NP, j, j)];
      if (!(d > 0.0) || !isfinite(d))
        *fail_sh = j + 1;
      else
        S[pk_idx(NP, j, j)] = sqrt(d);
    }
    __syncthreads();
    if (*fail_sh) return *fail_sh;
    const double rjj = S[pk_idx(NP, j, j)];
    for (int l = j + 1 + tid; l < n; l += nt) S[pk_idx(NP, j, l)] = S[pk_idx(NP, j, l)] / rjj;
    __syncthreads();
    for (int i = j + 1 + warp; i < n; i += nw) {
      const double rji = S[pk_idx(NP, j, i)];
      for (int l = i + lane; l < n; l += 32)
        S[pk_idx(NP, i, l)] = fma(-rji, S[pk_idx(NP, j, l)], S[pk_idx(NP, i, l)]);
    }
    __syncthreads();
  }
  return 0;
}

// S (packed A, then R_k) and Ra (packed R accumulation) are E doubles each,
// in shared memory for NP <= 128 and in workspace memory for NP = 256.
template <int NP>
__device__ __forceinline__ void chol_body(const Params& P, int pass, const double* __restrict__ gram,
                                          double* __restrict__ rstack, double* __restrict__ racc,
                                          double* __restrict__ Rout, double* __restrict__ Rpass,
                                          DevState* __restrict__ st, scqr3_info* __restrict__ info,
                                          double* S, double* Ra) {
  constexpr int E = pk_size(NP);
  __shared__ int fail_sh;
  __shared__ double s_sh, nrm_sh;
  __shared__ int shifted_sh, ufail_sh;
  __shared__ double red_sh[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = P.n;

  if (pass > 0 && !st->gram_after[pass - 1]) return;
  if (st->status != SCQR3_OK) {  // e.g. a block of B that is not SPD
    if (pass == 0 && tid == 0) info->status = st->status;
    return;
  }

  for (int e = tid; e < E; e += nt) S[e] = gram[e];
  __syncthreads();
  if (tid == 0) {
    // ||Q||^2 estimate: trace of the Gram matrix (B = I), else the sum of
    // squares accumulated in the same pass (Sec. 4.1: ||.||_F for ||.||_2).
    double nrm2 = 0.0;
    if (is_oblique(P)) {
      nrm2 = gram[E];
    } else {
      for (int j = 0; j < n; ++j) nrm2 = nrm2 + S[pk_idx(NP, j, j)];
    }
    if (pass == 0 && P.norm_x2 > 0.0) nrm2 = P.norm_x2;
    if (pass == 0 && is_oblique(P))
      st->normb = P.normb_in > 0.0 ? P.normb_in : st->normb_bits_max;
    nrm_sh = nrm2;
    // Alg. 3 shifts pass 1 unconditionally; Alg. 2 tries the plain Cholesky first
    shifted_sh = (pass == 0 && P.algorithm != 2);
    ufail_sh = 0;
  }
  __syncthreads();
  if (P.norm_x2 < 0.0) {  // SCQR3_NORM_X2_TWO_EST: ||Q||_2^2 of this pass's iterate, estimated
    __shared__ double pw[2][256];
    const double e = normest2<NP>(S, n, pw[0], pw[1], red_sh);
    if (tid == 0) nrm_sh = e;
    __syncthreads();
  }
  if (!isfinite(nrm_sh)) {
    if (tid == 0) {
      st->status = SCQR3_E_NONFINITE;
      info->status = SCQR3_E_NONFINITE;
    }
    return;
  }
  if (P.algorithm == 2 && pass > 0) {
    // Alg. 2's stopping test, on the Gram matrix of the current iterate
    const double d2 = dev_from_identity2<NP>(S, n, red_sh);
    if (sqrt(d2) <= P.tol) {
      if (tid == 0) {
        st->status = SCQR3_OK;
        info->status = SCQR3_OK;
        info->passes = pass;
      }
      return;
    }
  }

  if (!shifted_sh) {  // Alg. 2: plain Cholesky first
    const int f = chol_packed<NP>(S, n, &fail_sh);
    if (f) {
      if (tid == 0) {
        ufail_sh = f;
        shifted_sh = 1;
      }
      __syncthreads();
      for (int e = tid; e < E; e += nt) S[e] = gram[e];
      __syncthreads();
    }
  }
  if (tid == 0) s_sh = 0.0;
  if (shifted_sh) {  // Alg. 1 / Alg. 2: shifted Cholesky
    int f = 1;
    if (P.shift_scale > 0.0) {  // the smaller shift first (remark of Sec. 6.1)
      if (tid == 0) {
        s_sh = small_shift_value(P, nrm_sh, st->normb);
        for (int j = 0; j < n; ++j) S[pk_idx(NP, j, j)] = S[pk_idx(NP, j, j)] + s_sh;
      }
      __syncthreads();
      f = chol_packed<NP>(S, n, &fail_sh);
      if (f) {
        __syncthreads();
        for (int e = tid; e < E; e += nt) S[e] = gram[e];
        __syncthreads();
      }
    }
    if (f) {
      if (tid == 0) {
        s_sh = shift_value(P, nrm_sh, st->normb);
        for (int j = 0; j < n; ++j) S[pk_idx(NP, j, j)] = S[pk_idx(NP, j, j)] + s_sh;
      }
      __syncthreads();
      f = chol_packed<NP>(S, n, &fail_sh);
    }
    if (f) {
      if (tid == 0) {
        st->status = f;
        st->passes = pass + 1;
        info->status = f;
        info->passes = pass + 1;
        info->shifted[pass] = 1;
        info->unshifted_fail[pass] = ufail_sh;
        info->s[pass] = s_sh;
        info->norm2[pass] = nrm_sh;
      }
      return;
    }
  }
  __syncthreads();
  // Padding rows/columns n..NP-1 of R_k are the identity; lower part zero.
  for (int e = tid; e < E; e += nt) {
    // recover (j, k) of packed entry e
    int j = 0;
    while (pk_row(NP, j + 1) <= e) ++j;
    const int k = j + (e - pk_row(NP, j));
    if (j >= n || k >= n) S[e] = (j == k) ? 1.0 : 0.0;
  }
  __syncthreads();
  double* rk = rstack + (int64_t)pass * E;
  for (int e = tid; e < E; e += nt) rk[e] = S[e];
  if (Rpass) {
    double* out = Rpass + (int64_t)pass * n * n;
    for (int idx = tid; idx < n * n; idx += nt) {
      const int i = idx / n, k = idx % n;
      out[idx] = (k >= i) ? S[pk_idx(NP, i, k)] : 0.0;
    }
  }

  // R := R_k R (the update of Alg. 2); row i of the product needs rows >= i of the
  // old R, so rows are formed in ascending order, in place.
  if (pass == 0) {
    for (int e = tid; e < E; e += nt) Ra[e] = S[e];
  } else {
    for (int e = tid; e < E; e += nt) Ra[e] = racc[e];
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      double v = 0.0;
      const int jj = i + tid;
      if (jj < n) {
        for (int k = i; k <= jj; ++k) v = fma(S[pk_idx(NP, i, k)], Ra[pk_idx(NP, k, jj)], v);
      }
      __syncthreads();
      if (jj < n) Ra[pk_idx(NP, i, jj)] = v;
      __syncthreads();
    }
  }
  __syncthreads();
  for (int e = tid; e < E; e += nt) racc[e] = Ra[e];
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, k = idx % n;
    Rout[idx] = (k >= i) ? Ra[pk_idx(NP, i, k)] : 0.0;
  }
  if (tid == 0) {
    const int plain = shifted_sh ? 0 : st->plain_in_a_row + 1;
    st->plain_in_a_row = plain;
    st->passes = pass + 1;
    st->run_trsm[pass] = 1;
    // Alg. 3 ends after two consecutive plain passes; Alg. 2 needs the Gram
    // of every iterate for its stopping test
    const bool done = P.algorithm != 2 && plain >= 2;
    const bool more = !done && pass + 1 < P.max_passes;
    st->gram_after[pass] = more ? 1 : 0;
    if (!done && !more) st->status = SCQR3_E_MAXPASS;
    info->status = st->status;
    info->passes = pass + 1;
    info->more = st->gram_after[pass];
    info->shifted[pass] = shifted_sh;
    info->unshifted_fail[pass] = ufail_sh;
    info->s[pass] = s_sh;
    info->norm2[pass] = nrm_sh;
  }
}


}  // namespace scqr3
