// tc_bwprod.cu -- the two row products of a reverse pass of the tensor-core
// adjoint at n = 64, in one sweep over the rows.
//
// The adjoint holds the iterate of reverse pass k as Z = [Q_k | Qbar_k J]
// (m x 128, row-major; J reverses the column order). Per row it needs
//   t J     = Qbar_k J - Q_k Bt   (Bt = -2 P_k J)          and, for k > 1,
//   Q_{k-1} = 0 - Q_k Bq          (Bq = -R_k),
// two products of the same 64 values of Q_k with 64 x 64 matrices. Here each
// 128-row tile of Q_k is read and cut once and both products come out of one
// launch, in four groups of 32 output columns: g = 0, 1 the columns 0..31 and
// 32..63 of t J (in place over Qbar_k J), g = 2, 3 those of Q_{k-1} (into the
// next iterate).
//
// The split is the balanced fixed-point split of tc_common.cuh, keeping the
// seven leading digits of each value: row i of Q_k gets the scale
// sigma_i = 2^E_i > 2 max_k |q_ik|, column l of B the scale tau_l; the
// digits are exact BF16 numbers in [-64, 64], so x = sigma_i sum_{s<7} a_s
// 2^(-7(s+1)) up to 2^-49 sigma_i (the dropped digit and the rounding, of
// zero mean). Tile e of an accumulator sums the pairs (s, t) with s + t = e
// <= 6 over the 64 values: at most 7 * 64 * 64^2 < 2^21, exact in FP32.
// Per entry W = sum_e D_e 2^(42 - 7e) (below 2^61), folded pairwise in 32
// bits, and the product is sigma_i tau_l 2^-56 W: within about
// 2^-49 (sigma_i ||b_l||_1 + tau_l ||q_i||_1) + 64 * 7 * 2^-51 sigma_i tau_l of
// q_i^T b_l -- a perturbation of B of order 2^-49 ||B||, well inside the
// O(kappa u) error of the adjoint (the pairs s + t >= 7 not formed are of zero
// mean as well).
//
// Kernel layout: one 128-row tile in flight per CTA, 256 slicer threads plus
// a producer warp. Shared memory holds the tile's 7 digit planes (A operand,
// M = 128 rows, K = 64, K-major, no swizzle) and the 7 digit planes of all
// four groups of B (32 columns each), cut once per CTA. Tensor memory holds
// two accumulators of 7 tiles x 32 columns: the producer issues group g's
// MMAs (digit s of Q against the planes t = 0 .. 6 - s of the group, side by
// side, N = 32 (7 - s), from tensor column 32 s, so that the pair (s, t)
// lands in tile s + t; K steps of 16 values, of which only the first two for
// group 2: R_k is upper triangular) into accumulator g % 2 while the slicers
// read group g - 1 back, fold it, apply it and store it. Every wait has a time
// limit; past it the kernel records SCQR3_E_TIMEOUT, waits (bounded) for its
// own MMAs and frees its tensor memory.
#include "tc_common.cuh"

namespace scqr3 {

namespace tcb {

constexpr int ROWS = 128;
constexpr int K = 64;                     // contraction length: the 64 values of a row of Q_k
constexpr int PL = 7;                     // digit planes kept per value
constexpr int THREADS = 256;              // slicer threads (the producer warp comes on top)
constexpr uint32_t LBO = 128;             // K-direction core-matrix stride (bytes)
constexpr uint32_t SBO = 16 * K;          // 8-row (A) or 8-column (B) group stride: K / 8 core matrices
constexpr int APLANE = ROWS * K * 2;      // 16 KB: one digit plane of the tile
constexpr int BPLANE = 32 * K * 2;        // 4 KB: one digit plane of a group (32 columns)
constexpr int BGROUP = PL * BPLANE;       // 28 KB: a group's planes, side by side in N
constexpr uint32_t TACC = 256;            // tensor-memory columns per accumulator (7 tiles x 32 used)
constexpr int kNonFinite = 0x7FFFFFFF;    // row-scale marker of a row holding Inf or NaN
constexpr size_t SMEM = (size_t)PL * APLANE + 4 * (size_t)BGROUP;  // 224 KB
static_assert(SMEM + 1024 <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// Group g's MMAs: digit S of the tile (A) against planes t = 0 .. 6 - S of the
// group (B, N = 32 (7 - S)), into the accumulator from column 32 S; K step KK.
// The first MMA (S = 0, KK = 0) covers all 7 tiles and starts them.
template <int S, int KK, int KS>
__device__ __forceinline__ void issue(uint64_t adesc, uint64_t bdesc, uint32_t tmem, uint32_t idesc0) {
  constexpr uint32_t NS = 32 * (PL - S);
  constexpr uint64_t aoff = ((uint32_t)S * APLANE + KK * 2 * LBO) >> 4;
  constexpr uint64_t boff = (KK * 2 * LBO) >> 4;
  tc::mma(tmem + 32 * S, adesc + aoff, bdesc + boff, idesc0 | ((NS >> 3) << 17), (S > 0 || KK > 0) ? 1u : 0u);
  if constexpr (KK + 1 < KS) {
    issue<S, KK + 1, KS>(adesc, bdesc, tmem, idesc0);
  } else if constexpr (S + 1 < PL) {
    issue<S + 1, 0, KS>(adesc, bdesc, tmem, idesc0);
  }
}

// Eight values as their seven leading digit planes (one core-matrix row each).
__device__ __forceinline__ void cut7(const double* x, int E, uint8_t* dst, uint32_t plane) {
  unsigned long long M[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) M[r] = tc::biased56(x[r], E);
  uint4 w[8];
  tc::planes8(M, w);
#pragma unroll
  for (int s = 0; s < PL; ++s) *(uint4*)(dst + s * plane) = w[s];
}

// W 2^e2 as a double from the bits of W (integer operations): W's leading 53
// bits (truncated), exponent 63 - clz(|W|) + e2; zero below the normal range.
__device__ __forceinline__ double scaled_int(long long W, int e2) {
  const unsigned long long sgn = (unsigned long long)W & 0x8000000000000000ull;
  unsigned long long a = W < 0 ? 0ull - (unsigned long long)W : (unsigned long long)W;
  const int lz = __clzll((long long)a);
  a <<= (lz & 63);
  const int ex = 1023 + 63 - lz + e2;
  unsigned long long bits = sgn | ((unsigned long long)(ex < 2047 ? ex : 2047) << 52);
  if (ex < 2047) bits |= (a >> 11) & 0xFFFFFFFFFFFFFull;
  return (W == 0 || ex <= 0) ? 0.0 : __longlong_as_double((long long)bits);
}

// Barrier of the 256 slicer threads (id 1), returning whether any passed a
// non-zero pred.
__device__ __forceinline__ int slicers_any(int pred) {
  int r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.b32 %0, 1, 0, q;\n}"
               : "=r"(r) : "r"(pred), "r"(THREADS) : "memory");
  return r;
}

}  // namespace tcb

// z: the iterate [Q_k | Qbar_k J], m x 128 (ldz = 128); zn: the next one
// (its left half receives Q_{k-1} when groups == 4); bt, bq: the dense 64 x 64
// matrices -2 P_k J and -R_k (row stride ldb). groups: 4 (t J and Q_{k-1}) or
// 2 (t J only, pass 1).
__global__ void __launch_bounds__(tcb::THREADS + 32, 1)
tc_bwprod_kernel(double* z, double* zn, int64_t m, const double* __restrict__ bt, const double* __restrict__ bq,
                 int ldb, int groups, DevState* __restrict__ st, long long wait_ns) {
  using namespace tcb;
  using tc::smem_u32;
  constexpr int64_t LDZ = 2 * K;
  extern __shared__ __align__(16) uint8_t dsm[];
  uint8_t* abuf = dsm;                    // the tile's 7 planes
  uint8_t* bbuf = dsm + PL * APLANE;      // 4 groups x 7 planes
  __shared__ __align__(8) uint64_t afull;     // the tile's planes written (256 arrivals)
  __shared__ __align__(8) uint64_t mdone[2];  // MMAs of the accumulator's group done (commit)
  __shared__ __align__(8) uint64_t tfree[2];  // accumulator read back (256 arrivals)
  __shared__ uint32_t tslot;
  __shared__ int Eb[4 * 32];  // tau of group g, column c: 2^Eb[32 g + c]
  __shared__ int erow[ROWS];  // sigma of the tile's row r: 2^erow[r] (kNonFinite: the row holds Inf/NaN)
  __shared__ volatile int err_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == THREADS / 32;

  // column scales of the four groups (a column of Bt or Bq over its 64 rows)
  if (tid < 4 * 32) {
    const int g = tid >> 5, c = 32 * (g & 1) + (tid & 31);
    const double* b = g < 2 ? bt : bq;
    unsigned long long mx = 0;
    for (int k = 0; k < K; ++k) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(b[(int64_t)k * ldb + c]) &
                                   0x7FFFFFFFFFFFFFFFull;
      mx = mx > v ? mx : v;
    }
    Eb[tid] = tc::split_exp(mx);
  }
  if (tid == 0) {
    err_sh = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&afull)), "r"(THREADS));
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mdone[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&tfree[i])), "r"(THREADS));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  // B planes: group g, column c (32), K group kg (8 values)
  for (int u = tid; u < 4 * 32 * (K / 8); u += THREADS + 32) {
    const int g = u / (32 * (K / 8)), c = u % 32, kg = (u / 32) % (K / 8);
    const double* b = (g < 2 ? bt : bq) + 32 * (g & 1) + c;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = b[(int64_t)(8 * kg + q) * ldb];
    cut7(v, Eb[32 * g + c], bbuf + g * BGROUP + (c >> 3) * SBO + kg * LBO + (c & 7) * 16, BPLANE);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  // D F32, A and B BF16, both K-major, M = 128 (N set per MMA)
  const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);

  auto tile_row0 = [&](uint32_t j) -> int64_t {
    const int64_t r0 = ((int64_t)blockIdx.x + (int64_t)j * gridDim.x) * ROWS;
    return r0 < m ? r0 : -1;
  };

  uint32_t committed = 0;  // producer: groups whose MMAs were committed
  if (producer) {
    if (lane == 0) {
      const uint64_t ad = desc(smem_u32(abuf));
      for (uint32_t j = 0; tile_row0(j) >= 0; ++j) {
        if (!tc::wait_parity(smem_u32(&afull), j & 1, wait_ns) || err_sh) {
          err_sh = 1;
          break;
        }
        bool ok = true;
        for (int g = 0; g < groups; ++g) {
          const uint32_t u = j * groups + g, b = u & 1;
          // the previous group in this accumulator has been read back
          if (u >= 2 && (!tc::wait_parity(smem_u32(&tfree[b]), ((u >> 1) - 1) & 1, wait_ns) || err_sh)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t bd = desc(smem_u32(bbuf + g * BGROUP));
          if (g == 2)
            tcb::issue<0, 0, 2>(ad, bd, tmem + b * TACC, idesc0);
          else
            tcb::issue<0, 0, 4>(ad, bd, tmem + b * TACC, idesc0);
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(smem_u32(&mdone[b])) : "memory");
          committed = u + 1;
        }
        if (!ok) {
          err_sh = 1;
          break;
        }
      }
    }
  } else {
    // cut: row 16 warp + lane / 2, half lane % 2 (32 values: columns 32 h ..)
    const int rc = 16 * warp + (lane >> 1), hc = lane & 1;
    // read-back: tensor lane / row 32 (warp % 4) + lane, columns 16 (warp / 4) .. of the group
    const int rr = 32 * (warp & 3) + lane, hr = warp >> 2;
    const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    uint8_t* arow = abuf + (rc >> 3) * SBO + (rc & 7) * 16;
    for (uint32_t j = 0;; ++j) {
      const int64_t row0 = tile_row0(j);
      if (slicers_any(row0 < 0 || err_sh)) break;
      const int rows = (int)((m - row0) < ROWS ? (m - row0) : ROWS);
      // this thread's 32 values of Q_k (zeros past m), the row's scale from both halves
      double v[32];
      {
        const bool ok = rc < rows;
        const double* src = z + (row0 + (ok ? rc : 0)) * LDZ + 32 * hc;
        if (ok) {
#pragma unroll
          for (int c = 0; c < 32; c += 4)
            asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(v[c]), "=d"(v[c + 1]), "=d"(v[c + 2]), "=d"(v[c + 3]) : "l"(src + c) : "memory");
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c) v[c] = 0.0;
        }
      }
      unsigned long long mx = 0;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[c]) & 0x7FFFFFFFFFFFFFFFull;
        mx = mx > b ? mx : b;
      }
      {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, 1);
        mx = mx > o ? mx : o;
      }
      const bool finite_c = (mx >> 52) != 0x7FF;
      const int Ec = finite_c ? tc::split_exp(mx) : 0;
      // the previous tile's MMAs are complete: its last group was read back
#pragma unroll
      for (int kh = 0; kh < 4; ++kh) cut7(v + 8 * kh, Ec, arow + (4 * hc + kh) * LBO, APLANE);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&afull)) : "memory");
      // the row's scale for the read-back threads (another mapping of rows to
      // threads; read after the group loop's first barrier)
      if (hc == 0) erow[rc] = finite_c ? Ec : kNonFinite;
      bool failed = false;
      int Erow = 0;
      bool finite_r = true;
      for (int g = 0; g < groups; ++g) {
        const uint32_t u = j * groups + g, b = u & 1;
        const int col0 = 32 * (g & 1) + 16 * hr;  // first output column of this thread
        const bool rok = rr < rows;
        double x[16];
        double* dst = (g < 2 ? z + K : zn) + (row0 + (rok ? rr : 0)) * LDZ + col0;
        if (g < 2 && rok) {
#pragma unroll
          for (int c = 0; c < 16; c += 4)
            asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(x[c]), "=d"(x[c + 1]), "=d"(x[c + 2]), "=d"(x[c + 3]) : "l"(dst + c) : "memory");
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) x[c] = 0.0;
        }
        const bool ok = tc::wait_parity(smem_u32(&mdone[b]), (u >> 1) & 1, wait_ns);
        if (slicers_any(!ok)) {
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (g == 0) {
          const int e = erow[rr];
          finite_r = e != kNonFinite;
          Erow = finite_r ? e : 0;
        }
        constexpr uint32_t C129 = 0x4B400000u * 129u;  // mod 2^32
#pragma unroll
        for (int c4 = 0; c4 < 16; c4 += 4) {
          uint32_t t[PL][4];
#pragma unroll
          for (int e = 0; e < PL; ++e) tc::ld4(tq + b * TACC + 32 * e + 16 * hr + c4, t[e]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t w[PL];
#pragma unroll
            for (int e = 0; e < PL; ++e) w[e] = __float_as_uint(__uint_as_float(t[e][q]) + 12582912.0f);
            const long long p01 = (int32_t)(w[0] * 128u + w[1] - C129), p23 = (int32_t)(w[2] * 128u + w[3] - C129);
            const long long p45 = (int32_t)(w[4] * 128u + w[5] - C129);
            const long long d6 = (int32_t)(w[6] - 0x4B400000u);
            const long long W = (long long)(((unsigned long long)p01 << 35) + ((unsigned long long)p23 << 21) +
                                            ((unsigned long long)p45 << 7)) + d6;
            const int l = 32 * g + 16 * hr + c4 + q;  // Eb index of the output column
            x[c4 + q] = x[c4 + q] - scaled_int(W, Erow + Eb[l] - 56);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&tfree[b])) : "memory");
        if (rok) {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (!finite_r) x[c] = (double)NAN;
#pragma unroll
          for (int c = 0; c < 16; c += 4)
            asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};"
                         :: "l"(dst + c), "d"(x[c]), "d"(x[c + 1]), "d"(x[c + 2]), "d"(x[c + 3]) : "memory");
        }
      }
      if (failed) {
        err_sh = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (err_sh) {
    atomicCAS(&st->status, SCQR3_OK, SCQR3_E_TIMEOUT);
    // the MMAs already issued finish (bounded) before the memory goes away
    if (producer && lane == 0 && committed > 0) {
      const uint32_t u = committed - 1;
      tc::wait_parity(smem_u32(&mdone[u & 1]), (u >> 1) & 1, tc::kWaitNs);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// ---- host side ----------------------------------------------------------------------------

bool tc_bwprod_supported(int n) { return n == 64; }

// The products of reverse pass k at n = 64: t J in place over the right half
// of z and, when both (k > 1), Q_{k-1} into the left half of zn.
void launch_tc_bwprod(int sms, cudaStream_t s, double* z, double* zn, int64_t m, const double* bt,
                      const double* bq, int ldb, bool both, DevState* st, long long wait_ns) {
  cudaFuncSetAttribute(tc_bwprod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcb::SMEM);
  const int64_t tiles = (m + tcb::ROWS - 1) / tcb::ROWS;
  const int grid = (int)(tiles < sms ? (tiles < 1 ? 1 : tiles) : sms);
  tc_bwprod_kernel<<<grid, tcb::THREADS + 32, tcb::SMEM, s>>>(z, zn, m, bt, bq, ldb, both ? 4 : 2, st, wait_ns);
}

}  // namespace scqr3
