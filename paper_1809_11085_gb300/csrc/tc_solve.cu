// tc_solve.cu -- the row-wise substitution Q := X R^{-1} (Eq. backward2) for
// n <= 128 with its off-diagonal blocks on the tensor cores.
//
// Blocking R in diagonal blocks of w = 16 or 32 columns splits the
// substitution of each row x^T = [x_0^T .. x_{nb-1}^T] into, for J = 0, 1, ..:
//   y_J^T = x_J^T R_JJ^{-1},   x_K^T := x_K^T - y_J^T R_JK  (K > J):
// the same terms forward substitution over columns takes, grouped by block.
// The triangular solves run in FP64 on the pass kernel. The products
// y_J^T R_JK -- most of the substitution's flops, and dense contractions --
// run here on the BF16 tensor cores (one launch per 32 columns to update;
// written below as Y = Y_J with k = w columns and R01 = the updated columns
// of R_JK) through the exact digit split of the Gram kernel:
//  * row i of Y gets the scale sigma_i = 2^E_i > 2 max_k |y_ik| (its own k
//    values), column l of R01 the scale tau_l = 2^E_l > 2 max_k |r_kl|;
//  * both are rounded to 2^-56 of their scale and cut into eight signed
//    digits in [-64, 64] (the balanced split of tc_common.cuh); digit products
//    are exact in FP32, and tile e of tensor memory sums the pairs (s, t) with
//    s + t = e over the k columns: at most 8 * 32 * 64^2 = 2^20, exact;
//  * per entry the tile sums fold exactly into
//    W = sum_e D_e 2^{7(7-e)-7} = 2^21 U + floor(T / 2^7) with
//    U = sum_{e<=3} D_e 2^{7(3-e)} and T = sum_{e>=4} D_e 2^{7(7-e)}
//    (truncation below 2^-56 of sigma_i tau_l), formed pairwise in 32 bits:
//    |D_e| <= 2^20, so D_e + 1.5 2^23 is exact in FP32 with bit pattern
//    b_e = 0x4B400000 + D_e, and b_e 2^7 + b_{e+1} - 129 * 0x4B400000 =
//    D_e 2^7 + D_{e+1} (mod 2^32; below 2^28 in magnitude); then W =
//    P01 2^35 + P23 2^21 + P45 2^7 + floor(P67 / 2^7);
//    sigma_i tau_l 2^-56 W is assembled as a double from the bits of W
//    (integer operations), and x'_il = x_il - that, one FP64 subtraction per
//    entry.
// The computed product differs from y_i^T r_l by less than
// 2^-57 (sigma_i ||r_l||_1 + tau_l ||y_i||_1) + k 2^-55 sigma_i tau_l (the
// rounding of each value, and the digit pairs s + t > 7 not formed, both of
// zero mean), plus 2^-56 sigma_i tau_l for the fold: at most about
// 4 k u ||y_i|| ||r_l||, a perturbation of R01 of norm O(u ||R||),
// the order of the row-wise backward error of FP64 substitution
// (Eq. backward2) on which the analysis of Sec. 3 rests.
//
// Kernel layout: 2 slots of 256 threads (one 128-row tile each; threads r and
// r + 128 of a slot share the tile's row r and tensor-memory lane r, each with
// half of the row) plus a producer warp. A slot stages its tile of Y in shared
// memory (coalesced loads, rows padded to an odd number of words; for k = 16
// the next tile is prefetched by cp.async into a second buffer), each thread
// cuts its half row into 8 digit planes (A operand, M = 128 rows, K = k,
// K-major, no swizzle: core matrices of 8 rows x 16 bytes, K step 128 B,
// 8-row step 16 k bytes) and the slot signals the producer. The producer
// issues one MMA per digit s and K step, digit s of Y against the planes
// t = 0 .. 7 - s of R01 side by side (M = 128, N = 32 (8 - s), K = 16), into
// the slot's 256 columns of tensor memory from column 32 s, so that the pair
// (s, t) lands in tile e = s + t, and commits them to the slot's mbarrier.
// Meanwhile the slot stages its tile of x; then each thread reads its row's
// sums back (tcgen05.ld 32x32b), updates its row of x in shared memory, and the
// slot writes the tile out coalesced. While one slot waits for its MMAs the
// other cuts or applies. Every wait has an iteration limit; past it the kernel
// records SCQR3_E_TIMEOUT, waits (bounded) for its own MMAs and copies and
// frees its tensor memory.
#include "tc_common.cuh"

namespace scqr3 {

namespace tcs {

constexpr int ROWS = 128;                // rows per tile
constexpr int SLOTS = 2;                 // tiles in flight per CTA
constexpr int SLOT_THREADS = 2 * ROWS;  // two threads per row: each cuts and applies half of it
constexpr int THREADS = SLOT_THREADS * SLOTS;  // slot threads (the producer warp comes on top)
constexpr uint32_t LBO = 128;            // K-direction core-matrix stride
constexpr uint32_t TSLOT = 256;          // tensor-memory columns per slot: 8 tiles x 32
constexpr int YLD = 33;                  // row stride (doubles) of a slot's staged tile: conflict-free rows
constexpr int YSLOT = ROWS * YLD * 8;    // 33 KB: the slot's Y tile, then its x tile (<= 32 columns each)

// Geometry for a block of K = 16 or 32 columns (the contraction length).
// K = 16 leaves room to prefetch each slot's next tile of Y (two buffers per
// slot, filled by cp.async while the current tile is cut, multiplied and
// applied).
template <int K>
struct UGeo {
  static constexpr uint32_t SBO = 16 * K;     // 8-row (A) or 8-column (B) group stride: K / 8 core matrices
  static constexpr int APLANE = ROWS * K * 2;  // per digit plane of a tile (8 KB for K = 32)
  static constexpr int ASLOT = 8 * APLANE;     // the slot's 8 planes
  static constexpr int BPLANE = 32 * K * 2;    // per digit plane of R_JK (32 columns)
  static constexpr bool PREF = K == 16;        // prefetch the next tile of Y
  static constexpr int YPLD = K + 1;           // row stride of a prefetch buffer: conflict-free rows
  static constexpr size_t YPRE = PREF ? SLOTS * 2 * (size_t)ROWS * YPLD * 8 : 0;
  static constexpr size_t SMEM =
      SLOTS * (size_t)ASLOT + 8 * (size_t)BPLANE + SLOTS * (size_t)YSLOT + YPRE + 1024;
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Barrier among the 256 threads of a slot (ids 1, 2), returning whether any
// of them passed a non-zero `pred`: decisions that must be uniform in the slot.
__device__ __forceinline__ int slot_any(int slot, int pred) {
  int r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.b32 %0, 1, 0, q;\n}"
               : "=r"(r) : "r"(pred), "r"(1 + slot), "r"(SLOT_THREADS) : "memory");
  return r;
}
__device__ __forceinline__ void slot_sync(int slot) {
  asm volatile("bar.sync %0, %1;" :: "r"(1 + slot), "r"(SLOT_THREADS) : "memory");
}

template <int K>
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(UGeo<K>::SBO >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// The MMAs of a tile (16 for K = 32, 8 for K = 16): digit s of Y (A) against the planes t = 0 .. 7 - s
// of R01 side by side (B, N = 32 (8 - s): the planes are contiguous, 32
// columns each), accumulating at tensor-memory column 32 s, so that the pair
// (s, t) lands in tile e = s + t; K step kk. Descriptor offsets stay inside
// the start-address field (all of shared memory lies below 256 KB).
template <int K, int S, int KK>
__device__ __forceinline__ void issue(uint64_t adesc, uint64_t bdesc, uint32_t tmem, uint32_t idesc0) {
  constexpr uint32_t NS = 32 * (8 - S);
  constexpr uint64_t aoff = ((uint32_t)S * UGeo<K>::APLANE + KK * 2 * LBO) >> 4;
  constexpr uint64_t boff = (KK * 2 * LBO) >> 4;
  tc::mma(tmem + 32 * S, adesc + aoff, bdesc + boff, idesc0 | ((NS >> 3) << 17), (S > 0 || KK > 0) ? 1u : 0u);
  if constexpr (KK + 1 < K / 16) {
    issue<K, S, KK + 1>(adesc, bdesc, tmem, idesc0);
  } else if constexpr (S < 7) {
    issue<K, S + 1, 0>(adesc, bdesc, tmem, idesc0);
  }
}

// W 2^e2 as a double, built from the bits of W with integer operations (the
// FP64 pipe, the scarce one, is left for the update itself): W's leading 53
// bits (truncated: relative error below 2^-52), exponent 63 - clz(|W|) + e2.
// Zero for W = 0 or a value below the normal range (an update below 2^-1022),
// +-Inf above it.
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

}  // namespace tcs

// The diagonal blocks R_JJ (w = 16 or 32 columns each, the last one n - w J
// wide) of the packed np x np R_k, each packed 32 x 32 (16 x 16 when at most
// 16 wide) at rdiag + J * pk_size(32); the padding of R_k is the identity,
// and so is theirs.
__global__ void tc_split_r_kernel(const double* __restrict__ rk, int np, int n, int w, int pass,
                                  const DevState* __restrict__ st, double* __restrict__ rdiag) {
  if (!st->run_trsm[pass]) return;
  const int nb = (n + w - 1) / w;
  for (int e = threadIdx.x; e < nb * 32 * 32; e += blockDim.x) {
    const int J = e >> 10, j = (e >> 5) & 31, k = e & 31;
    const int wj = n - w * J < w ? n - w * J : w;
    const int npj = wj <= 16 ? 16 : 32;
    if (k < j || k >= npj) continue;
    rdiag[J * pk_size(32) + pk_idx(npj, j, k)] = rk[pk_idx(np, w * J + j, w * J + k)];
  }
}

// x' = x - Y R01 for rows [0, m): y holds Y (K = 16 or 32 columns, the first
// ky of them read, the rest taken as zero), x1 and q1 the n1 <= N columns to
// update of the pass's input and output (they may be the same memory; x1 null:
// x = 0); R01 is rows r0 .. r0 + K - 1, columns c0 .. c0 + n1 - 1 of R_k,
// packed np x np (ldb = 0), or of a dense row-major matrix with row stride ldb
// (ldb > 0; the adjoint's products).
template <int K, int N>
__global__ void __launch_bounds__(tcs::THREADS + 32, 1)
tc_update_kernel(const double* __restrict__ y, int64_t ldy, const double* x1, int64_t ldx, double* q1, int64_t ldq,
                 int64_t m, int n1, int pass, const double* __restrict__ rk, int np, int r0, int c0, int ldb, int ky,
                 DevState* __restrict__ st, long long wait_ns) {
  using namespace tcs;
  using tc::smem_u32;
  constexpr uint32_t SBO = UGeo<K>::SBO;
  constexpr int APLANE = UGeo<K>::APLANE, ASLOT = UGeo<K>::ASLOT, BPLANE = UGeo<K>::BPLANE;
  if (!st->run_trsm[pass]) return;
  extern __shared__ uint8_t dsm[];
  uint8_t* abuf = (uint8_t*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  uint8_t* bbuf = abuf + SLOTS * ASLOT;
  double* ystage = (double*)(bbuf + 8 * BPLANE);
  __shared__ __align__(8) uint64_t pfull[SLOTS];  // A planes of the slot's tile written (256 arrivals)
  __shared__ __align__(8) uint64_t mdone[SLOTS];  // MMAs of the slot's tile done (tcgen05.commit)
  __shared__ uint32_t tslot;
  __shared__ int Eb[32];  // tau_l = 2^Eb[l]
  __shared__ unsigned long long mxs[SLOTS][2][ROWS];  // K = 32: partial row maxima of the two half rows
  __shared__ volatile int err_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == THREADS / 32;
  const int slot = (warp >> 3) & 1;
  const int tis = tid & (SLOT_THREADS - 1);  // thread within the slot
  const int r = tis & (ROWS - 1);  // tile row and tensor-memory lane (warp w serves lanes 32 (w % 4) ..)
  const int hf = tis >> 7;         // which half of the row: K groups hf K/16 ..; columns N/2 hf ..
  auto bval = [&](int k, int l) -> double {  // entry (k, l) of R01
    return ldb > 0 ? rk[(int64_t)(r0 + k) * ldb + c0 + l] : rk[pk_idx(np, r0 + k, c0 + l)];
  };

  // column scales of R01 (columns >= n1: zero)
  if (tid < 32) {
    unsigned long long mx = 0;
    if (tid < n1)
      for (int k = 0; k < K; ++k) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(bval(k, tid)) & 0x7FFFFFFFFFFFFFFFull;
        mx = mx > b ? mx : b;
      }
    Eb[tid] = tc::split_exp(mx);
  }
  if (tid == 0) {
    err_sh = 0;
    for (int g = 0; g < SLOTS; ++g) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&pfull[g])), "r"(SLOT_THREADS));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mdone[g])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  // R_JK digit planes (B operand: 32 columns, zero past n1, x K rows, K-major)
  for (int u = tid; u < 32 * (K / 8); u += THREADS + 32) {
    const int l = u & 31, kg = u >> 5;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = l < n1 ? bval(8 * kg + q, l) : 0.0;
    tc::cut8(v, Eb[l], bbuf + (l >> 3) * SBO + kg * LBO + (l & 7) * 16, BPLANE);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  // D F32, A and B BF16, both K-major, M = 128 (N set per MMA)
  const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);

  // this CTA's tiles: ordinal k is tile blockIdx.x + k gridDim.x; slot k % 2
  auto tile_row0 = [&](uint32_t k) -> int64_t {
    const int64_t r0 = ((int64_t)blockIdx.x + (int64_t)k * gridDim.x) * ROWS;
    return r0 < m ? r0 : -1;
  };

  uint32_t committed = 0;
  if (producer) {
    if (lane == 0) {
      for (uint32_t k = 0; tile_row0(k) >= 0; ++k) {
        const int g = k & 1;
        if (!tc::wait_parity(smem_u32(&pfull[g]), (k >> 1) & 1, wait_ns) || err_sh) {
          err_sh = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue<K, 0, 0>(desc<K>(smem_u32(abuf + g * ASLOT)), desc<K>(smem_u32(bbuf)), tmem + g * TSLOT, idesc0);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&mdone[g])) : "memory");
        committed = k + 1;
      }
    }
  } else {
    constexpr bool PREF = UGeo<K>::PREF;
    constexpr int YPLD = UGeo<K>::YPLD;
    uint8_t* arow = abuf + slot * ASLOT + (r >> 3) * SBO + (r & 7) * 16;
    const uint32_t tq = tmem + slot * TSLOT + ((uint32_t)(32 * (warp & 3)) << 16);
    double* ys = ystage + slot * (ROWS * YLD);  // the slot's staged tile: Y (without prefetch), then x / x'
    double* ypre = ystage + SLOTS * (ROWS * YLD) + slot * 2 * (ROWS * YPLD);  // PREF: two Y buffers
    // PREF: copy the Y rows of the tile at row r0n into buf asynchronously
    // (zeros past m; nothing for r0n < 0), as one cp.async group
    auto prefetch_y = [&](int64_t r0n, double* buf) {
      if (r0n >= 0) {
        constexpr int IT = ROWS * K / SLOT_THREADS;
#pragma unroll
        for (int it = 0; it < IT; ++it) {
          const int rr = (tis + SLOT_THREADS * it) / K, c = tis % K;
          const bool ok = r0n + rr < m && c < ky;
          const double* g = ok ? y + (r0n + rr) * ldy + c : y;
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;"
                       :: "r"(smem_u32(buf + rr * YPLD + c)), "l"(g), "r"(ok ? 8 : 0) : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (PREF) prefetch_y(tile_row0(slot), ypre);
    // K = 32: rows of Y start on 32-byte boundaries (vector loads of half rows)
    const bool yvec = ((uintptr_t)y & 31) == 0 && (ldy & 3) == 0;
    for (uint32_t j = 0;; ++j) {
      const int64_t row0 = tile_row0(2 * j + slot);
      if (slot_any(slot, row0 < 0 || err_sh)) break;
      const int rows = (int)((m - row0) < ROWS ? (m - row0) : ROWS);
      // the tile's rows of x into ys by asynchronous copies (zeros past m, past
      // n1 and for x1 null), in flight while Y is cut and multiplied (ys is
      // free: the previous tile's stores from it ended at the loop's last barrier)
      {
        constexpr int IT = ROWS * N / SLOT_THREADS;
        const int c = tis % N;
#pragma unroll
        for (int it = 0; it < IT; ++it) {
          const int rr = (tis + SLOT_THREADS * it) / N;
          const bool ok = x1 && rr < rows && c < n1;
          const double* g = ok ? x1 + (row0 + rr) * ldx + c : y;
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;"
                       :: "r"(smem_u32(ys + rr * YLD + c)), "l"(g), "r"(ok ? 8 : 0) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      unsigned long long mx = 0;
      bool finite;
      int E;
      if constexpr (PREF) {
        // the next tile of this slot into the other Y buffer; copy groups
        // pending, oldest first: Y of this tile, x of this tile, Y of the next
        prefetch_y(tile_row0(2 * (j + 1) + slot), ypre + ((j + 1) & 1) * (ROWS * YPLD));
        asm volatile("cp.async.wait_group 2;" ::: "memory");
        slot_sync(slot);
        const double* yb = ypre + (j & 1) * (ROWS * YPLD);
        // the row's scale from all K values; this thread cuts its half
#pragma unroll
        for (int c = 0; c < K; ++c) {
          const unsigned long long b =
              (unsigned long long)__double_as_longlong(yb[r * YPLD + c]) & 0x7FFFFFFFFFFFFFFFull;
          mx = mx > b ? mx : b;
        }
        finite = (mx >> 52) != 0x7FF;
        E = finite ? tc::split_exp(mx) : 0;
#pragma unroll
        for (int kh = 0; kh < K / 16; ++kh) {
          const int kg = (K / 16) * hf + kh;
          double v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = yb[r * YPLD + 8 * kg + q];
          tc::cut8(v, E, arow + kg * LBO, APLANE);
        }
      } else {
        // this thread's half row of Y (columns 16 hf .. 16 hf + 15: one
        // 128-byte line), straight from global memory; the row's scale from
        // both halves (partial maxima exchanged through shared memory)
        static_assert(K == 32, "half rows of 16 values");
        const bool rok = r < rows;
        const double* yr = y + (row0 + (rok ? r : 0)) * ldy + 16 * hf;
        double yv[16];
        if (yvec && rok && 16 * hf + 16 <= ky) {  // four 32-byte loads
#pragma unroll
          for (int c = 0; c < 16; c += 4)
            asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(yv[c]), "=d"(yv[c + 1]), "=d"(yv[c + 2]), "=d"(yv[c + 3]) : "l"(yr + c) : "memory");
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) yv[c] = (rok && 16 * hf + c < ky) ? yr[c] : 0.0;
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const unsigned long long b = (unsigned long long)__double_as_longlong(yv[c]) & 0x7FFFFFFFFFFFFFFFull;
          mx = mx > b ? mx : b;
        }
        mxs[slot][hf][r] = mx;
        slot_sync(slot);
        const unsigned long long m0 = mxs[slot][0][r], m1 = mxs[slot][1][r];
        mx = m0 > m1 ? m0 : m1;
        finite = (mx >> 52) != 0x7FF;
        E = finite ? tc::split_exp(mx) : 0;
        tc::cut8(yv, E, arow + (2 * hf) * LBO, APLANE);
        tc::cut8(yv + 8, E, arow + (2 * hf + 1) * LBO, APLANE);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&pfull[slot])) : "memory");
      // this thread's copies of x done (the barrier below makes all of them visible)
      if constexpr (PREF) asm volatile("cp.async.wait_group 1;" ::: "memory");
      else asm volatile("cp.async.wait_group 0;" ::: "memory");
      const bool ok = tc::wait_parity(smem_u32(&mdone[slot]), j & 1, wait_ns);
      if (slot_any(slot, !ok)) {  // also: the tile of x is complete
        err_sh = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      // four columns at a time: the 8 tile sums of each (one wait for all
      // 32 words), folded pairwise in 32 bits (see the header)
      constexpr uint32_t C129 = 0x4B400000u * 129u;  // mod 2^32
#pragma unroll
      for (int c4 = hf * (N / 2); c4 < (hf + 1) * (N / 2); c4 += 4) {
        uint32_t t[8][4];
#pragma unroll
        for (int e = 0; e < 8; ++e) tc::ld4(tq + 32 * e + c4, t[e]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t b[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) b[e] = __float_as_uint(__uint_as_float(t[e][q]) + 12582912.0f);
          const long long p01 = (int32_t)(b[0] * 128u + b[1] - C129), p23 = (int32_t)(b[2] * 128u + b[3] - C129);
          const long long p45 = (int32_t)(b[4] * 128u + b[5] - C129), p67 = (int32_t)(b[6] * 128u + b[7] - C129);
          const long long W = (long long)(((unsigned long long)p01 << 35) + ((unsigned long long)p23 << 21) +
                                          ((unsigned long long)p45 << 7)) + (p67 >> 7);
          const int l = c4 + q;
          const double upd = scaled_int(W, E + Eb[l] - 56);  // sigma_i tau_l 2^-56 W
          ys[r * YLD + l] = finite ? ys[r * YLD + l] - upd : (double)NAN;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      slot_sync(slot);
      {
        constexpr int IT = ROWS * N / SLOT_THREADS;
        const int c = tis % N;
#pragma unroll
        for (int it = 0; it < IT; ++it) {
          const int rr = (tis + SLOT_THREADS * it) / N;
          if (rr < rows && c < n1) q1[(row0 + rr) * ldq + c] = ys[rr * YLD + c];
        }
      }
      slot_sync(slot);  // the tile is out before the next one is staged
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy into shared memory outlives the CTA
  __syncthreads();
  if (err_sh) {
    atomicCAS(&st->status, SCQR3_OK, SCQR3_E_TIMEOUT);
    // let the MMAs already issued finish (bounded) before the memory goes away
    if (producer && lane == 0 && committed > 0) {
      const uint32_t k = committed - 1;
      tc::wait_parity(smem_u32(&mdone[k & 1]), (k >> 1) & 1, tc::kWaitNs);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// ---- host side ----------------------------------------------------------------------------

cudaError_t tc_solve_setup() {
  cudaError_t e = cudaFuncSetAttribute(tc_update_kernel<16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tcs::UGeo<16>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_update_kernel<16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tcs::UGeo<16>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_update_kernel<32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tcs::UGeo<32>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_update_kernel<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tcs::UGeo<32>::SMEM);
  return e;
}

void launch_tc_split_r(cudaStream_t s, const double* rk, int np, int n, int w, int pass, const DevState* st,
                       double* rdiag) {
  tc_split_r_kernel<<<1, 256, 0, s>>>(rk, np, n, w, pass, st, rdiag);
}

// x1' = x1 - Y R_JK over rows [0, m); Y has k = 16 or 32 columns (the first
// ky read), n1 in 1 .. 32 columns are updated; R_JK at (r0, c0) of R_k (packed
// np; ldb > 0: a dense matrix with row stride ldb).
void launch_tc_update(int sms, cudaStream_t s, int k, const double* y, int64_t ldy, const double* x1,
                      int64_t ldx, double* q1, int64_t ldq, int64_t m, int n1, int pass, const double* rk, int np,
                      int r0, int c0, int ldb, int ky, DevState* st, long long wait_ns) {
  const int64_t tiles = (m + tcs::ROWS - 1) / tcs::ROWS;
  const int grid = (int)(tiles < sms ? (tiles < 1 ? 1 : tiles) : sms);
#define SCQR3_UPD(KV, NV)                                                                                   \
  tc_update_kernel<KV, NV><<<grid, tcs::THREADS + 32, tcs::UGeo<KV>::SMEM, s>>>(y, ldy, x1, ldx, q1, ldq, m, n1, \
                                                                             pass, rk, np, r0, c0, ldb, ky, st, wait_ns)
  if (k == 16) {
    if (n1 <= 16) SCQR3_UPD(16, 16);
    else SCQR3_UPD(16, 32);
  } else {
    if (n1 <= 16) SCQR3_UPD(32, 16);
    else SCQR3_UPD(32, 32);
  }
#undef SCQR3_UPD
}

}  // namespace scqr3
