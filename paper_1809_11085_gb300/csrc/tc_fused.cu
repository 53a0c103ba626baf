// tc_fused.cu -- one pass's row-wise substitution Q := X R_k^{-1}
// (Eq. backward2) for 16 < n <= 64 in a single sweep over the rows: every row
// is read once and written once, and the column maxima of the result (the
// scales of the next tensor-core Gram matrix) come out of the same sweep.
//
// The substitution of a row x^T groups its terms by 16-column blocks of R
// (as in tc_solve.cu), recursively halved: for n <= 64 (NP = 64)
//   y_0 = x_0 R_00^-1;        x_1 -= y_0 R_01               (K = 16, N = 16)
//   y_1 = x_1 R_11^-1;        [x_2 x_3] -= [y_0 y_1] R_{01,23}  (K = 32, N = 32)
//   y_2 = x_2 R_22^-1;        x_3 -= y_2 R_23               (K = 16, N = 16)
//   y_3 = x_3 R_33^-1
// and for n <= 32 (NP = 32) the first two lines. The triangular solves of the
// 16 x 16 diagonal blocks run in FP64, one thread per row, with the row held
// in registers; the products with the off-diagonal blocks run on the BF16
// tensor cores through the exact digit split of tc_solve.cu (a scale per row
// of Y -- here the common one of all K values multiplied, y_0 and y_1 together
// in the middle update -- and per column of R_JK; eight signed 7-bit digits;
// tile e of tensor memory sums the digit pairs with s + t = e, at most
// 8 * 32 * 127^2 < 2^22 per entry, exact in FP32; int64 folding; one FP64
// subtraction per updated entry). Error: as for tc_solve.cu, a perturbation
// of R_JK of norm O(u ||R||) per row, the form of the row-wise backward error
// that the analysis of Sec. 3 assumes.
//
// FP64 work per row: 4 (16 * 15 / 2 FMAs + 16 multiplies) + 64 subtractions
// = 608 at NP = 64, against 2112 for the unblocked substitution.
//
// Layout: one CTA per SM, two slots of 128 threads; a slot owns one 128-row
// tile at a time (thread r of the slot holds row r, which is tensor-memory
// lane r: warp w of the slot reads lane quadrant w). Each warp loads its 32
// rows with cp.async into the slot's 64 KB buffer (a 128-byte XOR swizzle
// per 16-column box, so that a thread reading its own row with 16-byte loads
// meets no bank conflict), then the thread keeps its row in registers. For an
// update the slot cuts its rows' K values into 8 digit planes in the same
// buffer (A operand: M = 128, K-major, no swizzle), thread 0 of the slot issues
// one MMA per digit s and K step (digit s of Y against the planes t = 0 .. 7 - s
// of R_JK side by side: N = N_u (8 - s), accumulating from tensor-memory column
// N_u s, so the pair (s, t) lands in tile e = s + t) into the slot's 256
// columns and commits them to the slot's mbarrier; every thread then reads its
// row's tile sums back (tcgen05.ld 32x32b) and applies them. While one slot
// cuts, waits or applies, the other keeps the FP64 pipe busy. The finished
// rows go out through the buffer, coalesced, and each lane keeps the largest
// |q_ij| of the columns it stores. Waits are bounded in time; a wait that
// runs out records SCQR3_E_TIMEOUT, and before the tensor memory is freed the
// CTA waits (bounded) for its last MMAs.
#include "tc_common.cuh"

namespace scqr3 {

namespace tcf {

constexpr int ROWS = 128;              // rows per tile = tensor-memory lanes
constexpr int SLOTS = 3;               // tiles in flight per CTA, 128 threads each
constexpr int THREADS = ROWS * SLOTS;
constexpr uint32_t LBO = 128;          // K-direction core-matrix stride
constexpr uint32_t TSLOT = 128;        // tensor-memory columns per slot: 8 tiles x 16 columns

// Off-diagonal products x[C0, C0 + 16) -= y[K0, K0 + K) R[K0.., C0..]: B planes
// at byte BOFF of the B area (8 planes of K x 16 BF16 digits), column
// exponents at EOFF.
struct Upd {
  int k0, K, c0, boff, eoff;
};
// NP = 64: U0 = y_0 R_01; U1a, U1b = [y_0 y_1] R_{01,2}, R_{01,3}; U2 = y_2 R_23.
// NP = 32: U0 only.
template <int NP> struct Plan;
template <> struct Plan<32> {
  static constexpr int NU = 1, BBYTES = 4096, NEB = 16;
};
template <> struct Plan<64> {
  static constexpr int NU = 4, BBYTES = 24576, NEB = 64;
};
template <int NP, int UI>
__host__ __device__ constexpr Upd plan() {
  return UI == 0 ? Upd{0, 16, 16, 0, 0}
       : UI == 1 ? Upd{0, 32, 32, 4096, 16}
       : UI == 2 ? Upd{0, 32, 48, 12288, 32}
                 : Upd{32, 16, 48, 20480, 48};
}

template <int NP> struct FGeo {
  static constexpr int NB = NP / 16;                               // diagonal blocks
  static constexpr int SBUF = NP == 64 ? 65536 : 32768;            // A planes of one update (K <= NP / 2)
  static constexpr size_t OFF_B = (size_t)SLOTS * SBUF;
  static constexpr size_t OFF_R = OFF_B + Plan<NP>::BBYTES;        // dense 16 x 16 diagonal blocks of R_k
  static constexpr size_t OFF_RINV = OFF_R + (size_t)NB * 256 * 8;  // 1 / r_jj
  static constexpr size_t SMEM = OFF_RINV + (size_t)NP * 8 + 1024;  // + alignment slack
  static_assert(SMEM + 512 <= 227 * 1024, "shared memory");
};

template <int K>
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)((16u * K) >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// The MMAs of one product: digit s of Y (A: plane s at s * 256 K bytes)
// against the B planes t = 0 .. 7 - s side by side, 16 (8 - s) columns from
// tensor column 16 s, so that the pair (s, t) lands in tile e = s + t; K step
// kk (two core matrices, 256 bytes, per K = 16).
template <int K, int S, int KK>
__device__ __forceinline__ void issue(uint64_t adesc, uint64_t bdesc, uint32_t tmem, uint32_t idesc0) {
  constexpr uint32_t NS = 16 * (8 - S);
  constexpr uint64_t aoff = ((uint32_t)S * (ROWS * K * 2) + KK * 2 * LBO) >> 4;
  constexpr uint64_t boff = (KK * 2 * LBO) >> 4;
  tc::mma(tmem + 16 * S, adesc + aoff, bdesc + boff, idesc0 | ((NS >> 3) << 17), (S > 0 || KK > 0) ? 1u : 0u);
  if constexpr (KK + 1 < K / 16) {
    issue<K, S, KK + 1>(adesc, bdesc, tmem, idesc0);
  } else if constexpr (S < 7) {
    issue<K, S + 1, 0>(adesc, bdesc, tmem, idesc0);
  }
}

// Barrier among the 128 threads of a slot (ids 1..SLOTS); the second form
// returns whether any of them passed a non-zero `pred` (slot-uniform decisions).
__device__ __forceinline__ void slot_sync(int slot) {
  asm volatile("bar.sync %0, %1;" :: "r"(1 + slot), "r"(ROWS) : "memory");
}
__device__ __forceinline__ int slot_any(int slot, int pred) {
  int r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.b32 %0, 1, 0, q;\n}"
               : "=r"(r) : "r"(pred), "r"(1 + slot), "r"(ROWS) : "memory");
  return r;
}

// W 2^e2 as a double from the bits of W (integer operations only): W's
// leading 53 bits (truncated), zero for W = 0 or below the normal range.
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

// y = h[OFF, OFF + 16) R_JJ^{-1} in place: forward substitution over the
// block's columns (multiply by the rounded reciprocal of r_jj); rb = the dense
// 16 x 16 block, ri = its 16 reciprocals (shared memory).
template <int OFF>
__device__ __forceinline__ void solve16(double (&h)[32], const double* __restrict__ rb,
                                        const double* __restrict__ ri) {
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    double rc;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(rc) : "r"(tc::smem_u32(ri + c)));
    const double y = h[OFF + c] * rc;
    h[OFF + c] = y;
#pragma unroll
    for (int c2 = c + 1; c2 < 16; ++c2) {
      // an explicit shared load: left to itself the compiler hoists the
      // block's R values into registers ahead of their use
      double rv;
      asm volatile("ld.shared.f64 %0, [%1];" : "=d"(rv) : "r"(tc::smem_u32(rb + c * 16 + c2)));
      h[OFF + c2] = fma(-y, rv, h[OFF + c2]);
    }
  }
}

// Per-slot state of the update pipeline.
struct SlotCtx {
  uint8_t* sbuf;     // the slot's A planes
  uint8_t* bb;       // B planes of the off-diagonal blocks
  const int* Eb;     // their column exponents
  uint32_t tmem;     // the slot's first tensor-memory column (lane 0)
  uint32_t tq;       // this thread's lane of it
  uint32_t mbar;     // the slot's MMA-completion mbarrier
  uint32_t idesc0;
  int slot, r;
  long long wait_ns;
};

// The scale exponent of h[0, K) and its digit planes (A operand, K-major) in
// the slot's buffer. Returns false for a non-finite row.
template <int K>
__device__ __forceinline__ bool cut_rows(const double (&h)[32], const SlotCtx& c, int& E) {
  unsigned long long mx = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(h[k]) & 0x7FFFFFFFFFFFFFFFull;
    mx = mx > b ? mx : b;
  }
  const bool finite = (mx >> 52) != 0x7FF;
  E = finite ? tc::split_exp(mx) : 0;
  slot_sync(c.slot);  // the slot's previous planes are consumed (its MMAs have completed)
  uint8_t* ar = c.sbuf + (c.r >> 3) * (16 * K) + (c.r & 7) * 16;
#pragma unroll
  for (int kg = 0; kg < K / 8; ++kg) tc::cut8(&h[8 * kg], E, ar + kg * LBO, ROWS * K * 2);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  return finite;
}

// Thread 0 of the slot issues product UI's MMAs (after the slot's barrier) and
// commits them to the slot's mbarrier.
template <int NP, int UI>
__device__ __forceinline__ void mma_product(const SlotCtx& c, uint32_t& commits) {
  constexpr Upd U = plan<NP, UI>();
  slot_sync(c.slot);  // planes written; the tensor-memory sums of the previous product read back
  if (c.r == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    issue<U.K, 0, 0>(desc<U.K>(tc::smem_u32(c.sbuf)), desc<U.K>(tc::smem_u32(c.bb + U.boff)), c.tmem, c.idesc0);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(c.mbar)
                 : "memory");
    ++commits;
  }
}

// Thread 0 waits for the slot's last commit; the barrier releases the slot.
// False (slot-uniformly) if the wait ran out.
__device__ __forceinline__ bool mma_wait(const SlotCtx& c, uint32_t& phase) {
  bool ok = true;
  if (c.r == 0) ok = tc::wait_parity(c.mbar, phase & 1, c.wait_ns);
  ++phase;
  if (slot_any(c.slot, !ok)) return false;
  asm volatile("tcgen05.fence::after_thread_sync;");
  return true;
}

// h[OFF, OFF + 16) -= the product just read back: per column, the 8 tile sums
// folded exactly into int64 and assembled as sigma_i tau_l 2^-56 W.
template <int OFF>
__device__ __forceinline__ void fold16(double (&h)[32], const SlotCtx& c, int E, bool finite, const int* eb) {
  constexpr unsigned long long BIAS = 0x4B400000ull * ((1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);
#pragma unroll
  for (int c4 = 0; c4 < 16; c4 += 4) {
    uint32_t v[8][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) tc::ld4(c.tq + 16 * e + c4, v[e]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // |D_e| <= 8 * 32 * 64^2 = 2^20: D_e + 1.5 2^23 is exact, with bit pattern 0x4B400000 + D_e
      // (the constant leaves with BIAS). U takes D_0..3 with weights 2^21, 2^14,
      // 2^7, 1; T takes D_4..7 with the same weights.
      unsigned long long Uu = 0, Tt = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const uint32_t b = __float_as_uint(__uint_as_float(v[e][q]) + 12582912.0f);
        const uint32_t w = 1u << (7 * (3 - (e & 3)));
        if (e < 4) Uu += (unsigned long long)b * w;
        else Tt += (unsigned long long)b * w;
      }
      const long long Us = (long long)(Uu - BIAS), Ts = (long long)(Tt - BIAS);
      const long long W = (Us << 21) + (Ts >> 7);  // 2^56 (y r) / (sigma tau), truncated
      const double upd = scaled_int(W, E + eb[c4 + q] - 56);
      h[OFF + c4 + q] = finite ? h[OFF + c4 + q] - upd : (double)NAN;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
}

// 32 columns [c0, c0 + 32) of the row into h (zeros past m and past n). vec:
// the half lies within n and starts on a 32-byte boundary (X 32-byte aligned,
// ldx a multiple of 4), so it moves as eight 256-bit loads.
__device__ __forceinline__ void load_half(double (&h)[32], const double* X, int64_t ldx, int64_t g, int64_t m,
                                          int c0, int n, bool vec) {
  const double* src = X + g * ldx + c0;
  if (g >= m) {
#pragma unroll
    for (int c = 0; c < 32; ++c) h[c] = 0.0;
  } else if (vec) {
#pragma unroll
    for (int c = 0; c < 32; c += 4)
      asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                   : "=d"(h[c]), "=d"(h[c + 1]), "=d"(h[c + 2]), "=d"(h[c + 3]) : "l"(src + c) : "memory");
  } else {
#pragma unroll
    for (int c = 0; c < 32; ++c) h[c] = c0 + c < n ? src[c] : 0.0;
  }
}

// h -> columns [c0, c0 + 32) of the row (256-bit stores when vec); the warp's
// largest |q| per column (the high word of its bit pattern) joins lane c's
// running maximum cm.
__device__ __forceinline__ void store_half(const double (&h)[32], double* Q, int64_t ldq, int64_t g, int64_t m,
                                           int c0, int n, bool vec, int lane, uint32_t& cm) {
  double* dst = Q + g * ldq + c0;
  if (g < m) {
    if (vec) {
#pragma unroll
      for (int c = 0; c < 32; c += 4)
        asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};"
                     :: "l"(dst + c), "d"(h[c]), "d"(h[c + 1]), "d"(h[c + 2]), "d"(h[c + 3]) : "memory");
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c0 + c < n) dst[c] = h[c];
    }
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const uint32_t hi = (uint32_t)((unsigned long long)__double_as_longlong(h[c]) >> 32) & 0x7FFFFFFFu;
    const uint32_t wm = __reduce_max_sync(0xffffffffu, hi);
    if (lane == c) cm = cm > wm ? cm : wm;
  }
}

// Column exponents of product UI's block of R_k (tau_l = 2^Eb > max_k |r_kl|).
template <int NP, int UI>
__device__ __forceinline__ void setup_eb(const double* __restrict__ rk, int np, int* Eb) {
  constexpr Upd U = plan<NP, UI>();
  for (int l = threadIdx.x; l < 16; l += THREADS) {
    unsigned long long mx = 0;
    for (int k = 0; k < U.K; ++k) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(rk[pk_idx(np, U.k0 + k, U.c0 + l)]) & 0x7FFFFFFFFFFFFFFFull;
      mx = mx > b ? mx : b;
    }
    Eb[U.eoff + l] = tc::split_exp(mx);
  }
}

// Digit planes of product UI's block of R_k (B operand: 16 columns, K-major;
// plane t at t * 32 K bytes), units (column l, K group kg).
template <int NP, int UI>
__device__ __forceinline__ void setup_b(const double* __restrict__ rk, int np, const int* Eb, uint8_t* bb) {
  constexpr Upd U = plan<NP, UI>();
  for (int u = threadIdx.x; u < 16 * (U.K / 8); u += THREADS) {
    const int l = u % 16, kg = u / 16;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = rk[pk_idx(np, U.k0 + 8 * kg + q, U.c0 + l)];
    tc::cut8(v, Eb[U.eoff + l], bb + U.boff + (l >> 3) * (16 * U.K) + kg * LBO + (l & 7) * 16, 32 * U.K);
  }
}

}  // namespace tcf

// X: rows [0, P.m) of the pass's input (ldx), Q: its output (ldq; may be X
// itself). rk: R_k packed P.np x P.np. colmax (may be null): receives, by
// atomicMax, a bit pattern with the exponent of max |q_ij| per column j < n
// (the high word of the pattern; the low word zero).
template <int NP>
__global__ void __launch_bounds__(tcf::THREADS, 1)
tc_fused_solve_kernel(const double* X, int64_t ldx, double* Q, int64_t ldq, Params P, int pass,
                      const double* __restrict__ rk, unsigned long long* __restrict__ colmax,
                      DevState* __restrict__ st, int stagger_ns) {
  using namespace tcf;
  using tc::smem_u32;
  using G = FGeo<NP>;
  using PL = Plan<NP>;
  if (!st->run_trsm[pass]) return;
  extern __shared__ uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  uint8_t* bb = base + G::OFF_B;
  double* rdb = (double*)(base + G::OFF_R);
  double* rinv = (double*)(base + G::OFF_RINV);
  __shared__ __align__(8) uint64_t mdone[SLOTS];  // the slot's MMAs done (tcgen05.commit)
  __shared__ uint32_t tslot;
  __shared__ int Eb[PL::NEB];  // column exponents of the B planes
  __shared__ int err_sh[SLOTS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slot = tid >> 7, r = tid & (ROWS - 1), ws = warp & 3;
  const int n = P.n, np = P.np;
  const int64_t m = P.m;

  // R_k: the diagonal blocks (dense 16 x 16, upper part), 1 / r_jj, and the
  // digit planes of the off-diagonal blocks with their column exponents
  for (int e = tid; e < G::NB * 256; e += THREADS) {
    const int J = e >> 8, c = (e >> 4) & 15, c2 = e & 15;
    rdb[e] = c2 >= c ? rk[pk_idx(np, 16 * J + c, 16 * J + c2)] : 0.0;
  }
  for (int j = tid; j < NP; j += THREADS) rinv[j] = 1.0 / rk[pk_idx(np, j, j)];
  setup_eb<NP, 0>(rk, np, Eb);
  if constexpr (NP == 64) {
    setup_eb<NP, 1>(rk, np, Eb);
    setup_eb<NP, 2>(rk, np, Eb);
    setup_eb<NP, 3>(rk, np, Eb);
  }
  if (tid < SLOTS) err_sh[tid] = 0;
  if (tid == 0) {
    for (int g = 0; g < SLOTS; ++g)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mdone[g])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  setup_b<NP, 0>(rk, np, Eb, bb);
  if constexpr (NP == 64) {
    setup_b<NP, 1>(rk, np, Eb, bb);
    setup_b<NP, 2>(rk, np, Eb, bb);
    setup_b<NP, 3>(rk, np, Eb, bb);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  SlotCtx ctx;
  ctx.sbuf = base + slot * G::SBUF;
  ctx.bb = bb;
  ctx.Eb = Eb;
  ctx.tmem = tmem + slot * TSLOT;
  ctx.tq = tmem + slot * TSLOT + ((uint32_t)(32 * ws) << 16);  // this thread's lane, the slot's columns
  ctx.mbar = smem_u32(&mdone[slot]);
  // D F32, A and B BF16, both K-major, M = 128 (N set per MMA)
  ctx.idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);
  ctx.slot = slot;
  ctx.r = r;
  ctx.wait_ns = P.wait_ns;

  // 256-bit row accesses for halves that lie within n, 32-byte aligned
  const bool vx0 = n >= 32 && ((uintptr_t)X & 31) == 0 && (ldx & 3) == 0;
  const bool vq0 = n >= 32 && ((uintptr_t)Q & 31) == 0 && (ldq & 3) == 0;
  const bool vx1 = vx0 && n >= 64, vq1 = vq0 && n >= 64;

  // The slots start apart, so that one slot's integer and tensor-core phases
  // meet the others' FP64 phases rather than their own.
  for (int t = 0; t < slot; ++t) __nanosleep(stagger_ns);

  uint32_t cm[NP / 32];  // lane c: the largest |q| high word of column 32 h + c
#pragma unroll
  for (int h = 0; h < NP / 32; ++h) cm[h] = 0;
  uint32_t phase = 0;    // completed waits on mdone[slot]
  uint32_t commits = 0;  // commits to mdone[slot] (thread 0 of the slot)
  bool failed = false;

  for (int64_t it = 0;; ++it) {
    const int64_t row0 = ((it * gridDim.x + blockIdx.x) * SLOTS + slot) * (int64_t)ROWS;
    if (row0 >= m) break;  // uniform in the slot
    const int64_t g = row0 + r;
    double h[32];
    int E;
    bool fin;
    load_half(h, X, ldx, g, m, 0, n, vx0);
    solve16<0>(h, rdb, rinv);
    // U0: x_1 -= y_0 R_01
    fin = cut_rows<16>(h, ctx, E);
    mma_product<NP, 0>(ctx, commits);
    if (!mma_wait(ctx, phase)) {
      failed = true;
      break;
    }
    fold16<16>(h, ctx, E, fin, Eb + plan<NP, 0>().eoff);
    solve16<16>(h, rdb + 256, rinv + 16);
    if constexpr (NP == 64) {
      // U1: [x_2 x_3] -= [y_0 y_1] R_{01,23}, as two 16-column products on
      // the same digit planes; the first runs while y_0, y_1 go out and
      // x_2, x_3 come in
      fin = cut_rows<32>(h, ctx, E);
      mma_product<NP, 1>(ctx, commits);
      store_half(h, Q, ldq, g, m, 0, n, vq0, lane, cm[0]);
      load_half(h, X, ldx, g, m, 32, n, vx1);
      if (!mma_wait(ctx, phase)) {
        failed = true;
        break;
      }
      fold16<0>(h, ctx, E, fin, Eb + plan<NP, 1>().eoff);
      mma_product<NP, 2>(ctx, commits);
      if (!mma_wait(ctx, phase)) {
        failed = true;
        break;
      }
      fold16<16>(h, ctx, E, fin, Eb + plan<NP, 2>().eoff);
      solve16<0>(h, rdb + 512, rinv + 32);
      // U2: x_3 -= y_2 R_23
      fin = cut_rows<16>(h, ctx, E);
      mma_product<NP, 3>(ctx, commits);
      if (!mma_wait(ctx, phase)) {
        failed = true;
        break;
      }
      fold16<16>(h, ctx, E, fin, Eb + plan<NP, 3>().eoff);
      solve16<16>(h, rdb + 768, rinv + 48);
      store_half(h, Q, ldq, g, m, 32, n, vq1, lane, cm[1]);
    } else {
      store_half(h, Q, ldq, g, m, 0, n, vq0, lane, cm[0]);
    }
  }
  if (failed && r == 0) err_sh[slot] = 1;
  __syncthreads();
  if (err_sh[slot]) {
    if (r == 0) {
      atomicCAS(&st->status, SCQR3_OK, SCQR3_E_TIMEOUT);
      // the slot's last MMAs finish (bounded) before the tensor memory is freed
      if (commits > 0) tc::wait_parity(ctx.mbar, (commits - 1) & 1, tc::kWaitNs);
    }
  } else if (colmax && st->gram_after[pass]) {
#pragma unroll
    for (int h = 0; h < NP / 32; ++h)
      if (32 * h + lane < n && cm[h]) atomicMax(&colmax[32 * h + lane], (unsigned long long)cm[h] << 32);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// ---- host side ----------------------------------------------------------------------------

cudaError_t tc_fused_setup() {
  cudaError_t e = cudaFuncSetAttribute(tc_fused_solve_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tcf::FGeo<32>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_fused_solve_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tcf::FGeo<64>::SMEM);
  return e;
}

// The fused substitution serves 16 < n <= 64.
bool tc_fused_supported(int n) { return n > 16 && n <= 64; }

// Pass k's substitution over rows [0, P.m) of X into Q; colmax (or null)
// receives the column maxima of Q for the next Gram matrix.
void launch_tc_fused(int sms, cudaStream_t s, const double* X, int64_t ldx, double* Q, int64_t ldq, const Params& P,
                     int pass, const double* rk, unsigned long long* colmax, DevState* st, int stagger_ns) {
  const int64_t tiles = (P.m + tcf::ROWS - 1) / tcf::ROWS;
  const int64_t want = (tiles + tcf::SLOTS - 1) / tcf::SLOTS;
  const int grid = (int)(want < sms ? (want < 1 ? 1 : want) : sms);
  if (P.n <= 32)
    tc_fused_solve_kernel<32><<<grid, tcf::THREADS, tcf::FGeo<32>::SMEM, s>>>(X, ldx, Q, ldq, P, pass, rk, colmax, st,
                                                                              stagger_ns);
  else
    tc_fused_solve_kernel<64><<<grid, tcf::THREADS, tcf::FGeo<64>::SMEM, s>>>(X, ldx, Q, ldq, P, pass, rk, colmax, st,
                                                                              stagger_ns);
}

}  // namespace scqr3
