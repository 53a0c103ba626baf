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

constexpr int ROWS = 128;                 // rows per tile = tensor-memory lanes
constexpr int SLOTS = 2;                  // tiles in flight per CTA
constexpr int THREADS = ROWS * SLOTS;     // one thread per row of each slot's tile
constexpr uint32_t LBO = 128;             // K-direction core-matrix stride
constexpr uint32_t TSLOT = 256;           // tensor-memory columns per slot
constexpr int SBUF = 65536;               // per slot: a staged tile of 128 x 64 doubles, or 8 digit planes (K <= 32)
constexpr int BOX = ROWS * 128;           // one 16-column box of a staged tile (16 KB)

// Off-diagonal updates x[C0, C0 + N) -= y[K0, K0 + K) R[K0.., C0..]: their B
// planes at byte BOFF of the B area and column exponents at EOFF.
struct Upd {
  int k0, K, c0, N, boff, eoff;
};
template <int NP> struct Plan;
template <> struct Plan<32> {
  static constexpr int NU = 1;
  static constexpr Upd u[1] = {{0, 16, 16, 16, 0, 0}};
  static constexpr int BBYTES = 4096, NEB = 16;
};
template <> struct Plan<64> {
  static constexpr int NU = 3;
  static constexpr Upd u[3] = {{0, 16, 16, 16, 0, 0}, {0, 32, 32, 32, 4096, 16}, {32, 16, 48, 16, 20480, 48}};
  static constexpr int BBYTES = 24576, NEB = 64;
};

template <int NP> struct FGeo {
  static constexpr int NB = NP / 16;  // diagonal blocks
  static constexpr size_t OFF_B = (size_t)SLOTS * SBUF;
  static constexpr size_t OFF_R = OFF_B + Plan<NP>::BBYTES;       // dense 16 x 16 diagonal blocks of R_k
  static constexpr size_t OFF_RINV = OFF_R + (size_t)NB * 256 * 8;  // 1 / r_jj
  static constexpr size_t SMEM = OFF_RINV + (size_t)NP * 8 + 1024;  // + alignment slack
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// byte offset of (row r, column c) in a staged tile: column box c / 16 (128
// bytes of each row), its 16-byte units XOR-swizzled by r % 8
__device__ __forceinline__ uint32_t stage_off(int r, int c) {
  return (uint32_t)((c >> 4) * BOX + r * 128 + ((((c >> 1) & 7) ^ (r & 7)) << 4) + ((c & 1) << 3));
}

template <int K>
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)((16u * K) >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// The MMAs of one update: digit s of Y (A: plane s at s * 256 K bytes) against
// the B planes t = 0 .. 7 - s side by side, N_u (8 - s) columns from tensor
// column N_u s; K step kk (two core matrices, 256 bytes, per K = 16).
template <int K, int N, int S, int KK>
__device__ __forceinline__ void issue(uint64_t adesc, uint64_t bdesc, uint32_t tmem, uint32_t idesc0) {
  constexpr uint32_t NS = N * (8 - S);
  constexpr uint64_t aoff = ((uint32_t)S * (ROWS * K * 2) + KK * 2 * LBO) >> 4;
  constexpr uint64_t boff = (KK * 2 * LBO) >> 4;
  tc::mma(tmem + N * S, adesc + aoff, bdesc + boff, idesc0 | ((NS >> 3) << 17), (S > 0 || KK > 0) ? 1u : 0u);
  if constexpr (KK + 1 < K / 16) {
    issue<K, N, S, KK + 1>(adesc, bdesc, tmem, idesc0);
  } else if constexpr (S < 7) {
    issue<K, N, S + 1, 0>(adesc, bdesc, tmem, idesc0);
  }
}

// Barrier among the 128 threads of a slot (ids 1, 2); the second form returns
// whether any of them passed a non-zero `pred` (slot-uniform decisions).
__device__ __forceinline__ void slot_sync(int slot) {
  asm volatile("bar.sync %0, %1;" :: "r"(1 + slot), "r"(ROWS) : "memory");
}
__device__ __forceinline__ int slot_any(int slot, int pred) {
  int r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.b32 %0, 1, 0, q;\n}"
               : "=r"(r) : "r"(pred), "r"(1 + slot), "r"(ROWS) : "memory");
  return r;
}

// Eight consecutive values as 8 digit planes of one core-matrix row each
// (16 bytes: 8 BF16 digits), at dst + s * plane; |x| < 2^E.
__device__ __forceinline__ void cut8(const double (&x)[8], int E, uint8_t* dst, uint32_t plane) {
  unsigned long long F[8];
  uint32_t sp[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    F[r] = tc::fixed56(x[r], E);
    const uint32_t sgn = (uint32_t)((unsigned long long)__double_as_longlong(x[r]) >> 32) & 0x80000000u;
    sp[r >> 1] |= (r & 1) ? sgn : (sgn >> 16);
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    uint4 w;
    switch (s) {  // digit_pair takes the digit as a template argument
#define SCQR3_CUTS(S)                                 \
  case S:                                             \
    w.x = tc::digit_pair<S>(F[0], F[1], sp[0]);       \
    w.y = tc::digit_pair<S>(F[2], F[3], sp[1]);       \
    w.z = tc::digit_pair<S>(F[4], F[5], sp[2]);       \
    w.w = tc::digit_pair<S>(F[6], F[7], sp[3]);       \
    break;
      SCQR3_CUTS(0) SCQR3_CUTS(1) SCQR3_CUTS(2) SCQR3_CUTS(3) SCQR3_CUTS(4) SCQR3_CUTS(5) SCQR3_CUTS(6)
      SCQR3_CUTS(7)
#undef SCQR3_CUTS
    }
    *(uint4*)(dst + s * plane) = w;
  }
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

// 2^E > the non-negative bit-pattern maximum mx (-1000 for zero)
__device__ __forceinline__ int scale_exp(unsigned long long mx) {
  if (mx == 0) return -1000;
  const int ex = (int)(mx >> 52);
  return (ex ? ex : 1) - 1023 + 1;
}

// The row of a thread lives in a register array x[NP]; the code that works on
// it is written once and reached with a runtime block index. These switches
// move 8, 16 or 4 values between x and small arrays with compile-time indices
// in every case, so x stays in registers while the tile's code stays small
// (a fully unrolled tile does not fit the instruction cache).
#define SCQR3_CASES8(M) M(0) M(1) M(2) M(3) M(4) M(5) M(6) M(7)
#define SCQR3_CASES16(M) SCQR3_CASES8(M) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15)
template <int NP>
__device__ __forceinline__ void get8(const double (&x)[NP], int g, double (&v)[8]) {
  switch (g) {
#define SCQR3_G8(I)                                           \
  case I:                                                     \
    if constexpr (8 * I < NP) {                               \
      _Pragma("unroll") for (int q = 0; q < 8; ++q) v[q] = x[8 * I + q]; \
    }                                                         \
    break;
    SCQR3_CASES8(SCQR3_G8)
#undef SCQR3_G8
    default: break;
  }
}
template <int NP>
__device__ __forceinline__ void get16(const double (&x)[NP], int J, double (&t)[16]) {
  switch (J) {
#define SCQR3_G16(I)                                            \
  case I:                                                       \
    if constexpr (16 * I < NP) {                                \
      _Pragma("unroll") for (int q = 0; q < 16; ++q) t[q] = x[16 * I + q]; \
    }                                                           \
    break;
    SCQR3_G16(0) SCQR3_G16(1) SCQR3_G16(2) SCQR3_G16(3)
#undef SCQR3_G16
    default: break;
  }
}
template <int NP>
__device__ __forceinline__ void put16(double (&x)[NP], int J, const double (&t)[16]) {
  switch (J) {
#define SCQR3_P16(I)                                            \
  case I:                                                       \
    if constexpr (16 * I < NP) {                                \
      _Pragma("unroll") for (int q = 0; q < 16; ++q) x[16 * I + q] = t[q]; \
    }                                                           \
    break;
    SCQR3_P16(0) SCQR3_P16(1) SCQR3_P16(2) SCQR3_P16(3)
#undef SCQR3_P16
    default: break;
  }
}
// x[4 g + q] -= upd[q] (NaN for a row whose scale is not finite)
template <int NP>
__device__ __forceinline__ void sub4(double (&x)[NP], int g, const double (&upd)[4], bool finite) {
  switch (g) {
#define SCQR3_S4(I)                                                                          \
  case I:                                                                                    \
    if constexpr (4 * I < NP) {                                                              \
      _Pragma("unroll") for (int q = 0; q < 4; ++q) x[4 * I + q] = finite ? x[4 * I + q] - upd[q] : (double)NAN; \
    }                                                                                        \
    break;
    SCQR3_CASES16(SCQR3_S4)
#undef SCQR3_S4
    default: break;
  }
}

// y = t R_JJ^{-1} in place for one 16-column diagonal block: forward
// substitution over its columns (multiply by the rounded reciprocal of r_jj).
__device__ __forceinline__ void solve16(double (&t)[16], const double* __restrict__ rb,
                                        const double* __restrict__ ri) {
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    double rc;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(rc) : "r"(tc::smem_u32(ri + c)));
    const double y = t[c] * rc;
    t[c] = y;
#pragma unroll
    for (int c2 = c + 1; c2 < 16; ++c2) {
      // an explicit shared load: left to itself the compiler hoists all of
      // the block's R values into registers, which the resident row needs
      double rv;
      asm volatile("ld.shared.f64 %0, [%1];" : "=d"(rv) : "r"(tc::smem_u32(rb + c * 16 + c2)));
      t[c2] = fma(-y, rv, t[c2]);
    }
  }
}

// Per-slot state of the update pipeline.
struct SlotCtx {
  uint8_t* sbuf;     // the slot's buffer (staged rows, A planes)
  uint8_t* bb;       // B planes of the off-diagonal blocks
  const int* Eb;     // their column exponents
  uint32_t tmem;     // the slot's first tensor-memory column (lane 0)
  uint32_t tq;       // this thread's lane of it
  uint32_t mbar;     // the slot's MMA-completion mbarrier
  uint32_t idesc0;
  int slot, r;
  long long wait_ns;
};

template <int NP>
__device__ __forceinline__ Upd plan_of(int ui) {
  if constexpr (NP == 32) {
    return Upd{0, 16, 16, 16, 0, 0};
  } else {
    return ui == 0 ? Upd{0, 16, 16, 16, 0, 0} : ui == 1 ? Upd{0, 32, 32, 32, 4096, 16} : Upd{32, 16, 48, 16, 20480, 48};
  }
}

// Update ui of Plan<NP> on this thread's row: x[C0, C0 + N) -= y[K0, K0 + K)
// R[K0.., C0..] on the tensor cores. Returns false (slot-uniformly) if the
// wait for the MMAs ran out.
template <int NP>
__device__ __forceinline__ bool update(double (&x)[NP], int ui, const SlotCtx& c, uint32_t& phase,
                                       uint32_t& commits) {
  const Upd U = plan_of<NP>(ui);
  // the row's scale over its K values
  unsigned long long mx = 0;
#pragma unroll 1
  for (int g = U.k0 / 8; g < (U.k0 + U.K) / 8; ++g) {
    double v[8];
    get8(x, g, v);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(v[q]) & 0x7FFFFFFFFFFFFFFFull;
      mx = mx > b ? mx : b;
    }
  }
  const bool finite = (mx >> 52) != 0x7FF;
  const int E = finite ? scale_exp(mx) : 0;
  slot_sync(c.slot);  // every warp of the slot is done with the buffer (staged rows, earlier planes)
  {
    uint8_t* ar = c.sbuf + (c.r >> 3) * (16 * U.K) + (c.r & 7) * 16;
    const uint32_t plane = ROWS * U.K * 2;
#pragma unroll 1
    for (int kg = 0; kg < U.K / 8; ++kg) {
      double v[8];
      get8(x, U.k0 / 8 + kg, v);
      cut8(v, E, ar + kg * LBO, plane);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  slot_sync(c.slot);
  bool ok = true;
  if (c.r == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (U.K == 16)
      issue<16, 16, 0, 0>(desc<16>(tc::smem_u32(c.sbuf)), desc<16>(tc::smem_u32(c.bb + U.boff)), c.tmem, c.idesc0);
    else
      issue<32, 32, 0, 0>(desc<32>(tc::smem_u32(c.sbuf)), desc<32>(tc::smem_u32(c.bb + U.boff)), c.tmem, c.idesc0);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(c.mbar)
                 : "memory");
    ++commits;
    // one thread waits; the barrier below releases the slot
    ok = tc::wait_parity(c.mbar, phase & 1, c.wait_ns);
  }
  ++phase;
  if (slot_any(c.slot, !ok)) return false;
  asm volatile("tcgen05.fence::after_thread_sync;");
  // read back the 8 tile sums of each updated column and apply them
  constexpr unsigned long long BIAS = 0x4B400000ull * ((1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);
#pragma unroll 1
  for (int c4 = 0; c4 < U.N; c4 += 4) {
    uint32_t v[8][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) tc::ld4(c.tq + U.N * e + c4, v[e]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    double upd[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // |D_e| < 2^22: D_e + 1.5 2^23 is exact, with bit pattern 0x4B400000 + D_e
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
      upd[q] = scaled_int(W, E + c.Eb[U.eoff + c4 + q] - 56);
    }
    sub4(x, (U.c0 + c4) / 4, upd, finite);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  return true;
}

// Column exponents of update UI's block of R_k (tau_l = 2^Eb > max_k |r_kl|).
template <int NP, int UI>
__device__ __forceinline__ void setup_eb(const double* __restrict__ rk, int np, int* Eb) {
  constexpr Upd U = Plan<NP>::u[UI];
  for (int l = threadIdx.x; l < U.N; l += THREADS) {
    unsigned long long mx = 0;
    for (int k = 0; k < U.K; ++k) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(rk[pk_idx(np, U.k0 + k, U.c0 + l)]) & 0x7FFFFFFFFFFFFFFFull;
      mx = mx > b ? mx : b;
    }
    Eb[U.eoff + l] = scale_exp(mx);
  }
}

// Digit planes of update UI's block of R_k (B operand: N columns, K-major;
// plane t at t * 2 K N bytes), units (column l, K group kg).
template <int NP, int UI>
__device__ __forceinline__ void setup_b(const double* __restrict__ rk, int np, const int* Eb, uint8_t* bb) {
  constexpr Upd U = Plan<NP>::u[UI];
  for (int u = threadIdx.x; u < U.N * (U.K / 8); u += THREADS) {
    const int l = u % U.N, kg = u / U.N;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = rk[pk_idx(np, U.k0 + 8 * kg + q, U.c0 + l)];
    cut8(v, Eb[U.eoff + l], bb + U.boff + (l >> 3) * (16 * U.K) + kg * LBO + (l & 7) * 16, 2 * U.K * U.N);
  }
}

}  // namespace tcf

// X: rows [0, P.m) of the pass's input (ldx), Q: its output (ldq; may be X
// itself). rk: R_k packed P.np x P.np. colmax (may be null): receives, by
// atomicMax, the bit pattern of max |q_ij| per column j < n.
template <int NP>
__global__ void __launch_bounds__(tcf::THREADS, 1)
tc_fused_solve_kernel(const double* X, int64_t ldx, double* Q, int64_t ldq, Params P, int pass,
                      const double* __restrict__ rk, unsigned long long* __restrict__ colmax,
                      DevState* __restrict__ st) {
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
  uint8_t* sbuf = base + slot * SBUF;

  // R_k: the diagonal blocks (dense 16 x 16, upper part), 1 / r_jj, and the
  // column exponents of the off-diagonal blocks
  for (int e = tid; e < G::NB * 256; e += THREADS) {
    const int J = e >> 8, c = (e >> 4) & 15, c2 = e & 15;
    rdb[e] = c2 >= c ? rk[pk_idx(np, 16 * J + c, 16 * J + c2)] : 0.0;
  }
  for (int j = tid; j < NP; j += THREADS) rinv[j] = 1.0 / rk[pk_idx(np, j, j)];
  setup_eb<NP, 0>(rk, np, Eb);
  if constexpr (PL::NU > 1) {
    setup_eb<NP, 1>(rk, np, Eb);
    setup_eb<NP, 2>(rk, np, Eb);
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
  if constexpr (PL::NU > 1) {
    setup_b<NP, 1>(rk, np, Eb, bb);
    setup_b<NP, 2>(rk, np, Eb, bb);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  SlotCtx ctx;
  ctx.sbuf = sbuf;
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

  unsigned long long cmax[NP / 32];  // max |q| bit patterns of columns 32 h + lane (store phase)
#pragma unroll
  for (int h = 0; h < NP / 32; ++h) cmax[h] = 0;
  uint32_t phase = 0;    // completed waits on mdone[slot]
  uint32_t commits = 0;  // commits to mdone[slot] (thread 0 of the slot)
  bool failed = false;

  for (int64_t it = 0;; ++it) {
    const int64_t row0 = ((it * gridDim.x + blockIdx.x) * SLOTS + slot) * (int64_t)ROWS;
    if (row0 >= m) break;  // uniform in the slot
    // ---- the warp's 32 rows into the buffer (zeros past m and past n)
#pragma unroll 2
    for (int rr = 0; rr < 32; ++rr) {
      const int row = 32 * ws + rr;
      const int64_t g = row0 + row;
#pragma unroll
      for (int h = 0; h < NP / 32; ++h) {
        const int c = 32 * h + lane;
        const bool ok = g < m && c < n;
        const double* src = ok ? X + g * ldx + c : X;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;"
                     :: "r"(smem_u32(sbuf + stage_off(row, c))), "l"(src), "r"(ok ? 8 : 0) : "memory");
      }
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    double x[NP];
#pragma unroll
    for (int c = 0; c < NP; c += 2) {
      const double2 v = *(const double2*)(sbuf + stage_off(r, c));
      x[c] = v.x;
      x[c + 1] = v.y;
    }
    // ---- diagonal blocks and off-diagonal updates (update J follows block J)
#pragma unroll 1
    for (int J = 0; J < G::NB; ++J) {
      double t[16];
      get16(x, J, t);
      solve16(t, rdb + J * 256, rinv + 16 * J);
      put16(x, J, t);
      if (J + 1 < G::NB && !update(x, J, ctx, phase, commits)) {
        failed = true;
        break;
      }
    }
    if (failed) break;
    // ---- the rows out through the buffer (the last MMAs have completed)
    __syncwarp();
#pragma unroll
    for (int c = 0; c < NP; c += 2) *(double2*)(sbuf + stage_off(r, c)) = make_double2(x[c], x[c + 1]);
    __syncwarp();
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const int row = 32 * ws + rr;
      const int64_t g = row0 + row;
#pragma unroll
      for (int h = 0; h < NP / 32; ++h) {
        const int c = 32 * h + lane;
        if (g < m && c < n) {
          const double v = *(const double*)(sbuf + stage_off(row, c));
          Q[g * ldq + c] = v;
          const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
          cmax[h] = cmax[h] > b ? cmax[h] : b;
        }
      }
    }
    __syncwarp();
  }
  if (failed && r == 0) err_sh[slot] = 1;
  __syncthreads();
  if (err_sh[slot]) {
    if (r == 0) {
      atomicCAS(&st->status, SCQR3_OK, SCQR3_E_TIMEOUT);
      // the slot's last MMAs finish (bounded) before the tensor memory is freed
      if (commits > 0) tc::wait_parity(ctx.mbar, (commits - 1) & 1, tc::kWaitNs);
    }
  } else if (colmax) {
#pragma unroll
    for (int h = 0; h < NP / 32; ++h)
      if (32 * h + lane < n && cmax[h]) atomicMax(&colmax[32 * h + lane], cmax[h]);
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
                     int pass, const double* rk, unsigned long long* colmax, DevState* st) {
  const int64_t tiles = (P.m + tcf::ROWS - 1) / tcf::ROWS;
  const int64_t want = (tiles + tcf::SLOTS - 1) / tcf::SLOTS;
  const int grid = (int)(want < sms ? (want < 1 ? 1 : want) : sms);
  if (P.n <= 32)
    tc_fused_solve_kernel<32><<<grid, tcf::THREADS, tcf::FGeo<32>::SMEM, s>>>(X, ldx, Q, ldq, P, pass, rk, colmax, st);
  else
    tc_fused_solve_kernel<64><<<grid, tcf::THREADS, tcf::FGeo<64>::SMEM, s>>>(X, ldx, Q, ldq, P, pass, rk, colmax, st);
}

}  // namespace scqr3
