// tc_fused.cu -- one pass's row-wise substitution Q := X R_k^{-1}
// (Eq. backward2) for 16 < n <= 64 in a single sweep over the rows: every row
// is read once and written once, and the column maxima of the result (the
// scales of the next tensor-core Gram matrix) come out of the same sweep.
//
// The substitution of a row x^T groups its terms by 16-column blocks of R
// (as in tc_solve.cu): for n <= 64 (NP = 64)
//   y_0 = x_0 R_00^-1;        x_1 -= y_0 R_01                    (K = 16)
//   y_1 = x_1 R_11^-1;        [x_2 x_3] -= [y_0 y_1] R_{01,23}   (K = 32)
//   y_2 = x_2 R_22^-1;        x_3 -= y_2 R_23                    (K = 16)
//   y_3 = x_3 R_33^-1
// and for n <= 32 (NP = 32) the first line and y_1. The triangular solves of
// the 16 x 16 diagonal blocks run in FP64, one thread per row, with the row
// in registers; the products with the off-diagonal blocks run on the BF16
// tensor cores through the exact digit split of tc_solve.cu (a scale per row
// of Y -- here the common one of all K values multiplied, y_0 and y_1
// together in the middle update -- and per column of R_JK; eight signed
// 7-bit digits; tile e of tensor memory sums the digit pairs with s + t = e,
// at most 8 * 32 * 64^2 = 2^20 per entry, exact in FP32; int64 folding; one
// FP64 subtraction per updated entry). Error: as for tc_solve.cu, a
// perturbation of R_JK of norm O(u ||R||) per row, the form of the row-wise
// backward error that the analysis of Sec. 3 assumes.
//
// FP64 work per row: 4 (16 * 15 / 2 FMAs + 16 multiplies) + 64 subtractions
// = 608 at NP = 64, against 2112 for the unblocked substitution.
//
// Layout: one CTA per SM, three slots of 128 threads; a slot owns one 128-row
// tile at a time (thread r of the slot holds row r, which is tensor-memory
// lane r: warp w of the slot reads lane quadrant w). A thread holds two
// 16-column blocks of its row in registers (lo, hi). A product's Y blocks are
// cut into digit planes in the slot's two 32 KB regions (A operand: M = 128,
// K = 16 per region, K-major, no swizzle); thread 0 of the slot issues one MMA
// per digit s and region (digit s of Y against the planes t = 0 .. 7 - s of
// R_JK side by side: N = 16 (8 - s), accumulating from tensor-memory column
// 16 s, so the pair (s, t) lands in tile e = s + t) into the slot's 128
// columns and commits them to the slot's mbarrier; every thread then reads its
// row's tile sums back (tcgen05.ld 32x32b) and folds them into hi.
//
// Scheduling: the slots take turns at the diagonal solves (at most two at a
// time), so that the FP64 pipe stays busy while the others cut digits, wait
// for their MMAs, fold, load and store. The work of
// a tile is a fixed program of steps (load, solve, scan, cut, swap, MMA, wait,
// fold, store) run by one loop over a switch, so that the code of each kind of
// step exists once: fully inlined, the kernel's code outgrew the instruction
// cache, and every step of every tile waited for its instructions. Waits are
// bounded in time; a wait that runs out records SCQR3_E_TIMEOUT, and before
// the tensor memory is freed the CTA waits (bounded) for its last MMAs.
#include <type_traits>

#include "tc_common.cuh"

namespace scqr3 {

namespace tcf {

constexpr int ROWS = 128;                       // rows per tile = tensor-memory lanes
constexpr int SLOTS = 3;                        // tiles in flight per CTA, 128 threads each
constexpr int THREADS = ROWS * SLOTS;
constexpr uint32_t LBO = 128;                   // K-direction core-matrix stride
constexpr uint32_t PLANE = ROWS * 16 * 2;       // one digit plane of a 128 x 16 block (4 KB)
constexpr uint32_t REGION = 8 * PLANE;          // the 8 planes of one block (32 KB)
constexpr uint32_t SBUF = 2 * REGION;           // a slot's A operand: up to K = 32
constexpr uint32_t TSLOT = 128;                 // tensor-memory columns per slot: 8 tiles x 16 columns

// Off-diagonal products x[c0, c0 + 16) -= y[k0, k0 + K) R[k0.., c0..]: B planes
// at byte boff of the B area (8 planes of K x 16 BF16 digits, plane t at
// t * 32 K), column exponents at eoff.
struct Upd {
  int k0, K, c0, boff, eoff;
};
// NP = 64: U0 = y_0 R_01; U1a, U1b = [y_0 y_1] R_{01,2}, R_{01,3}; U2 = y_2 R_23.
// NP = 32: U0 only.
__host__ __device__ constexpr Upd plan(int u) {
  return u == 0 ? Upd{0, 16, 16, 0, 0}
       : u == 1 ? Upd{0, 32, 32, 4096, 16}
       : u == 2 ? Upd{0, 32, 48, 12288, 32}
                : Upd{32, 16, 48, 20480, 48};
}
template <int NP> struct FGeo {
  static constexpr int NU = NP == 64 ? 4 : 1;                     // products
  static constexpr int BBYTES = NP == 64 ? 24576 : 4096;          // their B planes
  static constexpr int NB = NP / 16;                              // diagonal blocks
  static constexpr size_t OFF_B = (size_t)SLOTS * SBUF;
  static constexpr size_t OFF_R = OFF_B + BBYTES;                 // dense 16 x 16 diagonal blocks of R_k
  static constexpr size_t OFF_RINV = OFF_R + (size_t)NB * 256 * 8;  // 1 / r_jj
  static constexpr size_t SMEM = OFF_RINV + (size_t)NP * 8 + 1024;  // + alignment slack
  static_assert(SMEM + 512 <= 227 * 1024, "shared memory");
};

// Shared-memory matrix descriptor: K-major, no swizzle, core matrices of 8
// rows x 16 bytes, K-direction stride LBO, 8-row stride sbo.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// The FP64 turns: the slots run their diagonal solves in ring order, the j-th
// solve of slot s being turn t = SLOTS j + s, and turn t starts once turn
// t - TURNS has finished, so that at most TURNS slots issue FP64 work at a
// time while the others cut digits, wait for their MMAs, fold, load and
// store. (Left alone, the slots drift into step and meet in the same phase:
// all solving, then all on integer work with the FP64 pipe idle.) The slot of
// turn t - TURNS arrives on a named barrier that the slot of turn t waits on
// (2 x 128 threads); a producer's consecutive turns alternate between two
// barriers per consumer, and its turn k + 2 cannot start before the consumer
// has taken turn k, so no barrier ever holds two arrivals. Every slot runs
// the same number of solves; after the loop the slots with s < TURNS take
// the one arrival left for them.
constexpr int TURNS = 2;
__device__ __forceinline__ int turn_bar(int consumer, int k) { return 1 + SLOTS + 2 * consumer + (k & 1); }
__device__ __forceinline__ void turn_take(int slot, int j) {
  const int t = SLOTS * j + slot;
  if (t >= TURNS)
    asm volatile("bar.sync %0, %1;" :: "r"(turn_bar(slot, (t - TURNS) / SLOTS)), "r"(2 * ROWS) : "memory");
}
__device__ __forceinline__ void turn_pass(int slot, int j) {
  asm volatile("bar.arrive %0, %1;" :: "r"(turn_bar((slot + TURNS) % SLOTS, j)), "r"(2 * ROWS) : "memory");
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

// y = v R_JJ^{-1} in place: forward substitution over the block's columns
// (multiply by the rounded reciprocal of r_jj); rb = the dense 16 x 16 block,
// ri = its 16 reciprocals (shared memory).
__device__ __forceinline__ void solve16(double (&v)[16], const double* __restrict__ rb,
                                        const double* __restrict__ ri) {
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    double rc;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(rc) : "r"(tc::smem_u32(ri + c)));
    const double y = v[c] * rc;
    v[c] = y;
#pragma unroll
    for (int c2 = c + 1; c2 < 16; ++c2) {
      // an explicit shared load: left to itself the compiler hoists the
      // block's R values into registers ahead of their use
      double rv;
      asm volatile("ld.shared.f64 %0, [%1];" : "=d"(rv) : "r"(tc::smem_u32(rb + c * 16 + c2)));
      v[c2] = fma(-y, rv, v[c2]);
    }
  }
}

__device__ __forceinline__ void swap16(double (&a)[16], double (&b)[16]) {
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const double t = a[c];
    a[c] = b[c];
    b[c] = t;
  }
}

// The largest |v| bit pattern of 16 values.
__device__ __forceinline__ unsigned long long absmax16(const double (&v)[16]) {
  unsigned long long mx = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v[k]) & 0x7FFFFFFFFFFFFFFFull;
    mx = mx > b ? mx : b;
  }
  return mx;
}

// Per-slot state of the update pipeline.
struct SlotCtx {
  uint8_t* sbuf;     // the slot's A regions
  uint8_t* bb;       // B planes of the off-diagonal blocks
  const int* Eb;     // their column exponents
  uint32_t tmem;     // the slot's first tensor-memory column (lane 0)
  uint32_t tq;       // this thread's lane of it
  uint32_t mbar;     // the slot's MMA-completion mbarrier
  uint32_t idesc0;
  int slot, r;
  long long wait_ns;
};

// The digit planes of the thread's 16 values v (scale 2^E) in region q of the
// slot's A operand (row r of a K-major 128 x 16 block per plane).
__device__ __forceinline__ void cut16(const double (&v)[16], const SlotCtx& c, int E, int q) {
  uint8_t* ar = c.sbuf + q * REGION + (c.r >> 3) * 256 + (c.r & 7) * 16;
  tc::cut8(&v[0], E, ar, PLANE);
  tc::cut8(&v[8], E, ar + LBO, PLANE);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The MMAs of product U: per digit s of Y and region kk (K step), digit s
// against the B planes t = 0 .. 7 - s side by side (N = 16 (8 - s)) from
// tensor column 16 s, so that the pair (s, t) lands in tile e = s + t.
template <int U>
__device__ __forceinline__ void issue_product(const SlotCtx& c) {
  constexpr Upd P = plan(U);
  const uint64_t a0 = desc(tc::smem_u32(c.sbuf), 256);
  const uint64_t b0 = desc(tc::smem_u32(c.bb + P.boff), 16 * P.K);
#pragma unroll
  for (int sd = 0; sd < 8; ++sd) {
#pragma unroll
    for (int kk = 0; kk < P.K / 16; ++kk)
      tc::mma(c.tmem + 16 * sd, a0 + ((kk * REGION + sd * PLANE) >> 4), b0 + ((kk * 2 * LBO) >> 4),
              c.idesc0 | ((uint32_t)(2 * (8 - sd)) << 17), (sd > 0 || kk > 0) ? 1u : 0u);
  }
}

// After the slot's barrier (planes written; the previous product's sums read
// back), thread 0 issues product u and commits it to the slot's mbarrier.
__device__ __forceinline__ void mma_product(const SlotCtx& c, int u, uint32_t& commits) {
  slot_sync(c.slot);
  if (c.r == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    switch (u) {
      case 0: issue_product<0>(c); break;
      case 1: issue_product<1>(c); break;
      case 2: issue_product<2>(c); break;
      default: issue_product<3>(c); break;
    }
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

// v -= the product just read back: per column l, the 8 tile sums folded
// exactly into int64 and assembled as sigma_i tau_l 2^-56 W (eb: the 16
// column exponents tau_l = 2^eb[l]).
__device__ __forceinline__ void fold16(double (&v)[16], const SlotCtx& c, int E, bool finite, const int* eb) {
  constexpr uint32_t C129 = 0x4B400000u * 129u;  // mod 2^32
#pragma unroll
  for (int c4 = 0; c4 < 16; c4 += 4) {
    uint32_t t[8][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) tc::ld4(c.tq + 16 * e + c4, t[e]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // |D_e| <= 8 * 32 * 64^2 = 2^20: D_e + 1.5 2^23 is exact, with bit
      // pattern b_e = 0x4B400000 + D_e. Pairs of tiles combine in 32 bits:
      // b_0 2^7 + b_1 - 129 * 0x4B400000 = D_0 2^7 + D_1 (mod 2^32, and the
      // value is below 2^28 in magnitude); then
      // W = P01 2^35 + P23 2^21 + P45 2^7 + floor(P67 / 2^7)
      //   = floor(2^56 (y r) / (sigma tau)), the sum over e of D_e 2^(7 (7 - e) - 7).
      uint32_t b[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) b[e] = __float_as_uint(__uint_as_float(t[e][q]) + 12582912.0f);
      const long long p01 = (int32_t)(b[0] * 128u + b[1] - C129), p23 = (int32_t)(b[2] * 128u + b[3] - C129);
      const long long p45 = (int32_t)(b[4] * 128u + b[5] - C129), p67 = (int32_t)(b[6] * 128u + b[7] - C129);
      const long long W = (long long)(((unsigned long long)p01 << 35) + ((unsigned long long)p23 << 21) +
                                      ((unsigned long long)p45 << 7)) + (p67 >> 7);
      const double upd = scaled_int(W, E + eb[c4 + q] - 56);
      v[c4 + q] = finite ? v[c4 + q] - upd : (double)NAN;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
}

// Columns [c0, c0 + 16) of row g into v (zeros past m and past n). vec: the
// block lies within n and starts on a 32-byte boundary, so it moves as four
// 256-bit loads.
__device__ __forceinline__ void load16(double (&v)[16], const double* X, int64_t ldx, int64_t g, int64_t m, int c0,
                                       int n, bool vec) {
  const double* src = X + g * ldx + c0;
  if (g >= m) {
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = 0.0;
  } else if (vec) {
#pragma unroll
    for (int c = 0; c < 16; c += 4)
      asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                   : "=d"(v[c]), "=d"(v[c + 1]), "=d"(v[c + 2]), "=d"(v[c + 3]) : "l"(src + c) : "memory");
  } else {
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = c0 + c < n ? src[c] : 0.0;
  }
}

// v -> columns [c0, c0 + 16) of row g (256-bit stores when vec); the warp's
// largest |q| per column (the high word of its bit pattern) joins the running
// maximum of lane c0 + c mod 32, in cm[(c0 + c) / 32].
__device__ __forceinline__ void store16(const double (&v)[16], double* Q, int64_t ldq, int64_t g, int64_t m, int c0,
                                        int n, bool vec, int lane, uint32_t (&cm)[2]) {
  double* dst = Q + g * ldq + c0;
  if (g < m) {
    if (vec) {
#pragma unroll
      for (int c = 0; c < 16; c += 4)
        asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};"
                     :: "l"(dst + c), "d"(v[c]), "d"(v[c + 1]), "d"(v[c + 2]), "d"(v[c + 3]) : "memory");
    } else {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c0 + c < n) dst[c] = v[c];
    }
  }
  const bool upper = c0 >= 32;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const uint32_t hw = (uint32_t)((unsigned long long)__double_as_longlong(v[c]) >> 32) & 0x7FFFFFFFu;
    const uint32_t wm = __reduce_max_sync(0xffffffffu, hw);
    if (lane == ((c0 + c) & 31)) {
      if (upper) cm[1] = cm[1] > wm ? cm[1] : wm;
      else cm[0] = cm[0] > wm ? cm[0] : wm;
    }
  }
}

// Column exponents of product u's block of R_k (tau_l = 2^Eb > max_k |r_kl|).
__device__ __forceinline__ void setup_eb(const double* __restrict__ rk, int np, int u, int* Eb) {
  const Upd U = plan(u);
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

// Digit planes of product u's block of R_k (B operand: 16 columns, K-major;
// plane t at t * 32 K bytes), units (column l, K group kg).
__device__ __forceinline__ void setup_b(const double* __restrict__ rk, int np, int u, const int* Eb, uint8_t* bb) {
  const Upd U = plan(u);
  for (int w = threadIdx.x; w < 16 * (U.K / 8); w += THREADS) {
    const int l = w % 16, kg = w / 16;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = rk[pk_idx(np, U.k0 + 8 * kg + q, U.c0 + l)];
    tc::cut8(v, Eb[U.eoff + l], bb + U.boff + (l >> 3) * (16 * U.K) + kg * LBO + (l & 7) * 16, 32 * U.K);
  }
}

// The steps of one tile. Each thread holds two 16-column blocks of its row,
// lo and hi: solves, scans, cuts and stores work on lo, folds on hi. A step is
// one kind of work (op, arg) and optional trailing actions (post): store lo
// (ST, to column 16 * (post >> 2)) and swap lo and hi (SW). Arguments: LD
// (column of lo) / 16 | (column of hi) / 16 << 2; SOLVE the diagonal block;
// CUT the product's scale rule (C0: scale of lo; C0H: of lo with two bits of
// headroom; C1: the middle product, below); MMA, FOLD the product (FOLD first
// waits for its MMAs).
//
// The middle product needs one scale for y_0 and y_1. The first product cuts
// y_0 with two bits of headroom (2^(E-1) > 4 max |y_0|), and C1 keeps that
// scale when it also bounds y_1, so that only y_1 is cut and y_0's planes are
// used again; in the rare rows where y_1 is larger, the row takes y_1's scale
// and cuts its y_0 again. Either way every value multiplied is below 2^(E-1),
// and the scale is at most 8 times the largest of them (two bits of the 56
// given up in the first product), so the product error keeps its form.
enum : uint8_t { LD, SOLVE, CUT, MMA, FOLD, END };
enum : uint8_t { C0, C0H, C1 };
enum : uint8_t { ST = 1, SW = 2 };
struct Step {
  uint8_t op, arg, post;
};
constexpr uint8_t lohi(int lo, int hi) { return (uint8_t)(lo / 16 | (hi / 16) << 2); }
constexpr uint8_t st(int col) { return (uint8_t)(ST | (col / 16) << 2); }
constexpr int kMaxSteps = 24;
// NP = 64
__constant__ Step kProg64[] = {
    {LD, lohi(0, 16), 0},       // lo = x_0, hi = x_1
    {SOLVE, 0, 0},              // lo = y_0
    {CUT, C0H, 0},              // region 0
    {MMA, 0, st(0)},            // U0 = y_0 R_01; y_0 goes out
    {FOLD, 0, SW},              // lo = x_1 - U0, hi = y_0
    {SOLVE, 1, 0},              // lo = y_1
    {CUT, C1, 0},               // region 1 (and y_0 in region 0 again where needed)
    {MMA, 1, st(16)},           // U1a = [y_0 y_1] R_{01,2}; y_1 goes out
    {LD, lohi(48, 32), 0},      // lo = x_3, hi = x_2
    {FOLD, 1, 0},               // hi = x_2 - U1a
    {MMA, 2, SW},               // U1b = [y_0 y_1] R_{01,3}; lo = x_2', hi = x_3
    {SOLVE, 2, 0},              // lo = y_2
    {FOLD, 2, 0},               // hi = x_3 - U1b
    {CUT, C0, 0},               // region 0
    {MMA, 3, st(32)},           // U2 = y_2 R_23; y_2 goes out
    {FOLD, 3, SW},              // lo = x_3 - U1b - U2
    {SOLVE, 3, st(48)},         // y_3
    {END, 0, 0}};
// NP = 32
__constant__ Step kProg32[] = {
    {LD, lohi(0, 16), 0}, {SOLVE, 0, 0}, {CUT, C0, 0}, {MMA, 0, st(0)},
    {FOLD, 0, SW}, {SOLVE, 1, st(16)}, {END, 0, 0}};
static_assert(sizeof(kProg64) / sizeof(Step) <= kMaxSteps && sizeof(kProg32) / sizeof(Step) <= kMaxSteps,
              "program length");

}  // namespace tcf

// X: rows [0, P.m) of the pass's input (ldx), Q: its output (ldq; may be X
// itself). rk: R_k packed P.np x P.np. colmax (may be null): receives, by
// atomicMax, a bit pattern with the exponent of max |q_ij| per column j < n
// (the high word of the pattern; the low word zero).
template <int NP>
__global__ void __launch_bounds__(tcf::THREADS, 1)
tc_fused_solve_kernel(const double* X, int64_t ldx, double* Q, int64_t ldq, Params P, int pass,
                      const double* __restrict__ rk, unsigned long long* __restrict__ colmax,
                      DevState* __restrict__ st) {
  using namespace tcf;
  using tc::smem_u32;
  using G = FGeo<NP>;
  if (!st->run_trsm[pass]) return;
  extern __shared__ uint8_t dsm[];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  uint8_t* bb = base + G::OFF_B;
  double* rdb = (double*)(base + G::OFF_R);
  double* rinv = (double*)(base + G::OFF_RINV);
  __shared__ __align__(8) uint64_t mdone[SLOTS];  // the slot's MMAs done (tcgen05.commit)
  __shared__ uint32_t tslot;
  __shared__ int Eb[NP];  // column exponents of the B planes
  __shared__ int err_sh[SLOTS];
  __shared__ Step prog[kMaxSteps];
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
  for (int u = 0; u < G::NU; ++u) setup_eb(rk, np, u, Eb);
  if (tid < SLOTS) err_sh[tid] = 0;
  constexpr int NSTEPS = (NP == 64 ? sizeof(kProg64) : sizeof(kProg32)) / sizeof(Step);
  if (tid < NSTEPS) prog[tid] = NP == 64 ? kProg64[tid] : kProg32[tid];
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
  for (int u = 0; u < G::NU; ++u) setup_b(rk, np, u, Eb, bb);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  SlotCtx ctx;
  ctx.sbuf = base + slot * SBUF;
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

  // 256-bit row accesses for blocks that lie within n, 32-byte aligned
  const bool ax = ((uintptr_t)X & 31) == 0 && (ldx & 3) == 0;
  const bool aq = ((uintptr_t)Q & 31) == 0 && (ldq & 3) == 0;

  uint32_t cm[2] = {0, 0};  // lane c: the largest |q| high word of columns c and 32 + c
  uint32_t phase = 0;       // completed waits on mdone[slot]
  uint32_t commits = 0;     // commits to mdone[slot] (thread 0 of the slot)
  bool failed = false;      // slot-uniform: a wait ran out
  int nsolve = 0;           // the slot's solves so far

  // Every slot runs the same iterations (a slot whose tile lies past m works
  // on zero rows and stores nothing), so the turns stay matched; after a wait
  // has run out the slot skips its cuts, MMAs, waits and folds but keeps its
  // turns.
  for (int64_t it = 0;; ++it) {
    const int64_t tile0 = (it * gridDim.x + blockIdx.x) * SLOTS;
    if (tile0 * ROWS >= m) break;  // uniform in the CTA
    const int64_t g = (tile0 + slot) * ROWS + r;
    double lo[16], hi[16];
    int E = 0;         // the row's scale exponent for the current product
    bool fin = true;   // the values multiplied are finite
#pragma unroll 1
    for (int k = 0;; ++k) {
      const Step sp = prog[k];
      if (sp.op == END) break;
      switch (sp.op) {
        case LD: {
          const int c0 = 16 * (sp.arg & 3), c1 = 16 * (sp.arg >> 2);
          load16(lo, X, ldx, g, m, c0, n, ax && c0 + 16 <= n);
          load16(hi, X, ldx, g, m, c1, n, ax && c1 + 16 <= n);
          break;
        }
        case SOLVE:
          turn_take(slot, nsolve);
          solve16(lo, rdb + 256 * sp.arg, rinv + 16 * sp.arg);
          turn_pass(slot, nsolve);
          ++nsolve;
          break;
        case CUT: {
          const unsigned long long mx = absmax16(lo);
          const bool f = (mx >> 52) != 0x7FF;
          const int e = f ? tc::split_exp(mx) : 0;
          bool again = false;  // C1: the row cuts y_0 (hi) again with y_1's scale
          if (sp.arg == C1) {
            again = fin && f && e > E;
            if (again) E = e;
            fin = fin && f;
          } else {
            fin = f;
            E = sp.arg == C0H ? e + 2 : e;
          }
          if (failed) break;
          // q = 0: lo into region 0 (C0, C0H) or 1 (C1); q = 1 (C1 only, rows
          // with `again`): hi into region 0, between two swaps
#pragma unroll 1
          for (int q = 0; q < (sp.arg == C1 ? 2 : 1); ++q) {
            const bool other = q == 1;
            if (other && !__any_sync(0xffffffffu, again)) break;
            if (other) swap16(lo, hi);
            if (!other || again) cut16(lo, ctx, E, sp.arg == C1 && !other ? 1 : 0);
            if (other) swap16(lo, hi);
          }
          break;
        }
        case MMA:
          if (!failed) mma_product(ctx, sp.arg, commits);
          break;
        case FOLD:
          if (!failed) failed = !mma_wait(ctx, phase);
          if (!failed) fold16(hi, ctx, E, fin, Eb + plan(sp.arg).eoff);
          break;
      }
      if (sp.post & ST) {
        const int c0 = 16 * (sp.post >> 2);
        store16(lo, Q, ldq, g, m, c0, n, aq && c0 + 16 <= n, lane, cm);
      }
      if (sp.post & SW) swap16(lo, hi);
    }
  }
  if (slot < TURNS && nsolve > 0)  // the last arrival for this slot
    asm volatile("bar.sync %0, %1;" :: "r"(turn_bar(slot, nsolve - 1)), "r"(2 * ROWS) : "memory");
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
