// tc_gram.cu -- the Gram matrix A = Q^T Q on the BF16 tensor cores (tcgen05),
// accurate to FP64 level, for n <= 128.
//
// The FP64 pipe of this GPU issues 2 DFMA per clock per SM, so the Gram matrix
// of a tall-skinny matrix costs as much as the substitution. The tensor cores
// multiply BF16 exactly into FP32, which allows an exact fixed-point split:
//
//  * every column j gets a scale sigma_j = 2^E_j > 2 max_i |q_ij| (the column
//    maxima come from colmax_kernel, or from the one-sweep substitution that
//    wrote Q);
//  * q_ij / sigma_j * 2^56 is rounded to an integer N, |N| < 2^55, and cut
//    into eight signed digits a_0 .. a_7 (a_0 most significant; a_1 .. a_7 in
//    [-64, 63], a_0 in [-64, 64]: the balanced split of tc_common.cuh), so
//    q_ij = sigma_j * sum_s a_s 2^(-7(s+1)) up to at most sigma_j 2^-57, with
//    an error of zero mean; every digit is exactly a BF16 number;
//  * a product of two digits is at most 2^12 and the tensor core accumulates
//    it exactly in FP32 as long as a sum stays within 2^24: 1024 rows of up to
//    four digit pairs (4 * 1024 * 64^2 = 2^24);
//  * D_d = sum over digit pairs (s, t) with s + t = d, d = 0 .. 7, is read back
//    from tensor memory every 1024 rows (in two shares, lanes 0..63 of tile d
//    and lanes 64..127 of tile d - 1, added at the end). The digit sums are
//    exact integers, so U = D_0 2^21 + D_1 2^14 + D_2 2^7 + D_3 and
//    T = D_4 2^21 + ... + D_7 (per 1024 rows and share below 2^45.1) are
//    exact in int64; W = 2^17 U + round(T / 2^11) (below 2^62.2; the rounding
//    of T costs at most 2^-53 sigma_j sigma_k per group, zero mean) is the
//    group's 2^-35 U + 2^-63 T in units of 2^-52 sigma_j sigma_k, converted to
//    FP64 once per group and added up in FP64 over the CTA's groups (an FP64
//    sum of about m / 1024 terms, far inside the bound below). The FP64 pipe,
//    the scarce one, does no work per row. Pairs with s + t > 7 (at most
//    7 * 2^12 * 2^-70 < 2^-55 of sigma_j sigma_k per row, zero mean) are
//    dropped.
//
// The result differs from q_j^T q_k by at most about m 2^-54 sigma_j sigma_k
// (each value rounded to 2^-57 of its scale, and the pairs s + t > 7 not
// formed). With sigma <= 4 max |q| that is at most about 8.5 m u ||q_j||
// ||q_k||, so ||E|| <= 8.5 m n u ||Q||^2: a norm-wise Gram error of the FP64
// form's order, inside the 11 (mn + n(n+1)) u ||Q||^2 shift of Eq. (finds2),
// so the factorization keeps its guarantees. Unlike truncation, the rounding
// and the signed digits leave the error unbiased: the diagonal does not come
// out systematically low, which matters where a pass's plain Cholesky decides
// at the margin (Alg. 2's breakdown rule).
//
// Blocks: the columns form operand blocks of 64. For n <= 64 one block, and
// every CTA computes it; for 64 < n <= 128 the Gram matrix is the blocks
// (0,0), (1,1) and (0,1), each computed by its own set of CTAs over all rows.
// A CTA of block (J, K) cuts the digits of column blocks J (the A operand) and
// K (the B operand, the same planes when J = K) and writes its block's
// entries of the packed upper triangle into its partial slot, zeros elsewhere.
//
// Layout: the operands are the digit planes of a chunk of KC rows (KC = 64 for
// n <= 64, 32 above, so that two operand blocks fit a 64 KB stage), K-major
// (the chunk rows are the K dimension), no swizzle: core matrices of 8
// columns x 8 rows (16 bytes per column), the KC / 8 row groups of a column
// block contiguous (128 bytes apart), column blocks 16 KC bytes apart. A plane
// of one block is 128 KC bytes, and the planes lie in digit order, so that
// one A operand (M = 128) holds digits s and s + 1 of the block's columns and
// one B operand (N up to 256) the planes t .. t + 3 side by side: tile x of
// tensor memory (columns 64x .. 64x+63) accumulates the pairs (s, x - s) in
// lanes 0..63 (d = x) and (s + 1, x - s) in lanes 64..127 (d = x + 1), for
// s = 0, 2, 4, 6. Eight tiles use all 512 columns; six MMAs per K step cover
// every pair with s + t <= 7 (the issue of an MMA costs about as much for
// N = 256 as for N = 64, so wide ones are what keeps the tensor core busy).
//
// One CTA of 256 + 32 threads per SM. Two 64 KB digit-plane stages: the threads cut
// chunk c + 1 while the tensor core works on chunk c. When the rows are
// contiguous (ld = n, m n even, 16-byte aligned), thread 0 brings chunk c + 2
// into one of two 32 KB FP64 staging buffers with an asynchronous bulk copy
// (cp.async.bulk, completion counted in bytes on an mbarrier), so the global
// loads leave the critical path; otherwise the threads load the rows directly. Thread 0 issues the MMAs
// (descriptors are a base plus compile-time offsets) and commits them to the
// stage's mbarrier. For the read-back, warp w serves the tensor-memory lane
// quadrant w % 4 and the 32 columns 32 (w / 4) ..; on a diagonal block a warp
// whose rows all lie below its columns (strict lower triangle) skips it. Every
// wait has an iteration limit; past it the kernel records SCQR3_E_TIMEOUT,
// skips the rest and frees its tensor memory.
#include "tc_common.cuh"

namespace scqr3 {

namespace tc {

constexpr int BW = 64;              // columns of one operand block
constexpr int NPMAX = 256;          // largest padded n
constexpr int GROUP = 1024;         // rows per read-back group
constexpr int THREADS = 256;   // slicer and read-back threads (the producer warp comes on top)
constexpr uint32_t LBO = 128;       // K-direction core-matrix stride
constexpr int STAGE = 65536;        // digit planes of one chunk (one or two operand blocks)
constexpr int XSTAGE = 32768;       // FP64 rows of one chunk (KC n 8 bytes), staged by a bulk copy
constexpr size_t SMEM = 2 * (size_t)STAGE + 2 * (size_t)XSTAGE + 1024;  // + alignment slack

// Geometry of a chunk of KC rows.
template <int KC>
struct ChunkGeo {
  static constexpr int CHUNKS = GROUP / KC;    // chunks per read-back group
  static constexpr uint32_t SBO = 16 * KC;     // column-block stride
  static constexpr int PLANE = KC * BW * 2;    // bytes per digit plane of one block
  static constexpr int BREG = 8 * PLANE;       // the B operand's planes (off-diagonal block)
};
static_assert(8 * ChunkGeo<64>::PLANE == STAGE && 16 * ChunkGeo<32>::PLANE == STAGE, "stage size");
static_assert(32 * 128 * 8 == XSTAGE && 64 * 64 * 8 == XSTAGE, "staging size (bulk copies for n <= 128)");

template <int KC>
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(ChunkGeo<KC>::SBO >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// byte offset of digit plane s within an operand block's planes (natural
// order, so that planes s, s + 1 form one A operand of M = 128 and planes
// t .. t + 3 one B operand of N = 256)
template <int KC>
__host__ __device__ constexpr uint32_t plane_off(int s) {
  return s * ChunkGeo<KC>::PLANE;
}

// The MMAs of one chunk. A = digit planes s and s + 1 (M = 128: rows 0..63
// digit s, rows 64..127 digit s + 1, of the block's 64 columns), B = planes
// t0 .. t0 + nt - 1 side by side (N = 64 nt), written from tensor column
// 64 (s + t0): tile x (columns 64 x ..) then accumulates the pairs (s, x - s)
// in lanes 0..63 (d = x) and (s + 1, x - s) in lanes 64..127 (d = x + 1).
// For s = 0, 2, 4, 6 and t = 0 .. 7 - s that is every pair with s + t <= 7
// (and a few with d = 8 in the upper lanes of tile 7, never read), in six
// MMAs per K step: the cost of an MMA's issue does not grow with N, so few
// wide ones keep the tensor core busy. Tile x holds at most 4 pairs per lane
// half; per 1024 rows a sum stays within 4 * 1024 * 64^2 = 2^24, exact in
// FP32. OFFD: the B operand is the second block's planes. The start-address
// field of a descriptor is its low 14 bits (address / 16); the operands of a
// stage lie within 64 KB of its base and every stage below 256 KB, so offsets
// are added to the base descriptor without carrying out of the field.
template <int KC, bool OFFD, int S, int T0, int NT, int KK>
__device__ __forceinline__ void issue_one(uint64_t dbase, uint32_t tmem, uint32_t idesc, bool first_chunk) {
  constexpr uint64_t aoff = (plane_off<KC>(S) + KK * 2 * LBO) >> 4;
  constexpr uint64_t boff = ((OFFD ? ChunkGeo<KC>::BREG : 0) + plane_off<KC>(T0) + KK * 2 * LBO) >> 4;
  // the s = 0 MMAs of the first K step of a group's first chunk write all 8 tiles
  const uint32_t accum = (!first_chunk || S > 0 || KK > 0) ? 1u : 0u;
  mma(tmem + 64 * (S + T0), dbase + aoff, dbase + boff, idesc | ((uint32_t)(8 * NT) << 17), accum);
}
template <int KC, bool OFFD, int KK>
__device__ __forceinline__ void issue_k(uint64_t dbase, uint32_t tmem, uint32_t idesc, bool first_chunk) {
  issue_one<KC, OFFD, 0, 0, 4, KK>(dbase, tmem, idesc, first_chunk);
  issue_one<KC, OFFD, 0, 4, 4, KK>(dbase, tmem, idesc, first_chunk);
  issue_one<KC, OFFD, 2, 0, 4, KK>(dbase, tmem, idesc, first_chunk);
  issue_one<KC, OFFD, 2, 4, 2, KK>(dbase, tmem, idesc, first_chunk);
  issue_one<KC, OFFD, 4, 0, 4, KK>(dbase, tmem, idesc, first_chunk);
  issue_one<KC, OFFD, 6, 0, 2, KK>(dbase, tmem, idesc, first_chunk);
  if constexpr (KK + 1 < KC / 16) issue_k<KC, OFFD, KK + 1>(dbase, tmem, idesc, first_chunk);
}

}  // namespace tc

// Column scales: colmax[j] = max_i |q_ij| (pairs: max_i |hi_ij|) as the bit pattern of a double (the
// patterns of non-negative doubles order like the numbers; an Inf or NaN
// entry, exponent field all ones, orders above every finite one, so
// colmax[j] is then non-finite) over rows [0, m) of src. Integer operations
// only: the FP64 pipe is the slow one. Thread t serves column t % nc (nc = 64,
// 128 or 256 >= n) and row t / nc of each group of 256 / nc rows.
__global__ void __launch_bounds__(256)
colmax_kernel(const double* __restrict__ src, int64_t lds, int64_t m, int n, int pass,
              unsigned long long* __restrict__ colmax, const DevState* __restrict__ st, int pairs) {
  if (pass >= 0 && !(st->run_trsm[pass] && st->gram_after[pass])) return;
  __shared__ unsigned long long red[256];
  const int tid = threadIdx.x;
  const int nc = n > 128 ? 256 : n > 64 ? 128 : 64, rs = 256 / nc;
  const int j = tid % nc, r0 = tid / nc;
  const unsigned long long* s64 = reinterpret_cast<const unsigned long long*>(src);
  // pairs: the max of |hi| (the float's pattern in the low word; the Gram
  // kernel widens the scale by one bit for lo)
  const unsigned long long ABS = pairs ? 0x7FFFFFFFull : 0x7FFFFFFFFFFFFFFFull;
  unsigned long long mx = 0;
  if (j < n) {
    // 8 rows per thread in flight: the scan is bound by memory latency otherwise
    const int64_t step = (int64_t)gridDim.x * rs;
    int64_t i = (int64_t)blockIdx.x * rs + r0;
    for (; i + 7 * step < m; i += 8 * step) {
      unsigned long long v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = s64[(i + u * step) * lds + j];
#pragma unroll
      for (int u = 0; u < 8; ++u) mx = mx > (v[u] & ABS) ? mx : (v[u] & ABS);
    }
    for (; i < m; i += step) {
      const unsigned long long v = s64[i * lds + j] & ABS;
      mx = mx > v ? mx : v;
    }
  }
  red[tid] = mx;
  __syncthreads();
  if (tid < nc && j < n) {
    unsigned long long b = red[tid];
    for (int q = 1; q < rs; ++q) b = b > red[tid + nc * q] ? b : red[tid + nc * q];
    if (pairs) {  // the float's value as a double pattern (Inf/NaN: +Inf)
      const uint32_t fb = (uint32_t)b;
      b = ((fb >> 23) & 0xFF) == 0xFF ? 0x7FF0000000000000ull
                                      : (unsigned long long)__double_as_longlong((double)__uint_as_float(fb));
    }
    atomicMax(&colmax[j], b);
  }
}

namespace tc {
// z = L_b^T x for the 8 consecutive rows x of one column (BS-row blocks b, b + 1, ..),
// as the oblique Gram's Z = L^T Q of Alg. 4. Only the first nvalid rows exist;
// m is a multiple of BS, so a block lies wholly among them or wholly past them
// (past rows are zero, and their blocks are not read).
template <int BS>
__device__ __forceinline__ void apply_lt8(double (&x)[8], const double* __restrict__ lt, int64_t b, int nvalid) {
  constexpr int BSP = BS * (BS + 1) / 2;
#pragma unroll
  for (int o = 0; o < 8; o += BS) {
    if (o >= nvalid) break;
    const double* L = lt + (b + o / BS) * BSP;
#pragma unroll
    for (int i = 0; i < BS; ++i) {
      double z = 0.0;
#pragma unroll
      for (int l = i; l < BS; ++l) z = fma(__ldg(L + pk_idx(BS, i, l)), x[o + l], z);
      x[o + i] = z;
    }
  }
}
}  // namespace tc

// Oblique column scales: colmax[j] = max_i |z_ij| over Z = L^T Q (Alg. 4) as
// the bit pattern of a double, with z formed exactly as the Gram kernel forms
// it (tc::apply_lt8 on the same 8-row units), so the scales bound the values
// the kernel cuts. Thread units are (8-row group, column), consecutive columns
// in consecutive threads.
__global__ void __launch_bounds__(256)
colmax_obl_kernel(const double* __restrict__ src, int64_t lds, int64_t m, int n, int pass,
                  unsigned long long* __restrict__ colmax, const DevState* __restrict__ st,
                  const double* __restrict__ lt, int bs, int64_t blk0) {
  if (pass >= 0 && !(st->run_trsm[pass] && st->gram_after[pass])) return;
  __shared__ unsigned long long red[256];
  const int tid = threadIdx.x;
  const int nc = n > 64 ? 128 : 64, gs = 256 / nc;  // column slots, 8-row groups per block pass
  const int j = tid % nc, g0 = tid / nc;
  unsigned long long mx = 0;
  if (j < n) {
    for (int64_t g = blockIdx.x * (int64_t)gs + g0; g * 8 < m; g += (int64_t)gridDim.x * gs) {
      double x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) x[r] = g * 8 + r < m ? src[(g * 8 + r) * lds + j] : 0.0;
      const int64_t b = blk0 + (g * 8) / bs;
      const int nv = m - g * 8 < 8 ? (int)(m - g * 8) : 8;
      switch (bs) {
        case 1: tc::apply_lt8<1>(x, lt, b, nv); break;
        case 2: tc::apply_lt8<2>(x, lt, b, nv); break;
        case 4: tc::apply_lt8<4>(x, lt, b, nv); break;
        default: tc::apply_lt8<8>(x, lt, b, nv); break;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(x[r]) & 0x7FFFFFFFFFFFFFFFull;
        mx = mx > v ? mx : v;
      }
    }
  }
  red[tid] = mx;
  __syncthreads();
  if (tid < nc && j < n) {
    unsigned long long b = red[tid];
    for (int q = 1; q < gs; ++q) b = b > red[tid + nc * q] ? b : red[tid + nc * q];
    atomicMax(&colmax[j], b);
  }
}

// KC = 64: n <= 64, every CTA computes the one block. KC = 32: 64 < n <= 128;
// CTAs [0, gd) compute block (0,0), [gd, 2 gd) block (1,1), the rest (0,1).
// OBL: the Gram matrix Z^T Z of Z = L^T Q for an oblique B given by the
// packed L_j^T (lt; row 0 of src is in block blk0; B's blocks of bs = 1, 2, 4
// or 8 rows divide the 8-row units), with the column scales of Z from
// colmax_obl_kernel; the CTAs of the diagonal blocks also return ||Q||_F^2 of
// their rows and columns in the slot's last entry, for the oblique shift of
// Eq. (finds2B).
template <int KC, bool OBL>
__global__ void __launch_bounds__(tc::THREADS + 32, 1)
tc_gram_kernel(const double* __restrict__ src, int64_t lds, Params P, int pass,
               const unsigned long long* __restrict__ colmax, double* __restrict__ partials, int part_stride,
               DevState* __restrict__ st, int bulk, int pairs, int gd, const double* __restrict__ lt, int64_t blk0) {
  using namespace tc;
  using GK = ChunkGeo<KC>;
  constexpr int CHUNKS = GK::CHUNKS;
  const int NPK = KC == 64 ? 64 : P.np;  // packed layout of the slots (64, 128 or 256)
  if (pass >= 0 && !(st->run_trsm[pass] && st->gram_after[pass])) return;
  extern __shared__ uint8_t dsm[];
  uint8_t* stages = (uint8_t*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
  uint8_t* xst = stages + 2 * STAGE;           // two FP64 staging buffers
  __shared__ __align__(8) uint64_t bar[2];     // MMAs of the stage's chunk done (tcgen05.commit)
  __shared__ __align__(8) uint64_t full[2];    // staged rows of the buffer's chunk arrived (bytes)
  __shared__ __align__(8) uint64_t pfull[2];   // digit planes of the stage written (256 arrivals)
  __shared__ __align__(8) uint64_t tfree;      // tensor memory read back (256 arrivals)
  __shared__ uint32_t tslot;
  __shared__ int Esh[NPMAX];
  __shared__ double sig[NPMAX];
  __shared__ volatile int err_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == THREADS / 32;  // warp 8: copies and MMAs (lane 0)
  const int n = P.n;
  const int64_t m = P.m;
  double* part = partials + (int64_t)blockIdx.x * part_stride;

  // this CTA's block (cj, ck), its ordinal among the CTAs of the block, and
  // their count: nd = NPK / 64 diagonal blocks of gd CTAs each, then the
  // nd (nd - 1) / 2 off-diagonal blocks (0,1), (0,2), .., (1,2), .. sharing
  // the rest evenly (the last one takes the remainder)
  int cj = 0, ck = 0, cta = blockIdx.x, ncta = gridDim.x;
  if (KC == 32) {
    const int nd = NPK / BW, no = nd * (nd - 1) / 2;
    if ((int)blockIdx.x < nd * gd) {
      cj = ck = blockIdx.x / gd;
      cta = blockIdx.x % gd;
      ncta = gd;
    } else {
      const int r = blockIdx.x - nd * gd, rest = gridDim.x - nd * gd, go = rest / no;
      int p = go > 0 ? r / go : no - 1;
      if (p > no - 1) p = no - 1;
      cta = r - p * go;
      ncta = p == no - 1 ? rest - p * go : go;
      for (int a = 0, q = p; a < nd; ++a) {
        if (q < nd - 1 - a) {
          cj = a;
          ck = a + 1 + q;
          break;
        }
        q -= nd - 1 - a;
      }
    }
  }
  const bool offd = cj != ck;
  const int colA = BW * cj, colB = BW * ck;  // first columns of the A and B operand blocks

  int bad = 0;
  if (tid < NPMAX) {
    int E = -1000;
    double sg = 0.0;
    if (tid < n) {
      const double cm = __longlong_as_double((long long)colmax[tid]);
      if (!isfinite(cm)) {
        bad = 1;  // non-finite input: the Gram matrix is NaN
      } else if (cm > 0.0) {
        const int ex = (int)((colmax[tid] >> 52) & 0x7FF);
        E = (ex ? ex : 1) - 1023 + 2 + pairs;  // cm < 2^(E-1) (pairs: |hi| + |lo| < 2^(E-1))
        sg = ldexp(1.0, E);
      }
    }
    Esh[tid] = E;
    sig[tid] = sg;
  }
  if (__syncthreads_or(bad)) {
    for (int e = tid; e < part_stride; e += blockDim.x) part[e] = NAN;
    return;
  }

  if (tid == 0) {
    err_sh = 0;
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bar[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&full[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&pfull[i])), "r"(THREADS));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&tfree)), "r"(THREADS));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const uint32_t sbase = smem_u32(stages);
  // D F32, A and B BF16, both K-major, M = 128 (N set per MMA)
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);

  // This CTA's chunks in order: ordinal k is chunk k % CHUNKS of its group
  // cta + (k / CHUNKS) ncta; the sequence ends at the first chunk past m
  // (only the last group can be partial).
  auto row0_of = [&](uint32_t k) -> int64_t {
    const int64_t g = cta + (int64_t)(k / CHUNKS) * ncta;
    const int64_t r0 = (g * CHUNKS + (k % CHUNKS)) * KC;
    return r0 < m ? r0 : -1;
  };
  auto group_end = [&](uint32_t k) { return (k % CHUNKS) == CHUNKS - 1 || row0_of(k + 1) < 0; };

  // read-back of the slicer warps: lane quadrant qd = warp % 4 (row 32 qd +
  // lane of the tiles; rows 0..63 hold d = e, rows 64..127 d = e + 4),
  // columns 32 h .. 32 h + 31; on a diagonal block rows 32..63 x columns
  // 0..31 lie below the diagonal
  constexpr int CW = 32;
  const int qd = warp & 3, h = (warp >> 2) & 1;
  const int row = 32 * qd + lane;
  const int jr = row & 63;
  const bool upper = row < 64;
  const bool rb_skip = !offd && (qd & 1) == 1 && h == 0;
  double f2 = 0.0;  // OBL: ||Q||_F^2 of this thread's entries (diagonal-block CTAs)
  // diagonal-block CTAs: sum of the squares of digit 4 of this thread's
  // values (one column, tid % 64), the square pair (4, 4) of d = 8 that the
  // tiles do not hold; added to the diagonal it keeps the split unbiased there
  long long s44 = 0;
  // this thread's share of its 32 entries, in units of 2^-52 sigma_j sigma_k:
  // per 1024-row group the digit sums fold exactly into U (d = 0..3) and
  // T (d = 4..7), both below 2^45.1; W = 2^17 U + round(T / 2^11) (below
  // 2^62.2, so 2^-35 U + 2^-63 T to within 2^-53 of sigma_j sigma_k) goes to
  // FP64 once per group, and the groups add up in FP64
  double acc[CW];
#pragma unroll
  for (int k = 0; k < CW; ++k) acc[k] = 0.0;

  uint32_t issued = 0;     // producer: chunks whose rows were requested
  uint32_t committed = 0;  // producer: chunks whose MMAs were committed
  if (producer) {
    if (lane == 0) {
      auto stage_in = [&](uint32_t k) {
        const int64_t r0 = row0_of(k);
        if (r0 < 0) return;
        issued = k + 1;
        const int rows = (int)((m - r0) < KC ? (m - r0) : KC);
        const uint32_t bytes = (uint32_t)rows * (uint32_t)n * 8u;
        const uint32_t fb = smem_u32(&full[k & 1]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(fb), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(xst + (k & 1) * XSTAGE)), "l"(src + r0 * lds), "r"(bytes), "r"(fb) : "memory");
      };
      if (bulk) {
        stage_in(0);
        stage_in(1);
      }
      for (uint32_t k = 0; row0_of(k) >= 0; ++k) {
        const int stg = k & 1;
        const uint32_t q = k % CHUNKS, gi = k / CHUNKS;
        bool okw = wait_parity(smem_u32(&pfull[stg]), (k >> 1) & 1, P.wait_ns_gram);  // planes written, staging consumed
        if (okw && bulk) stage_in(k + 2);
        if (okw && q == 0 && gi > 0) okw = wait_parity(smem_u32(&tfree), (gi - 1) & 1, P.wait_ns_gram);  // tiles read back
        if (!okw || err_sh) {
          err_sh = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint64_t db = desc<KC>(sbase + stg * STAGE);
        if constexpr (KC == 32) {
          if (offd) tc::issue_k<KC, true, 0>(db, tmem, idesc, q == 0);
          else tc::issue_k<KC, false, 0>(db, tmem, idesc, q == 0);
        } else {
          tc::issue_k<KC, false, 0>(db, tmem, idesc, q == 0);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&bar[stg])) : "memory");
        committed = k + 1;
      }
    }
  } else {
    // units (j, ig): 8 consecutive rows of operand column j; j < 64 is block
    // cj (column colA + j), j >= 64 block ck (off-diagonal CTAs: colB + j - 64)
    const int lgc = offd ? 7 : 6;
    const int units = (KC / 8) << lgc;
    for (uint32_t chunk = 0;; ++chunk) {
      const int64_t row0 = row0_of(chunk);
      if (row0 < 0 || err_sh) break;
      const int rows = (int)((m - row0) < KC ? (m - row0) : KC);
      const int stg = chunk & 1;
      bool w = chunk < 2 || wait_parity(smem_u32(&bar[stg]), ((chunk - 2) >> 1) & 1, P.wait_ns_gram);  // planes free
      if (w && bulk) w = wait_parity(smem_u32(&full[stg]), (chunk >> 1) & 1, P.wait_ns_gram);            // rows staged
      if (!w) {
        err_sh = 1;
        break;
      }
      uint8_t* sb = stages + stg * STAGE;
      const double* xs = (const double*)(xst + stg * XSTAGE);
      if constexpr (!OBL) {
        // two units per thread at a time (the second empty when units run
        // out), so that their integer work interleaves
        for (int u = tid; u < units; u += 2 * THREADS) {
          const bool two = u + THREADS < units;
          unsigned long long F[2][8];
          int jj[2], igg[2];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int uu = u + h2 * THREADS;
            const bool live = h2 == 0 || two;
            const int j = uu & ((1 << lgc) - 1), ig = uu >> lgc;
            jj[h2] = j;
            igg[h2] = ig;
            const int col = j < BW ? colA + j : colB + (j - BW);
            const int E = Esh[col < NPMAX ? col : 0];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              const int i = ig * 8 + r;
              double x = 0.0;
              if (live && col < n && i < rows) x = bulk ? xs[i * n + col] : src[(row0 + i) * lds + col];
              F[h2][r] = pairs ? tc::biased56_pair((unsigned long long)__double_as_longlong(x), E)
                               : tc::biased56(x, E);
            }
          }
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            if (h2 == 1 && !two) break;
            if (!offd) {
#pragma unroll
              for (int r = 0; r < 8; ++r) {
                const int d4 = (int)((F[h2][r] >> 21) & 127) - 64;
                s44 += d4 * d4;
              }
            }
            const int j = jj[h2];
            uint8_t* dst = sb + (j >> 6) * GK::BREG + ((j & 63) >> 3) * GK::SBO + igg[h2] * LBO + (j & 7) * 16;
            uint4 w[8];
            tc::planes8(F[h2], w);
#pragma unroll
            for (int sd = 0; sd < 8; ++sd) *(uint4*)(dst + tc::plane_off<KC>(sd)) = w[sd];
          }
        }
      } else
      for (int u = tid; u < units; u += THREADS) {
        const int j = u & ((1 << lgc) - 1), ig = u >> lgc;
        const int col = j < BW ? colA + j : colB + (j - BW);
        const int E = Esh[col];
        unsigned long long F[8];  // biased fixed-point values (balanced split)
        if constexpr (!OBL) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = ig * 8 + r;
            double x = 0.0;
            if (col < n && i < rows) x = bulk ? xs[i * n + col] : src[(row0 + i) * lds + col];
            F[r] = pairs ? tc::biased56_pair((unsigned long long)__double_as_longlong(x), E) : tc::biased56(x, E);
          }
        } else {
          double xv[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = ig * 8 + r;
            xv[r] = 0.0;
            if (col < n && i < rows) xv[r] = bulk ? xs[i * n + col] : src[(row0 + i) * lds + col];
          }
          if (!offd) {
#pragma unroll
            for (int r = 0; r < 8; ++r) f2 = fma(xv[r], xv[r], f2);
          }
          // m is a multiple of bs: the unit's blocks lie wholly before or past the end
          if (ig * 8 < rows) {
            const int64_t b = blk0 + (row0 + ig * 8) / P.bs;
            const int nv = rows - ig * 8 < 8 ? rows - ig * 8 : 8;
            switch (P.bs) {
              case 1: tc::apply_lt8<1>(xv, lt, b, nv); break;
              case 2: tc::apply_lt8<2>(xv, lt, b, nv); break;
              case 4: tc::apply_lt8<4>(xv, lt, b, nv); break;
              default: tc::apply_lt8<8>(xv, lt, b, nv); break;
            }
          }
#pragma unroll
          for (int r = 0; r < 8; ++r) F[r] = tc::biased56(xv[r], E);
        }
        if (!offd) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int d4 = (int)((F[r] >> 21) & 127) - 64;
            s44 += d4 * d4;
          }
        }
        uint8_t* dst = sb + (j >> 6) * GK::BREG + ((j & 63) >> 3) * GK::SBO + ig * LBO + (j & 7) * 16;
        uint4 w[8];
        tc::planes8(F, w);
#pragma unroll
        for (int sd = 0; sd < 8; ++sd) *(uint4*)(dst + tc::plane_off<KC>(sd)) = w[sd];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&pfull[stg])) : "memory");
      if (!group_end(chunk)) continue;
      // end of a group: all its MMAs (the last commit covers every earlier one)
      if (!wait_parity(smem_u32(&bar[stg]), (chunk >> 1) & 1, P.wait_ns_gram)) {
        err_sh = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (!rb_skip) {
        const uint32_t tq = tmem + ((uint32_t)(32 * qd) << 16) + CW * h;
#pragma unroll
        for (int c = 0; c < CW; c += 8) {
          // upper rows hold d = e (tiles 0..7), lower rows d = e + 1 (tiles
          // 0..6; tile 7 would be d = 8). D_d enters U with weight
          // 2^(7 (3 - d)) (d <= 3) or T with weight 2^(7 (7 - d)).
          long long U[8], T[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) U[k] = T[k] = 0;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            if (!upper && e == 7) break;
            uint32_t v[8];
            tc::ld8(tq + 64 * e + c, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int d = upper ? e : e + 1;
            const int sh = d < 4 ? 7 * (3 - d) : 7 * (7 - d);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const long long dv = (long long)__float2int_rn(__uint_as_float(v[k])) << sh;
              if (d < 4) U[k] += dv;
              else T[k] += dv;
            }
          }
#pragma unroll
          for (int k = 0; k < 8; ++k)
            acc[c + k] += (double)((long long)((unsigned long long)U[k] << 17) + ((T[k] + 1024) >> 11));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&tfree)) : "memory");
    }
  }
  __syncthreads();
  if (err_sh) {
    atomicCAS(&st->status, SCQR3_OK, SCQR3_E_TIMEOUT);
    // let the MMAs and copies already issued finish (bounded) before the memory goes away
    if (producer && lane == 0) {
      if (committed > 0) wait_parity(smem_u32(&bar[(committed - 1) & 1]), ((committed - 1) >> 1) & 1, kWaitNs);
      for (uint32_t k = committed; k < issued; ++k) wait_parity(smem_u32(&full[k & 1]), (k >> 1) & 1, kWaitNs);
    }
  }

  // rows 64..127 hold the d + 1 share of the same entries: add them to rows 0..63
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  double* xch = (double*)stages;                    // 64 x 64 shares (32 KB) of stage 0,
  long long* s44sh = (long long*)(xch + BW * BW);  // then the slicers' digit-4 square sums
  if (!producer && !upper) {
#pragma unroll
    for (int k = 0; k < CW; ++k) xch[jr * BW + CW * h + k] = acc[k];
  }
  if (!producer) s44sh[tid] = s44;
  __syncthreads();
  if (!producer && upper && !rb_skip) {
    const double sj = sig[colA + jr];
#pragma unroll
    for (int k = 0; k < CW; ++k) {
      const int c = CW * h + k;
      if (offd || c >= jr) {
        double a = 0x1p-52 * (acc[k] + xch[jr * BW + c]);
        if (!offd && c == jr) {  // the diagonal: the square pair (4, 4), weight 2^-70
          long long q = 0;
          for (int t = jr; t < THREADS; t += BW) q += s44sh[t];
          a = fma(0x1p-70, (double)q, a);
        }
        part[pk_idx(NPK, colA + jr, colB + c)] = a * sj * sig[colB + c];
      }
    }
  }
  if (KC == 32) {  // the other blocks' entries of this slot
    for (int e = tid; e < NPK * NPK; e += blockDim.x) {
      const int r = e / NPK, c = e % NPK;
      if (c >= r && !((r >> 6) == cj && (c >> 6) == ck)) part[pk_idx(NPK, r, c)] = 0.0;
    }
  }
  if constexpr (OBL) {
    __shared__ double f2w[THREADS / 32 + 1];
    for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    if (lane == 0) f2w[warp] = f2;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < THREADS / 32; ++w) t += f2w[w];
      part[pk_size(NPK)] = t;
    }
  } else {
    if (tid == 0) part[pk_size(NPK)] = 0.0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// ---- host side ----------------------------------------------------------------------------

cudaError_t tc_setup() {
  cudaError_t e = cudaFuncSetAttribute(tc_gram_kernel<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_gram_kernel<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_gram_kernel<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_gram_kernel<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);
  return e;
}

int tc_groups(int64_t m) { return (int)((m + tc::GROUP - 1) / tc::GROUP); }

// CTAs of the tensor-core Gram of m rows (np = 64: one block; np = 128: three
// blocks, np = 256: ten, at least one CTA each).
int tc_grid(int64_t m, int np, int sms) {
  const int64_t g = tc_groups(m);
  if (np <= 64) return (int)(g < sms ? (g < 1 ? 1 : g) : sms);
  const int64_t t = (np <= 128 ? 3 : 10) * (g < 1 ? 1 : g);
  return (int)(t < sms ? t : sms);
}

// Column scales then the tensor-core Gram of rows [0, P.m) of src into `grid`
// slots; for an oblique B (P.bs > 0) of Z = L^T Q, with lt the packed L_j^T and
// row 0 of src in block blk0.
// scan = 0: colmax already holds the column maxima of src (the fused
// substitution that wrote it emitted them), so the scan is skipped.
// offd_only (np = 128, 256): only the off-diagonal 64-column block pairs are
// formed (every CTA serves them; the diagonal blocks of the result are zero).
void launch_tc_gram(int grid, int sms, cudaStream_t s, const double* src, int64_t lds, const Params& P, int pass,
                    unsigned long long* colmax, double* partials, int part_stride, DevState* st, int pairs,
                    const double* lt, int64_t blk0, int scan, int offd_only) {
  // the slots hold the packed np x np layout; np = 128 and 256 need a CTA per
  // block (3 and 10 blocks)
  const int nblk = P.np == 256 ? 10 : P.np == 128 ? 3 : 1;
  if ((P.np != 64 && P.np != 128 && P.np != 256) || part_stride != pk_size(P.np) + 1 || grid < nblk) return;
  if (scan) cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * tc::NPMAX, s);
  const int rs = P.n > 128 ? 1 : P.n > 64 ? 2 : 4;
  const int64_t want = (P.m + rs - 1) / rs;
  const int cg = (int)(want < (int64_t)sms * 8 ? (want < 1 ? 1 : want) : (int64_t)sms * 8);
  if (!scan) {
  } else if (P.bs > 0) {
    const int gs = P.n > 64 ? 2 : 4;
    const int64_t wg = (P.m / 8 + 1 + gs - 1) / gs;
    const int og = (int)(wg < (int64_t)sms * 8 ? (wg < 1 ? 1 : wg) : (int64_t)sms * 8);
    colmax_obl_kernel<<<og, 256, 0, s>>>(src, lds, P.m, P.n, pass, colmax, st, lt, P.bs, blk0);
  } else {
    colmax_kernel<<<cg, 256, 0, s>>>(src, lds, P.m, P.n, pass, colmax, st, pairs);
  }
  // bulk copies need contiguous rows, 16-byte aligned, and chunk sizes that are
  // multiples of 16 bytes (m n even)
  const int bulk = (P.n <= 128 && lds == P.n && ((uintptr_t)src & 15) == 0 && ((P.m * P.n) & 1) == 0) ? 1 : 0;
  const bool obl = P.bs > 0;
  if (P.np == 64) {
    if (obl)
      tc_gram_kernel<64, true><<<grid, tc::THREADS + 32, tc::SMEM, s>>>(src, lds, P, pass, colmax, partials,
                                                                        part_stride, st, bulk, pairs, grid, lt, blk0);
    else
      tc_gram_kernel<64, false><<<grid, tc::THREADS + 32, tc::SMEM, s>>>(src, lds, P, pass, colmax, partials,
                                                                         part_stride, st, bulk, pairs, grid, lt, blk0);
    return;
  }
  // np = 128 (256): gd CTAs for each of the 2 (4) diagonal blocks, the rest
  // (which also cut twice the columns) for the 1 (6) off-diagonal ones
  const int g = tc_groups(P.m);
  const int nd = P.np / 64, no = nd * (nd - 1) / 2;
  int gd = grid >= (nd + no) * g ? g : (10 * grid) / (10 * nd + 12 * no);
  if (gd < 1) gd = 1;
  if (grid - nd * gd < no) gd = (grid - no) / nd;  // every block gets a CTA (grid >= nblk)
  if (offd_only) gd = 0;
  if (obl)
    tc_gram_kernel<32, true><<<grid, tc::THREADS + 32, tc::SMEM, s>>>(src, lds, P, pass, colmax, partials,
                                                                      part_stride, st, bulk, pairs, gd, lt, blk0);
  else
    tc_gram_kernel<32, false><<<grid, tc::THREADS + 32, tc::SMEM, s>>>(src, lds, P, pass, colmax, partials,
                                                                       part_stride, st, bulk, pairs, gd, lt, blk0);
}

}  // namespace scqr3
