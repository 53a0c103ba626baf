// tc_common.cuh -- device helpers shared by the tensor-core kernels: tcgen05
// issue and read-back, bounded mbarrier waits, and the balanced fixed-point
// digit split of FP64 values into signed 7-bit BF16 digits.
#pragma once
#include <cuda_bf16.h>

#include "fp64_device.cuh"

namespace scqr3 {

namespace tc {

// Waits on mbarriers are bounded in time (%globaltimer, nanoseconds). A
// hand-off wait (one warp waiting for another's work) uses the call's limit,
// Params::wait_ns (default kWaitNs; a test can shorten it to force the
// timeout path); a drain wait before tensor memory is freed always uses
// kWaitNs, so that no MMA or copy of the CTA is still in flight then.
constexpr long long kWaitNs = 2000000000ll;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of the phase with parity `parity`, for at most
// limit_ns nanoseconds; false if it did not complete in time. A limit of zero
// gives up at once (the test hook that drives the timeout path).
__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity, long long limit_ns) {
  if (limit_ns <= 0) return false;
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  if (done) return true;
  const unsigned long long t0 = globaltimer();
  for (;;) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if ((long long)(globaltimer() - t0) > limit_ns) return false;
  }
}

__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                 "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
               : "r"(taddr) : "memory");
}

// The balanced fixed-point split shared by the tensor-core kernels. A value x
// with |x| < 2^(E-1) becomes N = round(x 2^(56-E)), |N| < 2^55 (half-way cases
// away from zero: the error is at most 2^(E-57) and symmetric), written as
// N = sum_s d_s 2^(7 (7 - s)) with digits d_1 .. d_7 in [-64, 63] and d_0 in
// [-64, 64]. With M = N + BIAS56 (64 in every 7-bit field; 0 <= M < 129 2^49)
// the digits are the unsigned fields of M less 64: d_s = ((M >> (49 - 7 s)) &
// 127) - 64 for s >= 1 and d_0 = (M >> 49) - 64. Every digit is exactly a BF16
// number and a product of two is at most 2^12 in magnitude. The rounding and
// the signed digits make the error of the split zero-mean, unlike truncation,
// which biases every |x| low.
constexpr unsigned long long BIAS56 = 0x0081020408102040ull;  // 64 (1 + 2^7 + ... + 2^49)

// M = round(x 2^(56-E)) + BIAS56 for |x| < 2^(E-1) (integer operations only).
__device__ __forceinline__ unsigned long long biased56(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  if (ex) mant |= 1ull << 52; else ex = 1;
  const int sh = ex - 1019 - E;  // N = mant 2^sh, sh <= 2 when |x| < 2^(E-1)
  const unsigned long long F =
      sh >= 0 ? (sh <= 2 ? (mant << sh) : (1ull << 55) - 1) : (sh > -64 ? (mant + (1ull << (-sh - 1))) >> -sh : 0ull);
  return (long long)bits < 0 ? BIAS56 - F : BIAS56 + F;
}

// The same for an element held as a float pair (hi, lo), value hi + lo (the
// mixed form's iterates; hi in the low word): each float is rounded to the
// fixed point on its own and the two integers are added, so no FP64
// arithmetic is needed; E must leave |hi| + |lo| < 2^(E-1).
__device__ __forceinline__ long long fix_float(uint32_t f, int E) {
  int ex = (int)((f >> 23) & 0xFF);
  long long mant = (long long)(f & 0x7FFFFFu);
  if (ex) mant |= 0x800000ll; else ex = 1;
  const int sh = ex - 94 - E;  // value mant 2^(ex - 150), times 2^(56 - E)
  const long long F = sh >= 0 ? (sh <= 32 ? (mant << sh) : 0x7FFFFFFFFFFFFFll)
                              : (sh > -40 ? ((mant + (1ll << (-sh - 1))) >> -sh) : 0ll);
  return (f & 0x80000000u) ? -F : F;
}
__device__ __forceinline__ unsigned long long biased56_pair(unsigned long long bits, int E) {
  return BIAS56 + (unsigned long long)(fix_float((uint32_t)bits, E) + fix_float((uint32_t)(bits >> 32), E));
}

__device__ __forceinline__ void ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(taddr) : "memory");
}

__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr) : "memory");
}

// Digit s of two entries (biased M0, M1: rows r and r + 1 of a column) as a
// BF16 pair: the fields f (< 128; f <= 128 for s = 0) are placed side by side
// and added to the BF16 pattern of 128 (0x4300), which gives the exact BF16
// value 128 + f (BF16 resolves units between 128 and 256, and 0x4300 + 128 is
// the pattern of 256); one exact BF16x2 subtraction of 192 leaves f - 64.
template <int S>
__device__ __forceinline__ uint32_t digit_pair(unsigned long long M0, unsigned long long M1) {
  const uint32_t lo = (uint32_t)(M0 >> (49 - 7 * S)), hi = (uint32_t)(M1 >> (49 - 7 * S));
  const uint32_t w0 = __byte_perm(lo, hi, 0x5410);
  uint32_t w = S == 0 ? (w0 & 0x00FF00FFu) + 0x43004300u : (w0 & 0x007F007Fu) | 0x43004300u;
  __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&w);
  v = __hsub2(v, __floats2bfloat162_rn(192.0f, 192.0f));
  return *reinterpret_cast<uint32_t*>(&v);
}

// Eight consecutive values as 8 digit planes of one core-matrix row each (16
// bytes: 8 BF16 digits), at dst + s * plane; |x| < 2^(E-1).
__device__ __forceinline__ void cut8(const double* x, int E, uint8_t* dst, uint32_t plane) {
  unsigned long long M[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) M[r] = biased56(x[r], E);
#define SCQR3_CUTS(S)                                \
  {                                                  \
    uint4 w;                                         \
    w.x = digit_pair<S>(M[0], M[1]);                 \
    w.y = digit_pair<S>(M[2], M[3]);                 \
    w.z = digit_pair<S>(M[4], M[5]);                 \
    w.w = digit_pair<S>(M[6], M[7]);                 \
    *(uint4*)(dst + (S) * plane) = w;                \
  }
  SCQR3_CUTS(0) SCQR3_CUTS(1) SCQR3_CUTS(2) SCQR3_CUTS(3) SCQR3_CUTS(4) SCQR3_CUTS(5) SCQR3_CUTS(6)
  SCQR3_CUTS(7)
#undef SCQR3_CUTS
}

// Scale exponent of a non-negative bit-pattern maximum for the balanced
// split: 2^(E-1) > the value (-1000 for zero, so every digit is 0).
__device__ __forceinline__ int split_exp(unsigned long long mx) {
  if (mx == 0) return -1000;
  const int ex = (int)(mx >> 52);
  return (ex ? ex : 1) - 1023 + 2;
}

}  // namespace tc

}  // namespace scqr3
