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

// M = round(x 2^(56-E)) + BIAS56 for |x| < 2^(E-1) (integer operations only):
// with x = mant 2^(ex - 1075), N = mant 2^(ex - 1019 - E) = (4 mant) / 2^K,
// K = 1021 + E - ex >= 0, rounded by adding 2^(K-1) before the shift (for
// K <= 2 that adds less than 4 to a multiple of 4 and changes nothing; K is
// capped at 63, where N is 0 already).
__device__ __forceinline__ unsigned long long biased56(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  if (ex) mant |= 1ull << 52; else ex = 1;
  int K = 1021 + E - ex;
  K = K < 0 ? 0 : (K > 63 ? 63 : K);
  const unsigned long long F = ((mant << 2) + ((1ull << K) >> 1)) >> K;
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

// The 8 digit planes of 8 biased values M[0..7] as BF16 pairs: word p of w[s]
// holds digit s of M[2p] (low half) and of M[2p + 1] (high half). The fields
// are taken two digits at a time: chunk j of a value (bits 42 - 14 j up, 14
// bits; 15 for j = 0, whose top field d_0 + 64 <= 128 has 8) from two values
// side by side in one word; one shift and one mask give the fields f of digit
// 2 j, one mask those of digit 2 j + 1. A field f (< 128; <= 128 for s = 0)
// added to the BF16 pattern of 128 (0x4300) gives the exact BF16 value 128 + f
// (BF16 resolves units between 128 and 256, and 0x4300 + 128 is the pattern of
// 256); one exact BF16x2 subtraction of 192 leaves the digit f - 64.
__device__ __forceinline__ void planes8(const unsigned long long (&M)[8], uint4 (&w)[8]) {
  uint32_t d[8][4];
  const __nv_bfloat162 k192 = __floats2bfloat162_rn(192.0f, 192.0f);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t t0 = (uint32_t)(M[2 * p] >> (42 - 14 * j)), t1 = (uint32_t)(M[2 * p + 1] >> (42 - 14 * j));
      const uint32_t C = __byte_perm(t0, t1, 0x5410);
      uint32_t ev = j == 0 ? ((C >> 7) & 0x00FF00FFu) + 0x43004300u : ((C >> 7) & 0x007F007Fu) | 0x43004300u;
      uint32_t od = (C & 0x007F007Fu) | 0x43004300u;
      __nv_bfloat162 ve = __hsub2(*reinterpret_cast<__nv_bfloat162*>(&ev), k192);
      __nv_bfloat162 vo = __hsub2(*reinterpret_cast<__nv_bfloat162*>(&od), k192);
      d[2 * j][p] = *reinterpret_cast<uint32_t*>(&ve);
      d[2 * j + 1][p] = *reinterpret_cast<uint32_t*>(&vo);
    }
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) w[s] = make_uint4(d[s][0], d[s][1], d[s][2], d[s][3]);
}

// Eight consecutive values as 8 digit planes of one core-matrix row each (16
// bytes: 8 BF16 digits), at dst + s * plane; |x| < 2^(E-1).
__device__ __forceinline__ void cut8(const double* x, int E, uint8_t* dst, uint32_t plane) {
  unsigned long long M[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) M[r] = biased56(x[r], E);
  uint4 w[8];
  planes8(M, w);
#pragma unroll
  for (int s = 0; s < 8; ++s) *(uint4*)(dst + s * plane) = w[s];
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
