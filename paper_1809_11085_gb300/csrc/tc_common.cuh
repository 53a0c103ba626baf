// tc_common.cuh -- device helpers shared by the tensor-core kernels: tcgen05
// issue and read-back, bounded mbarrier waits, and the exact fixed-point digit
// split of FP64 values into 7-bit BF16 digits.
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

// |x| / 2^E * 2^56 truncated to an integer (< 2^56 when |x| < 2^E).
__device__ __forceinline__ unsigned long long fixed56(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  if (ex) mant |= 1ull << 52; else ex = 1;
  const int sh = ex - 1019 - E;  // F = mant * 2^sh
  return sh >= 0 ? (sh <= 3 ? (mant << sh) : (1ull << 56) - 1) : (sh > -64 ? (mant >> -sh) : 0ull);
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

// The same for an element held as a float pair (hi, lo), value hi + lo (the
// mixed form's iterates; hi in the low word). Each float becomes its own
// fixed-point integer and the two are added as signed integers, so no FP64
// arithmetic is needed; E must leave |hi + lo| < 2^E. Returns |F| and sets the
// sign bit (bit 31) in *sign.
__device__ __forceinline__ long long fix_float(uint32_t f, int E) {
  int ex = (int)((f >> 23) & 0xFF);
  long long mant = (long long)(f & 0x7FFFFFu);
  if (ex) mant |= 0x800000ll; else ex = 1;
  const int sh = ex - 94 - E;  // value mant 2^(ex - 150), times 2^(56 - E)
  const long long F = sh >= 0 ? (sh <= 32 ? (mant << sh) : 0x7FFFFFFFFFFFFFll) : (sh > -40 ? (mant >> -sh) : 0ll);
  return (f & 0x80000000u) ? -F : F;
}
__device__ __forceinline__ unsigned long long fixed56_pair(unsigned long long bits, int E, uint32_t* sign) {
  const long long S = fix_float((uint32_t)bits, E) + fix_float((uint32_t)(bits >> 32), E);
  *sign = S < 0 ? 0x80000000u : 0u;
  return (unsigned long long)(S < 0 ? -S : S);
}

// Digit s of two entries (rows r and r + 1 of a column) as a BF16 pair with
// their signs (bits 15 and 31 of `signs`). The digits a, b < 128 are placed
// side by side and ORed into the BF16 pattern of 128 (0x4300): that is the
// exact BF16 value 128 + a, since BF16 resolves units between 128 and 256;
// one exact BF16x2 subtraction of 128 leaves a and b.
template <int S>
__device__ __forceinline__ uint32_t digit_pair(unsigned long long F0, unsigned long long F1, uint32_t signs) {
  const uint32_t lo = (uint32_t)(F0 >> (49 - 7 * S)), hi = (uint32_t)(F1 >> (49 - 7 * S));
  uint32_t w = (__byte_perm(lo, hi, 0x5410) & 0x007F007Fu) | 0x43004300u;
  __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&w);
  v = __hsub2(v, __floats2bfloat162_rn(128.0f, 128.0f));
  return *reinterpret_cast<uint32_t*>(&v) | signs;
}

}  // namespace tc

}  // namespace scqr3
