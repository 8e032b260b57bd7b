// Conversions between FP64 and double-FP32 (hi + lo) from the IEEE bit
// patterns, with 32-bit integer and FP32 operations only.
//
// On this GPU a conversion between FP64 and FP32 issues at about a
// seventieth of the FP32 rate and an FP64 add at a twenty-fifth, so the
// split hi = fl32(x), lo = fl32(x - hi) by conversions costs some 45 issue
// cycles per warp and real on those pipes; the bit-level forms below give
// the same bits from about 30 integer and FP32 operations.  Values outside
// the ranges they handle (tiny, huge, subnormal or non-finite) take the
// conversions.
//
// The functions compile for host and device so that a host test can check
// them bit for bit against the host's own conversions.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define DFB_HD __host__ __device__ __forceinline__
#else
#define DFB_HD inline
#endif

namespace ntu {

DFB_HD uint64_t dfb_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
DFB_HD double dfb_double(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}
DFB_HD uint32_t dfb_fbits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
DFB_HD float dfb_float(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}
DFB_HD float dfb_add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}

// The value of an integer 0 <= v < 2^23 as a float, exactly: the bits of
// 2^23 + v minus 2^23.
DFB_HD float dfb_small_int(uint32_t v) { return dfb_float(0x4b000000u | v) - 8388608.0f; }

// hi = fl32(x) and lo = fl32(x - hi), both rounded to nearest even.  The
// bit path covers |x| in [2^-73, 2^127): the 53-bit significand m of x
// splits into its top 24 bits s (rounded to nearest even on the 29 bits r
// below them) and the remainder r - (carry ? 2^29 : 0), which is exact and
// at most 2^28 in magnitude; r's float is the once-rounded sum of its two
// exactly representable halves, and both results are normal floats there.
DFB_HD void df_split_real(double x, float& hi, float& lo) {
  const uint64_t b = dfb_bits(x);
  const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
  const int E = (int)((bh >> 20) & 0x7ffu);
  if (E < 950 || E > 1149) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
    return;
  }
  const uint32_t sign = bh & 0x80000000u;
  uint32_t s = (((bh & 0xfffffu) | 0x100000u) << 3) | (bl >> 29);   // 2^23 <= s < 2^24
  int32_t r = (int32_t)(bl & 0x1fffffffu);
  if (r > (1 << 28) || (r == (1 << 28) && (s & 1u))) {
    s += 1u;
    r -= 1 << 29;
  }
  uint32_t ef = (uint32_t)(E - 896);
  if (s == (1u << 24)) {
    s = 1u << 23;
    ef += 1u;
  }
  hi = dfb_float(sign | (ef << 23) | (s & 0x7fffffu));
  if (r == 0) {
    lo = 0.0f;                                    // x - hi = +0 exactly
    return;
  }
  const uint32_t a = (uint32_t)(r < 0 ? -r : r);
  const float fa = dfb_add_rn(dfb_small_int(a >> 12) * 4096.0f, dfb_small_int(a & 0xfffu));
  // fa 2^(E - 1075) with the sign of x (r) : the exponent field moves by E - 1075
  const uint32_t fb = dfb_fbits(fa) + (uint32_t)((E - 1075) << 23);
  lo = dfb_float(fb | (r < 0 ? sign ^ 0x80000000u : sign));
}

// (double)f exactly, from the bits for zeros and normal floats.
DFB_HD double df_widen(float f) {
  const uint32_t u = dfb_fbits(f);
  const uint32_t ex = (u >> 23) & 0xffu;
  if (ex == 0xffu || (ex == 0u && (u & 0x7fffffu) != 0u)) return (double)f;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if (ex == 0u) return dfb_double(sign);
  return dfb_double(sign | ((uint64_t)(ex + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
}

}  // namespace ntu
