// ig_f32.cuh -- exact conversions between FP64 and FP32 values done with integer instructions.
//
// On this GPU FP64 instructions, and the hardware conversions between double and float, run at 2
// per clock per SM, against 125 FP32 fused multiply-adds and about 32 integer-to-float
// conversions. The FP32 face-geometry kernels therefore move their data between the two formats
// with the bit manipulations below instead of the conversion instructions.
#pragma once

#include <cuda_runtime.h>

namespace ig {

// x = hi + lo: hi holds the leading 24 significant bits of x (truncated toward zero), lo = x - hi
// rounded to float (its own relative error is 2^-24, so hi + lo carries about 47 significant bits).
// Differences of neighbouring values, (hi_a - hi_b) + (lo_a - lo_b), then keep FP32 relative
// accuracy even when they cancel most of the leading digits of a and b.
// Values below the float normal range (including zero) give hi = lo = 0 (an absolute error below
// 2^-126); values at or above 2^128, infinities and NaNs give hi = NaN.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned top = (unsigned)(b >> 32), bot = (unsigned)b;
  const unsigned sign = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7ffu);  // biased FP64 exponent
  const int ef = e - 896;                      // biased FP32 exponent of the same power of two
  if (ef >= 1 && ef <= 254) {
    hi = __uint_as_float(sign | ((unsigned)ef << 23) | ((top & 0xfffffu) << 3) | (bot >> 29));
    // lo = (low 29 mantissa bits) * 2^(e - 1075); that power of two has FP32 biased exponent e - 948
    const int es = e - 948;
    const float scale = es >= 1 ? __uint_as_float((unsigned)es << 23) : 0.0f;
    lo = __uint_as_float(__float_as_uint(__uint2float_rn(bot & 0x1fffffffu) * scale) | sign);
  } else if (ef < 1) {
    hi = 0.0f;
    lo = 0.0f;
  } else {
    hi = __uint_as_float(0x7fc00000u);
    lo = 0.0f;
  }
}

// x rounded to float, to nearest with ties to even (IEEE 754 binary64 -> binary32): the 29
// mantissa bits that binary32 drops decide the rounding; a carry out of the kept 23 bits moves into
// the exponent field, and past the largest float it gives infinity, as the rule requires. Zeros,
// results below the float normal range, infinities and NaNs (rare in the operator) take the
// hardware conversion.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned top = (unsigned)(b >> 32), bot = (unsigned)b;
  const unsigned e = (top >> 20) & 0x7ffu;  // biased FP64 exponent
  if (e < 897u || e > 1150u) return __double2float_rn(x);
  const unsigned m = ((top & 0xfffffu) << 3) | (bot >> 29);  // the kept 23 mantissa bits
  const unsigned rest = bot & 0x1fffffffu;                    // the dropped 29
  const unsigned up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
  return __uint_as_float(((top & 0x80000000u) | ((e - 896u) << 23) | m) + up);
}

// The FP64 value of a float, exactly (denormal floats are taken as zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double((long long)sign);
  const unsigned long long eo = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (eo << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

}  // namespace ig
