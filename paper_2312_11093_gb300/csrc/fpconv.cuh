// FP32 <-> FP64 conversions in integer arithmetic.
//
// On this GPU the FP64 pipe retires about 1.7 lanes per SM per clock, and the
// hardware conversions between FP32 and FP64 run on that pipe.  The residual
// (FP64 -> FP32 for the network input) and the update (FP32 correction ->
// FP64) convert once per unknown and cycle, so they rebuild the IEEE-754 bit
// patterns with integer operations instead: exact for FP32 -> FP64, round to
// nearest even for FP64 -> FP32 (results below the FP32 normal range, which
// need denormal rounding, take the hardware conversion).
#pragma once

#include <cstdint>

namespace mgcnn {

__device__ __forceinline__ double f32_to_f64_exact(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t ex = (b >> 23) & 0xffu, man = b & 0x7fffffu;
  uint64_t r;
  if (ex == 0xffu) {
    r = sign | 0x7ff0000000000000ull | ((uint64_t)man << 29);             // inf, nan
  } else if (ex != 0u) {
    r = sign | ((uint64_t)(ex + 896u) << 52) | ((uint64_t)man << 29);       // normal: 1023 - 127 = 896
  } else if (man == 0u) {
    r = sign;                                                               // signed zero
  } else {
    const int lz = __clz(man) - 8;                                          // FP32 denormal: normalise
    r = sign | ((uint64_t)(897 - lz) << 52) | ((uint64_t)((man << lz) & 0x7fffffu) << 29);
  }
  return __longlong_as_double((long long)r);
}

__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int ex = (int)((b >> 52) & 0x7ffu);
  const uint64_t man = b & 0xfffffffffffffull;
  if (ex == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (man ? 0x400000u : 0u));
  const int e32 = ex - 896;
  if (e32 >= 0xff) return __uint_as_float(sign | 0x7f800000u);            // overflow
  if (e32 <= 0) return (float)x;                                           // FP32 denormal range
  const uint32_t m = (uint32_t)(man >> 29), rem = (uint32_t)(man & 0x1fffffffull);
  uint32_t r = ((uint32_t)e32 << 23) | m;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) r += 1u;      // carry may reach the exponent
  return __uint_as_float(sign | r);
}

// FP64 reciprocal and 16th root with few FP64 instructions, for the setup
// kernels (every FP64 instruction per grid node there costs ~30 us at 4095^2).
// Both start from an FP32 value and refine it by Newton-Raphson iteration in
// FP64 fused multiply-adds (quadratic convergence: an FP32 start, relative error
// ~1e-7, is below FP64 rounding after two steps); results within a few units
// in the last place of the correctly rounded value.

// 1 / d for d > 0 with binary exponent in [-1000, 1000] (callers check): d =
// m 2^e with m in [1, 2); start from the FP32 reciprocal of m truncated to
// FP32 (from the bit pattern, no FP64 conversion), iterate r <- r + r (1 - m r)
// twice, scale by 2^-e (exact).
__device__ __forceinline__ double recip_newton(double d) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  const float mf = __uint_as_float(0x3f800000u | (uint32_t)((b >> 29) & 0x7fffffu));
  double r = f32_to_f64_exact(__frcp_rn(mf));
  r = fma(r, fma(-m, r, 1.0), r);
  r = fma(r, fma(-m, r, 1.0), r);
  return r * __longlong_as_double((long long)(1023 - e) << 52);
}

// x^(1/16) for x in [1, 2^16): z = x^(-1/16) starts in FP32 (exp2f of -log2f(x)
// / 16) and takes two Newton-Raphson steps for z^-16 = x, z <- z + z (1 - x z^16)
// / 16 (no division); then x^(1/16) = 1 / z.
__device__ __forceinline__ double root16_newton(double x) {
  const long long b = __double_as_longlong(x);
  const float xf = __uint_as_float((uint32_t)(((b >> 52) & 0x7ff) - 896) << 23 | (uint32_t)((b >> 29) & 0x7fffffu));
  double z = f32_to_f64_exact(exp2f(-0.0625f * log2f(xf)));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double z2 = z * z, z4 = z2 * z2, z8 = z4 * z4, z16 = z8 * z8;
    z = fma(z, 0.0625 * fma(-x, z16, 1.0), z);
  }
  return recip_newton(z);
}

}  // namespace mgcnn
