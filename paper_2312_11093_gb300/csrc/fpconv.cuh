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

}  // namespace mgcnn
