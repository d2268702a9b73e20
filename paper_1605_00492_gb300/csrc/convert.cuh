// FP64 <-> FP32 conversions on the integer pipe.
//
// On GB300 a hardware FP64<->FP32 conversion issues on the FP64 pipe, which
// retires one warp instruction per 64 cycles per sub-partition, as slow as an
// FP64 FMA.  These conversions use integer operations on the bit patterns:
//   float -> double is exact: re-bias the exponent by 1023 - 127 = 896 and
//     shift the 23-bit significand into the top of the 52-bit one;
//   double -> float rounds to nearest, ties to even (IEEE 754-2008,
//     roundTiesToEven): keep the top 23 significand bits, round up when the
//     29 dropped bits exceed half an ulp, or equal it with an odd kept part; a
//     carry out of the significand increments the exponent, which is the
//     correctly rounded result (up to infinity).
// Values outside the range where these bit manipulations apply (zero,
// subnormal results, infinities, NaN) use the hardware conversion.
#pragma once

namespace hmg {

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(e + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  // biased double exponents 897..1150 map to float exponents 1..254
  if (e < 897u || e > 1150u) return (float)d;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const unsigned kept = (unsigned)(mant >> 29);
  const unsigned long long dropped = mant & 0x1FFFFFFFull;
  unsigned v = ((e - 896u) << 23) | kept;
  const unsigned long long half = 0x10000000ull;
  if (dropped > half || (dropped == half && (kept & 1u))) v += 1u;
  return __uint_as_float(sign | v);
}

template <typename To, typename From>
__device__ __forceinline__ To cvt(From x) {
  return (To)x;
}
// FP64 -> FP32 inside the kernels stays on the hardware conversion: the
// rounding in integer operations measured slower there than the FP64-pipe
// conversion (f64_to_f32 serves the exported conversion utility).
template <>
__device__ __forceinline__ double cvt<double, float>(float x) {
  return f32_to_f64(x);
}

}  // namespace hmg
