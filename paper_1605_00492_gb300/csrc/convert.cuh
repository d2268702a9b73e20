// FP64 <-> FP32 conversions on the integer pipe.
//
// On GB300 a hardware FP64<->FP32 conversion issues on the FP64 pipe, which
// retires one warp instruction per 64 cycles per sub-partition, as slow as an
// FP64 FMA.  f32_to_f64 / f64_to_f32 use integer operations on the bit patterns
// (IEEE 754 binary32 and binary64 layouts):
//   float -> double is exact.  Normal values re-bias the exponent by
//     1023 - 127 = 896 and shift the 23-bit significand into the top of the
//     52-bit one.  A subnormal float m * 2^-149 (m < 2^23) becomes a normal
//     double: with k the index of m's leading one bit, the value is
//     2^(k - 149) * (m / 2^k), exponent field k + 874, significand m shifted
//     so that bit k lands on the implicit bit.  Zeros keep their sign,
//     infinities map to infinities, NaNs keep sign and payload with the quiet
//     bit set.  No branch reaches the FP64 pipe.
//   double -> float rounds to nearest, ties to even (IEEE 754-2008,
//     roundTiesToEven): keep the top 23 significand bits, round up when the
//     29 dropped bits exceed half an ulp, or equal it with an odd kept part; a
//     carry out of the significand increments the exponent, which is the
//     correctly rounded result (up to infinity).  Values outside the range
//     where this applies (zero, subnormal results, infinities, NaN) use the
//     hardware conversion.
#pragma once

namespace hmg {

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  unsigned long long ex = e + 896u, mm = (unsigned long long)m << 29;
  if (e == 0u) {
    const int k = 31 - __clz(m | 1u);  // m = 0 gives k = 0; its fields are cleared below
    ex = m ? (unsigned long long)(k + 874) : 0ull;
    mm = m ? (((unsigned long long)m << (52 - k)) & 0xFFFFFFFFFFFFFull) : 0ull;
  } else if (e == 0xFFu) {
    ex = 0x7FFull;
    if (m) mm |= 1ull << 51;
  }
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) | (ex << 52) | mm;
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

// Inside the kernels both directions use the hardware conversion: a single
// instruction keeps the unrolled column sweeps small, and there the FP64-pipe
// cost of a conversion overlaps memory time.  The integer forms above serve
// the exported conversion utility (hmg_convert_*).
template <typename To, typename From>
__device__ __forceinline__ To cvt(From x) {
  return (To)x;
}

}  // namespace hmg
