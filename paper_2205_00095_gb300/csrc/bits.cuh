// FP64 <-> FP32 conversions on the bit patterns, and two FP64 primitives built on them.
//
// On this GPU FP64<->FP32 conversion instructions issue on the FP64 pipe at the DFMA rate,
// which is the bottleneck of every FP64 kernel here, so conversions are done with integer
// operations (FP32-normal range; smaller magnitudes flush to zero, larger saturate to
// infinity).
#pragma once

#include <cuda_runtime.h>

namespace dgsrhd {

// double -> float by truncating the mantissa, via bit operations only
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const int hw = __double2hiint(x);
  const unsigned lw = (unsigned)__double2loint(x);
  const unsigned sign = (unsigned)hw & 0x80000000u;
  const int e = (hw >> 20) & 0x7ff;
  const unsigned mant = (((unsigned)hw & 0xfffffu) << 3) | (lw >> 29);
  const int ef = e - 896;  // rebias 1023 -> 127
  unsigned bits;
  if (ef <= 0)
    bits = sign;  // zero, subnormal or below the FP32-normal range
  else if (ef >= 255)
    bits = sign | 0x7f800000u | (e == 0x7ff && ((hw & 0xfffff) | lw) ? 0x400000u : 0u);
  else
    bits = sign | ((unsigned)ef << 23) | mant;
  return __uint_as_float(bits);
}

// float -> double (exact for FP32-normal values), via bit operations only
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned ef = (b >> 23) & 0xffu;
  const unsigned mf = b & 0x7fffffu;
  int hw;
  unsigned lw;
  if (ef == 0) {
    hw = (int)sign;
    lw = 0u;
  } else if (ef == 255) {
    hw = (int)(sign | 0x7ff00000u | (mf >> 3));
    lw = mf << 29;
  } else {
    hw = (int)(sign | ((ef + 896u) << 20) | (mf >> 3));
    lw = mf << 29;
  }
  return __hiloint2double(hw, (int)lw);
}

// x minus its FP32 truncation (f64_to_f32_bits keeps the top 23 of the 52 mantissa bits), as an
// FP32 truncated to 24 significant bits, from the bit pattern alone: the low 29 mantissa bits,
// normalised.  Zero when they are zero, for zeros, subnormals, infinities and NaNs, and where
// the part falls below the FP32-normal range.
__device__ __forceinline__ float f64_lo_f32_bits(double x) {
  const int hw = __double2hiint(x);
  const unsigned rem = (unsigned)__double2loint(x) & 0x1fffffffu;
  const int e = (hw >> 20) & 0x7ff;
  const int lz = __clz(rem);                  // 3..32; the leading one of rem at bit 31 - lz
  const int ef = e - 917 - lz;                // FP32 biased exponent of that leading one
  const unsigned mant = ((rem << (lz & 31)) >> 8) & 0x7fffffu;
  const unsigned bits = ((unsigned)hw & 0x80000000u) | ((unsigned)ef << 23) | mant;
  return (rem == 0u || e == 0x7ff || ef <= 0) ? 0.0f : __uint_as_float(bits);
}

// FP32 head and tail of an FP64 value (integer operations only)
struct F32Pair {
  float hi, lo;
};

__device__ __forceinline__ F32Pair f32_pair(double x) {
  F32Pair q;
  q.hi = f64_to_f32_bits(x);
  q.lo = f64_lo_f32_bits(x);
  return q;
}

// Reciprocal by the Newton-Raphson iteration r <- r + r (1 - x r), which squares the relative
// error at every step (the classical iteration for division, e.g. P. Markstein, IBM J. Res.
// Dev. 34 (1990) 111), from an FP32 seed: the seed is within ~2^-21, so two steps reach FP64
// rounding (each step is two DFMAs, against the ~8.6 DFMA-equivalents of a division here).
// For |x| outside [2^-100, 2^100] (where the FP32 seed would not be normal), and for zero,
// infinity or NaN, the reciprocal is a true division.
__device__ __forceinline__ double recip_nr(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;
  if (e < 1023 - 100 || e > 1023 + 100) return 1.0 / x;
  double r = f32_to_f64_bits(__fdividef(1.0f, f64_to_f32_bits(x)));
  double t = fma(-x, r, 1.0);
  r = fma(r, t, r);
  t = fma(-x, r, 1.0);
  return fma(r, t, r);
}

// sqrt(y) as y rsqrt(y) (about 1.7 DFMA-equivalents cheaper than sqrt here) for finite y > 0,
// within a few ulp of sqrt; y for y = +-0, NaN for y < 0, y = +inf or NaN.
__device__ __forceinline__ double sqrt_rs(double y) {
  return (__double_as_longlong(y) << 1) == 0 ? y : y * rsqrt(y);
}

}  // namespace dgsrhd
