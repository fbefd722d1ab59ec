// FP64 <-> FP32 conversions on the bit patterns, and the FP64 reciprocal and roots built on them.
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

// Products and sums of FP32 head-and-tail pairs (the value is hi + lo), on the FP32 pipe, for
// quantities that need about 44 bits rather than FP64's 53 (those the split-precision path
// feeds its FP32 deviations with, and the adjoint's transposed contractions).  mul_pair: the product of
// the heads, its rounding error by one fused multiply-add (exact, Dekker's two-product) and the
// two cross terms; the lo x lo term and the roundings of the cross terms leave it within about
// 2^-46 of the exact product.  add_pair: Knuth's two-sum of the heads (the exact sum as s + e)
// with both tails added to e; it is within about 2^-46 (|a| + |b|) of the exact sum (relative
// to the sum itself for addends of one sign).
__device__ __forceinline__ F32Pair mul_pair(F32Pair a, F32Pair b) {
  const float h = __fmul_rn(a.hi, b.hi);
  return F32Pair{h, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -h)))};
}

__device__ __forceinline__ F32Pair add_pair(F32Pair a, F32Pair b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return F32Pair{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

// x 2^k for a runtime k in [-1023, 1023]: exponent arithmetic on the integer pipe for a normal x
// (zero when the result leaves the normal range downwards, infinity upwards), x itself for zero,
// infinity and NaN, and one FP64 multiplication for a subnormal x.
__device__ __forceinline__ double scale_pow2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0x7ff || (b << 1) == 0) return x;
  if (ex == 0) return x * __longlong_as_double((long long)(1023 + k) << 52);
  const long long sign = b & (long long)0x8000000000000000ULL;
  const int ne = ex + k;
  if (ne <= 0) return __longlong_as_double(sign);
  if (ne >= 0x7ff) return __longlong_as_double(sign | 0x7ff0000000000000LL);
  return __longlong_as_double(b + ((long long)k << 52));
}

// x 2^k for a normal x whose result stays normal, by adding k to the exponent field on the
// integer pipe (exact, like the multiplication it replaces); zero (and a subnormal) is returned
// unchanged.
template <int K>
__device__ __forceinline__ double ldexp_bits(double x) {
  const long long b = __double_as_longlong(x);
  return (b & 0x7ff0000000000000LL) == 0 ? x : __longlong_as_double(b + ((long long)K << 52));
}

// Reciprocal from an FP32 seed r0 and one third-order correction: with h = 1 - x r0 (one fused
// multiply-add), 1/x = r0 / (1 - h) = r0 (1 + h + h^2 + h^3 + ...), so r0 + r0 (h + h^2) leaves
// a truncation error h^3.  The seed is within ~2^-21 (the FP32 truncation of x and MUFU's
// reciprocal), so h^3 < 2^-63 and the result is within one rounding of 1/x: three FP64
// instructions, where two Newton-Raphson steps r + r (1 - x r) (the classical iteration for
// division, e.g. P. Markstein, IBM J. Res. Dev. 34 (1990) 111) take four and CUDA's division
// about eight DFMA-equivalents.  For |x| outside [2^-100, 2^100] (where the FP32 seed would not
// be normal), and for zero, infinity or NaN, the reciprocal is a true division.
__device__ __forceinline__ double recip_nr(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;
  if (e < 1023 - 100 || e > 1023 + 100) return 1.0 / x;
  const double r0 = f32_to_f64_bits(__fdividef(1.0f, f64_to_f32_bits(x)));
  const double h = fma(-x, r0, 1.0);
  return fma(r0, fma(h, h, h), r0);
}

// Roots from an FP32 seed and one third-order correction.  The seed r0 ~ x^(-1/2) (MUFU's FP32
// reciprocal square root, within 2 FP32 ulp) or r0 ~ |x|^(-1/3) (below) has relative error below
// 2^-20; with h = 1 - x r0^2 (resp. 1 - |x| r0^3), formed by one fused multiply-add, the
// binomial series
//   (1 - h)^(-1/2) = 1 + h/2 + 3h^2/8 + O(h^3),   (1 - h)^(-1/3) = 1 + h/3 + 2h^2/9 + O(h^3)
// gives x^(-1/2) = r0 (1 - h)^(-1/2), sqrt(x) = x r0 (1 - h)^(-1/2) and x^(-1/3) = r0 (1 - h)^(-1/3)
// with a truncation error O(h^3) < 2^-60: the result is within about one ulp.  The second-order
// term lies below 2^-40, so FP32 carries it to within 2^-62: it is formed from h truncated to
// FP32 and added to the FP64 first-order term by one fused multiply-add.  That leaves four FP64
// instructions for the square root and the reciprocal square root and five for the reciprocal
// cube root, where CUDA's sqrt, rsqrt and rcbrt take about 7.5, 4.8 and 15 DFMA-equivalents.
// Outside [2^-120, 2^120] (where the FP32 seed would not be a normal number), for zero, negative
// (square roots), infinite or NaN arguments, CUDA's own function is used.
__device__ __forceinline__ bool seed_range(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;
  return e >= 1023 - 120 && e <= 1023 + 120;
}

// c h^2 for |h| < 2^-18, in FP32 (h truncated to FP32; zero once h^2 leaves the FP32-normal range)
__device__ __forceinline__ double sq_term_f32(double h, float c) {
  const float hf = f64_to_f32_bits(h);
  return f32_to_f64_bits(c * hf * hf);
}

// sqrt(y) for y >= 0 (y itself for +-0, NaN for y < 0)
__device__ __forceinline__ double sqrt_nr(double y) {
  if (__double2hiint(y) < 0 || !seed_range(y))
    return (__double_as_longlong(y) << 1) == 0 ? y : y * rsqrt(y);
  const double r0 = f32_to_f64_bits(rsqrtf(f64_to_f32_bits(y)));
  const double s0 = y * r0;
  const double h = fma(-s0, r0, 1.0);
  return fma(s0, fma(h, 0.5, sq_term_f32(h, 0.375f)), s0);
}

// 1/sqrt(y), with CUDA's rsqrt semantics outside the seed range (+inf at +0, -inf at -0, NaN
// below zero, 0 at +inf)
__device__ __forceinline__ double rsqrt_nr(double y) {
  if (__double2hiint(y) < 0 || !seed_range(y)) return rsqrt(y);
  const double r0 = f32_to_f64_bits(rsqrtf(f64_to_f32_bits(y)));
  const double h = fma(-(y * r0), r0, 1.0);
  return fma(r0, fma(h, 0.5, sq_term_f32(h, 0.375f)), r0);
}

// y^(-1/3) with the sign of y (y != 0).  FP32 seed: the bit pattern of |y|^(-1/3) is about
// K - bits(|y|)/3 with K = (4/3) 127 2^23 (the exponent field read as a logarithm), refined by
// three FP32 Newton steps r <- r (4 - a r^3)/3 to within ~5e-7.
__device__ __forceinline__ double rcbrt_nr(double y) {
  if (!seed_range(y)) return rcbrt(y);
  const long long sign = __double_as_longlong(y) & (long long)0x8000000000000000ULL;
  const double ay = __longlong_as_double(__double_as_longlong(y) ^ sign);  // |y|
  const float a = f64_to_f32_bits(ay);
  float r = __uint_as_float(0x54aaaaaau - __float_as_uint(a) / 3u);
#pragma unroll
  for (int k = 0; k < 3; ++k) r = r * (4.0f - (a * r) * (r * r)) * (1.0f / 3.0f);
  const double r0 = f32_to_f64_bits(r);
  const double h = fma(-(ay * r0), r0 * r0, 1.0);
  const double q = fma(r0, fma(h, 1.0 / 3.0, sq_term_f32(h, 2.0f / 9.0f)), r0);
  return __longlong_as_double(__double_as_longlong(q) | sign);
}

}  // namespace dgsrhd
