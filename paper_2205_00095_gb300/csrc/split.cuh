// Split-precision basis contractions on tensor cores (3xTF32, FP32 accumulation).
//
// The volume term, the face-trace extrapolation and the lift are small dense contractions along
// one axis of an element: out[i] = sum_a C[i][a] x[a] for every line of N nodes.  Gathered over
// a block they are matrix products of shape (lines x N) * (N x N) (or N x 2 for traces, 2 x N
// for the lift), done here with mma.sync.m16n8k8 TF32: a warp multiplies 16 lines (rows of A)
// by the coefficient matrix (B, 8 x 8 with zero padding).  Each operand x is split as
// x = hi + lo with hi, lo TF32 and the product formed as hi*hi + lo*hi + hi*lo in FP32.
//
// The splits and the conversions of FP32 results back to FP64 use the integer bit-pattern
// conversions of bits.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bits.cuh"

namespace dgsrhd {

// TF32 split of a float: hi keeps the top 10 explicit mantissa bits, lo = x - hi (exact in
// FP32), rounded to TF32 by the tensor core's truncation of its low 13 bits.
struct Tf32Pair {
  unsigned hi, lo;
};

__device__ __forceinline__ Tf32Pair split_tf32(float x) {
  const unsigned h = __float_as_uint(x) & 0xffffe000u;
  const float lo = x - __uint_as_float(h);
  Tf32Pair p;
  p.hi = h;
  p.lo = __float_as_uint(lo) & 0xffffe000u;
  return p;
}

__device__ __forceinline__ Tf32Pair split_tf32_f64(double x) { return split_tf32(f64_to_f32_bits(x)); }

// x - r in FP32 from the pairs: (x_hi - r_hi) + (x_lo - r_lo).  The head difference is exact
// when x_hi and r_hi lie within a factor 2 of each other (Sterbenz) and within 2^-24 of itself
// otherwise, so the result is within about 2^-23 of x - r, the accuracy of the FP32 truncation
// of an exact FP64 difference, at no FP64 operation.
__device__ __forceinline__ float dev_f32(F32Pair x, F32Pair r) {
  return __fadd_rn(__fsub_rn(x.hi, r.hi), __fsub_rn(x.lo, r.lo));
}

// D (16x8, f32) += A (16x8, tf32, row) * B (8x8, tf32, col)
__device__ __forceinline__ void mma_tf32(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 3xTF32 product: c += A_lo B_hi + A_hi B_lo + A_hi B_hi (small terms first)
__device__ __forceinline__ void mma_3xtf32(float c[4], const unsigned ahi[4], const unsigned alo[4],
                                           const unsigned bhi[2], const unsigned blo[2]) {
  mma_tf32(c, alo, bhi);
  mma_tf32(c, ahi, blo);
  mma_tf32(c, ahi, bhi);
}

}  // namespace dgsrhd
