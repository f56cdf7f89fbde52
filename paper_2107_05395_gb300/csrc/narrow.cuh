// FP64 -> FP32 truncation with integer operations, for the refinement residuals
// (host and device; the host build serves the CPU tests).
#pragma once

#include "arith.cuh"

namespace sb {

// FP64 -> FP32 by truncation toward zero with integer operations: for |v| in
// FP32's normal range the sign, the re-biased exponent and the top 23 fraction
// bits.  Smaller magnitudes give a signed zero (used for refinement residuals,
// which are often exactly zero once x has converged; one below 2^-126 is far under
// what an FP32 correction resolves).  Magnitudes from 2^128 up, infinities and
// NaNs take the rounding conversion (an infinity or a NaN), out of line, so that
// its FP64 instruction is issued only where it is needed.
#if defined(__CUDACC__)
static __host__ __device__ __noinline__
#else
static inline
#endif
float f64_to_f32_slow(double v) {
  return (float)v;
}

SB_HD float f64_to_f32_trunc(double v) {
  const uint32_t hi = d_hi(v), lo = d_lo(v);
  const uint32_t E = (hi >> 20) & 0x7FFu;
  if (SB_LIKELY(E - 897u < 254u))  // E in [897, 1150]: exponent in [-126, 127]
    return u2f((funnel_l(lo, hi, 3) - (896u << 23)) | (hi & 0x80000000u));
  if (E < 897u) return u2f(hi & 0x80000000u);
  return f64_to_f32_slow(v);
}

}  // namespace sb
