// Arithmetic policies for the batched sweeps.
//
// Every sweep step has the same shape (coefficients prescaled on the host):
//     out = C0 * in - C1 * v1 - C2 * v2          (C2 only for pentadiagonal)
// NativeArith<T> evaluates it in T (FP64 or FP32) with fused multiply-adds.
// DFArith evaluates it in double-float ("df") arithmetic: every value is an
// unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h), giving about 48
// significant bits with the FP32 pipe (GB300 issues 64x more FP32 than FP64
// operations per clock).  The building blocks are the classical error-free
// transformations: TwoSum (Knuth), Fast2Sum (Dekker) and TwoProd with an FMA.
// FP64 <-> df conversions of the inputs and outputs use integer operations only
// (the FP64 conversion instructions run on the slow FP64 pipe); values outside
// the exponent window of the integer path take an exact FP64 fallback.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define SB_HD __host__ __device__ __forceinline__
#define SB_LIKELY(c) __builtin_expect(!!(c), 1)
#else
#define SB_HD inline
#define SB_LIKELY(c) (c)
#endif

namespace sb {

// ------------------------------------------------- portable primitives
// On the device these are the round-to-nearest intrinsics (never contracted into
// FMAs); the host versions exist so the same code can be unit-tested on a CPU
// (compile host code with -ffp-contract=off).
SB_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
SB_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
SB_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
SB_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
SB_HD uint32_t f2u(float v) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(v);
#else
  uint32_t u;
  std::memcpy(&u, &v, 4);
  return u;
#endif
}
SB_HD float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float v;
  std::memcpy(&v, &u, 4);
  return v;
#endif
}
SB_HD uint32_t d_hi(double v) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__double2hiint(v);
#else
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return (uint32_t)(u >> 32);
#endif
}
SB_HD uint32_t d_lo(double v) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__double2loint(v);
#else
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return (uint32_t)u;
#endif
}
SB_HD double hilo2d(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double v;
  std::memcpy(&v, &u, 8);
  return v;
#endif
}
// upper 32 bits of (hi:lo) << s, 0 <= s < 32
SB_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, uint32_t s) {
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lo, hi, s);
#else
  return (uint32_t)(((((uint64_t)hi << 32) | lo) << s) >> 32);
#endif
}
// (hi:lo) + (bhi:blo) modulo 2^64
SB_HD void add64(uint32_t lo, uint32_t hi, uint32_t blo, uint32_t bhi, uint32_t* rlo,
                 uint32_t* rhi) {
#ifdef __CUDA_ARCH__
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;"
      : "=r"(*rlo), "=r"(*rhi)
      : "r"(lo), "r"(blo), "r"(hi), "r"(bhi));
#else
  const uint64_t r = (((uint64_t)hi << 32) | lo) + (((uint64_t)bhi << 32) | blo);
  *rlo = (uint32_t)r;
  *rhi = (uint32_t)(r >> 32);
#endif
}

// ------------------------------------------- FP64 multiply on the integer pipe

SB_HD uint64_t d_bits(double v) { return ((uint64_t)d_hi(v) << 32) | d_lo(v); }
SB_HD double bits_d(uint64_t u) { return hilo2d((uint32_t)(u >> 32), (uint32_t)u); }
SB_HD uint64_t umul64hi(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Plain FP64 product, kept out of line so that the fallback below is a real
// branch (an if-converted DMUL would be issued for every element).
#if defined(__CUDACC__)
static __host__ __device__ __noinline__
#else
static inline
#endif
double dmul_slow(double a, double b) {
  return a * b;
}

// a * b in IEEE binary64 with round-to-nearest-even, computed with integer
// instructions only: the 53 x 53-bit significand product, normalisation, and
// rounding on the guard bit and the sticky bits.  The result is bit-identical to
// the FP64 multiply instruction; zero, subnormal, infinite or NaN operands and
// products outside the normal range take that instruction instead.  On GB300 the
// integer pipes issue 64x more operations per clock than the FP64 pipe, so this
// moves one multiply per element off the pipe that bounds the FP64 sweeps.
SB_HD double dmul_int(double a, double b) {
  const uint32_t ah = d_hi(a), al = d_lo(a), bh = d_hi(b), bl = d_lo(b);
  const uint32_t ea = (ah >> 20) & 0x7FFu, eb = (bh >> 20) & 0x7FFu;
  const int e = (int)(ea + eb) - 1023;  // product exponent if the significand product were < 2
  if (SB_LIKELY(ea - 1u < 2046u && eb - 1u < 2046u && (unsigned)(e - 1) < 2044u)) {
    // significands A = Ah 2^32 + al, B = Bh 2^32 + bl with the implicit bit in Ah, Bh;
    // P = A B = H 2^64 + mlo 2^32 + l0 from four 32 x 32 -> 64-bit multiply-adds
    const uint32_t Ah = (ah & 0xFFFFFu) | 0x100000u, Bh = (bh & 0xFFFFFu) | 0x100000u;
    const uint64_t ll = (uint64_t)al * bl;
    const uint64_t t = (uint64_t)al * Bh + (ll >> 32);
    const uint64_t mid = (uint64_t)Ah * bl + t;
    const uint64_t H = (uint64_t)Ah * Bh + (mid >> 32);  // bits 64 .. 105 of P
    const uint32_t mlo = (uint32_t)mid, l0 = (uint32_t)ll;
    const uint32_t top = (uint32_t)(H >> 41) & 1u;  // P >= 2^105
    // 53-bit significand P >> (52 + top), its guard bit and the sticky bits below
    const uint32_t sh = 12u - top;
    const uint64_t m0 = (H << sh) | (uint64_t)(mlo >> (32u - sh));
    const uint32_t gpos = 19u + top;
    const uint32_t guard = (mlo >> gpos) & 1u;
    const uint32_t sticky = ((mlo & ((1u << gpos) - 1u)) | l0) != 0u;
    uint64_t m = m0 + (uint64_t)(guard & (sticky | (uint32_t)(m0 & 1u)));
    const uint32_t carry = (uint32_t)(m >> 53);  // rounding reached the next binade
    m >>= carry;
    const int ex = e + (int)top + (int)carry;
    if ((unsigned)(ex - 1) < 2046u) {
      const uint32_t hi = ((ah ^ bh) & 0x80000000u) | ((uint32_t)ex << 20) |
                          ((uint32_t)(m >> 32) & 0xFFFFFu);
      return hilo2d(hi, (uint32_t)m);
    }
  }
  return dmul_slow(a, b);
}

// ------------------------------------------------------------- native T

template <typename T>
struct NativeArith {
  using V = T;  // working value
  using C = T;  // coefficient
  using S = T;  // stored intermediate
  static SB_HD V zero() { return T(0); }
  // in * c0: for FP64 on the integer pipe (bit-identical, see dmul_int) since this
  // product is off the recurrence's dependent chain
  static SB_HD V scale(C c, V v) {
    if constexpr (sizeof(T) == 8)
      return dmul_int(v, c);
    else
      return v * c;
  }
  // out = c0*in - c1*v1 (- c2*v2); C0ONE skips the c0 product.
  template <int P, bool C0ONE>
  static SB_HD V step(const C* c, V in, V v1, V v2) {
    V u = C0ONE ? in : scale(c[0], in);
    u = std::fma(-c[1], v1, u);
    if constexpr (P == 2) u = std::fma(-c[2], v2, u);
    return u;
  }
  static SB_HD S to_store(V v) { return v; }
  static SB_HD V from_store(S s) { return s; }
  // value operations used to build right-hand sides
  static SB_HD V add(V a, V b) { return a + b; }
  static SB_HD V mulc(C c, V v) { return c * v; }
  static SB_HD V fmac(C c, V v, V acc) { return std::fma(c, v, acc); }  // acc + c*v
  static SB_HD V cubic(V c) { return std::fma(c * c, c, -c); }        // c^3 - c
};

// ---------------------------------------------------------- double-float

struct alignas(8) df {
  float h, l;
};

// Knuth's TwoSum: s + e == a + b exactly.
SB_HD df two_sum(float a, float b) {
  const float s = f_add(a, b);
  const float bb = f_sub(s, a);
  const float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
  return {s, e};
}

// Dekker's Fast2Sum, valid when |a| >= |b| (or a == 0).
SB_HD df fast_two_sum(float a, float b) {
  const float s = f_add(a, b);
  const float e = f_sub(b, f_sub(s, a));
  return {s, e};
}

// Product of a df coefficient and a df value as an unnormalised pair (p, e):
// p = fl(ch*vh) and e = its exact rounding error + ch*vl + cl*vh (the cl*vl
// term is below 2^-48 relative and dropped).
SB_HD df df_mul(df c, df v) {
  const float p = f_mul(c.h, v.h);
  float e = f_fma(c.h, v.h, -p);
  e = f_fma(c.h, v.l, e);
  e = f_fma(c.l, v.h, e);
  return {p, e};
}

// FP64 -> df.  Integer path for 2^-60 <= |v| < 2^100: the high part keeps the
// sign, exponent and top 23 fraction bits (truncated), the low part the next 23
// bits, made exact by the subtraction of a power of two (Sterbenz).  The 6
// lowest fraction bits are dropped (relative error < 2^-47).
// Exact slow paths of the conversions, kept out of line: if they were inlined the
// compiler may if-convert them and issue their FP64 instructions (on GB300's slow
// FP64 pipe) for every element, not only for the rare values that need them.
#if defined(__CUDACC__)
static __host__ __device__ __noinline__
#else
static inline
#endif
df double_to_df_slow(double v) {
  const float h = (float)v;  // round to nearest, then the rest
  return {h, (float)(v - (double)h)};
}


SB_HD df double_to_df(double v) {
  const uint32_t hi = d_hi(v), lo = d_lo(v);
  const uint32_t E = (hi >> 20) & 0x7FFu;
  if (SB_LIKELY(E - 963u < 160u)) {  // E in [963, 1122]: exponent in [-60, 99]
    const uint32_t t = funnel_l(lo, hi, 3);                // E[8:0] | top 23 bits
    const uint32_t hb = (t - (896u << 23)) | (hi & 0x80000000u);
    const uint32_t bb = (hb & 0xFF800000u) - (23u << 23);  // 2^(e-23) with the sign
    const uint32_t fb = bb | ((lo >> 6) & 0x7FFFFFu);
    return {u2f(hb), f_sub(u2f(fb), u2f(bb))};
  }
  return double_to_df_slow(v);  // exact fallback (rare)
}

// FP32 -> FP64 widening with integer operations only (exact): sign, exponent
// re-biased by 1023 - 127 = 896, fraction shifted into the upper bits.  Zero and
// FP32 subnormals give (signed) zero; infinities stay infinite and NaNs NaN.
SB_HD double widen_f32(float v) {
  const uint32_t b = f2u(v);
  const uint32_t mag = b & 0x7FFFFFFFu;
  uint32_t hi = (mag >= 0x00800000u) ? ((mag >> 3) + (896u << 20)) : 0u;
  uint32_t lo = (mag >= 0x00800000u) ? (b << 29) : 0u;
  if (mag >= 0x7F800000u) {  // infinity or NaN
    hi = (mag == 0x7F800000u) ? 0x7FF00000u : 0x7FF80000u;
    lo = 0u;
  }
  return hilo2d(hi | (b & 0x80000000u), lo);
}

// df -> FP64: h + l rounded to the nearest double.  Both parts are widened exactly
// with integer operations and added with a single FP64 addition (one FP64-pipe
// instruction per value instead of two conversions and an addition).
SB_HD double df_to_double(df x) { return widen_f32(x.h) + widen_f32(x.l); }

struct DFArith {
  using V = df;
  using C = df;  // (hi, lo) of a coefficient
  using S = df;  // stored intermediate (8 bytes, same as FP64)
  static SB_HD V zero() { return {0.f, 0.f}; }
  static SB_HD V scale(C c, V v) { return mulc(c, v); }
  template <int P, bool C0ONE>
  static SB_HD V step(const C* c, V in, V v1, V v2) {
    df t0 = C0ONE ? in : df_mul(c[0], in);
    const df t1 = df_mul(c[1], v1);
    const df s1 = two_sum(t0.h, -t1.h);
    float lo = f_sub(t0.l, t1.l);
    float hi = s1.h;
    lo = f_add(lo, s1.l);
    if constexpr (P == 2) {
      const df t2 = df_mul(c[2], v2);
      const df s2 = two_sum(hi, -t2.h);
      lo = f_sub(lo, t2.l);
      lo = f_add(lo, s2.l);
      hi = s2.h;
    }
    return fast_two_sum(hi, lo);
  }
  static SB_HD S to_store(V v) { return v; }
  static SB_HD V from_store(S s) { return s; }
  // value operations used to build right-hand sides (all results normalised)
  static SB_HD V add(V a, V b) {
    const df s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, f_add(s.l, f_add(a.l, b.l)));
  }
  static SB_HD V mulc(C c, V v) {
    const df p = df_mul(c, v);
    return fast_two_sum(p.h, p.l);
  }
  static SB_HD V fmac(C c, V v, V acc) {  // acc + c*v
    const df p = df_mul(c, v);
    const df s = two_sum(acc.h, p.h);
    return fast_two_sum(s.h, f_add(s.l, f_add(acc.l, p.l)));
  }
  static SB_HD V cubic(V c) {  // c^3 - c = c * (c*c - 1)
    const df sq = mulc(c, c);
    const df s = two_sum(sq.h, -1.0f);
    const df q = fast_two_sum(s.h, f_add(s.l, sq.l));
    return mulc(q, c);
  }
};

}  // namespace sb
