// dog_math.cuh -- device arithmetic shared by the filter kernels.
//
// Every floating-point operation on the filter's path is an explicit IEEE binary32
// round-to-nearest intrinsic (__fadd_rn, __fmul_rn, ...; the code is compiled without
// contraction), so the sequence of roundings is fixed.  The transcendentals the filter
// needs (ln and sin/cos of 2 pi u for Box-Muller, exp for the radar likelihood) are this
// file's own series evaluations, not CUDA's math library; their Horner steps are explicit
// fused multiply-adds (__fmaf_rn, one rounding each, as C's fmaf).
#pragma once
#include <cstdint>

namespace dog {

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplications with
// the Weyl-sequence key schedule.  Counter = (element, frame, purpose tag, 0).
// ------------------------------------------------------------------------------------
struct U4 {
  uint32_t a, b, c, d;
};

__device__ __forceinline__ U4 philox(uint32_t e, uint32_t frame, uint32_t tag, uint32_t k0,
                                     uint32_t k1) {
  uint32_t x0 = e, x1 = frame, x2 = tag, x3 = 0u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
    const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
    const uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{x0, x1, x2, x3};
}

// The same generator with its key schedule (the ten round keys, which depend on the seed
// only) computed once: kernels that draw for several elements keep them in registers.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};
__device__ __forceinline__ PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys K;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
    K.k1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  return K;
}
__device__ __forceinline__ U4 philox(uint32_t e, uint32_t frame, uint32_t tag, const PhiloxKeys &K) {
  uint32_t x0 = e, x1 = frame, x2 = tag, x3 = 0u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
    const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
    const uint32_t y0 = hi1 ^ x1 ^ K.k0[r], y2 = hi0 ^ x3 ^ K.k1[r];
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
  }
  return U4{x0, x1, x2, x3};
}

enum : uint32_t { TAG_INIT = 0, TAG_PREDICT = 1, TAG_BIRTH = 2, TAG_RESAMPLE = 3 };

// uniform draws from the top 24 bits: [0,1) and (0,1]
__device__ __forceinline__ float u01_co(uint32_t r) { return __fmul_rn((float)(r >> 8), 0x1p-24f); }
__device__ __forceinline__ float u01_oc(uint32_t r) { return __fmul_rn((float)((r >> 8) + 1u), 0x1p-24f); }

// ln(u) for a positive normal u: fold the mantissa into [sqrt(1/2), sqrt(2)], then
// ln m = 2 atanh((m-1)/(m+1)) by its odd series to the 11th power (Horner in s^2), and
// add e*ln2 with ln2 split in a short high part (exact products) and a correction.
__device__ __forceinline__ float ln_f(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)((bits >> 23) & 0xffu) - 127;
  float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float f = __fsub_rn(m, 1.0f);
  const float s = __fdiv_rn(f, __fadd_rn(2.0f, f));
  const float z = __fmul_rn(s, s);
  float p = 0x1.745d18p-4f;
  p = __fmaf_rn(p, z, 0x1.c71c72p-4f);
  p = __fmaf_rn(p, z, 0x1.24924ap-3f);
  p = __fmaf_rn(p, z, 0x1.99999ap-3f);
  p = __fmaf_rn(p, z, 0x1.555556p-2f);
  p = __fmaf_rn(p, z, 1.0f);
  const float lnm = __fmul_rn(__fadd_rn(s, s), p);
  const float ef = (float)e;
  const float lo = __fmaf_rn(ef, 0x1.7f7d1cp-20f, lnm);
  return __fmaf_rn(ef, 0x1.62e4p-1f, lo);  // e ln2_hi is exact: one rounding either way
}

// sin and cos of 2*pi*u, u = k 2^-24 in [0,1): octant by the exact value 8u, reduced angle
// in [0, pi/4] (odd octants mirrored to 1 - t), Taylor series of sin (to theta^9) and
// cos (to theta^10), then the octant's symmetry.
__device__ __forceinline__ void sincos2pi_f(float u, float &sn, float &cs) {
  const float v = __fmul_rn(u, 8.0f);
  const int k = (int)v;
  const float t = __fsub_rn(v, (float)k);
  const float tt = (k & 1) ? __fsub_rn(1.0f, t) : t;
  const float th = __fmul_rn(tt, 0x1.921fb6p-1f);
  const float z = __fmul_rn(th, th);
  float ps = 0x1.71de3ap-19f;
  ps = __fmaf_rn(ps, z, -0x1.a01a02p-13f);
  ps = __fmaf_rn(ps, z, 0x1.111112p-7f);
  ps = __fmaf_rn(ps, z, -0x1.555556p-3f);
  ps = __fmaf_rn(ps, z, 1.0f);
  const float S = __fmul_rn(th, ps);
  float pc = -0x1.27e4fcp-22f;
  pc = __fmaf_rn(pc, z, 0x1.a01a02p-16f);
  pc = __fmaf_rn(pc, z, -0x1.6c16c2p-10f);
  pc = __fmaf_rn(pc, z, 0x1.555556p-5f);
  pc = __fmaf_rn(pc, z, -0.5f);
  pc = __fmaf_rn(pc, z, 1.0f);
  const float Cc = pc;
  // octant k: (sin, cos) = k0 (S, C)  k1 (C, S)  k2 (C,-S)  k3 (S,-C)
  //                        k4 (-S,-C) k5 (-C,-S) k6 (-C, S) k7 (-S, C)
  const bool swap = ((k + 1) & 2) != 0;  // k = 1, 2, 5, 6
  const float a = swap ? Cc : S;
  const float b = swap ? S : Cc;
  sn = (k >= 4) ? -a : a;
  cs = (k >= 2 && k <= 5) ? -b : b;
}

// e^x for x <= 0: x = k ln2 + r, k = floor(x/ln2 + 1/2), r by a two-part ln2, Taylor
// series of e^r to r^7, scaled by 2^k through the exponent field; 0 below -87.
__device__ __forceinline__ float exp_f(float x) {
  if (!(x > -87.0f)) return 0.0f;
  const float kf = floorf(__fmaf_rn(x, 0x1.715476p+0f, 0.5f));
  const int k = (int)kf;
  // k ln2_hi is exact, so x - k ln2_hi rounds once either way
  const float r = __fmaf_rn(-kf, 0x1.7f7d1cp-20f, __fmaf_rn(-kf, 0x1.62e4p-1f, x));
  float p = 0x1.a01a02p-13f;
  p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
  p = __fmaf_rn(p, r, 0x1.111112p-7f);
  p = __fmaf_rn(p, r, 0x1.555556p-5f);
  p = __fmaf_rn(p, r, 0x1.555556p-3f);
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  return __fmul_rn(p, __uint_as_float((uint32_t)(k + 127) << 23));
}

// Box-Muller pair from two 32-bit draws
__device__ __forceinline__ void gauss2(uint32_t ra, uint32_t rb, float &n0, float &n1) {
  const float rad = __fsqrt_rn(__fmul_rn(-2.0f, ln_f(u01_oc(ra))));
  float sn, cs;
  sincos2pi_f(u01_co(rb), sn, cs);
  n0 = __fmul_rn(rad, cs);
  n1 = __fmul_rn(rad, sn);
}

// ------------------------------------------------------------------------------------
// Fixed point.  Weights: unsigned 64-bit, scale 2^40, truncation; back to float by
// round-to-nearest.  Moment terms (products of a cell-normalised weight with velocities):
// two's-complement 64-bit, scale 2^40, truncation toward 0, saturated at +-2^62.
// ------------------------------------------------------------------------------------
// |t| * 2^40 truncated toward zero, from the float's bits with integer shifts only (the
// hardware float -> 64-bit integer conversion runs on the FP64 pipe, 1/64 of the FP32 rate
// on this GPU); saturates at 2^62.  Equal to the truncating conversion of t * 2^40.
__device__ __forceinline__ unsigned long long fx40_mag(uint32_t bits) {
  const int ex = (int)((bits >> 23) & 0xffu);
  if (ex == 0) return 0ull;  // zero or subnormal: |t| 2^40 < 1
  const unsigned long long m = (unsigned long long)((bits & 0x7fffffu) | 0x800000u);
  const int sh = ex - 110;   // |t| 2^40 = m 2^(ex - 150 + 40)
  if (sh >= 39) return 1ull << 62;
  if (sh >= 0) return m << sh;
  if (sh <= -24) return 0ull;
  return m >> (-sh);
}
__device__ __forceinline__ unsigned long long q40(float w) {
  return (w > 0.0f) ? fx40_mag(__float_as_uint(w)) : 0ull;
}
// u64 -> float, round to nearest even, with integer operations only (equal to the hardware
// conversion, which runs on the FP64 pipe)
__device__ __forceinline__ float u64_to_f32_rn(unsigned long long x) {
  if (x < (1ull << 24)) return (float)(uint32_t)x;  // exact
  const int shift = 40 - __clzll(x);                  // bits beyond the 24 kept, >= 1
  unsigned long long m = x >> shift;                  // 24 bits, leading bit at 23
  const unsigned long long rem = x & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
  int e = shift;
  if (rem > half || (rem == half && (m & 1ull))) {
    ++m;
    if (m == (1ull << 24)) {
      m >>= 1;
      ++e;
    }
  }
  return __uint_as_float(((uint32_t)(e + 150) << 23) | ((uint32_t)m & 0x7fffffu));
}
__device__ __forceinline__ float fx40_to_f(unsigned long long s) {
  return __fmul_rn(u64_to_f32_rn(s), 0x1p-40f);
}
__device__ __forceinline__ unsigned long long q40s(float t) {
  const uint32_t b = __float_as_uint(t);
  const unsigned long long mag = fx40_mag(b);
  return (b >> 31) ? 0ull - mag : mag;
}
// signed fixed point (two's complement, scale 2^40) -> float with 32-bit operations: the
// two halves are converted separately (at most one extra rounding)
__device__ __forceinline__ float fx40s_to_f(unsigned long long s) {
  const int hi = (int)(uint32_t)(s >> 32);
  const uint32_t lo = (uint32_t)s;
  return __fmul_rn(__fadd_rn(__fmul_rn((float)hi, 0x1p32f), (float)lo), 0x1p-40f);
}

// ------------------------------------------------------------------------------------
// Compensated (double-float) arithmetic for the per-cell velocity moments: a value is an
// unevaluated sum hi + lo of two binary32 numbers.  two_sum (Knuth) and two_prod (with one
// fused multiply-add) return the exact rounding error of a sum / product, so sums of
// double-float terms carry about 48 significant bits whatever their number and order.
// ------------------------------------------------------------------------------------
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, e};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return DF{p, __fmaf_rn(a, b, -p)};
}
// a + b; the low parts are added without compensation (their error is second order)
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return DF{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ DF df_norm(DF a) {  // hi = RN(hi + lo)
  const float s = __fadd_rn(a.hi, a.lo);
  return DF{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const DF p = two_prod(a.hi, b);
  return df_norm(DF{p.hi, __fmaf_rn(a.lo, b, p.lo)});
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const DF p = two_prod(a.hi, b.hi);
  const float c = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
  return df_norm(DF{p.hi, __fadd_rn(p.lo, c)});
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
// a / b for b > 0: quotient, exact remainder by one fused multiply-add, one correction
__device__ __forceinline__ DF df_div_f(DF a, float b) {
  const float q1 = __fdiv_rn(a.hi, b);
  const float r = __fadd_rn(__fmaf_rn(-q1, b, a.hi), a.lo);
  return df_norm(DF{q1, __fdiv_rn(r, b)});
}
__device__ __forceinline__ float df_to_f(DF a) { return __fadd_rn(a.hi, a.lo); }

// signed 2^-40 fixed point -> double-float: the binary32 value and the exact integer
// remainder below it
__device__ __forceinline__ DF fx40s_to_df(unsigned long long s) {
  const float hi = fx40s_to_f(s);
  return DF{hi, fx40s_to_f(s - q40s(hi))};
}

// ------------------------------------------------------------------------------------
// 128-bit helpers for the exact integer allocation rules
// ------------------------------------------------------------------------------------
struct U128 {
  unsigned long long hi, lo;
};
__device__ __forceinline__ U128 mul_64x64(unsigned long long a, unsigned long long b) {
  return U128{__umul64hi(a, b), a * b};
}
__device__ __forceinline__ U128 add_128_64(U128 a, unsigned long long b) {
  const unsigned long long lo = a.lo + b;
  return U128{a.hi + (lo < b ? 1ull : 0ull), lo};
}
__device__ __forceinline__ bool lt_128(U128 a, U128 b) {
  return (a.hi < b.hi) || (a.hi == b.hi && a.lo < b.lo);
}
// floor(a * b / d) for b <= d (so the result lies in [0, a]), exactly: a float estimate
// brackets the quotient (+-16; the bracket is checked and widened to [0, a] if it fails),
// then bisection with exact 128-bit comparisons
__device__ __forceinline__ uint32_t floor_muldiv(uint32_t a, unsigned long long b, unsigned long long d) {
  const U128 ab = mul_64x64(a, b);
  const float est = __fmul_rn((float)a, __fdiv_rn(u64_to_f32_rn(b), u64_to_f32_rn(d)));
  const uint32_t q = est >= (float)a ? a : (uint32_t)est;
  uint32_t lo = q > 16u ? q - 16u : 0u;
  uint32_t hi = (a - q) > 16u ? q + 16u : a;
  if (lt_128(ab, mul_64x64(lo, d)) || (hi < a && !lt_128(ab, mul_64x64((unsigned long long)hi + 1, d)))) {
    lo = 0;
    hi = a;
  }
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1) / 2;
    if (lt_128(ab, mul_64x64(mid, d))) hi = mid - 1; else lo = mid;
  }
  return lo;
}

}  // namespace dog
