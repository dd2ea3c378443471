// Pairs of FP32 numbers ("double-float"): x = hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits, evaluated on the FP32 pipes.  On GB300 the FP64
// pipe runs at about 1/62 of the FP32 rate; the QMC_FP32X2 form computes the atomic
// orbitals and the AO->MO contraction in this arithmetic so that the MO
// channels reach near-FP64 accuracy at FP32-pipe cost.
//
// The building blocks are the classical error-free transformations:
//   two_sum(a, b)      = (s, e), s = fl(a + b), s + e = a + b exactly   (Knuth)
//   fast_two_sum(a, b) = the same for |a| >= |b|                        (Dekker)
//   two_prod(a, b)     = (p, e), p = fl(a b), p + e = a b exactly (one FMA)
// and from them addition, multiplication, division, square root and the
// exponential.  exp uses table-driven argument reduction in the manner of
// Tang (ACM TOMS 15, 1989): x = (64 m + j) ln2/64 + r with |r| <= ln2/128,
// exp(x) = 2^m 2^(j/64) exp(r), the 64 values 2^(j/64) held as pairs (built
// on the host), exp(r) from its Taylor polynomial to r^5 (truncation below
// 2^-54 relative).
//
// Everything here is __host__ __device__ so that host tests can compile it
// (without FMA contraction) and compare it with long-double references.
// On the device the primitives use the _rn intrinsics, which the compiler
// never contracts into FMAs (an error-free transformation needs its products
// and sums rounded exactly as written).
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define QMC_HD __host__ __device__ __forceinline__
#else
#define QMC_HD inline
#endif

namespace qmc {

#if defined(__CUDA_ARCH__)
QMC_HD float x2_add_rn(float a, float b) { return __fadd_rn(a, b); }
QMC_HD float x2_sub_rn(float a, float b) { return __fsub_rn(a, b); }
QMC_HD float x2_mul_rn(float a, float b) { return __fmul_rn(a, b); }
QMC_HD float x2_fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
QMC_HD float x2_sqrt_rn(float a) { return __fsqrt_rn(a); }
QMC_HD float x2_rcp(float a) { return __frcp_rn(a); }
QMC_HD float x2_rsqrt(float a) { return rsqrtf(a); }
// round to the nearest integer (ties to even) by adding and subtracting
// 1.5 x 2^23, for |a| < 2^22 (every use here: digits below 2^9, exponential
// arguments below 2^13): two FP32 adds on the FMA pipe
QMC_HD float x2_rint(float a) { return __fsub_rn(__fadd_rn(a, 12582912.0f), 12582912.0f); }
QMC_HD float x2_bits_f(uint32_t u) { return __uint_as_float(u); }
#else
QMC_HD float x2_add_rn(float a, float b) { return a + b; }
QMC_HD float x2_sub_rn(float a, float b) { return a - b; }
QMC_HD float x2_mul_rn(float a, float b) { return a * b; }
QMC_HD float x2_fma_rn(float a, float b, float c) { return std::fma(a, b, c); }
QMC_HD float x2_sqrt_rn(float a) { return std::sqrt(a); }
QMC_HD float x2_rcp(float a) { return 1.0f / a; }
QMC_HD float x2_rsqrt(float a) { return 1.0f / std::sqrt(a); }
QMC_HD float x2_rint(float a) { return std::nearbyint(a); }
QMC_HD float x2_bits_f(uint32_t u) {
  union {
    uint32_t u;
    float f;
  } c;
  c.u = u;
  return c.f;
}
#endif

struct f32x2 {
  float hi, lo;
  f32x2() = default;
  QMC_HD constexpr f32x2(float h, float l) : hi(h), lo(l) {}
  QMC_HD constexpr f32x2(float h) : hi(h), lo(0.0f) {}
  QMC_HD constexpr f32x2(int k) : hi((float)k), lo(0.0f) {}  // |k| < 2^24: exact
};

QMC_HD f32x2 two_sum(float a, float b) {
  const float s = x2_add_rn(a, b);
  const float bb = x2_sub_rn(s, a);
  const float e = x2_add_rn(x2_sub_rn(a, x2_sub_rn(s, bb)), x2_sub_rn(b, bb));
  return f32x2(s, e);
}
QMC_HD f32x2 fast_two_sum(float a, float b) {
  const float s = x2_add_rn(a, b);
  return f32x2(s, x2_sub_rn(b, x2_sub_rn(s, a)));
}
QMC_HD f32x2 two_prod(float a, float b) {
  const float p = x2_mul_rn(a, b);
  return f32x2(p, x2_fma_rn(a, b, -p));
}

QMC_HD f32x2 operator-(f32x2 a) { return f32x2(-a.hi, -a.lo); }

// sum with relative error about 2^-47 of max(|a|, |b|)
QMC_HD f32x2 operator+(f32x2 a, f32x2 b) {
  const f32x2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, x2_add_rn(s.lo, x2_add_rn(a.lo, b.lo)));
}
QMC_HD f32x2 operator-(f32x2 a, f32x2 b) { return a + (-b); }

QMC_HD f32x2 operator*(f32x2 a, f32x2 b) {
  const f32x2 p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, x2_fma_rn(a.hi, b.lo, x2_fma_rn(a.lo, b.hi, p.lo)));
}
QMC_HD f32x2 operator*(f32x2 a, float b) {
  const f32x2 p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, x2_fma_rn(a.lo, b, p.lo));
}
QMC_HD f32x2 operator*(float a, f32x2 b) { return b * a; }

// reciprocal: one Newton step y + y (1 - b y) from the FP32 reciprocal
QMC_HD f32x2 recip_x2(f32x2 b) {
  const float y = x2_rcp(b.hi);
  // 1 - b y with b y as an exact pair: the residual is formed to 2^-48
  const f32x2 p = two_prod(b.hi, y);
  const float res = x2_sub_rn(x2_sub_rn(1.0f, p.hi), x2_fma_rn(b.lo, y, p.lo));
  return fast_two_sum(y, x2_mul_rn(y, res));
}
QMC_HD f32x2 operator/(f32x2 a, f32x2 b) { return a * recip_x2(b); }

QMC_HD f32x2& operator+=(f32x2& a, f32x2 b) { return a = a + b; }
QMC_HD f32x2& operator-=(f32x2& a, f32x2 b) { return a = a - b; }
QMC_HD f32x2& operator*=(f32x2& a, f32x2 b) { return a = a * b; }

// sqrt: s = sqrt(hi) correctly rounded, then s + (a - s^2) / (2 s)
QMC_HD f32x2 sqrt_x2(f32x2 a) {
  if (!(a.hi > 0.0f)) return f32x2(x2_sqrt_rn(a.hi), 0.0f);
  const float s = x2_sqrt_rn(a.hi);
  const f32x2 p = two_prod(s, s);
  const float d = x2_add_rn(x2_sub_rn(x2_sub_rn(a.hi, p.hi), p.lo), a.lo);
  return fast_two_sum(s, x2_mul_rn(d, x2_mul_rn(0.5f, x2_rcp(s))));
}

// 1 / sqrt(a): one Newton step y + y (1 - a y^2) / 2 from the FP32 estimate
QMC_HD f32x2 rsqrt_x2(f32x2 a) {
  const float y = x2_rsqrt(a.hi);
  const f32x2 y2 = two_prod(y, y);
  const f32x2 ay2 = a * y2;
  const float res = x2_sub_rn(x2_sub_rn(1.0f, ay2.hi), ay2.lo);
  return fast_two_sum(y, x2_mul_rn(x2_mul_rn(0.5f, y), res));
}

// ln2/64 as three parts: the first (1420 * 2^-17) has 11 significant bits, so
// that n times it is exact for |n| < 2^13; the three sum to ln2/64 within
// 2^-72 relative.
constexpr float kLn2By64A = 0.010833740234375f;
constexpr float kLn2By64B = -3.3155381515825866e-06f;
constexpr float kLn2By64C = 2.572804640231345e-14f;
constexpr float k64ByLn2 = 92.332482616893656877f;

// exp of a pair for x <= about 0 (the orbital exponentials); tab holds
// 2^(j/64) as pairs (hi, lo) for j = 0..63.  Results below FLT_MIN (x < -87)
// are flushed to 0; x > 80 is outside the contract (never met: the
// arguments are -alpha r^2 and -zeta r).
QMC_HD f32x2 exp_x2(f32x2 x, const float* tab) {
  if (x.hi < -87.0f) return f32x2(0.0f, 0.0f);
  const float nf = x2_rint(x2_mul_rn(x.hi, k64ByLn2));
  const int n = (int)nf;
  // r = x - n ln2/64 as a pair: x.hi - n A is exact (n A has at most 24
  // bits and is within a factor 2 of x.hi, or n = 0)
  const float r0 = x2_sub_rn(x.hi, x2_mul_rn(nf, kLn2By64A));
  // (x.lo, up to 2^-24 |x|, enters through its own two_sum: rounding it with
  // the small terms would cost 2^-24 |x.lo| absolute)
  const f32x2 nb = two_prod(nf, kLn2By64B);
  const f32x2 r1 = two_sum(r0, -nb.hi);
  const f32x2 r2 = two_sum(r1.hi, x.lo);
  const f32x2 r =
      fast_two_sum(r2.hi, x2_add_rn(x2_add_rn(r1.lo, r2.lo), -x2_fma_rn(nf, kLn2By64C, nb.lo)));
  // exp(r) - 1 = r + r^2/2 + r^3 (1/6 + r (1/24 + r/120)), |r| <= 0.0055
  f32x2 q = two_prod(r.hi, r.hi);
  q = f32x2(x2_mul_rn(0.5f, q.hi), x2_mul_rn(0.5f, x2_fma_rn(2.0f * r.hi, r.lo, q.lo)));
  const float r3 = x2_mul_rn(r.hi, x2_mul_rn(r.hi, r.hi));
  const float tail =
      x2_mul_rn(r3, x2_fma_rn(r.hi, x2_fma_rn(r.hi, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f));
  f32x2 em1 = r + q;
  em1 = fast_two_sum(em1.hi, x2_add_rn(em1.lo, tail));
  const f32x2 one_p = fast_two_sum(1.0f, em1.hi);
  const f32x2 er = fast_two_sum(one_p.hi, x2_add_rn(one_p.lo, em1.lo));
  const int j = n & 63, m = n >> 6;  // floor division for negative n too
  const f32x2 t(tab[2 * j], tab[2 * j + 1]);
  f32x2 v = er * t;
  // times 2^m: one normal factor for m in [-126, 127] (x >= -87 keeps m >= -126);
  // two factors outside that range
  if (m >= -126 && m <= 127) {
    const float sc = x2_bits_f((uint32_t)(m + 127) << 23);
    return f32x2(x2_mul_rn(v.hi, sc), x2_mul_rn(v.lo, sc));
  }
  const int m1 = m / 2, m2 = m - m1;
  const float s1 = x2_bits_f((uint32_t)(m1 + 127) << 23), s2 = x2_bits_f((uint32_t)(m2 + 127) << 23);
  v = f32x2(x2_mul_rn(x2_mul_rn(v.hi, s1), s2), x2_mul_rn(x2_mul_rn(v.lo, s1), s2));
  return v;
}

// Multiply-accumulate into an unnormalised pair (acc.hi + acc.lo): the
// product a b is formed exactly up to its 2^-48 cross terms, its high part
// enters acc.hi through two_sum and everything else is gathered in acc.lo.
// Normalise with fast_two_sum(acc.hi, acc.lo) after the last term.
QMC_HD void mac_x2(f32x2& acc, f32x2 a, f32x2 b) {
  const float p = x2_mul_rn(a.hi, b.hi);
  const float pe = x2_fma_rn(a.hi, b.hi, -p);
  const float cross = x2_fma_rn(a.hi, b.lo, x2_fma_rn(a.lo, b.hi, pe));
  const f32x2 s = two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = x2_add_rn(acc.lo, x2_add_rn(s.lo, cross));
}

QMC_HD f32x2 normalize_x2(f32x2 a) { return fast_two_sum(a.hi, a.lo); }

}  // namespace qmc
