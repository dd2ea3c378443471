// Exact AO->MO contraction of pairs of FP32 on BF16 tensor cores: operands
// cut into signed 8-bit digits (an error-free slicing in the manner of the
// Ozaki scheme: Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012;
// Ootomo, Ozaki and Yokota, IJHPCA 2024).
//
// A row of AO values a_b (one walker, one electron, one channel) is scaled by
// a power of two 2^-e with |a_b| 2^-e <= 1 (e from an upper bound of the
// row), an MO column c_bm by 2^-f_m with |c_bm| 2^-f_m <= 1, and each is
// written as six digits
//     a 2^-e = sum_{k=1..6} d_k 2^-8k + r,   |r| <= 2^-49,
// d_k integers with |d_1|, |d_4| <= 256 and the others <= 129: every digit
// is exact in BF16 (8 significant bits).  The product of two digits is exact
// in FP32 and, for at most 110 AO terms, every partial sum of the digit
// products of one weight class g = k + l - 2 (0..5) is an integer below
// 2^24, so a tensor core accumulating D_g = sum_{k+l=g+2} A_k B_l in FP32
// adds exactly.  Classes k + l > 7 are dropped (below 2^-48 of |a||c|), and
//     Phi_m = 2^(e + f_m - 16) sum_{g=0..5} D_g 2^-8g
// is recombined as a pair of FP32 by error-free sums (oz_combine).
//
// Everything here is __host__ __device__: tests/f32x2_check.cpp runs the
// same code on the host against long-double references.
#pragma once

#include "f32x2.cuh"

namespace qmc {

constexpr int kOzDigits = 6;
constexpr int kOzClasses = 6;

// digits d[0..5] of x = (hi, lo), a normalised pair with |x| <= 1:
// three from the high word by exact steps, then the low word folded in with
// one two_sum, then three more; |residual| <= 2^-49
QMC_HD void oz_digits(f32x2 x, float d[kOzDigits]) {
  float h = x2_mul_rn(x.hi, 256.0f);
  d[0] = x2_rint(h);
  h = x2_mul_rn(x2_sub_rn(h, d[0]), 256.0f);
  d[1] = x2_rint(h);
  h = x2_mul_rn(x2_sub_rn(h, d[1]), 256.0f);
  d[2] = x2_rint(h);
  h = x2_mul_rn(x2_sub_rn(h, d[2]), 256.0f);  // units of 2^-32
  const f32x2 s = two_sum(h, x2_mul_rn(x.lo, 4294967296.0f));
  d[3] = x2_rint(s.hi);
  float r = x2_add_rn(x2_mul_rn(x2_sub_rn(s.hi, d[3]), 256.0f), x2_mul_rn(s.lo, 256.0f));
  d[4] = x2_rint(r);
  r = x2_mul_rn(x2_sub_rn(r, d[4]), 256.0f);
  d[5] = x2_rint(r);
}

// sum_{g} acc[g] 2^-8g as a normalised pair (acc[g] exact integers below 2^24)
QMC_HD f32x2 oz_combine(const float acc[kOzClasses]) {
  constexpr float kScale[kOzClasses] = {1.0f, 0.00390625f, 1.52587890625e-05f, 5.9604644775390625e-08f,
                                        2.3283064365386963e-10f, 9.094947017729282e-13f};
  float s = x2_mul_rn(acc[kOzClasses - 1], kScale[kOzClasses - 1]), e = 0.0f;
  for (int g = kOzClasses - 2; g >= 0; --g) {
    const f32x2 t = two_sum(x2_mul_rn(acc[g], kScale[g]), s);
    s = t.hi;
    e = x2_add_rn(e, t.lo);
  }
  return fast_two_sum(s, e);
}

// BF16 bit pattern of a digit (an integer of magnitude <= 256: the FP32
// pattern's upper half is exact)
QMC_HD uint16_t oz_bf16(float d) {
#if defined(__CUDA_ARCH__)
  return (uint16_t)(__float_as_uint(d) >> 16);
#else
  union {
    float f;
    uint32_t u;
  } c;
  c.f = d;
  return (uint16_t)(c.u >> 16);
#endif
}

}  // namespace qmc
