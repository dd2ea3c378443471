// Host check of the pair-of-FP32 arithmetic (paper_2506_09743_gb300/csrc/f32x2.cuh)
// against long-double references.  Prints one "name max_rel_err" line per
// operation; the Python test reads them.  Built with -ffp-contract=off so
// that the error-free transformations are evaluated as written.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <random>

#include "../paper_2506_09743_gb300/csrc/f32x2.cuh"
#include "../paper_2506_09743_gb300/csrc/oz_digits.cuh"

using qmc::f32x2;

static long double val(f32x2 a) { return (long double)a.hi + (long double)a.lo; }
static f32x2 from_ld(long double x) {
  const float h = (float)x;
  return f32x2(h, (float)(x - (long double)h));
}
static double rel(long double got, long double ref) {
  const long double d = fabsl(got - ref), s = fabsl(ref);
  return (double)(s > 0 ? d / s : d);
}

int main() {
  float tab[128];
  for (int j = 0; j < 64; ++j) {
    const long double v = exp2l((long double)j / 64.0L);
    tab[2 * j] = (float)v;
    tab[2 * j + 1] = (float)(v - (long double)tab[2 * j]);
  }
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> u01(0.0, 1.0);
  double e_exp = 0, e_exp_tiny = 0, e_mul = 0, e_add = 0, e_div = 0, e_sqrt = 0, e_rsqrt = 0, e_dot = 0, e_norm = 0;
  int bad_norm = 0;
  for (int t = 0; t < 200000; ++t) {
    // exponential over the orbital range, arguments given as pairs
    const long double x = -87.0L * powl(u01(rng), 3.0L) + (t % 97 == 0 ? 0.9L * u01(rng) : 0.0L);
    const f32x2 xa = from_ld(x);
    const f32x2 ex = qmc::exp_x2(xa, tab);
    // full pair precision while the low part stays a normal float (results
    // above 2^-100); below that the low part loses bits and the error is
    // bounded by 2^-149 absolute
    const double ee = rel(val(ex), expl(val(xa)));
    if (val(ex) > 0x1p-100L) e_exp = std::fmax(e_exp, ee);
    else e_exp_tiny = std::fmax(e_exp_tiny, (double)fabsl(val(ex) - expl(val(xa))));
    if (fabsf(ex.lo) > 0.5f * ldexpf(1.0f, ilogbf(ex.hi) - 23) * 1.0001f && ex.hi != 0.0f) ++bad_norm;
    // arithmetic on random pairs of mixed magnitude
    const long double a = (u01(rng) - 0.5) * powl(10.0L, 6.0L * u01(rng) - 3.0L);
    const long double b = (u01(rng) - 0.5) * powl(10.0L, 6.0L * u01(rng) - 3.0L);
    const f32x2 pa = from_ld(a), pb = from_ld(b);
    e_mul = std::fmax(e_mul, rel(val(pa * pb), val(pa) * val(pb)));
    // addition: error relative to the larger operand (cancellation allowed)
    {
      const long double ref = val(pa) + val(pb), scale = fmaxl(fabsl(val(pa)), fabsl(val(pb)));
      e_add = std::fmax(e_add, (double)(fabsl(val(pa + pb) - ref) / scale));
    }
    e_div = std::fmax(e_div, rel(val(pa / pb), val(pa) / val(pb)));
    const f32x2 ap(fabsf(pa.hi), pa.hi < 0 ? -pa.lo : pa.lo);
    e_sqrt = std::fmax(e_sqrt, rel(val(qmc::sqrt_x2(ap)), sqrtl(val(ap))));
    e_rsqrt = std::fmax(e_rsqrt, rel(val(qmc::rsqrt_x2(ap)), 1.0L / sqrtl(val(ap))));
  }
  // 64-term dot products with cancellation, error relative to sum |a_k b_k|
  for (int t = 0; t < 20000; ++t) {
    f32x2 acc(0.0f, 0.0f);
    long double ref = 0, mag = 0;
    for (int k = 0; k < 64; ++k) {
      const f32x2 a = from_ld((u01(rng) - 0.5) * powl(10.0L, 4.0L * u01(rng) - 2.0L));
      const f32x2 b = from_ld(u01(rng) - 0.5);
      qmc::mac_x2(acc, a, b);
      ref += val(a) * val(b);
      mag += fabsl(val(a) * val(b));
    }
    const f32x2 s = qmc::normalize_x2(acc);
    e_dot = std::fmax(e_dot, (double)(fabsl(val(s) - ref) / mag));
    e_norm = std::fmax(e_norm, fabsf(s.lo) / fmaxf(fabsf(s.hi), 1e-30f));
  }
  // digit-sliced contraction (oz_digits.cuh): rows of 58 pair values of
  // spread magnitude against FP64 columns, digits of both, exact integer
  // class sums (checked below 2^24 and against the BF16 range), recombined;
  // error relative to K 2^(e + f), the scale of the dropped digit classes
  double e_oz = 0;
  long long max_class = 0;
  int bad_digit = 0;
  for (int t = 0; t < 4000; ++t) {
    const int K = 58;
    f32x2 a[K];
    double c[K];
    long double amax = 0, cmax = 0;
    for (int b = 0; b < K; ++b) {
      a[b] = from_ld((u01(rng) - 0.5) * expl(-30.0L * u01(rng)));
      c[b] = (u01(rng) - 0.5) * pow(10.0, -3.0 * u01(rng));
      amax = fmaxl(amax, fabsl(val(a[b])));
      cmax = fmaxl(cmax, fabsl((long double)c[b]));
    }
    // row scale from a bound within 2x of the maximum (the kernel's slack)
    const int ea = ilogbl(amax * (1.0L + u01(rng))) + 2;
    const int fc = ilogbl(cmax) + 1;
    long long cls[qmc::kOzClasses] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < K; ++b) {
      const f32x2 xs(ldexpf(a[b].hi, -ea), ldexpf(a[b].lo, -ea));
      float d[qmc::kOzDigits];
      qmc::oz_digits(xs, d);
      double y = ldexp(c[b], -fc), dl[qmc::kOzDigits];
      for (int l = 0; l < qmc::kOzDigits; ++l) {
        y *= 256.0;
        dl[l] = nearbyint(y);
        y -= dl[l];
      }
      for (int k = 0; k < qmc::kOzDigits; ++k) {
        if (fabsf(d[k]) > 256.0f || d[k] != nearbyintf(d[k])) ++bad_digit;
        for (int l = 0; l < qmc::kOzDigits; ++l)
          if (k + l <= 5) cls[k + l] += (long long)d[k] * (long long)dl[l];
      }
    }
    float acc[qmc::kOzClasses];
    for (int g = 0; g < qmc::kOzClasses; ++g) {
      max_class = std::max(max_class, std::llabs(cls[g]));
      acc[g] = (float)cls[g];
    }
    const f32x2 s = qmc::oz_combine(acc);
    const long double got = ldexpl(val(s), ea + fc - 16);
    long double ref = 0;
    for (int b = 0; b < K; ++b) ref += val(a[b]) * (long double)c[b];
    // the scheme's scale: K terms of at most 2^(ea + fc) each
    e_oz = std::fmax(e_oz, (double)(fabsl(got - ref) / ldexpl((long double)K, ea + fc)));
  }
  std::printf("oz_contraction %.3e\noz_max_class_log2 %.3f\noz_bad_digits %d\n", e_oz,
              std::log2((double)max_class), bad_digit);
  std::printf("exp %.3e\nexp_tiny_abs %.3e\nmul %.3e\nadd %.3e\ndiv %.3e\nsqrt %.3e\nrsqrt %.3e\ndot %.3e\nnorm %.3e\nexp_unnormalised %d\n",
              e_exp, e_exp_tiny, e_mul, e_add, e_div, e_sqrt, e_rsqrt, e_dot, e_norm, bad_norm);
  return 0;
}
