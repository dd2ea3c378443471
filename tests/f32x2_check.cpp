// Host check of the pair-of-FP32 arithmetic (paper_2506_09743_gb300/csrc/f32x2.cuh)
// against long-double references.  Prints one "name max_rel_err" line per
// operation; the Python test reads them.  Built with -ffp-contract=off so
// that the error-free transformations are evaluated as written.
#include <cmath>
#include <cstdio>
#include <random>

#include "../paper_2506_09743_gb300/csrc/f32x2.cuh"

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
  std::printf("exp %.3e\nexp_tiny_abs %.3e\nmul %.3e\nadd %.3e\ndiv %.3e\nsqrt %.3e\nrsqrt %.3e\ndot %.3e\nnorm %.3e\nexp_unnormalised %d\n",
              e_exp, e_exp_tiny, e_mul, e_add, e_div, e_sqrt, e_rsqrt, e_dot, e_norm, bad_norm);
  return 0;
}
