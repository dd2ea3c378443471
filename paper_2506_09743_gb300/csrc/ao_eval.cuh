// Atomic-orbital evaluation shared by the SIMT and tensor-core AO->MO kernels.
//
// phi = P(d) f(|d|), d = r - R_atom, P = dx^a dy^b dz^c (Sec. 2.1):
//   STO  f = c rho^kn exp(-zeta rho)
//   GTO  f = sum_p c_p exp(-alpha_p rho^2)
// (radial normalisation folded into c; angular factor folded into the MO
// table).  With g1 = f'/rho and f2 = f'':
//   grad phi = f grad P + P g1 d
//   lap phi  = f lap P + P (f2 + 2 (l + 1) g1)      (d . grad P = l P, Euler)
// The kinetic channel written for the determinant stage is the one-body
// operator O = lap + 2 grad_i J . grad applied to phi (App. F: the Jastrow
// cross term 2 grad J/J . grad Sigma/Sigma and lap Sigma/Sigma are both
// traces of one-body operators, so their sum is one trace).
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

template <typename T>
__device__ __forceinline__ void pow_table(T x, T* p) {  // p[0..4] = x^0..x^4
  p[0] = T(1); p[1] = x; p[2] = x * x; p[3] = p[2] * x; p[4] = p[2] * p[2];
}

// Shell parameters in the arithmetic type (FP32 copies avoid conversions).
__device__ __forceinline__ double sh_expo(const ShellDev& sh, int p, double) { return sh.expo[p]; }
__device__ __forceinline__ float sh_expo(const ShellDev& sh, int p, float) { return sh.expo_f[p]; }
__device__ __forceinline__ double sh_coef(const ShellDev& sh, int p, double) { return sh.coef[p]; }
__device__ __forceinline__ float sh_coef(const ShellDev& sh, int p, float) { return sh.coef_f[p]; }

// Radial part and its derivatives for one shell at distance rho (rho^2 = r2).
template <typename T>
__device__ __forceinline__ void shell_radial(const ShellDev& sh, T r2, T rho, T inv_rho, T& f, T& g1, T& f2,
                                             bool deriv) {
  if (sh.kind == 0) {
    const T zeta = sh_expo(sh, 0, T(0));
    T rk = T(1);
    for (int k = 0; k < sh.kn; ++k) rk *= rho;
    f = sh_coef(sh, 0, T(0)) * rk * exp(-zeta * rho);
    if (deriv) {
      const T q = T(sh.kn) * inv_rho - zeta;
      g1 = q * f * inv_rho;
      f2 = (q * q - T(sh.kn) * inv_rho * inv_rho) * f;
    }
  } else {
    f = T(0); g1 = T(0); f2 = T(0);
    for (int p = 0; p < sh.n_prim; ++p) {
      const T al = sh_expo(sh, p, T(0));
      const T e = sh_coef(sh, p, T(0)) * exp(-al * r2);
      f += e;
      if (deriv) {
        g1 -= T(2) * al * e;
        f2 += (T(4) * al * al * r2 - T(2) * al) * e;
      }
    }
  }
}

// p[k] for k in 0..4 (k < 0 gives p[0]; callers multiply it by zero) as a
// chain of selects, so that the power tables stay in registers.
template <typename T>
__device__ __forceinline__ T pick(const T* p, int k) {
  T r = p[0];
  r = k == 1 ? p[1] : r;
  r = k == 2 ? p[2] : r;
  r = k == 3 ? p[3] : r;
  r = k == 4 ? p[4] : r;
  return r;
}

// Angular monomial and derivatives for powers (a, b, c).
template <typename T>
__device__ __forceinline__ void angular(int pw, const T* px, const T* py, const T* pz, T& P, T& Px, T& Py, T& Pz,
                                        T& lapP, bool deriv) {
  const int a = pw & 15, b = (pw >> 4) & 15, c = (pw >> 8) & 15;
  const T xa = pick(px, a), yb = pick(py, b), zc = pick(pz, c);
  P = xa * yb * zc;
  if (deriv) {
    Px = a ? T(a) * pick(px, a - 1) * yb * zc : T(0);
    Py = b ? T(b) * xa * pick(py, b - 1) * zc : T(0);
    Pz = c ? T(c) * xa * yb * pick(pz, c - 1) : T(0);
    lapP = T(0);
    if (a >= 2) lapP += T(a * (a - 1)) * pick(px, a - 2) * yb * zc;
    if (b >= 2) lapP += T(b * (b - 1)) * xa * pick(py, b - 2) * zc;
    if (c >= 2) lapP += T(c * (c - 1)) * xa * yb * pick(pz, c - 2);
  }
}

// Electron - nucleus displacement in the arithmetic type.  FP64: plain
// differences.  FP32: both positions are split into float pairs first, so
// the difference is accurate to 2^-24 relative even for an electron close to
// the nucleus, without any FP64 instruction.
__device__ __forceinline__ void displacement(double rx, double ry, double rz, const double* a, double& dx,
                                             double& dy, double& dz) {
  dx = rx - a[0]; dy = ry - a[1]; dz = rz - a[2];
}
__device__ __forceinline__ void displacement(double rx, double ry, double rz, const double* a, float& dx,
                                             float& dy, float& dz) {
  float xh, xl, yh, yl, zh, zl, ah, al;
  split_f64(rx, xh, xl); split_f64(ry, yh, yl); split_f64(rz, zh, zl);
  split_f64(a[0], ah, al); dx = (xh - ah) + (xl - al);
  split_f64(a[1], ah, al); dy = (yh - ah) + (yl - al);
  split_f64(a[2], ah, al); dz = (zh - ah) + (zl - al);
}

// r - a for a position r and a nucleus a given in FP64, as a normalised pair:
// one FP64 subtraction (exact when r is next to a, Sterbenz), then the split.
// (Splitting r and a first keeps only 2^-48 of |r| in each, which is a
// relative error of 2^-48 |r| / |r - a| in the difference.)
__device__ __forceinline__ f32x2 diff_x2(double r, double a) {
  float h, l;
  split_f64(r - a, h, l);
  return fast_two_sum(h, l);
}

}  // namespace qmc
