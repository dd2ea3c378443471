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

// Radial part and its derivatives for one shell at distance rho (rho^2 = r2).
template <typename T>
__device__ __forceinline__ void shell_radial(const ShellDev& sh, T r2, T rho, T inv_rho, T& f, T& g1, T& f2,
                                             bool deriv) {
  if (sh.kind == 0) {
    const T zeta = T(sh.expo[0]);
    T rk = T(1);
    for (int k = 0; k < sh.kn; ++k) rk *= rho;
    f = T(sh.coef[0]) * rk * exp(-zeta * rho);
    if (deriv) {
      const T q = T(sh.kn) * inv_rho - zeta;
      g1 = q * f * inv_rho;
      f2 = (q * q - T(sh.kn) * inv_rho * inv_rho) * f;
    }
  } else {
    f = T(0); g1 = T(0); f2 = T(0);
    for (int p = 0; p < sh.n_prim; ++p) {
      const T al = T(sh.expo[p]);
      const T e = T(sh.coef[p]) * exp(-al * r2);
      f += e;
      if (deriv) {
        g1 -= T(2) * al * e;
        f2 += (T(4) * al * al * r2 - T(2) * al) * e;
      }
    }
  }
}

// Angular monomial and derivatives for powers (a, b, c).
template <typename T>
__device__ __forceinline__ void angular(int pw, const T* px, const T* py, const T* pz, T& P, T& Px, T& Py, T& Pz,
                                        T& lapP, bool deriv) {
  const int a = pw & 15, b = (pw >> 4) & 15, c = (pw >> 8) & 15;
  P = px[a] * py[b] * pz[c];
  if (deriv) {
    Px = a ? T(a) * px[a - 1] * py[b] * pz[c] : T(0);
    Py = b ? T(b) * px[a] * py[b - 1] * pz[c] : T(0);
    Pz = c ? T(c) * px[a] * py[b] * pz[c - 1] : T(0);
    lapP = T(0);
    if (a >= 2) lapP += T(a * (a - 1)) * px[a - 2] * py[b] * pz[c];
    if (b >= 2) lapP += T(b * (b - 1)) * px[a] * py[b - 2] * pz[c];
    if (c >= 2) lapP += T(c * (c - 1)) * px[a] * py[b] * pz[c - 2];
  }
}

}  // namespace qmc
