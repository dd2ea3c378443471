// Device code shared by the general FP64 kernels (k_general.cu: local
// energy and log|Psi|; k_general_grad.cu: forces and parameter gradient).
//
// General single-determinant path in FP64: backflow-transformed orbitals
// (Sec. 2.1, Sec. 3: r~_i = r_i + sum_{j!=i} (w / r_ij)(r_i - r_j)), the full
// determinant Laplacian of App. F, nuclear forces by forward-mode tangents and
// the parameter gradient of log|Psi|.  One thread per walker; everything is
// recomputed from the coordinates (no AO tables are stored).
//
// Per electron coordinate x_k (k = 3 kk + e):
//   d_k A_{i,m}   = sum_d d_d phi_m(r~_i) J1[i,d;k]
//   d_k^2 A_{i,m} = sum_{d,f} H_df phi_m(r~_i) J1[i,d;k] J1[i,f;k] + sum_d d_d phi_m(r~_i) J2[i,d;k]
// with J1 = d r~ / d x_k and J2 = d^2 r~ / d x_k^2 built from the pair terms of
// g(v) = eta(|v|) v, eta = w/rho:
//   dg_d/dv_e      = eta delta_de + e1 v_d v_e,              e1 = eta'/rho = -w/rho^3
//   d2g_d/dv_e^2   = 2 delta_de e1 v_e + e1 v_d + e2 v_d v_e^2, e2 = eta''/rho^2 - eta'/rho^3 = 3w/rho^5
//   J1[i,.;i,e] = e_e + sum_j dg(.,e)(r_i - r_j),  J1[i,.;k,e] = -dg(.,e)(r_i - r_k)   (k != i)
//   J2[i,.;i,e] = sum_j d2g(.,e)(r_i - r_j),       J2[i,.;k,e] = d2g(.,e)(r_i - r_k)
// Eq. nabla_d per spin: d_k^2 D / D = Tr(A^-1 d_k^2 A) + Tr(A^-1 d_k A)^2 - Tr((A^-1 d_k A)^2),
// Eqs. nabla_sigma / delta_sigma (single determinant, with the up-down cross
// term), and App. F's decomposition with the Jastrow on the original
// coordinates:
//   E_L = -1/2 sum_k [d_k^2 J + (d_k J)^2 + 2 d_k J d_k Sigma/Sigma + d_k^2 Sigma/Sigma] + V.
#pragma once

#include <type_traits>

#include "ao_eval.cuh"
#include "dual.cuh"
#include "qmc_internal.cuh"

namespace qmc {

namespace {

template <typename T>
__device__ __forceinline__ T mono(const T& x, const T& y, const T& z, int a, int b, int c) {
  if (a < 0 || b < 0 || c < 0) return T(0.0);
  T r = T(1.0);
  for (int k = 0; k < a; ++k) r = r * x;
  for (int k = 0; k < b; ++k) r = r * y;
  for (int k = 0; k < c; ++k) r = r * z;
  return r;
}

// radial factor f, g1 = f'/rho, f2 = f'' of a shell (normalisation folded in)
template <typename T>
__device__ __forceinline__ void radial(const ShellDev& sh, const T& r2, const T& rho, T& f, T& g1, T& f2,
                                       const T* irho = nullptr) {
  if (sh.kind == 0) {
    const double z = sh.expo[0];
    T rk = T(1.0);
    for (int k = 0; k < sh.kn; ++k) rk = rk * rho;
    f = sh.coef[0] * rk * exp(-z * rho);
    const T inv = irho ? *irho : 1.0 / rho;
    const T q = double(sh.kn) * inv - z;
    g1 = q * f * inv;
    f2 = (q * q - double(sh.kn) * inv * inv) * f;
  } else {
    f = T(0.0);
    g1 = T(0.0);
    f2 = T(0.0);
    for (int p = 0; p < sh.n_prim; ++p) {
      const double al = sh.expo[p];
      const T e = sh.coef[p] * exp(-al * r2);
      f += e;
      g1 -= 2.0 * al * e;
      f2 += (4.0 * al * al * r2 - 2.0 * al) * e;
    }
  }
}

// Hessian component index for (d, f): xx yy zz xy xz yz
__device__ __forceinline__ int hidx(int d, int f) {
  if (d == f) return d;
  const int s = d + f;  // xy = 1, xz = 2, yz = 3
  return s == 1 ? 3 : (s == 2 ? 4 : 5);
}

struct GenShared {
  const ShellDev* sh;
  const int* pw;
  const double* C;     // [n_ao][n_mo] (angular factors folded in)
  const float2* Cx2;   // the same as pairs of FP32 (FP32X2 form), or null
};

// One shell's AO value, gradient and Hessian channels at displacement
// (dx, dy, dz) from its nucleus, accumulated into the MO channels.  U is the
// arithmetic type of the AO (double, or a dual number when the nucleus
// carries tangents); T that of the accumulators.
template <typename U, typename T, int NO>
__device__ __forceinline__ void shell_channels(const WfDev& wf, const GenShared& g, const ShellDev& sh, const U& dx,
                                               const U& dy, const U& dz, const U& r2, const U& rho, const U& ir2,
                                               const U& irho, int n_occ, T* phi, T (*dphi)[3], T (*hphi)[6],
                                               bool deriv) {
  U f, g1, f2;
  radial(sh, r2, rho, f, g1, f2, &irho);
  const U dv[3] = {dx, dy, dz};
  auto add = [&](int b, const U& val, const U* grad, const U* hess) {
    const double* Cb = g.C + (size_t)b * wf.n_mo;
    for (int m = 0; m < NO; ++m) {
      if (m < n_occ) {
        const double c = Cb[m];
        phi[m] += c * val;
        if (deriv) {
          for (int d = 0; d < 3; ++d) dphi[m][d] += c * grad[d];
          for (int q = 0; q < 6; ++q) hphi[m][q] += c * hess[q];
        }
      }
    }
  };
  if (sh.l <= 1) {
    // closed forms: phi = f (s) or d_c f (p), with
    //   grad_d (d_c f) = f delta_dc + d_c g1 d_d,
    //   H_de f         = g1 delta_de + q d_d d_e,    q = (f2 - g1) / rho^2,
    //   H_de (d_c f)   = g1 (delta_dc d_e + delta_ec d_d) + d_c H_de f
    const U q = deriv ? (f2 - g1) * ir2 : U(0.0);
    U hs[6], gs[3];
    if (deriv) {
      for (int d = 0; d < 3; ++d) gs[d] = g1 * dv[d];
      hs[0] = g1 + q * dx * dx;
      hs[1] = g1 + q * dy * dy;
      hs[2] = g1 + q * dz * dz;
      hs[3] = q * dx * dy;
      hs[4] = q * dx * dz;
      hs[5] = q * dy * dz;
    }
    for (int k = 0; k < sh.n_ao; ++k) {
      const int b = sh.ao_first + k;
      const int pw = g.pw[b];
      if (sh.l == 0) {
        add(b, f, gs, hs);
        continue;
      }
      const int c = (pw & 15) ? 0 : ((pw >> 4) & 15) ? 1 : 2;
      const U& x = dv[c];
      U grad[3], hess[6];
      if (deriv) {
        for (int d = 0; d < 3; ++d) grad[d] = x * gs[d];
        grad[c] += f;
        for (int q2 = 0; q2 < 6; ++q2) hess[q2] = x * hs[q2];
        // g1 (delta_dc d_e + delta_ec d_d): the diagonal element (c, c) gets
        // 2 g1 d_c, the off-diagonal elements (c, e) get g1 d_e
        hess[c] += 2.0 * gs[c];
        for (int e = 0; e < 3; ++e)
          if (e != c) hess[hidx(c, e)] += gs[e];
      }
      add(b, x * f, grad, hess);
    }
    return;
  }
  for (int k = 0; k < sh.n_ao; ++k) {
    const int b = sh.ao_first + k;
    const int pw = g.pw[b];
    const int pa[3] = {pw & 15, (pw >> 4) & 15, (pw >> 8) & 15};
    const U P = mono(dx, dy, dz, pa[0], pa[1], pa[2]);
    const U val = P * f;
    U grad[3], hess[6];
    if (deriv) {
      U dP[3];
      for (int d = 0; d < 3; ++d) {
        const int q[3] = {pa[0] - (d == 0), pa[1] - (d == 1), pa[2] - (d == 2)};
        dP[d] = double(pa[d]) * mono(dx, dy, dz, q[0], q[1], q[2]);
        grad[d] = f * dP[d] + P * g1 * dv[d];
      }
      for (int d = 0; d < 3; ++d)
        for (int e = d; e < 3; ++e) {
          const int q[3] = {pa[0] - (d == 0) - (e == 0), pa[1] - (d == 1) - (e == 1), pa[2] - (d == 2) - (e == 2)};
          const double cde = double(pa[d]) * double(pa[e] - (d == e ? 1 : 0));
          const U d2P = cde * mono(dx, dy, dz, q[0], q[1], q[2]);
          U h = f * d2P + g1 * (dP[d] * dv[e] + dP[e] * dv[d]) + P * (f2 - g1) * dv[d] * dv[e] * ir2;
          if (d == e) h += P * g1;
          hess[hidx(d, e)] = h;
        }
    }
    const double* Cb = g.C + (size_t)b * wf.n_mo;
    for (int m = 0; m < NO; ++m) {
      if (m < n_occ) {
        const double c = Cb[m];
        phi[m] += c * val;
        if (deriv) {
          for (int d = 0; d < 3; ++d) dphi[m][d] += c * grad[d];
          for (int q = 0; q < 6; ++q) hphi[m][q] += c * hess[q];
        }
      }
    }
  }
}

// MO value, gradient and Hessian channels of the occupied orbitals at one
// (possibly backflow-transformed) position p, with nuclei at R.  With dual
// numbers, only the nucleus `seeded` carries tangents: the other nuclei's
// shells are evaluated in plain doubles and enter as constants.
template <typename T, int NO>
__device__ void mo_channels(const WfDev& wf, const GenShared& g, const double p[3], const T (*R)[3], int n_occ,
                            T* phi, T (*dphi)[3], T (*hphi)[6], bool deriv, int seeded = -1) {
  for (int m = 0; m < NO; ++m) {
    phi[m] = T(0.0);
    for (int d = 0; d < 3; ++d) dphi[m][d] = T(0.0);
    for (int c = 0; c < 6; ++c) hphi[m][c] = T(0.0);
  }
  constexpr bool kDual = !std::is_same<T, double>::value;
  int cur_atom = -1;  // shells come grouped by atom: one displacement and distance per atom
  T dx = T(0.0), dy = T(0.0), dz = T(0.0), r2 = T(0.0), rho = T(0.0), ir2 = T(0.0), irho = T(0.0);
  double xd = 0.0, yd = 0.0, zd = 0.0, r2d = 0.0, rhod = 0.0, ir2d = 0.0, irhod = 0.0;
  bool plain = !kDual;
  for (int s = 0; s < wf.n_shell; ++s) {
    const ShellDev& sh = g.sh[s];
    if (sh.atom != cur_atom) {
      cur_atom = sh.atom;
      plain = !kDual || cur_atom != seeded;
      if (plain) {
        xd = p[0] - value_of(R[cur_atom][0]);
        yd = p[1] - value_of(R[cur_atom][1]);
        zd = p[2] - value_of(R[cur_atom][2]);
        r2d = xd * xd + yd * yd + zd * zd;
        rhod = sqrt(r2d);
        irhod = 1.0 / rhod;
        ir2d = irhod * irhod;
      } else {
        dx = p[0] - R[cur_atom][0];
        dy = p[1] - R[cur_atom][1];
        dz = p[2] - R[cur_atom][2];
        r2 = dx * dx + dy * dy + dz * dz;
        rho = sqrt(r2);
        irho = 1.0 / rho;
        ir2 = irho * irho;
      }
    }
    if (plain)
      shell_channels<double, T, NO>(wf, g, sh, xd, yd, zd, r2d, rhod, ir2d, irhod, n_occ, phi, dphi, hphi, deriv);
    else
      shell_channels<T, T, NO>(wf, g, sh, dx, dy, dz, r2, rho, ir2, irho, n_occ, phi, dphi, hphi, deriv);
  }
}

// The FP32X2 form of mo_channels (shells with l <= 1): displacements, radial
// factors, the closed-form derivative set and the contraction in pairs of
// FP32 (f32x2.cuh: error-free products and sums, table-driven exponential),
// widened to FP64 once per channel.  C is the pair table g.Cx2 [n_ao][n_mo]
// (angular factors folded in).  dphi / hphi may be null when !deriv.
template <int NO>
__device__ void mo_channels_x2(const WfDev& wf, const GenShared& g, const double p[3], int n_occ, double* phi,
                               double (*dphi)[3], double (*hphi)[6], bool deriv) {
  f32x2 aphi[NO], adphi[NO][3], ahphi[NO][6];
  for (int m = 0; m < NO; ++m) {
    aphi[m] = f32x2(0.f);
    for (int d = 0; d < 3; ++d) adphi[m][d] = f32x2(0.f);
    for (int q = 0; q < 6; ++q) ahphi[m][q] = f32x2(0.f);
  }
  int cur_atom = -1;
  f32x2 dv[3], r2(0.f), rho(0.f), irho(0.f), ir2(0.f);
  for (int s = 0; s < wf.n_shell; ++s) {
    const ShellDev& sh = g.sh[s];
    if (sh.atom != cur_atom) {
      cur_atom = sh.atom;
      for (int d = 0; d < 3; ++d) dv[d] = diff_x2(p[d], wf.atom_xyz[cur_atom][d]);
      r2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
      rho = sqrt_x2(r2);
      irho = recip_x2(rho);
      ir2 = irho * irho;
    }
    f32x2 f(0.f), g1(0.f), f2(0.f);
    if (sh.kind == 0) {
      const f32x2 z(sh.expo_f[0], sh.expo_lo[0]);
      f32x2 rk(1.f);
      for (int k = 0; k < sh.kn; ++k) rk = rk * rho;
      f = f32x2(sh.coef_f[0], sh.coef_lo[0]) * rk * exp_x2(-(z * rho), wf.exp_tab);
      if (deriv) {
        const f32x2 q = irho * (float)sh.kn - z;
        g1 = q * f * irho;
        f2 = (q * q - ir2 * (float)sh.kn) * f;
      }
    } else {
      for (int k = 0; k < sh.n_prim; ++k) {
        const f32x2 al(sh.expo_f[k], sh.expo_lo[k]);
        const f32x2 ce = f32x2(sh.coef_f[k], sh.coef_lo[k]) * exp_x2(-(al * r2), wf.exp_tab);
        f = f + ce;
        if (deriv) {
          const f32x2 t = (al * ce) * 2.0f;
          g1 = g1 - t;
          f2 = f2 + ((al * r2) * 2.0f - 1.0f) * t;
        }
      }
    }
    // closed forms as in shell_channels: q = (f2 - g1) / rho^2
    f32x2 gs[3], hs[6];
    if (deriv) {
      const f32x2 q = (f2 - g1) * ir2;
      for (int d = 0; d < 3; ++d) gs[d] = g1 * dv[d];
      hs[0] = g1 + q * dv[0] * dv[0];
      hs[1] = g1 + q * dv[1] * dv[1];
      hs[2] = g1 + q * dv[2] * dv[2];
      hs[3] = q * dv[0] * dv[1];
      hs[4] = q * dv[0] * dv[2];
      hs[5] = q * dv[1] * dv[2];
    }
    for (int k = 0; k < sh.n_ao; ++k) {
      const int b = sh.ao_first + k;
      f32x2 val = f, grad[3], hess[6];
      if (deriv)
        for (int d = 0; d < 3; ++d) grad[d] = gs[d];
      if (deriv)
        for (int q = 0; q < 6; ++q) hess[q] = hs[q];
      if (sh.l == 1) {
        const int pw = g.pw[b];
        const int c = (pw & 15) ? 0 : ((pw >> 4) & 15) ? 1 : 2;
        const f32x2 x = dv[c];
        val = x * f;
        if (deriv) {
          for (int d = 0; d < 3; ++d) grad[d] = x * gs[d];
          grad[c] = grad[c] + f;
          for (int q = 0; q < 6; ++q) hess[q] = x * hs[q];
          hess[c] = hess[c] + gs[c] * 2.0f;
          for (int e = 0; e < 3; ++e)
            if (e != c) hess[hidx(c, e)] = hess[hidx(c, e)] + gs[e];
        }
      }
      const float2* Cb = g.Cx2 + (size_t)b * wf.n_mo;
      for (int m = 0; m < NO; ++m) {
        if (m < n_occ) {
          const float2 cc = Cb[m];
          const f32x2 c(cc.x, cc.y);
          mac_x2(aphi[m], c, val);
          if (deriv) {
            for (int d = 0; d < 3; ++d) mac_x2(adphi[m][d], c, grad[d]);
            for (int q = 0; q < 6; ++q) mac_x2(ahphi[m][q], c, hess[q]);
          }
        }
      }
    }
  }
  for (int m = 0; m < NO; ++m) {
    phi[m] = widen(normalize_x2(aphi[m]));
    if (deriv) {
      for (int d = 0; d < 3; ++d) dphi[m][d] = widen(normalize_x2(adphi[m][d]));
      for (int q = 0; q < 6; ++q) hphi[m][q] = widen(normalize_x2(ahphi[m][q]));
    }
  }
}

// in-place inverse of a[0:n][0:n] (rows electrons, columns orbitals ->
// a[m][r] = (A^-1)_{m r}) by Gauss-Jordan with partial pivoting; returns det
template <typename T, int NO>
__device__ T small_inverse(T (*a)[NO], int n) {
  int piv[NO];
  T det = T(1.0);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(value_of(a[k][k]));
    for (int i = k + 1; i < n; ++i)
      if (fabs(value_of(a[i][k])) > best) { best = fabs(value_of(a[i][k])); p = i; }
    piv[k] = p;
    if (p != k) {
      for (int j = 0; j < n; ++j) { const T t = a[k][j]; a[k][j] = a[p][j]; a[p][j] = t; }
      det = -det;
    }
    const T pv = a[k][k];
    det = det * pv;
    const T inv = 1.0 / pv;
    a[k][k] = T(1.0);
    for (int j = 0; j < n; ++j) a[k][j] = a[k][j] * inv;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const T f = a[i][k];
      a[i][k] = T(0.0);
      for (int j = 0; j < n; ++j) a[i][j] -= f * a[k][j];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = 0; i < n; ++i) { const T t = a[i][k]; a[i][k] = a[i][p]; a[i][p] = t; }
  }
  return det;
}

// pair geometry of the original coordinates
template <int NE>
struct Pairs {
  double inv[NE][NE];  // 1 / r_ij (0 on the diagonal)
};

template <int NE>
__device__ void pair_geometry(const double (&r)[NE][3], int n, Pairs<NE>& P) {
  for (int i = 0; i < NE; ++i) P.inv[i][i] = 0.0;
  for (int i = 0; i < NE; ++i)
    for (int j = i + 1; j < NE; ++j) {
      double v = 0.0;
      if (i < n && j < n) {
        const double dx = r[i][0] - r[j][0], dy = r[i][1] - r[j][1], dz = r[i][2] - r[j][2];
        v = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
      }
      P.inv[i][j] = v;
      P.inv[j][i] = v;
    }
}

// The pair blocks of the backflow Jacobian, tabulated once per walker.  For
// the ordered pair (a, b), v = r_a - r_b, eta = w / r, e1 = -w / r^3,
// e2 = 3 w / r^5:
//   G1_ab[d][e] = delta_de eta + e1 v_d v_e                (even in v: G1_ba = G1_ab)
//   G2_ab[d][e] = 2 delta_de e1 v_e + e1 v_d + e2 v_d v_e^2  (odd in v:  G2_ba = -G2_ab)
// and the rows of backflow_rows follow as
//   i == k:  J1[i,d;i,e] = delta_de + sum_{j != i} G1_ij[d][e],  J2[i,d;i,e] = sum_{j != i} G2_ij[d][e]
//   i != k:  J1[i,d;k,e] = -G1_ik[d][e],                          J2[i,d;k,e] = G2_ik[d][e].
// G1 keeps its six distinct components (xx yy zz xy xz yz), G2 all nine;
// pairs are stored once (a < b).
template <int NE>
struct BackflowTables {
  static constexpr int kPairs = NE * (NE - 1) / 2;
  double G1[kPairs][6], G2[kPairs][9];
  double S1[NE][6], S2[NE][9];
};

__host__ __device__ constexpr int pair_index(int a, int b, int ne) { return a * ne - a * (a + 1) / 2 + (b - a - 1); }

template <int NE>
__device__ void backflow_tables(const double (&r)[NE][3], const Pairs<NE>& P, int n, double w, BackflowTables<NE>& T) {
  for (int i = 0; i < NE; ++i) {
    for (int q = 0; q < 6; ++q) T.S1[i][q] = 0.0;
    for (int q = 0; q < 9; ++q) T.S2[i][q] = 0.0;
  }
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      const int pi = pair_index(a, b, NE);
      const double iv = P.inv[a][b];
      const double v[3] = {r[a][0] - r[b][0], r[a][1] - r[b][1], r[a][2] - r[b][2]};
      const double iv2 = iv * iv, eta = w * iv, e1 = -w * iv * iv2, e2 = 3.0 * w * iv * iv2 * iv2;
      for (int d = 0; d < 3; ++d)
        for (int e = d; e < 3; ++e) {
          const double g = (d == e ? eta : 0.0) + e1 * v[d] * v[e];
          T.G1[pi][hidx(d, e)] = g;
          T.S1[a][hidx(d, e)] += g;
          T.S1[b][hidx(d, e)] += g;
        }
      for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e) {
          const double g = (d == e ? 2.0 * e1 * v[e] : 0.0) + e1 * v[d] + e2 * v[d] * v[e] * v[e];
          T.G2[pi][3 * d + e] = g;
          T.S2[a][3 * d + e] += g;
          T.S2[b][3 * d + e] -= g;
        }
    }
}

// J1[i,.;k,e] and J2[i,.;k,e] from the tables
template <int NE>
__device__ __forceinline__ void backflow_rows_t(const BackflowTables<NE>& T, int i, int k, int e, double j1[3],
                                                double j2[3]) {
  if (i == k) {
    for (int d = 0; d < 3; ++d) {
      j1[d] = (d == e ? 1.0 : 0.0) + T.S1[i][hidx(d, e)];
      j2[d] = T.S2[i][3 * d + e];
    }
  } else {
    const int pi = i < k ? pair_index(i, k, NE) : pair_index(k, i, NE);
    const double sg = i < k ? 1.0 : -1.0;  // G2_ik = -G2_ki
    for (int d = 0; d < 3; ++d) {
      j1[d] = -T.G1[pi][hidx(d, e)];
      j2[d] = sg * T.G2[pi][3 * d + e];
    }
  }
}

// Pade Jastrow (Eq. pade_kernel) on the original coordinates: J, lap J
// summed over electrons, grad_i J; and the Coulomb potential V (Eq. Hmol)
// with nuclei at R.
template <typename T, int NE>
__device__ void jastrow_coulomb(const WfDev& wf, const double (&r)[NE][3], const T (*R)[3], const Pairs<NE>& P,
                                double& J, double& lapJ, double (&gJ)[NE][3], T& V) {
  const int N = wf.n_elec, nu = wf.n_up;
  double Vee = 0.0;
  J = 0.0;
  lapJ = 0.0;
  for (int i = 0; i < NE; ++i)
    for (int d = 0; d < 3; ++d) gJ[i][d] = 0.0;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      const double iv = P.inv[i][j], dist = 1.0 / iv;
      const double w0 = ((i < nu) == (j < nu)) ? wf.w0_par : wf.w0_anti;
      const double rd = 1.0 / (1.0 + wf.jb * dist);
      const double u1 = w0 * rd * rd, u2 = -2.0 * w0 * wf.jb * rd * rd * rd;
      J += w0 * dist * rd;
      Vee += iv;
      lapJ += 2.0 * (u2 + 2.0 * u1 * iv);
      for (int d = 0; d < 3; ++d) {
        const double s = u1 * iv * (r[i][d] - r[j][d]);
        gJ[i][d] += s;
        gJ[j][d] -= s;
      }
    }
  V = T(Vee);
  for (int a = 0; a < wf.n_atom; ++a) {
    for (int i = 0; i < N; ++i) {
      const T dx = r[i][0] - R[a][0], dy = r[i][1] - R[a][1], dz = r[i][2] - R[a][2];
      V -= wf.atom_z[a] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    for (int b = a + 1; b < wf.n_atom; ++b) {
      const T dx = R[a][0] - R[b][0], dy = R[a][1] - R[b][1], dz = R[a][2] - R[b][2];
      V += wf.atom_z[a] * wf.atom_z[b] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
}

// backflow positions r~_i = r_i + sum_{j != i} (w / r_ij)(r_i - r_j)
template <int NE>
__device__ void backflow_positions(const double (&r)[NE][3], const Pairs<NE>& P, int N, double w,
                                   double (&rt)[NE][3]) {
  for (int i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) {
      double acc = r[i][d];
      for (int j = 0; j < N; ++j)
        if (j != i) acc += w * P.inv[i][j] * (r[i][d] - r[j][d]);
      rt[i][d] = acc;
    }
}

// Orbital values alone at one position: the value part of mo_channels, in
// the same order of operations.
template <int NO>
__device__ __forceinline__ void mo_values(const WfDev& wf, const GenShared& g, const double (&p)[3], int n_occ, double (&phi)[NO]) {
#pragma unroll
  for (int m = 0; m < NO; ++m) phi[m] = 0.0;
  int cur_atom = -1;  // shells come grouped by atom: one displacement and distance per atom
  double dx = 0.0, dy = 0.0, dz = 0.0, r2 = 0.0, rho = 0.0;
  for (int s = 0; s < wf.n_shell; ++s) {
    const ShellDev& sh = g.sh[s];
    if (sh.atom != cur_atom) {
      cur_atom = sh.atom;
      dx = p[0] - wf.atom_xyz[cur_atom][0];
      dy = p[1] - wf.atom_xyz[cur_atom][1];
      dz = p[2] - wf.atom_xyz[cur_atom][2];
      r2 = dx * dx + dy * dy + dz * dz;
      rho = sqrt(r2);
    }
    double f, g1, f2;
    radial(sh, r2, rho, f, g1, f2);
    for (int k = 0; k < sh.n_ao; ++k) {
      const int b = sh.ao_first + k;
      const int pw = g.pw[b];
      const double val = mono(dx, dy, dz, pw & 15, (pw >> 4) & 15, (pw >> 8) & 15) * f;
      const double* Cb = g.C + (size_t)b * wf.n_mo;
#pragma unroll
      for (int m = 0; m < NO; ++m)
        if (m < n_occ) phi[m] += Cb[m] * val;
    }
  }
}

// Determinant alone: the pivots of small_inverse's elimination (partial
// pivoting, scaled pivot row), restricted to the rows and columns that later
// pivots depend on.  Fully unrolled with opaque selects for the row
// exchanges, so the matrix stays in registers.
template <int NO>
__device__ __forceinline__ double det_pivots(double (&a)[NO][NO], int n) {
  double det = 1.0;
#pragma unroll
  for (int k = 0; k < NO; ++k) {
    if (k < n) {
      int p = k;
      double best = fabs(a[k][k]);
#pragma unroll
      for (int i = k + 1; i < NO; ++i)
        if (i < n && fabs(a[i][k]) > best) { best = fabs(a[i][k]); p = i; }
      if (p != k) det = -det;
#pragma unroll
      for (int i = k + 1; i < NO; ++i) {
        const bool sw = i == p;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          const double t = a[k][j];
          a[k][j] = dsel(sw, a[i][j], t);
          a[i][j] = dsel(sw, t, a[i][j]);
        }
      }
      const double pv = a[k][k];
      det = det * pv;
      const double inv = 1.0 / pv;
#pragma unroll
      for (int j = k + 1; j < NO; ++j) a[k][j] = a[k][j] * inv;
#pragma unroll
      for (int i = k + 1; i < NO; ++i) {
        if (i < n) {
          const double f = a[i][k];
#pragma unroll
          for (int j = k + 1; j < NO; ++j) a[i][j] -= f * a[k][j];
        }
      }
    }
  }
  return det;
}

}  // namespace

// log|Psi| alone of a single-determinant walker (the Metropolis value path):
// Pade J, backflow positions, orbital values and the two determinants --
// eval_walker's value part without its derivative channels.  Loops over the
// electron-count bracket are unrolled (guards on the actual counts) so that
// every array stays in registers; the pair terms are visited in eval_walker's
// order.
template <int NE, int NO, bool PAIRS = false>
__device__ __forceinline__ double logpsi_walker(const WfDev& wf, const GenShared& g, const double (&r)[NE][3]) {
  const int N = wf.n_elec, nu = wf.n_up, nd = wf.n_down;
  const double w = wf.bf_w;
  double J = 0.0, rt[NE][3];
#pragma unroll
  for (int i = 0; i < NE; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) rt[i][d] = r[i][d];
#pragma unroll
  for (int i = 0; i < NE; ++i)
#pragma unroll
    for (int j = i + 1; j < NE; ++j)
      if (j < N) {
        const double dx = r[i][0] - r[j][0], dy = r[i][1] - r[j][1], dz = r[i][2] - r[j][2];
        const double iv = 1.0 / sqrt(dx * dx + dy * dy + dz * dz), dist = 1.0 / iv;
        const double w0 = ((i < nu) == (j < nu)) ? wf.w0_par : wf.w0_anti;
        const double rd = 1.0 / (1.0 + wf.jb * dist);
        J += w0 * dist * rd;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          rt[i][d] += w * iv * (r[i][d] - r[j][d]);
          rt[j][d] += w * iv * (r[j][d] - r[i][d]);
        }
      }
  const int n_occ = nu > nd ? nu : nd;
  double phi[NE][NO];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    if (q < N) {
      if constexpr (PAIRS) mo_channels_x2<NO>(wf, g, rt[q], n_occ, phi[q], nullptr, nullptr, false);
      else mo_values<NO>(wf, g, rt[q], n_occ, phi[q]);
    }
    else
#pragma unroll
      for (int m = 0; m < NO; ++m) phi[q][m] = 0.0;
  }
  double logdet = log(fabs(wf.det_w[0]));
  double a[NO][NO];
  if (nu > 0) {  // spin up: electrons 0 .. nu-1
#pragma unroll
    for (int e = 0; e < NO; ++e)
#pragma unroll
      for (int m = 0; m < NO; ++m) a[e][m] = phi[e < NE ? e : 0][m];
    logdet += log_abs(det_pivots<NO>(a, nu));
  }
  if (nd > 0) {  // spin down: electrons nu .. nu+nd-1 (rows picked by selects)
#pragma unroll
    for (int e = 0; e < NO; ++e)
#pragma unroll
      for (int m = 0; m < NO; ++m) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < NE; ++q) v = dsel(q == nu + e, phi[q][m], v);
        a[e][m] = v;
      }
    logdet += log_abs(det_pivots<NO>(a, nd));
  }
  return J + logdet;
}

// Local energy and log|Psi| of one walker.  T = double, or Dual<K> with the
// nuclear coordinates R seeded for forces.  NE >= n_elec, NO >= occupied
// orbitals per spin.
template <typename T, int NE, int NO, bool PAIRS = false>
__device__ void eval_walker(const WfDev& wf, const GenShared& g, const double (&r)[NE][3], const T (*R)[3],
                            bool kinetic, T& eloc, T& logpsi, int seeded = -1) {
  const int N = wf.n_elec, nu = wf.n_up;
  const double w = wf.bf_w;
  Pairs<NE> P;
  pair_geometry<NE>(r, N, P);
  double J, lapJ, gJ[NE][3], rt[NE][3];
  T V;
  jastrow_coulomb<T, NE>(wf, r, R, P, J, lapJ, gJ, V);
  backflow_positions<NE>(r, P, N, w, rt);
  // orbitals at the backflow positions
  const int n_occ = nu > wf.n_down ? nu : wf.n_down;
  BackflowTables<NE> BT;
  if (kinetic && w != 0.0) backflow_tables<NE>(r, P, N, w, BT);
  T phi[NE][NO], dphi[NE][NO][3], hphi[NE][NO][6];
  for (int i = 0; i < N; ++i) {
    if constexpr (PAIRS) mo_channels_x2<NO>(wf, g, rt[i], n_occ, phi[i], dphi[i], hphi[i], kinetic);
    else mo_channels<T, NO>(wf, g, rt[i], R, n_occ, phi[i], dphi[i], hphi[i], kinetic, seeded);
  }
  // reference determinants (the expansion holds one determinant)
  T ainv[2][NO][NO];
  T logdet = T(log(fabs(wf.det_w[0])));
  for (int s = 0; s < 2; ++s) {
    const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
    if (n == 0) continue;
    for (int a = 0; a < n; ++a)
      for (int m = 0; m < n; ++m) ainv[s][a][m] = phi[i0 + a][m];
    const T det = small_inverse<T, NO>(ainv[s], n);
    logdet += log_abs(det);
  }
  logpsi = J + logdet;
  if (!kinetic) return;
  // Per spin, the orbital gradients and Hessians of each row contracted with
  // A^-1 once per walker:
  //   M_d[a][b] = sum_m d_d phi_m(r~_{i_a}) (A^-1)_{m b},   Hc[i_a][q] = sum_m (A^-1)_{m a} H_q phi_m(r~_{i_a}).
  // Per coordinate x_k, with Y = (d_k A) A^-1, Y[a][b] = sum_d J1_a(k)_d M_d[a][b]:
  //   Tr(A^-1 d_k A) = Tr Y,  Tr((A^-1 d_k A)^2) = Tr(Y^2),
  //   Tr(A^-1 d_k^2 A) = sum_a [sum_q cq_a(k) Hc[i_a][q] + sum_d J2_a(k)_d M_d[a][a]].
  T Md[2][3][NO][NO], Hc[NE][6];
  for (int s = 0; s < 2; ++s) {
    const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
    for (int a = 0; a < n; ++a) {
      const int i = i0 + a;
      for (int d = 0; d < 3; ++d)
        for (int b = 0; b < n; ++b) {
          T acc = T(0.0);
          for (int m = 0; m < n; ++m) acc += dphi[i][m][d] * ainv[s][m][b];
          Md[s][d][a][b] = acc;
        }
      for (int q = 0; q < 6; ++q) {
        T acc = T(0.0);
        for (int m = 0; m < n; ++m) acc += ainv[s][m][a] * hphi[i][m][q];
        Hc[i][q] = acc;
      }
    }
  }
  T kin = T(lapJ);
  for (int kk = 0; kk < N; ++kk) {
    const int sk = kk < nu ? 0 : 1;
    for (int e = 0; e < 3; ++e) {
      T a_s[2] = {T(0.0), T(0.0)}, b_s[2] = {T(0.0), T(0.0)};
      for (int s = 0; s < 2; ++s) {
        const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
        if (n == 0 || (w == 0.0 && s != sk)) continue;
        T Y[NO][NO];
        T tr2 = T(0.0);
        for (int a = 0; a < n; ++a) {
          const int i = i0 + a;
          if (w == 0.0 && i != kk) {
            for (int b = 0; b < n; ++b) Y[a][b] = T(0.0);
            continue;
          }
          double j1[3], j2[3];
          if (w != 0.0) {
            backflow_rows_t<NE>(BT, i, kk, e, j1, j2);
          } else {  // no backflow: only the moving electron's own row, J1 = unit, J2 = 0
            for (int d = 0; d < 3; ++d) { j1[d] = d == e ? 1.0 : 0.0; j2[d] = 0.0; }
          }
          // sum_{d,f} j1_d j1_f H_df = sum_q cq[q] H_q over the six distinct
          // Hessian components (xx yy zz xy xz yz)
          const double cq[6] = {j1[0] * j1[0], j1[1] * j1[1], j1[2] * j1[2],
                                2.0 * j1[0] * j1[1], 2.0 * j1[0] * j1[2], 2.0 * j1[1] * j1[2]};
          for (int q = 0; q < 6; ++q) tr2 += cq[q] * Hc[i][q];
          for (int d = 0; d < 3; ++d) tr2 += j2[d] * Md[s][d][a][a];
          for (int b = 0; b < n; ++b) {
            T v1 = T(0.0);
            for (int d = 0; d < 3; ++d) v1 += j1[d] * Md[s][d][a][b];
            Y[a][b] = v1;
          }
        }
        T tr1 = T(0.0), trsq = T(0.0);
        for (int a = 0; a < n; ++a) {
          tr1 += Y[a][a];
          for (int b = 0; b < n; ++b) trsq += Y[a][b] * Y[b][a];
        }
        a_s[s] = tr1;
        b_s[s] = tr2 + tr1 * tr1 - trsq;
      }
      const T dS = a_s[0] + a_s[1];
      const T d2S = b_s[0] + 2.0 * a_s[0] * a_s[1] + b_s[1];
      const double gj = gJ[kk][e];
      kin += gj * gj + 2.0 * gj * dS + d2S;
    }
  }
  eloc = -0.5 * kin + V;
}

// Multi-determinant local energy with backflow (FP64).  Every coordinate
// x_k moves every row of both spins' matrices, so per coordinate and spin the
// excited determinants' first and second log-derivatives come from tables of
// the reference inverse (Eq. table for Tr(A_X^-1 d A_X) and
// Tr(A_X^-1 d^2 A_X), Eq. table_squared for Tr((A_X^-1 d A_X)^2); App. F, H).
// With t_p = A0^-1 Phi_p, X1 = A0^-1 dA, X2 = A0^-1 d^2A (all columns) and
//   m1_p = X1[:, p] - X1[:, occ] t_p,  m2_p likewise from X2,  y_p = X1[:, occ] m1_p,
// an excitation X (holes h_a, particles p_b) has S_ab = t_{p_b}[h_a],
// (PMP)_ab = m1_{p_b}[h_a], (PYP)_ab = y_{p_b}[h_a], (PM2P)_ab = m2_{p_b}[h_a]
// and, with R = det S and adj S its adjugate (k = 1, 2), division-free:
//   R d D_X/D_X   = R tr1 + Tr(adj S PMP)
//   R d^2 D_X/D_X = R (tr2 + tr1^2 - trsq) + Tr(adj S PM2P) + 2 tr1 Tr(adj S PMP)
//                   + 2 det(PMP) - 2 Tr(adj S PYP)
// (Eq. nabla_d; for k = 2 the terms (Tr Z)^2 - Tr(Z^2) = 2 det Z of
// Z = S^-1 PMP collapse to 2 det(PMP) / R; for k = 1 they cancel), where
// tr1 = Tr X1_occ, trsq = Tr(X1_occ^2), tr2 = Tr X2_occ.  Then
// Eqs. nabla_sigma / delta_sigma with the up-down cross term.
template <int NE, int NC, bool PAIRS = false>
__device__ void eval_walker_md(const WfDev& wf, const GenShared& g, const double (&r)[NE][3], bool kinetic,
                               double& eloc, double& logpsi) {
  constexpr int NS = 4;  // occupied orbitals per spin
  const int N = wf.n_elec, nu = wf.n_up;
  const double w = wf.bf_w;
  Pairs<NE> P;
  pair_geometry<NE>(r, N, P);
  double J, lapJ, gJ[NE][3], rt[NE][3], V;
  jastrow_coulomb<double, NE>(wf, r, wf.atom_xyz, P, J, lapJ, gJ, V);
  backflow_positions<NE>(r, P, N, w, rt);
  BackflowTables<NE> BT;
  if (kinetic) backflow_tables<NE>(r, P, N, w, BT);
  const int ncol = wf.p_hi[0] > wf.p_hi[1] ? wf.p_hi[0] : wf.p_hi[1];
  double phi[NE][NC], dphi[NE][NC][3], hphi[NE][NC][6];
  for (int i = 0; i < N; ++i) {
    if constexpr (PAIRS) mo_channels_x2<NC>(wf, g, rt[i], ncol, phi[i], dphi[i], hphi[i], kinetic);
    else mo_channels<double, NC>(wf, g, rt[i], wf.atom_xyz, ncol, phi[i], dphi[i], hphi[i], kinetic);
  }
  // reference inverses and the value tables t_p
  double ainv[2][NS][NS], tv[2][NS][NC], det0 = 1.0;
  for (int s = 0; s < 2; ++s) {
    const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
    if (n == 0) continue;
    for (int a = 0; a < n; ++a)
      for (int m = 0; m < n; ++m) ainv[s][a][m] = phi[i0 + a][m];
    det0 *= small_inverse<double, NS>(ainv[s], n);
    for (int m = 0; m < n; ++m)
      for (int c = n; c < wf.p_hi[s]; ++c) {
        double acc = 0.0;
        for (int a = 0; a < n; ++a) acc += ainv[s][m][a] * phi[i0 + a][c];
        tv[s][m][c] = acc;
      }
  }
  // determinant ratios R_s of every determinant (coordinate independent)
  auto ratio = [&](int s, const int* e) -> double {
    if (e[0] == 0) return 1.0;
    if (e[0] == 1) return tv[s][e[1]][e[3]];
    return tv[s][e[1]][e[3]] * tv[s][e[2]][e[4]] - tv[s][e[1]][e[4]] * tv[s][e[2]][e[3]];
  };
  double sum_r = 0.0;
  for (int d = 0; d < wf.n_det; ++d) {
    const int* eu = wf.exc + (0 * kMaxExc + wf.det_idx[2 * d]) * 5;
    const int* ed = wf.exc + (1 * kMaxExc + wf.det_idx[2 * d + 1]) * 5;
    sum_r += wf.det_w[d] * ratio(0, eu) * ratio(1, ed);
  }
  logpsi = J + log(fabs(det0 * sum_r));
  if (!kinetic) return;
  double kin = lapJ;
  for (int kk = 0; kk < N; ++kk)
    for (int e = 0; e < 3; ++e) {
      double tr1[2] = {0.0, 0.0}, trsq[2] = {0.0, 0.0}, tr2[2] = {0.0, 0.0};
      double pm1[2][NS][NC], py[2][NS][NC], pm2[2][NS][NC];
      for (int s = 0; s < 2; ++s) {
        const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
        if (n == 0) continue;
        double dA[NS][NC], d2A[NS][NC];
        for (int a = 0; a < n; ++a) {
          const int i = i0 + a;
          double j1[3], j2[3];
          backflow_rows_t<NE>(BT, i, kk, e, j1, j2);
          const double cq[6] = {j1[0] * j1[0], j1[1] * j1[1], j1[2] * j1[2],
                                2.0 * j1[0] * j1[1], 2.0 * j1[0] * j1[2], 2.0 * j1[1] * j1[2]};
          for (int c = 0; c < wf.p_hi[s]; ++c) {
            double v1 = 0.0, v2 = 0.0;
            for (int dd = 0; dd < 3; ++dd) {
              v1 += j1[dd] * dphi[i][c][dd];
              v2 += j2[dd] * dphi[i][c][dd];
            }
            for (int q = 0; q < 6; ++q) v2 += cq[q] * hphi[i][c][q];
            dA[a][c] = v1;
            d2A[a][c] = v2;
          }
        }
        double X1[NS][NC], X2[NS][NC];
        for (int m = 0; m < n; ++m)
          for (int c = 0; c < wf.p_hi[s]; ++c) {
            double a1 = 0.0, a2 = 0.0;
            for (int a = 0; a < n; ++a) {
              a1 += ainv[s][m][a] * dA[a][c];
              a2 += ainv[s][m][a] * d2A[a][c];
            }
            X1[m][c] = a1;
            X2[m][c] = a2;
          }
        for (int m = 0; m < n; ++m) {
          tr1[s] += X1[m][m];
          tr2[s] += X2[m][m];
          for (int q = 0; q < n; ++q) trsq[s] += X1[m][q] * X1[q][m];
        }
        for (int c = n; c < wf.p_hi[s]; ++c) {
          double m1[NS];
          for (int m = 0; m < n; ++m) {
            double a1 = X1[m][c], a2 = X2[m][c];
            for (int q = 0; q < n; ++q) {
              a1 -= X1[m][q] * tv[s][q][c];
              a2 -= X2[m][q] * tv[s][q][c];
            }
            m1[m] = a1;
            pm1[s][m][c] = a1;
            pm2[s][m][c] = a2;
          }
          for (int m = 0; m < n; ++m) {
            double acc = 0.0;
            for (int q = 0; q < n; ++q) acc += X1[m][q] * m1[q];
            py[s][m][c] = acc;
          }
        }
      }
      // R, R dD/D and R d^2D/D of one spin excitation
      auto terms = [&](int s, const int* e, double& R, double& RG, double& RB) {
        const double base = tr2[s] + tr1[s] * tr1[s] - trsq[s];
        if (e[0] == 0) {
          R = 1.0;
          RG = tr1[s];
          RB = base;
        } else if (e[0] == 1) {
          const int h = e[1], p = e[3];
          R = tv[s][h][p];
          const double q1 = pm1[s][h][p];
          RG = R * tr1[s] + q1;
          RB = R * base + pm2[s][h][p] + 2.0 * (tr1[s] * q1 - py[s][h][p]);
        } else {
          const int h1 = e[1], h2 = e[2], p1 = e[3], p2 = e[4];
          const double s00 = tv[s][h1][p1], s01 = tv[s][h1][p2], s10 = tv[s][h2][p1], s11 = tv[s][h2][p2];
          R = s00 * s11 - s01 * s10;
          auto adj_tr = [&](const double (*Q)[NC]) {
            return s11 * Q[h1][p1] - s01 * Q[h2][p1] - s10 * Q[h1][p2] + s00 * Q[h2][p2];
          };
          const double t1 = adj_tr(pm1[s]);
          const double detq = pm1[s][h1][p1] * pm1[s][h2][p2] - pm1[s][h1][p2] * pm1[s][h2][p1];
          RG = R * tr1[s] + t1;
          RB = R * base + adj_tr(pm2[s]) + 2.0 * tr1[s] * t1 + 2.0 * detq - 2.0 * adj_tr(py[s]);
        }
      };
      double acc_g = 0.0, acc_b = 0.0;
      for (int d = 0; d < wf.n_det; ++d) {
        double R0, G0, B0, R1, G1, B1;
        terms(0, wf.exc + (0 * kMaxExc + wf.det_idx[2 * d]) * 5, R0, G0, B0);
        terms(1, wf.exc + (1 * kMaxExc + wf.det_idx[2 * d + 1]) * 5, R1, G1, B1);
        const double dw = wf.det_w[d];
        acc_g += dw * (G0 * R1 + R0 * G1);
        acc_b += dw * (B0 * R1 + 2.0 * G0 * G1 + R0 * B1);
      }
      const double dS = acc_g / sum_r, d2S = acc_b / sum_r;
      const double gj = gJ[kk][e];
      kin += gj * gj + 2.0 * gj * dS + d2S;
    }
  eloc = -0.5 * kin + V;
}

// ----------------------------------------------------------------------------
// kernels

template <int NE>
__device__ __forceinline__ void load_walker(const double* walkers, int64_t ldw, int64_t w, int n, double (&r)[NE][3]) {
  for (int i = 0; i < NE; ++i)
    for (int d = 0; d < 3; ++d) r[i][d] = i < n ? walkers[(int64_t)(3 * i + d) * ldw + w] : 0.0;
}

__device__ __forceinline__ void stage_tables(const WfDev& wf, GenShared& g, unsigned char* smem) {
  ShellDev* sh = reinterpret_cast<ShellDev*>(smem);
  int* pw = reinterpret_cast<int*>(sh + wf.n_shell);
  for (int k = threadIdx.x; k < wf.n_shell * (int)(sizeof(ShellDev) / 4); k += blockDim.x)
    reinterpret_cast<int*>(sh)[k] = reinterpret_cast<const int*>(wf.shells)[k];
  for (int k = threadIdx.x; k < wf.n_ao; k += blockDim.x) pw[k] = wf.ao_pow[k];
  __syncthreads();
  g.sh = sh;
  g.pw = pw;
  g.C = wf.mo64;
  g.Cx2 = wf.mo_x2n;
}

inline size_t gen_table_bytes(const WfDev& wf) {
  return (sizeof(ShellDev) * wf.n_shell + sizeof(int) * wf.n_ao + 15) & ~size_t(15);
}

#define QMC_GEN_DISPATCH(CALL)                                        \
  {                                                                   \
    const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;         \
    if (wf.n_elec <= 2 && ns <= 1) { constexpr int NE = 2, NO = 1; CALL; } \
    else if (wf.n_elec <= 4 && ns <= 2) { constexpr int NE = 4, NO = 2; CALL; } \
    else if (wf.n_elec <= 6 && ns <= 3) { constexpr int NE = 6, NO = 3; CALL; } \
    else if (wf.n_elec <= 8 && ns <= 4) { constexpr int NE = 8, NO = 4; CALL; } \
    else return cudaErrorInvalidValue;                                \
  }

}  // namespace qmc
