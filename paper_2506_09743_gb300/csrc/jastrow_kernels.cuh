// Pade electron-electron Jastrow and Coulomb potential, one thread per walker.
//
//   J        = sum_{i<j} u(r_ij),  u(r) = w0 r / (1 + b r)   (Eqs. jastrow, pade_kernel)
//   grad_i J = sum_{j!=i} u'(r_ij) (r_i - r_j) / r_ij,  u' = w0 / (1 + b r)^2
//   kinJ     = sum_i lap_i J + |grad_i J|^2,  lap_i J = sum_j u'' + 2 u'/r_ij,
//              u'' = -2 w0 b / (1 + b r)^3                     (App. F, lap e^J / e^J)
//   V        = sum_{i<j} 1/r_ij - sum_{i,a} Z_a / r_ia + V_nn  (Eq. Hmol)
// Each pair is visited once.
//
// Many-body Jastrow (App. D), compiled in only when the wavefunction has it:
//   K_en(r)  = (w0 r + w1 r^2) / (1 + w2 r) per electron i and atom a, r = r_ai:
//              K' = (w0 + 2 w1 r + w1 w2 r^2) / (1 + w2 r)^2,  K'' = 2 (w1 - w0 w2) / (1 + w2 r)^3
//   K_een    = sum_mu c_mu f(a1, b1; x) f(a2, b2; y) f(a3, b3; z), f(a, b; r) = a r / (1 + b r),
//              x = r_ai, y = r_aj, z = r_ij, summed over atoms and ordered pairs with 1/2,
//              i.e. G(x, y, z) = (K_een(x, y, z) + K_een(y, x, z)) / 2 per unordered pair;
//   grad_i += G_x u_ai + G_z u_ij,  grad_j += G_y u_aj - G_z u_ij,
//   lap_i  += G_xx + 2 G_x / x + G_zz + 2 G_z / z + 2 G_xz (u_ai . u_ij),
//   lap_j  += G_yy + 2 G_y / y + G_zz + 2 G_z / z - 2 G_yz (u_aj . u_ij).
//
// FP64 form: everything in double.  Other forms: positions are split into
// float pairs (hi + lo, integer operations only), pair differences
// (hi_i - hi_j) + (lo_i - lo_j) keep 2^-24 relative accuracy even for close
// pairs, pair terms are FP32 and the sums J, V, kinJ are carried as
// compensated (Kahan) FP32 pairs; on GB300 the FP64 pipe runs at 1/64 of the
// FP32 rate, so this kernel issues no FP64 instruction until the three final
// sums are widened.
#pragma once

#include "qmc_internal.cuh"

namespace qmc {

// f(a, b; r) = a r / (1 + b r) and its first two derivatives
template <typename T>
__device__ __forceinline__ void rational3(T a, T b, T r, T& f, T& f1, T& f2) {
  const T id = T(1) / (T(1) + b * r);
  f1 = a * id * id;
  f = a * r * id;
  f2 = T(-2) * b * f1 * id;
}

// Many-body Jastrow contributions (App. D) of one walker.  disp_en(i, a, v)
// writes r_i - R_a, disp_ee(i, j, v) writes r_i - r_j, both in T; par_en
// [3] and par_een [n_een][7] are the kernel parameters in T; J and lap are
// accumulators with add(T); g [NMAX][3] the electron gradients.
template <typename T, int NMAX, typename DispEn, typename DispEe, typename Acc>
__device__ __forceinline__ void manybody_terms(const WfDev& wf, const T* par_en, const T (*par_een)[7], int n,
                                               DispEn disp_en, DispEe disp_ee, Acc& J, Acc& lap, T (&g)[NMAX][3],
                                               bool deriv) {
  for (int a = 0; a < wf.n_atom; ++a) {
    if (wf.mb_en) {
      const T w0 = par_en[0], w1 = par_en[1], w2 = par_en[2];
#pragma unroll
      for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
          T v[3];
          disp_en(i, a, v);
          const T r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
          const T ir = T(1) / sqrt(r2), r = r2 * ir;
          const T id = T(1) / (T(1) + w2 * r);
          J.add((w0 * r + w1 * r * r) * id);
          if (deriv) {
            const T k1 = (w0 + T(2) * w1 * r + w1 * w2 * r * r) * id * id;
            const T k2 = T(2) * (w1 - w0 * w2) * id * id * id;
            lap.add(k2 + T(2) * k1 * ir);
            const T s = k1 * ir;
            g[i][0] += s * v[0]; g[i][1] += s * v[1]; g[i][2] += s * v[2];
          }
        }
      }
    }
    if (wf.n_een == 0) continue;
    // runtime pair loop (the electron gradients go to local memory in this
    // variant; fully unrolled triplet sums cost minutes of compile time)
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
#pragma unroll 1
      for (int j = i + 1; j < n; ++j) {
        {
          T vi[3], vj[3], vij[3];
          disp_en(i, a, vi);
          disp_en(j, a, vj);
          disp_ee(i, j, vij);
          const T x2 = vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2];
          const T y2 = vj[0] * vj[0] + vj[1] * vj[1] + vj[2] * vj[2];
          const T z2 = vij[0] * vij[0] + vij[1] * vij[1] + vij[2] * vij[2];
          const T ix = T(1) / sqrt(x2), iy = T(1) / sqrt(y2), iz = T(1) / sqrt(z2);
          const T x = x2 * ix, y = y2 * iy, z = z2 * iz;
          T G = T(0), Gx = T(0), Gy = T(0), Gz = T(0), Gxx = T(0), Gyy = T(0), Gzz = T(0), Gxz = T(0), Gyz = T(0);
          for (int t = 0; t < wf.n_een; ++t) {
            const T c = T(0.5) * par_een[t][0];
            T p1x, p1x1, p1x2, p2y, p2y1, p2y2, p1y, p1y1, p1y2, p2x, p2x1, p2x2, q, q1, q2;
            rational3(par_een[t][1], par_een[t][2], x, p1x, p1x1, p1x2);
            rational3(par_een[t][3], par_een[t][4], y, p2y, p2y1, p2y2);
            rational3(par_een[t][1], par_een[t][2], y, p1y, p1y1, p1y2);
            rational3(par_een[t][3], par_een[t][4], x, p2x, p2x1, p2x2);
            rational3(par_een[t][5], par_een[t][6], z, q, q1, q2);
            const T P = p1x * p2y + p1y * p2x;  // symmetrised in x and y
            const T Px = p1x1 * p2y + p1y * p2x1, Py = p1x * p2y1 + p1y1 * p2x;
            G += c * P * q;
            if (deriv) {
              Gx += c * Px * q;
              Gy += c * Py * q;
              Gz += c * P * q1;
              Gxx += c * (p1x2 * p2y + p1y * p2x2) * q;
              Gyy += c * (p1x * p2y2 + p1y2 * p2x) * q;
              Gzz += c * P * q2;
              Gxz += c * Px * q1;
              Gyz += c * Py * q1;
            }
          }
          J.add(G);
          if (deriv) {
            T ui[3], uj[3], u[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) { ui[d] = vi[d] * ix; uj[d] = vj[d] * iy; u[d] = vij[d] * iz; }
            const T cij = ui[0] * u[0] + ui[1] * u[1] + ui[2] * u[2];
            const T cji = uj[0] * u[0] + uj[1] * u[1] + uj[2] * u[2];
            lap.add(Gxx + T(2) * Gx * ix + Gyy + T(2) * Gy * iy + T(2) * (Gzz + T(2) * Gz * iz) +
                    T(2) * (Gxz * cij - Gyz * cji));
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              g[i][d] += Gx * ui[d] + Gz * u[d];
              g[j][d] += Gy * uj[d] - Gz * u[d];
            }
          }
        }
      }
    }
  }
}

struct PlainD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
};

template <int NMAX, bool MB>
__global__ void __launch_bounds__(128) k_jastrow_f64(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                     int64_t ldw, double* __restrict__ gradJ,
                                                     double* __restrict__ jscal, int64_t ldm, bool deriv) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int n = wf.n_elec;
  double r[NMAX][3], g[NMAX][3];
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      r[i][d] = (i < n) ? walkers[(int64_t)(3 * i + d) * ldw + w] : 0.0;
      g[i][d] = 0.0;
    }
  double J = 0.0, lap = 0.0, V = wf.vnn;
  const double b = wf.jb;
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
#pragma unroll
    for (int j = i + 1; j < NMAX; ++j) {
      if (j < n) {
        const double dx = r[i][0] - r[j][0], dy = r[i][1] - r[j][1], dz = r[i][2] - r[j][2];
        const double d2 = dx * dx + dy * dy + dz * dz;
        const double inv = 1.0 / sqrt(d2);
        const double dist = d2 * inv;
        const double w0 = ((i < wf.n_up) == (j < wf.n_up)) ? wf.w0_par : wf.w0_anti;
        const double rden = 1.0 / (1.0 + b * dist);
        const double u1 = w0 * rden * rden;
        J += w0 * dist * rden;
        V += inv;
        if (deriv) {
          lap += 2.0 * (-2.0 * b * u1 * rden + 2.0 * u1 * inv);
          const double s = u1 * inv;
          g[i][0] += s * dx; g[i][1] += s * dy; g[i][2] += s * dz;
          g[j][0] -= s * dx; g[j][1] -= s * dy; g[j][2] -= s * dz;
        }
      }
    }
  }
  for (int a = 0; a < wf.n_atom; ++a) {
    double va = 0.0;
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < n) {
        const double dx = r[i][0] - wf.atom_xyz[a][0], dy = r[i][1] - wf.atom_xyz[a][1],
                     dz = r[i][2] - wf.atom_xyz[a][2];
        va += 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
      }
    V -= wf.atom_z[a] * va;
  }
  if (MB) {
    PlainD Jm, lm;
    auto disp_en = [&](int i, int a, double* v) {
      for (int d = 0; d < 3; ++d) v[d] = r[i][d] - wf.atom_xyz[a][d];
    };
    auto disp_ee = [&](int i, int j, double* v) {
      for (int d = 0; d < 3; ++d) v[d] = r[i][d] - r[j][d];
    };
    manybody_terms<double, NMAX>(wf, wf.jen, wf.jeen, n, disp_en, disp_ee, Jm, lm, g, deriv);
    J += Jm.s;
    lap += lm.s;
  }
  double kin = lap;
  if (deriv) {
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < n)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          kin += g[i][d] * g[i][d];
          gradJ[(int64_t)(3 * i + d) * ldm + w] = g[i][d];
        }
  }
  jscal[w] = J;
  jscal[ldm + w] = kin;
  jscal[2 * ldm + w] = V;
}

// compensated FP32 accumulator
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int NMAX, bool MB>
__global__ void __launch_bounds__(128) k_jastrow_f32(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                     int64_t ldw, float* __restrict__ gradJ,
                                                     double* __restrict__ jscal, int64_t ldm, float b, float w0p,
                                                     float w0a, bool deriv) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int n = wf.n_elec;
  float rh[NMAX][3], rl[NMAX][3], g[NMAX][3];
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (i < n) split_f64(walkers[(int64_t)(3 * i + d) * ldw + w], rh[i][d], rl[i][d]);
      else { rh[i][d] = 0.f; rl[i][d] = 0.f; }
      g[i][d] = 0.f;
    }
  KahanF J, V, lap;
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
#pragma unroll
    for (int j = i + 1; j < NMAX; ++j) {
      if (j < n) {
        const float dx = (rh[i][0] - rh[j][0]) + (rl[i][0] - rl[j][0]);
        const float dy = (rh[i][1] - rh[j][1]) + (rl[i][1] - rl[j][1]);
        const float dz = (rh[i][2] - rh[j][2]) + (rl[i][2] - rl[j][2]);
        const float d2 = dx * dx + dy * dy + dz * dz;
        const float inv = 1.0f / sqrtf(d2);
        const float dist = d2 * inv;
        const float w0 = ((i < wf.n_up) == (j < wf.n_up)) ? w0p : w0a;
        const float rden = 1.0f / (1.0f + b * dist);
        const float u1 = w0 * rden * rden;
        J.add(w0 * dist * rden);
        V.add(inv);
        if (deriv) {
          lap.add(2.0f * (-2.0f * b * u1 * rden + 2.0f * u1 * inv));
          const float s = u1 * inv;
          g[i][0] += s * dx; g[i][1] += s * dy; g[i][2] += s * dz;
          g[j][0] -= s * dx; g[j][1] -= s * dy; g[j][2] -= s * dz;
        }
      }
    }
  }
  for (int a = 0; a < wf.n_atom; ++a) {
    float ah[3], al[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) split_f64(wf.atom_xyz[a][d], ah[d], al[d]);
    float zh, zl;
    split_f64(wf.atom_z[a], zh, zl);
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < n) {
        const float dx = (rh[i][0] - ah[0]) + (rl[i][0] - al[0]);
        const float dy = (rh[i][1] - ah[1]) + (rl[i][1] - al[1]);
        const float dz = (rh[i][2] - ah[2]) + (rl[i][2] - al[2]);
        V.add(-zh / sqrtf(dx * dx + dy * dy + dz * dz));
      }
  }
  if (MB) {
    auto disp_en = [&](int i, int a, float* v) {
      for (int d = 0; d < 3; ++d) {
        float ah, al;
        split_f64(wf.atom_xyz[a][d], ah, al);
        v[d] = (rh[i][d] - ah) + (rl[i][d] - al);
      }
    };
    auto disp_ee = [&](int i, int j, float* v) {
      for (int d = 0; d < 3; ++d) v[d] = (rh[i][d] - rh[j][d]) + (rl[i][d] - rl[j][d]);
    };
    manybody_terms<float, NMAX>(wf, wf.jen_f, wf.jeen_f, n, disp_en, disp_ee, J, lap, g, deriv);
  }
  if (deriv) {
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
      if (i < n)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          lap.add(g[i][d] * g[i][d]);
          gradJ[(int64_t)(3 * i + d) * ldm + w] = g[i][d];
        }
  }
  jscal[w] = J.value();
  jscal[ldm + w] = lap.value();
  jscal[2 * ldm + w] = V.value() + wf.vnn;
}

// Launch one kernel instance; NM is the electron-count bracket.
template <int NM, bool MB>
cudaError_t launch_jastrow_nm(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                              const Workspace& ws, bool derivs, cudaStream_t st) {
  const dim3 block(128), grid((unsigned)((W + 127) / 128));
  if (prec == QMC_FP64)
    k_jastrow_f64<NM, MB><<<grid, block, 0, st>>>(wf, walkers, W, ldw, static_cast<double*>(ws.gradJ), ws.jscal,
                                                  ws.ldm, derivs);
  else
    k_jastrow_f32<NM, MB><<<grid, block, 0, st>>>(wf, walkers, W, ldw, static_cast<float*>(ws.gradJ), ws.jscal,
                                                  ws.ldm, wf.jb_f, wf.w0p_f, wf.w0a_f, derivs);
  return cudaGetLastError();
}

}  // namespace qmc
