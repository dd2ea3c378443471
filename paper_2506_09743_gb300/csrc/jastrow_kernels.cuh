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
// compensated (Kahan) FP32 pairs; on GB300 the FP64 pipe runs at about 1/62 of the
// FP32 rate, so this kernel issues no FP64 instruction until the three final
// sums are widened.
#pragma once

#include <type_traits>

#include "ao_eval.cuh"
#include "qmc_internal.cuh"

namespace qmc {

// 1 / d: IEEE division in FP64; the correctly rounded reciprocal in FP32
// (one reciprocal instead of a division per kernel evaluation)
__device__ __forceinline__ double recip_t(double d) { return 1.0 / d; }
__device__ __forceinline__ float recip_t(float d) { return __frcp_rn(d); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// f(a, b; r) = a r / (1 + b r) and its first two derivatives
template <typename T>
__device__ __forceinline__ void rational3(T a, T b, T r, T& f, T& f1, T& f2) {
  const T id = recip_t(T(1) + b * r);
  f1 = a * id * id;
  f = a * r * id;
  f2 = T(-2) * b * f1 * id;
}

// Electron-nucleus Jastrow kernel (App. D) of one walker.  disp_en(i, a, v)
// writes r_i - R_a in T; par_en [3] are (w0, w1, w2) in T; J and lap are
// accumulators with add(T); g [NMAX][3] the electron gradients.  (The
// electron-electron-nucleus terms run in k_jastrow_een, after this stage.)
template <typename T, int NMAX, typename DispEn, typename Acc>
__device__ __forceinline__ void en_terms(const WfDev& wf, const T* par_en, int n, DispEn disp_en, Acc& J, Acc& lap,
                                         T (&g)[NMAX][3], bool deriv) {
  if (!wf.mb_en) return;
  const T w0 = par_en[0], w1 = par_en[1], w2 = par_en[2];
  for (int a = 0; a < wf.n_atom; ++a) {
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
}

// Electron positions as kept in shared memory by k_jastrow_een: plain in
// FP64, float pairs hi + lo (integer splitting only) in FP32.
struct EenPosD {
  double x[3];
};
struct EenPosF {
  float h[3], l[3];
};
__device__ __forceinline__ EenPosD een_pos(const double* r, double) { return EenPosD{{r[0], r[1], r[2]}}; }
__device__ __forceinline__ EenPosF een_pos(const double* r, float) {
  EenPosF p;
  for (int d = 0; d < 3; ++d) split_f64(r[d], p.h[d], p.l[d]);
  return p;
}
__device__ __forceinline__ void een_diff(const EenPosD& a, const EenPosD& b, double* v) {
  for (int d = 0; d < 3; ++d) v[d] = a.x[d] - b.x[d];
}
__device__ __forceinline__ void een_diff(const EenPosF& a, const EenPosF& b, float* v) {
  for (int d = 0; d < 3; ++d) v[d] = (a.h[d] - b.h[d]) + (a.l[d] - b.l[d]);
}

// Electron-electron-nucleus Jastrow terms (App. D), added to the outputs of
// the Jastrow stage.  Sixteen lanes per walker (N <= 16), kEenWalkers walkers
// per block.
//  1. lane e tabulates, for its electron and every atom a, the distance x =
//     r_ae, its unit vector u_ae and, per term, f(a1, b1; x) and f(a2, b2; x)
//     with their first two derivatives (f(a, b; r) = a r / (1 + b r));
//  2. the unordered pairs (i < j) are dealt to the lanes; per pair the lane
//     forms z = r_ij and the terms' f(a3, b3; z) once, and per atom the
//     symmetrised kernel
//       G(x, y, z) = (K_een(x, y, z) + K_een(y, x, z)) / 2,  x = r_ai, y = r_aj,
//     from the tables, with both electrons' derivatives:
//       grad_i += G_x u_ai + G_z u_ij,   grad_j += G_y u_aj - G_z u_ij,
//       lap_i  += G_xx + 2 G_x / x + G_zz + 2 G_z / z + 2 G_xz (u_ai . u_ij),
//       lap_j  += G_yy + 2 G_y / y + G_zz + 2 G_z / z - 2 G_yz (u_aj . u_ij),
//       J      += G;
//  3. lane e gathers its electron's pair terms in a fixed pair order
//     (deterministic sums).  The electron's total gradient is grad J (Pade and
//     electron-nucleus parts, already written) plus this part, so kinJ gains
//     lap_e + 2 g0 . g + |g|^2; the lane sums of a walker are reduced by
//     shuffles in a fixed order and added by one lane.
constexpr int kEenWalkers = 4;
constexpr int kEenMaxPairs = 120;  // 16 x 15 / 2

// shared-memory layout of k_jastrow_een (dynamic part), in elements of T.
// The tables are read as two-element vectors; their electron stride is 2
// (mod 4) elements, so that the 16 lanes of a walker reading 16 different
// electrons hit distinct banks.
struct EenLayout {
  int per_ea;    // values per (electron, atom): x, 1/x, u (3), a pad, then 6 per term
  int per_e;     // per electron: n_atom x per_ea, rounded up to 2 (mod 4)
  int per_walk;  // per walker: n x per_e
  int np_pad;    // pair stride of the two-sided pair terms, = 2 (mod 4): the
                 // two walkers of a warp write opposite halves of the banks
  int pair_walk; // per walker: 8 x np_pad (value-major [8][np_pad])
  __host__ __device__ EenLayout(int n, int n_atom, int n_een)
      : per_ea(6 + 6 * n_een),
        per_e(n_atom * per_ea + ((n_atom * per_ea) % 4 == 0 ? 2 : 0)),
        per_walk(n * per_e),
        np_pad(((n * (n - 1) / 2 + 1) / 4) * 4 + 2),
        pair_walk(8 * np_pad) {}
};

// 2 K consecutive table values as K two-element vector loads (p is aligned to
// two elements)
template <int K>
__device__ __forceinline__ void ld_vec2(const float* p, float* v) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 q = reinterpret_cast<const float2*>(p)[k];
    v[2 * k] = q.x;
    v[2 * k + 1] = q.y;
  }
}
template <int K>
__device__ __forceinline__ void ld_vec2(const double* p, double* v) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double2 q = reinterpret_cast<const double2*>(p)[k];
    v[2 * k] = q.x;
    v[2 * k + 1] = q.y;
  }
}
template <typename T>
size_t een_smem_bytes(const WfDev& wf) {
  const EenLayout L(wf.n_elec, wf.n_atom, wf.n_een);
  return sizeof(T) * (size_t)kEenWalkers * (L.per_walk + L.pair_walk);
}

template <typename T>
__global__ void __launch_bounds__(16 * kEenWalkers) k_jastrow_een(WfDev wf, const double* __restrict__ walkers,
                                                                  int64_t W, int64_t ldw, T* __restrict__ gradJ,
                                                                  double* __restrict__ jscal, int64_t ldm, bool deriv) {
  using Pos = decltype(een_pos((const double*)nullptr, T(0)));
  __shared__ Pos pos_s[kEenWalkers][16];
  __shared__ Pos atom_s[QMC_MAX_ATOMS];
  __shared__ T par_s[kMaxEen][7];
  __shared__ unsigned char pair_i[kEenMaxPairs], pair_j[kEenMaxPairs], pair_of[16][16];
  extern __shared__ __align__(16) unsigned char een_raw[];
  const int n = wf.n_elec, na = wf.n_atom, nt = wf.n_een;
  const EenLayout L(n, na, nt);
  T* tab_all = reinterpret_cast<T*>(een_raw);                         // [kEenWalkers][per_walk]
  T* contrib_all = tab_all + (size_t)kEenWalkers * L.per_walk;        // [kEenWalkers][2][4][np_pad]
  const T* par_src = std::is_same<T, double>::value ? reinterpret_cast<const T*>(&wf.jeen[0][0])
                                                     : reinterpret_cast<const T*>(&wf.jeen_f[0][0]);
  const int grp = threadIdx.x >> 4, lane = threadIdx.x & 15;
  const int n_pairs = n * (n - 1) / 2;
  const int64_t w = (int64_t)blockIdx.x * kEenWalkers + grp;
  const bool wl = w < W;
  T* tab = tab_all + (size_t)grp * L.per_walk;
  T* contrib = contrib_all + (size_t)grp * L.pair_walk;
  if (wl && lane < n) {
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = walkers[(int64_t)(3 * lane + d) * ldw + w];
    pos_s[grp][lane] = een_pos(r, T(0));
  }
  if (threadIdx.x < na) atom_s[threadIdx.x] = een_pos(wf.atom_xyz[threadIdx.x], T(0));
  for (int k = threadIdx.x; k < nt * 7; k += blockDim.x) par_s[k / 7][k % 7] = par_src[k];
  if (threadIdx.x < n) {  // pair numbering: (0,1), (0,2), ..., (1,2), ...
    const int i = threadIdx.x;
    for (int j = i + 1; j < n; ++j) {
      const int k = i * n - i * (i + 1) / 2 + (j - i - 1);
      pair_i[k] = (unsigned char)i;
      pair_j[k] = (unsigned char)j;
      pair_of[i][j] = pair_of[j][i] = (unsigned char)k;
    }
  }
  __syncthreads();
  // ---- 1. electron-atom tables
  if (wl && lane < n) {
    const Pos pe = pos_s[grp][lane];
    for (int a = 0; a < na; ++a) {
      T v[3];
      een_diff(pe, atom_s[a], v);
      const T x2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      const T ix = rsqrt_t(x2), x = x2 * ix;
      T* e = tab + lane * L.per_e + a * L.per_ea;
      e[0] = x;
      e[1] = ix;
      for (int d = 0; d < 3; ++d) e[2 + d] = v[d] * ix;
      e[5] = T(0);
      for (int t = 0; t < nt; ++t) {
        rational3(par_s[t][1], par_s[t][2], x, e[6 + 6 * t], e[7 + 6 * t], e[8 + 6 * t]);
        rational3(par_s[t][3], par_s[t][4], x, e[9 + 6 * t], e[10 + 6 * t], e[11 + 6 * t]);
      }
    }
  }
  __syncthreads();
  // ---- 2. pairs
  T jv = T(0);
  if (wl) {
    for (int k = lane; k < n_pairs; k += 16) {
      const int i = pair_i[k], j = pair_j[k];
      T vij[3];
      een_diff(pos_s[grp][i], pos_s[grp][j], vij);
      const T z2 = vij[0] * vij[0] + vij[1] * vij[1] + vij[2] * vij[2];
      const T iz = rsqrt_t(z2), z = z2 * iz;
      T u[3];
      for (int d = 0; d < 3; ++d) u[d] = vij[d] * iz;
      T ci[4] = {T(0), T(0), T(0), T(0)}, cj[4] = {T(0), T(0), T(0), T(0)};
      T qz[kMaxEen][3];  // c / 2 times f(a3, b3; z) and its derivatives, per term
#pragma unroll
      for (int t = 0; t < kMaxEen; ++t)
        if (t < nt) {
          rational3(par_s[t][5], par_s[t][6], z, qz[t][0], qz[t][1], qz[t][2]);
          const T c = T(0.5) * par_s[t][0];
          qz[t][0] *= c;
          qz[t][1] *= c;
          qz[t][2] *= c;
        }
      for (int a = 0; a < na; ++a) {
        const T* ei = tab + i * L.per_e + a * L.per_ea;
        const T* ej = tab + j * L.per_e + a * L.per_ea;
        T G = T(0), Gx = T(0), Gy = T(0), Gz = T(0), Gxx = T(0), Gyy = T(0), Gzz = T(0), Gxz = T(0), Gyz = T(0);
#pragma unroll
        for (int t = 0; t < kMaxEen; ++t) {
          if (t >= nt) break;
          const T q = qz[t][0], q1 = qz[t][1], q2 = qz[t][2];
          T fi[6], fj[6];  // f1(x), f1', f1'', f2(x), f2', f2''; the same at y
          ld_vec2<3>(ei + 6 + 6 * t, fi);
          ld_vec2<3>(ej + 6 + 6 * t, fj);
          const T P = fi[0] * fj[3] + fj[0] * fi[3];  // symmetrised in x and y
          const T Px = fi[1] * fj[3] + fj[0] * fi[4], Py = fi[0] * fj[4] + fj[1] * fi[3];
          G += P * q;
          if (deriv) {
            Gx += Px * q;
            Gy += Py * q;
            Gz += P * q1;
            Gxx += (fi[2] * fj[3] + fj[0] * fi[5]) * q;
            Gyy += (fi[0] * fj[5] + fj[2] * fi[3]) * q;
            Gzz += P * q2;
            Gxz += Px * q1;
            Gyz += Py * q1;
          }
        }
        jv += G;
        if (deriv) {
          T hi[6], hj[6];  // x, 1/x, u (3), pad
          ld_vec2<3>(ei, hi);
          ld_vec2<3>(ej, hj);
          const T ix = hi[1], iy = hj[1];
          const T cij = hi[2] * u[0] + hi[3] * u[1] + hi[4] * u[2];
          const T cji = hj[2] * u[0] + hj[3] * u[1] + hj[4] * u[2];
          for (int d = 0; d < 3; ++d) {
            ci[d] += Gx * hi[2 + d] + Gz * u[d];
            cj[d] += Gy * hj[2 + d] - Gz * u[d];
          }
          ci[3] += Gxx + T(2) * Gx * ix + Gzz + T(2) * Gz * iz + T(2) * Gxz * cij;
          cj[3] += Gyy + T(2) * Gy * iy + Gzz + T(2) * Gz * iz - T(2) * Gyz * cji;
        }
      }
      if (deriv)
        for (int q = 0; q < 4; ++q) {
          contrib[q * L.np_pad + k] = ci[q];
          contrib[(4 + q) * L.np_pad + k] = cj[q];
        }
    }
  }
  __syncthreads();
  // ---- 3. per-electron gather
  T corr = T(0);
  if (deriv && wl && lane < n) {
    const int e = lane;
    T g[4] = {T(0), T(0), T(0), T(0)};
    for (int o = 0; o < n; ++o) {
      if (o == e) continue;
      const int k = pair_of[e][o], side = e < o ? 0 : 4;
      for (int q = 0; q < 4; ++q) g[q] += contrib[(side + q) * L.np_pad + k];
    }
    T* g0p = gradJ + (int64_t)(3 * e) * ldm + w;
    const T g0x = g0p[0], g0y = g0p[ldm], g0z = g0p[2 * ldm];
    g0p[0] = g0x + g[0];
    g0p[ldm] = g0y + g[1];
    g0p[2 * ldm] = g0z + g[2];
    corr = g[3] + T(2) * (g0x * g[0] + g0y * g[1] + g0z * g[2]) + (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    jv += __shfl_xor_sync(0xffffffffu, jv, o);
    corr += __shfl_xor_sync(0xffffffffu, corr, o);
  }
  if (lane == 0 && wl) {
    jscal[w] += widen(jv);
    if (deriv) jscal[ldm + w] += widen(corr);
  }
}

struct PlainD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
};

template <int NMAX, bool MB>
__global__ void __launch_bounds__(128) k_jastrow_f64(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                     int64_t ldw, double* __restrict__ copy,
                                                     double* __restrict__ gradJ, double* __restrict__ jscal,
                                                     int64_t ldm, bool deriv) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int n = wf.n_elec;
  double r[NMAX][3], g[NMAX][3];
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      r[i][d] = (i < n) ? walkers[(int64_t)(3 * i + d) * ldw + w] : 0.0;
      if (copy && i < n) copy[(int64_t)(3 * i + d) * ldw + w] = r[i][d];
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
    en_terms<double, NMAX>(wf, wf.jen, n, disp_en, Jm, lm, g, deriv);
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

// r_i - r_j (d) of two positions held as float pairs, as a pair
// (the low words' difference is formed exactly too: near a nucleus, where
// |a - b| is far below |a|, rounding it would cost 2^-48 |a| absolute, a
// relative error of 2^-48 |a| / |a - b| in 1 / |a - b|)
__device__ __forceinline__ f32x2 pair_diff_x2(float ah, float al, float bh, float bl) {
  const f32x2 s = two_sum(ah, -bh);
  const f32x2 t = two_sum(al, -bl);
  const f32x2 u = two_sum(s.hi, t.hi);
  return fast_two_sum(u.hi, x2_add_rn(u.lo, x2_add_rn(s.lo, t.lo)));
}
// 1 / |v| of a difference vector given as pairs
__device__ __forceinline__ f32x2 inv_dist_x2(f32x2 x, f32x2 y, f32x2 z) { return rsqrt_x2(x * x + y * y + z * z); }

// VX2 (the QMC_FP32X2 form): the electron-nucleus potential is summed in
// pairs of FP32 (Z/r_ia grows without bound near a nucleus, where FP32 terms
// would cost 2^-24 of several hundred Ha); the electron-electron terms are
// FP32 reciprocals refined to about one ulp and summed with compensation
// (within 2^-22 V_ee: an emulation over 100,000 CO walkers gives at most
// 4.7e-6 Ha); pairs closer than 0.01 bohr take 1/r_ij and the Jastrow
// Laplacian term 2u'/r_ij (both unbounded at coalescence) in FP64; the other
// Jastrow terms are bounded and stay FP32.
template <int NMAX, bool MB, bool VX2>
__global__ void __launch_bounds__(128) k_jastrow_f32(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                     int64_t ldw, double* __restrict__ copy,
                                                     float* __restrict__ gradJ, double* __restrict__ jscal,
                                                     int64_t ldm, float b, float w0p, float w0a, bool deriv) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int n = wf.n_elec;
  float rh[NMAX][3], rl[NMAX][3], g[NMAX][3];
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (i < n) {
        const double v = walkers[(int64_t)(3 * i + d) * ldw + w];
        if (copy) copy[(int64_t)(3 * i + d) * ldw + w] = v;
        split_f64(v, rh[i][d], rl[i][d]);
      } else {
        rh[i][d] = 0.f;
        rl[i][d] = 0.f;
      }
      g[i][d] = 0.f;
    }
  KahanF J, V, lap;
  f32x2 vx(0.f, 0.f);           // V in pairs (VX2)
  double Vd = 0.0, lapd = 0.0;  // close pairs in FP64 (VX2)
  bool any_close = false;
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
#pragma unroll
    for (int j = i + 1; j < NMAX; ++j) {
      if (j < n) {
        const float dx = (rh[i][0] - rh[j][0]) + (rl[i][0] - rl[j][0]);
        const float dy = (rh[i][1] - rh[j][1]) + (rl[i][1] - rl[j][1]);
        const float dz = (rh[i][2] - rh[j][2]) + (rl[i][2] - rl[j][2]);
        // (the order of the roundings is fixed: the close-pair pass below
        // repeats this test bit for bit)
        const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        const float inv = rsqrtf(d2);  // hardware reciprocal square root and reciprocal:
        const float dist = d2 * inv;    // a few ulp, far inside the FP32 pair-term budget
        const float w0 = ((i < wf.n_up) == (j < wf.n_up)) ? w0p : w0a;
        const float rden = __frcp_rn(1.0f + b * dist);
        const float u1 = w0 * rden * rden;
        J.add(w0 * dist * rden);
        // FP32X2: electrons within 0.01 bohr (1/r_ij > 100, and the Jastrow
        // Laplacian 2u'/r_ij as large, where FP32 terms would cost 2^-22 of
        // them) are left out here and taken in FP64 after the loop
        const bool close = VX2 && d2 < 1e-4f;
        any_close |= close;
        if (VX2) {
          // 1/r_ij to about one ulp (one Newton step on the hardware
          // estimate, residual by FMA), summed with compensation: each term
          // within 2^-22 of itself, at most 2.4e-5 Ha
          const float e = fmaf(-d2 * inv, inv, 1.0f);
          V.add(close ? 0.0f : fmaf(0.5f * inv, e, inv));
        } else {
          V.add(inv);
        }
        if (deriv) {
          lap.add(close ? 0.0f : 2.0f * (-2.0f * b * u1 * rden + 2.0f * u1 * inv));
          const float s = u1 * inv;
          g[i][0] += s * dx; g[i][1] += s * dy; g[i][2] += s * dz;
          g[j][0] -= s * dx; g[j][1] -= s * dy; g[j][2] -= s * dz;
        }
      }
    }
  }
  if (VX2 && any_close) {
    // the close pairs (the same FP32 test as above, on the same splits) in
    // FP64 from the FP64 coordinates and parameters; rare (the cusp), so one
    // rolled loop over the pairs
    const double* src = copy ? copy : walkers;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        float d2 = 0.f;
        for (int d = 0; d < 3; ++d) {
          float ih, il, jh, jl;
          split_f64(src[(int64_t)(3 * i + d) * ldw + w], ih, il);
          split_f64(src[(int64_t)(3 * j + d) * ldw + w], jh, jl);
          const float v = (ih - jh) + (il - jl);
          d2 = d == 0 ? __fmul_rn(v, v) : __fmaf_rn(v, v, d2);
        }
        if (!(d2 < 1e-4f)) continue;
        double dd2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double v = src[(int64_t)(3 * i + d) * ldw + w] - src[(int64_t)(3 * j + d) * ldw + w];
          dd2 += v * v;
        }
        const double invd = 1.0 / sqrt(dd2), distd = dd2 * invd;
        const double w0d = ((i < wf.n_up) == (j < wf.n_up)) ? wf.w0_par : wf.w0_anti;
        const double rdd = 1.0 / (1.0 + wf.jb * distd), u1d = w0d * rdd * rdd;
        Vd += invd;
        if (deriv) lapd += 2.0 * (-2.0 * wf.jb * u1d * rdd + 2.0 * u1d * invd);
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
        if (VX2) {
          // r_i - R_a from the FP64 coordinates (one FP64 subtraction each,
          // exact for an electron next to the nucleus), then split: the float
          // split of a coordinate alone keeps only 2^-48 of |r_i|, which is
          // 2^-48 |r_i| / |r_i - R_a| of Z / |r_i - R_a|
          const double* src = copy ? copy : walkers;
          f32x2 dv[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) dv[d] = diff_x2(src[(int64_t)(3 * i + d) * ldw + w], wf.atom_xyz[a][d]);
          vx = vx - inv_dist_x2(dv[0], dv[1], dv[2]) * f32x2(zh, zl);
        } else {
          const float dx = (rh[i][0] - ah[0]) + (rl[i][0] - al[0]);
          const float dy = (rh[i][1] - ah[1]) + (rl[i][1] - al[1]);
          const float dz = (rh[i][2] - ah[2]) + (rl[i][2] - al[2]);
          V.add(-zh * rsqrtf(dx * dx + dy * dy + dz * dz));
        }
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
    en_terms<float, NMAX>(wf, wf.jen_f, n, disp_en, J, lap, g, deriv);
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
  jscal[ldm + w] = VX2 ? lap.value() + lapd : lap.value();
  jscal[2 * ldm + w] = (VX2 ? widen(vx) + V.value() + Vd : V.value()) + wf.vnn;
}

// Launch one kernel instance; NM is the electron-count bracket.  If copy is
// not null the kernel also writes the positions it reads there (same layout):
// walkers may then be mapped host memory, read once over the host link, and
// the later stages read the device copy.
template <int NM, bool MB>
cudaError_t launch_jastrow_nm(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                              double* copy, const Workspace& ws, bool derivs, cudaStream_t st) {
  const dim3 block(128), grid((unsigned)((W + 127) / 128));
  if (prec == QMC_FP64)
    k_jastrow_f64<NM, MB><<<grid, block, 0, st>>>(wf, walkers, W, ldw, copy, static_cast<double*>(ws.gradJ),
                                                  ws.jscal, ws.ldm, derivs);
  else if (prec == QMC_FP32X2)
    k_jastrow_f32<NM, MB, true><<<grid, block, 0, st>>>(wf, walkers, W, ldw, copy, static_cast<float*>(ws.gradJ),
                                                        ws.jscal, ws.ldm, wf.jb_f, wf.w0p_f, wf.w0a_f, derivs);
  else
    k_jastrow_f32<NM, MB, false><<<grid, block, 0, st>>>(wf, walkers, W, ldw, copy, static_cast<float*>(ws.gradJ),
                                                         ws.jscal, ws.ldm, wf.jb_f, wf.w0p_f, wf.w0a_f, derivs);
  return cudaGetLastError();
}

}  // namespace qmc
