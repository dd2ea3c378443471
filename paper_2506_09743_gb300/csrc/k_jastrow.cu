// Pade electron-electron Jastrow and Coulomb potential, one thread per walker.
//
//   J        = sum_{i<j} u(r_ij),  u(r) = w0 r / (1 + b r)   (Eqs. jastrow, pade_kernel)
//   grad_i J = sum_{j!=i} u'(r_ij) (r_i - r_j) / r_ij,  u' = w0 / (1 + b r)^2
//   kinJ     = sum_i lap_i J + |grad_i J|^2,  lap_i J = sum_j u'' + 2 u'/r_ij,
//              u'' = -2 w0 b / (1 + b r)^3                     (App. F, lap e^J / e^J)
//   V        = sum_{i<j} 1/r_ij - sum_{i,a} Z_a / r_ia + V_nn  (Eq. Hmol)
// Each pair is visited once.
//
// FP64 form: everything in double.  Other forms: positions are split into
// float pairs (hi + lo, integer operations only), pair differences
// (hi_i - hi_j) + (lo_i - lo_j) keep 2^-24 relative accuracy even for close
// pairs, pair terms are FP32 and the sums J, V, kinJ are carried as
// compensated (Kahan) FP32 pairs; on GB300 the FP64 pipe runs at 1/64 of the
// FP32 rate, so this kernel issues no FP64 instruction until the three final
// sums are widened.
#include "qmc_internal.cuh"

namespace qmc {

template <int NMAX>
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

template <int NMAX>
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

cudaError_t launch_jastrow(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                           const Workspace& ws, bool derivs, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  const dim3 block(128), grid((unsigned)((W + 127) / 128));
  const float b = (float)wf.jb, w0p = (float)wf.w0_par, w0a = (float)wf.w0_anti;
#define QMC_JAS(NM)                                                                                          \
  if (wf.n_elec <= NM) {                                                                                     \
    if (prec == QMC_FP64)                                                                                    \
      k_jastrow_f64<NM><<<grid, block, 0, st>>>(wf, walkers, W, ldw, static_cast<double*>(ws.gradJ), ws.jscal, \
                                                ws.ldm, derivs);                                             \
    else                                                                                                     \
      k_jastrow_f32<NM><<<grid, block, 0, st>>>(wf, walkers, W, ldw, static_cast<float*>(ws.gradJ), ws.jscal,  \
                                                ws.ldm, b, w0p, w0a, derivs);                                \
    return cudaGetLastError();                                                                               \
  }
  QMC_JAS(2)
  QMC_JAS(4)
  QMC_JAS(8)
  QMC_JAS(16)
#undef QMC_JAS
  return cudaErrorInvalidValue;
}

}  // namespace qmc
