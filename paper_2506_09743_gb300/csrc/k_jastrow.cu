// Pade electron-electron Jastrow and Coulomb potential, one thread per walker.
//
//   J        = sum_{i<j} u(r_ij),  u(r) = w0 r / (1 + b r)   (Eqs. jastrow, pade_kernel)
//   grad_i J = sum_{j!=i} u'(r_ij) (r_i - r_j) / r_ij
//   kinJ     = sum_i lap_i J + |grad_i J|^2                  (App. F, lap e^J / e^J)
//   V        = sum_{i<j} 1/r_ij - sum_{i,a} Z_a / r_ia + V_nn  (Eq. Hmol)
//
// Each pair is visited once.  PT is the pair arithmetic type: double in the
// FP64 form; float in the other forms, where every coordinate difference is
// still taken in double (so a close pair keeps its relative accuracy) and all
// sums of pair terms are accumulated in double.
#include "qmc_internal.cuh"

namespace qmc {

template <int NMAX, typename PT, bool DERIV>
__global__ void __launch_bounds__(128) k_jastrow(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                 int64_t ldw, PT* __restrict__ gradJ, double* __restrict__ jscal,
                                                 int64_t ldm) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int n = wf.n_elec;
  double r[NMAX][3];
  PT g[NMAX][3];
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      r[i][d] = (i < n) ? walkers[(int64_t)(3 * i + d) * ldw + w] : 0.0;
      g[i][d] = PT(0);
    }
  }
  double J = 0.0, lap = 0.0, V = wf.vnn;
  const PT b = PT(wf.jb);
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
#pragma unroll
    for (int j = i + 1; j < NMAX; ++j) {
      if (j < n) {
        const PT dx = PT(r[i][0] - r[j][0]), dy = PT(r[i][1] - r[j][1]), dz = PT(r[i][2] - r[j][2]);
        const PT d2 = dx * dx + dy * dy + dz * dz;
        const PT inv = PT(1) / sqrt(d2);
        const PT dist = d2 * inv;
        const bool same = (i < wf.n_up) == (j < wf.n_up);
        const PT w0 = PT(same ? wf.w0_par : wf.w0_anti);
        const PT rden = PT(1) / (PT(1) + b * dist);
        const PT u1 = w0 * rden * rden;
        J += double(w0 * dist * rden);
        V += double(inv);
        if (DERIV) {
          const PT u2 = PT(-2) * b * u1 * rden;
          lap += 2.0 * double(u2 + PT(2) * u1 * inv);
          const PT s = u1 * inv;
          g[i][0] += s * dx; g[i][1] += s * dy; g[i][2] += s * dz;
          g[j][0] -= s * dx; g[j][1] -= s * dy; g[j][2] -= s * dz;
        }
      }
    }
  }
  for (int a = 0; a < wf.n_atom; ++a) {
    double va = 0.0;
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
      if (i < n) {
        const PT dx = PT(r[i][0] - wf.atom_xyz[a][0]), dy = PT(r[i][1] - wf.atom_xyz[a][1]),
                 dz = PT(r[i][2] - wf.atom_xyz[a][2]);
        va += double(PT(1) / sqrt(dx * dx + dy * dy + dz * dz));
      }
    }
    V -= wf.atom_z[a] * va;
  }
  double kin = lap;
  if (DERIV) {
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
      if (i < n) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          kin += double(g[i][d]) * double(g[i][d]);
          gradJ[(int64_t)(3 * i + d) * ldm + w] = g[i][d];
        }
      }
    }
  }
  jscal[w] = J;
  jscal[ldm + w] = kin;
  jscal[2 * ldm + w] = V;
}

template <typename PT>
static cudaError_t launch_t(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                            bool derivs, cudaStream_t st) {
  const dim3 block(128), grid((unsigned)((W + 127) / 128));
  PT* gj = static_cast<PT*>(ws.gradJ);
#define QMC_JAS(NM)                                                                                     \
  if (wf.n_elec <= NM) {                                                                                \
    if (derivs) k_jastrow<NM, PT, true><<<grid, block, 0, st>>>(wf, walkers, W, ldw, gj, ws.jscal, ws.ldm); \
    else k_jastrow<NM, PT, false><<<grid, block, 0, st>>>(wf, walkers, W, ldw, gj, ws.jscal, ws.ldm);       \
    return cudaGetLastError();                                                                          \
  }
  QMC_JAS(2)
  QMC_JAS(4)
  QMC_JAS(8)
  QMC_JAS(16)
#undef QMC_JAS
  return cudaErrorInvalidValue;
}

cudaError_t launch_jastrow(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                           const Workspace& ws, bool derivs, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  return prec == QMC_FP64 ? launch_t<double>(wf, walkers, W, ldw, ws, derivs, st)
                          : launch_t<float>(wf, walkers, W, ldw, ws, derivs, st);
}

}  // namespace qmc
