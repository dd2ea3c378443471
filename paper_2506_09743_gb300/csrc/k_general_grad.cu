// Nuclear forces (Eq. force, forward tangents) and the parameter gradient of
// log|Psi| (Eq. nabla_loss) on the general FP64 path; the shared device
// code is in general_eval.cuh.
#include "general_eval.cuh"

namespace qmc {

// Forces, Eq. force: per walker the tangents of E_L and log|Psi| along the
// three coordinates of nucleus `atom` (forward mode), combined as
//   f = -(d E_L + (E_L - E_v) 2 d log|Psi|) / M
// and summed per block in a fixed order.  With raw = true the kernel keeps
// the three sums the estimator is assembled from instead (sharded batches):
//   sum d E_L,  sum d ln rho,  sum E_L d ln rho      (ln rho = 2 log|Psi|)
// in rows q * 3 n_atom + 3 atom + c, q = 0, 1, 2.
template <int NE, int NO>
__global__ void __launch_bounds__(128) k_forces(WfDev wf, const double* __restrict__ walkers, int64_t W, int64_t ldw,
                                                const double* __restrict__ e_loc, const double* __restrict__ stats,
                                                double* __restrict__ partial, bool raw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GenShared g;
  stage_tables(wf, g, smem_raw);
  __shared__ double red[9][128];
  const int atom = blockIdx.y;
  const int nq = raw ? 9 : 3;
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double f[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (w < W) {
    double r[NE][3];
    load_walker<NE>(walkers, ldw, w, wf.n_elec, r);
    Dual<3> R[QMC_MAX_ATOMS][3];
    for (int a = 0; a < wf.n_atom; ++a)
      for (int c = 0; c < 3; ++c) {
        R[a][c] = Dual<3>(wf.atom_xyz[a][c]);
        if (a == atom) R[a][c].d[c] = 1.0;
      }
    Dual<3> e, lp;
    eval_walker<Dual<3>, NE, NO>(wf, g, r, R, true, e, lp, atom);
    if (raw) {
      const double el = e_loc[w];
      for (int c = 0; c < 3; ++c) {
        f[c] = e.d[c];
        f[3 + c] = 2.0 * lp.d[c];
        f[6 + c] = el * 2.0 * lp.d[c];
      }
    } else {
      const double M = (double)W, de = e_loc[w] - stats[0];
      for (int c = 0; c < 3; ++c) f[c] = -(e.d[c] + de * 2.0 * lp.d[c]) / M;
    }
  }
  for (int q = 0; q < nq; ++q) red[q][threadIdx.x] = f[q];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int q = 0; q < nq; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < nq; ++q) {
      const size_t row = (size_t)(q / 3) * 3 * wf.n_atom + (size_t)atom * 3 + q % 3;
      partial[row * gridDim.x + blockIdx.x] = red[q][0];
    }
}

// Parameter gradient of log|Psi| per walker (reverse mode written out), weighted
// by 2 (E_L - E_v) / M (Eq. nabla_loss) and summed per block in a fixed order.
//   d log|Psi| / d C_{b,m}   = sum_{i in spin s, m < n_s} phi_b(r~_i) (A_s^-1)_{m i}
//   d log|Psi| / d zeta_p    = sum_i d phi_b(r~_i)/d zeta_p sum_m C_{b,m} (A^-1)_{m i}
//        STO: d phi / d zeta = phi ((n + 1/2)/zeta - rho);
//        GTO: d phi / d alpha_p = (prim p term) ((3/4 + l/2)/alpha_p - rho^2)
//   d log|Psi| / d d_0       = 1 / d_0
//   d log|Psi| / d b         = -sum_{i<j} w0 r_ij^2 / (1 + b r_ij)^2
//   d log|Psi| / d w         = sum_i sum_m (A^-1)_{m i} grad phi_m(r~_i) . sum_{j!=i} (r_i - r_j)/r_ij
//
// weight selects the per-walker factor: 0 the estimator's 2 (E_L - E_v) / M,
// 1 one (sum d log|Psi|), 2 E_L (sum E_L d log|Psi|): the raw sums of a
// sharded batch.
template <int NE, int NO>
__global__ void __launch_bounds__(128) k_grad_logpsi(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                     int64_t ldw, const double* __restrict__ e_loc,
                                                     const double* __restrict__ stats, const double* __restrict__ ang,
                                                     const int* __restrict__ prim_start, int n_param,
                                                     double* __restrict__ partial, int weight) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GenShared g;
  stage_tables(wf, g, smem_raw);
  const size_t tab_bytes = (sizeof(ShellDev) * wf.n_shell + sizeof(int) * wf.n_ao + 15) & ~size_t(15);
  double* acc = reinterpret_cast<double*>(smem_raw + tab_bytes);  // [n_param][blockDim]
  const int T = blockDim.x, tid = threadIdx.x;
  for (int k = 0; k < n_param; ++k) acc[(size_t)k * T + tid] = 0.0;
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n_prim = prim_start[wf.n_ao];
  const int off_c = n_prim, off_d = off_c + wf.n_ao * wf.n_mo, off_b = off_d + wf.n_det, off_w = off_b + 1;
  if (w < W) {
    const int N = wf.n_elec, nu = wf.n_up;
    const double M = (double)W;
    const double wt = weight == 0 ? 2.0 * (e_loc[w] - stats[0]) / M : weight == 1 ? 1.0 : e_loc[w];
    double r[NE][3];
    load_walker<NE>(walkers, ldw, w, N, r);
    Pairs<NE> P;
    pair_geometry<NE>(r, N, P);
    double rt[NE][3], drt[NE][3];
    for (int i = 0; i < N; ++i)
      for (int d = 0; d < 3; ++d) {
        double a = 0.0;
        for (int j = 0; j < N; ++j)
          if (j != i) a += P.inv[i][j] * (r[i][d] - r[j][d]);
        drt[i][d] = a;
        rt[i][d] = r[i][d] + wf.bf_w * a;
      }
    const int n_occ = nu > wf.n_down ? nu : wf.n_down;
    double phi[NE][NO], dphi[NE][NO][3], hphi[NE][NO][6];
    for (int i = 0; i < N; ++i)
      mo_channels<double, NO>(wf, g, rt[i], wf.atom_xyz, n_occ, phi[i], dphi[i], hphi[i], true);
    double ainv[2][NO][NO];
    for (int s = 0; s < 2; ++s) {
      const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
      if (n == 0) continue;
      for (int a = 0; a < n; ++a)
        for (int m = 0; m < n; ++m) ainv[s][a][m] = phi[i0 + a][m];
      small_inverse<double, NO>(ainv[s], n);
    }
    // MO coefficients and exponents: loop over AOs and electrons
    for (int s = 0; s < wf.n_shell; ++s) {
      const ShellDev& sh = g.sh[s];
      for (int i = 0; i < N; ++i) {
        const int sp = i < nu ? 0 : 1, n = sp == 0 ? nu : wf.n_down, a = sp == 0 ? i : i - nu;
        const double dx = rt[i][0] - wf.atom_xyz[sh.atom][0], dy = rt[i][1] - wf.atom_xyz[sh.atom][1],
                     dz = rt[i][2] - wf.atom_xyz[sh.atom][2];
        const double r2 = dx * dx + dy * dy + dz * dz, rho = sqrt(r2);
        double f, g1, f2;
        radial(sh, r2, rho, f, g1, f2);
        for (int k = 0; k < sh.n_ao; ++k) {
          const int b = sh.ao_first + k;
          const int pw = g.pw[b];
          const double Pm = mono(dx, dy, dz, pw & 15, (pw >> 4) & 15, (pw >> 8) & 15);
          const double* Cb = g.C + (size_t)b * wf.n_mo;
          double cw = 0.0;  // sum_m C_{b,m} (A^-1)_{m i}  (angular factor folded in C)
          for (int m = 0; m < n; ++m) {
            const double ai = ainv[sp][m][a];
            cw += Cb[m] * ai;
            acc[(size_t)(off_c + b * wf.n_mo + m) * T + tid] += wt * ang[b] * Pm * f * ai;
          }
          const int p0 = prim_start[b];
          if (sh.kind == 0) {
            const int nq = sh.kn + (pw & 15) + ((pw >> 4) & 15) + ((pw >> 8) & 15) + 1;
            acc[(size_t)p0 * T + tid] += wt * cw * Pm * f * ((nq + 0.5) / sh.expo[0] - rho);
          } else {
            for (int p = 0; p < sh.n_prim; ++p) {
              const double al = sh.expo[p];
              const double term = sh.coef[p] * exp(-al * r2);
              acc[(size_t)(p0 + p) * T + tid] += wt * cw * Pm * term * ((0.75 + 0.5 * sh.l) / al - r2);
            }
          }
        }
      }
    }
    acc[(size_t)off_d * T + tid] += wt / wf.det_w[0];
    double gb = 0.0;
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j) {
        const double dist = 1.0 / P.inv[i][j];
        const double w0 = ((i < nu) == (j < nu)) ? wf.w0_par : wf.w0_anti;
        const double den = 1.0 + wf.jb * dist;
        gb -= w0 * dist * dist / (den * den);
      }
    acc[(size_t)off_b * T + tid] += wt * gb;
    {  // also at w = 0: the derivative of turning the backflow on
      double gw = 0.0;
      for (int i = 0; i < N; ++i) {
        const int sp = i < nu ? 0 : 1, n = sp == 0 ? nu : wf.n_down, a = sp == 0 ? i : i - nu;
        for (int m = 0; m < n; ++m)
          gw += ainv[sp][m][a] * (dphi[i][m][0] * drt[i][0] + dphi[i][m][1] * drt[i][1] + dphi[i][m][2] * drt[i][2]);
      }
      acc[(size_t)off_w * T + tid] += wt * gw;
    }
  }
  __syncthreads();
  for (int o = T / 2; o > 0; o >>= 1) {
    if (tid < o)
      for (int k = 0; k < n_param; ++k) acc[(size_t)k * T + tid] += acc[(size_t)k * T + tid + o];
    __syncthreads();
  }
  for (int k = tid; k < n_param; k += T) partial[(size_t)k * gridDim.x + blockIdx.x] = acc[(size_t)k * T];
}

// Row sums of partial[n_rows][n_cols] in column order (deterministic).
__global__ void k_row_sums(const double* __restrict__ partial, int n_rows, int n_cols, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_rows) return;
  double s = 0.0;
  for (int c = 0; c < n_cols; ++c) s += partial[(size_t)k * n_cols + c];
  out[k] = s;
}

cudaError_t launch_row_sums(const double* partial, int n_rows, int n_cols, double* out, cudaStream_t st) {
  k_row_sums<<<(n_rows + 127) / 128, 128, 0, st>>>(partial, n_rows, n_cols, out);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// launchers

cudaError_t launch_forces(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const double* e_loc,
                          const double* stats, double* partial, double* forces, cudaStream_t st, bool raw) {
  const size_t smem = gen_table_bytes(wf);
  const dim3 grid((unsigned)general_blocks(W), (unsigned)wf.n_atom);
  QMC_GEN_DISPATCH((k_forces<NE, NO><<<grid, 128, smem, st>>>(wf, walkers, W, ldw, e_loc, stats, partial, raw)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int rows = (raw ? 9 : 3) * wf.n_atom;
  k_row_sums<<<(rows + 127) / 128, 128, 0, st>>>(partial, rows, grid.x, forces);
  return cudaGetLastError();
}

size_t grad_smem_bytes(const WfDev& wf, int n_param) { return gen_table_bytes(wf) + sizeof(double) * 128 * n_param; }

cudaError_t launch_grad(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const double* e_loc,
                        const double* stats, const double* ang, const int* prim_start, int n_param, double* partial,
                        double* grad, cudaStream_t st, int weight) {
  const size_t smem = grad_smem_bytes(wf, n_param);
  const dim3 grid((unsigned)general_blocks(W));
  QMC_GEN_DISPATCH((cudaFuncSetAttribute(k_grad_logpsi<NE, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem),
                    k_grad_logpsi<NE, NO><<<grid, 128, smem, st>>>(wf, walkers, W, ldw, e_loc, stats, ang,
                                                                   prim_start, n_param, partial, weight)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_row_sums<<<(n_param + 127) / 128, 128, 0, st>>>(partial, n_param, grid.x, grad);
  return cudaGetLastError();
}

// M, sum E_L and sum E_L^2 of a batch in a fixed order (one block)
__global__ void k_energy_sums(const double* __restrict__ e, int64_t W, double* __restrict__ out) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int64_t w = threadIdx.x; w < W; w += blockDim.x) {
    a += e[w];
    b += e[w] * e[w];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = (double)W;
    out[1] = s1[0];
    out[2] = s2[0];
  }
}

cudaError_t launch_energy_sums(const double* e_loc, int64_t W, double* out, cudaStream_t st) {
  k_energy_sums<<<1, 256, 0, st>>>(e_loc, W, out);
  return cudaGetLastError();
}

}  // namespace qmc
