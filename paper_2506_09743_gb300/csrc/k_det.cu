// Determinants, excited-determinant tables and local-energy assembly.
// All arithmetic in FP64.  One thread per walker, both spin channels.
//
// Per spin channel s with n = n_s electrons (rows) and reference columns
// 0..n-1 (A0 = Phi[:, 0:n], B = O Phi with O = lap + 2 grad J . grad):
//   1. A0^-1 by Gauss-Jordan elimination with partial pivoting; det A0 is the
//      signed product of the pivots.
//   2. tr0 = Tr(A0^-1 B0)                           (Jacobi / eq. claudia_trace)
//   3. for every virtual column p that an excitation uses:
//        t      = A0^-1 Phi[:, p]                   (T_val column, all rows)
//        y      = B[:, p] - B0 t
//        Top[h] = (A0^-1 y)[h]   for holes h        (= (P M P) entries of Eq. table)
//      so that for an excitation X with holes h_a, particles p_b:
//        S_ab = T_val[h_a][p_b] = (P A0^-1 A_X P),   Mk_ab = Top[h_a][p_b] = (P M P)
//        D_X / D_0 = det S                          (the k x k minor, k <= 2)
//        Tr(A_X^-1 B_X) = tr0 + Tr(S^-1 Mk)         (Eq. table, App. F)
//      and R Tr(S^-1 Mk) = Tr(adj(S) Mk) needs no division.
//   4. Sigma / (D0_up D0_dn) = sum_n d_n R_n^up R_n^dn; the Slater kinetic part
//        [lap Sigma + 2 grad J . grad Sigma] / Sigma
//          = sum_n d_n (R^up R^dn)(Tr_n^up + Tr_n^dn) / sum_n d_n R^up R^dn
//      (Eqs. nabla_sigma, delta_sigma with the one-body operator O; the up-down
//      cross term is zero without backflow).
//   5. E_L = -1/2 (kinJ + Slater kinetic part) + V,  log|Psi| = J + log|Sigma|.
#include "qmc_internal.cuh"

namespace qmc {

// Read MO channel c, row i (electron), column m for walker w.
template <typename TA>
__device__ __forceinline__ double ld_mo(const TA* __restrict__ mo, int nch, int nmo, int64_t ldm, int i, int c,
                                        int m, int64_t w) {
  return double(mo[((int64_t)(i * nch + c) * nmo + m) * ldm + w]);
}

// In-place Gauss-Jordan inverse of a[0:n][0:n] (NS compile-time bound, rows
// in registers) with partial pivoting.  Returns det through (sign, prod).
template <int NS>
__device__ __forceinline__ void gj_inverse(double (&a)[NS][NS], int n, double& det) {
  int piv[NS];
  det = 1.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    if (k < n) {
      int p = k;
      double best = fabs(a[k][k]);
#pragma unroll
      for (int i = k + 1; i < NS; ++i) {
        if (i < n && fabs(a[i][k]) > best) { best = fabs(a[i][k]); p = i; }
      }
      piv[k] = p;
      if (p != k) det = -det;
#pragma unroll
      for (int i = k + 1; i < NS; ++i) {
        const bool sw = (i == p);
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          const double t = a[k][j];
          a[k][j] = sw ? a[i][j] : a[k][j];
          a[i][j] = sw ? t : a[i][j];
        }
      }
      const double pv = a[k][k];
      det *= pv;
      const double inv = 1.0 / pv;
      a[k][k] = 1.0;
#pragma unroll
      for (int j = 0; j < NS; ++j) a[k][j] *= inv;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        if (i != k && i < n) {
          const double f = a[i][k];
          a[i][k] = 0.0;
#pragma unroll
          for (int j = 0; j < NS; ++j) a[i][j] -= f * a[k][j];
        }
      }
    }
  }
  // undo the row interchanges as column interchanges, last first
#pragma unroll
  for (int k = NS - 1; k >= 0; --k) {
    if (k < n) {
      const int p = piv[k];
#pragma unroll
      for (int j = k + 1; j < NS; ++j) {
        const bool sw = (j == p);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          const double t = a[i][k];
          a[i][k] = sw ? a[i][j] : a[i][k];
          a[i][j] = sw ? t : a[i][j];
        }
      }
    }
  }
}

template <int NS, typename TA, bool KIN>
__global__ void __launch_bounds__(64) k_det(WfDev wf, int64_t W, const TA* __restrict__ mo, int64_t ldm,
                                            const double* __restrict__ jscal, double* __restrict__ e_loc,
                                            double* __restrict__ log_psi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // excitation tables, [element][thread] so that 64-bit accesses are conflict-free
  double* tab = reinterpret_cast<double*>(smem_raw);
  int* exc_s = reinterpret_cast<int*>(tab + (size_t)wf.tab_elems * blockDim.x);
  int* didx_s = exc_s + 2 * 5 * (wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1]);
  const int nexc_max = wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1];
  for (int s = 0; s < 2; ++s)
    for (int k = threadIdx.x; k < wf.n_exc[s] * 5; k += blockDim.x)
      exc_s[(s * nexc_max) * 5 + k] = wf.exc[s * kMaxExc * 5 + k];
  for (int k = threadIdx.x; k < wf.n_det * 2; k += blockDim.x) didx_s[k] = wf.det_idx[k];
  __syncthreads();

  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int nch = KIN ? 2 : 1;
  const int nmo = wf.n_mo;
  const int T = blockDim.x, tid = threadIdx.x;

  double logdet = 0.0, tr0u = 0.0, tr0d = 0.0;
  int tab_off = 0;
  for (int s = 0; s < 2; ++s) {
    const int n = s == 0 ? wf.n_up : wf.n_down;
    const int i0 = s == 0 ? 0 : wf.n_up;
    if (n == 0) continue;
    double a[NS][NS];
#pragma unroll
    for (int r = 0; r < NS; ++r)
#pragma unroll
      for (int m = 0; m < NS; ++m) a[r][m] = (r < n && m < n) ? ld_mo(mo, nch, nmo, ldm, i0 + r, 0, m, w) : 0.0;
    double det;
    gj_inverse<NS>(a, n, det);  // a[m][r] = (A0^-1)_{m r}
    logdet += log(fabs(det));
    if (KIN) {
      double t = 0.0;
#pragma unroll
      for (int m = 0; m < NS; ++m)
#pragma unroll
        for (int r = 0; r < NS; ++r)
          if (m < n && r < n) t += a[m][r] * ld_mo(mo, nch, nmo, ldm, i0 + r, 1, m, w);
      if (s == 0) tr0u = t; else tr0d = t;
    }
    const int hl = wf.h_lo[s], nh = wf.nh[s], nv = wf.nv[s];
    for (int pv = 0; pv < nv; ++pv) {
      const int p = n + pv;
      double phi[NS], t[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) phi[r] = r < n ? ld_mo(mo, nch, nmo, ldm, i0 + r, 0, p, w) : 0.0;
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < NS; ++r) acc += a[m][r] * phi[r];
        t[m] = acc;
      }
#pragma unroll
      for (int m = 0; m < NS; ++m)
        if (m >= hl && m < n) tab[(size_t)(tab_off + (m - hl) * nv + pv) * T + tid] = t[m];
      if (KIN) {
        double y[NS];
#pragma unroll
        for (int r = 0; r < NS; ++r) {
          double acc = 0.0;
          if (r < n) {
            acc = ld_mo(mo, nch, nmo, ldm, i0 + r, 1, p, w);
#pragma unroll
            for (int m = 0; m < NS; ++m)
              if (m < n) acc -= ld_mo(mo, nch, nmo, ldm, i0 + r, 1, m, w) * t[m];
          }
          y[r] = acc;
        }
#pragma unroll
        for (int m = 0; m < NS; ++m) {
          if (m >= hl && m < n) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < NS; ++r) acc += a[m][r] * y[r];
            tab[(size_t)(tab_off + nh * nv + (m - hl) * nv + pv) * T + tid] = acc;
          }
        }
      }
    }
    tab_off += (KIN ? 2 : 1) * nh * nv;
  }

  // determinant expansion
  double sum_r = 0.0, sum_k = 0.0;
  for (int d = 0; d < wf.n_det; ++d) {
    double R[2], RT[2];
    int off = 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const double tr0s = s == 0 ? tr0u : tr0d;
      const int n = s == 0 ? wf.n_up : wf.n_down;
      const int hl = wf.h_lo[s], nh = wf.nh[s], nv = wf.nv[s];
      const int* e = exc_s + (s * nexc_max + didx_s[2 * d + s]) * 5;
      const int rank = e[0];
      const double* tv = tab + (size_t)off * T + tid;
      const double* tk = tab + (size_t)(off + nh * nv) * T + tid;
      if (rank == 0) {
        R[s] = 1.0; RT[s] = tr0s;
      } else if (rank == 1) {
        const int q = (e[1] - hl) * nv + (e[3] - n);
        R[s] = tv[(size_t)q * T];
        RT[s] = R[s] * tr0s + (KIN ? tk[(size_t)q * T] : 0.0);
      } else {
        const int q00 = (e[1] - hl) * nv + (e[3] - n), q01 = (e[1] - hl) * nv + (e[4] - n);
        const int q10 = (e[2] - hl) * nv + (e[3] - n), q11 = (e[2] - hl) * nv + (e[4] - n);
        const double s00 = tv[(size_t)q00 * T], s01 = tv[(size_t)q01 * T];
        const double s10 = tv[(size_t)q10 * T], s11 = tv[(size_t)q11 * T];
        R[s] = s00 * s11 - s01 * s10;
        RT[s] = R[s] * tr0s;
        if (KIN)
          RT[s] += s11 * tk[(size_t)q00 * T] - s01 * tk[(size_t)q10 * T] - s10 * tk[(size_t)q01 * T] +
                   s00 * tk[(size_t)q11 * T];
      }
      off += (KIN ? 2 : 1) * nh * nv;
    }
    const double dw = wf.det_w[d];
    sum_r += dw * R[0] * R[1];
    if (KIN) sum_k += dw * (RT[0] * R[1] + R[0] * RT[1]);
  }
  const double J = jscal[w];
  const double lp = J + logdet + log(fabs(sum_r));
  if (log_psi) log_psi[w] = lp;
  if (KIN) {
    const double kinJ = jscal[ldm + w], V = jscal[2 * ldm + w];
    e_loc[w] = -0.5 * (kinJ + sum_k / sum_r) + V;
  }
}

template <int NS, typename TA>
static cudaError_t launch_ns(const WfDev& wf, int64_t W, const Workspace& ws, bool kin, double* e_loc,
                             double* log_psi, cudaStream_t st) {
  const int block = 64;
  const dim3 grid((unsigned)((W + block - 1) / block));
  const int nexc_max = wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1];
  const int tab = kin ? wf.tab_elems : (wf.nh[0] * wf.nv[0] + wf.nh[1] * wf.nv[1]);
  const size_t smem = sizeof(double) * (size_t)tab * block + sizeof(int) * (10 * nexc_max + 2 * wf.n_det);
  WfDev w2 = wf;
  w2.tab_elems = tab;
  const TA* mo = static_cast<const TA*>(ws.mo);
  if (kin) {
    auto kern = k_det<NS, TA, true>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, block, smem, st>>>(w2, W, mo, ws.ldm, ws.jscal, e_loc, log_psi);
  } else {
    auto kern = k_det<NS, TA, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, block, smem, st>>>(w2, W, mo, ws.ldm, ws.jscal, e_loc, log_psi);
  }
  return cudaGetLastError();
}

template <typename TA>
static cudaError_t launch_t(const WfDev& wf, int64_t W, const Workspace& ws, bool kin, double* e_loc,
                           double* log_psi, cudaStream_t st) {
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  if (ns <= 1) return launch_ns<1, TA>(wf, W, ws, kin, e_loc, log_psi, st);
  if (ns <= 2) return launch_ns<2, TA>(wf, W, ws, kin, e_loc, log_psi, st);
  if (ns <= 4) return launch_ns<4, TA>(wf, W, ws, kin, e_loc, log_psi, st);
  if (ns <= 8) return launch_ns<8, TA>(wf, W, ws, kin, e_loc, log_psi, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_det(const WfDev& wf, int prec, int64_t W, const Workspace& ws, bool kinetic, double* e_loc,
                       double* log_psi, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  return prec == QMC_FP64 ? launch_t<double>(wf, W, ws, kinetic, e_loc, log_psi, st)
                          : launch_t<float>(wf, W, ws, kinetic, e_loc, log_psi, st);
}

}  // namespace qmc
