// Determinants, excited-determinant tables and local-energy assembly.
// All arithmetic in FP64 (the inputs are widened to FP64 exactly).
//
// Work decomposition: a team of TS threads (TS = 1, 2, 4 or 8, a divisor of
// the warp) owns one walker.  FP64 issue slots are the scarce resource on
// GB300 (the FP64 pipe runs at 1/64 of the FP32 rate), so the work is split
// without redundancy and the team keeps enough warps resident to hide
// latency:
//   0. stage: the walker's MO block of one spin (value channel Phi and
//      kinetic channel B = (lap + 2 grad J . grad) Phi, rows = electrons,
//      columns = orbitals) is read as one contiguous chunk, widened to FP64
//      with integer bit operations and kept in shared memory;
//   1. A0^-1 (A0 = Phi[:, 0:n]) by Gauss-Jordan elimination with partial
//      pivoting, thread q owning column q; the pivot row index and pivot
//      column are broadcast by warp shuffles; det A0 is the signed pivot
//      product;
//   2. tr0 = Tr(A0^-1 B0) (Jacobi formula / eq. claudia_trace), and per
//      virtual column p (thread q takes p = n + q, n + q + TS, ...):
//        t      = A0^-1 Phi[:, p]          T_val column
//        y      = B[:, p] - B0 t
//        Top[h] = (A0^-1 y)[h]             for the holes h
//      which gives, for an excitation X with holes h_a and particles p_b,
//        S_ab = T_val[h_a][p_b] = (P A0^-1 A_X P),  Mk_ab = Top[h_a][p_b] = (P M P)
//        D_X / D_0 = det S,  Tr(A_X^-1 B_X) = tr0 + Tr(S^-1 Mk)   (Eq. table, App. F)
//      with R Tr(S^-1 Mk) = Tr(adj(S) Mk), free of divisions;
//   3. the determinant list is split over the team:
//        Sigma / (D0_up D0_dn) = sum_n d_n R_n^up R_n^dn
//        [lap Sigma + 2 grad J . grad Sigma] / Sigma
//             = sum_n d_n (RT^up R^dn + R^up RT^dn) / sum_n d_n R^up R^dn
//      (Eqs. nabla_sigma, delta_sigma; the up-down cross term vanishes
//      without backflow) and reduced across the team by shuffles;
//   4. E_L = -1/2 (kinJ + Slater kinetic part) + V, log|Psi| = J + log|Sigma|.
#include "qmc_internal.cuh"

namespace qmc {

template <int NS, int TS, typename TA, bool KIN>
__global__ void __launch_bounds__(256) k_det(WfDev wf, int64_t W, const TA* __restrict__ mo, int nmp,
                                             const double* __restrict__ jscal, int64_t ldm, int stride,
                                             double* __restrict__ e_loc, double* __restrict__ log_psi) {
  constexpr int WPB = 256 / TS;
  constexpr int NCH = KIN ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nexc = wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1];
  double* walk_s = reinterpret_cast<double*>(smem_raw);  // [WPB][stride]
  double* dw_s = walk_s + (size_t)WPB * stride;          // [n_det]
  int* exc_s = reinterpret_cast<int*>(dw_s + wf.n_det);  // [2][nexc][5]
  int* didx_s = exc_s + 10 * nexc;                       // [n_det][2]
  for (int s = 0; s < 2; ++s)
    for (int k = threadIdx.x; k < wf.n_exc[s] * 5; k += blockDim.x) exc_s[s * nexc * 5 + k] = wf.exc[s * kMaxExc * 5 + k];
  for (int k = threadIdx.x; k < wf.n_det * 2; k += blockDim.x) didx_s[k] = wf.det_idx[k];
  for (int k = threadIdx.x; k < wf.n_det; k += blockDim.x) dw_s[k] = wf.det_w[k];
  __syncthreads();

  const int team = threadIdx.x / TS, q = threadIdx.x % TS;
  const int lane0 = (threadIdx.x & 31) - q;  // first lane of the team
  const int64_t w = (int64_t)blockIdx.x * WPB + team;
  const bool live = w < W;
  const int nmo = wf.n_mo, N = wf.n_elec;
  double* my = walk_s + (size_t)team * stride;
  // per-walker shared layout: stage [NCH][NS][nmo] (input type, widened on
  // read: halves the footprint in the FP32 forms) | ainv [NS][NS] | tables
  TA* stage = reinterpret_cast<TA*>(my);
  double* ainv = my + (NCH * NS * nmo * (int)sizeof(TA) + 7) / 8;
  double* tab = ainv + NS * NS;
  const TA* blk = mo + (size_t)(live ? w : 0) * N * NCH * nmp;

  double detprod = 1.0, tr0u = 0.0, tr0d = 0.0;
  int tab_off = 0;
  for (int s = 0; s < 2; ++s) {
    const int n = s == 0 ? wf.n_up : wf.n_down;
    const int i0 = s == 0 ? 0 : wf.n_up;
    if (n == 0) continue;
    // ---- 0. stage rows i0 .. i0+n-1 (contiguous in the walker block)
    {
      const TA* src = blk + (size_t)i0 * NCH * nmp;
      const int total = n * NCH * nmp;
      for (int k = q; k < total; k += TS) {
        const int m = k % nmp, rc = k / nmp, c = rc % NCH, r = rc / NCH;
        if (m < nmo) stage[(c * NS + r) * nmo + m] = live ? src[k] : TA(r == m ? 1 : 0);
      }
    }
    __syncwarp();
    // ---- 1. Gauss-Jordan inverse, thread q owns column q
    double col[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) col[r] = (r < n && q < n) ? widen(stage[r * nmo + q]) : 0.0;
    int piv[NS];
    double det = 1.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (k < n) {
        int p = k;
        long long best = abs_key(col[k]);
#pragma unroll
        for (int i = k + 1; i < NS; ++i)
          if (i < n && abs_key(col[i]) > best) { best = abs_key(col[i]); p = i; }
        p = __shfl_sync(0xffffffffu, p, lane0 + k);
        piv[k] = p;
#pragma unroll
        for (int i = k + 1; i < NS; ++i) {
          const bool sw = (i == p);
          const double t = col[k];
          col[k] = sw ? col[i] : col[k];
          col[i] = sw ? t : col[i];
        }
        double f[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) f[i] = __shfl_sync(0xffffffffu, col[i], lane0 + k);
        const double pv = f[k];
        det *= (p != k) ? -pv : pv;
        const double inv = recip(pv);
        const double ak = ((q == k) ? 1.0 : col[k]) * inv;
        col[k] = ak;
#pragma unroll
        for (int i = 0; i < NS; ++i)
          if (i != k && i < n) col[i] = ((q == k) ? 0.0 : col[i]) - f[i] * ak;
      }
    }
    {  // undo the row interchanges as column interchanges
      int src = q;
#pragma unroll
      for (int k = 0; k < NS; ++k)
        if (k < n) src = (src == k) ? piv[k] : (src == piv[k] ? k : src);
#pragma unroll
      for (int r = 0; r < NS; ++r) col[r] = __shfl_sync(0xffffffffu, col[r], lane0 + (src < TS ? src : 0));
    }
    if (q < n) {
#pragma unroll
      for (int m = 0; m < NS; ++m)
        if (m < n) ainv[m * NS + q] = col[m];  // (A0^-1)_{m q}
    }
    detprod *= det;  // one logarithm per walker, taken at the end
    __syncwarp();
    // ---- 2. tr0 and the excitation tables
    if (KIN) {
      double c = 0.0;
      if (q < n) {
#pragma unroll
        for (int r = 0; r < NS; ++r)
          if (r < n) c += ainv[q * NS + r] * widen(stage[(NS + r) * nmo + q]);
      }
      c = team_sum<TS>(c);
      if (s == 0) tr0u = c; else tr0d = c;
    }
    const int hl = wf.h_lo[s], nh = wf.nh[s], nv = wf.nv[s];
    for (int pv = q; pv < nv; pv += TS) {
      const int p = n + pv;
      double t[NS];
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        double acc = 0.0;
        if (m < n) {
#pragma unroll
          for (int r = 0; r < NS; ++r)
            if (r < n) acc += ainv[m * NS + r] * widen(stage[r * nmo + p]);
        }
        t[m] = acc;
      }
#pragma unroll
      for (int m = 0; m < NS; ++m)
        if (m >= hl && m < n) tab[tab_off + (m - hl) * nv + pv] = t[m];
      if (KIN) {
        double y[NS];
#pragma unroll
        for (int r = 0; r < NS; ++r) {
          double acc = 0.0;
          if (r < n) {
            acc = widen(stage[(NS + r) * nmo + p]);
#pragma unroll
            for (int m = 0; m < NS; ++m)
              if (m < n) acc -= widen(stage[(NS + r) * nmo + m]) * t[m];
          }
          y[r] = acc;
        }
#pragma unroll
        for (int m = 0; m < NS; ++m) {
          if (m >= hl && m < n) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < NS; ++r)
              if (r < n) acc += ainv[m * NS + r] * y[r];
            tab[tab_off + nh * nv + (m - hl) * nv + pv] = acc;
          }
        }
      }
    }
    tab_off += NCH * nh * nv;
    __syncwarp();
  }

  // ---- 3. determinant expansion, split over the team
  double sum_r = 0.0, sum_k = 0.0;
  for (int d = q; d < wf.n_det; d += TS) {
    double R[2], RT[2];
    int off = 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const double tr0s = s == 0 ? tr0u : tr0d;
      const int n = s == 0 ? wf.n_up : wf.n_down;
      const int hl = wf.h_lo[s], nh = wf.nh[s], nv = wf.nv[s];
      const int* e = exc_s + (s * nexc + didx_s[2 * d + s]) * 5;
      const int rank = e[0];
      const double* tv = tab + off;
      const double* tk = tab + off + nh * nv;
      if (rank == 0) {
        R[s] = 1.0;
        RT[s] = tr0s;
      } else if (rank == 1) {
        const int qq = (e[1] - hl) * nv + (e[3] - n);
        R[s] = tv[qq];
        RT[s] = KIN ? R[s] * tr0s + tk[qq] : 0.0;
      } else {
        const int q00 = (e[1] - hl) * nv + (e[3] - n), q01 = (e[1] - hl) * nv + (e[4] - n);
        const int q10 = (e[2] - hl) * nv + (e[3] - n), q11 = (e[2] - hl) * nv + (e[4] - n);
        const double s00 = tv[q00], s01 = tv[q01], s10 = tv[q10], s11 = tv[q11];
        R[s] = s00 * s11 - s01 * s10;
        RT[s] = KIN ? R[s] * tr0s + s11 * tk[q00] - s01 * tk[q10] - s10 * tk[q01] + s00 * tk[q11] : 0.0;
      }
      off += NCH * nh * nv;
    }
    const double dw = dw_s[d];
    sum_r += dw * R[0] * R[1];
    if (KIN) sum_k += dw * (RT[0] * R[1] + R[0] * RT[1]);
  }
  sum_r = team_sum<TS>(sum_r);
  if (KIN) sum_k = team_sum<TS>(sum_k);
  if (q == 0 && live) {
    const double lp = jscal[w] + log(fabs(detprod * sum_r));
    if (log_psi) log_psi[w] = lp;
    if (KIN) e_loc[w] = -0.5 * (jscal[ldm + w] + sum_k / sum_r) + jscal[2 * ldm + w];
  }
}

// doubles per walker in shared memory, padded to 8 mod 16: 64-bit shared
// accesses are served per half warp (two teams of 8), and this offset puts
// the second team on the other 16 bank pairs both for broadcast reads and
// for row reads of 8 consecutive doubles
static int walker_stride(const WfDev& wf, int NS, bool kin, int ta_bytes) {
  const int nch = kin ? 2 : 1;
  const int tab = kin ? wf.tab_elems : (wf.nh[0] * wf.nv[0] + wf.nh[1] * wf.nv[1]);
  int s = (nch * NS * wf.n_mo * ta_bytes + 7) / 8 + NS * NS + tab;
  while (s % 16 != 8) ++s;
  return s;
}

size_t det_smem_bytes(const WfDev& wf, int NS, int TS, bool kin, int ta_bytes) {
  const int nexc = wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1];
  return sizeof(double) * ((size_t)(256 / TS) * walker_stride(wf, NS, kin, ta_bytes) + wf.n_det) +
         sizeof(int) * (10 * (size_t)nexc + 2 * (size_t)wf.n_det);
}

template <int NS, int TS, typename TA>
static cudaError_t launch_ns(const WfDev& wf, int64_t W, const Workspace& ws, bool kin, double* e_loc,
                             double* log_psi, cudaStream_t st) {
  constexpr int WPB = 256 / TS;
  const dim3 grid((unsigned)((W + WPB - 1) / WPB));
  const int stride = walker_stride(wf, NS, kin, (int)sizeof(TA));
  const size_t smem = det_smem_bytes(wf, NS, TS, kin, (int)sizeof(TA));
  const TA* mo = static_cast<const TA*>(ws.mo);
  auto kern = kin ? k_det<NS, TS, TA, true> : k_det<NS, TS, TA, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, 256, smem, st>>>(wf, W, mo, ws.nmp, ws.jscal, ws.ldm, stride, e_loc, log_psi);
  return cudaGetLastError();
}

// team size: enough threads for the widest of the n columns and nv virtual
// columns, at most 8
int det_team_size(const WfDev& wf) {
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  const int nv = wf.nv[0] > wf.nv[1] ? wf.nv[0] : wf.nv[1];
  const int need = ns > nv ? ns : nv;
  return need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : 8;
}

template <typename TA>
static cudaError_t launch_t(const WfDev& wf, int64_t W, const Workspace& ws, bool kin, double* e_loc,
                           double* log_psi, cudaStream_t st) {
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  const int ts = det_team_size(wf);
#define QMC_DET(NS_, TS_) \
  if (ns == NS_ && ts == TS_) return launch_ns<NS_, TS_, TA>(wf, W, ws, kin, e_loc, log_psi, st);
  QMC_DET(1, 1) QMC_DET(1, 2) QMC_DET(1, 4) QMC_DET(1, 8)
  QMC_DET(2, 2) QMC_DET(2, 4) QMC_DET(2, 8)
  QMC_DET(3, 4) QMC_DET(3, 8) QMC_DET(4, 4) QMC_DET(4, 8)
  QMC_DET(5, 8) QMC_DET(6, 8) QMC_DET(7, 8) QMC_DET(8, 8)
#undef QMC_DET
  return cudaErrorInvalidValue;
}

cudaError_t launch_det(const WfDev& wf, int prec, int64_t W, const Workspace& ws, bool kinetic, double* e_loc,
                       double* log_psi, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  return prec == QMC_FP64 ? launch_t<double>(wf, W, ws, kinetic, e_loc, log_psi, st)
                          : launch_t<float>(wf, W, ws, kinetic, e_loc, log_psi, st);
}

}  // namespace qmc
