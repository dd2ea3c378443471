// Determinants, excited-determinant tables and local-energy assembly.
// All arithmetic in FP64 (the MO channels arrive in FP64 in every form).
//
// Work decomposition: one thread per (walker, spin); the two spins of a
// walker are adjacent lanes of one warp.  FP64 issue slots are the scarce
// resource on GB300 (the FP64 pipe runs at about 1/62 of the FP32 rate), so each
// thread keeps its reference inverse in registers and runs long chains of
// independent FMAs (no shuffles inside the linear algebra, no idle lanes,
// no duplicated per-walker work):
//   1. A0^-1 (A0 = Phi[:, 0:n], rows = electrons of the spin, columns =
//      orbitals) by Gauss-Jordan elimination with partial pivoting in
//      registers; rows are exchanged with selects, and the exchanges are
//      undone on the columns of the inverse at the end; det A0 is the signed
//      pivot product;
//   2. tr0 = Tr(A0^-1 B0) (Jacobi formula / eq. claudia_trace), B the kinetic
//      channel (lap + 2 grad J . grad) Phi, and per virtual column p:
//        t      = A0^-1 Phi[:, p]          T_val column
//        y      = B[:, p] - B0 t
//        Top[h] = (A0^-1 y)[h]             for the holes h
//      stored in shared memory; for an excitation X with holes h_a and
//      particles p_b,
//        S_ab = T_val[h_a][p_b] = (P A0^-1 A_X P),  Mk_ab = Top[h_a][p_b] = (P M P)
//        D_X / D_0 = det S,  Tr(A_X^-1 B_X) = tr0 + Tr(S^-1 Mk)   (Eq. table, App. F)
//      with R Tr(S^-1 Mk) = Tr(adj(S) Mk), free of divisions;
//   3. the two threads of a walker split its determinant list (both spins'
//      tables are in shared memory):
//        Sigma / (D0_up D0_dn) = sum_n d_n R_n^up R_n^dn
//        [lap Sigma + 2 grad J . grad Sigma] / Sigma
//             = (tr0_up + tr0_dn) + sum_n d_n (K^up R^dn + R^up K^dn) / sum_n d_n R^up R^dn,
//        K = R (Tr(A_X^-1 B_X) - tr0)
//      (Eqs. nabla_sigma, delta_sigma; the up-down cross term vanishes
//      without backflow), and combine their sums with one shuffle;
//   4. E_L = -1/2 (kinJ + Slater kinetic part) + V, log|Psi| = J + log|Sigma|.
//
// MO input layout (walker fastest, so that a warp's loads are coalesced):
// element (electron i, channel c, orbital m) of walker w at
// mo[((i * NCH + c) * nmp + m) * ldm + w].
#include "qmc_internal.cuh"

namespace qmc {

namespace {

constexpr int kWalkersPerBlock = 32;  // 64 threads: (walker, spin) pairs

}  // namespace

template <int NS, bool KIN>
__global__ void __launch_bounds__(2 * kWalkersPerBlock)
    k_det(WfDev wf, int64_t W, const double* __restrict__ mo, int nmp, int64_t ldm, const double* __restrict__ jscal,
          int stride, double* __restrict__ e_loc, double* __restrict__ log_psi) {
  constexpr int NCH = KIN ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* tab_all = reinterpret_cast<double*>(smem_raw);       // [kWalkersPerBlock][stride]
  double* dw_s = tab_all + (size_t)kWalkersPerBlock * stride;  // [n_det]
  int4* dt_s = reinterpret_cast<int4*>(dw_s + ((wf.n_det + 1) & ~1));  // [n_det] determinant records
  for (int k = threadIdx.x; k < wf.n_det; k += blockDim.x) {
    dw_s[k] = wf.det_w[k];
    dt_s[k] = wf.det_tab[k];
  }
  __syncthreads();

  const int wl = threadIdx.x >> 1, s = threadIdx.x & 1;
  const int64_t w = (int64_t)blockIdx.x * kWalkersPerBlock + wl;
  const bool live = w < W;
  const int64_t wc = live ? w : 0;  // column read by threads past the end (their results are discarded)
  const int n = s == 0 ? wf.n_up : wf.n_down;
  const int i0 = s == 0 ? 0 : wf.n_up;
  const int hl = wf.h_lo[s], nh = wf.nh[s], nv = wf.nv[s];
  double* tab = tab_all + (size_t)wl * stride;
  const int tab_off = s == 0 ? 0 : NCH * wf.nh[0] * wf.nv[0];
  // channel c (0 = Phi, 1 = B) of electron row r, orbital m
  auto ld = [&](int c, int r, int m) -> double {
    return mo[((int64_t)((i0 + r) * NCH + c) * nmp + m) * ldm + wc];
  };

  // ---- 1. Gauss-Jordan inverse in registers: a[m][r] ends as (A0^-1)_{m r}
  double a[NS][NS];
#pragma unroll
  for (int r = 0; r < NS; ++r)
#pragma unroll
    for (int c = 0; c < NS; ++c) a[r][c] = (r < n && c < n) ? ld(0, r, c) : (r == c ? 1.0 : 0.0);
  int piv[NS];
  double det = 1.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    piv[k] = k;
    if (k < n) {
      int p = k;
      long long best = abs_key(a[k][k]);
#pragma unroll
      for (int i = k + 1; i < NS; ++i)
        if (i < n && abs_key(a[i][k]) > best) { best = abs_key(a[i][k]); p = i; }
      piv[k] = p;
#pragma unroll
      for (int i = k + 1; i < NS; ++i) {
        const bool sw = i == p;
#pragma unroll
        for (int c = 0; c < NS; ++c) {
          const double t = a[k][c];
          a[k][c] = dsel(sw, a[i][c], t);
          a[i][c] = dsel(sw, t, a[i][c]);
        }
      }
      const double pv = a[k][k];
      det *= (p != k) ? -pv : pv;
      const double inv = recip(pv);
#pragma unroll
      for (int c = 0; c < NS; ++c) a[k][c] = (c == k) ? inv : a[k][c] * inv;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        if (i != k && i < n) {
          const double f = a[i][k];
#pragma unroll
          for (int c = 0; c < NS; ++c) a[i][c] = (c == k) ? -f * inv : fma(-f, a[k][c], a[i][c]);
        }
      }
    }
  }
  // undo the row exchanges as column exchanges of the inverse, last first
#pragma unroll
  for (int k = NS - 1; k >= 0; --k) {
    const int p = piv[k];
#pragma unroll
    for (int c = k + 1; c < NS; ++c) {
      const bool sw = c == p;
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        const double t = a[m][k];
        a[m][k] = dsel(sw, a[m][c], t);
        a[m][c] = dsel(sw, t, a[m][c]);
      }
    }
  }

  // ---- 2. tr0 and the excitation tables
  double tr0 = 0.0;
  if (KIN) {
    double part[NS];  // independent partial sums (no serial FMA chain)
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      part[m] = 0.0;
#pragma unroll
      for (int r = 0; r < NS; ++r)
        if (m < n && r < n) part[m] = fma(a[m][r], ld(1, r, m), part[m]);
    }
#pragma unroll
    for (int m = 0; m < NS; ++m) tr0 += part[m];
  }
  // virtual columns Phi_p and B_p are loaded one column ahead (software
  // pipelining: their global-load latency overlaps the previous column's FMAs)
  double nphi[NS], nbp[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) {
    nphi[r] = (r < n && nv > 0) ? ld(0, r, n) : 0.0;
    nbp[r] = (KIN && r < n && nv > 0) ? ld(1, r, n) : 0.0;
  }
  for (int pv = 0; pv < nv; ++pv) {
    const int p = n + pv;
    double cphi[NS], cbp[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      cphi[r] = nphi[r];
      cbp[r] = nbp[r];
    }
    if (pv + 1 < nv) {
#pragma unroll
      for (int r = 0; r < NS; ++r)
        if (r < n) {
          nphi[r] = ld(0, r, p + 1);
          if (KIN) nbp[r] = ld(1, r, p + 1);
        }
    }
    double t[NS];
#pragma unroll
    for (int m = 0; m < NS; ++m) t[m] = 0.0;
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      if (r < n) {
        const double phi = cphi[r];
#pragma unroll
        for (int m = 0; m < NS; ++m) t[m] = fma(a[m][r], phi, t[m]);
      }
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
          acc = cbp[r];
#pragma unroll
          for (int m = 0; m < NS; ++m)
            if (m < n) acc = fma(-ld(1, r, m), t[m], acc);
        }
        y[r] = acc;
      }
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        if (m >= hl && m < n) {
          double acc = 0.0;
#pragma unroll
          for (int r = 0; r < NS; ++r)
            if (r < n) acc = fma(a[m][r], y[r], acc);
          tab[tab_off + nh * nv + (m - hl) * nv + pv] = acc;
        }
      }
    }
  }
  const double tr0_other = __shfl_xor_sync(0xffffffffu, tr0, 1);
  const double det_other = __shfl_xor_sync(0xffffffffu, det, 1);
  __syncwarp();

  // ---- 3. determinant expansion: thread s takes determinants d = s, s + 2, ...
  double sum_r = 0.0, sum_k = 0.0;
  for (int d = s; d < wf.n_det; d += 2) {
    const int4 rec = dt_s[d];
    double R[2], K[2];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const int packed = sp == 0 ? rec.x : rec.z, rank = sp == 0 ? rec.y : rec.w;
      const int off = sp == 0 ? 0 : NCH * wf.nh[0] * wf.nv[0];
      const double* tv = tab + off;
      const double* tk = tab + off + wf.nh[sp] * wf.nv[sp];
      const int q00 = packed & 0xff, q01 = (packed >> 8) & 0xff, q10 = (packed >> 16) & 0xff, q11 = packed >> 24;
      if (rank == 0) {
        R[sp] = 1.0;
        K[sp] = 0.0;
      } else if (rank == 1) {
        R[sp] = tv[q00];
        K[sp] = KIN ? tk[q00] : 0.0;
      } else {
        const double s00 = tv[q00], s01 = tv[q01], s10 = tv[q10], s11 = tv[q11];
        R[sp] = fma(s00, s11, -s01 * s10);
        K[sp] = KIN ? fma(s11, tk[q00], fma(-s01, tk[q10], fma(-s10, tk[q01], s00 * tk[q11]))) : 0.0;
      }
    }
    const double dw = dw_s[d];
    const double dr1 = dw * R[1];
    sum_r = fma(dr1, R[0], sum_r);
    if (KIN) sum_k = fma(dr1, K[0], fma(dw * R[0], K[1], sum_k));
  }
  sum_r += __shfl_xor_sync(0xffffffffu, sum_r, 1);
  if (KIN) sum_k += __shfl_xor_sync(0xffffffffu, sum_k, 1);
  if (s == 0 && live) {
    const double lp = jscal[w] + log(fabs(det * det_other * sum_r));
    if (log_psi) log_psi[w] = lp;
    if (KIN) e_loc[w] = -0.5 * (jscal[ldm + w] + tr0 + tr0_other + sum_k / sum_r) + jscal[2 * ldm + w];
  }
}

namespace {

// doubles of tables per walker in shared memory, made odd so that the 32
// walkers of a block start on different banks (the threads of a warp read
// the same table offset of different walkers)
int table_stride(const WfDev& wf, bool kin) {
  const int tab = kin ? wf.tab_elems : (wf.nh[0] * wf.nv[0] + wf.nh[1] * wf.nv[1]);
  return tab | 1;
}

template <int NS>
cudaError_t launch_ns(const WfDev& wf, int64_t W, const Workspace& ws, bool kin, double* e_loc, double* log_psi,
                      cudaStream_t st) {
  const dim3 grid((unsigned)((W + kWalkersPerBlock - 1) / kWalkersPerBlock));
  const int stride = table_stride(wf, kin);
  const size_t smem = det_smem_bytes(wf, kin);
  auto kern = kin ? k_det<NS, true> : k_det<NS, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, 2 * kWalkersPerBlock, smem, st>>>(wf, W, ws.mo, ws.nmp, ws.ldm, ws.jscal, stride, e_loc, log_psi);
  return cudaGetLastError();
}

}  // namespace

size_t det_smem_bytes(const WfDev& wf, bool kin) {
  return sizeof(double) * ((size_t)kWalkersPerBlock * table_stride(wf, kin) + ((wf.n_det + 1) & ~1)) +
         sizeof(int4) * (size_t)wf.n_det;
}

cudaError_t launch_det(const WfDev& wf, int prec, int64_t W, const Workspace& ws, bool kinetic, double* e_loc,
                       double* log_psi, cudaStream_t st) {
  (void)prec;  // the MO channels are FP64 in every form
  if (W == 0) return cudaSuccess;
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  switch (ns) {
    case 1: return launch_ns<1>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 2: return launch_ns<2>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 3: return launch_ns<3>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 4: return launch_ns<4>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 5: return launch_ns<5>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 6: return launch_ns<6>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 7: return launch_ns<7>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 8: return launch_ns<8>(wf, W, ws, kinetic, e_loc, log_psi, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qmc
