// Explicit multi-determinant evaluation: the baseline of the paper's
// comparison between explicit and table-accelerated excited determinants
// (Sec. 2.2, App. A, Fig. xt_bench).  Every distinct spin excitation X gets
// its own matrix A_X (ground-state columns h replaced in place by virtual
// orbitals p, Eq. AX), factorised by LU with partial pivoting, with
//     D_X = det A_X,   t_X = Tr(A_X^-1 B_X)       (Jacobi formula)
// where B = (lap + 2 grad J . grad) Phi is the kinetic channel.  Then
//     Sigma = sum_n d_n D_n^up D_n^dn,
//     [lap Sigma + 2 grad J . grad Sigma] / Sigma
//           = sum_n d_n D_n^up D_n^dn (t_n^up + t_n^dn) / Sigma,
//     E_L = -1/2 (kinJ + that) + V,   log|Psi| = J + log|Sigma|.
// Cost: O(n^3) per distinct excitation instead of O(k^3) minors of tables.
// All arithmetic in FP64.
//
// Decomposition: a team of 8 threads per walker (four walkers per warp); the
// walker's MO block of one spin is staged in shared memory, the team's threads take distinct excitations in turn,
// each factorising its A_X in registers; (D_X, t_X) go to shared memory and
// the determinant list is then split over the team.
#include "qmc_internal.cuh"

namespace qmc {

constexpr int kTS = 8;
constexpr int kWPB = 8;  // walkers per CTA (64 threads)

template <int NS, bool KIN>
__global__ void __launch_bounds__(kWPB * kTS) k_det_explicit(WfDev wf, int64_t W, const double* __restrict__ mo, int nmp,
                                                             const double* __restrict__ jscal, int64_t ldm,
                                                             int stride, double* __restrict__ e_loc,
                                                             double* __restrict__ log_psi) {
  constexpr int NCH = KIN ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nexc = wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1];
  double* walk_s = reinterpret_cast<double*>(smem_raw);   // [kWPB][stride]
  double* dw_s = walk_s + (size_t)kWPB * stride;          // [n_det]
  int* exc_s = reinterpret_cast<int*>(dw_s + wf.n_det);   // [2][nexc][5]
  int* didx_s = exc_s + 10 * nexc;                        // [n_det][2]
  for (int s = 0; s < 2; ++s)
    for (int k = threadIdx.x; k < wf.n_exc[s] * 5; k += blockDim.x) exc_s[s * nexc * 5 + k] = wf.exc[s * kMaxExc * 5 + k];
  for (int k = threadIdx.x; k < wf.n_det * 2; k += blockDim.x) didx_s[k] = wf.det_idx[k];
  for (int k = threadIdx.x; k < wf.n_det; k += blockDim.x) dw_s[k] = wf.det_w[k];
  __syncthreads();

  const int team = threadIdx.x / kTS, q = threadIdx.x % kTS;
  const int64_t w = (int64_t)blockIdx.x * kWPB + team;
  const bool live = w < W;
  const int nmo = wf.n_mo;
  double* my = walk_s + (size_t)team * stride;
  // per-walker shared layout: results [2][nexc][2] (D_X, t_X) | stage [NCH][NS][nmo]
  double* res = my;
  double* stage = my + 4 * nexc;
  const int64_t wc = live ? w : 0;

  for (int s = 0; s < 2; ++s) {
    const int n = s == 0 ? wf.n_up : wf.n_down;
    const int i0 = s == 0 ? 0 : wf.n_up;
    double* rs = res + 2 * s * nexc;
    if (n == 0) {
      for (int u = q; u < wf.n_exc[s]; u += kTS) { rs[2 * u] = 1.0; rs[2 * u + 1] = 0.0; }
      __syncwarp();
      continue;
    }
    {  // MO layout [N][NCH][nmp][ldm], walker fastest
      const int total = n * NCH * nmo;
      for (int k = q; k < total; k += kTS) {
        const int m = k % nmo, rc = k / nmo, c = rc % NCH, r = rc / NCH;
        stage[(c * NS + r) * nmo + m] =
            live ? mo[((int64_t)((i0 + r) * NCH + c) * nmp + m) * ldm + wc] : (r == m ? 1.0 : 0.0);
      }
    }
    __syncwarp();
    for (int u = q; u < wf.n_exc[s]; u += kTS) {
      const int* e = exc_s + (s * nexc + u) * 5;
      const int h1 = e[1], h2 = e[2], p1 = e[3], p2 = e[4];
      // column c of A_X is orbital c, or its particle if c is a hole
      int orb[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) orb[c] = c == h1 ? p1 : c == h2 ? p2 : c;
      double a[NS][NS];
#pragma unroll
      for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int c = 0; c < NS; ++c)
          a[r][c] = (r < n && c < n) ? (stage[r * nmo + orb[c]]) : (r == c ? 1.0 : 0.0);
      // LU with partial pivoting, P A = L U (L unit lower, stored below the diagonal)
      int perm[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) perm[r] = r;
      double det = 1.0, dinv[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        dinv[k] = 1.0;
        if (k < n) {
          int p = k;
          long long best = abs_key(a[k][k]);
#pragma unroll
          for (int i = k + 1; i < NS; ++i)
            if (i < n && abs_key(a[i][k]) > best) { best = abs_key(a[i][k]); p = i; }
#pragma unroll
          for (int i = k + 1; i < NS; ++i) {
            const bool sw = i == p;
#pragma unroll
            for (int c = 0; c < NS; ++c) {
              const double t = a[k][c];
              a[k][c] = dsel(sw, a[i][c], t);
              a[i][c] = dsel(sw, t, a[i][c]);
            }
            const int tp = perm[k];
            perm[k] = isel(sw, perm[i], tp);
            perm[i] = isel(sw, tp, perm[i]);
          }
          const double pv = a[k][k];
          det *= (p != k) ? -pv : pv;
          const double inv = recip(pv);
          dinv[k] = inv;
#pragma unroll
          for (int i = k + 1; i < NS; ++i) {
            if (i < n) {
              const double l = a[i][k] * inv;
              a[i][k] = l;
#pragma unroll
              for (int c = k + 1; c < NS; ++c) a[i][c] -= l * a[k][c];
            }
          }
        }
      }
      double tr = 0.0;
      if (KIN) {
        // t_X = sum_c (A_X^-1 B_X)[c][c]: solve A_X y = B_X[:, c] per column
#pragma unroll
        for (int c = 0; c < NS; ++c) {
          if (c < n) {
            double y[NS];
#pragma unroll
            for (int r = 0; r < NS; ++r) y[r] = r < n ? (stage[(NS + perm[r]) * nmo + orb[c]]) : 0.0;
#pragma unroll
            for (int r = 0; r < NS; ++r)
#pragma unroll
              for (int j = 0; j < r; ++j) y[r] -= a[r][j] * y[j];
#pragma unroll
            for (int r = NS - 1; r >= 0; --r) {
              if (r < n) {
#pragma unroll
                for (int j = r + 1; j < NS; ++j)
                  if (j < n) y[r] -= a[r][j] * y[j];
                y[r] *= dinv[r];
              }
            }
            tr += y[c];
          }
        }
      }
      rs[2 * u] = det;
      rs[2 * u + 1] = tr;
    }
    __syncwarp();
  }

  double sum_r = 0.0, sum_k = 0.0;
  for (int d = q; d < wf.n_det; d += kTS) {
    const int iu = didx_s[2 * d], id = didx_s[2 * d + 1];
    const double du = res[2 * iu], tu = res[2 * iu + 1];
    const double dd = res[2 * nexc + 2 * id], td = res[2 * nexc + 2 * id + 1];
    const double c = dw_s[d] * du * dd;
    sum_r += c;
    if (KIN) sum_k += c * (tu + td);
  }
  sum_r = team_sum<kTS>(sum_r);
  if (KIN) sum_k = team_sum<kTS>(sum_k);
  if (q == 0 && live) {
    const double lp = jscal[w] + log(fabs(sum_r));
    if (log_psi) log_psi[w] = lp;
    if (KIN) e_loc[w] = -0.5 * (jscal[ldm + w] + sum_k / sum_r) + jscal[2 * ldm + w];
  }
}

namespace {

int explicit_stride(const WfDev& wf, int NS, bool kin) {
  const int nexc = wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1];
  const int nch = kin ? 2 : 1;
  int s = 4 * nexc + nch * NS * wf.n_mo;
  return s | 1;  // odd: the teams' rows start on different banks
}

template <int NS>
cudaError_t launch_x(const WfDev& wf, int64_t W, const Workspace& ws, bool kin, double* e_loc, double* log_psi,
                     cudaStream_t st) {
  const int stride = explicit_stride(wf, NS, kin);
  const size_t smem = det_explicit_smem_bytes(wf, kin);
  const dim3 grid((unsigned)((W + kWPB - 1) / kWPB));
  auto kern = kin ? k_det_explicit<NS, true> : k_det_explicit<NS, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, kWPB * kTS, smem, st>>>(wf, W, ws.mo, ws.nmp, ws.jscal, ws.ldm, stride, e_loc, log_psi);
  return cudaGetLastError();
}

}  // namespace

size_t det_explicit_smem_bytes(const WfDev& wf, bool kin) {
  const int nexc = wf.n_exc[0] > wf.n_exc[1] ? wf.n_exc[0] : wf.n_exc[1];
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  return sizeof(double) * ((size_t)kWPB * explicit_stride(wf, ns, kin) + wf.n_det) +
         sizeof(int) * (10 * (size_t)nexc + 2 * (size_t)wf.n_det);
}

cudaError_t launch_det_explicit(const WfDev& wf, int prec, int64_t W, const Workspace& ws, bool kinetic,
                                double* e_loc, double* log_psi, cudaStream_t st) {
  (void)prec;  // the MO channels are FP64 in every form
  if (W == 0) return cudaSuccess;
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  switch (ns) {
    case 1: return launch_x<1>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 2: return launch_x<2>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 3: return launch_x<3>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 4: return launch_x<4>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 5: return launch_x<5>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 6: return launch_x<6>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 7: return launch_x<7>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 8: return launch_x<8>(wf, W, ws, kinetic, e_loc, log_psi, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qmc
