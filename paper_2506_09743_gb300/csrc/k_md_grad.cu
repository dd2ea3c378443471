// Parameter gradient of log|Psi| for a multi-determinant expansion without
// backflow (FP64): the estimator of Eq. nabla_loss for Psi of Eq. psimol
// with the CI sum, through the tables of the reference inverse (Eq. table).
//
// Per spin (n electrons a, orbitals m, Phi_{a m} = phi_m(r_a), A = Phi[:, occ]
// the reference matrix, T = A^-1 Phi, so that an excitation X with holes h
// and particles p has D_X / D_0 = R_X = det T[h, p]):
//   log|Psi| = log|D_0^up| + log|D_0^dn| + log|S|,   S = sum_n d_n R_n^up R_n^dn.
// The derivative of log|Psi| with respect to Phi_{a m} is Gamma_{m a}:
//   d log|D_0| / d Phi_{a m} = (A^-1)_{m a}                 (m occupied)
//   d log S / d Phi_{a m}    = [(I - P T) Y A^-1]_{m a},
// where Y_{p h} = (dS / dT_{h p}) / S collects, per unique excitation e of
// the spin, c_e = sum_{n: e_n = e} d_n R_n^(other spin) / S times dR_e/dT_{hp}
// (rank 1: 1; rank 2: the 2x2 cofactors), and P selects the occupied rows
// (dT = A^-1 (dPhi - dPhi[:, occ] T)).  Y has rows for particles only, so
//   Gamma_{m a} = (A^-1)_{m a} - sum_p T_{m p} Z_{p a}   (m occupied),
//   Gamma_{p a} = Z_{p a}                                 (particles),
//   Z = Y A^-1.
// Then with AO values phi_b (angular normalisation ang_b), MO coefficients
// C_{b m} and u_b = sum_m C_{b m} ang_b Gamma_{m a} per electron row:
//   d log|Psi| / d C_{b m}  = sum_a ang_b phi_b(r_a) Gamma_{m a}
//   d log|Psi| / d alpha_p  = sum_a u_b d phi_b / d alpha_p      (as k_grad_logpsi)
//   d log|Psi| / d d_n      = R_n^up R_n^dn / S
//   d log|Psi| / d b        = -sum_{i<j} w0 r_ij^2 / (1 + b r_ij)^2
//   d log|Psi| / d w        = sum_a sum_b u_b grad phi_b(r_a) . sum_{j != a} (r_a - r_j) / r_ij
// (the last at w = 0: the derivative of turning the backflow on).
//
// Two kernels: k_md_gamma (one thread per walker: the reference inverses,
// tables, CI sum, Gamma, the CI-weight and Jastrow terms) writes Gamma to
// scratch; k_md_rows (one thread per electron row) evaluates the AOs and
// adds the coefficient, exponent and backflow terms.  Per-walker values are
// weighted (estimator 2 (E_L - E_v) / M, one, or E_L) and summed per warp by
// shuffles in a fixed order (a butterfly reduce-scatter for the outputs of
// two AOs at a time), per block over the warps in order, and over the blocks
// by k_row_sums: the result is bitwise reproducible.
#include "general_eval.cuh"

namespace qmc {

namespace {

constexpr int kMdNS = 8;        // electrons per spin
constexpr int kMdNM = 16;       // orbitals
constexpr int kMdThreads = 128;
constexpr int kMdWarps = kMdThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;  // lane 0 holds the sum
}

__device__ __forceinline__ double walker_weight(int weight, const double* e_loc, const double* stats, int64_t w,
                                                int64_t W) {
  if (weight == 1) return 1.0;
  if (weight == 2) return e_loc[w];
  return 2.0 * (e_loc[w] - stats[0]) / (double)W;
}

// per-warp accumulators [kMdWarps][n_param] -> partial[k][col] in a fixed order
__device__ void flush_acc(const double* acc, int n_param, double* partial, int64_t ld_partial, int col) {
  __syncthreads();
  for (int k = threadIdx.x; k < n_param; k += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kMdWarps; ++q) s += acc[(size_t)q * n_param + k];
    partial[(size_t)k * ld_partial + col] = s;
  }
}

}  // namespace

__global__ void __launch_bounds__(kMdThreads) k_md_gamma(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                          int64_t ldw, const double* __restrict__ mo, int nmp,
                                                          int64_t ldm, const double* __restrict__ e_loc,
                                                          const double* __restrict__ stats, int weight, int n_param,
                                                          int off_d, double* __restrict__ gam,
                                                          double* __restrict__ partial, int64_t ld_partial) {
  extern __shared__ __align__(16) double acc[];  // [kMdWarps][n_param]
  for (int k = threadIdx.x; k < kMdWarps * n_param; k += blockDim.x) acc[k] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nu = wf.n_up, N = wf.n_elec, nmo = wf.n_mo;
  const int off_b = off_d + wf.n_det;
  const int64_t n_iter = (W + (int64_t)gridDim.x * kMdThreads - 1) / ((int64_t)gridDim.x * kMdThreads);
  for (int64_t it = 0; it < n_iter; ++it) {
    const int64_t w = (it * gridDim.x + blockIdx.x) * kMdThreads + threadIdx.x;
    const bool live = w < W;
    const double wt = live ? walker_weight(weight, e_loc, stats, w, W) : 0.0;
    double R[2][kMaxExc > 128 ? 128 : kMaxExc];  // ratios of the unique excitations
    double ainv[2][kMdNS][kMdNS], T[2][kMdNS][kMdNM];
    for (int s = 0; s < 2; ++s) {
      const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
      const int p_hi = wf.p_hi[s];
      for (int a = 0; a < n; ++a)
        for (int m = 0; m < n; ++m)
          ainv[s][a][m] = live ? mo[((size_t)((i0 + a) * 2) * nmp + m) * ldm + w] : (a == m ? 1.0 : 0.0);
      if (n > 0) small_inverse<double, kMdNS>(ainv[s], n);
      // T_{h p} = sum_a (A^-1)_{h a} Phi_{a p} for every occupied row h and particle p
      for (int h = 0; h < n; ++h)
        for (int p = n; p < p_hi; ++p) {
          double t = 0.0;
          for (int a = 0; a < n; ++a)
            t += ainv[s][h][a] * (live ? mo[((size_t)((i0 + a) * 2) * nmp + p) * ldm + w] : 0.0);
          T[s][h][p] = t;
        }
      for (int e = 0; e < wf.n_exc[s]; ++e) {
        const int* x = wf.exc + (s * kMaxExc + e) * 5;
        const int rank = x[0];
        R[s][e] = rank == 0 ? 1.0
                  : rank == 1 ? T[s][x[1]][x[3]]
                              : T[s][x[1]][x[3]] * T[s][x[2]][x[4]] - T[s][x[1]][x[4]] * T[s][x[2]][x[3]];
      }
    }
    double S = 0.0;
    for (int n = 0; n < wf.n_det; ++n) S += wf.det_w[n] * R[0][wf.det_idx[2 * n]] * R[1][wf.det_idx[2 * n + 1]];
    const double iS = live ? 1.0 / S : 0.0;
    // CI weights (stored sorted; the gradient goes to the original order)
    for (int n = 0; n < wf.n_det; ++n) {
      const double v = warp_sum(wt * R[0][wf.det_idx[2 * n]] * R[1][wf.det_idx[2 * n + 1]] * iS);
      if (lane == 0) acc[(size_t)warp * n_param + off_d + wf.det_orig[n]] += v;
    }
    // Jastrow b
    {
      double gb = 0.0;
      if (live)
        for (int i = 0; i < N; ++i)
          for (int j = i + 1; j < N; ++j) {
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
              const double dd = walkers[(int64_t)(3 * i + c) * ldw + w] - walkers[(int64_t)(3 * j + c) * ldw + w];
              d2 += dd * dd;
            }
            const double dist = sqrt(d2);
            const double w0 = ((i < nu) == (j < nu)) ? wf.w0_par : wf.w0_anti;
            const double den = 1.0 + wf.jb * dist;
            gb -= w0 * dist * dist / (den * den);
          }
      const double v = warp_sum(wt * gb);
      if (lane == 0) acc[(size_t)warp * n_param + off_b] += v;
    }
    // many-body Jastrow (App. D), after the backflow weight:
    //   K_en = (w0 r + w1 r^2) / (1 + w2 r) over atoms and electrons:
    //     d/dw0 = r / d, d/dw1 = r^2 / d, d/dw2 = -(w0 r + w1 r^2) r / d^2, d = 1 + w2 r;
    //   K_een = 1/2 sum over atoms, ordered pairs i != j and terms of
    //     c f(a1, b1; r_ai) f(a2, b2; r_aj) f(a3, b3; r_ij), f(a, b; r) = a r / (1 + b r):
    //     df/da = r / (1 + b r), df/db = -a r^2 / (1 + b r)^2
    if (wf.mb_en || wf.n_een) {
      int k = off_b + 2;
      if (wf.mb_en) {
        double g3[3] = {0.0, 0.0, 0.0};
        if (live)
          for (int a = 0; a < wf.n_atom; ++a)
            for (int i = 0; i < N; ++i) {
              double d2 = 0.0;
              for (int c = 0; c < 3; ++c) {
                const double dd = walkers[(int64_t)(3 * i + c) * ldw + w] - wf.atom_xyz[a][c];
                d2 += dd * dd;
              }
              const double r = sqrt(d2), d = 1.0 + wf.jen[2] * r;
              g3[0] += r / d;
              g3[1] += r * r / d;
              g3[2] -= (wf.jen[0] * r + wf.jen[1] * r * r) * r / (d * d);
            }
        for (int q = 0; q < 3; ++q) {
          const double v = warp_sum(wt * g3[q]);
          if (lane == 0) acc[(size_t)warp * n_param + k + q] += v;
        }
        k += 3;
      }
      for (int t = 0; t < wf.n_een; ++t) {
        const double c = wf.jeen[t][0], a1 = wf.jeen[t][1], b1 = wf.jeen[t][2], a2 = wf.jeen[t][3],
                     b2 = wf.jeen[t][4], a3 = wf.jeen[t][5], b3 = wf.jeen[t][6];
        double g7[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (live)
          for (int a = 0; a < wf.n_atom; ++a)
            for (int i = 0; i < N; ++i)
              for (int j = 0; j < N; ++j) {
                if (i == j) continue;
                double x2 = 0.0, y2 = 0.0, z2 = 0.0;
                for (int q = 0; q < 3; ++q) {
                  const double ri = walkers[(int64_t)(3 * i + q) * ldw + w], rj = walkers[(int64_t)(3 * j + q) * ldw + w];
                  x2 += (ri - wf.atom_xyz[a][q]) * (ri - wf.atom_xyz[a][q]);
                  y2 += (rj - wf.atom_xyz[a][q]) * (rj - wf.atom_xyz[a][q]);
                  z2 += (ri - rj) * (ri - rj);
                }
                const double x = sqrt(x2), y = sqrt(y2), z = sqrt(z2);
                const double d1 = 1.0 + b1 * x, d2 = 1.0 + b2 * y, d3 = 1.0 + b3 * z;
                const double h1 = x / d1, h2 = y / d2, h3 = z / d3;  // df/da
                const double f1 = a1 * h1, f2 = a2 * h2, f3 = a3 * h3;
                g7[0] += 0.5 * f1 * f2 * f3;
                g7[1] += 0.5 * c * h1 * f2 * f3;
                g7[2] -= 0.5 * c * a1 * h1 * h1 * f2 * f3;
                g7[3] += 0.5 * c * f1 * h2 * f3;
                g7[4] -= 0.5 * c * f1 * a2 * h2 * h2 * f3;
                g7[5] += 0.5 * c * f1 * f2 * h3;
                g7[6] -= 0.5 * c * f1 * f2 * a3 * h3 * h3;
              }
        for (int q = 0; q < 7; ++q) {
          const double v = warp_sum(wt * g7[q]);
          if (lane == 0) acc[(size_t)warp * n_param + k + q] += v;
        }
        k += 7;
      }
    }
    if (!live) continue;
    // Gamma per spin
    for (int s = 0; s < 2; ++s) {
      const int n = s == 0 ? nu : wf.n_down, i0 = s == 0 ? 0 : nu;
      const int p_hi = wf.p_hi[s];
      // c_e and Y_{p h}
      double c[kMaxExc > 128 ? 128 : kMaxExc];
      for (int e = 0; e < wf.n_exc[s]; ++e) c[e] = 0.0;
      for (int k = 0; k < wf.n_det; ++k)
        c[wf.det_idx[2 * k + s]] += wf.det_w[k] * R[1 - s][wf.det_idx[2 * k + 1 - s]] * iS;
      double Y[kMdNM][kMdNS];
      for (int p = n; p < p_hi; ++p)
        for (int h = 0; h < n; ++h) Y[p][h] = 0.0;
      for (int e = 0; e < wf.n_exc[s]; ++e) {
        const int* x = wf.exc + (s * kMaxExc + e) * 5;
        if (x[0] == 1) {
          Y[x[3]][x[1]] += c[e];
        } else if (x[0] == 2) {
          Y[x[3]][x[1]] += c[e] * T[s][x[2]][x[4]];
          Y[x[4]][x[2]] += c[e] * T[s][x[1]][x[3]];
          Y[x[4]][x[1]] -= c[e] * T[s][x[2]][x[3]];
          Y[x[3]][x[2]] -= c[e] * T[s][x[1]][x[4]];
        }
      }
      // Z = Y A^-1 (particle rows), then Gamma
      double Z[kMdNM][kMdNS];
      for (int p = n; p < p_hi; ++p)
        for (int a = 0; a < n; ++a) {
          double z = 0.0;
          for (int h = 0; h < n; ++h) z += Y[p][h] * ainv[s][h][a];
          Z[p][a] = z;
        }
      for (int a = 0; a < n; ++a) {
        double* g = gam + (size_t)((i0 + a) * nmo) * ldm + w;
        for (int m = 0; m < nmo; ++m) {
          double v = 0.0;
          if (m < n) {
            v = ainv[s][m][a];
            for (int p = n; p < p_hi; ++p) v -= T[s][m][p] * Z[p][a];
          } else if (m < p_hi) {
            v = Z[m][a];
          }
          g[(size_t)m * ldm] = v;
        }
      }
    }
  }
  flush_acc(acc, n_param, partial, ld_partial, blockIdx.x);
}

// Sum over the warp's lanes of 32 values per lane: afterwards lane L holds the
// sum of every lane's v[L].  Butterfly reduce-scatter in five exchange
// stages (31 adds per lane for 32 outputs, instead of five per output for a
// per-output tree); the order of the additions is fixed.
__device__ __forceinline__ double reduce_scatter32(double (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const double send = upper ? v[k] : v[k + s];
      const double keep = upper ? v[k + s] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

__global__ void __launch_bounds__(kMdThreads) k_md_rows(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                         int64_t ldw, const double* __restrict__ gam, int64_t ldm,
                                                         const double* __restrict__ e_loc,
                                                         const double* __restrict__ stats, int weight,
                                                         const double* __restrict__ ang,
                                                         const int* __restrict__ prim_start, int n_param,
                                                         double* __restrict__ partial, int64_t ld_partial, int col0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GenShared g;
  stage_tables(wf, g, smem_raw);
  const size_t tab_bytes = (sizeof(ShellDev) * wf.n_shell + sizeof(int) * wf.n_ao + 15) & ~size_t(15);
  double* acc = reinterpret_cast<double*>(smem_raw + tab_bytes);  // [kMdWarps][n_param]
  for (int k = threadIdx.x; k < kMdWarps * n_param; k += blockDim.x) acc[k] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = wf.n_elec, nmo = wf.n_mo;
  const int n_prim = prim_start[wf.n_ao];
  const int off_c = n_prim, off_w = off_c + wf.n_ao * nmo + wf.n_det + 1;
  double* my = acc + (size_t)warp * n_param;
  const int64_t rows = (int64_t)N * W;
  const int64_t n_iter = (rows + (int64_t)gridDim.x * kMdThreads - 1) / ((int64_t)gridDim.x * kMdThreads);
  for (int64_t it = 0; it < n_iter; ++it) {
    const int64_t q = (it * gridDim.x + blockIdx.x) * kMdThreads + threadIdx.x;
    const bool live = q < rows;
    const int i = live ? (int)(q / W) : 0;
    const int64_t w = live ? q % W : 0;
    const double wt = live ? walker_weight(weight, e_loc, stats, w, W) : 0.0;
    double r[3], drt[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3; ++c) r[c] = walkers[(int64_t)(3 * i + c) * ldw + w];
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      double v[3], d2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        v[c] = r[c] - walkers[(int64_t)(3 * j + c) * ldw + w];
        d2 += v[c] * v[c];
      }
      const double inv = 1.0 / sqrt(d2);
      for (int c = 0; c < 3; ++c) drt[c] += inv * v[c];
    }
    double G[kMdNM];
    for (int m = 0; m < kMdNM; ++m) G[m] = (live && m < nmo) ? gam[((size_t)i * nmo + m) * ldm + w] : 0.0;
    double gw = 0.0;
    for (int s = 0; s < wf.n_shell; ++s) {
      const ShellDev& sh = g.sh[s];
      const double dx = r[0] - wf.atom_xyz[sh.atom][0], dy = r[1] - wf.atom_xyz[sh.atom][1],
                   dz = r[2] - wf.atom_xyz[sh.atom][2];
      const double r2 = dx * dx + dy * dy + dz * dz, rho = sqrt(r2);
      // radial factor, f'/rho, and per primitive the exponent derivative of
      // its normalised term: d(N_p e^(-alpha r^2)) / d alpha = term ((3/4 + l/2)/alpha - r^2)
      double f = 0.0, g1 = 0.0, dexp[QMC_MAX_PRIM];
      if (sh.kind == 0) {
        double rk = 1.0;
        for (int k = 0; k < sh.kn; ++k) rk *= rho;
        f = sh.coef[0] * rk * exp(-sh.expo[0] * rho);
        g1 = (sh.kn / rho - sh.expo[0]) * f / rho;
        const int nq = sh.kn + sh.l + 1;
        dexp[0] = f * ((nq + 0.5) / sh.expo[0] - rho);
      } else {
        for (int p = 0; p < sh.n_prim; ++p) {
          const double al = sh.expo[p];
          const double term = sh.coef[p] * exp(-al * r2);
          f += term;
          g1 -= 2.0 * al * term;
          dexp[p] = term * ((0.75 + 0.5 * sh.l) / al - r2);
        }
      }
      const double dv[3] = {dx, dy, dz};
      // AOs two at a time: MO-coefficient terms of AO k in slots [16 (k & 1), +16)
      for (int k0 = 0; k0 < sh.n_ao; k0 += 2) {
        double vc[32];
        double ub[2] = {0.0, 0.0}, Pm[2] = {0.0, 0.0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = k0 + h;
          const bool has = k < sh.n_ao;
          const int b = has ? sh.ao_first + k : sh.ao_first;
          const int pw = g.pw[b];
          const int pa[3] = {pw & 15, (pw >> 4) & 15, (pw >> 8) & 15};
          Pm[h] = has ? mono(dx, dy, dz, pa[0], pa[1], pa[2]) : 0.0;
          const double sb = wt * ang[b] * Pm[h] * f;
          const double* Cb = g.C + (size_t)b * nmo;  // angular factor folded in
          double u = 0.0;
#pragma unroll
          for (int m = 0; m < kMdNM; ++m) {
            vc[16 * h + m] = sb * G[m];
            if (m < nmo) u += Cb[m] * G[m];
          }
          ub[h] = has ? u : 0.0;
          // grad (P f) . sum_j (r_a - r_j) / r_aj
          if (has) {
            double gd = 0.0;
            for (int d = 0; d < 3; ++d) {
              double dP = 0.0;
              if (pa[d] > 0) {
                const int e[3] = {pa[0] - (d == 0), pa[1] - (d == 1), pa[2] - (d == 2)};
                dP = pa[d] * mono(dx, dy, dz, e[0], e[1], e[2]);
              }
              gd += (f * dP + Pm[h] * g1 * dv[d]) * drt[d];
            }
            gw += u * gd;
          }
        }
        const double oc = reduce_scatter32(vc, lane);
        {
          const int k = k0 + (lane >> 4), m = lane & 15;
          if (k < sh.n_ao && m < nmo) my[off_c + (sh.ao_first + k) * nmo + m] += oc;
        }
        // exponent terms of the same two AOs: slots [8 h + p]
        double ve[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) ve[t] = 0.0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const double qb = wt * ub[h] * Pm[h];
          for (int p = 0; p < sh.n_prim && p < QMC_MAX_PRIM; ++p) ve[8 * h + p] = qb * dexp[p];
        }
        const double oe = reduce_scatter32(ve, lane);
        {
          const int h = lane >> 3, p = lane & 7, k = k0 + h;
          if (h < 2 && k < sh.n_ao && p < (sh.kind == 0 ? 1 : sh.n_prim)) my[prim_start[sh.ao_first + k] + p] += oe;
        }
      }
    }
    const double v = warp_sum(wt * gw);
    if (lane == 0) my[off_w] += v;
  }
  flush_acc(acc, n_param, partial, ld_partial, col0 + blockIdx.x);
}

bool md_grad_supported(const WfDev& wf) {
  if (wf.bf_w != 0.0) return false;
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  if (ns > kMdNS || wf.n_mo > kMdNM || wf.n_exc[0] > 128 || wf.n_exc[1] > 128) return false;
  return true;
}

size_t md_grad_smem_bytes(const WfDev& wf, int n_param) {
  return gen_table_bytes(wf) + sizeof(double) * kMdWarps * (size_t)n_param;
}

// Scratch of launch_md_grad: Gamma [n_elec][n_mo][ldm] and the partial sums
// [n_param][2 x blocks].
size_t md_grad_scratch_bytes(const WfDev& wf, int64_t ldm, int n_param, int n_sm) {
  return sizeof(double) * ((size_t)wf.n_elec * wf.n_mo * ldm + (size_t)n_param * 2 * 4 * n_sm);
}

cudaError_t launch_md_grad(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                           const double* e_loc, const double* stats, int n_prim, int n_param, double* scratch,
                           double* grad, cudaStream_t st, int weight) {
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int nb = 4 * n_sm;
  double* gam = scratch;
  double* partial = scratch + (size_t)wf.n_elec * wf.n_mo * ws.ldm;
  const int64_t ldp = 2 * nb;
  // parameter blocks of qmc_param_layout: exponents (n_prim), MO
  // coefficients, CI weights, Jastrow b, backflow w
  const int off_d = n_prim + wf.n_ao * wf.n_mo;
  const size_t smem_a = sizeof(double) * kMdWarps * (size_t)n_param;
  cudaError_t e = cudaFuncSetAttribute(k_md_gamma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
  if (e != cudaSuccess) return e;
  k_md_gamma<<<nb, kMdThreads, smem_a, st>>>(wf, walkers, W, ldw, ws.mo, ws.nmp, ws.ldm, e_loc, stats, weight,
                                             n_param, off_d, gam, partial, ldp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem_b = md_grad_smem_bytes(wf, n_param);
  e = cudaFuncSetAttribute(k_md_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
  if (e != cudaSuccess) return e;
  k_md_rows<<<nb, kMdThreads, smem_b, st>>>(wf, walkers, W, ldw, gam, ws.ldm, e_loc, stats, weight, wf.ao_ang,
                                            wf.ao_prim, n_param, partial, ldp, nb);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_row_sums(partial, n_param, (int)ldp, grad, st);
}

}  // namespace qmc
