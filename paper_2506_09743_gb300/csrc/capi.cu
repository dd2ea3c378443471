// C ABI of the engine: wavefunction construction, workspace management and
// the launch sequences of qmc_local_energy / qmc_sample.
//
// Launch sequence of one local-energy evaluation (Sec. 2.2, App. F):
//   k_jastrow   J, grad J, kinJ, V                  (thread per walker)
//   k_ao_mo_*   Phi and (lap + 2 grad J . grad) Phi  (SIMT, or tcgen05 for the
//               mixed forms)
//   k_det       A0^-1, tables, excited determinants, E_L, log|Psi|
// One Metropolis step (App. B): k_propose, the value-only form of the same
// three stages on the proposal, k_accept.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qmc_internal.cuh"
#include "wf_internal.cuh"

using namespace qmc;

namespace {

thread_local std::string g_err;

qmc_status fail(qmc_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

qmc_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return QMC_ERR_CUDA;
}

}  // namespace

qmc_status set_error(qmc_status s, const std::string& msg) { return fail(s, msg); }

namespace {

double dfact(int n) {
  double r = 1.0;
  while (n > 1) { r *= n; n -= 2; }
  return r;
}

double fact(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= k;
  return r;
}



}  // namespace



namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// FP64 flops per walker of the table-method determinant stage (k_det): per
// spin with n electrons, nh holes and nv virtual columns 2n^3 (inverse),
// 2n^2 (Jacobi trace) and nv 2(2n^2 + nh n) (tables); 2 per distinct rank-1
// and 12 per distinct rank-2 spin excitation; 8 per determinant.  exc holds
// the distinct excitation records per spin ([2][kMaxExc][5], rank first).
double det_stage_flops(const WfDev& d, const std::vector<int>& exc) {
  double f = 8.0 * d.n_det;
  for (int s = 0; s < 2; ++s) {
    const double n = s == 0 ? d.n_up : d.n_down;
    if (n == 0) continue;
    f += 2 * n * n * n + 2 * n * n + d.nv[s] * 2.0 * (2 * n * n + d.nh[s] * n);
    for (int i = 1; i < d.n_exc[s]; ++i) {
      const int rank = exc[(s * kMaxExc + i) * 5];
      f += rank == 1 ? 2.0 : rank == 2 ? 12.0 : 0.0;
    }
  }
  return f;
}

size_t ta_size(int prec) { return prec == QMC_FP64 ? 8 : 4; }

size_t workspace_bytes(const qmc_wf* wf, int64_t W) {
  const int64_t ldm = round_up(W > 0 ? W : 1, 32);
  const int N = wf->dev.n_elec;
  const size_t ta = ta_size(wf->precision);
  size_t b = 0;
  b += align256(3 * N * ldm * ta);                     // gradJ
  b += align256(3 * ldm * sizeof(double));             // jscal
  const bool tc = wf->precision == QMC_MIXED_TF32 || wf->precision == QMC_MIXED_BF16;
  b += align256((size_t)N * 2 * mo_row_pad(wf->dev.n_mo, tc) * ldm * sizeof(double));  // MO channels (FP64)
  b += align256(3 * N * ldm * sizeof(double));         // proposals
  b += 2 * align256(ldm * sizeof(double));             // lp, lp_new
  b += align256(sizeof(uint64_t));                     // step counter
  b += align256(sizeof(int));                          // device error flag
  return b;
}

Workspace carve(const qmc_wf* wf, void* base, int64_t W, int** err_flag) {
  Workspace ws{};
  ws.ldm = round_up(W > 0 ? W : 1, 32);
  const int N = wf->dev.n_elec;
  const size_t ta = ta_size(wf->precision);
  char* p = static_cast<char*>(base);
  ws.gradJ = p; p += align256(3 * N * ws.ldm * ta);
  ws.jscal = reinterpret_cast<double*>(p); p += align256(3 * ws.ldm * sizeof(double));
  const bool tc = wf->precision == QMC_MIXED_TF32 || wf->precision == QMC_MIXED_BF16;
  ws.nmp = mo_row_pad(wf->dev.n_mo, tc);
  ws.mo = reinterpret_cast<double*>(p); p += align256((size_t)N * 2 * ws.nmp * ws.ldm * sizeof(double));
  ws.prop = reinterpret_cast<double*>(p); p += align256(3 * N * ws.ldm * sizeof(double));
  ws.lp = reinterpret_cast<double*>(p); p += align256(ws.ldm * sizeof(double));
  ws.lp_new = reinterpret_cast<double*>(p); p += align256(ws.ldm * sizeof(double));
  ws.ctr = reinterpret_cast<uint64_t*>(p); p += align256(sizeof(uint64_t));
  *err_flag = reinterpret_cast<int*>(p);
  return ws;
}

qmc_status get_workspace(qmc_wf* wf, int64_t W, void* user, size_t user_bytes, void** out) {
  const size_t need = workspace_bytes(wf, W);
  if (user) {
    if (user_bytes < need)
      return fail(QMC_ERR_OOM, "workspace too small: need " + std::to_string(need) + " bytes");
    *out = user;
    return QMC_OK;
  }
  if (wf->ws_bytes < need) {
    if (wf->ws) cudaFree(wf->ws);
    wf->ws = nullptr;
    wf->ws_bytes = 0;
    cudaError_t e = cudaMalloc(&wf->ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(QMC_ERR_OOM, std::string("workspace allocation: ") + cudaGetErrorString(e));
    }
    wf->ws_bytes = need;
  }
  *out = wf->ws;
  return QMC_OK;
}

double vnn_of(const WfDev& d) {
  double v = 0.0;
  for (int a = 0; a < d.n_atom; ++a)
    for (int b = a + 1; b < d.n_atom; ++b) {
      const double dx = d.atom_xyz[a][0] - d.atom_xyz[b][0], dy = d.atom_xyz[a][1] - d.atom_xyz[b][1],
                   dz = d.atom_xyz[a][2] - d.atom_xyz[b][2];
      v += d.atom_z[a] * d.atom_z[b] / std::sqrt(dx * dx + dy * dy + dz * dz);
    }
  return v;
}

// Split an FP32 value into TF32 high part (round to nearest, 10 explicit
// mantissa bits) and the FP32 remainder.
uint32_t tf32_hi_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return u;
  u += 0x1000u;  // round half away from zero at bit 13
  return u & 0xffffe000u;
}

float bits_f(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Offset (in 32-bit words) of element (row, k) of a K-major operand stored as
// 8-row x 16-byte core matrices, core matrices along K contiguous (128 B
// apart) and 8-row groups k_pad*4 bytes apart.
size_t core_offset_words(int row, int k, int k_pad) {
  return (size_t)(row / 8) * (k_pad / 4) * 32 + (size_t)(k / 4) * 32 + (row % 8) * 4 + (k % 4);
}

// Position of the Cartesian monomial x^a y^b z^c (a + b + c = l <= 2) in the
// canonical order s; x, y, z; xx, xy, xz, yy, yz, zz.
int tc_canonical_index(int l, int a, int b, int c) {
  if (l == 0) return 0;
  if (l == 1) return a ? 0 : b ? 1 : 2;
  if (a == 2) return 0;
  if (a == 1) return b ? 1 : 2;
  if (b == 2) return 3;
  return b ? 4 : 5;
}

// Row-scale tables of the FP32X2 tensor-core AO stage: for every atom and
// bin [r_lo^2, r_hi^2] of the squared electron-nucleus distance, upper bounds
// over the AOs of the atom's shells of |AO value| (bv) and of the kinetic
// channel, |lap phi + 2 grad J . grad phi| <= bk0 + |grad J| bk1.  Per shell
// (radial sums at rho_lo, powers of rho at rho_hi, the terms of the bound
// the kernel's shells would give one by one):
//   R0 >= sum |c| e^(-a rho^2), R1 >= |f'/rho|, R2 >= |f''|,
//   bv  = R0 rho^l,
//   bk0 = R0 l (l - 1) rho^(l-2) + rho^l (R2 + 2 (l + 1) R1),
//   bk1 = 2 R1 rho^(l+1) + 2 R0 l rho^(l-1).
// The last bin (rho >= 256) takes rho_lo for every factor, valid once each
// radial factor times rho^(l+2) decreases beyond 256 bohr (checked: else no
// table).  Bins are widened by 1e-6 on both sides and the bounds rounded up,
// so FP32 rounding of r^2 on the device cannot leave a bin's bound.
bool oz_bound_table(const std::vector<ShellDev>& shells, int n_atom, std::vector<float>& tab) {
  for (const ShellDev& sh : shells) {
    if (sh.kind == 0) {
      if (sh.expo[0] * 256.0 < sh.kn + sh.l + 3) return false;
    } else {
      for (int p = 0; p < sh.n_prim; ++p)
        if (2.0 * sh.expo[p] * 65536.0 < sh.l + 3) return false;
    }
  }
  std::vector<double> acc((size_t)n_atom * kOzBoundBins * 3, 0.0);
  for (int k = 1; k < kOzBoundBins; ++k) {
    double rlo, rhi;
    if (k == kOzBoundBins - 1) {
      rlo = 256.0 * (1.0 - 1e-6);
      rhi = rlo;
    } else {
      const uint32_t u0 = (uint32_t)(k - 1 + kOzBoundBase) << 19, u1 = (uint32_t)(k + kOzBoundBase) << 19;
      float f0, f1;
      std::memcpy(&f0, &u0, 4);
      std::memcpy(&f1, &u1, 4);
      rlo = std::sqrt((double)f0) * (1.0 - 1e-6);
      rhi = std::sqrt((double)f1) * (1.0 + 1e-6);
    }
    for (const ShellDev& sh : shells) {
      double R0 = 0.0, R1 = 0.0, R2 = 0.0;
      if (sh.kind == 0) {
        const double F = std::fabs(sh.coef[0]) * std::pow(rhi, sh.kn) * std::exp(-sh.expo[0] * rlo);
        const double Q = sh.kn / rlo + sh.expo[0];
        R0 = F;
        R1 = Q * F / rlo;
        R2 = (Q * Q + sh.kn / (rlo * rlo)) * F;
      } else {
        for (int p = 0; p < sh.n_prim; ++p) {
          const double a = sh.expo[p], ce = std::fabs(sh.coef[p]) * std::exp(-a * rlo * rlo);
          R0 += ce;
          R1 += 2.0 * a * ce;
          R2 += (4.0 * a * a * rhi * rhi + 2.0 * a) * ce;
        }
      }
      const int l = sh.l;
      const double rl = std::pow(rhi, l), rl1 = l >= 1 ? std::pow(rhi, l - 1) : 0.0,
                   rl2 = l >= 2 ? std::pow(rhi, l - 2) : 0.0;
      const double bv = R0 * rl;
      const double bk0 = R0 * l * (l - 1) * rl2 + rl * (R2 + 2.0 * (l + 1) * R1);
      const double bk1 = 2.0 * R1 * rhi * rl + 2.0 * R0 * l * rl1;
      double* t = &acc[((size_t)sh.atom * kOzBoundBins + k) * 3];
      t[0] = std::max(t[0], bv);
      t[1] = std::max(t[1], bk0);
      t[2] = std::max(t[2], bk1);
    }
  }
  tab.assign((size_t)n_atom * kOzBoundBins * 4, 0.0f);
  for (size_t i = 0; i < (size_t)n_atom * kOzBoundBins; ++i)
    for (int c = 0; c < 3; ++c) {
      const double v = acc[i * 3 + c] * (1.0 + 1e-6);
      float f = (float)v;
      if ((double)f < v) f = std::nextafter(f, std::numeric_limits<float>::infinity());
      tab[i * 4 + c] = f;
    }
  return true;
}

qmc_status launch_status(cudaError_t e, const char* where) {
  return e == cudaSuccess ? QMC_OK : cuda_fail(e, where);
}

// Validate wf->spec and (re)build every device table from it.  On failure the
// previous tables (if any) are kept.
qmc_status build_tables(qmc_wf* wf) {
  const HostSpec& h = wf->spec;
  const int na = h.na, nup = h.nup, ndn = h.ndn, nao = h.nao, nmo = h.nmo, ndet = h.ndet;
  const int prec = wf->precision;
  const bool tc = prec == QMC_MIXED_TF32 || prec == QMC_MIXED_BF16;
  if (tc && nmo > 16) return fail(QMC_ERR_UNSUPPORTED, "tensor-core forms need n_mo <= 16");
  if (prec == QMC_MIXED_BF16) return fail(QMC_ERR_UNSUPPORTED, "BF16 form not built");
  WfDev d{};
  d.n_atom = na;
  d.n_up = nup;
  d.n_down = ndn;
  d.n_elec = nup + ndn;
  d.n_ao = nao;
  d.n_mo = nmo;
  d.n_det = ndet;
  d.w0_par = h.w0p;
  d.w0_anti = h.w0a;
  d.jb = h.b;
  d.w0p_f = (float)h.w0p;
  d.w0a_f = (float)h.w0a;
  d.jb_f = (float)h.b;
  d.bf_w = h.w;
  for (int a = 0; a < na; ++a) {
    for (int k = 0; k < 3; ++k) d.atom_xyz[a][k] = h.xyz[3 * a + k];
    d.atom_z[a] = h.z[a];
  }
  d.vnn = vnn_of(d);
  d.wait_cycles = wf->wait_cycles;
  if (h.w != 0.0 && prec != QMC_FP64 && prec != QMC_FP32X2)
    return fail(QMC_ERR_UNSUPPORTED, "backflow wavefunctions run in the FP64 and FP32X2 forms only");
  // FP32X2 with backflow: the general kernels take the orbitals in pairs of FP32
  d.gen_x2 = (h.w != 0.0 && prec == QMC_FP32X2) ? 1 : 0;
  d.mb_en = h.jen.empty() ? 0 : 1;
  d.n_een = (int)(h.jeen.size() / 7);
  for (int k = 0; k < 3; ++k) {
    d.jen[k] = d.mb_en ? h.jen[k] : 0.0;
    d.jen_f[k] = (float)d.jen[k];
  }
  for (int t = 0; t < d.n_een; ++t)
    for (int k = 0; k < 7; ++k) {
      d.jeen[t][k] = h.jeen[7 * t + k];
      d.jeen_f[t][k] = (float)d.jeen[t][k];
    }
  if (h.w != 0.0 && (d.mb_en || d.n_een))
    return fail(QMC_ERR_UNSUPPORTED, "the many-body Jastrow is not combined with backflow");
  if (d.n_een && een_shared_bytes(d, prec == QMC_FP64) > 227 * 1024)
    return fail(QMC_ERR_UNSUPPORTED, "electron-electron-nucleus Jastrow tables exceed shared memory");

  // ---- basis: shells, normalisation, angular factors
  std::vector<ShellDev> shells;
  std::vector<int> ao_pow(nao);
  std::vector<double> ang(nao);
  for (int b = 0; b < nao; ++b) {
    const int atom = h.ao_atom[b], kind = h.ao_kind[b];
    const int kx = h.ao_pow[4 * b], ky = h.ao_pow[4 * b + 1], kz = h.ao_pow[4 * b + 2], kn = h.ao_pow[4 * b + 3];
    const int s0 = h.prim_start[b], s1 = h.prim_start[b + 1];
    if (atom < 0 || atom >= na || (kind != 0 && kind != 1) || kx < 0 || ky < 0 || kz < 0 || kn < 0 || kx > 4 ||
        ky > 4 || kz > 4 || kx + ky + kz > 4 || kn > 8 || s1 <= s0 || (kind == 0 && s1 - s0 != 1) ||
        s1 - s0 > QMC_MAX_PRIM)
      return fail(QMC_ERR_ARG, "bad AO " + std::to_string(b));
    for (int p = s0; p < s1; ++p)
      if (!(h.prim_exp[p] > 0.0) || !std::isfinite(h.prim_exp[p]))
        return fail(QMC_ERR_ARG, "AO exponents must be positive and finite (AO " + std::to_string(b) + ")");
    const int l = kx + ky + kz;
    ao_pow[b] = kx | (ky << 4) | (kz << 8);
    const double df = dfact(2 * kx - 1) * dfact(2 * ky - 1) * dfact(2 * kz - 1);
    ShellDev sh{};
    sh.atom = atom;
    sh.kind = kind;
    sh.kn = kind == 0 ? kn : 0;
    sh.l = l;
    sh.n_prim = s1 - s0;
    sh.ao_first = b;
    sh.n_ao = 1;
    if (kind == 0) {
      const double zeta = h.prim_exp[s0];
      const int n = kn + l + 1;
      ang[b] = std::sqrt(dfact(2 * l + 1) / (4.0 * M_PI * df));
      sh.expo[0] = zeta;
      sh.coef[0] = h.prim_coef[s0] * std::pow(2.0 * zeta, n + 0.5) / std::sqrt(fact(2 * n));
      sh.expo_f[0] = (float)sh.expo[0];
      sh.coef_f[0] = (float)sh.coef[0];
    } else {
      ang[b] = 1.0 / std::sqrt(df);
      for (int p = s0; p < s1; ++p) {
        const double al = h.prim_exp[p];
        sh.expo[p - s0] = al;
        sh.coef[p - s0] = h.prim_coef[p] * std::pow(2.0 * al / M_PI, 0.75) * std::pow(4.0 * al, 0.5 * l);
        sh.expo_f[p - s0] = (float)sh.expo[p - s0];
        sh.coef_f[p - s0] = (float)sh.coef[p - s0];
      }
    }
    bool merged = false;
    if (!shells.empty()) {
      ShellDev& q = shells.back();
      if (q.atom == sh.atom && q.kind == sh.kind && q.kn == sh.kn && q.l == sh.l && q.n_prim == sh.n_prim &&
          q.ao_first + q.n_ao == b && q.n_ao < kMaxShellAo) {
        bool same = true;
        for (int p = 0; p < sh.n_prim; ++p) same = same && q.expo[p] == sh.expo[p] && q.coef[p] == sh.coef[p];
        if (same) { q.n_ao += 1; merged = true; }
      }
    }
    if (!merged) shells.push_back(sh);
  }
  if ((int)shells.size() > kMaxShells) return fail(QMC_ERR_UNSUPPORTED, "too many shells");
  d.n_shell = (int)shells.size();
  // ---- pairs of FP32 of the shell parameters (FP32X2 form), and the
  // canonical order of complete s, p and d shells: the FP32X2 kernel
  // evaluates such a shell's AOs in closed form in the order s; x, y, z; xx,
  // xy, xz, yy, yz, zz and reads MO-table row x2_row[b] for AO b
  std::vector<int> x2_row(nao);
  for (ShellDev& q : shells) {
    for (int p = 0; p < q.n_prim; ++p) {
      q.expo_lo[p] = (float)(q.expo[p] - (double)q.expo_f[p]);
      q.coef_lo[p] = (float)(q.coef[p] - (double)q.coef_f[p]);
      // 2 alpha c and 4 alpha^2 c: the GTO kinetic radial sums as pair
      // multiply-accumulates with e^(-alpha r^2)
      const double c2 = 2.0 * q.expo[p] * q.coef[p], c4 = 4.0 * q.expo[p] * q.expo[p] * q.coef[p];
      q.c2a_f[p] = (float)c2;
      q.c2a_lo[p] = (float)(c2 - (double)q.c2a_f[p]);
      q.c4a_f[p] = (float)c4;
      q.c4a_lo[p] = (float)(c4 - (double)q.c4a_f[p]);
    }
    std::vector<int> canon(q.n_ao, -1);
    bool complete = q.l <= 2 && q.n_ao == (q.l + 1) * (q.l + 2) / 2;
    for (int k = 0; k < q.n_ao && complete; ++k) {
      const int pw = ao_pow[q.ao_first + k];
      const int j = tc_canonical_index(q.l, pw & 15, (pw >> 4) & 15, (pw >> 8) & 15);
      for (int k2 = 0; k2 < k; ++k2) complete = complete && canon[k2] != j;
      canon[k] = j;
    }
    q.canon = complete ? 1 + q.l : 0;
    for (int k = 0; k < q.n_ao; ++k) x2_row[q.ao_first + k] = q.ao_first + (complete ? canon[k] : k);
  }
  // ---- tensor-core AO stage: pack the shells into K-passes of kTcPass
  // columns, then deal each pass's shells to the four thread parts by
  // estimated cost, largest first, each part's list kept in shell order so
  // that shells of one atom stay together.  Within each atom the complete d
  // shells are placed first, on columns = 0 (mod 4), then the complete p
  // shells on even columns, then the rest into the first free columns (the
  // gaps the alignment leaves), so that the kernel writes a d shell's first
  // four columns with one 16-byte store and pairs of p and d columns with
  // 8-byte stores; a shell that does not fit in the pass starts the next one.
  std::vector<int> ao_col(nao, 0), tc_shells;
  d.n_pass = 0;
  if (tc || prec == QMC_FP32X2) {
    std::vector<int> shell_col(d.n_shell), shell_type(d.n_shell), shell_pass(d.n_shell);
    std::vector<int> canon_all(nao, 0);
    for (int s = 0; s < d.n_shell; ++s) {
      const ShellDev& q = shells[s];
      // a complete Cartesian s, p or d shell gets its columns in the
      // canonical order (x, y, z / xx, xy, xz, yy, yz, zz), which the kernel
      // evaluates without per-AO power lookups
      std::vector<int> canon(q.n_ao, -1);
      bool complete = q.l <= 2 && q.n_ao == (q.l + 1) * (q.l + 2) / 2;
      for (int k = 0; k < q.n_ao && complete; ++k) {
        const int pw = ao_pow[q.ao_first + k];
        const int j = tc_canonical_index(q.l, pw & 15, (pw >> 4) & 15, (pw >> 8) & 15);
        for (int k2 = 0; k2 < k; ++k2) complete = complete && canon[k2] != j;
        canon[k] = j;
      }
      shell_type[s] = complete ? 1 + q.l : 0;
      for (int k = 0; k < q.n_ao; ++k) canon_all[q.ao_first + k] = complete ? canon[k] : k;
    }
    // placement order: atom by atom (shell order), d first, then p, then the rest
    std::vector<int> order;
    for (int s0 = 0; s0 < d.n_shell;) {
      int s1 = s0;
      while (s1 < d.n_shell && shells[s1].atom == shells[s0].atom) ++s1;
      for (int want : {3, 2, -1})
        for (int s = s0; s < s1; ++s)
          if ((want >= 0 && shell_type[s] == want) || (want < 0 && shell_type[s] != 3 && shell_type[s] != 2))
            order.push_back(s);
      s0 = s1;
    }
    unsigned used = 0;  // columns taken in the current pass
    int pass = 0;
    std::vector<unsigned> pass_used;
    for (int s : order) {
      const ShellDev& q = shells[s];
      const int align = shell_type[s] == 3 ? 4 : shell_type[s] == 2 ? 2 : 1;
      const unsigned span = q.n_ao >= 32 ? 0xFFFFFFFFu : ((1u << q.n_ao) - 1u);
      int c = -1;
      for (int tries = 0; tries < 2 && c < 0; ++tries) {
        for (int k = 0; k + q.n_ao <= kTcPass; k += align)
          if (((span << k) & used) == 0) { c = k; break; }
        if (c < 0) {  // start the next pass
          pass_used.push_back(used);
          used = 0;
          ++pass;
        }
      }
      if (c < 0) return fail(QMC_ERR_UNSUPPORTED, "an AO shell wider than a tensor-core pass");
      used |= span << c;
      shell_col[s] = c;
      shell_pass[s] = pass;
      for (int k = 0; k < q.n_ao; ++k) ao_col[q.ao_first + k] = pass * kTcPass + c + canon_all[q.ao_first + k];
    }
    pass_used.push_back(used);
    d.n_pass = (int)pass_used.size();
    std::vector<int> lists, lists2;  // shell lists in four and in two parts per row
    if (d.n_pass > kMaxTcPass) return fail(QMC_ERR_UNSUPPORTED, "too many AO passes");
    for (int p = 0; p < d.n_pass; ++p) {
      d.pass_zero[p] = ~pass_used[p];
      std::vector<int> by_cost;
      for (int s = 0; s < d.n_shell; ++s)
        if (shell_pass[s] == p) by_cost.push_back(s);
      // issue cost of a shell in the pair kernels: ~140 FP32 operations per
      // primitive (exponential, radial sums), ~100 per AO (angular factor,
      // kinetic channel, digits of both channels), ~40 per shell
      auto cost = [&](int s) { return 14 * shells[s].n_prim + 10 * shells[s].n_ao + 4; };
      std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return cost(a) > cost(b); });
      // split of the pass's shells over np parts: greedy, largest cost first;
      // two parts of at most 20 shells take the best of all subsets instead
      auto split = [&](int np, int* off) {
        std::vector<std::vector<int>> part(np);
        std::vector<int> load(np, 0);
        const int n = (int)by_cost.size();
        if (np == 2 && n <= 20) {
          int total = 0;
          for (int s : by_cost) total += cost(s);
          unsigned best = 0;
          int best_max = total + 1;
          for (unsigned m = 0; m < (1u << n); m += 2) {  // shell 0 (the costliest) stays in part 0
            int a = 0;
            for (int k = 0; k < n; ++k)
              if ((m >> k) & 1u) a += cost(by_cost[k]);
            const int mx = std::max(a, total - a);
            if (mx < best_max) { best_max = mx; best = m; }
          }
          for (int k = 0; k < n; ++k) part[(best >> k) & 1u].push_back(by_cost[k]);
        } else {
          for (int s : by_cost) {
            const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            part[q].push_back(s);
            load[q] += cost(s);
          }
        }
        for (int q = 0; q < np; ++q) {
          std::sort(part[q].begin(), part[q].end());
          off[q] = (int)lists.size();
          for (int s : part[q]) lists.push_back(s | (shell_col[s] << 8) | (shell_type[s] << 16));
        }
        off[np] = (int)lists.size();
      };
      split(4, d.part_off[p]);
      std::swap(lists, lists2);
      split(2, d.part2_off[p]);
      std::swap(lists, lists2);
    }
    // the two-part lists follow the four-part ones
    for (int p = 0; p < d.n_pass; ++p)
      for (int q = 0; q < 3; ++q) d.part2_off[p][q] += d.n_shell;
    tc_shells = lists;
    tc_shells.insert(tc_shells.end(), lists2.begin(), lists2.end());
  }
  if (d.gen_x2)
    for (const ShellDev& q : shells)
      if (q.l > 1) return fail(QMC_ERR_UNSUPPORTED, "the FP32X2 form with backflow covers s and p shells");
  std::vector<double> mo64((size_t)nao * nmo);
  std::vector<float> mo32((size_t)nao * nmo);
  std::vector<float> mo_x2((size_t)nao * nmo * 2);  // rows in x2_row order, (hi, lo)
  std::vector<float> mo_x2n((size_t)nao * nmo * 2);  // rows in AO order, (hi, lo)
  for (int b = 0; b < nao; ++b)
    for (int m = 0; m < nmo; ++m) {
      const double c = h.mo[(size_t)b * nmo + m] * ang[b];
      mo64[(size_t)b * nmo + m] = c;
      mo32[(size_t)b * nmo + m] = (float)c;
      const size_t o = 2 * ((size_t)x2_row[b] * nmo + m);
      mo_x2[o] = (float)c;
      mo_x2[o + 1] = (float)(c - (double)(float)c);
      mo_x2n[2 * ((size_t)b * nmo + m)] = (float)c;
      mo_x2n[2 * ((size_t)b * nmo + m) + 1] = (float)(c - (double)(float)c);
    }
  // 2^(j/64), j = 0..63, as pairs of FP32 for the FP32X2 exponential
  std::vector<float> exp_tab(128);
  for (int j = 0; j < 64; ++j) {
    const long double v = std::exp2((long double)j / 64.0L);
    exp_tab[2 * j] = (float)v;
    exp_tab[2 * j + 1] = (float)(v - (long double)exp_tab[2 * j]);
  }

  // ---- determinants: unique excitation records per spin.  The expansion is
  // stored sorted by (rank up, rank down): the determinant stage hands
  // consecutive determinants to the lanes of a warp, and a sorted list keeps
  // their rank branches uniform (the sum is order independent).
  std::vector<int> order(ndet);
  for (int n = 0; n < ndet; ++n) order[n] = n;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return h.det_exc[a * 10] * 3 + h.det_exc[a * 10 + 5] < h.det_exc[b * 10] * 3 + h.det_exc[b * 10 + 5];
  });
  std::vector<double> det_w_sorted(ndet);
  for (int n = 0; n < ndet; ++n) det_w_sorted[n] = h.det_w[order[n]];
  std::vector<int> exc(2 * kMaxExc * 5, -1);
  std::vector<int> det_idx(2 * ndet);
  for (int s = 0; s < 2; ++s) {
    const int ns = s == 0 ? nup : ndn;
    std::map<std::vector<int>, int> seen;
    std::vector<int> g = {0, -1, -1, -1, -1};
    seen[g] = 0;
    for (int k = 0; k < 5; ++k) exc[(s * kMaxExc + 0) * 5 + k] = g[k];
    int h_lo = ns, p_hi = ns;
    for (int n = 0; n < ndet; ++n) {
      const int src = order[n];
      std::vector<int> e(h.det_exc.begin() + (src * 2 + s) * 5, h.det_exc.begin() + (src * 2 + s) * 5 + 5);
      const int rank = e[0];
      bool ok = rank >= 0 && rank <= 2;
      if (ok && rank == 0) e = g;
      if (ok && rank >= 1) ok = e[1] >= 0 && e[1] < ns && e[3] >= ns && e[3] < nmo;
      if (ok && rank == 2) ok = e[2] > e[1] && e[2] < ns && e[4] > e[3] && e[4] < nmo;
      if (ok && rank == 1) { e[2] = -1; e[4] = -1; }
      if (!ok) return fail(QMC_ERR_ARG, "bad excitation record of determinant " + std::to_string(src));
      auto it = seen.find(e);
      int idx;
      if (it == seen.end()) {
        idx = (int)seen.size();
        if (idx >= kMaxExc) return fail(QMC_ERR_UNSUPPORTED, "too many distinct excitations");
        seen[e] = idx;
        for (int k = 0; k < 5; ++k) exc[(s * kMaxExc + idx) * 5 + k] = e[k];
      } else {
        idx = it->second;
      }
      det_idx[2 * n + s] = idx;
      if (rank >= 1) { h_lo = std::min(h_lo, e[1]); p_hi = std::max(p_hi, e[3] + 1); }
      if (rank == 2) { p_hi = std::max(p_hi, e[4] + 1); }
    }
    d.n_exc[s] = (int)seen.size();
    d.h_lo[s] = h_lo;
    d.p_hi[s] = p_hi;
    d.nh[s] = ns - h_lo;
    d.nv[s] = p_hi - ns;
  }
  d.tab_elems = 2 * (d.nh[0] * d.nv[0] + d.nh[1] * d.nv[1]);
  // per determinant and spin: the table offsets (h_a - h_lo) nv + (p_b - n_s)
  // of its k x k block packed into one word (8 bits each; nh nv <= 8 x 24)
  // and its rank, so the determinant stage reads one record per determinant
  std::vector<int> det_tab(4 * (size_t)ndet);
  for (int n = 0; n < ndet; ++n)
    for (int s = 0; s < 2; ++s) {
      const int ns = s == 0 ? nup : ndn, hl = d.h_lo[s], nv = d.nv[s];
      const int* e = &exc[(s * kMaxExc + det_idx[2 * n + s]) * 5];
      auto q = [&](int hh, int pp) { return (hh - hl) * nv + (pp - ns); };
      int packed = 0;
      if (e[0] >= 1) packed = q(e[1], e[3]);
      if (e[0] == 2) packed |= (q(e[1], e[4]) << 8) | (q(e[2], e[3]) << 16) | (q(e[2], e[4]) << 24);
      det_tab[4 * n + 2 * s] = packed;
      det_tab[4 * n + 2 * s + 1] = e[0];
    }
  // The FP32X2 form's determinant stage.  k_det_x2 (pairs of FP32, eight
  // lanes per spin block) has a fixed cost per walker that the FP64 stage
  // k_det (one thread per spin block) does not; it pays where the tables and
  // the expansion make the FP64 work large.  Measured det-stage times on
  // 262,144 walkers of the CO basis with n electrons per spin (k_det /
  // k_det_x2, ms): one determinant 0.09 / 0.31 (n = 2) ... 0.52 / 0.61 (n = 7);
  // 100 determinants 0.66 / 0.72 (n = 3, 2,484 FP64 flops per walker),
  // 0.89 / 0.81 (n = 4, 3,462 flops), 1.72 / 1.14 (n = 7, 6,486 flops).
  d.det_x2 = (prec == QMC_FP32X2 && det_stage_flops(d, exc) >= 3000.0) ? 1 : 0;
  if (d.det_x2 && det_x2_smem_bytes(d, true) > 227 * 1024) d.det_x2 = 0;
  if (h.w != 0.0 && !general_supported(d) && !bf_multidet_supported(d))
    return fail(QMC_ERR_UNSUPPORTED,
                "backflow needs <= 8 electrons, <= 4 per spin and (several determinants) <= 8 orbital columns");
  if (det_smem_bytes(d, true) > 227 * 1024)
    return fail(QMC_ERR_UNSUPPORTED, "determinant stage exceeds shared memory (too many MOs or excitations)");

  // ---- tensor-core B operand (MO^T, N = 16 rows, K = k_pad), TF32 hi/lo
  d.k_pad = (tc || prec == QMC_FP32X2) ? d.n_pass * kTcPass : 0;
  if (tc && tc_smem_bytes(d, 2) > 227 * 1024)
    return fail(QMC_ERR_UNSUPPORTED, "tensor-core AO stage exceeds shared memory (too many AOs or shells)");
  // the FP32X2 form's Metropolis value path (log|Psi| for the acceptance
  // test) runs the FP32-AO tensor-core stage when it fits
  d.tc_value = (prec == QMC_FP32X2 && nmo <= 16 && d.n_pass > 0 && tc_smem_bytes(d, 1) <= 227 * 1024) ? 1 : 0;
  std::vector<uint32_t> tc_hi, tc_lo;
  if (tc || d.tc_value) {
    tc_hi.assign((size_t)16 * d.k_pad, 0u);
    tc_lo.assign((size_t)16 * d.k_pad, 0u);
    for (int m = 0; m < nmo; ++m)
      for (int b = 0; b < nao; ++b) {
        const float v = mo32[(size_t)b * nmo + m];
        const uint32_t hi = tf32_hi_bits(v);
        const float lo = v - bits_f(hi);
        uint32_t lo_bits;
        std::memcpy(&lo_bits, &lo, 4);
        const size_t off = core_offset_words(m, ao_col[b], d.k_pad);
        tc_hi[off] = hi;
        tc_lo[off] = tf32_hi_bits(bits_f(lo_bits));
      }
  }

  // ---- FP32X2 form on the tensor cores: MO column m scaled by 2^-f_m
  // (max |C_bm| < 2^f_m) and written as six balanced digits of 8 bits,
  // exactly (FP64 steps), as BF16 in the K-major core-matrix layout
  std::vector<uint16_t> mo_oz;
  d.oz = 0;
  for (int m = 0; m < 16; ++m) d.oz_colexp[m] = 0;
  if (prec == QMC_FP32X2 && nmo <= 16 && d.n_pass > 0) {
    const int kp = d.k_pad;
    mo_oz.assign((size_t)6 * 16 * kp, 0);
    for (int m = 0; m < nmo; ++m) {
      double cmax = 0.0;
      for (int b = 0; b < nao; ++b) cmax = std::max(cmax, std::fabs(mo64[(size_t)b * nmo + m]));
      int f = 0;
      if (cmax > 0.0) std::frexp(cmax, &f);  // cmax = x 2^f, x in [0.5, 1)
      d.oz_colexp[m] = f;
      for (int b = 0; b < nao; ++b) {
        double y = std::ldexp(mo64[(size_t)b * nmo + m], -f);
        const int k = ao_col[b];
        const size_t off = (size_t)(m / 8) * (kp / 8) * 64 + (size_t)(k / 8) * 64 + (m % 8) * 8 + (k % 8);
        for (int l = 0; l < 6; ++l) {
          y *= 256.0;
          const double dl = std::nearbyint(y);
          y -= dl;
          const float df = (float)dl;  // |dl| <= 256: exact in BF16
          uint32_t u;
          std::memcpy(&u, &df, 4);
          mo_oz[(size_t)l * 16 * kp + off] = (uint16_t)(u >> 16);
        }
      }
    }
    d.oz = 1;  // confirmed by oz_supported below, once the other tables are known
  }
  std::vector<float> oz_bnd;
  const bool have_bnd = d.oz && oz_bound_table(shells, d.n_atom, oz_bnd);

  // ---- upload everything in one blob
  DeviceGuard guard(wf->device);
  std::vector<std::pair<const void*, size_t>> parts = {
      {shells.data(), sizeof(ShellDev) * shells.size()}, {ao_pow.data(), sizeof(int) * nao},
      {mo64.data(), sizeof(double) * mo64.size()},       {mo32.data(), sizeof(float) * mo32.size()},
      {exc.data(), sizeof(int) * exc.size()},           {det_idx.data(), sizeof(int) * det_idx.size()},
      {det_w_sorted.data(), sizeof(double) * ndet},      {tc_hi.data(), sizeof(uint32_t) * tc_hi.size()},
      {tc_lo.data(), sizeof(uint32_t) * tc_lo.size()},  {ang.data(), sizeof(double) * nao},
      {h.prim_start.data(), sizeof(int) * (nao + 1)}, {ao_col.data(), sizeof(int) * nao},
      {tc_shells.data(), sizeof(int) * tc_shells.size()}, {det_tab.data(), sizeof(int) * det_tab.size()},
      {mo_x2.data(), sizeof(float) * mo_x2.size()},      {exp_tab.data(), sizeof(float) * exp_tab.size()},
      {mo_oz.data(), sizeof(uint16_t) * mo_oz.size()},  {oz_bnd.data(), sizeof(float) * oz_bnd.size()},
      {order.data(), sizeof(int) * order.size()},        {mo_x2n.data(), sizeof(float) * mo_x2n.size()}};
  size_t total = 0;
  for (auto& p : parts) total += align256(p.second);
  void* blob = nullptr;
  cudaError_t e = cudaMalloc(&blob, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(QMC_ERR_OOM, std::string("table allocation: ") + cudaGetErrorString(e));
  }
  std::vector<char*> ptr;
  char* base = static_cast<char*>(blob);
  for (auto& p : parts) {
    ptr.push_back(base);
    if (p.second) {
      e = cudaMemcpy(base, p.first, p.second, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        cudaFree(blob);
        return cuda_fail(e, "table upload");
      }
    }
    base += align256(p.second);
  }
  d.shells = reinterpret_cast<const ShellDev*>(ptr[0]);
  d.ao_pow = reinterpret_cast<const int*>(ptr[1]);
  d.mo64 = reinterpret_cast<const double*>(ptr[2]);
  d.mo32 = reinterpret_cast<const float*>(ptr[3]);
  d.exc = reinterpret_cast<const int*>(ptr[4]);
  d.det_idx = reinterpret_cast<const int*>(ptr[5]);
  d.det_w = reinterpret_cast<const double*>(ptr[6]);
  d.mo_tc_hi = reinterpret_cast<const uint32_t*>(ptr[7]);
  d.mo_tc_lo = reinterpret_cast<const uint32_t*>(ptr[8]);
  d.ao_ang = reinterpret_cast<const double*>(ptr[9]);
  d.ao_prim = reinterpret_cast<const int*>(ptr[10]);
  d.ao_col = reinterpret_cast<const int*>(ptr[11]);
  d.tc_shells = reinterpret_cast<const int*>(ptr[12]);
  d.det_tab = reinterpret_cast<const int4*>(ptr[13]);
  d.mo_x2 = reinterpret_cast<const float2*>(ptr[14]);
  d.exp_tab = reinterpret_cast<const float*>(ptr[15]);
  d.mo_oz = reinterpret_cast<const uint16_t*>(ptr[16]);
  d.oz_bound = have_bnd ? reinterpret_cast<const float4*>(ptr[17]) : nullptr;
  d.det_orig = reinterpret_cast<const int*>(ptr[18]);
  d.mo_x2n = reinterpret_cast<const float2*>(ptr[19]);
  // the SIMT pair kernel serves this wavefunction when the tensor-core stage
  // does not fit, or when the contraction is too small to pay for it (H2 and
  // LiH: n_ao x n_mo of 2 and 72, where k_ao_mo_x2 measured 1.1-2.1x faster at
  // 1,024-65,536 walkers; CO, 812: k_ao_mo_oz 1.2x faster at every size)
  if (d.oz && (!oz_supported(d) || nao * nmo < 256)) d.oz = 0;
  // the previous tables may still be read by work in flight on any stream
  if (wf->blob) {
    cudaDeviceSynchronize();
    cudaFree(wf->blob);
  }
  wf->blob = blob;
  wf->dev = d;
  return QMC_OK;
}

}  // namespace

extern "C" {

qmc_status qmc_create_wf(const qmc_atoms* atoms, const qmc_basis* basis, const qmc_mos* mos, const qmc_dets* dets,
                         const qmc_jastrow* jastrow, const qmc_options* opt, qmc_wf** out) {
  if (!atoms || !basis || !mos || !dets || !jastrow || !opt || !out) return fail(QMC_ERR_ARG, "null argument");
  *out = nullptr;
  const int na = atoms->n_atom, nup = atoms->n_up, ndn = atoms->n_down;
  if (na < 1 || na > QMC_MAX_ATOMS || !atoms->xyz || !atoms->z) return fail(QMC_ERR_ARG, "bad atoms");
  if (nup < 0 || ndn < 0 || nup + ndn < 1) return fail(QMC_ERR_ARG, "bad electron counts");
  if (nup > QMC_MAX_SPIN_ELECTRONS || ndn > QMC_MAX_SPIN_ELECTRONS)
    return fail(QMC_ERR_UNSUPPORTED, "more than 8 electrons per spin");
  const int nao = basis->n_ao, nmo = mos->n_mo;
  if (nao < 1 || nao > QMC_MAX_AO || !basis->ao_atom || !basis->ao_kind || !basis->ao_pow ||
      !basis->ao_prim_start || !basis->prim_exp || !basis->prim_coef)
    return fail(QMC_ERR_ARG, "bad basis");
  if (nmo < 1 || nmo > QMC_MAX_MO || !mos->coeff) return fail(QMC_ERR_ARG, "bad MO table");
  if (nmo < nup || nmo < ndn) return fail(QMC_ERR_ARG, "fewer MOs than electrons of one spin");
  const int prec = opt->precision;
  if (prec < QMC_FP64 || prec > QMC_FP32X2) return fail(QMC_ERR_ARG, "bad precision");
  if (!dets->weight || !dets->exc || dets->n_det < 1 || dets->n_det > kMaxDets)
    return fail(QMC_ERR_ARG, "bad determinant list");
  const int n_prim = basis->ao_prim_start[nao];
  if (basis->ao_prim_start[0] != 0 || n_prim < nao || n_prim > nao * QMC_MAX_PRIM)
    return fail(QMC_ERR_ARG, "bad primitive offsets");

  qmc_wf* wf = new qmc_wf();
  wf->device = opt->device;
  wf->precision = prec;
  HostSpec& h = wf->spec;
  h.na = na; h.nup = nup; h.ndn = ndn; h.nao = nao; h.nmo = nmo; h.ndet = dets->n_det;
  h.xyz.assign(atoms->xyz, atoms->xyz + 3 * na);
  h.z.assign(atoms->z, atoms->z + na);
  h.ao_atom.assign(basis->ao_atom, basis->ao_atom + nao);
  h.ao_kind.assign(basis->ao_kind, basis->ao_kind + nao);
  h.ao_pow.assign(basis->ao_pow, basis->ao_pow + 4 * nao);
  h.prim_start.assign(basis->ao_prim_start, basis->ao_prim_start + nao + 1);
  h.prim_exp.assign(basis->prim_exp, basis->prim_exp + n_prim);
  h.prim_coef.assign(basis->prim_coef, basis->prim_coef + n_prim);
  h.mo.assign(mos->coeff, mos->coeff + (size_t)nao * nmo);
  h.det_w.assign(dets->weight, dets->weight + dets->n_det);
  h.det_exc.assign(dets->exc, dets->exc + 10 * (size_t)dets->n_det);
  h.w0p = jastrow->w0_par; h.w0a = jastrow->w0_anti; h.b = jastrow->b; h.w = jastrow->backflow_w;
  qmc_status st = build_tables(wf);
  if (st == QMC_OK) {  // the sticky status word of the bounded device waits, and its host mirror
    DeviceGuard guard(wf->device);
    cudaError_t e = cudaMalloc(&wf->err_wf, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(wf->err_wf, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&wf->status_host), sizeof(int), 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = fail(QMC_ERR_OOM, std::string("status word: ") + cudaGetErrorString(e));
    }
  }
  if (st == QMC_OK) {  // the proposal kernels' Box-Muller tables on this device
    DeviceGuard guard(wf->device);
    const cudaError_t e = init_box_muller_tables();
    if (e != cudaSuccess) st = cuda_fail(e, "Box-Muller tables");
  }
  if (st != QMC_OK) {
    qmc_destroy_wf(wf);
    return st;
  }
  *out = wf;
  return QMC_OK;
}

void qmc_destroy_wf(qmc_wf* wf) {
  if (!wf) return;
  {
    DeviceGuard guard(wf->device);
    // a failure here has no caller to report to: it is recorded as the
    // thread's qmc_last_error() text and cleared from the runtime
    auto rel = [](cudaError_t e, const char* what) {
      if (e != cudaSuccess) {
        cudaGetLastError();
        g_err = std::string("qmc_destroy_wf: ") + what + ": " + cudaGetErrorString(e);
      }
    };
    if (wf->blob) rel(cudaFree(wf->blob), "tables");
    if (wf->ws) rel(cudaFree(wf->ws), "workspace");
    if (wf->stage) rel(cudaFree(wf->stage), "staging buffer");
    if (wf->gws) rel(cudaFree(wf->gws), "gradient scratch");
    if (wf->err_wf) rel(cudaFree(wf->err_wf), "status word");
    if (wf->status_host) rel(cudaFreeHost(wf->status_host), "host status word");
    for (auto& e : wf->tev)
      if (e) rel(cudaEventDestroy(e), "timing event");
    if (wf->cap_stream) rel(cudaStreamDestroy(wf->cap_stream), "capture stream");
  }
  delete wf;
}

qmc_status qmc_set_geometry(qmc_wf* wf, const double* xyz) {
  if (!wf || !xyz) return fail(QMC_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lock(wf->mu);
  for (int a = 0; a < wf->dev.n_atom; ++a)
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(xyz[3 * a + k])) return fail(QMC_ERR_ARG, "non-finite nuclear coordinate");
      wf->dev.atom_xyz[a][k] = xyz[3 * a + k];
    }
  wf->dev.vnn = vnn_of(wf->dev);
  wf->spec.xyz.assign(xyz, xyz + 3 * wf->dev.n_atom);
  return QMC_OK;
}

size_t qmc_workspace_size(const qmc_wf* wf, int64_t n_walkers) {
  if (!wf || n_walkers < 0) return 0;
  return workspace_bytes(wf, n_walkers);
}

qmc_status qmc_param_layout(const qmc_wf* wf, int64_t* n_param, int64_t offsets[6]) {
  if (!wf || !n_param) return fail(QMC_ERR_ARG, "null argument");
  int64_t o[6];
  o[0] = 0;
  o[1] = o[0] + (int64_t)wf->spec.prim_exp.size();
  o[2] = o[1] + (int64_t)wf->dev.n_ao * wf->dev.n_mo;
  o[3] = o[2] + wf->dev.n_det;
  o[4] = o[3] + 1;
  // with a many-body Jastrow its parameters follow the backflow weight:
  // K_en (w0, w1, w2), then per K_een term (c, a1, b1, a2, b2, a3, b3)
  o[5] = o[4] + 1 + (wf->dev.mb_en ? 3 : 0) + 7 * (int64_t)wf->dev.n_een;
  *n_param = o[5];
  if (offsets)
    for (int k = 0; k < 6; ++k) offsets[k] = o[k];
  return QMC_OK;
}

static void mark(qmc_wf* wf, int k, cudaStream_t st) {
  if (wf->timing) cudaEventRecord(wf->tev[k], st);
}

// Local-energy (kinetic) or value-only evaluation of W walkers.
// Stages: Jastrow + Coulomb, AO + AO->MO contraction, determinants (table
// method, or explicit per-excitation LU when selected), in order on the
// caller's stream.  (A two-stream pipeline over walker chunks, with each
// chunk's determinant stage overlapping the next chunk's AO stage, was
// measured slower on CO: a determinant block sharing an SM keeps half of its
// warps and loses more FP64 throughput than the overlap gains.)  Backflow
// wavefunctions run the general FP64 kernel.
//
// mapped: null, or walkers [3N][ldw] in mapped host memory.  Then `stage` is a
// device buffer of the same shape: the Jastrow kernel reads the positions
// over the host link once and writes them there, and the later stages read
// the device copy (the upload overlaps the Jastrow stage's arithmetic).
static qmc_status eval_path(qmc_wf* wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                            int* err_flag, bool kinetic, double* e_loc, double* log_psi, cudaStream_t st,
                            const double* mapped = nullptr, double* stage = nullptr) {
  const WfDev& d = wf->dev;
  if (d.bf_w != 0.0) {  // backflow: one general kernel (Jastrow, orbitals, Eq. nabla_d, E_L)
    mark(wf, 0, st);
    qmc_status s = launch_status(launch_eloc_general(d, walkers, W, ldw, kinetic, e_loc, log_psi, st), "general");
    if (s) return s;
    for (int k = 1; k < 6; ++k) mark(wf, k, st);
    if (wf->timing) wf->timed_once = true;
    return QMC_OK;
  }
  const bool tc = wf->precision == QMC_MIXED_TF32 || wf->precision == QMC_MIXED_BF16;
  const int nch = kinetic ? 2 : 1;
  const Workspace& v = ws;
  // FP32X2 value path: log|Psi| for the Metropolis acceptance test needs
  // FP32-level MO values only (the 2e-4 Ha gate concerns E_L); it runs the
  // Jastrow and FP32-AO tensor-core stages of the mixed form
  const bool x2_value = wf->precision == QMC_FP32X2 && !kinetic && d.tc_value;
  mark(wf, 0, st);
  qmc_status s = launch_status(launch_jastrow(d, x2_value ? QMC_MIXED_TF32 : wf->precision, mapped ? mapped : walkers, W,
                                              ldw, mapped ? stage : nullptr, v, kinetic, st),
                               "jastrow");
  if (s) return s;
  if (mapped) walkers = stage;
  mark(wf, 1, st);
  mark(wf, 2, st);
  const bool x2 = wf->precision == QMC_FP32X2;
  s = launch_status(x2_value    ? launch_ao_mo_tc(d, QMC_MIXED_TF32, walkers, W, ldw, v, nch, err_flag, wf->err_wf, st)
                    : tc        ? launch_ao_mo_tc(d, wf->precision, walkers, W, ldw, v, nch, err_flag, wf->err_wf, st)
                    : x2 && d.oz ? launch_ao_mo_oz(d, walkers, W, ldw, v, nch, err_flag, wf->err_wf, st)
                    : x2         ? launch_ao_mo_x2(d, walkers, W, ldw, v, nch, st)
                                 : launch_ao_mo_simt(d, wf->precision, walkers, W, ldw, v, nch, st),
                    "ao_mo");
  if (s) return s;
  mark(wf, 3, st);
  mark(wf, 4, st);
  s = launch_status(wf->det_method == QMC_DET_EXPLICIT
                        ? launch_det_explicit(d, wf->precision, W, v, kinetic, e_loc, log_psi, st)
                        : x2 && d.det_x2 ? launch_det_x2(d, W, v, kinetic, e_loc, log_psi, st)
                             : launch_det(d, wf->precision, W, v, kinetic, e_loc, log_psi, st),
                    "det");
  if (s) return s;
  mark(wf, 5, st);
  if (wf->timing) wf->timed_once = true;
  return QMC_OK;
}

}  // extern "C"

// Only the tensor-core forms run bounded device waits; their calls clear the
// workspace's status word first (a later read tells whether this call's waits
// gave up).
static bool has_device_waits(const qmc_wf* wf) {
  return wf->precision == QMC_MIXED_TF32 || wf->precision == QMC_MIXED_BF16 ||
         (wf->precision == QMC_FP32X2 && (wf->dev.oz || wf->dev.tc_value));
}

static qmc_status reset_status(const qmc_wf* wf, int* err_flag, cudaStream_t st) {
  if (!has_device_waits(wf)) return QMC_OK;
  return launch_status(cudaMemsetAsync(err_flag, 0, sizeof(int), st), "status word reset");
}

qmc_status local_energy_call(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, double* e_loc,
                             double* log_psi, void* workspace, size_t workspace_bytes_, void* stream, bool reset) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (n_walkers < 0 || ldw < n_walkers) return fail(QMC_ERR_ARG, "bad walker count or leading dimension");
  if (n_walkers == 0) return QMC_OK;
  if (!walkers || !e_loc) return fail(QMC_ERR_ARG, "null walkers or e_loc");
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  void* base;
  qmc_status s = get_workspace(wf, n_walkers, workspace, workspace_bytes_, &base);
  if (s) return s;
  int* err_flag;
  Workspace ws = carve(wf, base, n_walkers, &err_flag);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (reset && (s = reset_status(wf, err_flag, st))) return s;
  return eval_path(wf, walkers, n_walkers, ldw, ws, err_flag, true, e_loc, log_psi, st);
}

extern "C" {

qmc_status qmc_local_energy(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, double* e_loc,
                            double* log_psi, void* workspace, size_t workspace_bytes_, void* stream) {
  return local_energy_call(wf, walkers, n_walkers, ldw, e_loc, log_psi, workspace, workspace_bytes_, stream, true);
}

qmc_status qmc_local_energy_host(qmc_wf* wf, const double* walkers, int64_t n_walkers, double* e_loc,
                                 double* log_psi, void* stream) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (n_walkers < 0) return fail(QMC_ERR_ARG, "bad walker count");
  if (n_walkers == 0) return QMC_OK;
  if (!walkers || !e_loc) return fail(QMC_ERR_ARG, "null walkers or e_loc");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t W = n_walkers;
  const size_t in_bytes = sizeof(double) * 3 * wf->dev.n_elec * W;
  const size_t need = align256(in_bytes) + 2 * align256(sizeof(double) * W);
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  if (wf->stage_bytes < need) {
    if (wf->stage) cudaFree(wf->stage);
    wf->stage = nullptr;
    wf->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&wf->stage, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(QMC_ERR_OOM, std::string("staging allocation: ") + cudaGetErrorString(e));
    }
    wf->stage_bytes = need;
  }
  char* p = reinterpret_cast<char*>(wf->stage);
  double* d_in = reinterpret_cast<double*>(p);
  double* d_e = reinterpret_cast<double*>(p + align256(in_bytes));
  double* d_lp = reinterpret_cast<double*>(p + align256(in_bytes) + align256(sizeof(double) * W));
  // Page-locked host walkers that the runtime maps into this device's address
  // space are read by the first kernel directly (one pass over the host link,
  // overlapped with its arithmetic); any other host memory is uploaded first.
  // Backflow wavefunctions run one general kernel and always take the upload.
  const double* mapped = nullptr;
  if (wf->dev.bf_w == 0.0) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, walkers) == cudaSuccess) {
      if (pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr && pa.device == wf->device)
        mapped = static_cast<const double*>(pa.devicePointer);
    } else {
      cudaGetLastError();
    }
  }
  if (!mapped) {
    cudaError_t e = cudaMemcpyAsync(d_in, walkers, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "walker upload");
  }
  void* base;
  qmc_status s = get_workspace(wf, W, nullptr, 0, &base);
  if (s) return s;
  int* err_flag;
  Workspace ws = carve(wf, base, W, &err_flag);
  if ((s = reset_status(wf, err_flag, st))) return s;
  s = eval_path(wf, d_in, W, W, ws, err_flag, true, d_e, log_psi ? d_lp : nullptr, st, mapped, d_in);
  if (s) return s;
  cudaError_t e = cudaMemcpyAsync(e_loc, d_e, sizeof(double) * W, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && log_psi) e = cudaMemcpyAsync(log_psi, d_lp, sizeof(double) * W, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && has_device_waits(wf))
    e = cudaMemcpyAsync(wf->status_host, err_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "result download");
  if (has_device_waits(wf) && *wf->status_host != 0)
    return fail(QMC_ERR_TIMEOUT, "a bounded device wait gave up: the affected walkers' results are NaN");
  return QMC_OK;
}

// Metropolis steps as a CUDA graph: one step (proposal, value path on the
// proposals, acceptance, step-counter advance) is captured once on the
// wavefunction's capture stream and replayed n_steps times on st, so a
// launch-bound chain (small walker counts) pays one graph launch per step
// instead of five to seven kernel launches.  The step index comes from a
// device counter (zeroed first), so every replay draws its own Philox
// numbers and the chain is the one the plain loop gives.  *done = false with
// QMC_OK when capture is not possible here (the caller then runs the loop).
static constexpr int kGraphMinSteps = 4;

static qmc_status sample_graph(qmc_wf* wf, double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                               int* err_flag, int32_t n_steps, double step, uint64_t seed, uint64_t first_walker,
                               uint64_t step_offset, int64_t* n_accept, cudaStream_t st, bool* done) {
  *done = false;
  if (!wf->cap_stream && cudaStreamCreateWithFlags(&wf->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return QMC_OK;
  }
  cudaStream_t cs = wf->cap_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return QMC_OK;
  }
  Workspace wp = ws;
  qmc_status s = launch_status(
      launch_propose(wf->dev, walkers, W, ldw, ws, step, seed, first_walker, step_offset, ws.ctr, cs), "propose");
  if (!s) s = eval_path(wf, ws.prop, W, ws.ldm, wp, err_flag, false, nullptr, ws.lp_new, cs);
  if (!s)
    s = launch_status(
        launch_accept(wf->dev, walkers, W, ldw, ws, seed, first_walker, step_offset, ws.ctr, n_accept, cs), "accept");
  if (!s) s = launch_status(launch_step_advance(ws.ctr, cs), "step counter");
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (s || e != cudaSuccess || !graph) {  // not capturable here: the plain loop runs instead
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return QMC_OK;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QMC_OK;
  }
  e = cudaMemsetAsync(ws.ctr, 0, sizeof(uint64_t), st);
  for (int t = 0; e == cudaSuccess && t < n_steps; ++t) e = cudaGraphLaunch(exec, st);
  cudaGraphExecDestroy(exec);  // freed once the launched replays complete
  if (e != cudaSuccess) return cuda_fail(e, "step graph launch");
  *done = true;
  return QMC_OK;
}

}  // extern "C"

qmc_status sample_call(qmc_wf* wf, double* walkers, int64_t n_walkers, int64_t ldw, int32_t n_steps, double step,
                       uint64_t seed, uint64_t first_walker, uint64_t step_offset, double* log_psi, int64_t* n_accept,
                       void* workspace, size_t workspace_bytes_, void* stream, bool reset) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (n_walkers < 0 || ldw < n_walkers || n_steps < 0) return fail(QMC_ERR_ARG, "bad sizes");
  if (n_walkers == 0) return QMC_OK;
  if (!walkers) return fail(QMC_ERR_ARG, "null walkers");
  if (!(step > 0.0) || !std::isfinite(step)) return fail(QMC_ERR_ARG, "step must be positive and finite");
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  void* base;
  qmc_status s = get_workspace(wf, n_walkers, workspace, workspace_bytes_, &base);
  if (s) return s;
  int* err_flag;
  Workspace ws = carve(wf, base, n_walkers, &err_flag);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (reset && (s = reset_status(wf, err_flag, st))) return s;
  s = eval_path(wf, walkers, n_walkers, ldw, ws, err_flag, false, nullptr, ws.lp, st);
  if (s) return s;
  Workspace wp = ws;  // value path on the proposals: walkers = prop, ldw = ldm
  bool done = false;
  if (n_steps >= kGraphMinSteps && !wf->timing) {
    s = sample_graph(wf, walkers, n_walkers, ldw, ws, err_flag, n_steps, step, seed, first_walker, step_offset,
                     n_accept, st, &done);
    if (s) return s;
  }
  for (int t = 0; !done && t < n_steps; ++t) {
    const uint64_t g = step_offset + (uint64_t)t;
    s = launch_status(launch_propose(wf->dev, walkers, n_walkers, ldw, ws, step, seed, first_walker, g, nullptr, st),
                      "propose");
    if (s) return s;
    s = eval_path(wf, ws.prop, n_walkers, ws.ldm, wp, err_flag, false, nullptr, ws.lp_new, st);
    if (s) return s;
    s = launch_status(
        launch_accept(wf->dev, walkers, n_walkers, ldw, ws, seed, first_walker, g, nullptr, n_accept, st), "accept");
    if (s) return s;
  }
  if (log_psi) {
    cudaError_t e = cudaMemcpyAsync(log_psi, ws.lp, sizeof(double) * n_walkers, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "log_psi copy");
  }
  return QMC_OK;
}

extern "C" {

qmc_status qmc_sample(qmc_wf* wf, double* walkers, int64_t n_walkers, int64_t ldw, int32_t n_steps, double step,
                      uint64_t seed, uint64_t first_walker, uint64_t step_offset, double* log_psi,
                      int64_t* n_accept, void* workspace, size_t workspace_bytes_, void* stream) {
  return sample_call(wf, walkers, n_walkers, ldw, n_steps, step, seed, first_walker, step_offset, log_psi, n_accept,
                     workspace, workspace_bytes_, stream, true);
}

}  // extern "C"

int* workspace_status(const qmc_wf* wf, void* workspace, int64_t n_walkers) {
  int* flag = nullptr;
  carve(wf, workspace, n_walkers, &flag);
  return flag;
}

extern "C" {

qmc_status qmc_check_status(qmc_wf* wf, void* stream) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(wf->status_host, wf->err_wf, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (*wf->status_host == 0) return QMC_OK;
  e = cudaMemsetAsync(wf->err_wf, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status reset");
  return fail(QMC_ERR_TIMEOUT,
              "a bounded device wait gave up since the last check: the affected walkers' results are NaN");
}

qmc_status qmc_set_wait_limit(qmc_wf* wf, int64_t cycles) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (cycles < 0) return fail(QMC_ERR_ARG, "negative wait budget");
  std::lock_guard<std::mutex> lock(wf->mu);
  wf->wait_cycles = cycles;
  wf->dev.wait_cycles = wf->wait_cycles;
  return QMC_OK;
}

// ---- allocation-free variant of qmc_local_energy ---------------------------
// The scratch lives in a static device array of this translation unit; host
// code only ever uses the address obtained for it by cudaGetSymbolAddress (the
// array's name is a host-side shadow in host code), looked up once per device
// with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QMC_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256] = {};

qmc_status qmc_local_energy_noalloc(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw,
                                    double* e_loc, double* log_psi, void* stream) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (n_walkers < 0 || ldw < n_walkers) return fail(QMC_ERR_ARG, "bad walker count or leading dimension");
  if (n_walkers == 0) return QMC_OK;
  if (!walkers || !e_loc) return fail(QMC_ERR_ARG, "null walkers or e_loc");
  const size_t need = workspace_bytes(wf, n_walkers);
  if (need > QMC_NOALLOC_SCRATCH_BYTES) {
    int64_t lo = 0, hi = n_walkers;  // largest admissible batch, for the message
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) / 2;
      if (workspace_bytes(wf, mid) <= QMC_NOALLOC_SCRATCH_BYTES) lo = mid; else hi = mid - 1;
    }
    return fail(QMC_ERR_ARG, "n_walkers = " + std::to_string(n_walkers) + " needs " + std::to_string(need) +
                                 " bytes of scratch; the static scratch holds " +
                                 std::to_string((size_t)QMC_NOALLOC_SCRATCH_BYTES) +
                                 " bytes (at most " + std::to_string(lo) +
                                 " walkers for this wavefunction per call)");
  }
  if (wf->device < 0 || wf->device >= 256) return fail(QMC_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  void* base;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[wf->device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "static scratch address");
      g_noalloc_ptr[wf->device] = p;
    }
    base = g_noalloc_ptr[wf->device];
  }
  int* err_flag;
  Workspace ws = carve(wf, base, n_walkers, &err_flag);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  qmc_status s = reset_status(wf, err_flag, st);
  if (s) return s;
  return eval_path(wf, walkers, n_walkers, ldw, ws, err_flag, true, e_loc, log_psi, st);
}

qmc_status qmc_set_params(qmc_wf* wf, const double* params) {
  if (!wf || !params) return fail(QMC_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lock(wf->mu);
  HostSpec old = wf->spec;
  HostSpec& h = wf->spec;
  size_t k = 0;
  for (auto& v : h.prim_exp) v = params[k++];
  for (auto& v : h.mo) v = params[k++];
  for (auto& v : h.det_w) v = params[k++];
  h.b = params[k++];
  h.w = params[k++];
  for (auto& v : h.jen) v = params[k++];
  for (auto& v : h.jeen) v = params[k++];
  for (size_t q = 0; q < k; ++q)
    if (!std::isfinite(params[q])) {
      wf->spec = old;
      return fail(QMC_ERR_ARG, "non-finite parameter " + std::to_string(q));
    }
  qmc_status st = build_tables(wf);
  if (st != QMC_OK) wf->spec = old;
  return st;
}

}  // extern "C"

// Preconditions and scratch of the energy-gradient calls: the library-owned
// workspace, and in the gradient scratch e_loc [W], stats [4] and the block
// partial sums (rows x blocks, rows up to max(n_param, 9 n_atom)).
// The energy-gradient path of a wavefunction: the general kernels (one
// determinant, <= 8 electrons, <= 4 per spin; gradient and forces) or the
// multi-determinant kernels (no backflow; gradient only).
static qmc_status grad_setup(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, bool want_grad,
                             int64_t* n_param, Workspace* ws, int** err_flag, double** e_loc, double** stats,
                             double** partial, bool* md) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (n_walkers < 1 || ldw < n_walkers) return fail(QMC_ERR_ARG, "need n_walkers >= 1 and ldw >= n_walkers");
  if (!walkers) return fail(QMC_ERR_ARG, "null walkers");
  if (wf->precision != QMC_FP64) return fail(QMC_ERR_UNSUPPORTED, "energy gradients are computed in the FP64 form");
  // the many-body Jastrow's parameters are in the multi-determinant kernels
  *md = !general_supported(wf->dev) || wf->dev.mb_en || wf->dev.n_een;
  if (*md && !md_grad_supported(wf->dev))
    return fail(QMC_ERR_UNSUPPORTED,
                "energy gradients need one determinant with <= 8 electrons (<= 4 per spin), or no backflow with "
                "<= 8 electrons per spin, <= 16 orbitals and <= 128 distinct excitations per spin");
  qmc_param_layout(wf, n_param, nullptr);
  const size_t smem = *md ? md_grad_smem_bytes(wf->dev, (int)*n_param) : grad_smem_bytes(wf->dev, (int)*n_param);
  if (want_grad && smem > 227 * 1024)
    return fail(QMC_ERR_UNSUPPORTED, "too many parameters for the gradient kernel's shared memory");
  void* base;
  qmc_status s = get_workspace(wf, n_walkers, nullptr, 0, &base);
  if (s) return s;
  *ws = carve(wf, base, n_walkers, err_flag);
  const int64_t nb = general_blocks(n_walkers);
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const size_t part = *md ? md_grad_scratch_bytes(wf->dev, ws->ldm, (int)*n_param, n_sm)
                          : sizeof(double) * nb * std::max<int64_t>(*n_param, 9 * wf->dev.n_atom);
  const size_t need = align256(sizeof(double) * n_walkers) + align256(sizeof(double) * 4) + align256(part);
  if (wf->gws_bytes < need) {
    if (wf->gws) cudaFree(wf->gws);
    wf->gws = nullptr;
    wf->gws_bytes = 0;
    cudaError_t e = cudaMalloc(&wf->gws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(QMC_ERR_OOM, std::string("gradient scratch allocation: ") + cudaGetErrorString(e));
    }
    wf->gws_bytes = need;
  }
  char* p = static_cast<char*>(wf->gws);
  *e_loc = reinterpret_cast<double*>(p);
  *stats = reinterpret_cast<double*>(p + align256(sizeof(double) * n_walkers));
  *partial = reinterpret_cast<double*>(p + align256(sizeof(double) * n_walkers) + align256(sizeof(double) * 4));
  return QMC_OK;
}

extern "C" {

qmc_status qmc_energy_grad(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, double* e_stats,
                           double* grad, double* forces, void* stream) {
  if (!e_stats) return fail(QMC_ERR_ARG, "null e_stats");
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t n_param = 0;
  Workspace ws;
  int* err_flag;
  double *e_loc, *stats, *partial;
  bool md = false;
  qmc_status s = grad_setup(wf, walkers, n_walkers, ldw, grad != nullptr, &n_param, &ws, &err_flag, &e_loc, &stats,
                            &partial, &md);
  if (s) return s;
  if (md && forces)
    return fail(QMC_ERR_UNSUPPORTED,
                "forces need one determinant with <= 8 electrons and no many-body Jastrow (pass forces = NULL)");
  s = eval_path(wf, walkers, n_walkers, ldw, ws, err_flag, true, e_loc, nullptr, st);
  if (s) return s;
  s = launch_status(launch_mean_var(e_loc, n_walkers, stats, st), "mean/variance");
  if (s) return s;
  if (grad && md) {
    s = launch_status(launch_md_grad(wf->dev, walkers, n_walkers, ldw, ws, e_loc, stats, wf->spec.prim_start[wf->dev.n_ao],
                                     (int)n_param, partial, grad, st),
                      "parameter gradient (several determinants)");
    if (s) return s;
  } else if (grad) {
    s = launch_status(launch_grad(wf->dev, walkers, n_walkers, ldw, e_loc, stats, wf->dev.ao_ang, wf->dev.ao_prim,
                                  (int)n_param, partial, grad, st),
                      "parameter gradient");
    if (s) return s;
  }
  if (forces) {
    s = launch_status(launch_forces(wf->dev, walkers, n_walkers, ldw, e_loc, stats, partial, forces, st), "forces");
    if (s) return s;
  }
  cudaError_t e = cudaMemcpyAsync(e_stats, stats, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? QMC_OK : cuda_fail(e, "energy statistics");
}

int64_t qmc_energy_grad_sums_size(const qmc_wf* wf) {
  if (!wf) return 0;
  int64_t n_param = 0;
  qmc_param_layout(wf, &n_param, nullptr);
  return 3 + 2 * n_param + 9 * (int64_t)wf->dev.n_atom;
}

qmc_status qmc_energy_grad_sums(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, double* sums,
                                void* stream) {
  if (!sums) return fail(QMC_ERR_ARG, "null sums");
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t n_param = 0;
  Workspace ws;
  int* err_flag;
  double *e_loc, *stats, *partial;
  bool md = false;
  qmc_status s =
      grad_setup(wf, walkers, n_walkers, ldw, true, &n_param, &ws, &err_flag, &e_loc, &stats, &partial, &md);
  if (s) return s;
  s = eval_path(wf, walkers, n_walkers, ldw, ws, err_flag, true, e_loc, nullptr, st);
  if (s) return s;
  s = launch_status(launch_energy_sums(e_loc, n_walkers, sums, st), "energy sums");
  if (s) return s;
  if (md) {  // gradient sums; the force blocks are NaN (forces need path (a))
    for (int weight = 1; weight <= 2 && !s; ++weight)
      s = launch_status(launch_md_grad(wf->dev, walkers, n_walkers, ldw, ws, e_loc, stats,
                                       wf->spec.prim_start[wf->dev.n_ao], (int)n_param, partial,
                                       sums + 3 + (weight - 1) * n_param, st, weight),
                        "parameter gradient sums (several determinants)");
    if (s) return s;
    return launch_status(cudaMemsetAsync(sums + 3 + 2 * n_param, 0xFF, sizeof(double) * 9 * wf->dev.n_atom, st),
                         "force sums");
  }
  for (int weight = 1; weight <= 2 && !s; ++weight)
    s = launch_status(launch_grad(wf->dev, walkers, n_walkers, ldw, e_loc, stats, wf->dev.ao_ang, wf->dev.ao_prim,
                                  (int)n_param, partial, sums + 3 + (weight - 1) * n_param, st, weight),
                      "parameter gradient sums");
  if (s) return s;
  return launch_status(launch_forces(wf->dev, walkers, n_walkers, ldw, e_loc, stats, partial, sums + 3 + 2 * n_param,
                                     st, true),
                       "force sums");
}

qmc_status qmc_assemble_energy_grad(int64_t n_param, int32_t n_atom, const double* sums, double* e_stats,
                                    double* grad, double* forces) {
  if (n_param < 0 || n_atom < 1 || !sums || !e_stats) return fail(QMC_ERR_ARG, "bad sizes or null sums / e_stats");
  const double M = sums[0];
  if (!(M >= 1.0)) return fail(QMC_ERR_ARG, "the sums cover no walker");
  const double ev = sums[1] / M;
  e_stats[0] = ev;
  e_stats[1] = sums[2] / M - ev * ev;
  const double* s_dlp = sums + 3;
  const double* s_edlp = sums + 3 + n_param;
  if (grad)
    for (int64_t k = 0; k < n_param; ++k) grad[k] = 2.0 * (s_edlp[k] - ev * s_dlp[k]) / M;
  const int64_t na3 = 3 * (int64_t)n_atom;
  const double* s_de = sums + 3 + 2 * n_param;
  const double* s_dr = s_de + na3;
  const double* s_edr = s_dr + na3;
  if (forces)
    for (int64_t k = 0; k < na3; ++k) forces[k] = -(s_de[k] + s_edr[k] - ev * s_dr[k]) / M;
  return QMC_OK;
}

qmc_status qmc_set_manybody_jastrow(qmc_wf* wf, const double* en, int32_t n_een, const double* een) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (n_een < 0 || n_een > kMaxEen || (n_een > 0 && !een)) return fail(QMC_ERR_ARG, "bad electron-electron-nucleus terms");
  if (en && (!std::isfinite(en[0]) || !std::isfinite(en[1]) || !(en[2] >= 0.0) || !std::isfinite(en[2])))
    return fail(QMC_ERR_ARG, "electron-nucleus kernel: finite w0, w1 and w2 >= 0 required");
  for (int t = 0; t < n_een; ++t)
    for (int k = 0; k < 7; ++k) {
      const double v = een[7 * t + k];
      if (!std::isfinite(v) || ((k == 2 || k == 4 || k == 6) && v < 0.0))
        return fail(QMC_ERR_ARG, "electron-electron-nucleus terms: finite values and b >= 0 required");
    }
  std::lock_guard<std::mutex> lock(wf->mu);
  HostSpec old = wf->spec;
  wf->spec.jen.clear();
  if (en) wf->spec.jen.assign(en, en + 3);
  wf->spec.jeen.clear();
  if (n_een > 0) wf->spec.jeen.assign(een, een + 7 * n_een);
  qmc_status st = build_tables(wf);
  if (st != QMC_OK) wf->spec = old;
  return st;
}

qmc_status qmc_set_det_method(qmc_wf* wf, int32_t method) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  if (method != QMC_DET_TABLE && method != QMC_DET_EXPLICIT) return fail(QMC_ERR_ARG, "unknown determinant method");
  std::lock_guard<std::mutex> lock(wf->mu);
  if (method == QMC_DET_EXPLICIT &&
      det_explicit_smem_bytes(wf->dev, true) > 227 * 1024)
    return fail(QMC_ERR_UNSUPPORTED, "explicit determinant stage exceeds shared memory");
  wf->det_method = method;
  return QMC_OK;
}

qmc_status qmc_set_timing(qmc_wf* wf, int32_t enable) {
  if (!wf) return fail(QMC_ERR_ARG, "null wavefunction");
  std::lock_guard<std::mutex> lock(wf->mu);
  DeviceGuard guard(wf->device);
  if (enable && !wf->tev[0])
    for (auto& e : wf->tev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return cuda_fail(r, "event create");
    }
  wf->timing = enable != 0;
  return QMC_OK;
}

qmc_status qmc_last_stage_ms(qmc_wf* wf, float* ms, int32_t n) {
  if (!wf || !ms || n < 0 || n > 3) return fail(QMC_ERR_ARG, "bad argument");
  std::lock_guard<std::mutex> lock(wf->mu);
  if (!wf->timed_once) return fail(QMC_ERR_ARG, "no timed evaluation yet");
  DeviceGuard guard(wf->device);
  cudaError_t r = cudaEventSynchronize(wf->tev[5]);
  for (int k = 0; k < n && r == cudaSuccess; ++k) r = cudaEventElapsedTime(&ms[k], wf->tev[2 * k], wf->tev[2 * k + 1]);
  if (r != cudaSuccess) return cuda_fail(r, "event timing");
  return QMC_OK;
}

const char* qmc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
