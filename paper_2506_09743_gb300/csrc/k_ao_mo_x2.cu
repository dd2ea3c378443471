// AO evaluation fused with the AO->MO contraction in pairs of FP32
// (QMC_FP32X2 form): near-FP64 MO channels from the FP32 pipes.
//
// Why: the local energy of an ill-conditioned walker (a reference matrix
// with a large condition number, or a CI expansion that nearly cancels) is
// so sensitive to its MO values that FP32 AOs leave about one CO walker in
// six more than 2e-4 Ha from the FP64 result.  Pairs of FP32 (f32x2.cuh,
// about 2^-47 per operation) bring the MO channels to within a few 2^-46 of
// |AO| |C|, and the FP64 determinant stage then matches the FP64 form to
// well under 2e-4 Ha on every walker short of the nodes.  GB300's FP64 pipe
// runs at about 1/62 of the FP32 rate, so pairs of FP32 cost far less than FP64.
//
// One thread per (walker, electron), 128 walkers per block, one block row
// per electron (the layout of the SIMT kernel of the other forms).  Per shell
// the radial factor and its derivatives (Sec. 2.1: STO and contracted GTO)
//   f,  g1 = f'/rho,  f2 = f''
// and the kinetic operator's radial part RL = f2 + 2 (l + 1) g1 + 2 g1 (gJ . d)
// give, for a complete Cartesian s, p or d shell (canonical order s; x, y, z;
// xx, xy, xz, yy, yz, zz; rows of the MO table permuted to match),
//   value   P f
//   kinetic (lap + 2 gJ . grad)(P f) = f lap P + P RL + 2 f gJ . grad P
// in closed form; other shells take the general power path.  Every AO value
// and kinetic value is multiplied into the MO accumulators as a pair
// (mac_x2: exact product, two_sum into the high word), normalised once at
// the end and written as FP64 (hi + lo is exact in FP64).
#include "ao_eval.cuh"

namespace qmc {

namespace {

constexpr int kX2Threads = 128;

__device__ __forceinline__ f32x2 ld_x2(const float2* p) {
  const float2 v = *p;
  return f32x2(v.x, v.y);
}

__device__ __forceinline__ f32x2 x2_expo(const ShellDev& sh, int p) { return f32x2(sh.expo_f[p], sh.expo_lo[p]); }
__device__ __forceinline__ f32x2 x2_coef(const ShellDev& sh, int p) { return f32x2(sh.coef_f[p], sh.coef_lo[p]); }

}  // namespace

template <int NMO, int NCH>
__global__ void __launch_bounds__(kX2Threads) k_ao_mo_x2(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                        int64_t ldw, const float* __restrict__ gradJ,
                                                        double* __restrict__ mo_out, int nmp, int64_t ldm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* C_s = reinterpret_cast<float2*>(smem_raw);                    // [n_ao][NMO], shell-canonical rows
  float* xtab = reinterpret_cast<float*>(C_s + (size_t)wf.n_ao * NMO);  // [64][2]
  ShellDev* sh_s = reinterpret_cast<ShellDev*>(xtab + 128);            // [n_shell]
  int* pow_s = reinterpret_cast<int*>(sh_s + wf.n_shell);               // [n_ao]
  for (int k = threadIdx.x; k < wf.n_ao * NMO; k += blockDim.x) {
    const int b = k / NMO, m = k % NMO;
    C_s[k] = m < wf.n_mo ? wf.mo_x2[b * wf.n_mo + m] : make_float2(0.f, 0.f);
  }
  for (int k = threadIdx.x; k < 128; k += blockDim.x) xtab[k] = wf.exp_tab[k];
  for (int k = threadIdx.x; k < wf.n_shell * (int)(sizeof(ShellDev) / 4); k += blockDim.x)
    reinterpret_cast<int*>(sh_s)[k] = reinterpret_cast<const int*>(wf.shells)[k];
  for (int k = threadIdx.x; k < wf.n_ao; k += blockDim.x) pow_s[k] = wf.ao_pow[k];
  __syncthreads();

  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (w >= W) return;
  const double rx = walkers[(int64_t)(3 * i) * ldw + w];
  const double ry = walkers[(int64_t)(3 * i + 1) * ldw + w];
  const double rz = walkers[(int64_t)(3 * i + 2) * ldw + w];
  float gjx = 0.f, gjy = 0.f, gjz = 0.f;
  if (NCH == 2) {
    gjx = gradJ[(int64_t)(3 * i) * ldm + w];
    gjy = gradJ[(int64_t)(3 * i + 1) * ldm + w];
    gjz = gradJ[(int64_t)(3 * i + 2) * ldm + w];
  }
  f32x2 acc0[NMO], acc1[NMO];
#pragma unroll
  for (int m = 0; m < NMO; ++m) {
    acc0[m] = f32x2(0.f, 0.f);
    acc1[m] = f32x2(0.f, 0.f);
  }
  auto emit = [&](int row, f32x2 v, f32x2 kin) {
    const float2* Cb = C_s + row * NMO;
#pragma unroll
    for (int m = 0; m < NMO; ++m) {
      const f32x2 c = ld_x2(Cb + m);
      mac_x2(acc0[m], v, c);
      if (NCH == 2) mac_x2(acc1[m], kin, c);
    }
  };

  int cur_atom = -1, pow_atom = -1;
  f32x2 dx(0.f), dy(0.f), dz(0.f), r2(0.f), G(0.f), rho(0.f), irho(0.f);
  bool have_rho = false;
  f32x2 px[5], py[5], pz[5];
  for (int s = 0; s < wf.n_shell; ++s) {
    const ShellDev& sh = sh_s[s];
    if (sh.atom != cur_atom) {
      cur_atom = sh.atom;
      dx = diff_x2(rx, wf.atom_xyz[cur_atom][0]);
      dy = diff_x2(ry, wf.atom_xyz[cur_atom][1]);
      dz = diff_x2(rz, wf.atom_xyz[cur_atom][2]);
      r2 = dx * dx + dy * dy + dz * dz;
      if (NCH == 2) G = dx * gjx + dy * gjy + dz * gjz;
      have_rho = false;
    }
    // radial factor f, g1 = f'/rho, f2 = f''
    f32x2 f(0.f), g1(0.f), f2(0.f);
    if (sh.kind == 0) {  // Slater: c rho^kn exp(-zeta rho)
      if (!have_rho) {
        rho = sqrt_x2(r2);
        irho = recip_x2(rho);
        have_rho = true;
      }
      const f32x2 zeta = x2_expo(sh, 0);
      f32x2 rk(1.f);
      for (int k = 0; k < sh.kn; ++k) rk = rk * rho;
      f = x2_coef(sh, 0) * rk * exp_x2(-(zeta * rho), xtab);
      if (NCH == 2) {
        const f32x2 q = irho * (float)sh.kn - zeta;
        g1 = q * f * irho;
        f2 = (q * q - irho * irho * (float)sh.kn) * f;
      }
    } else {  // contracted Gaussian: sum_p c_p exp(-alpha_p rho^2)
      // g1 = -sum 2 al c e, f2 = rho^2 sum (2 al)^2 c e - sum 2 al c e
      f32x2 t1(0.f), t2(0.f);
      for (int p = 0; p < sh.n_prim; ++p) {
        const f32x2 al = x2_expo(sh, p);
        const f32x2 ce = x2_coef(sh, p) * exp_x2(-(al * r2), xtab);
        f += ce;
        if (NCH == 2) {
          const f32x2 t = (al * ce) * 2.0f;  // 2 al c e (the factor 2 is exact)
          t1 += t;
          t2 += (al * t) * 2.0f;
        }
      }
      if (NCH == 2) {
        g1 = -t1;
        f2 = r2 * t2 - t1;
      }
    }
    f32x2 RL(0.f), tf(0.f);
    if (NCH == 2) {
      RL = f2 + g1 * (float)(2 * (sh.l + 1)) + (g1 * G) * 2.0f;
      tf = f * 2.0f;
    }
    const int row0 = sh.ao_first;
    if (sh.canon == 1) {  // s
      emit(row0, f, RL);
    } else if (sh.canon == 2) {  // p: x, y, z
      emit(row0 + 0, dx * f, NCH == 2 ? dx * RL + tf * gjx : f32x2(0.f));
      emit(row0 + 1, dy * f, NCH == 2 ? dy * RL + tf * gjy : f32x2(0.f));
      emit(row0 + 2, dz * f, NCH == 2 ? dz * RL + tf * gjz : f32x2(0.f));
    } else if (sh.canon == 3) {  // d: xx, xy, xz, yy, yz, zz
      const f32x2 fx = f * dx, fy = f * dy, fz = f * dz;
      if (NCH == 2) {
        const f32x2 Rx = RL * dx, Ry = RL * dy, Rz = RL * dz;
        const f32x2 tx = tf * gjx, ty = tf * gjy, tz = tf * gjz;
        emit(row0 + 0, fx * dx, tf + (Rx + tx * 2.0f) * dx);
        emit(row0 + 1, fx * dy, Rx * dy + tx * dy + ty * dx);
        emit(row0 + 2, fx * dz, Rx * dz + tx * dz + tz * dx);
        emit(row0 + 3, fy * dy, tf + (Ry + ty * 2.0f) * dy);
        emit(row0 + 4, fy * dz, Ry * dz + ty * dz + tz * dy);
        emit(row0 + 5, fz * dz, tf + (Rz + tz * 2.0f) * dz);
      } else {
        const f32x2 z0(0.f);
        emit(row0 + 0, fx * dx, z0);
        emit(row0 + 1, fx * dy, z0);
        emit(row0 + 2, fx * dz, z0);
        emit(row0 + 3, fy * dy, z0);
        emit(row0 + 4, fy * dz, z0);
        emit(row0 + 5, fz * dz, z0);
      }
    } else {  // general monomials
      if (pow_atom != cur_atom) {
        pow_atom = cur_atom;
        pow_table(dx, px);
        pow_table(dy, py);
        pow_table(dz, pz);
      }
      for (int k = 0; k < sh.n_ao; ++k) {
        f32x2 P, Px, Py, Pz, lapP;
        angular(pow_s[sh.ao_first + k], px, py, pz, P, Px, Py, Pz, lapP, NCH == 2);
        f32x2 kin(0.f);
        if (NCH == 2) kin = f * lapP + P * RL + tf * (Px * gjx + Py * gjy + Pz * gjz);
        emit(row0 + k, P * f, kin);
      }
    }
  }
  // walker-fastest FP64 MO layout [N][NCH][nmp][ldm] (columns >= n_mo are never read)
  double* dst = mo_out + (size_t)i * NCH * nmp * ldm + w;
#pragma unroll
  for (int m = 0; m < NMO; ++m) {
    dst[(size_t)m * ldm] = widen(normalize_x2(acc0[m]));
    if (NCH == 2) dst[(size_t)(nmp + m) * ldm] = widen(normalize_x2(acc1[m]));
  }
}

size_t x2_smem_bytes(const WfDev& wf, int nmo_inst) {
  return sizeof(float2) * (size_t)wf.n_ao * nmo_inst + sizeof(float) * 128 + sizeof(ShellDev) * wf.n_shell +
         sizeof(int) * wf.n_ao;
}

template <int NMO>
static cudaError_t launch_x2_nmo(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                                 int nch, cudaStream_t st) {
  const dim3 block(kX2Threads), grid((unsigned)((W + kX2Threads - 1) / kX2Threads), (unsigned)wf.n_elec);
  const size_t smem = x2_smem_bytes(wf, NMO);
  const float* gj = static_cast<const float*>(ws.gradJ);
  if (nch == 2) {
    cudaFuncSetAttribute(k_ao_mo_x2<NMO, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ao_mo_x2<NMO, 2><<<grid, block, smem, st>>>(wf, walkers, W, ldw, gj, ws.mo, ws.nmp, ws.ldm);
  } else {
    cudaFuncSetAttribute(k_ao_mo_x2<NMO, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ao_mo_x2<NMO, 1><<<grid, block, smem, st>>>(wf, walkers, W, ldw, gj, ws.mo, ws.nmp, ws.ldm);
  }
  return cudaGetLastError();
}

cudaError_t launch_ao_mo_x2(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                            int nch, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  if (ws.nmp < wf.n_mo) return cudaErrorInvalidValue;
  // one instance per orbital-count bracket (the accumulators live in registers)
  const int n = wf.n_mo;
  if (n <= 4) return launch_x2_nmo<4>(wf, walkers, W, ldw, ws, nch, st);
  if (n <= 8) return launch_x2_nmo<8>(wf, walkers, W, ldw, ws, nch, st);
  if (n <= 12) return launch_x2_nmo<12>(wf, walkers, W, ldw, ws, nch, st);
  if (n <= 14) return launch_x2_nmo<14>(wf, walkers, W, ldw, ws, nch, st);
  if (n <= 16) return launch_x2_nmo<16>(wf, walkers, W, ldw, ws, nch, st);
  if (n <= 24) return launch_x2_nmo<24>(wf, walkers, W, ldw, ws, nch, st);
  if (n <= 32) return launch_x2_nmo<32>(wf, walkers, W, ldw, ws, nch, st);
  return cudaErrorInvalidValue;
}

}  // namespace qmc
