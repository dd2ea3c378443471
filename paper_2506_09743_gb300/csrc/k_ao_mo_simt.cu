// AO evaluation fused with the AO->MO contraction on the SIMT pipes.
//
// One thread per (walker, electron): evaluates every shell's radial factor
// once, every AO's value and kinetic channel, and accumulates
// Phi_{i,m} = sum_b phi_b C_{b,m} (Sec. 2.1, MO layer) for both channels in
// registers.  The MO table sits in shared memory and is read as a warp-wide
// broadcast.  Used by the FP64 and FP32 forms (the mixed forms run the
// contraction on tcgen05, k_ao_mo_tc.cu).
#include "ao_eval.cuh"

namespace qmc {

template <typename T, int NMO, int NCH>
__global__ void __launch_bounds__(128) k_ao_mo_simt(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                    int64_t ldw, const T* __restrict__ gradJ,
                                                    double* __restrict__ mo_out, int64_t ldm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ShellDev* sh_s = reinterpret_cast<ShellDev*>(smem_raw);
  int* pow_s = reinterpret_cast<int*>(sh_s + wf.n_shell);
  T* C_s = reinterpret_cast<T*>(smem_raw + round_up(sizeof(ShellDev) * wf.n_shell + sizeof(int) * wf.n_ao, 16));
  const T* Cg = sizeof(T) == 8 ? reinterpret_cast<const T*>(wf.mo64) : reinterpret_cast<const T*>(wf.mo32);
  for (int k = threadIdx.x; k < wf.n_shell * (int)(sizeof(ShellDev) / 4); k += blockDim.x)
    reinterpret_cast<int*>(sh_s)[k] = reinterpret_cast<const int*>(wf.shells)[k];
  for (int k = threadIdx.x; k < wf.n_ao; k += blockDim.x) pow_s[k] = wf.ao_pow[k];
  for (int k = threadIdx.x; k < wf.n_ao * NMO; k += blockDim.x) {
    const int b = k / NMO, m = k % NMO;
    C_s[k] = m < wf.n_mo ? Cg[b * wf.n_mo + m] : T(0);
  }
  __syncthreads();

  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (w >= W) return;
  const double rx = walkers[(int64_t)(3 * i) * ldw + w];
  const double ry = walkers[(int64_t)(3 * i + 1) * ldw + w];
  const double rz = walkers[(int64_t)(3 * i + 2) * ldw + w];
  T gjx = T(0), gjy = T(0), gjz = T(0);
  if (NCH == 2) {
    gjx = gradJ[(int64_t)(3 * i) * ldm + w];
    gjy = gradJ[(int64_t)(3 * i + 1) * ldm + w];
    gjz = gradJ[(int64_t)(3 * i + 2) * ldm + w];
  }
  T acc0[NMO], acc1[NMO];
#pragma unroll
  for (int m = 0; m < NMO; ++m) { acc0[m] = T(0); acc1[m] = T(0); }

  int cur_atom = -1;
  T dx = T(0), dy = T(0), dz = T(0), r2 = T(0), rho = T(0), irho = T(0);
  T px[5], py[5], pz[5];
  for (int s = 0; s < wf.n_shell; ++s) {
    const ShellDev& sh = sh_s[s];
    if (sh.atom != cur_atom) {
      cur_atom = sh.atom;
      displacement(rx, ry, rz, wf.atom_xyz[cur_atom], dx, dy, dz);
      r2 = dx * dx + dy * dy + dz * dz;
      irho = T(1) / sqrt(r2);
      rho = r2 * irho;
      pow_table(dx, px); pow_table(dy, py); pow_table(dz, pz);
    }
    T f, g1, f2;
    shell_radial(sh, r2, rho, irho, f, g1, f2, NCH == 2);
    const T radial_lap = f2 + T(2 * (sh.l + 1)) * g1;
    for (int k = 0; k < sh.n_ao; ++k) {
      const int b = sh.ao_first + k;
      T P, Px, Py, Pz, lapP;
      angular(pow_s[b], px, py, pz, P, Px, Py, Pz, lapP, NCH == 2);
      const T v = P * f;
      T kin = T(0);
      if (NCH == 2) {
        const T gx = f * Px + P * g1 * dx, gy = f * Py + P * g1 * dy, gz = f * Pz + P * g1 * dz;
        kin = f * lapP + P * radial_lap + T(2) * (gjx * gx + gjy * gy + gjz * gz);
      }
      const T* Cb = C_s + b * NMO;
#pragma unroll
      for (int m = 0; m < NMO; ++m) {
        const T c = Cb[m];
        acc0[m] += v * c;
        if (NCH == 2) acc1[m] += kin * c;
      }
    }
  }
  // walker-fastest FP64 MO layout [N][NCH][NMO][ldm] (FP32 results widened exactly)
  double* dst = mo_out + (size_t)i * NCH * NMO * ldm + w;
#pragma unroll
  for (int m = 0; m < NMO; ++m) {
    dst[(size_t)m * ldm] = widen(acc0[m]);
    if (NCH == 2) dst[(size_t)(NMO + m) * ldm] = widen(acc1[m]);
  }
}

template <typename T>
static cudaError_t launch_t(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                            int nch, cudaStream_t st) {
  const dim3 block(128), grid((unsigned)((W + 127) / 128), (unsigned)wf.n_elec);
  const T* gj = static_cast<const T*>(ws.gradJ);
  double* mo = ws.mo;
#define QMC_AOMO(NM)                                                                                        \
  if (wf.n_mo <= NM) {                                                                                      \
    const size_t smem = round_up(sizeof(ShellDev) * wf.n_shell + sizeof(int) * wf.n_ao, 16) +              \
                        sizeof(T) * wf.n_ao * NM;                                                           \
    if (nch == 2) {                                                                                         \
      auto kern = k_ao_mo_simt<T, NM, 2>;                                                                   \
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                   \
      kern<<<grid, block, smem, st>>>(wf, walkers, W, ldw, gj, mo, ws.ldm);                                 \
    } else {                                                                                                \
      auto kern = k_ao_mo_simt<T, NM, 1>;                                                                   \
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                   \
      kern<<<grid, block, smem, st>>>(wf, walkers, W, ldw, gj, mo, ws.ldm);                                 \
    }                                                                                                       \
    return cudaGetLastError();                                                                              \
  }
  if (ws.nmp != mo_row_pad(wf.n_mo, false)) return cudaErrorInvalidValue;
  QMC_AOMO(8)
  QMC_AOMO(16)
  QMC_AOMO(32)
#undef QMC_AOMO
  return cudaErrorInvalidValue;
}

cudaError_t launch_ao_mo_simt(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                              const Workspace& ws, int nch, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  return prec == QMC_FP64 ? launch_t<double>(wf, walkers, W, ldw, ws, nch, st)
                          : launch_t<float>(wf, walkers, W, ldw, ws, nch, st);
}

}  // namespace qmc
