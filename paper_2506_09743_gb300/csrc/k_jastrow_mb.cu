// Many-body Jastrow instances of the Jastrow + Coulomb stage (App. D; kernels
// in jastrow_kernels.cuh), compiled apart from the Pade-only instances.
#include "jastrow_kernels.cuh"

namespace qmc {

size_t een_shared_bytes(const WfDev& wf, bool fp64) {
  return fp64 ? een_smem_bytes<double>(wf) : een_smem_bytes<float>(wf);
}

cudaError_t launch_jastrow_mb(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                              double* copy, const Workspace& ws, bool derivs, cudaStream_t st) {
  const int n = wf.n_elec;
  cudaError_t e;
  if (n <= 2) e = launch_jastrow_nm<2, true>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  else if (n <= 4) e = launch_jastrow_nm<4, true>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  else if (n <= 8) e = launch_jastrow_nm<8, true>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  else if (n <= 16) e = launch_jastrow_nm<16, true>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess || wf.n_een == 0) return e;
  // electron-electron-nucleus terms: 16 lanes per walker, kEenWalkers walkers
  // per block; they read the device copy when the first kernel made one
  if (copy) walkers = copy;
  const unsigned grid = (unsigned)((W + kEenWalkers - 1) / kEenWalkers);
  if (prec == QMC_FP64) {
    const size_t smem = een_smem_bytes<double>(wf);
    cudaFuncSetAttribute(k_jastrow_een<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jastrow_een<double><<<grid, 16 * kEenWalkers, smem, st>>>(wf, walkers, W, ldw, static_cast<double*>(ws.gradJ),
                                                                ws.jscal, ws.ldm, derivs);
  } else {
    const size_t smem = een_smem_bytes<float>(wf);
    cudaFuncSetAttribute(k_jastrow_een<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jastrow_een<float><<<grid, 16 * kEenWalkers, smem, st>>>(wf, walkers, W, ldw, static_cast<float*>(ws.gradJ),
                                                               ws.jscal, ws.ldm, derivs);
  }
  return cudaGetLastError();
}

}  // namespace qmc
