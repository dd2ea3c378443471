// Launchers of the Pade Jastrow + Coulomb stage (kernels in jastrow_kernels.cuh).
// The Pade-only instances live here, one per electron-count bracket; the
// many-body instances are compiled in k_jastrow_mb.cu (a separate translation
// unit keeps the parallel build short).
#include "jastrow_kernels.cuh"

namespace qmc {

cudaError_t launch_jastrow_mb(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                              double* copy, const Workspace& ws, bool derivs, cudaStream_t st);

cudaError_t launch_jastrow(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw, double* copy,
                           const Workspace& ws, bool derivs, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  if (wf.mb_en || wf.n_een > 0) return launch_jastrow_mb(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  // one instance per electron-count bracket: registers grow with NMAX, and
  // occupancy with them (14 electrons at NMAX 14: 155 registers, 12 warps/SM;
  // at NMAX 16: 179 registers, 8 warps/SM)
  const int n = wf.n_elec;
  if (n <= 2) return launch_jastrow_nm<2, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  if (n <= 4) return launch_jastrow_nm<4, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  if (n <= 6) return launch_jastrow_nm<6, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  if (n <= 8) return launch_jastrow_nm<8, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  if (n <= 10) return launch_jastrow_nm<10, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  if (n <= 12) return launch_jastrow_nm<12, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  if (n <= 14) return launch_jastrow_nm<14, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  if (n <= 16) return launch_jastrow_nm<16, false>(wf, prec, walkers, W, ldw, copy, ws, derivs, st);
  return cudaErrorInvalidValue;
}

}  // namespace qmc
