// Many-body Jastrow instances of the Jastrow + Coulomb stage (App. D; kernels
// in jastrow_kernels.cuh), compiled apart from the Pade-only instances.
#include "jastrow_kernels.cuh"

namespace qmc {

cudaError_t launch_jastrow_mb(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                              const Workspace& ws, bool derivs, cudaStream_t st) {
  const int n = wf.n_elec;
  if (n <= 2) return launch_jastrow_nm<2, true>(wf, prec, walkers, W, ldw, ws, derivs, st);
  if (n <= 4) return launch_jastrow_nm<4, true>(wf, prec, walkers, W, ldw, ws, derivs, st);
  if (n <= 8) return launch_jastrow_nm<8, true>(wf, prec, walkers, W, ldw, ws, derivs, st);
  if (n <= 16) return launch_jastrow_nm<16, true>(wf, prec, walkers, W, ldw, ws, derivs, st);
  return cudaErrorInvalidValue;
}

}  // namespace qmc
