// General FP64 path: local energy and log|Psi| kernels (backflow, several
// determinants with backflow) and their launchers; the shared device code
// (orbitals, backflow, determinant Laplacian) is in general_eval.cuh.
#include "general_eval.cuh"

namespace qmc {

template <int NE, int NC, bool PAIRS>
__global__ void __launch_bounds__(128) k_eloc_md(WfDev wf, const double* __restrict__ walkers, int64_t W, int64_t ldw,
                                                 bool kinetic, double* __restrict__ e_loc,
                                                 double* __restrict__ log_psi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GenShared g;
  stage_tables(wf, g, smem_raw);
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double r[NE][3];
  load_walker<NE>(walkers, ldw, w, wf.n_elec, r);
  double e = 0.0, lp = 0.0;
  eval_walker_md<NE, NC, PAIRS>(wf, g, r, kinetic, e, lp);
  if (kinetic) e_loc[w] = e;
  if (log_psi) log_psi[w] = lp;
}

template <int NE, int NO, bool PAIRS>
__global__ void __launch_bounds__(128, 4) k_eloc_general(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                      int64_t ldw, bool kinetic, double* __restrict__ e_loc,
                                                      double* __restrict__ log_psi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GenShared g;
  stage_tables(wf, g, smem_raw);
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double r[NE][3];
  load_walker<NE>(walkers, ldw, w, wf.n_elec, r);
  double e = 0.0, lp = 0.0;
  eval_walker<double, NE, NO, PAIRS>(wf, g, r, wf.atom_xyz, kinetic, e, lp);
  if (kinetic) e_loc[w] = e;
  if (log_psi) log_psi[w] = lp;
}

template <int NE, int NO, bool PAIRS>
__global__ void __launch_bounds__(128) k_logpsi_general(const __grid_constant__ WfDev wf,
                                                        const double* __restrict__ walkers, int64_t W,
                                                        int64_t ldw, double* __restrict__ log_psi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GenShared g;
  stage_tables(wf, g, smem_raw);
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double r[NE][3];
  load_walker<NE>(walkers, ldw, w, wf.n_elec, r);
  log_psi[w] = logpsi_walker<NE, NO, PAIRS>(wf, g, r);
}

// Sum of W values in a fixed order: [0] mean, [1] mean square deviation.
__global__ void k_mean_var(const double* __restrict__ x, int64_t W, double* __restrict__ stats) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < W; k += blockDim.x) s += x[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double mean = red[0] / (double)W;
  __syncthreads();
  s = 0.0;
  for (int64_t k = threadIdx.x; k < W; k += blockDim.x) s += (x[k] - mean) * (x[k] - mean);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[0] = mean;
    stats[1] = red[0] / (double)W;
  }
}

// ----------------------------------------------------------------------------
// launchers

bool general_supported(const WfDev& wf) {
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  return wf.n_det == 1 && wf.n_elec <= 8 && ns <= 4;
}

bool bf_multidet_supported(const WfDev& wf) {
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  const int nc = wf.p_hi[0] > wf.p_hi[1] ? wf.p_hi[0] : wf.p_hi[1];
  return wf.n_elec <= 8 && ns <= 4 && nc <= 8;
}

template <bool PAIRS>
static cudaError_t launch_eloc_general_t(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, bool kinetic,
                                         double* e_loc, double* log_psi, dim3 grid, size_t smem, cudaStream_t st) {
  if (wf.n_det > 1) {
    if (!bf_multidet_supported(wf)) return cudaErrorInvalidValue;
    if (wf.n_elec <= 2) k_eloc_md<2, 8, PAIRS><<<grid, 128, smem, st>>>(wf, walkers, W, ldw, kinetic, e_loc, log_psi);
    else if (wf.n_elec <= 4)
      k_eloc_md<4, 8, PAIRS><<<grid, 128, smem, st>>>(wf, walkers, W, ldw, kinetic, e_loc, log_psi);
    else k_eloc_md<8, 8, PAIRS><<<grid, 128, smem, st>>>(wf, walkers, W, ldw, kinetic, e_loc, log_psi);
    return cudaGetLastError();
  }
  if (!kinetic && log_psi) {  // value path: log|Psi| alone
    QMC_GEN_DISPATCH((k_logpsi_general<NE, NO, PAIRS><<<grid, 128, smem, st>>>(wf, walkers, W, ldw, log_psi)));
    return cudaGetLastError();
  }
  QMC_GEN_DISPATCH(
      (k_eloc_general<NE, NO, PAIRS><<<grid, 128, smem, st>>>(wf, walkers, W, ldw, kinetic, e_loc, log_psi)));
  return cudaGetLastError();
}

cudaError_t launch_eloc_general(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, bool kinetic,
                                double* e_loc, double* log_psi, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  const size_t smem = gen_table_bytes(wf);
  const dim3 grid((unsigned)((W + 127) / 128));
  // FP32X2 form: the orbitals in pairs of FP32 (mo_channels_x2)
  if (wf.gen_x2) return launch_eloc_general_t<true>(wf, walkers, W, ldw, kinetic, e_loc, log_psi, grid, smem, st);
  return launch_eloc_general_t<false>(wf, walkers, W, ldw, kinetic, e_loc, log_psi, grid, smem, st);
}

// As k_mean_var over the finite values only: [0] mean, [1] mean square
// deviation, [2] the number of non-finite values (a request's walkers on a
// nucleus, a coalescence point or a node).
__global__ void k_mean_var_finite(const double* __restrict__ x, int64_t W, double* __restrict__ stats) {
  __shared__ double red[256];
  __shared__ double cnt[256];
  double s = 0.0, c = 0.0;
  for (int64_t k = threadIdx.x; k < W; k += blockDim.x)
    if (isfinite(x[k])) {
      s += x[k];
      c += 1.0;
    }
  red[threadIdx.x] = s;
  cnt[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      cnt[threadIdx.x] += cnt[threadIdx.x + o];
    }
    __syncthreads();
  }
  const double n = cnt[0], mean = n > 0.0 ? red[0] / n : __longlong_as_double(0x7ff8000000000000ll);
  __syncthreads();
  s = 0.0;
  for (int64_t k = threadIdx.x; k < W; k += blockDim.x)
    if (isfinite(x[k])) s += (x[k] - mean) * (x[k] - mean);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[0] = mean;
    stats[1] = n > 0.0 ? red[0] / n : mean;
    stats[2] = (double)W - n;
  }
}

cudaError_t launch_mean_var_finite(const double* x, int64_t W, double* stats, cudaStream_t st) {
  k_mean_var_finite<<<1, 256, 0, st>>>(x, W, stats);
  return cudaGetLastError();
}

cudaError_t launch_mean_var(const double* x, int64_t W, double* stats, cudaStream_t st) {
  k_mean_var<<<1, 256, 0, st>>>(x, W, stats);
  return cudaGetLastError();
}

int general_blocks(int64_t W) { return (int)((W + 127) / 128); }

}  // namespace qmc
