// Wavefunction optimisation loop (App. B) and batched, axis-symmetrised
// forces (Sec. 3.3), composed from the sampling and energy-gradient entry
// points, with the ADAM update and the sample images as device kernels.
//
// ADAM (Kingma and Ba, ICLR 2015, Algorithm 1), per optimised parameter:
//   m = b1 m + (1 - b1) g,   v = b2 v + (1 - b2) g^2,
//   theta -= lr (m / c1) / (sqrt(v / c2) + eps),   c_k = 1 - b_k^t
// each operation rounded once in this order (no contraction into FMAs), with
// b_k^t formed on the host by repeated multiplication; the result is
// reproducible bit for bit.
#include <cmath>
#include <string>
#include <vector>

#include "wf_internal.cuh"

namespace qmc {

__global__ void k_adam(int n, double* __restrict__ theta, double* __restrict__ m, double* __restrict__ v,
                       const double* __restrict__ g, const unsigned char* __restrict__ mask, double lr, double b1,
                       double b2, double c1, double c2, double eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || !mask[k]) return;
  const double gk = g[k];
  const double mk = __dadd_rn(__dmul_rn(b1, m[k]), __dmul_rn(__dsub_rn(1.0, b1), gk));
  const double vk = __dadd_rn(__dmul_rn(b2, v[k]), __dmul_rn(__dsub_rn(1.0, b2), __dmul_rn(gk, gk)));
  const double mhat = __ddiv_rn(mk, c1), vhat = __ddiv_rn(vk, c2);
  m[k] = mk;
  v[k] = vk;
  theta[k] = __dsub_rn(theta[k], __ddiv_rn(__dmul_rn(lr, mhat), __dadd_rn(__dsqrt_rn(vhat), eps)));
}

// images of walkers [3N][ldw] (W of them) under x -> -x, y -> -y and both:
// out [3N][4W], image j of walker w in column j W + w
__global__ void k_axis_images(int n3, int64_t W, const double* __restrict__ r, int64_t ldw, double* __restrict__ out) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  for (int c = 0; c < n3; ++c) {
    const double x = r[(int64_t)c * ldw + w];
    const int d = c % 3;
    for (int j = 0; j < 4; ++j) {
      const bool flip = (d == 0 && (j & 1)) || (d == 1 && (j & 2));
      out[(int64_t)c * 4 * W + (int64_t)j * W + w] = flip ? -x : x;
    }
  }
}

}  // namespace qmc

using namespace qmc;

namespace {

std::vector<double> current_params(const qmc_wf* wf) {
  const HostSpec& h = wf->spec;
  std::vector<double> p;
  p.insert(p.end(), h.prim_exp.begin(), h.prim_exp.end());
  p.insert(p.end(), h.mo.begin(), h.mo.end());
  p.insert(p.end(), h.det_w.begin(), h.det_w.end());
  p.push_back(h.b);
  p.push_back(h.w);
  p.insert(p.end(), h.jen.begin(), h.jen.end());
  p.insert(p.end(), h.jeen.begin(), h.jeen.end());
  return p;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" {

qmc_status qmc_optimize(qmc_wf* wf, double* walkers, int64_t n_walkers, int64_t ldw, const qmc_opt_config* cfg,
                        double* history, void* stream) {
  if (!wf || !cfg) return set_error(QMC_ERR_ARG, "null wavefunction or configuration");
  if (!walkers || n_walkers < 1 || ldw < n_walkers) return set_error(QMC_ERR_ARG, "bad walkers");
  if (cfg->n_iter < 0 || cfg->n_equil < 0 || cfg->n_resample < 0 || !(cfg->step > 0.0))
    return set_error(QMC_ERR_ARG, "bad step counts or proposal width");
  if (!(cfg->lr >= 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) || !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0) ||
      !(cfg->eps > 0.0))
    return set_error(QMC_ERR_ARG, "bad ADAM hyper-parameters");
  if (cfg->n_iter > 0 && !history) return set_error(QMC_ERR_ARG, "null history");
  if (cfg->reserved != 0) return set_error(QMC_ERR_ARG, "reserved field must be 0");
  int64_t n_param = 0;
  qmc_status s = qmc_param_layout(wf, &n_param, nullptr);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DeviceGuard guard(wf->device);
  // device state: theta, m, v, g [n_param] doubles; mask [n_param] bytes; accept counts [W]
  DevBuf buf;
  const size_t nb = sizeof(double) * (size_t)n_param;
  cudaError_t e = cudaMalloc(&buf.p, 4 * nb + (size_t)n_param + 256 + sizeof(int64_t) * (size_t)n_walkers);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(QMC_ERR_OOM, std::string("optimiser state: ") + cudaGetErrorString(e));
  }
  char* base = static_cast<char*>(buf.p);
  double* theta = reinterpret_cast<double*>(base);
  double* m = theta + n_param;
  double* v = m + n_param;
  double* g = v + n_param;
  int64_t* nacc = reinterpret_cast<int64_t*>(base + 4 * nb);
  unsigned char* mask = reinterpret_cast<unsigned char*>(nacc + n_walkers);
  std::vector<unsigned char> hmask((size_t)n_param, 1);
  if (cfg->mask)
    for (int64_t k = 0; k < n_param; ++k) hmask[k] = cfg->mask[k] ? 1 : 0;
  std::vector<double> th = current_params(wf);
  e = cudaMemcpyAsync(theta, th.data(), nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, 2 * nb, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mask, hmask.data(), (size_t)n_param, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return set_error(QMC_ERR_CUDA, std::string("optimiser setup: ") + cudaGetErrorString(e));

  uint64_t offset = 0;
  if (cfg->n_equil > 0) {
    s = qmc_sample(wf, walkers, n_walkers, ldw, cfg->n_equil, cfg->step, cfg->seed, 0, offset, nullptr, nullptr,
                   nullptr, 0, stream);
    if (s) return s;
    offset += (uint64_t)cfg->n_equil;
  }
  double b1t = 1.0, b2t = 1.0;
  for (int32_t t = 1; t <= cfg->n_iter; ++t) {
    double stats[2];
    s = qmc_energy_grad(wf, walkers, n_walkers, ldw, stats, g, nullptr, stream);
    if (s) return s;
    b1t *= cfg->beta1;
    b2t *= cfg->beta2;
    const int threads = 128;
    k_adam<<<(unsigned)((n_param + threads - 1) / threads), threads, 0, st>>>(
        (int)n_param, theta, m, v, g, mask, cfg->lr, cfg->beta1, cfg->beta2, 1.0 - b1t, 1.0 - b2t, cfg->eps);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(th.data(), theta, nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(QMC_ERR_CUDA, std::string("ADAM update: ") + cudaGetErrorString(e));
    s = qmc_set_params(wf, th.data());
    if (s) return s;
    double acc = 0.0;
    if (cfg->n_resample > 0) {
      e = cudaMemsetAsync(nacc, 0, sizeof(int64_t) * (size_t)n_walkers, st);
      if (e != cudaSuccess) return set_error(QMC_ERR_CUDA, std::string("accept counts: ") + cudaGetErrorString(e));
      s = qmc_sample(wf, walkers, n_walkers, ldw, cfg->n_resample, cfg->step, cfg->seed, 0, offset, nullptr, nacc,
                     nullptr, 0, stream);
      if (s) return s;
      offset += (uint64_t)cfg->n_resample;
      std::vector<int64_t> hacc((size_t)n_walkers);
      e = cudaMemcpyAsync(hacc.data(), nacc, sizeof(int64_t) * (size_t)n_walkers, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return set_error(QMC_ERR_CUDA, std::string("accept counts: ") + cudaGetErrorString(e));
      int64_t tot = 0;
      for (int64_t x : hacc) tot += x;
      acc = (double)tot / ((double)n_walkers * cfg->n_resample);
    }
    history[3 * (t - 1) + 0] = stats[0];
    history[3 * (t - 1) + 1] = stats[1];
    history[3 * (t - 1) + 2] = acc;
  }
  return QMC_OK;
}

qmc_status qmc_force_batches(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, int32_t n_batches,
                             int32_t symmetrize, double* e_mean, double* forces, void* stream) {
  if (!wf || !walkers || !forces) return set_error(QMC_ERR_ARG, "null argument");
  if (n_batches < 1 || n_walkers < n_batches || ldw < n_walkers) return set_error(QMC_ERR_ARG, "bad batch count");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DeviceGuard guard(wf->device);
  const int n3 = 3 * wf->dev.n_elec, na = wf->dev.n_atom;
  const int64_t per = n_walkers / n_batches, last = n_walkers - per * (n_batches - 1);
  const int64_t cols = symmetrize ? 4 * last : 0;
  DevBuf buf;
  cudaError_t e = cudaMalloc(&buf.p, sizeof(double) * ((size_t)n3 * (size_t)cols + 3 * (size_t)na));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(QMC_ERR_OOM, std::string("force batches: ") + cudaGetErrorString(e));
  }
  double* fdev = static_cast<double*>(buf.p);
  double* img = fdev + 3 * na;
  for (int32_t b = 0; b < n_batches; ++b) {
    const int64_t nw = b == n_batches - 1 ? last : per;
    const double* src = walkers + (int64_t)b * per;
    const double* eval = src;
    int64_t W = nw, ld = ldw;
    if (symmetrize) {
      k_axis_images<<<(unsigned)((nw + 127) / 128), 128, 0, st>>>(n3, nw, src, ldw, img);
      e = cudaGetLastError();
      if (e != cudaSuccess) return set_error(QMC_ERR_CUDA, std::string("axis images: ") + cudaGetErrorString(e));
      eval = img;
      W = 4 * nw;
      ld = W;
    }
    double stats[2];
    qmc_status s = qmc_energy_grad(wf, eval, W, ld, stats, nullptr, fdev, stream);
    if (s) return s;
    e = cudaMemcpyAsync(forces + (size_t)b * 3 * na, fdev, sizeof(double) * 3 * na, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(QMC_ERR_CUDA, std::string("force copy: ") + cudaGetErrorString(e));
    if (e_mean) e_mean[b] = stats[0];
  }
  return QMC_OK;
}

}  // extern "C"
