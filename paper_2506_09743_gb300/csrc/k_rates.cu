// Measured arithmetic rates of the GPU the library runs on: the denominators
// of the FP64- and FP32-bound rooflines, and the cost of the FP64 special
// functions (exponential, square root, reciprocal) in FMA equivalents.
//
// Every kernel runs eight independent dependency chains per thread on
// 8 x 256 threads per SM, long enough (tens of milliseconds) for the launch
// to vanish, and is timed with CUDA events on the caller's stream.  The
// chains are contractive maps, so every value stays finite and normal.
#include <string>

#include "qmc_internal.cuh"
#include "wf_internal.cuh"

namespace qmc {

namespace {

constexpr int kChains = 8;
constexpr int kRateThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kRateThreads) k_rate_fma(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// op 0: exp(-x), op 1: sqrt(x + 1), op 2: 1 / (x + 1)
template <int OP>
__global__ void __launch_bounds__(kRateThreads) k_rate_special(double* out, int iters) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 0.25 + 1e-4 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (OP == 0) x[k] = exp(-x[k]);
      if (OP == 1) x[k] = sqrt(x[k] + 1.0);
      if (OP == 2) x[k] = 1.0 / (x[k] + 1.0);
    }
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace qmc

extern "C" qmc_status qmc_measure_rates(double rates[5], void* stream) {
  using namespace qmc;
  if (!rates) return set_error(QMC_ERR_ARG, "null rates");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = 8 * n_sm;
  const double threads = (double)blocks * kRateThreads;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * kRateThreads) != cudaSuccess) {
    cudaGetLastError();
    return set_error(QMC_ERR_OOM, "rate probe buffer");
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto timed = [&](auto launch) -> double {
    launch();  // warm-up
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms * 1e-3;
  };
  const int it_fma = 4096, it_special = 256;
  const double t64 = timed([&] {
    k_rate_fma<double><<<blocks, kRateThreads, 0, st>>>(out, it_fma, 0.999999, 1e-6);
  });
  const double t32 = timed([&] {
    k_rate_fma<float><<<blocks, kRateThreads, 0, st>>>(reinterpret_cast<float*>(out), it_fma * 16, 0.999999f,
                                                      1e-6f);
  });
  const double te = timed([&] { k_rate_special<0><<<blocks, kRateThreads, 0, st>>>(out, it_special); });
  const double ts = timed([&] { k_rate_special<1><<<blocks, kRateThreads, 0, st>>>(out, it_special); });
  const double tr = timed([&] { k_rate_special<2><<<blocks, kRateThreads, 0, st>>>(out, it_special); });
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return set_error(QMC_ERR_CUDA, std::string("rate probe: ") + cudaGetErrorString(e));
  rates[0] = threads * kChains * 8.0 * it_fma / t64;          // FP64 FMA / s
  rates[1] = threads * kChains * 8.0 * it_fma * 16 / t32;     // FP32 FMA instructions / s
  rates[2] = threads * kChains * (double)it_special / te;     // FP64 exp / s
  rates[3] = threads * kChains * (double)it_special / ts;     // FP64 sqrt / s
  rates[4] = threads * kChains * (double)it_special / tr;     // FP64 reciprocal / s
  return QMC_OK;
}
