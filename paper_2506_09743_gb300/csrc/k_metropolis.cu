// Metropolis-Hastings walker step (App. B): Gaussian proposal moving all
// electrons at once, acceptance min(1, |Psi'/Psi|^2) in log form.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
// key (seed lo, seed hi) and counter (block j, walker, step lo, step hi).
// Block j gives Gaussians 4j..4j+3 by Box-Muller on the word pairs
// (x0, x1), (x2, x3) with u(x) = (x + 0.5) 2^-32; block ceil(3N/4) word 0 is
// the acceptance uniform.  Both kernels regenerate their numbers from the
// counter, so nothing random is stored between them.  The step index is
// gstep plus, when gctr is not null, a device counter: a CUDA graph of one
// step is then replayed with the counter advanced by a one-thread kernel.
#include <cmath>
#include <mutex>
#include <vector>

#include "qmc_internal.cuh"

namespace qmc {

struct u4 { uint32_t x, y, z, w; };

// ---- Box-Muller in FP64 by table-driven argument reduction (in the manner
// of Tang, ACM TOMS 15 (1989) and 16 (1990)): the uniforms are 32-bit
// integers x with u = (x + 1/2) 2^-32, so
//   2 pi u = A + B,  A = 2 pi (x >> 16) 2^-16 (table: sin A, cos A),
//                    B = 2 pi ((x & 0xffff) + 1/2) 2^-32 < 1e-4 (short Taylor series),
//   sin(A + B) = sin A cos B + cos A sin B, cos(A + B) = cos A cos B - sin A sin B;
//   log u = (e - 32) ln 2 + log(1 + j 2^-16) + log1p(r),
//           x + 1/2 = 2^e m, j = the top 16 fraction bits of m,
//           r = (m - (1 + j 2^-16)) / (1 + j 2^-16) < 2^-16 (four Taylor terms),
// with ln 2 split so that (e - 32) ln2_hi is exact; for u within 2^-7 of 1
// the series of log1p(-(1 - u)) instead, which keeps a tiny log u accurate.  About a third of the FP64
// work of the library functions, to within a few ulp of them; the tables
// (2 x 65,536 pairs of doubles, 2 MB, L2-resident) are built on the host in
// extended precision, once per device.
constexpr int kBmBits = 16;
constexpr int kBmN = 1 << kBmBits;
__device__ double g_bm_sincos[2 * kBmN];  // [j] = sin, cos of 2 pi j 2^-16
__device__ double g_bm_log[2 * kBmN];     // [j] = log(1 + j 2^-16), 1 / (1 + j 2^-16)

__device__ __forceinline__ void sincos_2pi_u(uint32_t x, double* s, double* c) {
  const double sa = g_bm_sincos[2 * (x >> kBmBits)], ca = g_bm_sincos[2 * (x >> kBmBits) + 1];
  const double b = ((double)(x & (kBmN - 1)) + 0.5) * (6.283185307179586 * 0x1p-32);
  const double b2 = b * b;
  const double sb = b - b * b2 * (1.0 / 6.0);                  // next term < 1e-18 relative
  const double cb = 1.0 - b2 * (0.5 - b2 * (1.0 / 24.0));      // next term < 1e-27
  *s = sa * cb + ca * sb;
  *c = ca * cb - sa * sb;
}

__device__ __forceinline__ double log_u(uint32_t x) {
  if (x >= 0xFE000000u) {
    // u within 2^-7 of 1: log u = log1p(-w) = -(w + w^2/2 + ... + w^9/9), with
    // w = 1 - u exact (the table form would lose the digits of a tiny log u
    // to the cancellation of e ln2 against the table entry)
    const double w = ((double)(0xFFFFFFFFu - x) + 0.5) * 0x1p-32;
    double q = 1.0 / 9.0;
    q = 1.0 / 8.0 + w * q;
    q = 1.0 / 7.0 + w * q;
    q = 1.0 / 6.0 + w * q;
    q = 1.0 / 5.0 + w * q;
    q = 1.0 / 4.0 + w * q;
    q = 1.0 / 3.0 + w * q;
    q = 0.5 + w * q;
    return -(w + w * w * q);
  }
  const double v = (double)x + 0.5;  // exact
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int e = (int)(bits >> 52) - 1023;
  const unsigned j = (unsigned)(bits >> (52 - kBmBits)) & (kBmN - 1);
  const double m = __longlong_as_double((long long)((bits & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
  const double mh =
      __longlong_as_double((long long)((bits & (((1ull << kBmBits) - 1) << (52 - kBmBits))) | 0x3FF0000000000000ull));
  const double r = (m - mh) * g_bm_log[2 * j + 1];  // m - mh exact
  const double p = r - r * r * (0.5 - r * (1.0 / 3.0 - r * 0.25));
  const double k = (double)(e - 32);
  const double ln2_hi = 6.93147180369123816490e-01, ln2_lo = 1.90821492927058770002e-10;
  return (k * ln2_hi + g_bm_log[2 * j]) + (k * ln2_lo + p);
}

// four Gaussians from one Philox block: (x0, x1) and (x2, x3) -> z[0..3]
__device__ __forceinline__ void box_muller4(const u4& x, double z[4]) {
  const double r1 = sqrt(-2.0 * log_u(x.x)), r2 = sqrt(-2.0 * log_u(x.z));
  double s1, c1, s2, c2;
  sincos_2pi_u(x.y, &s1, &c1);
  sincos_2pi_u(x.w, &s2, &c2);
  z[0] = r1 * c1; z[1] = r1 * s1; z[2] = r2 * c2; z[3] = r2 * s2;
}

cudaError_t init_box_muller_tables() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (int d : done)
    if (d == dev) return cudaSuccess;
  std::vector<double> sc(2 * kBmN), lg(2 * kBmN);
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int j = 0; j < kBmN; ++j) {
    const long double a = two_pi * (long double)j / (long double)kBmN;
    sc[2 * j] = (double)sinl(a);
    sc[2 * j + 1] = (double)cosl(a);
    const long double m = 1.0L + (long double)j / (long double)kBmN;
    lg[2 * j] = (double)logl(m);
    lg[2 * j + 1] = (double)(1.0L / m);
  }
  e = cudaMemcpyToSymbol(g_bm_sincos, sc.data(), sizeof(double) * sc.size());
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bm_log, lg.data(), sizeof(double) * lg.size());
  if (e == cudaSuccess) done.push_back(dev);
  return e;
}

__device__ __forceinline__ u4 philox4x32_10(u4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = u4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

__global__ void __launch_bounds__(128) k_propose(int n3, const double* __restrict__ walkers, int64_t W, int64_t ldw,
                                                 double* __restrict__ prop, int64_t ldm, double step, uint64_t seed,
                                                 uint64_t first_walker, uint64_t gstep,
                                                 const unsigned long long* __restrict__ gctr) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  if (gctr) gstep += *gctr;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint32_t wi = (uint32_t)(first_walker + (uint64_t)w);
  for (int j = 0; 4 * j < n3; ++j) {
    const u4 x = philox4x32_10(u4{(uint32_t)j, wi, (uint32_t)gstep, (uint32_t)(gstep >> 32)}, k0, k1);
    double z[4];
    box_muller4(x, z);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * j + q;
      if (k < n3) prop[(int64_t)k * ldm + w] = walkers[(int64_t)k * ldw + w] + step * z[q];
    }
  }
}

__global__ void __launch_bounds__(128) k_accept(int n3, double* __restrict__ walkers, int64_t W, int64_t ldw,
                                                const double* __restrict__ prop, int64_t ldm,
                                                double* __restrict__ lp, const double* __restrict__ lp_new,
                                                uint64_t seed, uint64_t first_walker, uint64_t gstep,
                                                const unsigned long long* __restrict__ gctr,
                                                int64_t* __restrict__ n_accept) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  if (gctr) gstep += *gctr;
  const uint32_t wi = (uint32_t)(first_walker + (uint64_t)w);
  const int nblk = (n3 + 3) / 4;
  const u4 x = philox4x32_10(u4{(uint32_t)nblk, wi, (uint32_t)gstep, (uint32_t)(gstep >> 32)}, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
  const double lnew = lp_new[w], lold = lp[w];
  if (log(u01(x.x)) < 2.0 * (lnew - lold)) {
    for (int k = 0; k < n3; ++k) walkers[(int64_t)k * ldw + w] = prop[(int64_t)k * ldm + w];
    lp[w] = lnew;
    if (n_accept) n_accept[w] += 1;
  }
}

// Initial walkers for the serving loop: electron i at R_home(i) + N(0, 1) per
// coordinate, Gaussians from the same Philox stream layout with the reserved
// step index 2^64 - 1 (never reached by a chain).
__global__ void __launch_bounds__(128) k_init_walkers(InitSpec spec, int64_t W, int64_t ldw,
                                                      double* __restrict__ walkers, uint64_t seed) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int n3 = 3 * spec.n_elec;
  for (int j = 0; 4 * j < n3; ++j) {
    const u4 x = philox4x32_10(u4{(uint32_t)j, (uint32_t)w, 0xFFFFFFFFu, 0xFFFFFFFFu}, (uint32_t)seed,
                               (uint32_t)(seed >> 32));
    double z[4];
    box_muller4(x, z);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * j + q;
      if (k < n3) walkers[(int64_t)k * ldw + w] = spec.home_xyz[k / 3][k % 3] + z[q];
    }
  }
}

// the step counter of a replayed step graph: one more step done
__global__ void k_step_advance(unsigned long long* ctr) { *ctr += 1ull; }

// sum of the per-walker acceptance counts into out[0] (fixed order)
__global__ void k_sum_counts(const int64_t* __restrict__ c, int64_t W, double* __restrict__ out) {
  __shared__ long long red[256];
  long long s = 0;
  for (int64_t k = threadIdx.x; k < W; k += blockDim.x) s += c[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (double)red[0];
}

cudaError_t launch_init_walkers(const InitSpec& spec, int64_t W, int64_t ldw, double* walkers, uint64_t seed,
                                cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  k_init_walkers<<<(unsigned)((W + 127) / 128), 128, 0, st>>>(spec, W, ldw, walkers, seed);
  return cudaGetLastError();
}

cudaError_t launch_sum_counts(const int64_t* counts, int64_t W, double* out, cudaStream_t st) {
  k_sum_counts<<<1, 256, 0, st>>>(counts, W, out);
  return cudaGetLastError();
}

cudaError_t launch_propose(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                           double step, uint64_t seed, uint64_t first_walker, uint64_t gstep, const uint64_t* gctr,
                           cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  k_propose<<<(unsigned)((W + 127) / 128), 128, 0, st>>>(3 * wf.n_elec, walkers, W, ldw, ws.prop, ws.ldm, step,
                                                          seed, first_walker, gstep,
                                                          reinterpret_cast<const unsigned long long*>(gctr));
  return cudaGetLastError();
}

cudaError_t launch_step_advance(uint64_t* gctr, cudaStream_t st) {
  k_step_advance<<<1, 1, 0, st>>>(reinterpret_cast<unsigned long long*>(gctr));
  return cudaGetLastError();
}

cudaError_t launch_accept(const WfDev& wf, double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                          uint64_t seed, uint64_t first_walker, uint64_t gstep, const uint64_t* gctr,
                          int64_t* n_accept, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  k_accept<<<(unsigned)((W + 127) / 128), 128, 0, st>>>(3 * wf.n_elec, walkers, W, ldw, ws.prop, ws.ldm, ws.lp,
                                                         ws.lp_new, seed, first_walker, gstep,
                                                         reinterpret_cast<const unsigned long long*>(gctr), n_accept);
  return cudaGetLastError();
}

}  // namespace qmc
