// AO evaluation in pairs of FP32 with the AO->MO contraction on the tcgen05
// tensor cores, exact through digit slicing (QMC_FP32X2 form).
//
// The AO values and kinetic channels are those of k_ao_mo_x2 (pairs of FP32,
// closed forms for complete s, p and d shells).  Instead of multiplying them
// into pair accumulators on the SIMT pipes, each is cut into six signed
// 8-bit digits relative to a power-of-two scale of its row (oz_digits.cuh),
// written to shared memory as BF16, and contracted on the tensor cores:
//     D[ch][g] += A[ch][k] B[l]   for every digit pair with k + l = g,
//                                 g = 0..5   (kind::f16, BF16 in, FP32 out).
// The six MO digit slices are stacked along N behind one zero block of 16
// rows, [0 B_0 .. B_5], and the six class accumulators of a channel lie side
// by side in tensor memory (16 columns each).  One MMA per A digit k adds
// A_k B_{g-k} to every class g >= k at once: for even k the window B_0 ..
// B_{5-k} (N = 16 (6 - k)) lands on classes k .. 5; for odd k the window
// starts one block earlier, on the zero block (N = 16 (7 - k)), and lands on
// classes k - 1 .. 5, so that every accumulator address stays a multiple of
// 32 columns.  6 MMAs per channel and K step instead of 21.
// Every product and every partial sum of a class is an integer below 2^24,
// so the FP32 accumulation in tensor memory is exact; the epilogue
// recombines the six classes as a pair of FP32 and writes FP64.
//
// Row scales: before a tile's passes the four thread parts of a row compute,
// in FP32, an upper bound of every AO value and kinetic value of the row
// (radial sums of |c| e^(-alpha r^2) or the Slater radial factor, monomials
// bounded by powers of rho, the Jastrow-gradient term by |grad J|), and the
// row's scale 2^e is the power of two with bound <= 2^(e-1): every scaled
// value lies in [-1/2, 1/2], where the digits stay within the BF16-exact
// range.  MO columns are scaled by 2^f_m and sliced on the host.
//
// Layout as k_ao_mo_tc: persistent CTAs walk over tiles of 128 walkers x one
// electron (MMA M = 128), AO columns in K-passes of 32 (a shell never
// straddles a pass), one CTA of 512 threads per SM.  Where shared memory
// holds two sets of digit tiles (96 KB each), the CTA runs as two groups of
// eight warps on alternate tiles, each with its own digit tiles, mbarrier,
// named barrier and half of tensor memory: while one group waits for its
// MMAs or drains its accumulators, the other evaluates AOs.  Otherwise one
// group of sixteen warps (four threads per row).  Tensor memory per group:
// 2 channels x 6 classes x 16 MO columns.  Every mbarrier wait is bounded as
// in k_ao_mo_tc (error flags, drain of the issued MMAs, NaN outputs,
// QMC_ERR_TIMEOUT on the host).
#include <algorithm>

#include "ao_eval.cuh"
#include "oz_digits.cuh"

namespace qmc {

namespace {

constexpr int kRows = 128;
constexpr int kThreads = 512;
constexpr int kNPad = 16;
constexpr int kPass = kTcPass;
constexpr uint32_t kTmemCols = 256;              // per group: 2 x 6 x 16 = 192 used
constexpr int kStackBlocks = kOzDigits + 1;       // zero block + digit slices of the B stack
constexpr int kChCols = kOzClasses * kNPad;       // accumulator columns of one channel
constexpr int kTileBytes = kRows * kPass * 2;     // one digit slice of one channel (BF16)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// SM100 shared-memory matrix descriptor, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = n
// (a multiple of 16 up to 96 here).
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Barrier of one thread group: the whole CTA for one group, named barrier
// 1 + group (n threads) for two
template <int G>
__device__ __forceinline__ void group_sync(int grp, int n) {
  if (G == 1) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(n) : "memory");
  }
}

template <int G>
__device__ __forceinline__ bool group_and(int grp, int n, bool v) {
  if (G == 1) return __syncthreads_and(v) != 0;
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, %3, q;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + grp), "r"(n)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase, long long budget) {
  const long long t0 = clock64();
  for (int it = 0; it < (1 << 24); ++it) {
    if (clock64() - t0 >= budget) break;
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

constexpr long long kDrainCycles = 1ll << 31;

// byte offset of element (row, k) of a [128][32] BF16 K-major core-matrix
// tile: 8-row x 16-byte core matrices, LBO = 128 B along K, SBO = 512 B
__device__ __forceinline__ uint32_t a_off(int row, int k) {
  return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// power-of-two exponent e of a row scale: bound <= 2^(e - 1), clamped so that
// 2^-e stays a normal float
__device__ __forceinline__ int scale_exponent(uint32_t bound_bits) {
  const int E = (int)((bound_bits >> 23) & 0xffu) - 127;
  return max(-100, min(E + 2, 126));
}

// FP64 value of f * 2^k (f widened exactly, k added to the exponent field)
__device__ __forceinline__ double widen_scaled(float f, int k) {
  const double d = widen(f);
  if (d == 0.0) return d;
  return __longlong_as_double(__double_as_longlong(d) + ((long long)k << 52));
}

// The same for a normal float f when f 2^k is a normal double (always so in
// the epilogue: f is zero or a multiple of 2^-40 below 2^25, |k| < 300): the
// FP64 bit pattern is assembled by integer operations, so the epilogue
// spends one FP64 instruction (the final add) per output instead of five.
__device__ __forceinline__ double widen_scaled_int(float f, int k) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e32 = (u >> 23) & 0xffu;
  if (e32 == 0u || e32 == 0xffu) return widen_scaled(f, k);  // zero, subnormal, inf, NaN
  const uint32_t hi = (u & 0x80000000u) | ((e32 + 896u + (uint32_t)k) << 20) | ((u >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// FP32 upper bounds of |AO value| and |kinetic value| over the AOs of a shell
// at distance rho (r2 = rho^2) with |grad J| = gn
__device__ __forceinline__ void shell_bounds(const ShellDev& sh, float r2, float rho, float irho, float gn,
                                             float& bv, float& bk) {
  float rb0 = 0.f, rb1 = 0.f, rb2 = 0.f;
  if (sh.kind == 0) {
    float rk = 1.f;
    for (int k = 0; k < sh.kn; ++k) rk *= rho;
    const float f = fabsf(sh.coef_f[0]) * rk * __expf(-sh.expo_f[0] * rho);
    const float q = (float)sh.kn * irho + sh.expo_f[0];
    rb0 = f;
    rb1 = q * f * irho;
    rb2 = (q * q + (float)sh.kn * irho * irho) * f;
  } else {
    for (int p = 0; p < sh.n_prim; ++p) {
      const float al = sh.expo_f[p];
      const float ce = fabsf(sh.coef_f[p]) * __expf(-al * r2);
      rb0 += ce;
      rb1 += 2.f * al * ce;
      rb2 += (4.f * al * al * r2 + 2.f * al) * ce;
    }
  }
  const int l = sh.l;
  float rl = 1.f, rl1 = 0.f, rl2 = 0.f;  // rho^l, rho^(l-1), rho^(l-2) (0 for negative powers)
  for (int k = 0; k < l; ++k) {
    rl2 = rl1;
    rl1 = rl;
    rl *= rho;
  }
  bv = rb0 * rl;
  bk = rb0 * (float)(l * (l - 1)) * rl2 + rl * (rb2 + (float)(2 * (l + 1)) * rb1 + 2.f * rb1 * gn * rho) +
       2.f * rb0 * gn * (float)l * rl1;
}

// shared int words of the AO powers, AO columns and both shell lists (four
// and two parts per row), padded to 16 bytes
__host__ __device__ inline int oz_int_words(const WfDev& wf) { return (2 * wf.n_ao + 2 * wf.n_shell + 3) & ~3; }

}  // namespace

template <int NCH, int NG>
__global__ void __launch_bounds__(kThreads, 1) k_ao_mo_oz(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                         int64_t ldw, const float* __restrict__ gradJ,
                                                         double* __restrict__ mo_out, int nmp, int64_t ldm,
                                                         int* __restrict__ err_flag, int* __restrict__ err_wf) {
  constexpr int kGT = kThreads / NG;      // threads of a group
  constexpr int kGP = kGT / kRows;       // threads (parts) per row
  constexpr int kGWarps = kGT / 32;      // warps of a group
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int kp = wf.k_pad;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int grp = tid / kGT, gtid = tid % kGT;
  unsigned char* A = smem_raw + (size_t)grp * NCH * kOzDigits * kTileBytes;  // [NCH][6][128 x 32] BF16
  unsigned char* B = smem_raw + (size_t)NG * NCH * kOzDigits * kTileBytes;    // [7 x 16][kp] BF16 stack
  ShellDev* sh_s = reinterpret_cast<ShellDev*>(B + (size_t)kStackBlocks * kNPad * kp * 2);
  float* xtab = reinterpret_cast<float*>(sh_s + wf.n_shell);          // [64][2]
  int* pow_s = reinterpret_cast<int*>(xtab + 128);                    // [n_ao]
  int* col_s = pow_s + wf.n_ao;                                       // [n_ao]
  int* list_s = col_s + wf.n_ao;                                      // [2][n_shell]
  int* ints_end = pow_s + oz_int_words(wf);
  unsigned* rowb = reinterpret_cast<unsigned*>(ints_end) + grp * 2 * kRows;  // [NG][2][128] bound bits
  int* rowe_buf = ints_end + NG * 2 * kRows + grp * 4 * kRows;                // [NG][2 tiles][2][128] exponents
  int* colf = ints_end + NG * 6 * kRows;                                      // [16] MO column exponents
  uint64_t* mbar_all = reinterpret_cast<uint64_t*>(colf + kNPad);            // [NG]
  uint64_t* mbar = mbar_all + grp;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar_all + NG);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols * NG));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (gtid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  {  // the stack: one zero block, then the six digit slices of the MO table
    const uint32_t* src = reinterpret_cast<const uint32_t*>(wf.mo_oz);
    uint32_t* dst = reinterpret_cast<uint32_t*>(B);
    const int zero_words = (kStackBlocks - kOzDigits) * kNPad * kp / 2;
    for (int k = tid; k < kStackBlocks * kNPad * kp / 2; k += kThreads)
      dst[k] = k < zero_words ? 0u : src[k - zero_words];
  }
  for (int k = tid; k < wf.n_shell * (int)(sizeof(ShellDev) / 4); k += kThreads)
    reinterpret_cast<int*>(sh_s)[k] = reinterpret_cast<const int*>(wf.shells)[k];
  for (int k = tid; k < 128; k += kThreads) xtab[k] = wf.exp_tab[k];
  for (int k = tid; k < wf.n_ao; k += kThreads) {
    pow_s[k] = wf.ao_pow[k];
    col_s[k] = wf.ao_col[k];
  }
  for (int k = tid; k < 2 * wf.n_shell; k += kThreads) list_s[k] = wf.tc_shells[k];
  for (int k = tid; k < kNPad; k += kThreads) colf[k] = wf.oz_colexp[k];
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot + (uint32_t)(grp * kTmemCols);  // this group's columns

  const int row = gtid & (kRows - 1), part = gtid / kRows;
  // a row's shells of pass p: list_s[part_begin(p) .. part_end(p)), from the
  // four-part lists for one group, from the two-part lists for two
  auto part_begin = [&](int p) { return NG == 1 ? wf.part_off[p][part] : wf.part2_off[p][part]; };
  auto part_end = [&](int p) { return NG == 1 ? wf.part_off[p][part + 1] : wf.part2_off[p][part + 1]; };
  const uint32_t lbo = 128, sbo_a = 512, sbo_b = (uint32_t)(kp / 8) * 128;
  const int64_t n_wblk = (W + kRows - 1) / kRows;
  const int64_t n_tiles = n_wblk * wf.n_elec;
  uint32_t commits = 0, iter = 0;
  // a row's electron position and Jastrow gradient, fetched one tile ahead
  // (the loads of the next tile are in flight during this tile's epilogue)
  double nrx, nry, nrz;
  float ngx, ngy, ngz;
  auto fetch = [&](int64_t t) {
    nrx = nry = nrz = 0.0;
    ngx = ngy = ngz = 0.f;
    if (t >= n_tiles) return;
    const int ti = (int)(t % wf.n_elec);
    const int64_t tw = (t / wf.n_elec) * kRows + row;
    if (tw >= W) return;
    nrx = walkers[(int64_t)(3 * ti) * ldw + tw];
    nry = walkers[(int64_t)(3 * ti + 1) * ldw + tw];
    nrz = walkers[(int64_t)(3 * ti + 2) * ldw + tw];
    if (NCH == 2) {
      ngx = gradJ[(int64_t)(3 * ti) * ldm + tw];
      ngy = gradJ[(int64_t)(3 * ti + 1) * ldm + tw];
      ngz = gradJ[(int64_t)(3 * ti + 2) * ldm + tw];
    }
  };
  // group g takes tiles blockIdx.x + (NG j + g) gridDim.x
  const int64_t tile_step = (int64_t)NG * gridDim.x;
  fetch(blockIdx.x + (int64_t)grp * gridDim.x);
  for (int64_t tile = blockIdx.x + (int64_t)grp * gridDim.x; tile < n_tiles; tile += tile_step, ++iter) {
    // scale exponents of this tile's rows: written before its passes, read by
    // its epilogue; alternate buffers, so that the next tile may write its
    // own while this epilogue still reads (the group's pass barrier of the
    // tile after next orders the reuse)
    int* rowe = rowe_buf + (iter & 1u) * 2 * kRows;
    const int i = (int)(tile % wf.n_elec);
    const int64_t wb = tile / wf.n_elec;
    const double rx = nrx, ry = nry, rz = nrz;
    const float gjx = ngx, gjy = ngy, gjz = ngz;
    // ---- 1. row scales from FP32 upper bounds of every AO of the row
    const float gn = NCH == 2 ? sqrtf(gjx * gjx + gjy * gjy + gjz * gjz) : 0.f;
    int e0 = 0, e1 = 0;
    if (wf.oz_bound != nullptr) {
      // per-atom tables of bounds over bins of r^2: each thread reads its
      // row's bins (no reduction across the row's four parts, no barrier);
      // an electron within 2^-12 bohr of a nucleus falls back to the shells
      float bv = 0.f, bk = 0.f;
      bool direct = false;
      for (int a = 0; a < wf.n_atom; ++a) {
        float dx, dy, dz;
        displacement(rx, ry, rz, wf.atom_xyz[a], dx, dy, dz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const int idx = oz_bound_bin(r2);
        if (idx == 0) {
          direct = true;
          continue;
        }
        const float4 t = __ldg(wf.oz_bound + (size_t)a * kOzBoundBins + idx);
        bv = fmaxf(bv, t.x);
        bk = fmaxf(bk, fmaf(gn, t.z, t.y));
      }
      if (direct) {
        int cur_atom = -1;
        float r2 = 0.f, rho = 0.f, irho = 0.f;
        for (int q = 0; q < wf.n_shell; ++q) {
          const ShellDev& sh = sh_s[q];
          if (sh.atom != cur_atom) {
            cur_atom = sh.atom;
            float dx, dy, dz;
            displacement(rx, ry, rz, wf.atom_xyz[cur_atom], dx, dy, dz);
            r2 = dx * dx + dy * dy + dz * dz;
            irho = rsqrtf(r2);
            rho = r2 * irho;
          }
          float sv, sk;
          shell_bounds(sh, r2, rho, irho, gn, sv, sk);
          bv = fmaxf(bv, sv);
          bk = fmaxf(bk, sk);
        }
      }
      e0 = scale_exponent(__float_as_uint(bv));
      e1 = scale_exponent(__float_as_uint(bk));
      if (part == 0) {
        rowe[row] = e0;
        rowe[kRows + row] = e1;
      }
    } else {
      // the four parts of a row bound their own shells and meet in shared memory
      for (int k = gtid; k < 2 * kRows; k += kGT) rowb[k] = 0u;
      group_sync<NG>(grp, kGT);
      float bv = 0.f, bk = 0.f;
      int cur_atom = -1;
      float r2 = 0.f, rho = 0.f, irho = 0.f;
      for (int pass = 0; pass < wf.n_pass; ++pass)
        for (int q = part_begin(pass); q < part_end(pass); ++q) {
          const ShellDev& sh = sh_s[list_s[q] & 0xff];
          if (sh.atom != cur_atom) {
            cur_atom = sh.atom;
            float dx, dy, dz;
            displacement(rx, ry, rz, wf.atom_xyz[cur_atom], dx, dy, dz);
            r2 = dx * dx + dy * dy + dz * dz;
            irho = rsqrtf(r2);
            rho = r2 * irho;
          }
          float sv, sk;
          shell_bounds(sh, r2, rho, irho, gn, sv, sk);
          bv = fmaxf(bv, sv);
          bk = fmaxf(bk, sk);
        }
      // bounds are non-negative: their bit patterns order as unsigned ints
      // (a NaN bound, from an electron on a nucleus, orders above all)
      atomicMax(&rowb[row], __float_as_uint(bv));
      if (NCH == 2) atomicMax(&rowb[kRows + row], __float_as_uint(bk));
      group_sync<NG>(grp, kGT);
      for (int k = gtid; k < 2 * kRows; k += kGT) rowe[k] = scale_exponent(rowb[k]);
      group_sync<NG>(grp, kGT);
      e0 = rowe[row];
      e1 = rowe[kRows + row];
    }
    const float sc0 = __uint_as_float((unsigned)(127 - e0) << 23);
    const float sc1 = NCH == 2 ? __uint_as_float((unsigned)(127 - e1) << 23) : 0.f;

    // digits of one, two (k even) or four (k = 0 mod 4) columns of a channel,
    // written to the six digit tiles (a digit's BF16 pattern is the upper half
    // of its FP32 pattern: two of them are packed by one byte permute)
    auto put1 = [&](int ch, int k, f32x2 v) {
      const float s = ch == 0 ? sc0 : sc1;
      float d[kOzDigits];
      oz_digits(f32x2(v.hi * s, v.lo * s), d);
      const uint32_t off = a_off(row, k);
#pragma unroll
      for (int j = 0; j < kOzDigits; ++j)
        *reinterpret_cast<uint16_t*>(A + (size_t)(ch * kOzDigits + j) * kTileBytes + off) = oz_bf16(d[j]);
    };
    auto put2 = [&](int ch, int k, f32x2 v0, f32x2 v1) {
      const float s = ch == 0 ? sc0 : sc1;
      float d0[kOzDigits], d1[kOzDigits];
      oz_digits(f32x2(v0.hi * s, v0.lo * s), d0);
      oz_digits(f32x2(v1.hi * s, v1.lo * s), d1);
      const uint32_t off = a_off(row, k);
#pragma unroll
      for (int j = 0; j < kOzDigits; ++j)
        *reinterpret_cast<uint32_t*>(A + (size_t)(ch * kOzDigits + j) * kTileBytes + off) =
            __byte_perm(__float_as_uint(d0[j]), __float_as_uint(d1[j]), 0x7632);
    };
    auto put4 = [&](int ch, int k, f32x2 v0, f32x2 v1, f32x2 v2, f32x2 v3) {
      const float s = ch == 0 ? sc0 : sc1;
      float d0[kOzDigits], d1[kOzDigits], d2[kOzDigits], d3[kOzDigits];
      oz_digits(f32x2(v0.hi * s, v0.lo * s), d0);
      oz_digits(f32x2(v1.hi * s, v1.lo * s), d1);
      oz_digits(f32x2(v2.hi * s, v2.lo * s), d2);
      oz_digits(f32x2(v3.hi * s, v3.lo * s), d3);
      const uint32_t off = a_off(row, k);
#pragma unroll
      for (int j = 0; j < kOzDigits; ++j)
        *reinterpret_cast<uint2*>(A + (size_t)(ch * kOzDigits + j) * kTileBytes + off) =
            make_uint2(__byte_perm(__float_as_uint(d0[j]), __float_as_uint(d1[j]), 0x7632),
                       __byte_perm(__float_as_uint(d2[j]), __float_as_uint(d3[j]), 0x7632));
    };

    // ---- 2. passes: AO pairs -> digits -> MMAs per digit class
    bool ok = true;
    uint32_t written = 0u;  // accumulators (ch, class) already written in this tile
    for (int pass = 0; pass < wf.n_pass; ++pass) {
      if (pass > 0) ok = mbar_wait_bounded(smem_u32(mbar), (commits - 1) & 1, wf.wait_cycles) && ok;
      const unsigned zero_cols = wf.pass_zero[pass];
      for (int k = part; k < kPass; k += kGP)
        if ((zero_cols >> k) & 1u)
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
            for (int j = 0; j < kOzDigits; ++j)
              *reinterpret_cast<uint16_t*>(A + (size_t)(ch * kOzDigits + j) * kTileBytes + a_off(row, k)) = 0;
      int cur_atom = -1, pow_atom = -1;
      f32x2 dx(0.f), dy(0.f), dz(0.f), r2(0.f), G(0.f), rho(0.f), irho(0.f);
      bool have_rho = false;
      f32x2 px[5], py[5], pz[5];
      for (int q = part_begin(pass); q < part_end(pass); ++q) {
        const int ent = list_s[q];
        const ShellDev& sh = sh_s[ent & 0xff];
        const int c0 = (ent >> 8) & 0xff, type = ent >> 16;
        if (sh.atom != cur_atom) {
          cur_atom = sh.atom;
          dx = diff_x2(rx, wf.atom_xyz[cur_atom][0]);
          dy = diff_x2(ry, wf.atom_xyz[cur_atom][1]);
          dz = diff_x2(rz, wf.atom_xyz[cur_atom][2]);
          r2 = dx * dx + dy * dy + dz * dz;
          if (NCH == 2) G = dx * gjx + dy * gjy + dz * gjz;
          have_rho = false;
        }
        f32x2 f(0.f), g1(0.f), f2(0.f);
        if (sh.kind == 0) {
          if (!have_rho) {
            rho = sqrt_x2(r2);
            irho = recip_x2(rho);
            have_rho = true;
          }
          const f32x2 zeta(sh.expo_f[0], sh.expo_lo[0]);
          f32x2 rk(1.f);
          for (int k = 0; k < sh.kn; ++k) rk = rk * rho;
          f = f32x2(sh.coef_f[0], sh.coef_lo[0]) * rk * exp_x2(-(zeta * rho), xtab);
          if (NCH == 2) {
            const f32x2 qq = irho * (float)sh.kn - zeta;
            g1 = qq * f * irho;
            f2 = (qq * qq - irho * irho * (float)sh.kn) * f;
          }
        } else {
          // per primitive e = e^(-alpha r^2) and, as pair multiply-accumulates
          // (normalised once per shell), f = sum c e, t1 = sum 2 alpha c e,
          // t2 = sum 4 alpha^2 c e
          f32x2 t1(0.f), t2(0.f);
          for (int p = 0; p < sh.n_prim; ++p) {
            const f32x2 e = exp_x2(-(f32x2(sh.expo_f[p], sh.expo_lo[p]) * r2), xtab);
            mac_x2(f, f32x2(sh.coef_f[p], sh.coef_lo[p]), e);
            if (NCH == 2) {
              mac_x2(t1, f32x2(sh.c2a_f[p], sh.c2a_lo[p]), e);
              mac_x2(t2, f32x2(sh.c4a_f[p], sh.c4a_lo[p]), e);
            }
          }
          f = normalize_x2(f);
          t1 = normalize_x2(t1);
          t2 = normalize_x2(t2);
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
        if (type == 1) {
          put1(0, c0, f);
          if (NCH == 2) put1(1, c0, RL);
        } else if (type == 2) {
          const f32x2 v0 = dx * f, v1 = dy * f, v2 = dz * f;
          f32x2 k0(0.f), k1(0.f), k2(0.f);
          if (NCH == 2) {
            k0 = dx * RL + tf * gjx;
            k1 = dy * RL + tf * gjy;
            k2 = dz * RL + tf * gjz;
          }
          if ((c0 & 1) == 0) {  // uniform across the warp: every row has the same shell
            put2(0, c0, v0, v1);
            if (NCH == 2) put2(1, c0, k0, k1);
          } else {
            put1(0, c0, v0);
            put1(0, c0 + 1, v1);
            if (NCH == 2) {
              put1(1, c0, k0);
              put1(1, c0 + 1, k1);
            }
          }
          put1(0, c0 + 2, v2);
          if (NCH == 2) put1(1, c0 + 2, k2);
        } else if (type == 3) {
          const f32x2 fx = f * dx, fy = f * dy, fz = f * dz;
          const f32x2 v0 = fx * dx, v1 = fx * dy, v2 = fx * dz, v3 = fy * dy, v4 = fy * dz, v5 = fz * dz;
          if ((c0 & 3) == 0) {
            put4(0, c0, v0, v1, v2, v3);
            put2(0, c0 + 4, v4, v5);
          } else {
            put1(0, c0, v0);
            put1(0, c0 + 1, v1);
            put1(0, c0 + 2, v2);
            put1(0, c0 + 3, v3);
            put1(0, c0 + 4, v4);
            put1(0, c0 + 5, v5);
          }
          if (NCH == 2) {
            const f32x2 Rx = RL * dx, Ry = RL * dy, Rz = RL * dz;
            const f32x2 tx = tf * gjx, ty = tf * gjy, tz = tf * gjz;
            const f32x2 k0 = tf + (Rx + tx * 2.0f) * dx, k1 = Rx * dy + tx * dy + ty * dx,
                        k2 = Rx * dz + tx * dz + tz * dx, k3 = tf + (Ry + ty * 2.0f) * dy,
                        k4 = Ry * dz + ty * dz + tz * dy, k5 = tf + (Rz + tz * 2.0f) * dz;
            if ((c0 & 3) == 0) {
              put4(1, c0, k0, k1, k2, k3);
              put2(1, c0 + 4, k4, k5);
            } else {
              put1(1, c0, k0);
              put1(1, c0 + 1, k1);
              put1(1, c0 + 2, k2);
              put1(1, c0 + 3, k3);
              put1(1, c0 + 4, k4);
              put1(1, c0 + 5, k5);
            }
          }
        } else {  // general monomials
          if (pow_atom != cur_atom) {
            pow_atom = cur_atom;
            pow_table(dx, px);
            pow_table(dy, py);
            pow_table(dz, pz);
          }
          for (int k = 0; k < sh.n_ao; ++k) {
            const int b = sh.ao_first + k;
            const int col = col_s[b] - pass * kPass;
            f32x2 P, Px, Py, Pz, lapP;
            angular(pow_s[b], px, py, pz, P, Px, Py, Pz, lapP, NCH == 2);
            put1(0, col, P * f);
            if (NCH == 2) put1(1, col, f * lapP + P * RL + tf * (Px * gjx + Py * gjy + Pz * gjz));
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ok = group_and<NG>(grp, kGT, ok);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) break;
      if (gtid == 0) {
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
        for (int ch = 0; ch < NCH; ++ch)
          for (int ks = 0; ks < kPass / 16; ++ks)
            for (int k = 0; k < kOzDigits; ++k) {
              const uint32_t a = a0 + (uint32_t)(ch * kOzDigits + k) * kTileBytes + (uint32_t)ks * 256;
              // even k: window B_0 .. B_{5-k} (stack block 1 on) onto classes
              // k .. 5; odd k: the zero block first, onto classes k - 1 .. 5.
              // k = 0 comes first and writes all six classes of the channel.
              const int odd = k & 1;
              const int n = kNPad * (kOzDigits - k + odd);
              const uint32_t b = b0 + (uint32_t)(1 - odd) * (kNPad * kp * 2) +
                                 (uint32_t)(pass * (kPass / 8) + 2 * ks) * 128;
              const uint32_t d = tmem + (uint32_t)(ch * kChCols + kNPad * (k - odd));
              const uint32_t acc = (written >> ch) & 1u;
              mma_bf16(d, smem_desc(a, lbo, sbo_a), smem_desc(b, lbo, sbo_b), idesc_bf16(n), acc);
              written |= 1u << ch;
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(mbar))
                     : "memory");
      }
      ++commits;
    }
    if (ok) ok = mbar_wait_bounded(smem_u32(mbar), (commits - 1) & 1, wf.wait_cycles);
    ok = group_and<NG>(grp, kGT, ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      // record the failure, let the issued MMAs finish (at most one commit is
      // outstanding), poison this group's remaining outputs and stop
      if (gtid == 0) {
        atomicExch(err_flag, 1);
        atomicExch(err_wf, 1);
      }
      if (commits > 0) mbar_wait_bounded(smem_u32(mbar), (commits - 1) & 1, kDrainCycles);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int64_t t = tile; t < n_tiles; t += tile_step) {
        const int ti = (int)(t % wf.n_elec);
        const int64_t tw = (t / wf.n_elec) * kRows + row;
        if (tw < W)
          for (int ch = part; ch < NCH; ch += kGP)
            for (int m = 0; m < nmp; ++m)
              mo_out[((size_t)(ti * NCH + ch) * nmp + m) * ldm + tw] = __longlong_as_double(0x7ff8000000000000ll);
      }
      break;
    }
    fetch(tile + tile_step);
    // ---- 3. epilogue: the six classes of 8 MO columns per thread, recombined.
    // A warp reads the tensor-memory lanes of its rank mod 4 (a group starts
    // at a multiple of four warps); the jobs (channel, half of the 16 MO
    // columns) go round the group's roles.
    constexpr int kRoles = kGWarps / 4;
    const int quad = warp & 3, role = (warp % kGWarps) >> 2;
#pragma unroll
    for (int job = role; job < 2 * NCH; job += kRoles) {
      const int ch = job >> 1, half = job & 1;
      {
        uint32_t v[kOzClasses][8];
#pragma unroll
        for (int g = 0; g < kOzClasses; ++g) {
          const uint32_t taddr =
              tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)((ch * kOzClasses + g) * kNPad + half * 8);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(v[g][0]), "=r"(v[g][1]), "=r"(v[g][2]), "=r"(v[g][3]), "=r"(v[g][4]),
                         "=r"(v[g][5]), "=r"(v[g][6]), "=r"(v[g][7])
                       : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int rr = quad * 32 + (tid & 31);
        const int64_t wr = wb * kRows + rr;
        if (wr < W) {
          const int er = rowe[ch * kRows + rr];
          double* dst = mo_out + (size_t)(i * NCH + ch) * nmp * ldm + wr;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int m = half * 8 + c;
            if (m < nmp) {
              float acc[kOzClasses];
#pragma unroll
              for (int g = 0; g < kOzClasses; ++g) acc[g] = __uint_as_float(v[g][c]);
              const f32x2 s = oz_combine(acc);
              const int k = er + colf[m] - 16;
              dst[(size_t)m * ldm] = widen_scaled_int(s.hi, k) + widen_scaled_int(s.lo, k);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot), "r"(kTmemCols * NG));
}

size_t oz_smem_bytes(const WfDev& wf, int nch, int groups) {
  size_t b = (size_t)groups * nch * kOzDigits * kTileBytes + (size_t)kStackBlocks * kNPad * wf.k_pad * 2;
  b += sizeof(ShellDev) * wf.n_shell + sizeof(float) * 128 + 4 * (size_t)oz_int_words(wf);
  b += sizeof(int) * (groups * 6 * kRows + kNPad) + 8 * groups + 8;
  return b;
}

bool oz_supported(const WfDev& wf) {
  // N = 16 MO columns per MMA; the class sums stay below 2^24 for up to 110
  // AO terms (96 kept as the limit); the tiles must fit in shared memory
  return wf.n_pass > 0 && wf.n_mo <= kNPad && wf.n_ao <= 96 && oz_smem_bytes(wf, 2, 1) <= 227 * 1024;
}

int oz_groups(const WfDev& wf, int nch) { return oz_smem_bytes(wf, nch, 2) <= 227 * 1024 ? 2 : 1; }

namespace {

template <int NCH, int G>
cudaError_t launch_oz_t(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                        int* err_flag, int* err_wf, dim3 grid, cudaStream_t st) {
  const size_t smem = oz_smem_bytes(wf, NCH, G);
  cudaFuncSetAttribute(k_ao_mo_oz<NCH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_ao_mo_oz<NCH, G><<<grid, kThreads, smem, st>>>(wf, walkers, W, ldw, static_cast<const float*>(ws.gradJ), ws.mo,
                                                    ws.nmp, ws.ldm, err_flag, err_wf);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ao_mo_oz(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                            int nch, int* err_flag, int* err_wf, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n_tiles = ((W + kRows - 1) / kRows) * wf.n_elec;
  const dim3 grid((unsigned)std::min<int64_t>(n_tiles, std::max(n_sm, 1)));
  const bool two = oz_groups(wf, nch) == 2;
  if (nch == 2)
    return two ? launch_oz_t<2, 2>(wf, walkers, W, ldw, ws, err_flag, err_wf, grid, st)
               : launch_oz_t<2, 1>(wf, walkers, W, ldw, ws, err_flag, err_wf, grid, st);
  return two ? launch_oz_t<1, 2>(wf, walkers, W, ldw, ws, err_flag, err_wf, grid, st)
             : launch_oz_t<1, 1>(wf, walkers, W, ldw, ws, err_flag, err_wf, grid, st);
}

}  // namespace qmc
