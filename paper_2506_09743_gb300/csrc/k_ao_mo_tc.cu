// AO evaluation fused with the AO->MO contraction on the 5th-generation
// tensor cores (tcgen05, sm_103a).  Mixed forms only.
//
// Persistent CTAs (two per SM) walk over tiles of 128 walkers x one electron
// (MMA M = 128 rows) with the tables staged once; 512 threads.  The AO
// columns are packed on the host into K-passes of 32 columns (a shell never
// straddles two passes; unused columns are zero).  For each pass the four
// thread parts of a row evaluate the pass's shells (dealt to the parts by
// cost), write the FP32 AO channels into shared memory as the MMA A operand,
// split into TF32 high and low parts
//     a = a_hi + a_lo,  a_hi = rna_tf32(a),  a_lo = rna_tf32(a - a_hi),
// and one thread issues, per channel c (value / kinetic operator) and K step,
//     D_c += A_c,hi B_hi + A_c,hi B_lo + A_c,lo B_hi        (kind::tf32)
// with N = 16 (MOs, padded), K = 8 per instruction, accumulating in FP32 in
// tensor memory (two 16-column accumulators) across all passes.  The
// dropped a_lo b_lo term and the TF32 rounding of the low parts leave an
// error of order 2^-21 relative to |a||b|, i.e. FP32-level accuracy.
// B = MO^T (scaled by the AO angular factors) is prepared on the host in the
// same core-matrix layout, for all passes, and copied into shared memory.
// The A buffer holds one pass (64 KB), so two CTAs (32 warps) fit on an SM;
// a pass's buffer is reused once its MMAs have completed (mbarrier).
//
// Shared-memory operand layout (K-major, no swizzle): 8-row x 16-byte core
// matrices; element (row, k) at byte (row / 8) * SBO + (k / 4) * 128 +
// (row % 8) * 16 + (k % 4) * 4, LBO = 128 B (next core matrix along K) and
// SBO = (K extent / 4) * 128 B (next 8-row group).
//
// Every wait on an mbarrier is bounded (WfDev::wait_cycles, about one second
// by default), after which the CTA raises the error flags, waits (bounded
// again) for the MMAs it has issued, writes NaN for its remaining outputs,
// frees its tensor memory and stops instead of hanging; the host reports
// QMC_ERR_TIMEOUT (qmc_check_status, and the calls that synchronise).
#include <algorithm>

#include "ao_eval.cuh"

namespace qmc {

namespace {

constexpr int kRows = 128;
constexpr int kThreads = 512;
constexpr int kParts = kThreads / kRows;
constexpr int kNPad = 16;
constexpr int kPass = kTcPass;
constexpr uint32_t kTmemCols = 32;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// round to TF32 (10 stored mantissa bits), to nearest with ties away from
// zero, on the bit pattern: adding half a TF32 unit to the magnitude and
// clearing the 13 dropped bits (a carry moves into the exponent as it
// should; infinities and NaNs keep their class).  Two integer operations,
// measured slightly faster here than the conversion instruction.
__device__ __forceinline__ uint32_t tf32_rna(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }

// SM100 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, N = 16, M = 128.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kNPad >> 3) << 17) |
                                ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdescTf32), "r"(accumulate));
}

// Wait for the mbarrier phase of the given parity for at most `budget` SM
// clock cycles (and 2^24 tries); false if it did not complete in time.  A
// budget of 0 gives up before the first try (the timeout path's test).
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

// budget of the drain after a failed wait: the MMAs a CTA issued must have
// completed before its shared and tensor memory are released (~1 s)
constexpr long long kDrainCycles = 1ll << 31;

// int words of the AO power, column and shell-list tables, rounded up so that
// the mbarrier behind them is 16-byte aligned
__host__ __device__ inline int tc_int_words(const WfDev& wf) { return (2 * wf.n_ao + wf.n_shell + 3) & ~3; }

}  // namespace

// at most 64 registers per thread: two 512-thread CTAs per SM
template <int NCH>
__global__ void __launch_bounds__(kThreads, 2) k_ao_mo_tc(WfDev wf, const double* __restrict__ walkers, int64_t W,
                                                         int64_t ldw, const float* __restrict__ gradJ,
                                                         double* __restrict__ mo_out, int64_t ldm,
                                                         int* __restrict__ err_flag, int* __restrict__ err_wf) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int kp = wf.k_pad;
  constexpr size_t tile_words = (size_t)kRows * kPass;
  uint32_t* A = reinterpret_cast<uint32_t*>(smem_raw);                // [NCH][2][128][kPass]
  uint32_t* B = A + (size_t)NCH * 2 * tile_words;                     // [2][16][kp]
  ShellDev* sh_s = reinterpret_cast<ShellDev*>(B + 2 * kNPad * kp);  // [n_shell]
  int* pow_s = reinterpret_cast<int*>(sh_s + wf.n_shell);              // [n_ao]
  int* col_s = pow_s + wf.n_ao;                                         // [n_ao]
  int* list_s = col_s + wf.n_ao;                                        // [n_shell]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(pow_s + tc_int_words(wf));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int k = tid; k < 2 * kNPad * kp; k += kThreads)
    B[k] = k < kNPad * kp ? wf.mo_tc_hi[k] : wf.mo_tc_lo[k - kNPad * kp];
  for (int k = tid; k < wf.n_shell * (int)(sizeof(ShellDev) / 4); k += kThreads)
    reinterpret_cast<int*>(sh_s)[k] = reinterpret_cast<const int*>(wf.shells)[k];
  for (int k = tid; k < wf.n_ao; k += kThreads) {
    pow_s[k] = wf.ao_pow[k];
    col_s[k] = wf.ao_col[k];
  }
  for (int k = tid; k < wf.n_shell; k += kThreads) list_s[k] = wf.tc_shells[k];
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int row = tid & (kRows - 1), part = tid / kRows;
  const uint32_t lbo = 128, sbo_a = (uint32_t)(kPass / 4) * 128, sbo_b = (uint32_t)(kp / 4) * 128;
  const int64_t n_wblk = (W + kRows - 1) / kRows;
  const int64_t n_tiles = n_wblk * wf.n_elec;
  uint32_t commits = 0;  // mbarrier phases completed so far (each pass commits once)
  // persistent CTA: the tables stay in shared memory and the tensor memory
  // stays allocated while the CTA walks over (walker block, electron) tiles
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int i = (int)(tile % wf.n_elec);
    const int64_t wb = tile / wf.n_elec;
    const int64_t w = wb * kRows + row;
    const bool live = w < W;
    double rx = 0.0, ry = 0.0, rz = 0.0;
    float gjx = 0.f, gjy = 0.f, gjz = 0.f;
    if (live) {
      rx = walkers[(int64_t)(3 * i) * ldw + w];
      ry = walkers[(int64_t)(3 * i + 1) * ldw + w];
      rz = walkers[(int64_t)(3 * i + 2) * ldw + w];
      if (NCH == 2) {
        gjx = gradJ[(int64_t)(3 * i) * ldm + w];
        gjy = gradJ[(int64_t)(3 * i + 1) * ldm + w];
        gjz = gradJ[(int64_t)(3 * i + 2) * ldm + w];
      }
    }
    auto put = [&](int ch, int k, float v) {  // k: column within the pass
      const size_t off = (size_t)(row / 8) * (kPass / 4) * 32 + (size_t)(k / 4) * 32 + (row % 8) * 4 + (k % 4);
      const uint32_t hi = tf32_rna(v);
      const float lo = v - __uint_as_float(hi);
      A[(size_t)(ch * 2 + 0) * tile_words + off] = hi;
      A[(size_t)(ch * 2 + 1) * tile_words + off] = tf32_rna(lo);
    };
    // two or four consecutive columns of one 16-byte core-matrix row (k even,
    // resp. k = 0 mod 4) with one 8- or 16-byte store per buffer: a warp's 32
    // rows then cover every bank instead of a quarter of them
    auto put2 = [&](int ch, int k, float v0, float v1) {
      const size_t off = (size_t)(row / 8) * (kPass / 4) * 32 + (size_t)(k / 4) * 32 + (row % 8) * 4 + (k % 4);
      const uint32_t h0 = tf32_rna(v0), h1 = tf32_rna(v1);
      *reinterpret_cast<uint2*>(A + (size_t)(ch * 2 + 0) * tile_words + off) = make_uint2(h0, h1);
      *reinterpret_cast<uint2*>(A + (size_t)(ch * 2 + 1) * tile_words + off) =
          make_uint2(tf32_rna(v0 - __uint_as_float(h0)), tf32_rna(v1 - __uint_as_float(h1)));
    };
    auto put4 = [&](int ch, int k, float v0, float v1, float v2, float v3) {
      const size_t off = (size_t)(row / 8) * (kPass / 4) * 32 + (size_t)(k / 4) * 32 + (row % 8) * 4;
      const uint32_t h0 = tf32_rna(v0), h1 = tf32_rna(v1), h2 = tf32_rna(v2), h3 = tf32_rna(v3);
      *reinterpret_cast<uint4*>(A + (size_t)(ch * 2 + 0) * tile_words + off) = make_uint4(h0, h1, h2, h3);
      *reinterpret_cast<uint4*>(A + (size_t)(ch * 2 + 1) * tile_words + off) =
          make_uint4(tf32_rna(v0 - __uint_as_float(h0)), tf32_rna(v1 - __uint_as_float(h1)),
                     tf32_rna(v2 - __uint_as_float(h2)), tf32_rna(v3 - __uint_as_float(h3)));
    };
    bool ok = true;
    for (int pass = 0; pass < wf.n_pass; ++pass) {
      if (pass > 0) {
        // the previous pass's MMAs must have read the A buffer before it is overwritten
        ok = mbar_wait_bounded(smem_u32(mbar), (commits - 1) & 1, wf.wait_cycles) && ok;
      }
      // unused columns of the pass are zero (disjoint from the shells' columns)
      const unsigned zero_cols = wf.pass_zero[pass];
      for (int k = part; k < kPass; k += kParts)
        if ((zero_cols >> k) & 1u)
          for (int ch = 0; ch < NCH; ++ch) put(ch, k, 0.f);
      const int s_begin = wf.part_off[pass][part], s_end = wf.part_off[pass][part + 1];
      int cur_atom = -1, pow_atom = -1;
      float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f, rho = 0.f, irho = 0.f, G = 0.f;
      float px[5], py[5], pz[5];
      // value channel P f and kinetic channel
      //   (lap + 2 grad J . grad)(P f) = f lap P + P (f2 + 2 (l+1) g1 + 2 g1 gJ.d) + 2 f gJ.grad P
      auto emit = [&](int col, float v, float kin) {
        // rows past the last walker keep whatever their (zero) positions give:
        // an MMA row depends on its own A row only, and those rows are never stored
        put(0, col, v);
        if (NCH == 2) put(1, col, kin);
      };
      for (int q = s_begin; q < s_end; ++q) {
        const int ent = list_s[q];
        const ShellDev& sh = sh_s[ent & 0xff];
        const int c0 = (ent >> 8) & 0xff, type = ent >> 16;
        if (sh.atom != cur_atom) {
          cur_atom = sh.atom;
          displacement(rx, ry, rz, wf.atom_xyz[cur_atom], dx, dy, dz);
          r2 = dx * dx + dy * dy + dz * dz;
          irho = rsqrtf(r2);
          rho = r2 * irho;
          G = gjx * dx + gjy * dy + gjz * dz;
        }
        float f, g1 = 0.f, f2 = 0.f;
        shell_radial(sh, r2, rho, irho, f, g1, f2, NCH == 2);
        const float RL = f2 + float(2 * (sh.l + 1)) * g1 + 2.f * g1 * G;
        const float tf = 2.f * f;
        if (type == 1) {
          emit(c0, f, RL);
        } else if (type == 2) {
          const float v0 = dx * f, v1 = dy * f, v2 = dz * f;
          const float k0 = dx * RL + tf * gjx, k1 = dy * RL + tf * gjy, k2 = dz * RL + tf * gjz;
          if ((c0 & 1) == 0) {  // uniform across the warp: every row has the same shell
            put2(0, c0, v0, v1);
            if (NCH == 2) put2(1, c0, k0, k1);
          } else {
            emit(c0 + 0, v0, k0);
            emit(c0 + 1, v1, k1);
          }
          emit(c0 + 2, v2, k2);
        } else if (type == 3) {
          const float fx = f * dx, fy = f * dy, fz = f * dz;
          const float Rx = RL * dx, Ry = RL * dy, Rz = RL * dz;
          const float v0 = fx * dx, v1 = fx * dy, v2 = fx * dz, v3 = fy * dy, v4 = fy * dz, v5 = fz * dz;
          const float k0 = tf + Rx * dx + 2.f * tf * gjx * dx, k1 = Rx * dy + tf * (gjx * dy + gjy * dx),
                      k2 = Rx * dz + tf * (gjx * dz + gjz * dx), k3 = tf + Ry * dy + 2.f * tf * gjy * dy,
                      k4 = Ry * dz + tf * (gjy * dz + gjz * dy), k5 = tf + Rz * dz + 2.f * tf * gjz * dz;
          if ((c0 & 3) == 0) {
            put4(0, c0, v0, v1, v2, v3);
            put2(0, c0 + 4, v4, v5);
            if (NCH == 2) {
              put4(1, c0, k0, k1, k2, k3);
              put2(1, c0 + 4, k4, k5);
            }
          } else {
            emit(c0 + 0, v0, k0);
            emit(c0 + 1, v1, k1);
            emit(c0 + 2, v2, k2);
            emit(c0 + 3, v3, k3);
            emit(c0 + 4, v4, k4);
            emit(c0 + 5, v5, k5);
          }
        } else {
          if (pow_atom != cur_atom) {
            pow_atom = cur_atom;
            pow_table(dx, px); pow_table(dy, py); pow_table(dz, pz);
          }
          for (int k = 0; k < sh.n_ao; ++k) {
            const int b = sh.ao_first + k;
            const int col = col_s[b] - pass * kPass;
            float P, Px, Py, Pz, lapP;
            angular(pow_s[b], px, py, pz, P, Px, Py, Pz, lapP, NCH == 2);
            emit(col, P * f, f * lapP + P * RL + tf * (gjx * Px + gjy * Py + gjz * Pz));
          }
        }
      }
      // generic-proxy shared stores -> visible to the tensor core (async proxy);
      // every thread learns whether all the waits of this CTA succeeded
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ok = __syncthreads_and(ok) != 0;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) break;
      if (tid == 0) {
        const uint32_t b_hi = smem_u32(B), b_lo = smem_u32(B + kNPad * kp);
        for (int ch = 0; ch < NCH; ++ch) {
          const uint32_t a_hi = smem_u32(A + (size_t)(ch * 2) * tile_words);
          const uint32_t a_lo = smem_u32(A + (size_t)(ch * 2 + 1) * tile_words);
          const uint32_t d = tmem + (uint32_t)(ch * kNPad);
          for (int ks = 0; ks < kPass / 8; ++ks) {
            const uint32_t aoff = (uint32_t)ks * 256;                            // two core matrices along K
            const uint32_t boff = (uint32_t)(pass * (kPass / 4) + 2 * ks) * 128;  // same columns of B
            const uint32_t acc = (pass > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(d, smem_desc(a_hi + aoff, lbo, sbo_a), smem_desc(b_hi + boff, lbo, sbo_b), acc);
            mma_tf32(d, smem_desc(a_hi + aoff, lbo, sbo_a), smem_desc(b_lo + boff, lbo, sbo_b), 1u);
            mma_tf32(d, smem_desc(a_lo + aoff, lbo, sbo_a), smem_desc(b_hi + boff, lbo, sbo_b), 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(mbar))
                     : "memory");
      }
      ++commits;
    }
    if (ok) ok = mbar_wait_bounded(smem_u32(mbar), (commits - 1) & 1, wf.wait_cycles);
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      // an MMA did not complete in time: record it (per call and per
      // wavefunction), let the MMAs already issued finish (at most one commit
      // is outstanding: every pass waits for the previous one before it
      // commits), poison this CTA's remaining outputs (this tile and the
      // tiles it would have taken) and stop
      if (tid == 0) {
        atomicExch(err_flag, 1);
        atomicExch(err_wf, 1);
      }
      if (commits > 0) mbar_wait_bounded(smem_u32(mbar), (commits - 1) & 1, kDrainCycles);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int ch = tid >> 7;
      for (int64_t t = tile; t < n_tiles; t += gridDim.x) {
        const int ti = (int)(t % wf.n_elec);
        const int64_t tw = (t / wf.n_elec) * kRows + row;
        if (ch < NCH && tw < W)
          for (int m = 0; m < kNPad; ++m)
            mo_out[((size_t)(ti * NCH + ch) * kNPad + m) * ldm + tw] = __longlong_as_double(0x7ff8000000000000ll);
      }
      break;
    }
    // ---- epilogue: TMEM -> registers -> MO channels in HBM
    const int quad = warp & 3, ch = warp >> 2;
    if (ch < NCH) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(ch * kNPad);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int64_t wr = wb * kRows + quad * 32 + (tid & 31);
      if (wr < W) {  // walker-fastest MO layout: a warp stores 32 consecutive walkers per orbital
        double* dst = mo_out + (size_t)(i * NCH + ch) * kNPad * ldm + wr;
#pragma unroll
        for (int m = 0; m < kNPad; ++m) dst[(size_t)m * ldm] = widen(__uint_as_float(v[m]));
      }
    }
    // the next tile's first MMA overwrites the accumulators: the loads above
    // are complete (wait::ld) before the barrier that precedes it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

size_t tc_smem_bytes(const WfDev& wf, int nch) {
  size_t b = (size_t)nch * 2 * kRows * kPass * 4 + 2 * kNPad * (size_t)wf.k_pad * 4;
  b += sizeof(ShellDev) * wf.n_shell + 4 * (size_t)tc_int_words(wf) + 16;
  return b;
}

cudaError_t launch_ao_mo_tc(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                            const Workspace& ws, int nch, int* err_flag, int* err_wf, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  if (prec != QMC_MIXED_TF32) return cudaErrorInvalidValue;
  // persistent grid: two CTAs per SM (the occupancy the kernel is built
  // for), never more CTAs than tiles
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n_tiles = ((W + kRows - 1) / kRows) * wf.n_elec;
  const dim3 grid((unsigned)std::min<int64_t>(n_tiles, 2 * (int64_t)std::max(n_sm, 1)));
  const size_t smem = tc_smem_bytes(wf, nch);
  const float* gj = static_cast<const float*>(ws.gradJ);
  double* mo = ws.mo;
  if (nch == 2) {
    cudaFuncSetAttribute(k_ao_mo_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ao_mo_tc<2><<<grid, kThreads, smem, st>>>(wf, walkers, W, ldw, gj, mo, ws.ldm, err_flag, err_wf);
  } else {
    cudaFuncSetAttribute(k_ao_mo_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ao_mo_tc<1><<<grid, kThreads, smem, st>>>(wf, walkers, W, ldw, gj, mo, ws.ldm, err_flag, err_wf);
  }
  return cudaGetLastError();
}

}  // namespace qmc
