// Determinants, excited-determinant tables and local-energy assembly in
// pairs of FP32 (QMC_FP32X2 form, table method).
//
// The same computation as k_det (reference inverse by Gauss-Jordan
// elimination with partial pivoting, Jacobi trace, excitation tables T_val
// and Top, the determinant expansion of Eqs. nabla_sigma / delta_sigma with
// the table formulas of App. F), with the linear algebra in pairs of FP32 on
// the FP32 pipes instead of FP64: on GB300 the FP64 pipe runs at about 1/62 of the
// FP32 rate, and a pair multiply-accumulate costs about 12 FP32 instructions.
//
// Row scaling.  Each electron row r of a spin block is multiplied by an
// exact power of two 2^-e_r (e_r from the largest FP64 exponent of the row's
// occupied orbital values), in both channels and every orbital column.  With
// A = D A^, B = D B^ (D = diag 2^e_r):
//     A^-1 Phi_p = A^^-1 Phi^_p,   A^-1 (B_p - B_0 t) = A^^-1 (B^_p - B^_0 t),
//     Tr(A^-1 B_0) = Tr(A^^-1 B^_0),   det A = 2^(sum e_r) det A^,
// so the tables, the traces and the determinant ratios are those of the
// scaled rows, and only log|det| takes sum e_r ln 2.  The scaled values lie
// within the FP32 exponent range whatever the magnitude of the orbitals.
//
// FP64 -> pair conversion by integer operations on the bit pattern (the
// FP64 pipe is the resource this kernel frees): the high word is the value
// truncated to 24 significant bits, the low word the remaining 29 bits
// rounded to 24; values below 2^-126 of their row scale are flushed to zero
// (an absolute error below 2^-126 against entries of order one).
//
// Work decomposition: eight lanes per (walker, spin), lane r holding row r
// of the spin block (n <= 8 electrons), sixteen lanes per walker, eight
// walkers per block of 128 threads.  Gauss-Jordan elimination runs in place
// with implicit pivoting: at step k the unused row p_k with the largest
// |a[p_k][k]| is broadcast by shuffles and eliminated from every other row
// (the pivot row divided by its pivot in the same instruction stream, as
// 0 - (-1/pivot) a_p); afterwards lane i holds Z[i][k] = (A^^-1)[m_i][p_k],
// m_i being the step at which row i was the pivot (the in-place result of the
// row-permuted elimination).  The tables are then formed per virtual column
// p from three all-gathers within the group, each lane writing one pair to a
// shared-memory slot and reading the group's slots back in 16-byte loads:
//     t[m_i]   = sum_k Z[i][k] Phi^_p[p_k]         (lane i; slot m_r holds Phi^_p[r])
//     y[r]     = B^_p[r] - sum_m B^_0[r][m] t[m]   (lane r; slot m_i holds t[m_i])
//     Top[m_i] = sum_k Z[i][k] y[p_k]              (lane i; slot m_r holds y[r])
// and stored, as in k_det, per walker in shared memory; the sixteen lanes of
// a walker then split its determinant list and reduce their sums with
// shuffles.  det A^ = sgn(p) prod_k pivot_k is kept as a pair with a
// separate power-of-two exponent.
#include "qmc_internal.cuh"

namespace qmc {

namespace {

constexpr int kLanes = 8;                       // lanes (rows) per (walker, spin)
constexpr int kWalkersPerBlockX2 = 8;           // 16 lanes per walker
constexpr int kThreadsX2 = 16 * kWalkersPerBlockX2;

// x 2^-e as a pair of FP32 (see the header); NaN and infinity become NaN
__device__ __forceinline__ f32x2 split_scaled(double x, int e) {
  const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
  const int E = (int)((H >> 20) & 0x7ffu);
  if (E == 0x7ff) return f32x2(__int_as_float(0x7fc00000), 0.f);
  const int e32 = E - 1023 - e + 127;
  if (E == 0 || e32 <= 0) return f32x2(0.f, 0.f);
  const unsigned sign = H & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)min(e32, 254) << 23) | ((H & 0xfffffu) << 3) | (L >> 29));
  // the low 29 bits of the significand times 2^(e32 - 127 - 52), converted
  // on the FP32 pipe (an integer m < 2^23 is (2^23 + m) - 2^23 exactly; the
  // 29 bits as 23 + 6, joined by one rounding FMA)
  float lo = 0.f;
  if (e32 > 52) {
    const unsigned r29 = L & 0x1fffffffu;
    const float fh = x2_sub_rn(__uint_as_float(0x4b000000u | (r29 >> 6)), 8388608.f);
    const float fl = x2_sub_rn(__uint_as_float(0x4b000000u | (r29 & 63u)), 8388608.f);
    lo = x2_mul_rn(x2_fma_rn(fh, 64.f, fl), __uint_as_float((unsigned)(e32 - 52) << 23));
  }
  return fast_two_sum(hi, sign ? -lo : lo);
}

// biased FP64 exponent field of x (0 for zero and subnormals, 2047 for NaN / inf)
__device__ __forceinline__ int exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// c - a b as a pair: the product exact up to its 2^-48 cross terms
__device__ __forceinline__ f32x2 fms_x2(f32x2 c, f32x2 a, f32x2 b) {
  const float p = x2_mul_rn(a.hi, b.hi);
  const float pe = x2_fma_rn(a.hi, b.hi, -p);
  const float cross = x2_fma_rn(a.hi, b.lo, x2_fma_rn(a.lo, b.hi, pe));
  const f32x2 s = two_sum(c.hi, -p);
  return fast_two_sum(s.hi, x2_add_rn(s.lo, x2_sub_rn(c.lo, cross)));
}

__device__ __forceinline__ f32x2 shfl_x2(f32x2 v, int src) {
  return f32x2(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
__device__ __forceinline__ f32x2 shfl_xor_x2(f32x2 v, int m) {
  return f32x2(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

// v 2^-e with e the exponent of v.hi (v.hi in [1, 2) afterwards); returns e.
// Zero, NaN and infinity are left as they are (e = 0).
__device__ __forceinline__ int renorm_x2(f32x2& v) {
  const unsigned u = __float_as_uint(v.hi);
  const int ex = (int)((u >> 23) & 0xffu);
  if (ex == 0 || ex == 0xff) return 0;
  const int e = ex - 127;
  v.hi = __uint_as_float(u - ((unsigned)e << 23));
  const unsigned ul = __float_as_uint(v.lo);
  const int exl = (int)((ul >> 23) & 0xffu);
  v.lo = exl - e >= 1 && exl != 0 ? __uint_as_float(ul - ((unsigned)e << 23)) : 0.f;
  return e;
}

}  // namespace

template <int NS, bool KIN>
__global__ void __launch_bounds__(kThreadsX2, 7)
    k_det_x2(WfDev wf, int64_t W, const double* __restrict__ mo, int nmp, int64_t ldm,
             const double* __restrict__ jscal, int stride, double* __restrict__ e_loc, double* __restrict__ log_psi) {
  constexpr int NCH = KIN ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f32x2* tab_all = reinterpret_cast<f32x2*>(smem_raw);                 // [walkers][stride]
  f32x2* b0_all = tab_all + (size_t)kWalkersPerBlockX2 * stride;       // [2 x walkers][8 rows][8] scaled B_0
  f32x2* dw_s = b0_all + 2 * kWalkersPerBlockX2 * kLanes * kLanes;     // [n_det]
  int4* dt_s = reinterpret_cast<int4*>(dw_s + ((wf.n_det + 1) & ~1));  // [n_det] determinant records
  for (int k = threadIdx.x; k < wf.n_det; k += blockDim.x) {
    dw_s[k] = split_scaled(wf.det_w[k], 0);
    dt_s[k] = wf.det_tab[k];
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int wl = threadIdx.x >> 4, s = (threadIdx.x >> 3) & 1, r = threadIdx.x & 7;
  const int gbase = lane & ~7;  // first lane of this (walker, spin) group
  const int64_t w = (int64_t)blockIdx.x * kWalkersPerBlockX2 + wl;
  const bool live = w < W;
  const int64_t wc = live ? w : 0;  // column read by lanes past the end (their results are discarded)
  const int n = s == 0 ? wf.n_up : wf.n_down;
  const int i0 = s == 0 ? 0 : wf.n_up;
  const int hl = wf.h_lo[s], nh = wf.nh[s], nv = wf.nv[s];
  const bool row = r < n;
  f32x2* tab = tab_all + (size_t)wl * stride;
  const int tab_off = s == 0 ? 0 : NCH * wf.nh[0] * wf.nv[0];
  f32x2* b0_s = b0_all + (size_t)(threadIdx.x >> 3) * kLanes * kLanes;  // this group's [8][8]
  auto ld = [&](int c, int m) -> double {
    return mo[((int64_t)((i0 + r) * NCH + c) * nmp + m) * ldm + wc];
  };

  // ---- 0. this row, scaled by 2^-e_r
  double a64[NS];
  int emax = 0;
#pragma unroll
  for (int c = 0; c < NS; ++c) {
    a64[c] = (row && c < n) ? ld(0, c) : 0.0;
    emax = max(emax, exp_field(a64[c]));
  }
  const int er = row && emax > 0 ? emax - 1023 : 0;
  int esum = er;
#pragma unroll
  for (int m = 1; m < kLanes; m <<= 1) esum += __shfl_xor_sync(0xffffffffu, esum, m);
  f32x2 a[NS];
#pragma unroll
  for (int c = 0; c < NS; ++c) a[c] = c < n ? split_scaled(a64[c], er) : f32x2(0.f);
  if (KIN) {
#pragma unroll
    for (int c = 0; c < NS; ++c) b0_s[r * kLanes + c] = (row && c < n) ? split_scaled(ld(1, c), er) : f32x2(0.f);
  }

  // ---- 1. in-place Gauss-Jordan elimination with implicit pivoting
  bool used = !row;
  int mi = 0;          // the step at which this row was the pivot
  int pk[NS];          // pivot row of each step
  f32x2 detm(1.f);     // det A^ = detm 2^dete (sign included)
  int dete = 0;
  int perm_sign = 0;   // parity of the pivot sequence
  // Every shuffle below runs on all 32 lanes: the two spin groups of a warp
  // may have different n and nv, so group-dependent limits only predicate
  // the arithmetic around the shuffles.
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const bool act = k < n;
    // the unused row with the largest |a[.][k]| (lowest index on ties; a NaN
    // entry counts as the largest, so that every lane agrees on the pivot)
    float key = (act && !used) ? fabsf(a[k].hi) : -1.f;
    if (key != key) key = __int_as_float(0x7f800000);
    int p = r;
#pragma unroll
    for (int m = 1; m < kLanes; m <<= 1) {
      const float ok = __shfl_xor_sync(0xffffffffu, key, m);
      const int op = __shfl_xor_sync(0xffffffffu, p, m);
      if (ok > key || (ok == key && op < p)) { key = ok; p = op; }
    }
    pk[k] = p;
    // the pivot row as it stands; one instruction stream for every lane:
    // the pivot row becomes 0 - (-inv) a_p = a_p / pv, every other row
    // a - g a_p with g = a[k] / pv
    const f32x2 pv = shfl_x2(a[k], gbase + p);
    const f32x2 inv = recip_x2(pv);
    f32x2 prw[NS];
#pragma unroll
    for (int c = 0; c < NS; ++c) prw[c] = shfl_x2(a[c], gbase + p);
    if (act) {
      detm = detm * pv;
      dete += renorm_x2(detm);
      const bool piv = r == p;
      if (piv) {
        used = true;
        mi = k;
      }
      if (row) {
        const f32x2 g = a[k] * inv;
        const f32x2 gg = piv ? -inv : g;
#pragma unroll
        for (int c = 0; c < NS; ++c)
          a[c] = c == k ? (piv ? inv : -g) : fms_x2(piv ? f32x2(0.f) : a[c], gg, prw[c]);
      }
    }
  }
  // parity of the pivot sequence p_0 .. p_{n-1} (inversions)
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int l = k + 1; l < NS; ++l)
      if (l < n && pk[k] > pk[l]) perm_sign ^= 1;
  if (perm_sign) detm = -detm;

  // ---- 2. tr0 = sum_i sum_k Z[i][k] B^_0[p_k][m_i], and the excitation tables
  __syncwarp();
  f32x2 tr0(0.f);
  if (KIN) {
    f32x2 acc(0.f);
    if (row) {
#pragma unroll
      for (int k = 0; k < NS; ++k)
        if (k < n) mac_x2(acc, a[k], b0_s[pk[k] * kLanes + mi]);
    }
    tr0 = normalize_x2(acc);
#pragma unroll
    for (int m = 1; m < kLanes; m <<= 1) tr0 = tr0 + shfl_xor_x2(tr0, m);
  }
  f32x2 b0r[NS];  // this row of B^_0
  if (KIN) {
#pragma unroll
    for (int c = 0; c < NS; ++c) b0r[c] = b0_s[r * kLanes + c];
  }
  const bool hole = row && mi >= hl;
  // per group three broadcast buffers (Phi_p by pivot step, t by step, y by
  // pivot step), 10 pairs apart so that a warp's four groups read different
  // banks
  __shared__ __align__(16) f32x2 bc_all[3][kThreadsX2 / kLanes][10];
  f32x2* bcP = bc_all[0][threadIdx.x >> 3];
  f32x2* bcT = bc_all[1][threadIdx.x >> 3];
  f32x2* bcY = bc_all[2][threadIdx.x >> 3];
  // sum_k z[k] buf[k] over the n broadcast slots (two pairs per 16-byte load)
  auto dot_bc = [&](const f32x2* buf, const f32x2* z) -> f32x2 {
    f32x2 acc(0.f);
    const float4* b4 = reinterpret_cast<const float4*>(buf);
#pragma unroll
    for (int k2 = 0; k2 < (NS + 1) / 2; ++k2) {
      const float4 qv = b4[k2];
      if (2 * k2 < n) mac_x2(acc, z[2 * k2], f32x2(qv.x, qv.y));
      if (2 * k2 + 1 < NS)
        if (2 * k2 + 1 < n) mac_x2(acc, z[2 * k2 + 1], f32x2(qv.z, qv.w));
    }
    return acc;
  };
  const int nv_max = max(wf.nv[0], wf.nv[1]);
  double nphi = (row && nv > 0) ? ld(0, n) : 0.0;
  double nbp = (KIN && row && nv > 0) ? ld(1, n) : 0.0;
  for (int pv = 0; pv < nv_max; ++pv) {
    const bool pact = pv < nv;
    const f32x2 phi = split_scaled(nphi, er);
    const f32x2 bp = KIN ? split_scaled(nbp, er) : f32x2(0.f);
    if (pv + 1 < nv && row) {
      nphi = ld(0, n + pv + 1);
      if (KIN) nbp = ld(1, n + pv + 1);
    }
    // t[m_i] = sum_k Z[i][k] Phi^_p[p_k]: lane r puts Phi^_p[r] in slot m_r
    if (row) bcP[mi] = phi;
    __syncwarp();
    f32x2 t = normalize_x2(dot_bc(bcP, a));
    if (pact && hole) tab[tab_off + (mi - hl) * nv + pv] = t;
    if (KIN) {
      // y[r] = B^_p[r] - sum_m B^_0[r][m] t[m]: lane i puts t[m_i] in slot
      // m_i (accumulated unnormalised, normalised once)
      if (row) bcT[mi] = t;
      __syncwarp();
      f32x2 nb0[NS];
#pragma unroll
      for (int m = 0; m < NS; ++m) nb0[m] = -b0r[m];
      f32x2 y = dot_bc(bcT, nb0);
      y = normalize_x2(bp + y);
      // Top[m_i] = sum_k Z[i][k] y[p_k]: lane r puts y[r] in slot m_r
      if (row) bcY[mi] = y;
      __syncwarp();
      f32x2 acc = dot_bc(bcY, a);
      if (pact && hole) tab[tab_off + nh * nv + (mi - hl) * nv + pv] = normalize_x2(acc);
    }
  }
  __syncwarp();

  // ---- 3. determinant expansion: the 16 lanes of a walker take d = q, q + 16, ...
  const int q = threadIdx.x & 15;
  f32x2 sum_r(0.f), sum_k(0.f);
  for (int d = q; d < wf.n_det; d += 16) {
    const int4 rec = dt_s[d];
    f32x2 R[2], K[2];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const int packed = sp == 0 ? rec.x : rec.z, rank = sp == 0 ? rec.y : rec.w;
      const int off = sp == 0 ? 0 : NCH * wf.nh[0] * wf.nv[0];
      const f32x2* tv = tab + off;
      const f32x2* tk = tab + off + wf.nh[sp] * wf.nv[sp];
      const int q00 = packed & 0xff, q01 = (packed >> 8) & 0xff, q10 = (packed >> 16) & 0xff, q11 = packed >> 24;
      if (rank == 0) {
        R[sp] = f32x2(1.f);
        K[sp] = f32x2(0.f);
      } else if (rank == 1) {
        R[sp] = tv[q00];
        K[sp] = KIN ? tk[q00] : f32x2(0.f);
      } else {
        const f32x2 s00 = tv[q00], s01 = tv[q01], s10 = tv[q10], s11 = tv[q11];
        R[sp] = fms_x2(s00 * s11, s01, s10);
        if (KIN) {
          f32x2 kk(0.f);
          mac_x2(kk, s11, tk[q00]);
          mac_x2(kk, -s01, tk[q10]);
          mac_x2(kk, -s10, tk[q01]);
          mac_x2(kk, s00, tk[q11]);
          K[sp] = normalize_x2(kk);
        } else {
          K[sp] = f32x2(0.f);
        }
      }
    }
    const f32x2 dw = dw_s[d];
    const f32x2 dr1 = dw * R[1];
    mac_x2(sum_r, dr1, R[0]);
    if (KIN) {
      mac_x2(sum_k, dr1, K[0]);
      mac_x2(sum_k, dw * R[0], K[1]);
    }
  }
  sum_r = normalize_x2(sum_r);
  sum_k = normalize_x2(sum_k);
#pragma unroll
  for (int m = 1; m < 16; m <<= 1) {
    sum_r = sum_r + shfl_xor_x2(sum_r, m);
    if (KIN) sum_k = sum_k + shfl_xor_x2(sum_k, m);
  }
  // the other spin's determinant and trace (lanes 8 apart)
  const f32x2 detm_o = shfl_xor_x2(detm, 8);
  const int dete_o = __shfl_xor_sync(0xffffffffu, dete, 8);
  const int esum_o = __shfl_xor_sync(0xffffffffu, esum, 8);
  const f32x2 tr0_o = KIN ? shfl_xor_x2(tr0, 8) : f32x2(0.f);
  if (q == 0 && live) {
    // the products and the kinetic quotient in pairs; FP64 for the logarithm
    // and the final sums only (the FP64 pipe runs at about 1/62 of the FP32 rate)
    const double lp = jscal[w] + log(fabs(widen((detm * detm_o) * sum_r))) +
                      (double)(dete + dete_o + esum + esum_o) * 0.69314718055994530942;
    if (log_psi) log_psi[w] = lp;
    if (KIN) e_loc[w] = -0.5 * (jscal[ldm + w] + widen(tr0 + tr0_o + sum_k * recip_x2(sum_r))) + jscal[2 * ldm + w];
  }
}

namespace {

int table_stride_x2(const WfDev& wf, bool kin) {
  const int tab = kin ? wf.tab_elems : (wf.nh[0] * wf.nv[0] + wf.nh[1] * wf.nv[1]);
  return tab | 1;
}

template <int NS>
cudaError_t launch_x2_ns(const WfDev& wf, int64_t W, const Workspace& ws, bool kin, double* e_loc, double* log_psi,
                         cudaStream_t st) {
  const dim3 grid((unsigned)((W + kWalkersPerBlockX2 - 1) / kWalkersPerBlockX2));
  const int stride = table_stride_x2(wf, kin);
  const size_t smem = det_x2_smem_bytes(wf, kin);
  auto kern = kin ? k_det_x2<NS, true> : k_det_x2<NS, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, kThreadsX2, smem, st>>>(wf, W, ws.mo, ws.nmp, ws.ldm, ws.jscal, stride, e_loc, log_psi);
  return cudaGetLastError();
}

}  // namespace

size_t det_x2_smem_bytes(const WfDev& wf, bool kin) {
  return sizeof(f32x2) * ((size_t)kWalkersPerBlockX2 * table_stride_x2(wf, kin) +
                          2 * kWalkersPerBlockX2 * kLanes * kLanes + ((wf.n_det + 1) & ~1)) +
         sizeof(int4) * (size_t)wf.n_det;
}

cudaError_t launch_det_x2(const WfDev& wf, int64_t W, const Workspace& ws, bool kinetic, double* e_loc,
                          double* log_psi, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  const int ns = wf.n_up > wf.n_down ? wf.n_up : wf.n_down;
  switch (ns) {
    case 1: return launch_x2_ns<1>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 2: return launch_x2_ns<2>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 3: return launch_x2_ns<3>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 4: return launch_x2_ns<4>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 5: return launch_x2_ns<5>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 6: return launch_x2_ns<6>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 7: return launch_x2_ns<7>(wf, W, ws, kinetic, e_loc, log_psi, st);
    case 8: return launch_x2_ns<8>(wf, W, ws, kinetic, e_loc, log_psi, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qmc
