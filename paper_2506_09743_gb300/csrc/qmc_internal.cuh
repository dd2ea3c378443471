// Internal declarations of the GB300 VMC engine (not part of the C ABI).
//
// Data layout in HBM (W walkers, ldm = W rounded up to 32):
//   walkers        double [3N][ldw]            caller-owned, coordinate-major
//   grad J         TA     [3N][ldm]            Jastrow gradient per electron
//   jastrow scal.  double [3][ldm]             J, sum_i(lap_i J + |grad_i J|^2), V
//   MO channels    double [N][NCH][nmp][ldm]   walker fastest; channel 0 =
//                                              Phi_{i,m}, channel 1 =
//                                              (lap + 2 grad J . grad) Phi_{i,m};
//                                              orbitals padded to nmp (8/16/32)
// with TA = double (FP64 form) or float (other forms).  The MO channels are
// stored in FP64 in every form (FP32 results widened exactly): the
// determinant stage, bound by the FP64 pipe, then reads its operands
// without conversion.  Every array is
// walker fastest: the kernels map consecutive threads (or consecutive
// tensor-memory rows) to consecutive walkers, so each warp-wide load or
// store of one element touches one contiguous span.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qmc.h"
#include "f32x2.cuh"

namespace qmc {

constexpr int kMaxShells = 128;
constexpr int kMaxExc = 512;   // unique excitations per spin channel
constexpr int kMaxDets = 4096;
constexpr int kMaxEen = 8;       // electron-electron-nucleus Jastrow terms
constexpr int kMaxShellAo = 16;  // AOs of one shell record (longer runs are split)
constexpr int kTcPass = 32;      // AO columns per K-pass of the tensor-core AO stage
constexpr int kMaxTcPass = 16;   // passes (QMC_MAX_AO columns, gaps of < kMaxShellAo per pass)

// One radial function shared by the AOs of a shell (same atom, kind, kn, l
// and primitives).  Radial normalisation and contraction coefficients are
// folded into coef; the per-AO angular factor is folded into the MO table.
struct ShellDev {
  int atom, kind, kn, l;
  int n_prim, ao_first, n_ao;
  int canon;  // 1 + l for a complete Cartesian s, p or d shell, else 0 (FP32X2 form:
              // its MO table rows are in the canonical order s; x, y, z; xx, xy, xz, yy, yz, zz)
  double expo[QMC_MAX_PRIM];
  double coef[QMC_MAX_PRIM];
  float expo_f[QMC_MAX_PRIM];  // FP32 copies: FP32 kernels must not convert
  float coef_f[QMC_MAX_PRIM];  // (double->float runs on the FP64 pipe)
  float expo_lo[QMC_MAX_PRIM];  // expo - expo_f and coef - coef_f as floats: the
  float coef_lo[QMC_MAX_PRIM];  // pairs (hi, lo) of the FP32X2 form (2^-48)
  float c2a_f[QMC_MAX_PRIM], c2a_lo[QMC_MAX_PRIM];  // 2 alpha c as pairs (GTO kinetic sums)
  float c4a_f[QMC_MAX_PRIM], c4a_lo[QMC_MAX_PRIM];  // 4 alpha^2 c as pairs
};

// Bins of the squared electron-nucleus distance for the FP32X2 row-scale
// tables, read off the FP32 bit pattern of r^2: bin 0 holds r^2 < 2^-24, bins
// 1 .. 640 sixteen per octave of r^2 up to 2^16, bin 641 everything beyond.
constexpr int kOzBoundBins = 642;
constexpr int kOzBoundBase = (127 - 24) << 4;  // (biased exponent of 2^-24) x 16
__host__ __device__ inline int oz_bound_bin(float r2) {
#if defined(__CUDA_ARCH__)
  const uint32_t u = __float_as_uint(r2);
#else
  uint32_t u;
  __builtin_memcpy(&u, &r2, 4);
#endif
  const int idx = (int)(u >> 19) - kOzBoundBase + 1;
  return idx < 0 ? 0 : (idx > kOzBoundBins - 1 ? kOzBoundBins - 1 : idx);
}

// Everything a kernel needs, passed by value (pointers are device memory).
struct WfDev {
  int n_atom, n_up, n_down, n_elec;
  int n_ao, n_mo, n_shell, n_det;
  int n_exc[2];   // unique excitation records per spin (index 0 = ground)
  int h_lo[2];    // smallest hole index per spin (n_s if none)
  int p_hi[2];    // one past the largest particle index per spin (n_s if none)
  int nh[2], nv[2];  // table extents: holes n_s - h_lo, virtuals p_hi - n_s
  int tab_elems;  // doubles of excitation tables per walker
  double w0_par, w0_anti, jb, bf_w, vnn;
  float w0p_f, w0a_f, jb_f;  // FP32 copies for the FP32 kernels
  // many-body Jastrow (App. D): electron-nucleus kernel (w0, w1, w2) when
  // mb_en, and n_een electron-electron-nucleus terms (c, a1, b1, a2, b2, a3, b3)
  int mb_en, n_een;
  double jen[3];
  double jeen[kMaxEen][7];
  float jen_f[3];  // FP32 copies for the FP32 kernels
  float jeen_f[kMaxEen][7];
  double atom_xyz[QMC_MAX_ATOMS][3];
  double atom_z[QMC_MAX_ATOMS];
  const ShellDev* shells;  // [n_shell]
  const int* ao_pow;       // [n_ao] kx | ky << 4 | kz << 8
  const double* mo64;      // [n_ao][n_mo] MO coefficients x AO angular factors
  const float* mo32;       // same, FP32
  const float2* mo_x2;     // same as pairs of FP32 (hi, lo) for the FP32X2 form
  // FP32X2 form on the tensor cores: MO columns scaled by 2^-oz_colexp[m] and
  // cut into six signed 8-bit digits, BF16 [6][16][k_pad] in the K-major
  // core-matrix layout of the B operand (oz_digits.cuh, k_ao_mo_oz.cu)
  const uint16_t* mo_oz;
  int oz_colexp[16];
  int oz;                  // 1: the FP32X2 form contracts on the tensor cores
  // per-atom upper bounds for the row scales of k_ao_mo_oz, [n_atom][kOzBoundBins]
  // {|AO value|, |kinetic value| = x + |grad J| y} over bins of r^2 (oz_bound_bin);
  // nullptr: the kernel bounds every shell instead
  const float4* oz_bound;
  int tc_value;            // 1: the FP32X2 form's Metropolis value path runs k_ao_mo_tc (FP32 AOs)
  int det_x2;              // 1: the FP32X2 form's determinant stage runs k_det_x2 (pairs of FP32), 0: k_det (FP64)
  const float* exp_tab;    // [64][2] 2^(j/64) as pairs: exp of the FP32X2 form
  const float2* mo_x2n;    // [n_ao][n_mo] MO table (angular factors folded in) as pairs, AO order
  int gen_x2;              // 1: the general (backflow) kernels evaluate the orbitals in pairs of FP32
  const int* exc;          // [2][kMaxExc][5] rank, h1, h2, p1, p2
  const int* det_idx;      // [n_det][2] excitation index per spin
  const int* det_orig;     // [n_det] index of each (sorted) determinant in the caller's order
  const double* det_w;     // [n_det]
  // [n_det] {packed offsets up, rank up, packed offsets down, rank down}:
  // table offsets (h_a - h_lo) nv + (p_b - n_s) of the k x k block, 8 bits
  // each in the order (h1 p1), (h1 p2), (h2 p1), (h2 p2)
  const int4* det_tab;
  // tensor-core B operand: MO^T split into high and low parts, K-major
  // core-matrix layout [n_mo_pad=16][k_pad], 32-bit words
  const uint32_t* mo_tc_hi;
  const uint32_t* mo_tc_lo;
  const double* ao_ang;  // [n_ao] angular normalisation factors (folded into mo64)
  const int* ao_prim;    // [n_ao + 1] first input primitive of each AO (gradient layout)
  // tensor-core AO stage: AO b sits in column ao_col[b] of the K dimension,
  // packed into n_pass passes of kTcPass columns (no shell straddles two
  // passes); in pass p, thread part q evaluates the shells
  // tc_shells[part_off[p][q] .. part_off[p][q+1]), and the columns of
  // pass_zero[p] (bit k = column k) are unused (zero).  A list entry is
  // shell | first column within the pass << 8 | type << 16, type 1 + l for a
  // complete s, p or d shell whose AOs sit in canonical Cartesian order
  // (x, y, z; xx, xy, xz, yy, yz, zz) from that column, 0 otherwise.  The
  // same shells split into two parts per row follow in
  // tc_shells[part2_off[p][q] .. part2_off[p][q+1]) (k_ao_mo_oz with two
  // thread groups).
  const int* ao_col;     // [n_ao]
  const int* tc_shells;  // [2][n_shell]
  long long wait_cycles; // budget of a bounded device wait, SM clock cycles (qmc_set_wait_limit)
  int k_pad;             // n_pass * kTcPass (0 when the form has no tensor-core stage)
  int n_pass;
  unsigned pass_zero[kMaxTcPass];
  int part_off[kMaxTcPass][5];
  int part2_off[kMaxTcPass][3];
};

struct Workspace {
  int64_t ldm;
  int nmp;         // padded orbital count of an MO row
  void* gradJ;     // TA [3N][ldm]
  double* jscal;   // [3][ldm]
  double* mo;      // [N][NCH][nmp][ldm]
  double* prop;    // [3N][ldm] proposed positions (sampling)
  double* lp;      // [ldm] current log|Psi| (sampling)
  double* lp_new;  // [ldm] proposed log|Psi| (sampling)
  uint64_t* ctr;   // step counter of a replayed Metropolis step graph
};

__host__ __device__ inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// the precision form keeps its Jastrow gradient in FP64 (QMC_FP64) or FP32
inline bool grad_fp64(int prec) { return prec == QMC_FP64; }

// padded orbital count of an MO row: the tensor-core forms always use 16
inline int mo_row_pad(int n_mo, bool tensor_core) {
  if (tensor_core) return 16;
  return n_mo <= 8 ? 8 : n_mo <= 16 ? 16 : 32;
}

#ifdef __CUDACC__
// Split a double into two floats hi + lo (hi = d truncated to 24 bits,
// lo = the next 24 bits) using integer operations and an integer->float
// conversion only; relative error 2^-48.  Magnitudes below 2^-70 give 0.
__device__ __forceinline__ void split_f64(double d, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ffu);
  if (e < 953) {
    hi = __uint_as_float(sign);
    lo = 0.0f;
    return;
  }
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
  const float l = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull)) * __uint_as_float((unsigned)(e - 948) << 23);
  lo = sign ? -l : l;
}

// Exact float -> double widening with integer operations only (no FP64-pipe
// conversion).  Subnormal inputs are flushed to signed zero.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  unsigned hi;
  if (ex == 0u) hi = sign;
  else if (ex == 0xffu) hi = sign | 0x7ff00000u | (man >> 3);
  else hi = sign | ((ex + 896u) << 20) | (man >> 3);
  const unsigned lo = ex == 0u ? 0u : (man << 29);
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double d) { return d; }
// hi + lo of a pair, exact in FP64 (|lo| <= 2^-24 |hi|: at most 48 bits)
__device__ __forceinline__ double widen(f32x2 a) { return widen(a.hi) + widen(a.lo); }

// Bitwise select c ? x : y, opaque to the optimiser.  Register arrays that
// are permuted by runtime pivot indices stay in registers (a plain select
// chain over a row index may be turned into an indexed access, which moves
// the whole array to local memory).
__device__ __forceinline__ double dsel(bool c, double x, double y) {
  double r;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\tselp.b64 %0, %2, %3, q;\n\t}"
      : "=d"(r)
      : "r"((int)c), "d"(x), "d"(y));
  return r;
}
__device__ __forceinline__ int isel(bool c, int x, int y) {
  int r;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\tselp.b32 %0, %2, %3, q;\n\t}"
      : "=r"(r)
      : "r"((int)c), "r"(x), "r"(y));
  return r;
}

// |x| as an ordered integer key (the IEEE bit pattern with the sign cleared
// orders like |x| for finite x), so pivot search needs no FP64 compare.
__device__ __forceinline__ long long abs_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffll;
}

// Reciprocal by Newton-Raphson iteration r <- r + r (1 - a r) (quadratic
// convergence) from an FP32 seed: the seed is built from the top bits of a
// with integer operations, inverted with the FP32 reciprocal (error < 2^-22)
// and widened back; two iterations reach the FP64 rounding level.  4 FP64
// instructions instead of a full division.  Pivots outside the FP32 range
// (never met by orbital matrices) take the IEEE division.
__device__ __forceinline__ double recip(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const int e = (int)((u >> 52) & 0x7ffu);
  if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / a;
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const float af = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((u >> 29) & 0x7fffffu));
  const unsigned rb = __float_as_uint(__frcp_rn(af));
  const unsigned re = (rb >> 23) & 0xffu;
  double r = __hiloint2double((int)((rb & 0x80000000u) | ((re + 896u) << 20) | ((rb & 0x7fffffu) >> 3)),
                              (int)(rb << 29));
  r = fma(r, fma(-a, r, 1.0), r);
  r = fma(r, fma(-a, r, 1.0), r);
  return r;
}

template <int TS>
__device__ __forceinline__ double team_sum(double v) {
#pragma unroll
  for (int o = TS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
#endif

size_t tc_smem_bytes(const WfDev& wf, int nch);
size_t det_smem_bytes(const WfDev& wf, bool kin);
size_t det_x2_smem_bytes(const WfDev& wf, bool kin);  // k_det_x2 (QMC_FP32X2 form)

// initial walker positions for the serving loop: home nucleus per electron
struct InitSpec {
  int n_elec;
  double home_xyz[2 * QMC_MAX_SPIN_ELECTRONS][3];
};
cudaError_t launch_init_walkers(const InitSpec& spec, int64_t W, int64_t ldw, double* walkers, uint64_t seed,
                                cudaStream_t st);
cudaError_t launch_sum_counts(const int64_t* counts, int64_t W, double* out, cudaStream_t st);

// general single-determinant FP64 path (backflow, forces, parameter gradient)
bool general_supported(const WfDev& wf);
// backflow with several determinants: <= 8 electrons, <= 4 per spin, <= 8 orbital columns
bool bf_multidet_supported(const WfDev& wf);
int general_blocks(int64_t W);
size_t grad_smem_bytes(const WfDev& wf, int n_param);
// multi-determinant parameter gradient (no backflow; k_md_grad.cu)
bool md_grad_supported(const WfDev& wf);
size_t md_grad_smem_bytes(const WfDev& wf, int n_param);
size_t md_grad_scratch_bytes(const WfDev& wf, int64_t ldm, int n_param, int n_sm);
cudaError_t launch_row_sums(const double* partial, int n_rows, int n_cols, double* out, cudaStream_t st);
cudaError_t launch_md_grad(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                           const double* e_loc, const double* stats, int n_prim, int n_param, double* scratch,
                           double* grad, cudaStream_t st, int weight = 0);
cudaError_t launch_eloc_general(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, bool kinetic,
                                double* e_loc, double* log_psi, cudaStream_t st);
cudaError_t launch_mean_var(const double* x, int64_t W, double* stats, cudaStream_t st);
// mean and variance of the finite values; stats[2] = number of non-finite values
cudaError_t launch_mean_var_finite(const double* x, int64_t W, double* stats, cudaStream_t st);
// raw = false: the forces of Eq. force; raw = true: the three sums of a
// sharded batch (sum d E_L, sum d ln rho, sum E_L d ln rho), 9 n_atom values
cudaError_t launch_forces(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const double* e_loc,
                          const double* stats, double* partial, double* forces, cudaStream_t st, bool raw = false);
// weight 0: the gradient of Eq. nabla_loss; 1: sum d log|Psi|; 2: sum E_L d log|Psi|
cudaError_t launch_grad(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const double* e_loc,
                        const double* stats, const double* ang, const int* prim_start, int n_param, double* partial,
                        double* grad, cudaStream_t st, int weight = 0);
// out[0..2] = M, sum E_L, sum E_L^2 (one block, fixed order)
cudaError_t launch_energy_sums(const double* e_loc, int64_t W, double* out, cudaStream_t st);

// kernel launchers (return cudaError_t of the launch)
// dynamic shared memory of the electron-electron-nucleus Jastrow kernel
size_t een_shared_bytes(const WfDev& wf, bool fp64);
// copy: null, or a device buffer [3N][ldw] that receives the positions read
// from walkers (which may then be mapped host memory; later stages read copy)
cudaError_t launch_jastrow(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw, double* copy,
                           const Workspace& ws, bool derivs, cudaStream_t st);
cudaError_t launch_ao_mo_simt(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                              const Workspace& ws, int nch, cudaStream_t st);
// pairs of FP32 (QMC_FP32X2 form): SIMT contraction, and the digit-sliced
// tensor-core contraction where oz_supported
size_t oz_smem_bytes(const WfDev& wf, int nch, int groups);
bool oz_supported(const WfDev& wf);
int oz_groups(const WfDev& wf, int nch);  // thread groups of k_ao_mo_oz (1 or 2)
cudaError_t launch_ao_mo_oz(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                            int nch, int* err_flag, int* err_wf, cudaStream_t st);
cudaError_t launch_ao_mo_x2(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                            int nch, cudaStream_t st);
cudaError_t launch_ao_mo_tc(const WfDev& wf, int prec, const double* walkers, int64_t W, int64_t ldw,
                            const Workspace& ws, int nch, int* err_flag, int* err_wf, cudaStream_t st);
cudaError_t launch_det(const WfDev& wf, int prec, int64_t W, const Workspace& ws, bool kinetic,
                       double* e_loc, double* log_psi, cudaStream_t st);
// the same in pairs of FP32 (QMC_FP32X2 form, table method)
cudaError_t launch_det_x2(const WfDev& wf, int64_t W, const Workspace& ws, bool kinetic, double* e_loc,
                          double* log_psi, cudaStream_t st);
// explicit per-excitation determinants (the baseline of the table method)
size_t det_explicit_smem_bytes(const WfDev& wf, bool kin);
cudaError_t launch_det_explicit(const WfDev& wf, int prec, int64_t W, const Workspace& ws, bool kinetic,
                                double* e_loc, double* log_psi, cudaStream_t st);
cudaError_t launch_propose(const WfDev& wf, const double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                           double step, uint64_t seed, uint64_t first_walker, uint64_t gstep, const uint64_t* gctr,
                           cudaStream_t st);
cudaError_t launch_accept(const WfDev& wf, double* walkers, int64_t W, int64_t ldw, const Workspace& ws,
                          uint64_t seed, uint64_t first_walker, uint64_t gstep, const uint64_t* gctr,
                          int64_t* n_accept, cudaStream_t st);
// the Box-Muller tables of the proposal kernels on the current device (once
// per device; synchronous)
cudaError_t init_box_muller_tables();
// *gctr += 1 (one thread): the step counter of a replayed step graph
cudaError_t launch_step_advance(uint64_t* gctr, cudaStream_t st);

}  // namespace qmc
