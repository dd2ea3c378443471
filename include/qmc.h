/*
 * qmc.h - C ABI of the GB300 variational Monte Carlo local-energy engine.
 *
 * The library evaluates, for a batch of electron configurations ("walkers"),
 * the local energy E_L = H Psi / Psi of a Slater-Jastrow(-backflow)
 * wavefunction, samples |Psi|^2 with a Metropolis walker step, and returns
 * the low-variance energy gradient and the interatomic forces.  The method
 * is the one of QMCTorch (arXiv:2506.09743):
 *
 *   H      = -1/2 sum_i lap_i + sum_{i>j} 1/r_ij - sum_{i,a} Z_a/r_ia
 *            + sum_{a>b} Z_a Z_b / R_ab                          (Eq. Hmol)
 *   Psi    = exp(J(r)) sum_n d_n D_n^up(r~^up) D_n^dn(r~^dn)    (Eq. psimol)
 *   r~_i   = r_i + sum_{j!=i} (w / r_ij)(r_i - r_j)   (Sec. 2.1, Sec. 3)
 *   J      = sum_{i<j} w0 r_ij / (1 + b r_ij)       (Eqs. jastrow, pade_kernel)
 *   kinetic term by the trace formulas of App. F and App. G and the
 *   excited-determinant table method (Eq. table, App. F / App. H).
 *
 * Conventions (all calls):
 *  - Walker coordinates are float64, coordinate-major ("SoA"): element
 *    [k][w] at walkers[k * ldw + w], k = 3*i + d for electron i (up electrons
 *    first, 0 .. n_up-1) and axis d (x, y, z); ldw >= n_walkers.  Units bohr.
 *  - Device pointers are owned by the caller and are not retained after the
 *    call returns.  Host pointers are read (or written) before return.
 *  - Calls taking a `stream` (a cudaStream_t passed as void*; NULL = legacy
 *    default stream) are stream-ordered and asynchronous unless they return
 *    a value on the host, in which case they synchronise that stream.
 *  - Every call returns a qmc_status and never aborts the process; on error
 *    qmc_last_error() gives a message (thread-local, valid until the next
 *    call on the same thread).  A walker whose energy is not finite (an
 *    electron exactly on a nucleus or on another electron, or exactly on a
 *    node) gets NaN and does not fail the call.
 *  - A qmc_wf is not safe for concurrent calls on different streams when the
 *    library-owned workspace is used (workspace == NULL); pass a separate
 *    caller-owned workspace per concurrent call instead.
 */
#ifndef QMC_GB300_H
#define QMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qmc_wf qmc_wf; /* opaque; owns its device-resident tables */

typedef enum {
  QMC_OK = 0,
  QMC_ERR_ARG = 1,         /* invalid argument (null pointer, bad size, bad index) */
  QMC_ERR_OOM = 2,         /* device allocation failed or workspace too small */
  QMC_ERR_CUDA = 3,        /* a CUDA runtime error; message has the CUDA text */
  QMC_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  QMC_ERR_UNSUPPORTED = 5, /* shape outside the compiled limits (see below) */
  QMC_ERR_CANCELLED = 6    /* a server request cancelled by qmc_server_cancel */
} qmc_status;

/* Precision forms of the local energy.
 *  QMC_FP64        everything in FP64 (AO, AO->MO contraction, determinants).
 *  QMC_FP32        FP32 AOs and SIMT FP32 AO->MO contraction; determinant LU,
 *                  log|det|, inverse update and energy assembly in FP64.
 *  QMC_MIXED_TF32  FP32 AOs; AO->MO contraction on tcgen05 tensor cores with
 *                  TF32 inputs split into high and low parts (three products,
 *                  FP32 accumulation in tensor memory); FP64 determinants.
 *  QMC_MIXED_BF16  not built: QMC_ERR_UNSUPPORTED.
 *  QMC_FP32X2      local energies with AOs in pairs of FP32 (hi + lo, about
 *                  48 significant bits, on the FP32 pipes), the AO->MO
 *                  contraction exact on the tcgen05 tensor cores (the pairs
 *                  cut into BF16 digits; SIMT pairs when n_mo > 16,
 *                  n_ao > 96 or n_ao n_mo < 256), electron-nucleus potential in pairs of
 *                  FP32 and electron-electron terms in compensated FP32: MO
 *                  values within about 2^-43 of |AO||C|, so that the local
 *                  energy matches the FP64 form to 2e-4 Ha on every walker
 *                  away from the nodes (where FP32 AOs leave about one CO
 *                  walker in six beyond it).  The determinant stage (table
 *                  method) runs in pairs of FP32 on rows scaled by powers of
 *                  two where its FP64 form would cost at least 3,000 flops per
 *                  walker (CO with 100 determinants: 6,560), in FP64
 *                  otherwise; the explicit method stays FP64.  The Metropolis
 *                  value path (log|Psi| of the acceptance test) evaluates the
 *                  orbitals as MIXED_TF32 does: FP32-level log|Psi|.
 * Jastrow terms are FP64 in QMC_FP64 and use FP32 pair arithmetic with
 * compensated sums in the other forms; the Coulomb potential is FP64 in
 * QMC_FP64; in QMC_FP32X2 its electron-nucleus terms are pairs of FP32 and
 * its electron-electron terms refined FP32 reciprocals with compensated
 * sums; FP32 terms with compensated sums otherwise.  Backflow wavefunctions run in QMC_FP64 and QMC_FP32X2; in
 * QMC_FP32X2 only their orbitals (AO values, derivatives and the AO->MO
 * contraction, s and p shells) are in pairs of FP32, while the Jastrow
 * factor, the backflow map, the potential, the determinants and the
 * Laplacian stay FP64 (and so does the value path). */
typedef enum {
  QMC_FP64 = 0,
  QMC_FP32 = 1,
  QMC_MIXED_TF32 = 2,
  QMC_MIXED_BF16 = 3,
  QMC_FP32X2 = 4
} qmc_precision;

/* Compiled limits (QMC_ERR_UNSUPPORTED beyond them). */
#define QMC_MAX_ATOMS 16
#define QMC_MAX_SPIN_ELECTRONS 8 /* per spin channel */
#define QMC_MAX_MO 32            /* MOs (tensor-core forms: 16) */
#define QMC_MAX_AO 256           /* AOs */
#define QMC_MAX_PRIM 8           /* primitives per contracted Gaussian */

/* Nuclei and electron counts (Eq. Hmol).  Host arrays. */
typedef struct {
  int32_t n_atom;
  const double* xyz; /* [n_atom][3] nuclear positions, bohr */
  const double* z;   /* [n_atom] nuclear charges */
  int32_t n_up;      /* electrons of spin up (electrons 0 .. n_up-1) */
  int32_t n_down;    /* electrons of spin down */
} qmc_atoms;

/* Atomic orbitals (Sec. 2.1).  AO b is centred on atom ao_atom[b] with
 * d = r - R: kind 0 (Slater) phi = N dx^kx dy^ky dz^kz |d|^kn exp(-zeta |d|)
 * with one primitive (zeta = prim_exp, prim_coef scales it); kind 1
 * (contracted Cartesian Gaussian) phi = sum_p c_p N_p dx^kx dy^ky dz^kz
 * exp(-alpha_p |d|^2).  Normalisation: STO radial (2 zeta)^(n+1/2)/sqrt((2n)!),
 * n = kn + l + 1, times sqrt((2l+1)!!/(4 pi (2kx-1)!!(2ky-1)!!(2kz-1)!!));
 * GTO primitive (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2kx-1)!!(2ky-1)!!(2kz-1)!!).
 * Host arrays. */
typedef struct {
  int32_t n_ao;
  const int32_t* ao_atom;       /* [n_ao] */
  const int32_t* ao_kind;       /* [n_ao] 0 = STO, 1 = GTO */
  const int32_t* ao_pow;        /* [n_ao][4] kx, ky, kz, kn */
  const int32_t* ao_prim_start; /* [n_ao + 1] offsets into prim_exp / prim_coef */
  const double* prim_exp;       /* zeta (STO) or alpha (GTO) */
  const double* prim_coef;      /* contraction coefficients */
} qmc_basis;

/* Molecular orbitals phi_m = sum_b C[b][m] AO_b (Sec. 2.1; the paper's
 * c x mu product).  Host array [n_ao][n_mo], row-major. */
typedef struct {
  int32_t n_mo;
  const double* coeff;
} qmc_mos;

/* Determinant expansion sum_n d_n D_n^up D_n^dn (Eq. psimol).  Per
 * determinant and spin an excitation record (rank, h1, h2, p1, p2): the
 * ground-state columns h1 < h2 (orbitals 0 .. n_s-1) are replaced in place
 * by virtual orbitals p1 < p2 (Eq. AX, App. H); rank 0 = ground state, rank
 * at most 2, unused entries -1.  Host arrays. */
typedef struct {
  int32_t n_det;
  const double* weight; /* [n_det] CI weights d_n */
  const int32_t* exc;   /* [n_det][2][5] */
} qmc_dets;

/* Pade electron-electron Jastrow u(r) = w0 r / (1 + b r), w0 = w0_par for
 * parallel and w0_anti for antiparallel spins (Eq. pade_kernel, App. D),
 * and the inverse backflow kernel K(r) = backflow_w / r (Sec. 3; 0 = off). */
typedef struct {
  double w0_par;
  double w0_anti;
  double b;
  double backflow_w;
} qmc_jastrow;

typedef struct {
  int32_t precision; /* qmc_precision */
  int32_t device;    /* CUDA device ordinal the tables live on */
} qmc_options;

/* Build a wavefunction: validates the inputs, computes normalisations and the
 * device-resident tables on `opt->device`.  *out is set on QMC_OK.  Defines
 * Psi of Eq. psimol with the pieces above. */
qmc_status qmc_create_wf(const qmc_atoms* atoms, const qmc_basis* basis, const qmc_mos* mos,
                         const qmc_dets* dets, const qmc_jastrow* jastrow, const qmc_options* opt,
                         qmc_wf** out);

/* Free a wavefunction and its device tables (NULL is a no-op). */
void qmc_destroy_wf(qmc_wf* wf);

/* Move the nuclei (same basis, MOs and determinants), e.g. along a bond
 * (Sec. 3.3).  xyz: host [n_atom][3].  Stream-ordered on the legacy stream
 * (synchronous). */
qmc_status qmc_set_geometry(qmc_wf* wf, const double* xyz);

/* Bytes of device scratch that one call with n_walkers needs when a caller
 * workspace is passed (0 on error). */
size_t qmc_workspace_size(const qmc_wf* wf, int64_t n_walkers);

/* Local energies (Eq. Hmol, kinetic term by App. F / App. G and Eq. table):
 * e_loc[w] = E_L(r_w) and, if log_psi != NULL, log_psi[w] = log|Psi(r_w)|.
 * walkers: device [3N][ldw]; e_loc, log_psi: device [n_walkers].
 * workspace: device scratch of at least qmc_workspace_size(wf, n_walkers)
 * bytes, or NULL to use a library-owned buffer (grown on demand).
 * n_walkers = 0 is a no-op. */
qmc_status qmc_local_energy(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw,
                            double* e_loc, double* log_psi, void* workspace, size_t workspace_bytes,
                            void* stream);

/* As qmc_local_energy with HOST buffers: evaluates into library-owned device
 * memory and copies e_loc (and log_psi if not NULL) back; returns after the
 * results are on the host.  walkers: host [3N][n_walkers] (ldw = n_walkers).
 * Page-locked walkers mapped into the wavefunction's device (as
 * cudaHostAlloc / torch pin_memory give them) are read by the first kernel
 * directly and copied to device memory on the way; other host memory is
 * uploaded with one copy before it (backflow wavefunctions always take the
 * copy).  Results are identical either way.  Host buffers should be pinned
 * for full speed. */
qmc_status qmc_local_energy_host(qmc_wf* wf, const double* walkers, int64_t n_walkers,
                                 double* e_loc, double* log_psi, void* stream);

/* Bytes of the library's static device scratch array used by
 * qmc_local_energy_noalloc.  Every GPU that loads the library holds this
 * much device memory until the process exits. */
#define QMC_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* qmc_local_energy for callers that must not allocate device memory during a
 * call.  The paper has no counterpart; this is an integration aid.  Such
 * callers include a serving loop that runs requests concurrently on several
 * streams under a fixed device-memory budget (a cudaMalloc stalls the whole
 * device and can fail once memory is fragmented), processes whose device
 * memory is owned by another allocator (a framework's caching pool), and
 * latency-bound callers that cannot absorb an allocation inside a request.
 * Same computation and results as qmc_local_energy, but the device scratch is
 * a fixed static array of QMC_NOALLOC_SCRATCH_BYTES inside the library: no
 * cudaMalloc, cudaFree or allocating library routine is called.
 * Limit: qmc_workspace_size(wf, n_walkers) <= QMC_NOALLOC_SCRATCH_BYTES;
 * larger batches return QMC_ERR_ARG with the largest admissible count in the
 * message (split them into several calls).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * previous call's contents (what must start at zero is cleared by the call
 * itself): calls that overlap on the GPU, on any stream or from any thread,
 * race on it and must be serialised by the caller.
 * walkers, e_loc, log_psi: as for qmc_local_energy. */
qmc_status qmc_local_energy_noalloc(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw,
                                    double* e_loc, double* log_psi, void* stream);

/* Bounded device waits (an engineering aid; the paper has no counterpart).  The
 * tensor-core AO stage (QMC_MIXED_TF32) waits on mbarriers for its MMAs;
 * every such wait is bounded (about one second of SM clock).  A wait that
 * gives up makes its block record the failure, wait (bounded again) for the
 * MMAs it already issued, write NaN for the MO values of the walkers it had
 * left and stop, so the affected walkers' results are NaN; nothing hangs.
 * The failure is reported as QMC_ERR_TIMEOUT:
 *  - by qmc_local_energy_host, which synchronises anyway;
 *  - in the status of a server result (qmc_result.status);
 *  - for the stream-ordered calls (qmc_local_energy, qmc_local_energy_noalloc,
 *    qmc_sample), by qmc_check_status below.
 * The other precision forms run no device waits. */

/* Waits for the work queued on `stream` and returns QMC_ERR_TIMEOUT if a
 * bounded device wait of this wavefunction's kernels gave up since the last
 * check (then clears the record), QMC_OK otherwise. */
qmc_status qmc_check_status(qmc_wf* wf, void* stream);

/* Testing aid: the budget of each bounded device wait in SM clock cycles
 * (default 2^31, about one second).  0 makes every wait give up at once on a
 * healthy GPU, which exercises the timeout path (QMC_ERR_TIMEOUT, NaN
 * results); the drain of the MMAs already issued always keeps the default
 * budget.  Applies to the calls that follow.  QMC_ERR_ARG if negative. */
qmc_status qmc_set_wait_limit(qmc_wf* wf, int64_t cycles);

/* Metropolis-Hastings walker steps (App. B): every step moves all electrons
 * of a walker by step * z, z ~ N(0, 1) per coordinate, and accepts with
 * probability min(1, |Psi'/Psi|^2).  Random numbers: Philox4x32-10 with key
 * (seed mod 2^32, seed div 2^32) and counter (block, first_walker + w,
 * global step mod 2^32, global step div 2^32), global step = step_offset + t;
 * block j gives Gaussians 4j..4j+3 by Box-Muller on word pairs, block
 * ceil(3N/4) word 0 the acceptance uniform u, with u(x) = (x + 0.5) 2^-32;
 * accept iff log u < 2 (log|Psi'| - log|Psi|).  The result is therefore a
 * pure function of (wf, walkers, seed, first_walker, step_offset, n_steps,
 * step), independent of batching.
 * walkers: device [3N][ldw], updated in place.  log_psi: device [n_walkers],
 * if not NULL receives log|Psi| of the final positions.  n_accept: device
 * int64 [n_walkers], if not NULL incremented by each walker's accepted moves.
 * workspace as for qmc_local_energy (qmc_workspace_size covers it). */
qmc_status qmc_sample(qmc_wf* wf, double* walkers, int64_t n_walkers, int64_t ldw, int32_t n_steps,
                      double step, uint64_t seed, uint64_t first_walker, uint64_t step_offset,
                      double* log_psi, int64_t* n_accept, void* workspace, size_t workspace_bytes,
                      void* stream);

/* Mean and variance of E_L over the batch, the low-variance energy gradient
 * (Eq. nabla_loss, Sec. 2.2) and the forces on the nuclei (Eq. force,
 * Sec. 2.3), with E_v the batch mean and ln rho = 2 log|Psi|:
 *   grad[p]   = (2/M) sum_m d_p log|Psi(r_m)| (E_L(r_m) - E_v)
 *   forces[a] = -(1/M) sum_m [d_a E_L(r_m) + (E_L(r_m) - E_v) d_a ln rho(r_m)]
 * The parameter derivatives of log|Psi| are evaluated in closed form (Jacobi
 * formula through the backflow map, AOs recomputed per walker rather than
 * stored); the nuclear derivatives of E_L and log|Psi| by forward-mode
 * tangents through the whole local-energy evaluation.  Sums run in a fixed
 * order (results are bitwise reproducible).
 * Several determinants (Eq. psimol with the CI sum): d log|Psi| / d Phi_{a m}
 * from tables of the reference inverse (Eq. table): with T = A0^-1 Phi,
 * R_X = det T[h, p], S = sum_n d_n R_n^up R_n^dn and Y_{p h} = (dS/dT_{h p}) / S,
 *   d log|Psi| / d Phi_{a m} = [m occupied] (A0^-1)_{m a} + [(I - P T) Y A0^-1]_{m a},
 * contracted with the AOs for the MO coefficients and exponents;
 * d log|Psi| / d d_n = R_n^up R_n^dn / S.
 * Scope: FP64 form and either (a) one determinant, <= 8 electrons, <= 4 per
 * spin (gradient and forces; backflow allowed) or (b) no backflow, <= 8
 * electrons per spin, <= 16 orbitals, <= 128 distinct excitations per spin
 * (gradient only: forces must be NULL).  A many-body Jastrow takes path (b)
 * (its parameters are in the gradient; forces must be NULL)
 * (QMC_ERR_UNSUPPORTED otherwise).
 * walkers: device [3N][ldw].  e_stats: host [2] (mean, variance).  grad:
 * device [n_param] in qmc_param_layout order, or NULL.  forces: device
 * [n_atom][3], or NULL.  Synchronises the stream. */
qmc_status qmc_energy_grad(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, double* e_stats,
                           double* grad, double* forces, void* stream);

/* Sharded batches (several GPUs, or batches too large for one call): the
 * estimators of qmc_energy_grad are assembled from per-batch sums, so one
 * all-reduce (sum) of these sums across the shards gives the estimator of
 * the whole sample exactly (Eq. nabla_loss, Sec. 2.2; Eq. force, Sec. 2.3):
 *   E_v    = S_E / M,  var = S_EE / M - E_v^2
 *   grad   = 2 (S_E,dlogPsi - E_v S_dlogPsi) / M
 *   forces = -(S_dE + S_E,dlnrho - E_v S_dlnrho) / M,   ln rho = 2 log|Psi|
 * qmc_energy_grad_sums writes, stream-ordered into DEVICE memory `sums`
 * (qmc_energy_grad_sums_size(wf) doubles, ready for an all-reduce in place):
 *   [0] M (walkers), [1] S_E = sum E_L, [2] S_EE = sum E_L^2,
 *   [3, 3 + P)          sum d log|Psi| / d theta_p   (qmc_param_layout order, P = n_param)
 *   [3 + P, 3 + 2P)     sum E_L d log|Psi| / d theta_p
 *   then three blocks of 3 n_atom (atom-major, x y z):
 *                       sum d E_L / d R,  sum d ln rho / d R,  sum E_L d ln rho / d R.
 * Scope of qmc_energy_grad; on its path (b) (several determinants, or the
 * many-body Jastrow) the three force blocks are NaN (all bits set): the
 * forces need path (a).  Sums run in
 * a fixed order (bitwise reproducible).  qmc_assemble_energy_grad is the host
 * arithmetic above on the (reduced) sums, copied to the host: e_stats [2],
 * grad [n_param] (or NULL), forces [n_atom][3] (or NULL); QMC_ERR_ARG when
 * the sums count no walker. */
int64_t qmc_energy_grad_sums_size(const qmc_wf* wf);
qmc_status qmc_energy_grad_sums(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, double* sums,
                                void* stream);
qmc_status qmc_assemble_energy_grad(int64_t n_param, int32_t n_atom, const double* sums, double* e_stats,
                                    double* grad, double* forces);

/* Replace the variational parameters (host [n_param] in qmc_param_layout
 * order: exponents, MO coefficients, CI weights, Jastrow b, backflow w, then
 * the many-body Jastrow's when it is set) and
 * rebuild the device tables.  Waits for work in flight on the device.
 * Exponents must be positive; on error the previous parameters stay. */
qmc_status qmc_set_params(qmc_wf* wf, const double* params);

/* Number of variational parameters and the offsets of the gradient blocks:
 * offsets[0] exponents (one per primitive, prim_exp order), [1] MO
 * coefficients (row-major n_ao x n_mo), [2] CI weights, [3] Jastrow b,
 * [4] backflow w, [5] = n_param.  With a many-body Jastrow (App. D) its
 * parameters follow the backflow weight, from offsets[4] + 1 to n_param:
 * K_en (w0, w1, w2) if set, then per K_een term (c, a1, b1, a2, b2, a3, b3).
 * offsets may be NULL. */
qmc_status qmc_param_layout(const qmc_wf* wf, int64_t* n_param, int64_t offsets[6]);

/* Many-body Jastrow factor (App. D), added to the Pade electron-electron
 * kernel in J (Eq. jastrow):
 *   electron-nucleus        K_en(r) = (w0 r + w1 r^2) / (1 + w2 r), summed over
 *                           atoms a and electrons i, r = |r_i - R_a|;
 *   electron-electron-nucleus, n_een terms mu:
 *     K_een = sum_mu c_mu f(a1, b1; r_ai) f(a2, b2; r_aj) f(a3, b3; r_ij),
 *     f(a, b; r) = a r / (1 + b r), summed over atoms and ordered electron
 *     pairs i != j with a factor 1/2 (J stays symmetric under exchange).
 * Both are spin independent.  en: host [3] (w0, w1, w2) or NULL (no K_en);
 * een: host [n_een][7] (c, a1, b1, a2, b2, a3, b3), n_een <= 8 (0 = none).
 * Requires w2 >= 0 and b >= 0 (no pole at r >= 0): QMC_ERR_ARG otherwise.
 * Covers qmc_local_energy* and qmc_sample in every precision form;
 * QMC_ERR_UNSUPPORTED with backflow, or when the electron-electron-nucleus
 * tables (per walker: n_elec x n_atom x (6 + 6 n_een) values plus
 * 8 x n_elec (n_elec - 1) / 2 pair terms, four walkers per block) exceed the
 * 227 KB of shared memory of a block.  Its parameters join the gradient
 * layout (qmc_param_layout) and qmc_energy_grad's gradient (no forces).
 * On error the previous Jastrow stays.  Synchronous (rebuilds the device
 * tables). */
qmc_status qmc_set_manybody_jastrow(qmc_wf* wf, const double* en, int32_t n_een, const double* een);

/* Determinant method of the local-energy and sampling calls.
 *  QMC_DET_TABLE     (default) excited determinants from tables of the
 *                    reference inverse: D_X / D_0 and the kinetic trace of
 *                    each excitation from k x k minors (Eq. table, App. H).
 *  QMC_DET_EXPLICIT  every distinct spin excitation X gets its own matrix
 *                    A_X, factorised by LU with partial pivoting; D_X and
 *                    Tr(A_X^-1 B_X) (Jacobi formula) from the factors.  The
 *                    baseline of the paper's explicit-versus-table comparison
 *                    (Sec. 2.2, App. A); O(n^3) per distinct excitation.
 * Both give the same local energy up to rounding.  Backflow wavefunctions
 * (single determinant) ignore the setting.  QMC_ERR_ARG for an unknown
 * method; QMC_ERR_UNSUPPORTED when the explicit stage's shared-memory tables
 * (both spins' distinct excitations) do not fit. */
typedef enum { QMC_DET_TABLE = 0, QMC_DET_EXPLICIT = 1 } qmc_det_method;
qmc_status qmc_set_det_method(qmc_wf* wf, int32_t method);

/* ---- Wavefunction optimisation (App. B) and batched forces (Sec. 3.3) ----
 * qmc_optimize runs the optimisation loop of App. B on the FP64 form (within
 * the scope of qmc_energy_grad's gradient): n_equil Metropolis steps, then per optimisation step t = 1 ..
 * n_iter the energy gradient of Eq. nabla_loss at the current walkers, one
 * ADAM update of the optimised parameters (Kingma and Ba 2015, Algorithm 1;
 * App. B: lr 1e-2), the new parameters installed as by qmc_set_params, and
 * n_resample Metropolis steps with the updated wavefunction (App. B: 500).
 * Metropolis steps are numbered globally from 0 (step_offset of qmc_sample),
 * so the run is a pure function of its inputs; the ADAM moments start at zero
 * on every call.  ADAM rounds each operation once, in the order
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g*g;
 *   theta = theta - (lr (m / c1)) / (sqrt(v / c2) + eps),  c_k = 1 - b_k^t
 * with b_k^t formed by repeated multiplication.
 * walkers: device [3N][ldw], updated in place (the final samples).
 * cfg->mask: host [n_param] (qmc_param_layout order), nonzero = optimised;
 * NULL optimises every parameter.  history: host [n_iter][3]: E mean and
 * variance at the samples of step t (before its update) and the acceptance
 * rate of the resampling that follows it.  The wavefunction keeps the final
 * parameters.  Synchronous.  Errors of the composed calls are returned as
 * they are (the parameters then stay at the last successful update);
 * QMC_ERR_ARG for bad counts or hyper-parameters (0 <= beta < 1, eps > 0). */
typedef struct {
  int32_t n_iter;     /* optimisation steps */
  int32_t n_equil;    /* Metropolis steps before the first step */
  int32_t n_resample; /* Metropolis steps after each update */
  int32_t reserved;   /* must be 0 */
  double step;        /* Gaussian proposal width per coordinate, bohr */
  uint64_t seed;      /* Philox key */
  double lr, beta1, beta2, eps;
  const uint8_t* mask;
} qmc_opt_config;
qmc_status qmc_optimize(qmc_wf* wf, double* walkers, int64_t n_walkers, int64_t ldw, const qmc_opt_config* cfg,
                        double* history, void* stream);

/* Forces of Eq. force per batch of samples, as used along the dissociation
 * curves of Sec. 3.3: the walkers are split into n_batches consecutive
 * slices (the last takes the remainder) and, with symmetrize != 0, every
 * slice is joined by the images of its samples under x -> -x, y -> -y and
 * both (all electrons together; the symmetry of a molecule on the z axis),
 * before Eq. force is evaluated with that slice's mean energy.  FP64 form,
 * scope (a) of qmc_energy_grad (forces).  walkers: device [3N][ldw].
 * e_mean: host [n_batches] or NULL.  forces: host [n_batches][n_atom][3].
 * Synchronous; QMC_ERR_ARG unless 1 <= n_batches <= n_walkers. */
qmc_status qmc_force_batches(qmc_wf* wf, const double* walkers, int64_t n_walkers, int64_t ldw, int32_t n_batches,
                             int32_t symmetrize, double* e_mean, double* forces, void* stream);

/* Per-stage device timing (tracing aid; the paper has no counterpart).  When
 * enabled, every qmc_local_energy / qmc_sample evaluation records CUDA events
 * on its stream around its three stages: [0] Jastrow and Coulomb terms,
 * [1] AO evaluation and AO->MO contraction, [2] determinants, tables and
 * local-energy assembly.  Off by default (no events recorded). */
qmc_status qmc_set_timing(qmc_wf* wf, int32_t enable);

/* Milliseconds of each stage of the last timed evaluation on this wf
 * (ms[0..n-1], n <= 3).  Waits for that evaluation's last event.
 * QMC_ERR_ARG if timing was never enabled or nothing was timed yet. */
qmc_status qmc_last_stage_ms(qmc_wf* wf, float* ms, int32_t n);

/* ---- Continuous-batching request server --------------------------------
 * A request evaluates one registered wavefunction (a molecule at one
 * geometry): its walkers are uploaded or drawn on the device, n_steps
 * Metropolis steps are run (App. B), then the local energies (Eq. Hmol) and
 * their mean and variance, the Monte Carlo estimate of Sec. 1.  Requests are
 * queued on submission and admitted as soon as one of max_in_flight stream
 * slots is free and the request's device memory (walkers, scratch) fits in
 * the server's arena of hbm_budget_bytes; admitted requests run concurrently
 * on their own streams.  Admission policy (qmc_server_set_policy): requests
 * of at least big_walkers walkers ("large") are admitted in arrival order
 * with at most max_big of them in flight, on low-priority streams; the other
 * requests are admitted in arrival order, may pass a large request that is
 * waiting for its turn, and run on high-priority streams.  Memory is
 * first-come for all: a request that does not fit stops admission until
 * memory is released.  The arena is allocated
 * once at creation: admission allocates nothing.  A result depends only on
 * the request, not on the other requests in flight.  Single host thread:
 * call the server functions from one thread. */
typedef struct qmc_server qmc_server;

typedef struct {
  int32_t wf_id;          /* from qmc_server_add_wf */
  int64_t n_walkers;      /* >= 1 */
  int32_t n_steps;        /* Metropolis steps before the energy (>= 0) */
  double step;            /* proposal width, bohr (> 0 if n_steps > 0) */
  uint64_t seed;          /* Philox key of the chain (and of the initial positions) */
  const double* walkers;  /* host [3N][n_walkers] initial positions, kept valid until the
                             result is returned; or NULL: electron i drawn N(home nucleus,
                             1 bohr^2) on the device (nuclei dealt by Z, spins alternating,
                             Philox step index 2^64 - 1) */
} qmc_request;

typedef struct {
  int64_t ticket;
  int32_t status;       /* QMC_OK or the error of this request (QMC_ERR_TIMEOUT: a bounded
                           device wait gave up; the statistics are NaN) */
  int32_t wf_id;
  int64_t n_walkers;
  double e_mean;        /* mean local energy over the walkers with a finite one, Ha */
  double e_var;         /* variance of those local energies, Ha^2 */
  double accept_rate;   /* accepted moves / (n_walkers n_steps) */
  double t_submit;      /* qmc_server_clock() at submission, admission and completion, s */
  double t_admit;
  double t_done;
  int64_t n_nonfinite;  /* walkers whose local energy is not finite (left out of e_mean, e_var) */
} qmc_result;

/* Create a server on `device` with a device-memory arena of hbm_budget_bytes
 * and max_in_flight concurrent request slots (streams). */
qmc_status qmc_server_create(int32_t device, size_t hbm_budget_bytes, int32_t max_in_flight, qmc_server** out);

/* Wait for the requests in flight and free the server (not the wavefunctions). */
void qmc_server_destroy(qmc_server* srv);

/* Register a wavefunction (not owned; keep it alive while the server runs). */
qmc_status qmc_server_add_wf(qmc_server* srv, qmc_wf* wf, int32_t* wf_id);

/* Queue a request (never blocks).  QMC_ERR_OOM if it can never fit. */
qmc_status qmc_server_submit(qmc_server* srv, const qmc_request* req, int64_t* ticket);

/* Retire finished requests and admit queued ones; returns the numbers in
 * flight and still queued.  Call it repeatedly (it does not block). */
qmc_status qmc_server_progress(qmc_server* srv, int32_t* n_in_flight, int32_t* n_queued);

/* Cancel a request: a queued one is removed at once (no device work) and a
 * request in flight finishes its kernels but its statistics are dropped;
 * either way its result carries QMC_ERR_CANCELLED with NaN statistics and
 * its memory returns to the arena.  QMC_ERR_ARG for a ticket that is
 * neither queued nor in flight (unknown, or already finished). */
qmc_status qmc_server_cancel(qmc_server* srv, int64_t ticket);

/* Move up to `capacity` finished results into out (oldest first). */
qmc_status qmc_server_results(qmc_server* srv, qmc_result* out, int32_t capacity, int32_t* n_out);

/* Admission policy (see above): big_walkers = 0 treats every request alike
 * (plain arrival order); max_big_in_flight >= 1.  Defaults: 65536 and 2.
 * Applies to the admissions that follow. */
qmc_status qmc_server_set_policy(qmc_server* srv, int64_t big_walkers, int32_t max_big_in_flight);

/* Bytes of the arena currently free. */
size_t qmc_server_free_bytes(const qmc_server* srv);

/* The server's monotonic clock, seconds. */
double qmc_server_clock(void);

/* Message of the last failed qmc_server_* call on this thread. */
const char* qmc_server_last_error(void);

/* Message of the last failed call on this thread ("" if none yet).  The
 * pointer stays valid until the next library call on the same thread. */
const char* qmc_last_error(void);

/* Measured arithmetic rates of the current device, the denominators of the
 * FP64- and FP32-bound rooflines: rates[0] FP64 FMA/s, [1] FP32 FMA
 * instructions/s, [2] FP64 exp/s, [3] FP64 sqrt/s, [4] FP64 reciprocal (1/x)/s.
 * Each is timed with CUDA events over a probe kernel of eight independent
 * dependency chains per thread, 8 x 256 threads per SM (contractive maps:
 * every value stays finite).  Synchronous on `stream` (about 0.3 s); rates:
 * host [5].  QMC_ERR_ARG for NULL rates, QMC_ERR_OOM, QMC_ERR_CUDA. */
qmc_status qmc_measure_rates(double rates[5], void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QMC_GB300_H */
