"""Benchmark: walker local-energy evaluations per second, CO (14 electrons).

Workload: CO, 7 up + 7 down electrons, 58 contracted Cartesian GTOs (5s4p2d
per atom, 3 primitives), 14 MOs, 100 determinants of the (10e, 12o) active
space, Pade Jastrow; 262,144 seeded synthetic walkers per GPU.  One step =
one qmc_local_energy call over the whole batch (Jastrow + Coulomb, AO
evaluation, AO->MO contraction, reference inverse, excited-determinant
tables, E_L assembly).  The headline `value` is the FP32X2 form (AOs,
contraction, Coulomb potential and determinant stage in pairs of FP32), the
form that meets 2e-4 Ha per walker against the FP64 oracle; the plain FP64
form and the faster FP32-AO tensor-core form (mixed_tf32, which does not meet
that gate on ill-conditioned walkers) are timed on the same walkers and
reported beside it, each with its error against the FP64 form on every
walker.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 is launched with torchrun (one rank per GPU); walkers are independent,
so every rank evaluates its own batch with no collective on the data path
(weak scaling) and the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import qmc_inputs as qi  # noqa: E402

METRIC = "walker local-energy evals/s (CO, 14 e-) vs FP64 plain; p99 request latency"
UNIT = "walker-evals/s"
WORKLOAD = "CO 14e- 58 GTO 14 MO 100 det, 262144 walkers"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.26 TF)
# DRAM bytes (read + write) per walker of the k_det launch (the FP64 determinant stage of the
# mixed_tf32 and FP64 forms), from an ncu capture of that kernel on 131,072 CO walkers (418.6 MB per
# launch); set to None whenever the kernel changes.
DET_TRAFFIC_BYTES_PER_WALKER = (414.384128e6 + 4.216064e6) / 131072
# DRAM bytes (read + write) per walker of the k_ao_mo_oz launch, from an ncu capture of that kernel on
# 131,072 CO walkers (66.3 MB read, 409.0 MB written per launch); None whenever the kernel changes.
OZ_TRAFFIC_BYTES_PER_WALKER = (66.262016e6 + 408.966912e6) / 131072
# DRAM bytes (read + write) per walker of the k_det_x2 launch (FP32X2 determinant stage), from an ncu
# capture of that kernel on 131,072 CO walkers; None whenever the kernel changes (the last capture,
# 414.4 MB read and 1.2 MB written, was of the six-blocks-per-SM build).
DETX2_TRAFFIC_BYTES_PER_WALKER = None


def det_stage_flops(mol) -> float:
    """Algorithmic FP64 flops per walker of the determinant stage (FMA = 2):
    per spin with n electrons, nh holes, nv virtuals: reference inverse 2n^3,
    Tr(A0^-1 B0) 2n^2, per virtual column 2(2n^2 + nh n); per spin excitation
    rank 1: 2, rank 2: 12; per determinant 8 (ratio and kinetic numerator)."""
    tot = 0.0
    dets = np.asarray(mol.det_exc)
    for s, n in enumerate((mol.n_up, mol.n_down)):
        if n == 0:
            continue
        ex = dets[:, s, :]
        ranks = ex[:, 0]
        holes = [h for row in ex for h in row[1:1 + row[0]]]
        parts = [p for row in ex for p in row[3:3 + row[0]]]
        nh = n - min(holes) if holes else 0
        nv = max(parts) + 1 - n if parts else 0
        tot += 2 * n ** 3 + 2 * n * n + nv * 2 * (2 * n * n + nh * n)
        uniq = {tuple(row) for row in ex}
        tot += sum(2 if r[0] == 1 else 12 if r[0] == 2 else 0 for r in uniq)
    return tot + 8 * len(dets)


def ao_mo_stage_flops(mol) -> float:
    """Algorithmic flops per walker of the AO->MO contraction (two channels)."""
    return 2.0 * 2 * mol.n_elec * mol.n_ao * mol.n_mo


# FP32 operations of the pair-of-FP32 primitives (f32x2.cuh, as written):
# two_prod 2, fast_two_sum 3, two_sum 6; product of pairs 7, pair times a
# float 6, sum of pairs 11; multiply-accumulate into a pair 12; c - a b as a
# pair 15; reciprocal 10; renormalisation 3; exponential 69
X2_OPS = {"mac": 12, "mul": 7, "mulf": 6, "add": 11, "fms": 15, "recip": 10, "norm": 3, "exp": 69}


def x2_stage_ops(mol) -> float:
    """Algorithmic FP32 operations per walker of the FP32X2 AO stage
    (k_ao_mo_x2): per electron and Gaussian primitive the exponential of
    -alpha rho^2 and the radial sums (value, 2 alpha c e, (2 alpha)^2 c e);
    per electron and AO its value and kinetic channel from the shell's radial
    part (one product for the value, two products and one sum for the
    kinetic channel); per electron, AO and MO two multiply-accumulates
    (value and kinetic channel).  Displacements, shell set-up and stores are
    not counted."""
    n_prim = sum(int(mol.ao_prim_start[b + 1] - mol.ao_prim_start[b]) for b in range(mol.n_ao))
    # primitives are shared by the AOs of a shell: count each shell once
    shells = {}
    for b in range(mol.n_ao):
        key = (int(mol.ao_atom[b]), int(sum(mol.ao_pow[b][:3])), tuple(mol.prim_exp[mol.ao_prim_start[b]:mol.ao_prim_start[b + 1]]))
        shells[key] = int(mol.ao_prim_start[b + 1] - mol.ao_prim_start[b])
    n_shell_prim = sum(shells.values())
    o = X2_OPS
    per_prim = o["mul"] + o["exp"] + o["mul"] + o["add"] + (o["mul"] + o["mulf"] + o["add"]) * 2
    per_ao = o["mul"] + 2 * o["mul"] + o["add"]
    per_row = n_shell_prim * per_prim + mol.n_ao * per_ao + 2 * mol.n_ao * mol.n_mo * o["mac"]
    del n_prim
    return float(mol.n_elec * per_row)


def det_x2_stage_ops(mol) -> float:
    """Algorithmic FP32 operations per walker of k_det_x2, the FP32X2
    determinant stage (table method, kinetic channel), from its pair
    primitives (X2_OPS).  Per spin with n electrons, nh holes, nv virtuals:
      elimination: per pivot step one reciprocal, the pivot row's n - 1
                   products, per other row one product and n - 1 updates
                   c - a b, and the determinant's running product
      Tr(A0^-1 B0): n^2 multiply-accumulates, n renormalisations, n - 1 sums
      per virtual: t = A0^-1 Phi_p (n^2 multiply-accumulates), y = B_p - B0 t
                   (n^2 updates), Top on the holes (nh n multiply-accumulates),
                   n + nh renormalisations
      per distinct rank-2 spin excitation: the 2 x 2 minor (a product and an
                   update) and its kinetic numerator (4 multiply-accumulates
                   and a renormalisation)
      per determinant: two products and three multiply-accumulates (ratio and
                   kinetic numerator);
    plus, per FP64 input element (both channels of the occupied block and of
    the virtual columns), its split into a pair (7 FP32 operations; the
    integer bit operations are not counted), and the 16-lane reductions of the
    two sums (8 pair sums)."""
    o = X2_OPS
    tot = 8 * o["add"]
    dets = np.asarray(mol.det_exc)
    for s, n in enumerate((mol.n_up, mol.n_down)):
        if n == 0:
            continue
        ex = dets[:, s, :]
        holes = [h for row in ex for h in row[1:1 + row[0]]]
        parts = [p for row in ex for p in row[3:3 + row[0]]]
        nh = n - min(holes) if holes else 0
        nv = max(parts) + 1 - n if parts else 0
        tot += n * (o["recip"] + (n - 1) * o["mul"] + (n - 1) * (o["mul"] + (n - 1) * o["fms"]) + o["mul"])
        tot += n * n * o["mac"] + n * o["norm"] + (n - 1) * o["add"]
        tot += nv * (n * n * o["mac"] + n * n * o["fms"] + nh * n * o["mac"] + (n + nh) * o["norm"])
        uniq = {tuple(row) for row in ex}
        tot += sum(o["mul"] + o["fms"] + 4 * o["mac"] + o["norm"] for r in uniq if r[0] == 2)
        tot += 7 * 2 * n * (n + nv)
    return float(tot + len(dets) * (2 * o["mul"] + 3 * o["mac"]))


def fp64_ao_stage_ops(mol) -> dict:
    """Algorithmic FP64 work per walker of k_ao_mo_simt<double> (FP64 form):
    per electron and Gaussian primitive -alpha rho^2, c e and the value and
    kinetic radial sums (11 flops) and one exponential; per AO its value and
    kinetic channel (12 flops); the contraction (ao_mo_stage_flops)."""
    n_shell_prim = 0
    shells = set()
    for b in range(mol.n_ao):
        key = (int(mol.ao_atom[b]), int(sum(mol.ao_pow[b][:3])),
               tuple(mol.prim_exp[mol.ao_prim_start[b]:mol.ao_prim_start[b + 1]]))
        if key not in shells:
            shells.add(key)
            n_shell_prim += int(mol.ao_prim_start[b + 1] - mol.ao_prim_start[b])
    flops = mol.n_elec * (11 * n_shell_prim + 12 * mol.n_ao) + ao_mo_stage_flops(mol)
    return {"flops": float(flops), "exp": mol.n_elec * n_shell_prim}


def general_eloc_ops(mol) -> dict:
    """Algorithmic FP64 work per walker of the general kernel's local energy
    (k_eloc_general: one determinant, backflow), counted from its formulas:
    flops (an FMA counts 2) and the special functions separately.
      pairs:      geometry 8 flops, 1 sqrt, 1 division; Pade J, grad J, lap J
                  and 1/r_ij 31 flops, 2 divisions; backflow Jacobian blocks
                  G1, G2 and their row sums 110 flops (w != 0)
      e-n terms:  10 flops, 1 sqrt, 1 division per (electron, atom)
      backflow positions: 4 flops per (electron, coordinate, partner)
      orbitals per electron: per atom 9 flops, 1 sqrt, 1 division; per shell
                  the radial factor (STO 12 + kn flops + 1 exp; GTO 12 flops +
                  1 exp per primitive) and the closed-form s/p derivative set
                  (20); per AO 2 x 10 channels x n_occ flops (+ 15 for p)
      reference inverses: 2 n^3 + n^2 flops, n divisions, 1 log per spin
      contractions against A^-1: 6 n^3 (gradients) + 12 n per electron (Hessians)
      per coordinate and spin: per row 45 flops (Jacobian row, cq, Tr(A^-1 d^2 A)
                  terms, Y row), then Tr Y, Tr Y^2 and the second derivative 24"""
    N, nu, nd = int(mol.n_elec), int(mol.n_up), int(mol.n_down)
    n_occ = max(nu, nd)
    A = int(mol.n_atom)
    P = N * (N - 1) // 2
    bf = float(mol.backflow_w) != 0.0
    flops = P * (8 + 31 + (110 if bf else 0)) + N * A * 10 + (N * 3 * (N - 1) * 4)
    n_sqrt = P + N * A + N * A
    n_div = P + 2 * P + N * A + N * A
    n_exp = 0
    shells = {}
    for b in range(mol.n_ao):
        key = (int(mol.ao_atom[b]), int(sum(mol.ao_pow[b][:3])), int(mol.ao_kind[b]), int(mol.ao_pow[b][3]),
               tuple(mol.prim_exp[mol.ao_prim_start[b]:mol.ao_prim_start[b + 1]]))
        shells.setdefault(key, 0)
        shells[key] += 1
    per_elec = A * 9
    for (atom, l, kind, kn, ex), n_ao in shells.items():
        if kind == 0:
            per_elec += 12 + kn + 20
            n_exp += N
        else:
            per_elec += 12 * len(ex) + 20
            n_exp += N * len(ex)
        per_elec += n_ao * (2 * 10 * n_occ + (15 if l == 1 else 0))
    flops += N * per_elec
    for n in (nu, nd):
        if n:
            flops += 2 * n ** 3 + n * n + 6 * n ** 3
            n_div += n
    flops += N * 12 * n_occ
    for n in (nu, nd):
        if n:
            flops += 3 * N * (n * 45 + 24)
    return {"flops": float(flops), "exp": n_exp, "sqrt": n_sqrt, "div": n_div, "log": 2}


def oz_stage_alu_ops(mol) -> float:
    """Algorithmic FP32/ALU operations per walker of k_ao_mo_oz, the FP32X2
    AO stage with the contraction on the tensor cores.  Per electron: per
    Gaussian primitive of each shell -alpha rho^2 (7), the exponential (69)
    and three pair multiply-accumulates for the value and the two kinetic
    radial sums (3 x 12, coefficients 2 alpha c and 4 alpha^2 c folded on the
    host); per shell their three normalisations (3 x 3); per AO its value and
    kinetic channel (32, as x2_stage_ops); per AO value and channel the digit
    slicing (oz_digits: 26 FP32 operations, 2 for the row scale, 6 BF16
    packs); per MO and channel the recombination of the six classes
    (oz_combine: 44).  The contraction itself runs on the tensor pipe (BF16
    digit products, exact FP32 sums) and is not counted here; row-scale
    bounds, addressing and stores are not counted either."""
    o = X2_OPS
    shells = {}
    for b in range(mol.n_ao):
        key = (int(mol.ao_atom[b]), int(sum(mol.ao_pow[b][:3])), tuple(mol.prim_exp[mol.ao_prim_start[b]:mol.ao_prim_start[b + 1]]))
        shells[key] = int(mol.ao_prim_start[b + 1] - mol.ao_prim_start[b])
    per_prim = o["mul"] + o["exp"] + 3 * o["mac"]
    per_ao = o["mul"] + 2 * o["mul"] + o["add"]
    per_row = (sum(shells.values()) * per_prim + len(shells) * 9 + mol.n_ao * per_ao
               + 2 * mol.n_ao * (26 + 2 + 6) + 2 * mol.n_mo * 44)
    return float(mol.n_elec * per_row)


# GB300 issue rates from the unit counts and the maximum SM clock (152 SMs,
# 2.07 GHz): FP32 128 lanes per SM; FP64 2 FMA lanes per SM (4 flop/clk)
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12  # 40.3 T FP32 operations/s


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)  # let the sampler start before the timed region
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(n_walkers: int = 16384, n_walkers_1core: int = 1024):
    """The oracle (plain FP64 CPU, PyTorch vectorised over walkers) on a
    bounded sample of the same workload, on all host cores and on one."""
    import torch

    from oracle import qmc_oracle as O

    mol = qi.make_co()
    r = torch.tensor(qi.walkers(mol, n_walkers, seed=qi.SEED_WALKERS))
    wf = O.Wavefunction(mol)
    O.local_energy(wf, r[:64])  # warm the allocator
    t0 = time.perf_counter()
    O.local_energy(wf, r)
    dt = time.perf_counter() - t0
    cores = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        O.local_energy(wf, r[:n_walkers_1core])
        dt1 = time.perf_counter() - t0
    finally:
        torch.set_num_threads(cores)
    return {"value": n_walkers / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(), "value_1core": n_walkers_1core / dt1,
            "program": "the FP64 oracle (oracle/qmc_oracle.py: plain PyTorch CPU ops, explicit per-determinant "
                       "inverses), not a tuned C++ program",
            "sample": f"{n_walkers} of the 262144 CO walkers (same seed), one evaluation, {dt:.1f} s; "
                      f"1 core: {n_walkers_1core} walkers, {dt1:.1f} s"}


def run_reference(args, rank):
    """--impl reference: the oracle as it stands, on the host cores."""
    if rank != 0:
        return
    import torch

    from oracle import qmc_oracle as O

    mol = qi.make_co()
    per_step = 2048
    wf = O.Wavefunction(mol)
    total = args.warmup + args.steps
    r = torch.tensor(qi.walkers(mol, per_step * max(1, total), seed=qi.SEED_WALKERS))
    times = []
    for k in range(total):
        t0 = time.perf_counter()
        O.local_energy(wf, r[k * per_step:(k + 1) * per_step])
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = per_step / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "walkers_per_step": per_step, "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                         "sample": f"{per_step} CO walkers per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_serving(n_requests: int, with_fp64: bool, device: int, n_requests_fp64: int = 1000,
                n_capacity: int = 400):
    """Serving mix (H2, LiH, Li2, CO at 20 bond lengths each; 50 Metropolis
    steps + E_L mean/variance per request; walkers uniform on 4k..256k):
    a closed-loop run of n_capacity requests measures the capacity (requests/s
    with everything queued at once) and warms the server up, then Poisson
    arrivals at 80% of it give the latencies (n_requests in the FP32X2 form,
    n_requests_fp64 in the slower FP64 form)."""
    from paper_2506_09743_gb300 import serving

    out = {"n_steps": 50, "walker_choices": [4096, 16384, 65536, 262144], "molecules": ["h2", "lih", "li2", "co"],
           "note": "Li2 (backflow) requests run in the FP32X2 form in the FP32X2 mix",
           "policy": "large (>= 65,536 walkers) requests ordered, at most 2 in flight, low stream priority"}
    forms = ["fp32x2"] + (["fp64"] if with_fp64 else [])
    for form in forms:
        n = n_requests if form == "fp32x2" else min(n_requests, n_requests_fp64)
        wfs = serving.build_mix(form, device=device)
        srv = serving.Server(device=device, hbm_budget_bytes=48 << 30, max_in_flight=8)
        ids = {k: srv.add(wf) for k, wf in wfs.items()}
        cap_reqs = qi.serving_requests(min(n, n_capacity), rate_hz=0.0, seed=101)
        cap = serving.summarize(serving.run_stream(srv, ids, cap_reqs, n_steps=50, step=0.05), 50)
        rate = 0.8 * cap["requests_per_s"]
        reqs = qi.serving_requests(n, rate_hz=rate, seed=102)
        st = serving.summarize(serving.run_stream(srv, ids, reqs, n_steps=50, step=0.05, rate_hz=rate), 50)
        st["capacity_requests_per_s"] = cap["requests_per_s"]
        st["arrival_rate_hz"] = rate
        if form == "fp64" and n < n_requests:
            st["note"] = (f"{n} requests: at 80% of the FP64 capacity ({rate:.1f} req/s) {n_requests} requests "
                          f"would take {n_requests / rate:.0f} s; {n} keep the default run within minutes "
                          f"({n // 100} requests above the p99)")
        out[form] = st
        srv.close()
        for wf in wfs.values():
            wf.close()
    return out


def run_secondary(device, stream, barrier, flush, rates=None):
    """The other workloads: E_L throughput of H2 (1,024 walkers), LiH
    (65,536) and Li2 with backflow (131,072), and the Li2 energy gradient +
    forces (Eq. nabla_loss, Eq. force) on 131,072 walkers."""
    import torch

    from paper_2506_09743_gb300 import Wavefunction

    out = {}

    def rate(wf, x, W, steps=5):
        e = torch.empty(W, dtype=torch.float64, device="cuda")
        for _ in range(3):
            wf.local_energy(x, e_loc=e, want_log_psi=False)
        barrier()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            wf.local_energy(x, e_loc=e, want_log_psi=False)
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return W * steps / (tot / 1e3)

    for name in ("h2", "lih", "li2"):
        mol = qi.make_molecule(name)
        W = qi.WORKLOAD_WALKERS[name]
        x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=qi.SEED_WALKERS)), device="cuda")
        forms = ("fp64", "fp32x2") if mol.backflow_w != 0.0 else ("fp64", "fp32x2", "mixed_tf32")
        for form in forms:
            wf = Wavefunction(mol, precision=form, device=device)
            out[f"{name}_{form}_walker_evals_per_s"] = rate(wf, x, W)
            if name == "li2" and form == "fp64":
                # the general kernel's FP64 roofline: formula flops, and with
                # the special functions at their measured FMA equivalents
                ops = general_eloc_ops(mol)
                ms = 1e3 * W / out[f"{name}_{form}_walker_evals_per_s"]
                fl = ops["flops"] * W / (ms / 1e3) / 1e12
                eq = None
                if rates:
                    f = rates["fp64_fma_per_s"]
                    sp = (ops["exp"] * f / rates["fp64_exp_per_s"] + ops["sqrt"] * f / rates["fp64_sqrt_per_s"]
                          + ops["div"] * f / rates["fp64_recip_per_s"])
                    eq = (ops["flops"] + 2.0 * sp) * W / (ms / 1e3) / 1e12
                out["li2_eloc_roofline"] = {
                    "kernel": "k_eloc_general<6, 3>", "bound": "alu", "kernel_ms": ms, "unit": "TFLOP/s (FP64)",
                    "flops_per_walker": ops["flops"], "exp_per_walker": ops["exp"], "sqrt_per_walker": ops["sqrt"],
                    "div_per_walker": ops["div"], "achieved": fl, "peak": FP64_PEAK_TFLOPS,
                    "frac": fl / FP64_PEAK_TFLOPS, "achieved_with_special": eq,
                    "frac_with_special": None if eq is None else eq / FP64_PEAK_TFLOPS,
                    "ops_model": "bench.general_eloc_ops; exp, sqrt and division at the measured FMA equivalents"}
            if name == "li2" and form == "fp64":
                wf.energy_grad(x)
                barrier()
                t0 = time.perf_counter()
                wf.energy_grad(x)
                out["li2_energy_grad_ms"] = 1e3 * (time.perf_counter() - t0)
                out["li2_energy_grad_note"] = ("131,072 walkers: E_L, mean/variance, gradient of 83 parameters "
                                               "and forces on both nuclei, host-timed (synchronous call)")
            wf.close()
    # CO energy gradient (Eq. nabla_loss) with the 100-determinant expansion:
    # 1,008 parameters (exponents, MO coefficients, CI weights, b, w), FP64
    mol = qi.make_co()
    W = 131072
    x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=qi.SEED_WALKERS)), device="cuda")
    wf = Wavefunction(mol, precision="fp64", device=device)
    wf.energy_grad(x, want_forces=False)
    barrier()
    t0 = time.perf_counter()
    wf.energy_grad(x, want_forces=False)
    out["co_energy_grad_ms"] = 1e3 * (time.perf_counter() - t0)
    out["co_energy_grad_note"] = ("131,072 walkers, 100 determinants: E_L (FP64 form), mean/variance and the gradient "
                                  "of 1,008 parameters through tables of the reference inverse; host-timed")
    wf.close()
    del x
    # CO with the many-body Jastrow of App. D (K_en + 5 K_een terms), mixed form
    mol = qi.with_manybody_jastrow(qi.make_co())
    W = qi.WORKLOAD_WALKERS["co"]
    x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=qi.SEED_WALKERS)), device="cuda")
    for form in ("fp32x2", "mixed_tf32"):
        wf = Wavefunction(mol, precision=form, device=device)
        out[f"co_manybody_jastrow_{form}_walker_evals_per_s"] = rate(wf, x, W, steps=3)
        wf.close()
    del x
    # several determinants with backflow: Li2, SD(6e, 6o) = 118 determinants
    mol = qi.make_li2(n_mo=6, n_det=118)
    W = qi.WORKLOAD_WALKERS["li2"]
    x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=qi.SEED_WALKERS)), device="cuda")
    wf = Wavefunction(mol, precision="fp64", device=device)
    out["li2_sd118_backflow_fp64_walker_evals_per_s"] = rate(wf, x, W, steps=3)
    wf.close()
    # one optimisation step of App. B (10^4 walkers: Eq. nabla_loss gradient, ADAM
    # update, 500 Metropolis resampling steps), host-timed through qmc_optimize
    for name in ("lih", "li2"):
        mol = qi.make_molecule(name)
        x = torch.tensor(qi.to_soa(qi.walkers(mol, 10000, seed=qi.SEED_WALKERS)), device="cuda")
        wf = Wavefunction(mol, precision="fp64", device=device)
        wf.optimize(x, n_iter=1, n_equil=50, n_resample=20, step=0.05, seed=0x5EED)
        barrier()
        t0 = time.perf_counter()
        hist = wf.optimize(x, n_iter=2, n_equil=0, n_resample=500, step=0.05, seed=0x5EED)
        out[f"{name}_opt_step_ms"] = 1e3 * (time.perf_counter() - t0) / 2
        out[f"{name}_opt_accept"] = float(hist[:, 2].mean())
        wf.close()
    out["opt_step_note"] = ("one App. B optimisation step on 10^4 walkers: gradient (Eq. nabla_loss), ADAM "
                            "update, parameter upload, 500 Metropolis steps of 0.05 bohr; FP64 form")
    return out


DET_SWEEP = (1, 4, 100, 876, 1716)


def run_det_sweep(device, stream, barrier, flush, W=65536, steps=3):
    """Explicit versus table determinants across expansion sizes (the shape of
    the paper's comparison, Sec. 2.2 / App. A): CO-shaped wavefunction with
    n_det determinants drawn from the (10e, 12o) space, mixed form, E_L
    walker-evals/s for both methods on the same walkers."""
    import torch

    from paper_2506_09743_gb300 import Wavefunction

    rows = []
    for n_det in DET_SWEEP:
        mol = qi.make_co(n_det=n_det)
        x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=qi.SEED_WALKERS)), device="cuda")
        e = torch.empty(W, dtype=torch.float64, device="cuda")
        row = {"n_det": n_det}
        for method in ("table", "explicit"):
            wf = Wavefunction(mol, precision="mixed_tf32", device=device)
            wf.set_det_method(method)
            for _ in range(3):
                wf.local_energy(x, e_loc=e, want_log_psi=False)
            barrier()
            tot = 0.0
            for _ in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                wf.local_energy(x, e_loc=e, want_log_psi=False)
                b.record(stream)
                b.synchronize()
                tot += a.elapsed_time(b)
            row[f"{method}_walker_evals_per_s"] = W * steps / (tot / 1e3)
            wf.close()
        row["speedup"] = row["table_walker_evals_per_s"] / row["explicit_walker_evals_per_s"]
        rows.append(row)
    return {"walkers": W, "precision": "mixed_tf32", "rows": rows}


def run_sharded_energy_grad(device, rank, world, dist, barrier, W=131072):
    """One sharded energy-gradient step (Eq. nabla_loss, Eq. force) of Li2
    with backflow: every rank forms the per-batch sums of its own 131,072
    walkers (qmc_energy_grad_sums, device memory), one all-reduce adds them
    across ranks in place (NCCL), and the estimator is assembled on the host
    (qmc_assemble_energy_grad).  Host-timed, max over ranks."""
    import torch

    from paper_2506_09743_gb300 import Wavefunction, _lib

    mol = qi.make_li2()
    x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=rank_walker_seed(rank))), device="cuda")
    wf = Wavefunction(mol, precision="fp64", device=device)
    n_param, _ = wf.param_layout()

    def step():
        sums = wf.energy_grad_sums(x)
        if dist is not None:
            dist.all_reduce(sums, op=dist.ReduceOp.SUM)
        return _lib.assemble_energy_grad(sums.cpu().numpy(), n_param, mol.n_atom)

    step()
    barrier()
    t0 = time.perf_counter()
    ev, var, g, f = step()
    ms = reduce_max(1e3 * (time.perf_counter() - t0), dist)
    wf.close()
    return {"walkers_per_gpu": W, "n_gpus": world, "ms": ms, "e_mean": ev,
            "collective": f"one all-reduce of {3 + 2 * n_param + 9 * mol.n_atom} doubles" if world > 1 else "none",
            "note": "Li2 backflow, FP64: per-batch sums on each GPU, all-reduced, assembled on the host"}


def reduce_max(v: float, dist=None) -> float:
    """Maximum of a per-rank value over the process group (identity alone)."""
    if dist is None or not dist.is_initialized():
        return v
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, steps: int, max_total_ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank's time."""
    return world * units_per_rank * steps / (max_total_ms / 1e3)


def rank_walker_seed(rank: int) -> int:
    """Each rank draws its own walkers (weak scaling: a fixed batch per GPU)."""
    return qi.SEED_WALKERS + rank


PROFILE_CASES = ("co_fp32x2", "co_mixed_tf32", "co_fp64", "co_energy_grad", "li2_eloc", "li2_eloc_fp32x2",
                 "li2_energy_grad", "li2_sample")


def run_only(case: str, W: int, steps: int, warmup: int, device: int = 0) -> dict:
    """One workload alone (the small cases the ncu captures run): `warmup`
    untimed calls, then `steps` calls timed with CUDA events.  CO cases time
    qmc_local_energy in the named form (co_energy_grad: the FP64 gradient of
    the 100-determinant expansion); li2_eloc the backflow E_L (FP64),
    li2_energy_grad qmc_energy_grad, li2_sample ten Metropolis steps."""
    import torch

    from paper_2506_09743_gb300 import Wavefunction

    mol = qi.make_co() if case.startswith("co_") else qi.make_li2()
    form = (case[3:] if case.startswith("co_") and case != "co_energy_grad"
            else "fp32x2" if case.endswith("_fp32x2") else "fp64")
    x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=qi.SEED_WALKERS)), device="cuda")
    wf = Wavefunction(mol, precision=form, device=device)
    e = torch.empty(W, dtype=torch.float64, device="cuda")

    def call():
        if case == "li2_energy_grad":
            wf.energy_grad(x)
        elif case == "co_energy_grad":
            wf.energy_grad(x, want_forces=False)
        elif case == "li2_sample":
            wf.sample(x, n_steps=10, step=0.05, seed=0x5EED)
        else:
            wf.local_energy(x, e_loc=e, want_log_psi=False)

    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        call()
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    wf.close()
    return {"case": case, "walkers": W, "steps": steps, "ms_per_call": ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--walkers", type=int, default=qi.WORKLOAD_WALKERS["co"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests of the Poisson serving run, FP32X2 form (the FP64 form serves at most 1000; 0 = skip)")
    ap.add_argument("--no-serving-fp64", action="store_true", help="serve the mix in the mixed form only")
    ap.add_argument("--no-det-sweep", action="store_true", help="skip the explicit-versus-table sweep")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other molecules' measurements")
    ap.add_argument("--manybody-jastrow", action="store_true",
                    help="time CO with the many-body Jastrow of App. D (K_en + 5 K_een terms) instead")
    ap.add_argument("--only", choices=PROFILE_CASES,
                    help="run one workload alone and print its time per call (the cases the ncu captures use)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2506_09743_gb300 import Wavefunction

    torch.cuda.set_device(local)
    if args.only:
        print(json.dumps(run_only(args.only, args.walkers, args.steps, args.warmup, local)), flush=True)
        return
    from paper_2506_09743_gb300 import _lib as qlib

    rates = qlib.measure_rates()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, dist)

    mol = qi.with_manybody_jastrow(qi.make_co()) if args.manybody_jastrow else qi.make_co()
    W = args.walkers
    r = qi.walkers(mol, W, seed=rank_walker_seed(rank))
    soa = np.ascontiguousarray(qi.to_soa(r))
    x = torch.tensor(soa, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()

    last_e = torch.empty(W, dtype=torch.float64, device="cuda")

    def timed_device(wf, steps, warmup):
        e = last_e
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        wf.set_timing(True)
        for _ in range(warmup):
            wf.local_energy(x, e_loc=e, log_psi=lp)
        barrier()
        stage = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()  # evict L2 between steps (outside the timed events)
            ev[k][0].record(stream)
            wf.local_energy(x, e_loc=e, log_psi=lp)
            ev[k][1].record(stream)
            stage.append(wf.last_stage_ms())  # waits for this step; outside the events
        barrier()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        wf.set_timing(False)
        finite = float(torch.isfinite(e).double().mean().item())
        return float(np.sum(step_ms)), np.mean(np.asarray(stage), axis=0), finite

    wf_x2 = Wavefunction(mol, precision="fp32x2", device=local)
    wf_mixed = Wavefunction(mol, precision="mixed_tf32", device=local)
    wf_fp64 = Wavefunction(mol, precision="fp64", device=local)

    clk = ClockSampler(local).__enter__()
    tot_x2, stage_x2, fin_x2 = timed_device(wf_x2, args.steps, args.warmup)
    e_x2 = last_e.clone()
    k_mixed = max(3, args.steps // 2)
    tot_mixed, stage_mixed, fin_mixed = timed_device(wf_mixed, k_mixed, 3)
    e_mixed = last_e.clone()
    k64 = max(3, args.steps // 4)
    tot_fp64, stage_fp64, fin_fp64 = timed_device(wf_fp64, k64, 3)
    e_fp64 = last_e.clone()
    tot_x2 = max_over_ranks(tot_x2)
    tot_mixed = max_over_ranks(tot_mixed)
    tot_fp64 = max_over_ranks(tot_fp64)
    ms_step = tot_x2 / args.steps
    value = whole_job_rate(world, W, args.steps, tot_x2)
    value_mixed = whole_job_rate(world, W, k_mixed, tot_mixed)
    value_fp64 = whole_job_rate(world, W, k64, tot_fp64)

    # end to end through the host-buffer C call (pinned host memory)
    pin_in = torch.from_numpy(soa).pin_memory()
    pin_e = torch.empty(W, dtype=torch.float64).pin_memory()
    pin_lp = torch.empty(W, dtype=torch.float64).pin_memory()
    in_np, e_np, lp_np = pin_in.numpy(), pin_e.numpy(), pin_lp.numpy()
    for _ in range(args.warmup):
        wf_x2.local_energy_host(in_np, e_np, lp_np, stream=stream)
    barrier()
    e2e_steps = max(3, args.steps // 2)
    t_e2e = []
    for _ in range(e2e_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wf_x2.local_energy_host(in_np, e_np, lp_np, stream=stream)
        b.record(stream)
        b.synchronize()
        t_e2e.append(a.elapsed_time(b))
    barrier()
    clk.__exit__(None, None, None)
    clocks = clk.summary()
    e2e_ms = max_over_ranks(float(np.sum(t_e2e)))
    e2e_value = whole_job_rate(world, W, e2e_steps, e2e_ms)

    # Metropolis walker steps (value path: Jastrow value, orbital values, determinants, accept)
    def mh_rate(wf, n_mh=5):
        xs = x.clone()
        wf.sample(xs, n_steps=1, step=0.05, seed=0x5EED)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wf.sample(xs, n_steps=n_mh, step=0.05, seed=0x5EED, step_offset=1)
        b.record(stream)
        b.synchronize()
        return world * W * n_mh / (max_over_ranks(a.elapsed_time(b)) / 1e3)

    mh_x2 = mh_rate(wf_x2)
    mh_mixed = mh_rate(wf_mixed)

    sharded = run_sharded_energy_grad(local, rank, world, dist, barrier)
    secondary = (run_secondary(local, stream, barrier, flush, rates)
                 if world == 1 and not args.no_secondary else None)
    det_sweep = run_det_sweep(local, stream, barrier, flush) if world == 1 and not args.no_det_sweep else None

    serving_out = None
    if args.serving_requests > 0 and world == 1:
        serving_out = run_serving(args.serving_requests, not args.no_serving_fp64, local)

    # error of each form against the FP64 form on every walker of the batch
    # (the FP64 form matches the CPU oracle to 1e-10 relative: tests/)
    def accuracy(e_form):
        err = (e_form - e_fp64).abs()
        ok = torch.isfinite(err)
        err = err[ok].cpu().numpy()
        return {"within_2e-4_Ha": float((err <= 2e-4).mean()), "median_Ha": float(np.median(err)),
                "p99_Ha": float(np.quantile(err, 0.99)), "p999_Ha": float(np.quantile(err, 0.999)),
                "max_Ha": float(err.max()), "nonfinite": int((~ok).sum().item()), "walkers": W,
                "note": "against the FP64 form on the same walkers; the walkers beyond 2e-4 Ha are at nodes "
                        "(|E| of 1e4..1e7 Ha), outside the parity tests' conditioning cut"}

    # measured FP64 FMA and FP32 instruction rates of this GPU (probe kernels
    # of the library): beside the nominal peaks derived from the unit counts
    fp64_meas = 2.0 * rates["fp64_fma_per_s"] / 1e12 if rates else None
    fp32_meas = rates["fp32_fma_per_s"] / 1e12 if rates else None
    # rooflines: both FP32X2 stages are bound by FP32/ALU issue (the AO
    # stage's contraction runs on the tensor pipe, its determinant stage in
    # pairs of FP32); the FP64 determinant stage of the mixed_tf32 and FP64
    # forms (k_det) by the FP64 pipe
    oz_ops = oz_stage_alu_ops(mol) * W
    x2_ms = float(stage_x2[1])
    oz_rate = oz_ops / (x2_ms / 1e3) / 1e12
    x2_equiv = x2_stage_ops(mol) * W / (x2_ms / 1e3) / 1e12
    dx2_ops = det_x2_stage_ops(mol) * W
    dx2_ms = float(stage_x2[2])
    dx2_rate = dx2_ops / (dx2_ms / 1e3) / 1e12
    flops_det = det_stage_flops(mol) * W
    det_ms = float(stage_mixed[2])
    det_rate = flops_det / (det_ms / 1e3) / 1e12
    roofline = {"kernel": "k_ao_mo_oz (AOs in pairs of FP32, exact digit-sliced contraction on tcgen05; FP32X2 form)",
                "bound": "alu", "achieved": oz_rate, "peak": FP32_PEAK_TOPS, "unit": "T FP32 ops/s",
                "frac": oz_rate / FP32_PEAK_TOPS,
                "traffic": None if OZ_TRAFFIC_BYTES_PER_WALKER is None else OZ_TRAFFIC_BYTES_PER_WALKER * W,
                "traffic_note": "ncu dram read + write of one launch on 131,072 walkers, scaled by walkers",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (no FP32 figure in the measured peaks)",
                "peak_measured": fp32_meas, "frac_of_measured": oz_rate / fp32_meas if fp32_meas else None,
                "ops_per_launch": oz_ops,
                "ops_model": "bench.oz_stage_alu_ops: AO evaluation in pair arithmetic + digit slicing + class "
                             "recombination; the contraction runs on the tensor pipe",
                "simt_equivalent_tops": x2_equiv,
                "simt_equivalent_note": "the whole stage (bench.x2_stage_ops, contraction as pair multiply-"
                                        "accumulates) per second: what the SIMT pair kernel would have to issue",
                "kernel_ms": x2_ms}
    # the FP64 form's AO stage: contraction flops + AO flops + exponentials
    # (in FMA equivalents from the measured exp rate)
    fp64_ao = fp64_ao_stage_ops(mol)
    simt_ms = float(stage_fp64[1])
    exp_fma = rates["fp64_fma_per_s"] / rates["fp64_exp_per_s"] if rates else None
    simt_flops = fp64_ao["flops"] * W
    simt_equiv = simt_flops + (2.0 * exp_fma * fp64_ao["exp"] * W if exp_fma else 0.0)
    rooflines = {
        "k_det_x2": {"bound": "alu", "achieved": dx2_rate, "peak": FP32_PEAK_TOPS, "unit": "T FP32 ops/s",
                     "frac": dx2_rate / FP32_PEAK_TOPS, "kernel_ms": dx2_ms, "ops_per_launch": dx2_ops,
                     "traffic": (None if DETX2_TRAFFIC_BYTES_PER_WALKER is None
                                 else DETX2_TRAFFIC_BYTES_PER_WALKER * W),
                     "peak_measured": fp32_meas, "frac_of_measured": dx2_rate / fp32_meas if fp32_meas else None,
                     "ops_model": "bench.det_x2_stage_ops: pair-of-FP32 elimination, tables, minors and "
                                  "expansion (FP32X2 form's determinant stage)"},
        "k_det": {"bound": "alu", "achieved": det_rate, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s (FP64)",
                  "form": "mixed_tf32 (the same kernel runs the FP64 form's determinant stage)",
                  "frac": det_rate / FP64_PEAK_TFLOPS, "kernel_ms": det_ms, "flops_per_launch": flops_det,
                  "traffic": None if DET_TRAFFIC_BYTES_PER_WALKER is None else DET_TRAFFIC_BYTES_PER_WALKER * W,
                  "peak_source": "FP64 pipe: 152 SMs x 4 flop/clk x 2.07 GHz (nominal)",
                  "peak_measured": fp64_meas, "frac_of_measured": det_rate / fp64_meas if fp64_meas else None},
        "k_ao_mo_simt_fp64": {"bound": "alu", "kernel_ms": simt_ms, "unit": "TFLOP/s (FP64)",
                              "peak": FP64_PEAK_TFLOPS, "flops_per_launch": simt_flops,
                              "exp_per_launch": fp64_ao["exp"] * W,
                              "achieved": simt_flops / (simt_ms / 1e3) / 1e12,
                              "achieved_with_exp": simt_equiv / (simt_ms / 1e3) / 1e12,
                              "frac_with_exp": simt_equiv / (simt_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                              "exp_cost_fma": exp_fma,
                              "ops_model": "bench.fp64_ao_stage_ops: AO values and kinetic channels, contraction; "
                                           "each exponential as the measured FMA equivalents"},
        "k_ao_mo_tc": {"kernel_ms": float(stage_mixed[1]), "note": "FP32 AO stage + tcgen05 TF32x3 contraction"},
    }
    # whole step: the FP32X2 step cannot beat its AO stage plus its
    # determinant stage at the FP32 issue rate (the two run in turn)
    bound_ms = (oz_ops + dx2_ops) / (FP32_PEAK_TOPS * 1e12) * 1e3
    whole_step = {"ms_per_step": ms_step, "bound_ms": bound_ms, "frac": bound_ms / ms_step,
                  "note": "AO stage and determinant stage at the FP32 issue rate, in sequence"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2 (AO, MO, det; f64 in/out)", "data": "synthetic",
        "config": {"workload": (WORKLOAD.replace("262144 walkers", f"{W} walkers")
                                + (" + many-body Jastrow (K_en, 5 K_een terms)" if args.manybody_jastrow else "")),
                   "walkers_per_gpu": W, "precision": "fp32x2",
                   "l2": "flushed (256 MB write) between timed steps, outside the timed events",
                   "parallelism": f"walker shards x{world}, no data-path collective"},
        "stage_ms": {"jastrow_coulomb": float(stage_x2[0]), "ao_mo_oz": float(stage_x2[1]),
                     "det_eloc": float(stage_x2[2])},
        "finite_frac": fin_x2,
        "accuracy": accuracy(e_x2),
        "fp64_plain": {"value": value_fp64, "ms_per_step": tot_fp64 / k64,
                       "stage_ms": [float(v) for v in stage_fp64], "finite_frac": fin_fp64},
        "mixed_tf32": {"value": value_mixed, "ms_per_step": tot_mixed / k_mixed,
                       "stage_ms": [float(v) for v in stage_mixed], "finite_frac": fin_mixed,
                       "accuracy": accuracy(e_mixed),
                       "note": "FP32 AOs, tcgen05 TF32x3 contraction: faster, but not within 2e-4 Ha on "
                               "ill-conditioned walkers"},
        "fp32x2_vs_fp64": value / value_fp64,
        "roofline": roofline,
        "rooflines": rooflines,
        "measured_rates": rates,
        "whole_step": whole_step,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(soa.nbytes),
                "d2h_bytes_per_step": int(2 * 8 * W), "api": "qmc_local_energy_host (pinned host buffers), FP32X2 form"},
        # per E_L: Jastrow (+ e-e-n kernel with the many-body Jastrow), AO->MO, determinants
        "gpu_launches": (4 if args.manybody_jastrow else 3) * args.steps,
        "clocks": clocks,
        "p99_request_latency_ms": None if serving_out is None else serving_out["fp32x2"]["p99_ms"],
        "metropolis_walker_steps_per_s": mh_x2,
        "metropolis_walker_steps_per_s_mixed_tf32": mh_mixed,
        "serving": serving_out,
        "sharded_energy_grad": sharded,
        "secondary": secondary,
        "det_sweep": det_sweep,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
