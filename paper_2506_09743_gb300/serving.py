"""Python driver of the continuous-batching request server (qmc_server_* in
include/qmc.h): argument marshalling and a Poisson-arrival load generator
that reports request latencies (p50/p99) and aggregate throughput.  All
scheduling, admission and device work run in the native library."""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import Wavefunction, _lib, library


class Server:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 32 << 30, max_in_flight: int = 8,
                 big_walkers: int = 65536, max_big_in_flight: int = 2):
        """big_walkers / max_big_in_flight: the admission policy of
        qmc_server_set_policy (big_walkers = 0: plain arrival order)."""
        lib = library()
        h = ctypes.c_void_p()
        _lib.check_server(lib.qmc_server_create(device, int(hbm_budget_bytes), int(max_in_flight), ctypes.byref(h)))
        self._h, self._lib = h, lib
        _lib.check_server(lib.qmc_server_set_policy(h, int(big_walkers), int(max_big_in_flight)))
        self._wfs = []  # keep wavefunctions alive
        self._hold = {}  # host walker buffers of requests in flight
        self.budget = int(hbm_budget_bytes)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.qmc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, wf: Wavefunction) -> int:
        k = ctypes.c_int32()
        _lib.check_server(self._lib.qmc_server_add_wf(self._h, wf._h, ctypes.byref(k)))
        self._wfs.append(wf)
        return int(k.value)

    def submit(self, wf_id: int, n_walkers: int, n_steps: int, step: float, seed: int, walkers=None) -> int:
        ptr = None
        if walkers is not None:
            walkers = np.ascontiguousarray(walkers, dtype=np.float64)
            ptr = walkers.ctypes.data_as(ctypes.c_void_p)
        req = _lib.Request(int(wf_id), int(n_walkers), int(n_steps), float(step), int(seed), ptr)
        t = ctypes.c_int64()
        _lib.check_server(self._lib.qmc_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        if walkers is not None:
            self._hold[int(t.value)] = walkers
        return int(t.value)

    def progress(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        _lib.check_server(self._lib.qmc_server_progress(self._h, ctypes.byref(a), ctypes.byref(q)))
        return int(a.value), int(q.value)

    def results(self, capacity: int = 256):
        buf = (_lib.Result * capacity)()
        n = ctypes.c_int32()
        _lib.check_server(self._lib.qmc_server_results(self._h, buf, capacity, ctypes.byref(n)))
        out = []
        for k in range(n.value):
            r = buf[k]
            self._hold.pop(int(r.ticket), None)
            out.append({f: getattr(r, f) for f, _ in _lib.Result._fields_})
        return out

    def cancel(self, ticket: int):
        """Cancel a queued or running request (its result reports QMC_ERR_CANCELLED)."""
        _lib.check_server(self._lib.qmc_server_cancel(self._h, int(ticket)))

    def set_policy(self, big_walkers: int, max_big_in_flight: int):
        _lib.check_server(self._lib.qmc_server_set_policy(self._h, int(big_walkers), int(max_big_in_flight)))

    def free_bytes(self) -> int:
        return int(self._lib.qmc_server_free_bytes(self._h))

    def clock(self) -> float:
        return float(self._lib.qmc_server_clock())

    def drain(self, timeout_s: float = 600.0):
        out = []
        t0 = time.monotonic()
        while True:
            a, q = self.progress()
            out += self.results()
            if a == 0 and q == 0:
                return out
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(50e-6)


def build_mix(precision: str, molecules=("h2", "lih", "li2", "co"), n_bonds: int = 20, device: int = 0):
    """Wavefunctions of the serving mix: each molecule at n_bonds bond lengths
    from 0.6x to 2.5x equilibrium.  Backflow (Li2) has the FP64 and FP32X2
    forms only: it runs in FP32X2 in the FP32X2 mix and in FP64 otherwise."""
    import qmc_inputs as qi

    wfs = {}
    for name in molecules:
        base = qi.make_molecule(name)
        for k, s in enumerate(np.linspace(0.6, 2.5, n_bonds)):
            prec = precision if base.backflow_w == 0.0 or precision in ("fp64", "fp32x2") else "fp64"
            wfs[(name, k)] = Wavefunction(base.with_bond_scale(float(s)), precision=prec, device=device)
    return wfs


def run_stream(server: Server, ids: dict, requests, n_steps: int = 50, step: float = 0.2, rate_hz: float = 0.0,
               timeout_s: float = 900.0, n_bonds: int = 20):
    """Submit `requests` (from qmc_inputs.serving_requests) at their Poisson
    arrival times (rate_hz = 0: all at once, a closed-loop capacity run),
    keep the server progressing, and return per-request records."""
    scales = np.linspace(0.6, 2.5, n_bonds)
    t0 = time.monotonic()
    pending = list(requests)
    done, sub = [], {}
    while pending or len(done) < len(requests):
        now = time.monotonic() - t0
        while pending and (rate_hz == 0.0 or pending[0]["arrival_s"] <= now):
            r = pending.pop(0)
            k = int(np.argmin(np.abs(scales - r["bond_scale"])))
            t = server.submit(ids[(r["molecule"], k)], r["n_walkers"], n_steps, step, r["seed"])
            sub[t] = r
        server.progress()
        for res in server.results():
            res["request"] = sub.pop(res["ticket"])
            done.append(res)
        if time.monotonic() - t0 > timeout_s:
            raise TimeoutError("serving run did not finish")
        if pending and rate_hz > 0.0:
            time.sleep(min(50e-6, max(0.0, pending[0]["arrival_s"] - (time.monotonic() - t0))))
    return done


def summarize(done, n_steps: int):
    lat = np.array([d["t_done"] - d["t_submit"] for d in done])
    t_first = min(d["t_submit"] for d in done)
    t_last = max(d["t_done"] for d in done)
    evals = sum(d["n_walkers"] * (n_steps + 1) for d in done)
    return {
        "requests": len(done),
        "failed": int(sum(1 for d in done if d["status"] != 0)),
        "nonfinite_walkers": int(sum(d.get("n_nonfinite", 0) for d in done)),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "makespan_s": float(t_last - t_first),
        "walker_evals_per_s": float(evals / (t_last - t_first)),
        "requests_per_s": float(len(done) / (t_last - t_first)),
    }
