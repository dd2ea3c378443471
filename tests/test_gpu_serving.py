"""Continuous-batching server (qmc_server_*): results are the same alone and
in a mix of concurrent requests, admission respects the device-memory
budget, and a request equals the composition of the public calls."""
import numpy as np
import pytest
import torch

import qmc_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2506_09743_gb300 as p

    return p


@pytest.fixture(scope="module")
def mix(pkg):
    from paper_2506_09743_gb300 import serving

    wfs = serving.build_mix("mixed_tf32", n_bonds=4)
    return wfs


def _server(mix, budget, slots, **policy):
    from paper_2506_09743_gb300 import serving

    srv = serving.Server(hbm_budget_bytes=budget, max_in_flight=slots, **policy)
    ids = {k: srv.add(wf) for k, wf in mix.items()}
    return srv, ids


def test_same_result_alone_and_in_the_mix(mix):
    target = (("co", 1), 20000, 30, 0.05, 1234)
    srv, ids = _server(mix, 8 << 30, 8)
    srv.submit(ids[target[0]], *target[1:])
    alone = srv.drain()
    assert len(alone) == 1 and alone[0]["status"] == 0
    rng = np.random.default_rng(5)
    keys = list(mix)
    tickets = []
    for k in range(12):
        key = keys[int(rng.integers(len(keys)))]
        tickets.append(srv.submit(ids[key], int(rng.choice([4096, 16384, 40000])), 30, 0.05, int(rng.integers(1 << 30))))
        if k == 5:
            t_target = srv.submit(ids[target[0]], *target[1:])
    res = {r["ticket"]: r for r in srv.drain()}
    assert all(r["status"] == 0 for r in res.values())
    inmix = res[t_target]
    for f in ("e_mean", "e_var", "accept_rate"):
        assert inmix[f] == alone[0][f], f
    assert srv.free_bytes() == srv.budget
    srv.close()


def test_admission_respects_the_memory_budget(mix, pkg):
    wf = mix[("lih", 0)]
    per_req = wf.workspace_size(65536) + 65536 * (3 * wf.n_elec + 2) * 8 + 4096
    budget = int(2.5 * per_req)  # at most two such requests fit at once
    srv, ids = _server({("lih", 0): wf}, budget, 8)
    for k in range(6):
        srv.submit(ids[("lih", 0)], 65536, 5, 0.2, 100 + k)
    max_in_flight = 0
    done = []
    while len(done) < 6:
        a, q = srv.progress()
        max_in_flight = max(max_in_flight, a)
        done += srv.results()
    assert max_in_flight <= 2
    assert all(r["status"] == 0 for r in done)
    assert srv.free_bytes() == budget
    srv.close()


def test_request_larger_than_budget_is_rejected(mix):
    from paper_2506_09743_gb300 import QmcError

    srv, ids = _server(mix, 64 << 20, 2)
    with pytest.raises(QmcError) as ei:
        srv.submit(ids[("co", 0)], 262144, 10, 0.05, 1)
    assert "budget" in str(ei.value)
    srv.close()


def test_request_equals_composed_public_calls(mix, pkg):
    mol = qi.make_h2().with_bond_scale(float(np.linspace(0.6, 2.5, 4)[2]))
    wf = pkg.Wavefunction(mol, precision="mixed_tf32")
    r = qi.to_soa(qi.walkers(mol, 5000, seed=9))
    srv, ids = _server({("h2", 2): wf}, 1 << 30, 2)
    srv.submit(ids[("h2", 2)], 5000, 25, 0.2, 77, walkers=r)
    res = srv.drain()[0]
    x = torch.tensor(r, device="cuda")
    acc = torch.zeros(5000, dtype=torch.int64, device="cuda")
    wf.sample(x, n_steps=25, step=0.2, seed=77, n_accept=acc)
    e, _ = wf.local_energy(x)
    torch.cuda.synchronize()
    e = e.cpu().numpy()
    assert abs(res["e_mean"] - e.mean()) <= 1e-12 * max(1.0, abs(e.mean()))
    assert abs(res["e_var"] - e.var()) <= 1e-10 * max(1.0, e.var())
    assert res["accept_rate"] == acc.sum().item() / (5000 * 25)
    srv.close()


def test_poisson_stream_reports_latency(mix):
    from paper_2506_09743_gb300 import serving

    srv, ids = _server(mix, 16 << 30, 8)
    reqs = qi.serving_requests(24, rate_hz=40.0, seed=3, walker_choices=(4096, 16384), n_bonds=4)
    done = serving.run_stream(srv, ids, reqs, n_steps=10, step=0.05, rate_hz=40.0, n_bonds=4)
    st = serving.summarize(done, 10)
    assert st["requests"] == 24 and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    srv.close()


def test_large_requests_keep_order_and_limit(mix):
    """Policy: at most max_big large requests in flight, in arrival order among
    themselves; a small request submitted behind a waiting large one is
    admitted before it; every result matches the same request run alone."""
    srv, ids = _server(mix, 16 << 30, 8, big_walkers=40000, max_big_in_flight=1)
    key = ids[("lih", 1)]
    big = [srv.submit(key, 65536, 20, 0.1, 500 + k) for k in range(3)]
    small = srv.submit(ids[("h2", 1)], 4096, 20, 0.1, 9)
    res = {r["ticket"]: r for r in srv.drain()}
    assert all(r["status"] == 0 for r in res.values())
    spans = sorted((res[t]["t_admit"], res[t]["t_done"]) for t in big)
    assert [res[t]["t_admit"] for t in big] == sorted(res[t]["t_admit"] for t in big)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0  # never two large requests at once
    assert res[small]["t_admit"] < res[big[1]]["t_admit"]
    srv.set_policy(0, 1)  # plain arrival order: the same results
    again = srv.submit(key, 65536, 20, 0.1, 501)
    r2 = srv.drain()[0]
    assert r2["e_mean"] == res[big[1]]["e_mean"] and r2["e_var"] == res[big[1]]["e_var"]
    srv.close()


def test_policy_arguments_are_checked(mix):
    from paper_2506_09743_gb300 import QmcError

    srv, _ = _server(mix, 1 << 30, 2)
    with pytest.raises(QmcError):
        srv.set_policy(-1, 2)
    with pytest.raises(QmcError):
        srv.set_policy(1000, 0)
    srv.close()


def test_cancel_queued_and_running_requests(pkg):
    """qmc_server_cancel: a queued request is removed without device work, a
    running one finishes its kernels but reports QMC_ERR_CANCELLED; the other
    requests are unaffected and the arena is whole again."""
    from paper_2506_09743_gb300 import serving
    from paper_2506_09743_gb300._lib import QMC_ERR_ARG, QMC_ERR_CANCELLED, QmcError

    wf = pkg.Wavefunction(qi.make_lih(), precision="fp64")
    srv = serving.Server(hbm_budget_bytes=1 << 30, max_in_flight=1)
    i = srv.add(wf)
    t = [srv.submit(i, 4096, 10, 0.05, 100 + k) for k in range(5)]
    srv.progress()  # admits t[0] (one slot)
    srv.cancel(t[0])  # running
    srv.cancel(t[2])  # queued
    srv.cancel(t[3])  # queued
    res = {r["ticket"]: r for r in srv.drain()}
    assert sorted(res) == sorted(t)
    for k in (0, 2, 3):
        assert res[t[k]]["status"] == QMC_ERR_CANCELLED and np.isnan(res[t[k]]["e_mean"])
    for k in (1, 4):
        assert res[t[k]]["status"] == 0 and np.isfinite(res[t[k]]["e_mean"])
    with pytest.raises(QmcError) as ei:
        srv.cancel(t[1])  # already finished
    assert ei.value.status == QMC_ERR_ARG
    assert srv.free_bytes() == srv.budget
    # the cancelled requests' seeds give the same results when run afresh
    t2 = srv.submit(i, 4096, 10, 0.05, 101)
    again = srv.drain()
    assert again[0]["e_mean"] == res[t[1]]["e_mean"]
    srv.close()
    wf.close()


def test_nonfinite_walkers_are_counted_not_averaged(pkg):
    """A walker with an electron exactly on a nucleus has no finite local
    energy: the request's result counts it and averages the others."""
    from paper_2506_09743_gb300 import serving

    mol = qi.make_h2()
    W = 256
    r = qi.walkers(mol, W, seed=61)
    r[5, 0] = mol.atom_xyz[0]  # electron 0 of walker 5 on nucleus 0
    r[9, 1] = mol.atom_xyz[1]
    wf = pkg.Wavefunction(mol, precision="fp64")
    srv = serving.Server(hbm_budget_bytes=1 << 28, max_in_flight=2)
    i = srv.add(wf)
    srv.submit(i, W, 0, 0.05, 1, walkers=qi.to_soa(r))
    res = srv.drain()[0]
    e, _ = wf.local_energy(torch.tensor(qi.to_soa(r), device="cuda"))
    e = e.cpu().numpy()
    fin = np.isfinite(e)
    assert res["status"] == 0 and res["n_nonfinite"] == int((~fin).sum()) == 2
    assert abs(res["e_mean"] - e[fin].mean()) <= 1e-12 * abs(e[fin].mean())
    srv.close()
    wf.close()
