"""The timeout path of the bounded device waits (tensor-core AO stages).

With a wait budget of 0 cycles every mbarrier wait of k_ao_mo_tc or k_ao_mo_oz gives up at
once on a healthy GPU: the block records the failure, drains the MMAs it
issued (with the normal budget), writes NaN for its remaining MO values and
frees its tensor memory.  The host must then see QMC_ERR_TIMEOUT wherever
the status can be read (qmc_check_status after the stream-ordered calls,
qmc_local_energy_host, a server result), never QMC_OK with NaN energies, and
the context must stay usable: with the default budget restored the results
are the ones of an untouched wavefunction."""
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


# CO: two K-passes (the wait between passes and the final wait); LiH: one.
# mixed_tf32 runs k_ao_mo_tc; fp32x2 on CO runs k_ao_mo_oz (its value path
# k_ao_mo_tc; LiH's small contraction takes the SIMT pair kernel instead)
@pytest.mark.parametrize("name,precision", [("co", "mixed_tf32"), ("lih", "mixed_tf32"), ("co", "fp32x2")])
def test_timeout_is_reported_and_poisons_outputs(pkg, name, precision):
    from paper_2506_09743_gb300 import QmcError
    from paper_2506_09743_gb300._lib import QMC_ERR_TIMEOUT

    mol = qi.make_co(n_det=20) if name == "co" else qi.make_lih()
    W = 1000
    soa = np.ascontiguousarray(qi.to_soa(qi.walkers(mol, W, seed=31)))
    x = torch.tensor(soa, device="cuda")
    wf = pkg.Wavefunction(mol, precision=precision)
    e_ok, lp_ok = wf.local_energy(x)
    wf.check_status()

    wf.set_wait_limit(0)
    e, lp = wf.local_energy(x)
    with pytest.raises(QmcError) as ei:
        wf.check_status()
    assert ei.value.status == QMC_ERR_TIMEOUT
    assert torch.isnan(e).all() and torch.isnan(lp).all()
    wf.check_status()  # the record was cleared by the check

    e_h, lp_h = np.empty(W), np.empty(W)
    with pytest.raises(QmcError) as ei:
        wf.local_energy_host(soa, e_loc=e_h, log_psi=lp_h)
    assert ei.value.status == QMC_ERR_TIMEOUT
    assert np.isnan(e_h).all()

    xs = x.clone()
    wf.sample(xs, n_steps=2, step=0.05, seed=3)
    with pytest.raises(QmcError) as ei:
        wf.check_status()
    assert ei.value.status == QMC_ERR_TIMEOUT

    wf.set_wait_limit(1 << 31)
    e2, lp2 = wf.local_energy(x)
    wf.check_status()
    torch.cuda.synchronize()
    assert torch.equal(e2, e_ok) and torch.equal(lp2, lp_ok)
    wf.close()


def test_timeout_in_a_server_request(pkg):
    from paper_2506_09743_gb300 import serving
    from paper_2506_09743_gb300._lib import QMC_ERR_TIMEOUT

    good = pkg.Wavefunction(qi.make_lih(), precision="mixed_tf32")
    bad = pkg.Wavefunction(qi.make_lih(), precision="mixed_tf32")
    bad.set_wait_limit(0)
    srv = serving.Server(hbm_budget_bytes=1 << 30, max_in_flight=4)
    ig, ib = srv.add(good), srv.add(bad)
    tg = srv.submit(ig, 4096, 5, 0.05, 11)
    tb = srv.submit(ib, 4096, 5, 0.05, 11)
    res = {r["ticket"]: r for r in srv.drain()}
    assert res[tg]["status"] == 0 and np.isfinite(res[tg]["e_mean"])
    assert res[tb]["status"] == QMC_ERR_TIMEOUT and np.isnan(res[tb]["e_mean"])
    srv.close()
    good.close()
    bad.close()
