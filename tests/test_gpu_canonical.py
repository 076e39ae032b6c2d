"""The canonical method (MSD_CANONICAL: every determinant's own inverse, Sherman-Morrison
updates) against the oracle and against the table method on the same trajectory."""
import numpy as np
import pytest
import torch

import oracle
from paper_1106_2456_gb300 import msd, workloads as wl
from _parity import rel_err, replay, tol_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_canonical_water_every_move():
    w = wl.make_workload("water", n_walkers=32)
    out = replay(w, "canonical", n_steps=5 * w.problem.n_tot)
    for key in ("ratio", "grad", "lap"):
        assert max(out[key + "_n"]) <= 1.0, (key, max(out[key + "_n"]))
    assert out["sign0_ok"] and out["sign_final_ok"] and out["R_final_err"] == 0.0
    assert out["logabs_final"] <= 1.0


@pytest.mark.parametrize("orders", [wl.uniform_orders(1, 8)])
def test_canonical_equals_table(orders):
    """Orders 1..8 with sparse singles: the canonical and table methods give the same ratios."""
    wk = wl.custom_workload((11, 9), (25, 26), 300, orders, W=8, n_nuc=4, seed=11, K=7)
    p = wk.problem
    a = msd.MSD(p, wk.n_walkers, "canonical", refresh_K=wk.refresh_K)
    b = msd.MSD(p, wk.n_walkers, "fp64", refresh_K=wk.refresh_K)
    R = torch.tensor(wk.R0, device="cuda")
    a.set_positions(R)
    b.set_positions(R)
    eta, u = wk.proposals(3 * p.n_tot)
    Rh = wk.R0.copy()
    orc = oracle.Oracle(p)
    for t in range(3 * p.n_tot):
        e = t % p.n_tot
        rnew = Rh[:, e] + wk.tau * eta[t]
        ra, ga, la = a.ratio(e, torch.tensor(rnew, device="cuda"))
        rb, gb, lb = b.ratio(e, torch.tensor(rnew, device="cuda"))
        kap = max(orc.reference_condition(Rh[i], e, rnew[i]) for i in range(wk.n_walkers))
        tol = 10 * tol_fp64(kap)
        assert torch.allclose(ra, rb, rtol=tol, atol=tol), t
        assert torch.allclose(ga, gb, rtol=tol, atol=tol) and torch.allclose(la, lb, rtol=tol, atol=tol * 10), t
        acc = (u[t] < (rb * rb).cpu().numpy()).astype(np.uint8)
        a.accept(e, torch.tensor(acc, device="cuda"))
        b.accept(e, torch.tensor(acc, device="cuda"))
        Rh[acc.astype(bool), e] = rnew[acc.astype(bool)]
    _, la_, sa = a.get_state()
    _, lb_, sb = b.get_state()
    assert torch.equal(sa, sb) and torch.allclose(la_, lb_, rtol=0, atol=1e-8)
    a.close()
    b.close()


def test_canonical_rejects_table_only_calls():
    w = wl.make_workload("water", n_walkers=4)
    c = msd.MSD(w.problem, w.n_walkers, "canonical")
    c.set_positions(torch.tensor(w.R0, device="cuda"))
    with pytest.raises(msd.MSDError, match="canonical"):
        c.grad_lap(0)
    c.close()
