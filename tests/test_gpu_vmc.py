"""The VMC energy driver: the Jastrow ratio and the local energy against the oracle, and a
Metropolis walk of exp(J) Psi_MD through the driver replayed move by move by the oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import hamiltonian as H
from paper_1106_2456_gb300 import msd, vmc, workloads as wl
from _parity import tol_fp64, tol_mixed

pytestmark = pytest.mark.gpu

JASTROWS = [(0.0, 0.0), (1.0, 1.5)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _moved(ctx, w, n_moves, mask_u=0.6):
    """Apply n_moves proposals with a fixed accept mask (u < mask_u, independent of the ratio,
    so every precision follows the same positions); return the host positions."""
    p = w.problem
    eta, u = w.proposals(n_moves)
    Rh = w.R0.copy()
    for t in range(n_moves):
        e = (3 * t + 1) % p.n_tot
        rnew = Rh[:, e] + w.tau * eta[t]
        ctx.ratio(e, torch.tensor(rnew, device="cuda"), with_grad=False)
        acc = u[t] < mask_u
        ctx.accept(e, torch.tensor(acc.astype(np.uint8), device="cuda"))
        Rh[acc, e] = rnew[acc]
    return Rh


@pytest.mark.parametrize("label,W", [("water", 16), ("medium", 2)])
def test_local_energy(label, W):
    """E_L of every walker after a few Sherman-Morrison updates, FP64 and mixed, with and
    without the Jastrow: |E_gpu - E_oracle| <= tol(cond A_0) x the size of E_L's terms; the
    Coulomb parts are FP64 pair sums in both modes."""
    w = wl.make_workload(label, n_walkers=W)
    p = w.problem
    Z = wl.nuclear_charges(p)
    orc = oracle.Oracle(p)
    refs = None
    for prec in ("fp64", "mixed"):
        ctx = msd.MSD(p, W, prec, refresh_K=w.refresh_K)
        ctx.set_positions(torch.tensor(w.R0, device="cuda"))
        Rh = _moved(ctx, w, 7)
        Rg, _, _ = ctx.get_state()
        assert np.array_equal(Rg.cpu().numpy(), Rh)
        if refs is None:
            refs = {jas: H.local_energy(orc, Rh, Z, *jas) for jas in JASTROWS}
            kap = np.array([orc.reference_condition(Rh[i]) for i in range(W)])
        tol = (tol_fp64 if prec == "fp64" else tol_mixed)(kap)
        for jas in JASTROWS:
            ctx.set_hamiltonian(Z, *jas)
            e, parts = ctx.local_energy(with_parts=True)
            e, parts = e.cpu().numpy(), parts.cpu().numpy()
            ref = refs[jas]
            err = np.abs(e - ref["eloc"]) / ref["scale"]
            assert np.all(err <= tol), (prec, jas, float((err / tol).max()))
            assert np.allclose(parts[:, 1:], ref["parts"][:, 1:], rtol=1e-12, atol=1e-12), (prec, jas)
            assert np.allclose(parts.sum(axis=1), e, rtol=1e-13, atol=1e-12)
        ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_jastrow_ratio(prec):
    w = wl.make_workload("water", n_walkers=16)
    p = w.problem
    Z = wl.nuclear_charges(p)
    ctx = msd.MSD(p, w.n_walkers, prec, refresh_K=w.refresh_K)
    ctx.set_positions(torch.tensor(w.R0, device="cuda"))
    eta, _ = w.proposals(p.n_tot)
    for b_ee, b_en in ((1.0, 1.5), (0.7, 0.0), (0.0, 2.0)):
        ctx.set_hamiltonian(Z, b_ee, b_en)
        for e in range(p.n_tot):
            rnew = w.R0[:, e] + w.tau * eta[e]
            ratio = torch.full((w.n_walkers,), -2.0, dtype=torch.float64, device="cuda")
            ctx.jastrow_ratio_(e, torch.tensor(rnew, device="cuda"), ratio)
            ref = -2.0 * H.jastrow_ratio(w.R0, p.n_elec[0], e, rnew, p.nuc_xyz, Z, b_ee, b_en)
            assert np.allclose(ratio.cpu().numpy(), ref, rtol=1e-12, atol=0.0), (b_ee, b_en, e)
    # without a Jastrow term the ratio is left as it is
    ctx.set_hamiltonian(Z)
    ratio = torch.full((w.n_walkers,), 3.0, dtype=torch.float64, device="cuda")
    ctx.jastrow_ratio_(0, torch.tensor(w.R0[:, 0] + 0.1, device="cuda"), ratio)
    assert torch.all(ratio == 3.0)
    ctx.close()


def test_vmc_walk_matches_oracle_replay():
    """Two sweeps of exp(J) Psi_MD through the driver (msd_propose, msd_ratio,
    msd_jastrow_ratio, msd_metropolis, msd_accept) with the oracle's random numbers: the
    same accept decisions and positions, then the same local energies."""
    w = wl.make_workload("water", n_walkers=16)
    p = w.problem
    W = w.n_walkers
    Z = wl.nuclear_charges(p)
    b_ee, b_en = 1.0, 1.5
    n_sw = 2
    eta, u = w.proposals(n_sw * p.n_tot)
    ctx = msd.MSD(p, W, "fp64", refresh_K=w.refresh_K)
    ctx.set_positions(torch.tensor(w.R0, device="cuda"))
    drv = vmc.VMC(ctx, Z, b_ee, b_en, tau=w.tau)
    eta_t = torch.tensor(eta, device="cuda").view(n_sw, p.n_tot, W, 3)
    u_t = torch.tensor(u, device="cuda").view(n_sw, p.n_tot, W)
    for s in range(n_sw):
        drv.sweep(eta_t[s], u_t[s])
    orc = oracle.Oracle(p)
    recs, R_or = oracle.vmc_replay(orc, w.R0, eta, u, w.tau, jastrow=dict(Z=Z, b_ee=b_ee, b_en=b_en))
    # a decision within rounding of the threshold may legitimately differ: leave such walkers out
    ok = np.ones(W, dtype=bool)
    for t, r in enumerate(recs):
        a2 = r["ratio_T"] ** 2
        ok &= np.abs(u[t] - a2) > 1e-9 * np.maximum(u[t], a2)
    assert ok.sum() >= W - 1
    Rg = ctx.get_state()[0].cpu().numpy()
    assert np.allclose(Rg[ok], R_or[ok], rtol=0.0, atol=1e-12)
    e = drv.energy().cpu().numpy()
    ref = H.local_energy(orc, R_or, Z, b_ee, b_en)
    kap = np.array([orc.reference_condition(R_or[i]) for i in range(W)])
    assert np.all(np.abs(e[ok] - ref["eloc"][ok]) <= tol_fp64(kap[ok]) * ref["scale"][ok])
    acc = sum(r["accept"].sum() for r in recs) / (len(recs) * W)
    assert 0.05 < acc < 0.95
    # an unattended run: finite estimates and a plausible acceptance
    res = drv.run(n_sweeps=3, n_equil=1)
    assert np.isfinite(res["energy"]) and np.isfinite(res["stderr"]) and 0.0 < res["acceptance"] < 1.0
    ctx.close()


def test_hamiltonian_call_errors():
    w = wl.make_workload("water", n_walkers=4)
    p = w.problem
    ctx = msd.MSD(p, 4, "fp64", refresh_K=w.refresh_K)
    ctx.set_positions(torch.tensor(w.R0, device="cuda"))
    with pytest.raises(msd.MSDError) as ei:
        ctx.local_energy()
    assert ei.value.code == 6  # MSD_ERR_STATE: no Hamiltonian yet
    with pytest.raises(msd.MSDError) as ei:
        ctx.set_hamiltonian(np.array([8.0, -1.0, 1.0]))
    assert ei.value.code == 1
    with pytest.raises(msd.MSDError) as ei:
        ctx.set_hamiltonian(wl.nuclear_charges(p), b_ee=-1.0)
    assert ei.value.code == 1
    ctx.set_hamiltonian(wl.nuclear_charges(p), 1.0, 1.0)
    with pytest.raises(msd.MSDError) as ei:
        ctx.jastrow_ratio_(p.n_tot, torch.zeros((4, 3), dtype=torch.float64, device="cuda"),
                           torch.ones(4, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 1
    ctx.close()
    can = msd.MSD(p, 4, "canonical", refresh_K=w.refresh_K)
    can.set_positions(torch.tensor(w.R0, device="cuda"))
    can.set_hamiltonian(wl.nuclear_charges(p), 1.0, 1.0)
    with pytest.raises(msd.MSDError) as ei:
        can.local_energy()
    assert ei.value.code == 1
    can.close()
