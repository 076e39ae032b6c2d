"""msd_backward (adjoint of log|Psi| w.r.t. c_I and B) against the oracle's Jacobi-formula
adjoint, summed over walkers with random weights."""
import numpy as np
import pytest
import torch

import oracle
from paper_1106_2456_gb300 import msd, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _reference(p, R, gbar):
    orc = oracle.Oracle(p)
    dci = np.zeros(p.n_det)
    dB = [np.zeros((p.n_basis, p.n_orb[0])), np.zeros((p.n_basis, p.n_orb[1]))]
    kappa = 1.0
    for w in range(R.shape[0]):
        c, (b0, b1) = orc.dlogpsi(R[w])
        dci += gbar[w] * c
        dB[0] += gbar[w] * b0
        dB[1] += gbar[w] * b1
        kappa = max(kappa, orc.reference_condition(R[w]))
    return dci, dB, kappa


def _errors(ctx, p, R, gbar):
    dci, (b0, b1) = ctx.backward(torch.tensor(gbar, device="cuda"))
    ref_c, ref_B, kappa = _reference(p, R, gbar)
    e_c = np.max(np.abs(dci.cpu().numpy() - ref_c)) / np.max(np.abs(ref_c))
    e_B = max(np.max(np.abs(g.cpu().numpy() - r)) / np.max(np.abs(r)) for g, r in ((b0, ref_B[0]), (b1, ref_B[1])))
    return e_c, e_B, kappa


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_water(prec):
    w = wl.make_workload("water", n_walkers=6)
    p = w.problem
    ctx = msd.MSD(p, w.n_walkers, prec, refresh_K=w.refresh_K)
    ctx.set_positions(torch.tensor(w.R0, device="cuda"))
    gbar = np.random.default_rng(5).standard_normal(w.n_walkers)
    e_c, e_B, kappa = _errors(ctx, p, w.R0, gbar)
    # norm-wise relative errors; the table method passes every quantity through A_0^{-1}
    tol = (1e-10 if prec == "fp64" else 1e3 * 2.0 ** -24) * max(kappa, 10.0)
    assert e_c <= tol and e_B <= tol, (e_c, e_B, kappa)
    # after moves the adjoint is taken at the new positions
    eta, u = w.proposals(4)
    R = w.R0.copy()
    for t in range(4):
        e = (3 * t + 1) % p.n_tot
        rnew = R[:, e] + w.tau * eta[t]
        r, _, _ = ctx.ratio(e, torch.tensor(rnew, device="cuda"))
        acc = u[t] < (r * r).cpu().numpy()
        ctx.accept(e, torch.tensor(acc.astype(np.uint8), device="cuda"))
        R[acc, e] = rnew[acc]
    e_c, e_B, kappa = _errors(ctx, p, R, gbar)
    tol = (1e-10 if prec == "fp64" else 1e3 * 2.0 ** -24) * max(kappa, 10.0)
    assert e_c <= tol and e_B <= tol, (e_c, e_B, kappa)
    ctx.close()


def test_backward_all_orders():
    """Orders 1..8 with sparse singles, odd sizes."""
    wk = wl.custom_workload((11, 9), (25, 26), 300, wl.uniform_orders(1, 8), W=3, n_nuc=4, seed=11, K=7)
    p = wk.problem
    ctx = msd.MSD(p, wk.n_walkers, "fp64", refresh_K=wk.refresh_K)
    ctx.set_positions(torch.tensor(wk.R0, device="cuda"))
    gbar = np.array([1.0, -0.5, 2.0])
    e_c, e_B, kappa = _errors(ctx, p, wk.R0, gbar)
    tol = 1e-10 * max(kappa, 10.0)
    assert e_c <= tol and e_B <= tol, (e_c, e_B, kappa)
    ctx.close()


def test_backward_identities_medium():
    """Medium size (32 + 32 electrons, dense singles), FP64: the two exact identities of the
    adjoint on the GPU output, sum_I c_I dlog/dc_I = sum_w gbar_w (linearity in c) and
    sum B_s dlog/dB_s = n_s sum_w gbar_w (homogeneity in B), and the oracle on one walker."""
    wk = wl.make_workload("medium", n_walkers=4)
    p = wk.problem
    ctx = msd.MSD(p, wk.n_walkers, "fp64", refresh_K=wk.refresh_K)
    ctx.set_positions(torch.tensor(wk.R0, device="cuda"))
    gbar = np.array([0.7, -1.3, 0.4, 1.1])
    dci, (b0, b1) = ctx.backward(torch.tensor(gbar, device="cuda"))
    dci, b0, b1 = dci.cpu().numpy(), b0.cpu().numpy(), b1.cpu().numpy()
    scale = np.sum(np.abs(p.ci * dci))
    assert abs(np.dot(p.ci, dci) - gbar.sum()) <= 1e-9 * max(scale, 1.0)
    for s, b in ((0, b0), (1, b1)):  # each spin's determinants are homogeneous of degree n_s in B_s
        hom = np.sum(p.B[s] * b)
        assert abs(hom - p.n_elec[s] * gbar.sum()) <= 1e-8 * np.sum(np.abs(p.B[s] * b))
    one = np.array([1.0, 0.0, 0.0, 0.0])
    e_c, e_B, kappa = _errors(ctx, p, wk.R0, one)
    tol = 1e-10 * max(kappa, 10.0)
    assert e_c <= tol and e_B <= tol, (e_c, e_B, kappa)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_differentiation_config(prec):
    """The differentiation workload's shape (32 + 32 electrons, 160 orbitals per spin, 5e4
    determinants, orders 1-6): the adjoint of 2 walkers against the oracle."""
    wk = wl.make_workload("diff", n_walkers=2)
    p = wk.problem
    ctx = msd.MSD(p, wk.n_walkers, prec, refresh_K=wk.refresh_K)
    ctx.set_positions(torch.tensor(wk.R0, device="cuda"))
    gbar = np.array([1.0, -0.7])
    e_c, e_B, kappa = _errors(ctx, p, wk.R0, gbar)
    tol = (1e-10 if prec == "fp64" else 1e3 * 2.0 ** -24) * max(kappa, 10.0)
    assert e_c <= tol and e_B <= tol, (e_c, e_B, kappa)
    ctx.close()
