"""msd_backward (adjoint of log|Psi| w.r.t. c_I and B) against the oracle's Jacobi-formula
adjoint, summed over walkers with random weights, entry by entry:

    |dX_gpu - dX_oracle| <= tol(kappa) * max(|dX_oracle|, scale_X)

with scale_X the size of the terms that cancel in that entry (``_reference``) and tol the
parity bar of the precision at the walkers' reference condition number."""
import numpy as np
import pytest
import torch

import oracle
from paper_1106_2456_gb300 import msd, workloads as wl
from _parity import tol_fp64, tol_mixed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _reference(p, R, gbar, walkers=None):
    """Oracle adjoint summed over walkers with weights gbar, and the per-entry cancellation
    scale of every entry: sum_w |gbar_w| x (size of the terms forming that walker's entry).
    For d/dc_I = t_I / S the terms are those of S, so the scale is |t_I / S| max(1, sum_J
    |c_J t_J| / |S|); for d/dB it is the oracle's sum of absolute terms of Jacobi's formula."""
    orc = oracle.Oracle(p)
    dci = np.zeros(p.n_det)
    sci = np.zeros(p.n_det)
    dB = [np.zeros((p.n_basis, p.n_orb[0])), np.zeros((p.n_basis, p.n_orb[1]))]
    sB = [np.zeros_like(dB[0]), np.zeros_like(dB[1])]
    kappa = 1.0
    for w in (range(R.shape[0]) if walkers is None else walkers):
        if gbar[w] == 0.0:
            continue
        c, (b0, b1), (s0, s1) = orc.dlogpsi(R[w], with_scale=True)
        absum = orc.eval(R[w])["absum"][0, 0]
        dci += gbar[w] * c
        sci += abs(gbar[w]) * np.abs(c) * max(1.0, absum)
        dB[0] += gbar[w] * b0
        dB[1] += gbar[w] * b1
        sB[0] += abs(gbar[w]) * s0
        sB[1] += abs(gbar[w]) * s1
        kappa = max(kappa, orc.reference_condition(R[w]))
    return dci, dB, sci, sB, kappa


def _tol(prec, kappa):
    return float(tol_mixed(kappa) if prec == "mixed" else tol_fp64(kappa))


def _errors(ctx, p, R, gbar, walkers=None):
    """Element-wise errors in units of max(|ref_i|, scale_i): the largest over d/dc and d/dB."""
    dci, (b0, b1) = ctx.backward(torch.tensor(gbar, device="cuda"))
    ref_c, ref_B, sc_c, sc_B, kappa = _reference(p, R, gbar, walkers)
    tiny = 1e-300
    e_c = np.max(np.abs(dci.cpu().numpy() - ref_c) / np.maximum(np.maximum(np.abs(ref_c), sc_c), tiny))
    e_B = max(np.max(np.abs(g.cpu().numpy() - r) / np.maximum(np.maximum(np.abs(r), sc), tiny))
              for g, r, sc in ((b0, ref_B[0], sc_B[0]), (b1, ref_B[1], sc_B[1])))
    return e_c, e_B, kappa


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_water(prec):
    w = wl.make_workload("water", n_walkers=6)
    p = w.problem
    ctx = msd.MSD(p, w.n_walkers, prec, refresh_K=w.refresh_K)
    ctx.set_positions(torch.tensor(w.R0, device="cuda"))
    gbar = np.random.default_rng(5).standard_normal(w.n_walkers)
    e_c, e_B, kappa = _errors(ctx, p, w.R0, gbar)
    tol = _tol(prec, kappa)
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
    tol = _tol(prec, kappa)
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
    tol = _tol("fp64", kappa)
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
    tol = _tol("fp64", kappa)
    assert e_c <= tol and e_B <= tol, (e_c, e_B, kappa)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_differentiation_config(prec):
    """The differentiation workload in its own launch configuration (32 + 32 electrons, 160
    orbitals per spin, 5e4 determinants, orders 1-6, 4096 walkers): after three moves of every
    walker, the adjoint weighted on three sampled walkers (the others weighted 0), entry by
    entry against the oracle."""
    wk = wl.make_workload("diff")
    p = wk.problem
    W = wk.n_walkers
    ctx = msd.MSD(p, W, prec, refresh_K=wk.refresh_K)
    ctx.set_positions(torch.tensor(wk.R0, device="cuda"))
    eta, u = wk.proposals(3)
    R = wk.R0.copy()
    for t, e in enumerate((0, 33, 5)):
        rnew = R[:, e] + wk.tau * eta[t]
        r, _, _ = ctx.ratio(e, torch.tensor(rnew, device="cuda"))
        acc = u[t] < (r * r).cpu().numpy()
        ctx.accept(e, torch.tensor(acc.astype(np.uint8), device="cuda"))
        R[acc, e] = rnew[acc]
    sample = [3, 2048, 4095]
    gbar = np.zeros(W)
    gbar[sample] = [1.0, -0.7, 0.4]
    e_c, e_B, kappa = _errors(ctx, p, R, gbar, walkers=sample)
    tol = _tol(prec, kappa)
    print(f"diff {prec}: element-wise error / scale: dci {e_c:.3e}, dB {e_B:.3e}, bar {tol:.3e} (kappa {kappa:.3e})")
    assert e_c <= tol and e_B <= tol, (e_c, e_B, kappa)
    ctx.close()
