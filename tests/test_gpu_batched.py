"""Batched uneven systems (msd_init with n_systems > 1) against one single-system context per
system on the same inputs, and against the oracle on sampled walkers of every system."""
import numpy as np
import pytest
import torch

import oracle
from paper_1106_2456_gb300 import msd, workloads as wl
from _parity import rel_err, tol_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _systems():
    ws = [wl.make_workload("water", n_walkers=6),
          wl.custom_workload((11, 9), (25, 26), 300, wl.uniform_orders(1, 8), W=5, n_nuc=4, seed=11, K=7),
          wl.custom_workload((1, 1), (6, 4), 9, wl.uniform_orders(1, 2), W=3, n_nuc=2, seed=3, K=3)]
    ws += wl.batched_workloads(3, W=4, seed=21, n_range=(4, 20), det_range=(1e2, 3e3))
    return ws


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_single_contexts(prec):
    ws = _systems()
    Ks = [w.refresh_K for w in ws]
    b = msd.MSDBatch([w.problem for w in ws], [w.n_walkers for w in ws], prec, refresh_K=Ks)
    singles = [msd.MSD(w.problem, w.n_walkers, prec, refresh_K=w.refresh_K) for w in ws]
    R = np.concatenate([w.R0.reshape(-1) for w in ws])
    b.set_positions(torch.tensor(R, device="cuda"))
    for w, c in zip(ws, singles):
        c.set_positions(torch.tensor(w.R0, device="cuda"))
    W = b.W
    rng = np.random.default_rng(9)
    off = np.cumsum([0] + [w.n_walkers for w in ws])
    tol = 1e-12 if prec == "fp64" else 1e-5
    for t in range(30):
        eta = torch.tensor(rng.standard_normal((W, 3)), device="cuda")
        rnew = torch.empty(W, 3, dtype=torch.float64, device="cuda")
        b.propose(t, eta, 0.4, rnew)
        r, g, l = b.ratio(t, rnew)
        u = torch.tensor(rng.random(W), device="cuda")
        acc = torch.empty(W, dtype=torch.uint8, device="cuda")
        b.metropolis(u, r, acc)
        for s, (w, c) in enumerate(zip(ws, singles)):
            sl = slice(off[s], off[s + 1])
            e = t % w.problem.n_tot
            r1, g1, l1 = c.ratio(e, rnew[sl].contiguous())
            for x, y in ((r[sl], r1), (g[sl], g1), (l[sl], l1)):
                assert bool(((x - y).abs() <= tol * y.abs().clamp_min(1.0)).all()), (s, t)
            c.accept(e, acc[sl].contiguous())
        b.accept(t, acc)
    b.sync()
    Rb, lb, sb = b.get_state()
    pos = 0
    for s, (w, c) in enumerate(zip(ws, singles)):
        Rs, ls, ss = c.get_state()
        n = Rs.numel()
        assert torch.equal(Rb[pos:pos + n], Rs.reshape(-1))
        assert torch.equal(sb[off[s]:off[s + 1]], ss)
        assert torch.allclose(lb[off[s]:off[s + 1]], ls, rtol=0, atol=1e-9)
        pos += n
        c.close()
    b.close()


def test_batch_against_oracle_and_backward():
    ws = _systems()
    b = msd.MSDBatch([w.problem for w in ws], [w.n_walkers for w in ws], "fp64")
    R = np.concatenate([w.R0.reshape(-1) for w in ws])
    b.set_positions(torch.tensor(R, device="cuda"))
    e = 3
    rnew_parts = []
    for w in ws:
        rnew_parts.append(w.R0[:, e % w.problem.n_tot] + 0.3)
    rnew = np.concatenate(rnew_parts)
    r, g, l = b.ratio(e, torch.tensor(rnew, device="cuda"))
    r, g, l = r.cpu().numpy(), g.cpu().numpy(), l.cpu().numpy()
    off = np.cumsum([0] + [w.n_walkers for w in ws])
    for s, w in enumerate(ws):
        orc = oracle.Oracle(w.problem)
        es = e % w.problem.n_tot
        cur = orc.eval(w.R0)
        ref, new = orc.ratio(w.R0, es, rnew_parts[s], cur)
        kap = max(orc.reference_condition(w.R0[i], es, rnew_parts[s][i]) for i in range(w.n_walkers))
        sl = slice(off[s], off[s + 1])
        assert np.all(rel_err(r[sl], ref, new["absum"][:, 0] * np.abs(ref)) <= tol_fp64(kap)), s
        assert np.all(rel_err(g[sl], new["grad"], new["absum"][:, 1:4]) <= tol_fp64(kap)), s
        assert np.all(rel_err(l[sl], new["lap"], new["absum"][:, 4]) <= tol_fp64(kap)), s
    # the adjoint: concatenated per system
    gbar = np.linspace(-1.0, 1.0, b.W)
    dci, dB = b.backward(torch.tensor(gbar, device="cuda"))
    dci, dB = dci.cpu().numpy(), dB.cpu().numpy()
    pc = pb = 0
    for s, w in enumerate(ws):
        c = msd.MSD(w.problem, w.n_walkers, "fp64")
        c.set_positions(torch.tensor(w.R0, device="cuda"))
        d1, (b0, b1) = c.backward(torch.tensor(gbar[off[s]:off[s + 1]], device="cuda"))
        nd, nB = w.problem.n_det, b0.numel() + b1.numel()
        ref_B = np.concatenate([b0.cpu().numpy().ravel(), b1.cpu().numpy().ravel()])
        assert np.allclose(dci[pc:pc + nd], d1.cpu().numpy(), rtol=1e-10, atol=1e-12 * np.abs(dci[pc:pc + nd]).max())
        assert np.allclose(dB[pb:pb + nB], ref_B, rtol=1e-10, atol=1e-12 * np.abs(ref_B).max())
        pc += nd
        pb += nB
        c.close()
    b.close()
