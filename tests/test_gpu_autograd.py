"""LogPsi (torch.autograd over msd_set_params + msd_backward) against central finite
differences of the library's own log|Psi| (h = 1e-6), and msd_set_params against a context
built from the new parameters."""
import numpy as np
import pytest
import torch

from paper_1106_2456_gb300 import msd, workloads as wl
from paper_1106_2456_gb300.autograd import log_psi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_set_params_equals_fresh_context():
    w = wl.make_workload("water", n_walkers=8)
    p = w.problem
    rng = np.random.default_rng(3)
    ci2 = p.ci * (1 + 0.1 * rng.standard_normal(p.n_det))
    B2 = (p.B[0] + 0.05 * rng.standard_normal(p.B[0].shape), p.B[1] + 0.05 * rng.standard_normal(p.B[1].shape))
    R = torch.tensor(w.R0, device="cuda")
    a = msd.MSD(p, w.n_walkers, "fp64")
    a.set_positions(R)
    a.set_params(ci2, B2)
    p2 = wl.dataclasses.replace(p, ci=ci2, B=B2)
    b = msd.MSD(p2, w.n_walkers, "fp64")
    b.set_positions(R)
    _, la, sa = a.get_state()
    _, lb, sb = b.get_state()
    assert torch.equal(sa, sb) and torch.allclose(la, lb, rtol=0, atol=1e-12)
    rnew = R[:, 2] + 0.2
    ra, ga, lpa = a.ratio(2, rnew.contiguous())
    rb, gb, lpb = b.ratio(2, rnew.contiguous())
    assert torch.allclose(ra, rb, rtol=1e-12) and torch.allclose(ga, gb, rtol=1e-12, atol=1e-13)
    a.close()
    b.close()


def test_log_psi_gradient_matches_finite_differences():
    w = wl.make_workload("water", n_walkers=4)
    p = w.problem
    wf = msd.MSD(p, w.n_walkers, "fp64")
    wf.set_positions(torch.tensor(w.R0, device="cuda"))
    ci = torch.tensor(p.ci, dtype=torch.float64, requires_grad=True)
    B0 = torch.tensor(p.B[0], dtype=torch.float64, requires_grad=True)
    B1 = torch.tensor(p.B[1], dtype=torch.float64, requires_grad=True)
    gbar = torch.tensor([0.5, -1.0, 2.0, 0.25], dtype=torch.float64, device="cuda")
    loss = (log_psi(wf, ci, B0, B1) * gbar).sum()
    loss.backward()

    def f(c, b0, b1):
        with torch.no_grad():
            return float((log_psi(wf, c, b0, b1) * gbar).sum())

    h = 1e-6
    rng = np.random.default_rng(1)
    for I in [0, 1] + list(rng.choice(p.n_det, 6, replace=False)):
        cp, cm = ci.detach().clone(), ci.detach().clone()
        cp[I] += h
        cm[I] -= h
        fd = (f(cp, B0, B1) - f(cm, B0, B1)) / (2 * h)
        assert abs(fd - float(ci.grad[I])) <= 1e-5 * max(1.0, abs(fd)), (I, fd, float(ci.grad[I]))
    for s, (B, Bg) in enumerate(((B0, B0.grad), (B1, B1.grad))):
        for _ in range(6):
            mu, j = int(rng.integers(B.shape[0])), int(rng.integers(B.shape[1]))
            bp, bm = B.detach().clone(), B.detach().clone()
            bp[mu, j] += h
            bm[mu, j] -= h
            args_p = (ci, bp, B1) if s == 0 else (ci, B0, bp)
            args_m = (ci, bm, B1) if s == 0 else (ci, B0, bm)
            fd = (f(*args_p) - f(*args_m)) / (2 * h)
            assert abs(fd - float(Bg[mu, j])) <= 1e-5 * max(1.0, abs(fd)), (s, mu, j, fd, float(Bg[mu, j]))
    wf.close()
