"""Host logic of the VMC driver without a GPU: the blocking error estimate against the closed
form of an AR(1) series, the sweep/run bookkeeping through a stand-in context, and the
cross-replica combination on two gloo ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1106_2456_gb300 import vmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ar1(rng, phi, n):
    x = np.empty(n)
    x[0] = rng.standard_normal() / np.sqrt(1 - phi * phi)
    eps = rng.standard_normal(n)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + eps[t]
    return x


def test_blocking_matches_ar1_closed_form():
    """x_t = phi x_{t-1} + e_t, Var(e) = 1: Var(mean) -> (1 + phi) / ((1 - phi) (1 - phi^2) N)."""
    phi, n = 0.8, 1 << 16
    exact = np.sqrt((1 + phi) / ((1 - phi) * (1 - phi * phi) * n))
    rng = np.random.default_rng(7)
    est, naive = [], []
    for _ in range(8):
        x = _ar1(rng, phi, n)
        est.append(vmc.blocking_stderr(x))
        naive.append(x.std(ddof=1) / np.sqrt(n))
    r = np.mean(est) / exact
    assert 0.85 < r < 1.25, r
    # the naive error misses the correlation by sqrt((1 + phi) / (1 - phi)) = 3
    assert abs(np.mean(naive) / exact - 1 / 3) < 0.05


def test_blocking_on_independent_values_is_the_naive_error():
    x = np.random.default_rng(3).standard_normal(1 << 14)
    naive = x.std(ddof=1) / np.sqrt(x.size)
    assert 0.95 <= vmc.blocking_stderr(x) / naive < 1.3
    assert np.isnan(vmc.blocking_stderr([1.0]))
    assert vmc.blocking_stderr([1.0, 3.0]) == pytest.approx(1.0)


class _StandIn:
    """The calls VMC makes, on the CPU: even walkers always accept (ratio 2), odd never (0);
    the local energy of every walker after the t-th call is t."""

    def __init__(self, W=6, n_tot=3):
        self.W, self.n_tot, self.dev = W, n_tot, torch.device("cpu")
        self.t = 0
        self.jastrow_calls = 0
        self.accepted = 0

    def set_hamiltonian(self, Z, b_ee, b_en):
        self.ham = (list(Z), b_ee, b_en)

    def propose(self, e, eta, tau, out):
        out.copy_(tau * eta)

    def ratio_into(self, e, rnew, ratio, grad=None, lap=None):
        ratio.copy_(torch.where(torch.arange(self.W) % 2 == 0, 2.0, 0.0).to(torch.float64))

    def jastrow_ratio_(self, e, rnew, ratio):
        self.jastrow_calls += 1

    def metropolis(self, u, ratio, out):
        out.copy_((u < ratio * ratio).to(torch.uint8))

    def accept(self, e, acc):
        self.accepted += int(acc.sum())

    def local_energy_into(self, eloc, parts=None):
        self.t += 1
        eloc.fill_(float(self.t))


@pytest.mark.parametrize("b_ee", [0.0, 1.0])
def test_run_bookkeeping(b_ee):
    c = _StandIn()
    d = vmc.VMC(c, [1.0, 2.0], b_ee=b_ee, tau=0.3, seed=1)
    res = d.run(n_sweeps=4, n_equil=2)
    assert res["energy"] == pytest.approx(2.5)          # sweeps see E = 1, 2, 3, 4
    assert res["acceptance"] == pytest.approx(0.5)      # half the walkers always accept
    assert res["sweeps"] == 4 and np.isfinite(res["stderr"])
    assert c.jastrow_calls == (c.n_tot * 6 if b_ee > 0 else 0)
    assert c.accepted == (c.W // 2) * c.n_tot * 6
    # explicit random numbers: eta and u per electron
    eta = torch.zeros((c.n_tot, c.W, 3), dtype=torch.float64)
    u = torch.full((c.n_tot, c.W), 0.5, dtype=torch.float64)
    d.sweep(eta, u)
    assert c.accepted == (c.W // 2) * c.n_tot * 7


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_1106_2456_gb300 import vmc as v

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    W = 3 + rank
    sums = torch.tensor([10.0 * (rank + 1), 20.0 + rank, -5.0 * rank], dtype=torch.float64)
    means, acc = v.combine_replicas(sums, W, n_accepted=2.0 + rank, n_proposed=10.0 * (rank + 1))
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([means.numpy(), [acc]]))
    dist.destroy_process_group()


def test_combine_replicas_on_two_gloo_ranks(tmp_path):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    a, b = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    expect = np.array([(10.0 + 20.0) / 7, (20.0 + 21.0) / 7, (0.0 - 5.0) / 7, (2.0 + 3.0) / 30.0])
    assert np.allclose(a, expect) and np.allclose(b, expect)


def test_combine_replicas_single_process():
    means, acc = vmc.combine_replicas(torch.tensor([6.0, 9.0]), 3, 1.0, 4.0)
    assert means.tolist() == [2.0, 3.0] and acc == 0.25
