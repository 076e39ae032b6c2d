"""Step A1 (Algorithm 1 step 2) through msd_orbitals against the oracle's orbitals.

FP64 path: the SIMT product in FP64.  Mixed path: the tensor-core product (tcgen05, three TF32
pieces per operand, FP32 accumulator).  Each orbital value or derivative phi^a_j(r) is compared
with the oracle's FP64 value relative to the size of the terms it sums,
scale = sum_mu |d^a chi_mu(r)| |B[mu][j]|, so cancellation between basis functions is judged
against what rounding of those terms allows: 1e-13 (FP64) and 2e-6 (FP32: about 30 units of
the last place).  Shapes cover a ragged last tile of 128 rows, orbital counts that are not a
multiple of 32, and more than 256 orbitals (two column tiles)."""
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


def _reference(p, spin, pts):
    orc = oracle.Oracle(p)
    ref = np.stack([orc.orbitals(spin, r) for r in pts])              # [P][5][N]
    chi = np.stack([orc.basis(r) for r in pts])                        # [P][5][nb]
    scale = np.einsum("pan,nj->paj", np.abs(chi), np.abs(p.B[spin]))  # [P][5][N]
    return ref, scale


CASES = [
    ("water", lambda: wl.make_workload("water", n_walkers=2).problem),
    ("large", lambda: wl.make_workload("large", n_walkers=2, n_det=200).problem),
    ("n=50, N=300", lambda: wl.custom_workload((50, 6), (300, 40), 30, wl.uniform_orders(1, 3), W=2, n_nuc=5,
                                              seed=21, K=4).problem),
]


@pytest.mark.parametrize("label,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_orbitals_against_oracle(label, make, prec, tol):
    p = make()
    rng = np.random.default_rng(3)
    ctx = msd.MSD(p, 2, prec)
    worst = 0.0
    for spin in (0, 1):
        for P in (1, 77, 300):  # 300 points x 5 channels = 1500 rows: 11 full tiles of 128 and a tail
            pts = p.nuc_xyz[rng.integers(0, p.nuc_xyz.shape[0], P)] + rng.standard_normal((P, 3))
            ref, scale = _reference(p, spin, pts)
            for nch in (5, 1):
                out = ctx.orbitals(spin, torch.tensor(pts, device="cuda"), nch).double().cpu().numpy()
                err = np.abs(out - ref[:, :nch]) / np.maximum(scale[:, :nch], 1e-300)
                worst = max(worst, float(err.max()))
                assert err.max() <= tol, (label, prec, spin, P, nch, float(err.max()))
    print(f"{label} {prec}: largest error / scale {worst:.2e}")
    ctx.sync()
    ctx.close()
