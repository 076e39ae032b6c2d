"""The table method on a problem rewritten around another reference determinant (Section V):
every move of a walk against the oracle, which evaluates the unchanged wavefunction."""
import dataclasses

import pytest
import torch

from paper_1106_2456_gb300 import reference, workloads as wl
from _parity import replay

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_switched_reference_every_move(precision):
    w = wl.make_workload("water", n_walkers=16)
    q = reference.switch_reference(w.problem, reference.heaviest_term(w.problem))
    out = replay(dataclasses.replace(w, problem=q), precision, n_steps=2 * q.n_tot)
    for key in ("ratio", "grad", "lap"):
        assert max(out[key + "_n"]) <= 1.0, (key, max(out[key + "_n"]))
    assert out["sign0_ok"] and out["sign_final_ok"] and out["R_final_err"] == 0.0
