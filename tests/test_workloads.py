"""Sanity of the seeded input generator (shape and structure only, no method arithmetic)."""
import math
import os

import numpy as np
import pytest

from paper_1106_2456_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_water_geometry_matches_section_vi():
    g = _golden("water_geometry.txt")
    xyz = wl.water_nuclei() / wl.BOHR_PER_ANGSTROM
    d1 = np.linalg.norm(xyz[1] - xyz[0])
    d2 = np.linalg.norm(xyz[2] - xyz[0])
    cosang = np.dot(xyz[1] - xyz[0], xyz[2] - xyz[0]) / (d1 * d2)
    assert d1 == pytest.approx(g["r_OH_angstrom"], rel=1e-12)
    assert d2 == pytest.approx(g["r_OH_angstrom"], rel=1e-12)
    assert math.degrees(math.acos(cosang)) == pytest.approx(g["theta_HOH_degree"], rel=1e-12)
    # the stated H coordinates (+-0.757, 0, 0.586) A
    assert abs(xyz[1, 0]) == pytest.approx(0.757, abs=5e-4)
    assert xyz[1, 2] == pytest.approx(0.586, abs=5e-4)


@pytest.mark.parametrize("label", ["water", "medium"])
def test_strings_and_terms_are_well_formed(label):
    w = wl.make_workload(label, n_walkers=8)
    p = w.problem
    assert p.ci[0] == 1.0 and p.det_up[0] == 0 and p.det_dn[0] == 0
    keys = set()
    for I in range(p.n_det):
        keys.add((int(p.det_up[I]), int(p.det_dn[I])))
    assert len(keys) == p.n_det  # no duplicate terms
    for s in range(2):
        n, m = p.n_elec[s], p.n_orb[s] - p.n_elec[s]
        off, h, q = p.exc_off[s], p.exc_holes[s], p.exc_parts[s]
        assert off[0] == 0 and off[1] == 0  # string 0 is the reference
        seen = set()
        for u in range(p.n_exc(s)):
            hh = tuple(h[off[u]:off[u + 1]])
            qq = tuple(q[off[u]:off[u + 1]])
            assert list(hh) == sorted(set(hh)) and list(qq) == sorted(set(qq))
            assert all(x < n for x in hh) and all(x < m for x in qq)
            assert len(hh) <= wl.MAXK
            seen.add((hh, qq))
        assert len(seen) == p.n_exc(s)
        used = p.det_up if s == 0 else p.det_dn
        assert set(np.unique(used)) == set(range(p.n_exc(s)))
    assert w.R0.shape == (8, p.n_tot, 3)


def test_generator_is_deterministic():
    a = wl.make_workload("water", n_walkers=4)
    b = wl.make_workload("water", n_walkers=4)
    assert np.array_equal(a.problem.ci, b.problem.ci)
    assert np.array_equal(a.R0, b.R0)
    assert np.array_equal(a.problem.exc_holes[1], b.problem.exc_holes[1])


def test_nuclear_charges_make_every_system_neutral():
    w = wl.make_workload("water", n_walkers=1)
    assert list(wl.nuclear_charges(w.problem)) == [8.0, 1.0, 1.0]
    for n, n_nuc in (((5, 4), 4), ((7, 7), 3), ((3, 2), 6)):
        c = wl.custom_workload(n, (n[0] + 4, n[1] + 4), 10, wl.uniform_orders(1, 2), W=1, n_nuc=n_nuc, seed=2)
        Z = wl.nuclear_charges(c.problem)
        assert Z.sum() == sum(n) and Z.max() - Z.min() <= 1 and np.all(Z == np.round(Z))
