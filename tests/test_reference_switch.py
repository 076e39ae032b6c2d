"""Reference-determinant switching (Section V) on the host: the rewritten problem is the same
wavefunction (checked by the oracle's determinant-by-determinant evaluation), its excitation
orders grow by at most the new reference's order, and the library accepts it."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1106_2456_gb300 import build as libbuild
from paper_1106_2456_gb300 import msd, reference, workloads as wl


def test_permutation_sign_matches_permutation_matrix_determinant():
    rng = np.random.default_rng(2)
    for n in (1, 2, 3, 5, 8):
        for _ in range(20):
            b = list(rng.permutation(20)[:n])
            perm = rng.permutation(n)
            a = [b[i] for i in perm]
            P = np.zeros((n, n))
            P[np.arange(n), perm] = 1.0
            assert reference.permutation_sign(a, b) == round(np.linalg.det(P))


def test_canonical_string_reproduces_in_place_columns():
    n = 4
    for holes in itertools.combinations(range(n), 2):
        for parts in itertools.combinations(range(3), 2):
            cols = reference.string_columns(n, holes, parts)
            h, p, sign = reference.canonical_string(n, cols)
            assert (h, p, sign) == (holes, parts, 1)
            # a column swap flips the sign only
            swapped = cols[:]
            swapped[0], swapped[3] = swapped[3], swapped[0]
            assert reference.canonical_string(n, swapped) == (holes, parts, -1)


def _problems():
    water = wl.make_workload("water", n_walkers=3)
    custom = wl.custom_workload((4, 3), (9, 8), 60, wl.uniform_orders(1, 3), W=3, n_nuc=3, seed=5)
    return [water, custom]


@pytest.mark.parametrize("which", [0, 1])
def test_switched_problem_is_the_same_wavefunction(which):
    w = _problems()[which]
    p = w.problem
    orc = oracle.Oracle(p)
    R = w.R0
    cur = orc.eval(R)
    terms = [reference.heaviest_term(p)] + [int(t) for t in np.random.default_rng(4).choice(p.n_det, 3)]
    for I in terms:
        q = reference.switch_reference(p, I)
        assert q.det_up[I] == 0 and q.det_dn[I] == 0
        assert q.exc_off[0][1] == 0 and q.exc_off[1][1] == 0   # string 0 is the reference
        o2 = oracle.Oracle(q)
        new = o2.eval(R)
        # Psi is a sum over the same determinants: equal up to rounding of the sum
        assert np.allclose(new["logabs"], cur["logabs"], rtol=0, atol=1e-11 * max(1.0, cur["absum"][:, 0].max()))
        assert np.array_equal(new["sign"], cur["sign"])
        for e in (0, p.n_tot - 1):
            a, b = orc.eval(R, e), o2.eval(R, e)
            assert np.allclose(a["grad"], b["grad"], rtol=1e-9, atol=1e-9 * a["absum"][:, 1:4].max())
            assert np.allclose(a["lap"], b["lap"], rtol=1e-9, atol=1e-9 * a["absum"][:, 4].max())


def test_orders_grow_by_at_most_the_new_reference_order():
    w = _problems()[1]
    p = w.problem
    I = reference.heaviest_term(p)
    q = reference.switch_reference(p, I)
    for s, u in ((0, int(p.det_up[I])), (1, int(p.det_dn[I]))):
        k_ref = int(p.exc_orders(s)[u])
        assert q.exc_orders(s).max() <= p.exc_orders(s).max() + k_ref
        # the old reference is now a string of exactly the new reference's order
        old_ref_new_index = int(q.det_up[0] if s == 0 else q.det_dn[0]) if (p.det_up[0], p.det_dn[0]) == (0, 0) else None
        if old_ref_new_index is not None:
            assert q.exc_orders(s)[old_ref_new_index] == k_ref


def test_switching_back_restores_the_problem():
    w = _problems()[0]
    p = w.problem
    I = reference.heaviest_term(p)
    q = reference.switch_reference(p, I)
    J = int(np.flatnonzero((p.det_up == 0) & (p.det_dn == 0))[0])  # the term of the old reference
    r = reference.switch_reference(q, J)
    # the occupied and virtual orbital sets come back (their order within a set may differ:
    # the column permutation's sign sits in the CI coefficients)
    for s in range(2):
        n = p.n_elec[s]
        for lo, hi in ((0, n), (n, p.n_orb[s])):
            a = {tuple(col) for col in p.B[s][:, lo:hi].T}
            b = {tuple(col) for col in r.B[s][:, lo:hi].T}
            assert a == b
    orc, o2 = oracle.Oracle(p), oracle.Oracle(r)
    assert np.allclose(orc.eval(w.R0)["logabs"], o2.eval(w.R0)["logabs"], rtol=0, atol=1e-12)


def test_library_accepts_the_switched_problem():
    libbuild.build()
    for w in _problems():
        q = reference.switch_reference(w.problem, reference.heaviest_term(w.problem))
        for prec in ("fp64", "mixed"):
            lay = msd.describe(q, prec)
            assert lay.shape[0] == 2


def test_order_limit_is_enforced():
    """Two order-5 strings with disjoint holes are 10 apart: beyond the library's 8."""
    n, N = 10, 20
    ref = ((), ())
    a = (tuple(range(5)), tuple(range(5)))
    b = (tuple(range(5, 10)), tuple(range(5, 10)))
    B = np.eye(N)
    p = wl.explicit_problem(np.zeros((1, 3)), [0] * N, [0] * N, np.linspace(0.5, 2.0, N), (B, B), (n, n),
                            [ref, a, b], [ref], [0, 1, 2], [0, 0, 0], [1.0, 0.5, 0.25])
    with pytest.raises(ValueError):
        reference.switch_reference(p, 1)


def test_heaviest_term_is_the_largest_non_reference_term():
    p = _problems()[1].problem
    I = reference.heaviest_term(p)
    assert not (p.det_up[I] == 0 and p.det_dn[I] == 0)
    others = [abs(p.ci[J]) for J in range(p.n_det) if not (p.det_up[J] == 0 and p.det_dn[J] == 0)]
    assert abs(p.ci[I]) == max(others)
