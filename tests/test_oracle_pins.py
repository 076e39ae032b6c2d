"""Pins of the FP64 oracle against facts it does not compute itself.

Every check here compares the oracle with brute force, a library routine it does not
use, finite differences, a closed form, or an invariant -- never with a retyped copy
of its own formula.  A dropped term, a wrong sign or index, or a transposed operand in
``oracle/msd_oracle.c`` fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1106_2456_gb300 import workloads as wl

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------------------------
# determinants
# ---------------------------------------------------------------------------------

def leibniz_det(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1.0
        for i in range(n):
            prod *= A[i, perm[i]]
        tot += (-1) ** inv * prod
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_lu_matches_leibniz(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        A = rng.standard_normal((n, n))
        la, sg = oracle.lu_logdet(A)
        ref = leibniz_det(A)
        assert sg * math.exp(la) == pytest.approx(ref, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("n", [10, 37, 64])
def test_lu_matches_lapack(n):
    rng = np.random.default_rng(100 + n)
    A = rng.standard_normal((n, n))
    la, sg = oracle.lu_logdet(A)
    s_ref, l_ref = np.linalg.slogdet(A)
    assert sg == s_ref
    assert la == pytest.approx(l_ref, rel=1e-12)


def test_lu_singular_and_permutation():
    A = np.array([[1.0, 2.0], [2.0, 4.0]])
    la, sg = oracle.lu_logdet(A)
    assert sg == 0.0 and la == -np.inf
    # a permutation matrix: determinant is the permutation's sign
    P = np.eye(4)[[1, 0, 3, 2]]
    la, sg = oracle.lu_logdet(P)
    assert sg == 1.0 and la == pytest.approx(0.0, abs=1e-15)
    P = np.eye(3)[[1, 2, 0]]
    assert oracle.lu_logdet(P)[1] == 1.0
    P = np.eye(3)[[1, 0, 2]]
    assert oracle.lu_logdet(P)[1] == -1.0


# ---------------------------------------------------------------------------------
# basis and orbitals
# ---------------------------------------------------------------------------------

def _one_center_problem(alpha):
    nuc = np.array([[0.3, -0.2, 0.5]])
    B = (np.eye(4), np.eye(4))
    return wl.explicit_problem(nuc, [0, 0, 0, 0], [0, 1, 2, 3], [alpha] * 4, B, (1, 1),
                               [((), ())], [((), ())], [0], [0], [1.0])


def test_basis_special_values():
    al = 0.7
    o = oracle.Oracle(_one_center_problem(al))
    A = np.array([0.3, -0.2, 0.5])
    chi = o.basis(A)
    # at the centre: s = 1, p = 0, grad s = 0, grad p_c = e_c, lap s = -6 alpha
    assert chi[0] == pytest.approx([1.0, 0.0, 0.0, 0.0], abs=1e-15)
    assert chi[1:4, 0] == pytest.approx([0, 0, 0], abs=1e-15)
    assert chi[1:4, 1:4] == pytest.approx(np.eye(3), abs=1e-15)
    assert chi[4, 0] == pytest.approx(-6 * al)
    # one bohr along x: p_x = e^-alpha, p_y = p_z = 0
    chi = o.basis(A + np.array([1.0, 0, 0]))
    assert chi[0] == pytest.approx([math.exp(-al), math.exp(-al), 0.0, 0.0], abs=1e-15)


@pytest.mark.parametrize("al", [0.1, 1.3, 9.0])
def test_basis_finite_differences(al):
    o = oracle.Oracle(_one_center_problem(al))
    rng = np.random.default_rng(int(al * 10))
    h1, h2 = 1e-5, 1e-3
    for _ in range(4):
        r = np.array([0.3, -0.2, 0.5]) + rng.standard_normal(3) * 0.6
        chi = o.basis(r)
        lap_fd = np.zeros(4)
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1.0
            g_fd = (o.basis(r + h1 * e)[0] - o.basis(r - h1 * e)[0]) / (2 * h1)
            assert chi[1 + a] == pytest.approx(g_fd, rel=1e-7, abs=1e-9)
            lap_fd += (o.basis(r + h2 * e)[0] + o.basis(r - h2 * e)[0] - 2 * chi[0]) / h2 ** 2
        assert chi[4] == pytest.approx(lap_fd, rel=1e-4, abs=1e-5)


def test_orbitals_linear_in_basis_and_fd():
    w = wl.make_workload("water", n_walkers=2)
    o = oracle.Oracle(w.problem)
    r = w.R0[0, 0]
    phi = o.orbitals(0, r)
    chi = o.basis(r)
    # orbitals are the basis contracted with B (checked with numpy's matmul)
    assert phi == pytest.approx(chi @ w.problem.B[0], rel=1e-13, abs=1e-14)
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        g = (o.orbitals(0, r + e)[0] - o.orbitals(0, r - e)[0]) / (2 * h)
        assert phi[1 + a] == pytest.approx(g, rel=1e-6, abs=1e-8)


# ---------------------------------------------------------------------------------
# wavefunction pins
# ---------------------------------------------------------------------------------

def _slater(o, spin, R, n_up, n):
    off = 0 if spin == 0 else n_up
    return np.stack([o.orbitals(spin, R[off + r]) for r in range(n)], axis=1)  # [5, n, N]


def test_single_determinant_reduction():
    """n_det = 1: Psi = det M_up,0 det M_dn,0; the ratio is 1 + u^T M^-1 e_i (Section III)."""
    w = wl.make_workload("water", n_walkers=3)
    p = w.problem
    single = wl.explicit_problem(p.nuc_xyz, p.bas_center, p.bas_lm, p.bas_alpha, p.B, p.n_elec,
                                 [((), ())], [((), ())], [0], [0], [1.0])
    o = oracle.Oracle(single)
    n = p.n_elec[0]
    for wk in range(3):
        R = w.R0[wk]
        res = o.eval(R)
        Mu = _slater(o, 0, R, n, n)[0][:, :n]
        Md = _slater(o, 1, R, n, n)[0][:, :n]
        s1, l1 = np.linalg.slogdet(Mu)
        s2, l2 = np.linalg.slogdet(Md)
        assert res["logabs"][0] == pytest.approx(l1 + l2, rel=1e-12)
        assert res["sign"][0] == s1 * s2
        # move electron 2 (spin up): Sherman-Morrison denominator
        i = 2
        rn = R[i] + np.array([0.2, -0.1, 0.3])
        u = o.orbitals(0, rn)[0][:n] - Mu[i]
        sm = 1.0 + u @ np.linalg.inv(Mu)[:, i]
        ratio, new = o.ratio(R[None], i, rn[None])
        assert ratio[0] == pytest.approx(sm, rel=1e-11)
        # single-determinant gradient and laplacian: sum_c d^a phi_c(r_i) M^-1[c, i]
        Mn = Mu.copy()
        Mn[i] = o.orbitals(0, rn)[0][:n]
        d = o.orbitals(0, rn)[:, :n]
        x = np.linalg.inv(Mn)[:, i]
        assert new["grad"][0] == pytest.approx(d[1:4] @ x, rel=1e-10)
        assert new["lap"][0] == pytest.approx(d[4] @ x, rel=1e-10)


def _excitation_table(o, p, R, spin):
    n = p.n_elec[spin]
    M = _slater(o, spin, R, p.n_elec[0], n)[0]  # [n, N]
    A0 = M[:, :n]
    Phiv = M[:, n:]
    return np.linalg.solve(A0, Phiv)  # T[c, a] = (A0^-1 Phi_v)[c, a]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_excitation_is_small_det_of_table(k):
    """det A_u / det A_0 = det T[h_q, p_l] (Section III: singles read off T, r-fold = r x r det)."""
    w = wl.make_workload("water", n_walkers=2)
    p = w.problem
    n, m = p.n_elec[0], p.n_orb[0] - p.n_elec[0]
    rng = np.random.default_rng(k)
    strings = [((), ())]
    for _ in range(6):
        h = tuple(sorted(rng.choice(n, k, replace=False).tolist()))
        q = tuple(sorted(rng.choice(m, k, replace=False).tolist()))
        strings.append((h, q))
    # one term per up string, down fixed at the reference, c = 1: Psi_j = det A_up,j det A_dn,0
    o_ref = oracle.Oracle(wl.explicit_problem(p.nuc_xyz, p.bas_center, p.bas_lm, p.bas_alpha, p.B,
                                              p.n_elec, [((), ())], [((), ())], [0], [0], [1.0]))
    R = w.R0[0]
    base = o_ref.eval(R)
    T = _excitation_table(o_ref, p, R, 0)
    for h, q in strings[1:]:
        pr = wl.explicit_problem(p.nuc_xyz, p.bas_center, p.bas_lm, p.bas_alpha, p.B, p.n_elec,
                                 [((), ()), (h, q)], [((), ())], [1], [0], [1.0])
        ex = oracle.Oracle(pr).eval(R)
        t = ex["sign"][0] * base["sign"][0] * math.exp(ex["logabs"][0] - base["logabs"][0])
        sub = T[np.ix_(list(h), list(q))]
        assert t == pytest.approx(np.linalg.det(sub), rel=1e-9, abs=1e-12)


def _cauchy_binet_problem(seed=3, n=(2, 3), N=(5, 6)):
    """Full CI with c_(u,d) = det Q_up[cols(u)] det Q_dn[cols(d)]: Psi = det(Phi_up Q_up) det(Phi_dn Q_dn)."""
    rng = np.random.default_rng(seed)
    nuc = wl.chain_nuclei(rng, 3)
    bc, blm, bal = wl.gaussian_basis(rng, 3)
    nb = bal.shape[0]
    B = (rng.standard_normal((nb, N[0])) / math.sqrt(nb), rng.standard_normal((nb, N[1])) / math.sqrt(nb))
    Q = (rng.standard_normal((N[0], n[0])), rng.standard_normal((N[1], n[1])))
    strs = [wl.full_ci_strings(n[s], N[s]) for s in range(2)]

    def cols(s, hp):
        c = list(range(n[s]))
        for hq, pq in zip(*hp):
            c[hq] = n[s] + pq
        return c

    cq = [[np.linalg.det(Q[s][cols(s, hp), :]) for hp in strs[s]] for s in range(2)]
    du, dd, ci = [], [], []
    for a in range(len(strs[0])):
        for b in range(len(strs[1])):
            du.append(a)
            dd.append(b)
            ci.append(cq[0][a] * cq[1][b])
    prob = wl.explicit_problem(nuc, bc, blm, bal, B, n, strs[0], strs[1], du, dd, ci, name="cauchy-binet")
    R = nuc[np.arange(n[0] + n[1]) % 3] + rng.standard_normal((n[0] + n[1], 3))
    return prob, Q, R


def test_cauchy_binet_full_ci_closed_form():
    prob, Q, R = _cauchy_binet_problem()
    o = oracle.Oracle(prob)
    n = prob.n_elec

    def rotated(spin, RR):
        off = 0 if spin == 0 else n[0]
        return np.stack([o.orbitals(spin, RR[off + r]) @ Q[spin] for r in range(n[spin])], axis=1)  # [5, n, n]

    res = o.eval(R)
    Pu, Pd = rotated(0, R)[0], rotated(1, R)[0]
    s1, l1 = np.linalg.slogdet(Pu)
    s2, l2 = np.linalg.slogdet(Pd)
    assert res["logabs"][0] == pytest.approx(l1 + l2, rel=1e-10, abs=1e-10)
    assert res["sign"][0] == s1 * s2
    # moves of an up and a down electron: ratio, grad, lap of a single rotated determinant
    for e in (1, n[0] + 2):
        spin = 0 if e < n[0] else 1
        i = e if spin == 0 else e - n[0]
        rn = R[e] + np.array([0.15, -0.25, 0.1])
        ratio, new = o.ratio(R[None], e, rn[None])
        R2 = R.copy()
        R2[e] = rn
        P_old = rotated(spin, R)[0]
        P_new_all = rotated(spin, R2)
        P_new = P_new_all[0]
        assert ratio[0] == pytest.approx(np.linalg.det(P_new) / np.linalg.det(P_old), rel=1e-9)
        x = np.linalg.inv(P_new)[:, i]
        assert new["grad"][0] == pytest.approx(P_new_all[1:4, i, :] @ x, rel=1e-8, abs=1e-10)
        assert new["lap"][0] == pytest.approx(P_new_all[4, i, :] @ x, rel=1e-8, abs=1e-10)


def test_antisymmetry_under_same_spin_swap():
    w = wl.make_workload("water", n_walkers=2)
    o = oracle.Oracle(w.problem)
    R = w.R0[0]
    base = o.eval(R)
    n_up = w.problem.n_elec[0]
    for a, b in [(0, 3), (n_up + 1, n_up + 4)]:
        R2 = R.copy()
        R2[[a, b]] = R2[[b, a]]
        sw = o.eval(R2)
        assert sw["logabs"][0] == pytest.approx(base["logabs"][0], rel=1e-12)
        assert sw["sign"][0] == -base["sign"][0]


def test_grad_lap_finite_differences():
    w = wl.make_workload("water", n_walkers=2)
    o = oracle.Oracle(w.problem)
    R = w.R0[1]
    for e in (0, 7):
        res = o.eval(R, e)
        cur = o.eval(R)
        h1, h2 = 1e-5, 1e-3
        g_fd = np.zeros(3)
        lap_fd = 0.0
        for a in range(3):
            d = np.zeros(3)
            d[a] = 1.0
            rp, _ = o.ratio(R[None], e, (R[e] + h1 * d)[None], cur)
            rm, _ = o.ratio(R[None], e, (R[e] - h1 * d)[None], cur)
            g_fd[a] = (rp[0] - rm[0]) / (2 * h1)
            rp, _ = o.ratio(R[None], e, (R[e] + h2 * d)[None], cur)
            rm, _ = o.ratio(R[None], e, (R[e] - h2 * d)[None], cur)
            lap_fd += (rp[0] + rm[0] - 2.0) / h2 ** 2
        assert res["grad"][0] == pytest.approx(g_fd, rel=1e-6, abs=1e-7)
        assert res["lap"][0] == pytest.approx(lap_fd, rel=1e-4, abs=1e-4)


def test_ratio_of_trajectory_matches_fresh_evaluation():
    w = wl.make_workload("water", n_walkers=4)
    o = oracle.Oracle(w.problem)
    eta, u = w.proposals(12)
    recs, R = oracle.vmc_replay(o, w.R0, eta, u, w.tau)
    # product of accepted ratios equals Psi(R_final) / Psi(R_0)
    prod = np.ones(4)
    for r in recs:
        prod = np.where(r["accept"], prod * r["ratio"], prod)
    a, b = o.eval(w.R0), o.eval(R)
    assert prod == pytest.approx(b["sign"] * a["sign"] * np.exp(b["logabs"] - a["logabs"]), rel=1e-9)
    assert 0 < sum(int(r["accept"].sum()) for r in recs) < 48


# ---------------------------------------------------------------------------------
# parameter derivatives
# ---------------------------------------------------------------------------------

def test_adjoint_invariants_and_fd():
    w = wl.make_workload("water", n_walkers=1, n_det=40)
    p = w.problem
    o = oracle.Oracle(p)
    R = w.R0[0]
    dci, dB = o.dlogpsi(R)
    # Psi is linear in c: sum_I c_I dlog|Psi|/dc_I = 1
    assert float(np.dot(p.ci, dci)) == pytest.approx(1.0, rel=1e-11)
    # Psi_s is homogeneous of degree n_s in B_s
    assert float(np.sum(p.B[0] * dB[0]) + np.sum(p.B[1] * dB[1])) == pytest.approx(sum(p.n_elec), rel=1e-10)
    # central differences in a few c_I and B entries
    h = 1e-6
    rng = np.random.default_rng(5)
    base_ci = p.ci.copy()
    for I in rng.choice(p.n_det, 4, replace=False):
        cp = base_ci.copy(); cp[I] += h
        cm = base_ci.copy(); cm[I] -= h
        fp = oracle.Oracle(wl.dataclasses.replace(p, ci=cp)).eval(R)["logabs"][0]
        fm = oracle.Oracle(wl.dataclasses.replace(p, ci=cm)).eval(R)["logabs"][0]
        assert dci[I] == pytest.approx((fp - fm) / (2 * h), rel=1e-5, abs=1e-8)
    for s in range(2):
        for _ in range(3):
            mu = int(rng.integers(p.n_basis))
            j = int(rng.integers(p.n_orb[s]))
            Bp = [p.B[0].copy(), p.B[1].copy()]
            Bm = [p.B[0].copy(), p.B[1].copy()]
            Bp[s][mu, j] += h
            Bm[s][mu, j] -= h
            fp = oracle.Oracle(wl.dataclasses.replace(p, B=tuple(Bp))).eval(R)["logabs"][0]
            fm = oracle.Oracle(wl.dataclasses.replace(p, B=tuple(Bm))).eval(R)["logabs"][0]
            assert dB[s][mu, j] == pytest.approx((fp - fm) / (2 * h), rel=1e-5, abs=1e-8)


# ---------------------------------------------------------------------------------
# reference Slater matrices and their condition number (the kappa of every parity bar)
# ---------------------------------------------------------------------------------

def _known_condition_problem(R, targets, seed=5):
    """A problem whose reference Slater matrix of spin s at R is exactly targets[s].

    A_0 = X_s B_s with X_s[r, mu] = chi_mu(r_r) (the basis at the spin's electrons, from the
    oracle's basis evaluator, pinned above), so B_s = pinv(X_s) targets[s] reproduces any
    n_s x n_s target while n_s <= n_basis.
    """
    rng = np.random.default_rng(seed)
    nuc = wl.chain_nuclei(rng, 3)
    bc, blm, bal = wl.gaussian_basis(rng, 3)
    n = (targets[0].shape[0], targets[1].shape[0])
    probe = wl.explicit_problem(nuc, bc, blm, bal, (np.eye(len(bc))[:, :n[0]], np.eye(len(bc))[:, :n[1]]), n,
                                [((), ())], [((), ())], [0], [0], [1.0])
    o = oracle.Oracle(probe)
    B = []
    for s in range(2):
        off = 0 if s == 0 else n[0]
        X = np.stack([o.basis(R[off + r])[0] for r in range(n[s])])  # [n_s, n_basis]
        B.append(np.linalg.pinv(X) @ targets[s])
    return wl.explicit_problem(nuc, bc, blm, bal, tuple(B), n, [((), ())], [((), ())], [0], [0], [1.0])


def _matrix_with_condition(rng, n, kappa):
    """Q diag(s) V^T with singular values log-spaced from 1 to 1/kappa: 2-norm condition kappa."""
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(np.logspace(0.0, -np.log10(kappa), n)) @ V.T


def test_slater_and_reference_condition_known_kappa():
    """Oracle.slater rebuilds a chosen matrix per spin (a wrong down-spin row offset or a
    transposed A_0 fails), and reference_condition returns the 2-norm condition number of the
    worse spin, known here by construction, and of the moved spin's matrix at R'."""
    rng = np.random.default_rng(17)
    n_up, n_dn = 4, 3
    R = rng.standard_normal((n_up + n_dn, 3)) * 1.2
    targets = (_matrix_with_condition(rng, n_up, 40.0), _matrix_with_condition(rng, n_dn, 900.0))
    p = _known_condition_problem(R, targets)
    o = oracle.Oracle(p)
    for s in range(2):
        A = o.slater(s, R)
        assert np.allclose(A, targets[s], rtol=0, atol=1e-9 * np.abs(targets[s]).max())
        # rows are electrons: a transposed or row-shifted matrix differs from the target
        assert not np.allclose(A.T, targets[s], atol=1e-6)
    kap = o.reference_condition(R)
    assert kap == pytest.approx(900.0, rel=1e-6)
    # swap the roles: the up spin ill-conditioned, the down spin not
    targets2 = (_matrix_with_condition(rng, n_up, 2.5e4), _matrix_with_condition(rng, n_dn, 3.0))
    o2 = oracle.Oracle(_known_condition_problem(R, targets2))
    assert o2.reference_condition(R) == pytest.approx(2.5e4, rel=1e-6)
    # moved electron: the moved spin's matrix at R' is A_0 with the electron's row replaced by
    # the orbitals at r', built here from the orbital evaluator row by row
    e = 5  # second down electron, row 1 of the down matrix
    rnew = R[e] + np.array([0.3, -0.2, 0.1])
    R2 = R.copy()
    R2[e] = rnew
    row = np.stack([o.orbitals(1, R2[n_up + r])[0][:n_dn] for r in range(n_dn)])
    want = max(40.0, 900.0, np.linalg.cond(row))
    assert o.reference_condition(R, e, rnew) == pytest.approx(want, rel=1e-9)
    # an up-electron move is judged on the up matrix at R' (the down one is unchanged)
    R3 = R.copy()
    R3[1] = R[1] + np.array([-0.4, 0.2, 0.5])
    rowu = np.stack([o.orbitals(0, R3[r])[0][:n_up] for r in range(n_up)])
    assert o.reference_condition(R, 1, R3[1]) == pytest.approx(max(900.0, np.linalg.cond(rowu)), rel=1e-9)


@pytest.mark.parametrize("label", ["water", "medium"])
def test_slater_matches_orbital_rows_and_determinant(label):
    """On the generated workloads: Oracle.slater(s, R) stacks the occupied orbitals of the
    spin's own electrons (down electrons start at n_up), and det A_up det A_dn equals the
    single-determinant Psi that the oracle's LU evaluation gives independently."""
    w = wl.make_workload(label, n_walkers=2)
    p = w.problem
    single = wl.explicit_problem(p.nuc_xyz, p.bas_center, p.bas_lm, p.bas_alpha, p.B, p.n_elec,
                                 [((), ())], [((), ())], [0], [0], [1.0])
    o = oracle.Oracle(single)
    R = w.R0[1]
    logs = 0.0
    sign = 1.0
    for s in range(2):
        n = p.n_elec[s]
        off = 0 if s == 0 else p.n_elec[0]
        A = o.slater(s, R)
        rows = np.stack([o.orbitals(s, R[off + r])[0][:n] for r in range(n)])
        assert np.array_equal(A, rows)
        sg, ld = np.linalg.slogdet(A)
        logs += ld
        sign *= sg
        assert o.reference_condition(R) >= np.linalg.cond(A) * (1 - 1e-12)
    ev = o.eval(R)
    assert ev["logabs"][0] == pytest.approx(logs, rel=1e-11, abs=1e-11)
    assert ev["sign"][0] == sign


def test_adjoint_cancellation_scale():
    """The per-entry scale the adjoint parity bars use: it bounds |d log|Psi| / dB| entry by entry
    (triangle inequality) and, for a single determinant, is sum_r |chi_mu(r_r)| |A_0^{-1}[j, r]|
    (Jacobi: d log|det A_0| / dA_0[r, j] = A_0^{-1}[j, r]; zero on the virtual orbitals)."""
    w = wl.make_workload("water", n_walkers=1, n_det=40)
    p = w.problem
    R = w.R0[0]
    dci, dB, sc = oracle.Oracle(p).dlogpsi(R, with_scale=True)
    for s in range(2):
        assert np.all(sc[s] >= np.abs(dB[s]) * (1 - 1e-12))
        assert np.all(sc[s] > 0)
    single = wl.explicit_problem(p.nuc_xyz, p.bas_center, p.bas_lm, p.bas_alpha, p.B, p.n_elec,
                                 [((), ())], [((), ())], [0], [0], [-2.0])
    o = oracle.Oracle(single)
    _, dB1, sc1 = o.dlogpsi(R, with_scale=True)
    for s in range(2):
        n = p.n_elec[s]
        off = 0 if s == 0 else p.n_elec[0]
        X = np.stack([o.basis(R[off + r])[0] for r in range(n)])  # [n, n_basis]
        Ainv = np.linalg.inv(o.slater(s, R))                       # [j, r]
        want = np.zeros_like(sc1[s])
        want[:, :n] = np.abs(X).T @ np.abs(Ainv).T
        assert np.allclose(sc1[s], want, rtol=1e-10, atol=1e-14)
        # and the value itself: sum_r chi_mu(r_r) A_0^{-1}[j, r]
        val = np.zeros_like(dB1[s])
        val[:, :n] = X.T @ Ainv.T
        assert np.allclose(dB1[s], val, rtol=1e-9, atol=1e-12)
