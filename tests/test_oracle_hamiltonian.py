"""Pins of the oracle's Jastrow factor and local energy (CPU only).

Each test checks ``oracle.hamiltonian`` against something other than itself: finite
differences, a closed form, a physical constraint (the cusp conditions) or geometry.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import hamiltonian as H
from paper_1106_2456_gb300 import workloads as wl


def _random_system(seed=3, n_up=3, n_dn=2):
    rng = np.random.default_rng(seed)
    nuc = rng.uniform(-1.5, 1.5, (2, 3))
    Z = np.array([2.0, 3.0])
    R = rng.uniform(-2.0, 2.0, (n_up + n_dn, 3))
    return R, n_up, nuc, Z


def test_jastrow_derivatives_match_finite_differences():
    R, n_up, nuc, Z = _random_system()
    b_ee, b_en = 0.8, 1.3
    g, lap = H.jastrow_derivatives(R, n_up, nuc, Z, b_ee, b_en)
    J0 = H.jastrow(R, n_up, nuc, Z, b_ee, b_en)
    h1, h2 = 1e-5, 1e-4
    for i in range(R.shape[0]):
        lap_fd = 0.0
        for a in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, a] += h1
            Rm[i, a] -= h1
            d1 = (H.jastrow(Rp, n_up, nuc, Z, b_ee, b_en) - H.jastrow(Rm, n_up, nuc, Z, b_ee, b_en)) / (2 * h1)
            assert abs(d1 - g[i, a]) < 1e-8 * max(1.0, abs(g[i, a]))
            Rp, Rm = R.copy(), R.copy()
            Rp[i, a] += h2
            Rm[i, a] -= h2
            lap_fd += (H.jastrow(Rp, n_up, nuc, Z, b_ee, b_en) - 2 * J0 + H.jastrow(Rm, n_up, nuc, Z, b_ee, b_en)) / h2**2
        assert abs(lap_fd - lap[i]) < 1e-5 * max(1.0, abs(lap[i]))


def test_cusp_conditions():
    """Kato: d<J>/dr at coalescence is 1/2 for unlike spins, 1/4 for like spins, -Z at a nucleus.
    The particles not involved sit 1e4 bohr away, so their terms change the slope by < 1e-8."""
    far = 1e4
    nuc = np.array([[0.0, 0.0, 0.0], [far, 0.0, 0.0]])
    Z = np.array([2.0, 1.0])
    base = np.array([[0.3, 0.4, -0.2], [0.3, 0.4, -0.2], [0.0, far, 0.0]])  # 2 up, 1 down
    n_up = 2
    d = np.array([0.6, -0.48, 0.64])
    delta = 1e-7

    def slope(i, j, b_ee, b_en):
        R0 = base.copy()
        R0[i] = R0[j]
        R1 = R0.copy()
        R1[i] = R0[j] + delta * d
        return (H.jastrow(R1, n_up, nuc, Z, b_ee, b_en) - H.jastrow(R0, n_up, nuc, Z, b_ee, b_en)) / delta

    assert abs(slope(0, 1, 1.0, 0.0) - 0.25) < 1e-6      # electrons 0 and 1: both up
    base[1] = (0.0, 0.0, far)
    assert abs(slope(2, 0, 1.0, 0.0) - 0.5) < 1e-6       # electrons 2 (down) and 0 (up)
    base[0] = (0.0, 0.0, -far)
    R0 = base.copy()
    R0[2] = nuc[0]
    R1 = R0.copy()
    R1[2] = nuc[0] + delta * d
    s = (H.jastrow(R1, n_up, nuc, Z, 0.0, 1.7) - H.jastrow(R0, n_up, nuc, Z, 0.0, 1.7)) / delta
    assert abs(s + Z[0]) < 1e-6


def test_jastrow_invariant_under_like_spin_exchange():
    R, n_up, nuc, Z = _random_system(5, 3, 3)
    J = H.jastrow(R, n_up, nuc, Z, 0.9, 1.1)
    for i, j in ((0, 2), (3, 5)):
        R2 = R.copy()
        R2[[i, j]] = R2[[j, i]]
        assert abs(H.jastrow(R2, n_up, nuc, Z, 0.9, 1.1) - J) < 1e-13 * max(1.0, abs(J))
    # exchanging an up and a down electron changes the pair coefficients, hence J
    R2 = R.copy()
    R2[[0, 4]] = R2[[4, 0]]
    assert abs(H.jastrow(R2, n_up, nuc, Z, 0.9, 1.1) - J) > 1e-6


def test_water_nuclear_repulsion_from_geometry():
    """V_nn of water, Z = (8, 1, 1), from the bond length 0.9572 A and angle 104.52 deg."""
    nuc = wl.water_nuclei()
    r_oh = 0.9572 * wl.BOHR_PER_ANGSTROM
    r_hh = 2.0 * r_oh * math.sin(math.radians(104.52) / 2.0)
    _, _, vnn = H.coulomb(np.full((1, 3), 5.0), nuc, np.array([8.0, 1.0, 1.0]))
    assert abs(vnn - (2 * 8.0 / r_oh + 1.0 / r_hh)) < 1e-12


def _two_electron_gaussian(alpha, Zc):
    """1 up + 1 down electron in the single s Gaussian exp(-alpha r^2) at one nucleus (charge Zc)."""
    nuc = np.zeros((1, 3))
    B = np.eye(2)  # orbital 0 = the s function, orbital 1 = a p_x function (an unused virtual)
    ref = [((), ())]
    return wl.explicit_problem(nuc, [0, 0], [0, 1], [alpha, alpha], (B, B), (1, 1), ref, ref, [0], [0], [1.0],
                               name="two-electron gaussian")


def test_two_electron_gaussian_closed_form():
    """Psi = g(r_1) g(r_2), g = exp(-alpha r^2): -1/2 lap g / g = 3 alpha - 2 alpha^2 r^2, so
    E_L = sum_i (3 alpha - 2 alpha^2 r_i^2 - Z / r_i) + 1 / r_12 (no Jastrow)."""
    alpha, Zc = 0.7, 2.0
    p = _two_electron_gaussian(alpha, Zc)
    orc = oracle.Oracle(p)
    rng = np.random.default_rng(11)
    R = rng.uniform(-1.2, 1.2, (4, 2, 3))
    out = H.local_energy(orc, R, [Zc])
    r = np.linalg.norm(R, axis=2)
    ref = np.sum(3 * alpha - 2 * alpha**2 * r**2 - Zc / r, axis=1) + 1.0 / np.linalg.norm(R[:, 0] - R[:, 1], axis=1)
    assert np.allclose(out["eloc"], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("b_ee,b_en", [(0.0, 0.0), (1.0, 1.5)])
def test_kinetic_energy_matches_finite_differences_of_log_psi(b_ee, b_en):
    """-1/2 sum_i lap_i Psi_T / Psi_T = -1/2 sum_i (lap_i log|Psi_T| + |grad_i log|Psi_T||^2), with
    log|Psi_T| = log|Psi_MD| (every determinant formed explicitly) + J, by central differences."""
    w = wl.make_workload("water", n_walkers=1)
    p = w.problem
    orc = oracle.Oracle(p)
    Z = np.array([8.0, 1.0, 1.0])
    R = w.R0[0]

    def logpsi(X):
        return float(orc.eval(X[None])["logabs"][0]) + H.jastrow(X, p.n_elec[0], p.nuc_xyz, Z, b_ee, b_en)

    f0 = logpsi(R)
    h = 2e-4  # O(h^2) truncation of the second differences: about 2e-4 Hartree here
    kin = 0.0
    for i in range(p.n_tot):
        for a in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, a] += h
            Rm[i, a] -= h
            fp, fm = logpsi(Rp), logpsi(Rm)
            d1 = (fp - fm) / (2 * h)
            d2 = (fp - 2 * f0 + fm) / h**2
            kin += -0.5 * (d2 + d1 * d1)
    out = H.local_energy(orc, R[None], Z, b_ee, b_en)
    # a dropped or mis-signed Jastrow term (cross term, |grad J|^2, lap J) moves it by > 2 Hartree
    assert abs(out["parts"][0, 0] - kin) < 2e-5 * max(1.0, abs(kin))
