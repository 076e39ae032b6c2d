"""Jastrow factor and local energy, plain FP64 -- TEST INFRASTRUCTURE ONLY (oracle).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
this module.  It shares no code with the CUDA library: every quantity is written out from
its definition with numpy, one walker and one pair at a time, and the determinant part comes
from the determinant-by-determinant evaluation of ``oracle.Oracle``.

Definitions (Hartree atomic units, clamped nuclei; the paper runs VMC on a Jastrow times
its multideterminant expansion in Section VI and leaves the Jastrow to standard methods in
Section II):

* Psi_T = exp(J) Psi_MD with the two-body Pade Jastrow
  J = sum_{i<j} a_ij r_ij / (1 + b_ee r_ij) + sum_{i,I} (-Z_I) r_iI / (1 + b_en r_iI),
  a_ij = 1/2 (unlike spins) or 1/4 (like spins), the values Kato's cusp conditions fix;
  a parameter of 0 removes its term.
* E_L = -1/2 sum_i lap_i Psi_T / Psi_T + sum_{i<j} 1/r_ij - sum_{i,I} Z_I / r_iI
  + sum_{I<J} Z_I Z_J / R_IJ, where for Psi_T = exp(J) D
  lap_i Psi_T / Psi_T = lap_i D / D + lap_i J + |grad_i J|^2 + 2 grad_i J . grad_i D / D.

Pins (tests/test_oracle_hamiltonian.py): finite differences of J; the kinetic energy against
finite differences of log|Psi_T| from full determinant evaluations; a two-electron
single-Gaussian closed form; the cusp values of J; the water nuclear repulsion from its
bond geometry; invariance of J under exchange of like-spin electrons.
"""
from __future__ import annotations

from typing import Dict

import numpy as np


def _pair_coeff(i: int, j: int, n_up: int) -> float:
    """a_ij: 1/4 when electrons i and j have the same spin, else 1/2."""
    return 0.25 if (i < n_up) == (j < n_up) else 0.5


def jastrow(R: np.ndarray, n_up: int, nuc: np.ndarray, Z: np.ndarray, b_ee: float, b_en: float) -> float:
    """J of one walker R [n_tot, 3]."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    J = 0.0
    if b_ee > 0.0:
        for i in range(n):
            for j in range(i + 1, n):
                r = np.linalg.norm(R[i] - R[j])
                J += _pair_coeff(i, j, n_up) * r / (1.0 + b_ee * r)
    if b_en > 0.0:
        for i in range(n):
            for I in range(nuc.shape[0]):
                r = np.linalg.norm(R[i] - nuc[I])
                J += -Z[I] * r / (1.0 + b_en * r)
    return float(J)


def jastrow_derivatives(R: np.ndarray, n_up: int, nuc: np.ndarray, Z: np.ndarray, b_ee: float, b_en: float):
    """grad_i J [n_tot, 3] and lap_i J [n_tot] of one walker.

    For a radial term f(r) of r = |r_i - c|: grad_i f = f'(r) (r_i - c) / r and
    lap_i f = f''(r) + 2 f'(r) / r.  For f = a r / (1 + b r): f' = a / (1 + b r)^2 and
    f'' = -2 a b / (1 + b r)^3.
    """
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    g = np.zeros((n, 3))
    lap = np.zeros(n)

    def add(i, d, a, b):
        r = np.linalg.norm(d)
        f1 = a / (1.0 + b * r) ** 2
        f2 = -2.0 * a * b / (1.0 + b * r) ** 3
        g[i] += f1 * d / r
        lap[i] += f2 + 2.0 * f1 / r

    for i in range(n):
        if b_ee > 0.0:
            for j in range(n):
                if j != i:
                    add(i, R[i] - R[j], _pair_coeff(i, j, n_up), b_ee)
        if b_en > 0.0:
            for I in range(nuc.shape[0]):
                add(i, R[i] - nuc[I], -Z[I], b_en)
    return g, lap


def coulomb(R: np.ndarray, nuc: np.ndarray, Z: np.ndarray):
    """(V_ee, V_en, V_nn) of one walker."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    vee = sum(1.0 / np.linalg.norm(R[i] - R[j]) for i in range(n) for j in range(i + 1, n))
    ven = -sum(Z[I] / np.linalg.norm(R[i] - nuc[I]) for i in range(n) for I in range(nuc.shape[0]))
    vnn = sum(Z[I] * Z[K] / np.linalg.norm(nuc[I] - nuc[K])
              for I in range(nuc.shape[0]) for K in range(I + 1, nuc.shape[0]) if Z[I] * Z[K] != 0.0)
    return float(vee), float(ven), float(vnn)


def jastrow_ratio(R: np.ndarray, n_up: int, elec: int, rnew: np.ndarray, nuc, Z, b_ee: float, b_en: float) -> np.ndarray:
    """exp(J(R') - J(R)) per walker for electron elec moved to rnew [W, 3], from two full J."""
    R = np.asarray(R, np.float64)
    out = np.zeros(R.shape[0])
    for w in range(R.shape[0]):
        R2 = R[w].copy()
        R2[elec] = rnew[w]
        out[w] = np.exp(jastrow(R2, n_up, nuc, Z, b_ee, b_en) - jastrow(R[w], n_up, nuc, Z, b_ee, b_en))
    return out


def local_energy(orc, R: np.ndarray, Z, b_ee: float = 0.0, b_en: float = 0.0) -> Dict[str, np.ndarray]:
    """E_L [W] and parts [W, 4] = (kinetic, V_ee, V_en, V_nn) of walkers R [W, n_tot, 3].

    Also returns `scale` [W]: the size of the terms E_L is formed from, with the determinant
    part's gradient and laplacian measured by their CI cancellation scales (the oracle's
    absum), against which a tolerance is stated:
    1/2 sum_i (max(|lap_i D/D|, s_lap) + 2 sum_a |d_a J| max(|d_a D/D|, s_a)) + |V_ee| + |V_en| + |V_nn|.
    """
    p = orc.p
    R = np.ascontiguousarray(R, np.float64)
    if R.ndim == 2:
        R = R[None]
    W, n = R.shape[0], p.n_tot
    Z = np.asarray(Z, np.float64)
    nuc = p.nuc_xyz
    gD = np.zeros((W, n, 3))
    lD = np.zeros((W, n))
    ab = np.zeros((W, n, 5))
    for e in range(n):
        ev = orc.eval(R, e)
        gD[:, e] = ev["grad"]
        lD[:, e] = ev["lap"]
        ab[:, e] = ev["absum"]
    parts = np.zeros((W, 4))
    scale = np.zeros(W)
    for w in range(W):
        gJ, lJ = jastrow_derivatives(R[w], p.n_elec[0], nuc, Z, b_ee, b_en)
        lap_psi = lD[w] + lJ + np.sum(gJ * gJ, axis=1) + 2.0 * np.sum(gJ * gD[w], axis=1)
        vee, ven, vnn = coulomb(R[w], nuc, Z)
        parts[w] = (-0.5 * np.sum(lap_psi), vee, ven, vnn)
        s_l = np.maximum(np.abs(lD[w]), ab[w, :, 4])
        s_g = np.maximum(np.abs(gD[w]), ab[w, :, 1:4])
        scale[w] = 0.5 * np.sum(s_l + 2.0 * np.sum(np.abs(gJ) * s_g, axis=1)) + abs(vee) + abs(ven) + abs(vnn)
    return dict(eloc=parts.sum(axis=1), parts=parts, scale=scale)
