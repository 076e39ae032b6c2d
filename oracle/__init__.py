"""FP64 CPU oracle for the multi-determinant wavefunction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library
(``paper_1106_2456_gb300``): its arithmetic lives in ``msd_oracle.c`` (plain C, FP64),
built by ``oracle/build.py`` with gcc, and this module only marshals arrays.

Functions and the passages they follow:

* :meth:`Oracle.eval` -- Psi, grad_i Psi / Psi and lap_i Psi / Psi from every
  determinant formed explicitly (Section II: Psi = sum_k alpha_k det M_up,k det M_dn,k,
  M(i, j) = phi_j(r_i); Section IV-A: a derivative of a determinant with respect to
  electron i is the determinant with row i replaced by the derivative row).
* :meth:`Oracle.ratio` -- Psi(R') / Psi(R) from two full evaluations (Section II).
* :meth:`Oracle.dlogpsi` -- d log|Psi| / d c_I and d log|Psi| / d B by Jacobi's formula
  (the paper is silent on derivatives with respect to parameters).
* :func:`vmc_replay` -- Metropolis sweeps (Section II: a step moves one electron, a
  sweep moves each once), accept iff u < |Psi(R') / Psi(R)|^2 (no Jastrow factor).
* :func:`lu_logdet` -- determinant by LU with partial pivoting.
* :mod:`oracle.hamiltonian` -- the Pade-Jastrow factor, its ratio for a move, and the local
  energy of Psi_T = exp(J) Psi_MD (numpy, from the definitions; Section VI runs VMC on such
  a Jastrow-multideterminant wavefunction).

Pins (tests/test_oracle_pins.py): Leibniz determinants, LAPACK determinants, finite
differences of the basis, orbitals and Psi, the single-determinant reduction, the
single-excitation table identity, a Cauchy-Binet full-CI closed form, antisymmetry, and
the adjoint's linearity and homogeneity identities.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np

from .build import build_oracle, library_path

_lib = None


class _OrcProblem(ctypes.Structure):
    _fields_ = [
        ("n_elec", ctypes.c_int32 * 2),
        ("n_orb", ctypes.c_int32 * 2),
        ("n_nuc", ctypes.c_int32),
        ("nuc_xyz", ctypes.c_void_p),
        ("n_basis", ctypes.c_int32),
        ("bas_center", ctypes.c_void_p),
        ("bas_lm", ctypes.c_void_p),
        ("bas_alpha", ctypes.c_void_p),
        ("B", ctypes.c_void_p * 2),
        ("n_exc", ctypes.c_int32 * 2),
        ("exc_off", ctypes.c_void_p * 2),
        ("exc_holes", ctypes.c_void_p * 2),
        ("exc_parts", ctypes.c_void_p * 2),
        ("n_det", ctypes.c_int64),
        ("det_up", ctypes.c_void_p),
        ("det_dn", ctypes.c_void_p),
        ("ci", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        vp, i32 = ctypes.c_void_p, ctypes.c_int
        lib.orc_lu_logdet.argtypes = [i32, vp, vp, vp]
        lib.orc_basis.argtypes = [vp, vp, vp]
        lib.orc_orbitals.argtypes = [vp, i32, vp, vp]
        lib.orc_slater.argtypes = [vp, i32, vp, vp]
        lib.orc_eval.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
        lib.orc_eval.restype = i32
        lib.orc_eval_batch.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp, vp, vp]
        lib.orc_dlogpsi.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.orc_dlogpsi.restype = i32
        lib.orc_num_threads.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    return int(_load().orc_num_threads())


def lu_logdet(A: np.ndarray):
    """(log|det A|, sign) by the oracle's LU with partial pivoting."""
    lib = _load()
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    la = np.zeros(1)
    sg = np.zeros(1)
    lib.orc_lu_logdet(a.shape[0], _ptr(a), _ptr(la), _ptr(sg))
    return float(la[0]), float(sg[0])


class Oracle:
    """Plain FP64 evaluation of one problem (a ``workloads.Problem``)."""

    def __init__(self, problem):
        self.p = problem
        lib = _load()
        self._lib = lib
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            if a.size == 0:
                a = np.zeros(1, dtype=dt)
            keep.append(a)
            return _ptr(a)

        s = _OrcProblem()
        s.n_elec[0], s.n_elec[1] = problem.n_elec
        s.n_orb[0], s.n_orb[1] = problem.n_orb
        s.n_nuc = problem.nuc_xyz.shape[0]
        s.nuc_xyz = arr(problem.nuc_xyz, np.float64)
        s.n_basis = problem.n_basis
        s.bas_center = arr(problem.bas_center, np.int32)
        s.bas_lm = arr(problem.bas_lm, np.int8)
        s.bas_alpha = arr(problem.bas_alpha, np.float64)
        for k in range(2):
            s.B[k] = arr(problem.B[k], np.float64)
            s.n_exc[k] = problem.n_exc(k)
            s.exc_off[k] = arr(problem.exc_off[k], np.int32)
            s.exc_holes[k] = arr(problem.exc_holes[k], np.uint8)
            s.exc_parts[k] = arr(problem.exc_parts[k], np.uint8)
        s.n_det = problem.n_det
        s.det_up = arr(problem.det_up, np.int32)
        s.det_dn = arr(problem.det_dn, np.int32)
        s.ci = arr(problem.ci, np.float64)
        self._keep = keep
        self._s = s
        self._sp = ctypes.addressof(s)

    # -- single-point helpers ---------------------------------------------------------
    def basis(self, r) -> np.ndarray:
        out = np.zeros((5, self.p.n_basis))
        r = np.ascontiguousarray(r, np.float64)
        self._lib.orc_basis(self._sp, _ptr(r), _ptr(out))
        return out

    def orbitals(self, spin: int, r) -> np.ndarray:
        out = np.zeros((5, self.p.n_orb[spin]))
        r = np.ascontiguousarray(r, np.float64)
        self._lib.orc_orbitals(self._sp, spin, _ptr(r), _ptr(out))
        return out

    def slater(self, spin: int, R) -> np.ndarray:
        """Reference Slater matrix A_0[r, c] = phi_c(r_r) of one spin at configuration R [n_tot, 3]."""
        n = self.p.n_elec[spin]
        out = np.zeros((n, n))
        R = np.ascontiguousarray(R, np.float64)
        self._lib.orc_slater(self._sp, spin, _ptr(R), _ptr(out))
        return out

    def reference_condition(self, R, elec: Optional[int] = None, rnew=None) -> float:
        """Largest 2-norm condition number of the reference matrices of both spins at R and, for a
        move of electron elec to rnew, of the moved spin's reference matrix at R'.  Every quantity
        the table method forms passes through A_0^{-1}, so its rounding errors scale with this."""
        kap = max(np.linalg.cond(self.slater(s, R)) for s in range(2))
        if elec is not None and elec >= 0 and rnew is not None:
            R2 = np.array(R, dtype=np.float64, copy=True)
            R2[elec] = rnew
            kap = max(kap, np.linalg.cond(self.slater(self.p.spin_of(elec), R2)))
        return float(kap)

    # -- wavefunction -----------------------------------------------------------------
    def eval(self, R: np.ndarray, elec: int = -1, rnew: Optional[np.ndarray] = None) -> Dict[str, np.ndarray]:
        """Evaluate walkers R [W, n_tot, 3] (electron `elec` moved to rnew [W, 3] if given).

        Returns logabs [W], sign [W], and for elec >= 0 grad [W, 3] = grad_elec Psi / Psi,
        lap [W] = lap_elec Psi / Psi; absum [W, 5] = sum_I |c_I X_I| / |Psi| per channel.
        """
        R = np.ascontiguousarray(R, np.float64)
        if R.ndim == 2:
            R = R[None]
        W = R.shape[0]
        out = dict(logabs=np.zeros(W), sign=np.zeros(W), grad=np.zeros((W, 3)), lap=np.zeros(W),
                   absum=np.zeros((W, 5)))
        rn = None
        if rnew is not None:
            rn = np.ascontiguousarray(rnew, np.float64).reshape(W, 3)
        self._lib.orc_eval_batch(self._sp, W, _ptr(R), int(elec), _ptr(rn) if rn is not None else None,
                                 _ptr(out["logabs"]), _ptr(out["sign"]), _ptr(out["grad"]),
                                 _ptr(out["lap"]), _ptr(out["absum"]))
        return out

    def ratio(self, R: np.ndarray, elec: int, rnew: np.ndarray, cur: Optional[Dict] = None):
        """Psi(R') / Psi(R) by two full evaluations, plus grad/lap at R' and their scales."""
        if cur is None:
            cur = self.eval(R)
        new = self.eval(R, elec, rnew)
        ratio = new["sign"] * cur["sign"] * np.exp(new["logabs"] - cur["logabs"])
        return ratio, new

    def dlogpsi(self, R: np.ndarray, with_scale: bool = False):
        """d log|Psi| / d c [n_det] and d log|Psi| / d B_s [n_basis, n_orb] per spin, one walker.

        with_scale=True also returns the per-entry cancellation scale of each d/dB_s (the sum of
        the absolute values of the terms of Jacobi's formula that form it)."""
        R = np.ascontiguousarray(R, np.float64).reshape(self.p.n_tot, 3)
        dci = np.zeros(self.p.n_det)
        dB0 = np.zeros((self.p.n_basis, self.p.n_orb[0]))
        dB1 = np.zeros((self.p.n_basis, self.p.n_orb[1]))
        s0 = np.zeros_like(dB0) if with_scale else None
        s1 = np.zeros_like(dB1) if with_scale else None
        rc = self._lib.orc_dlogpsi(self._sp, _ptr(R), _ptr(dci), _ptr(dB0), _ptr(dB1),
                                   _ptr(s0) if with_scale else None, _ptr(s1) if with_scale else None)
        if rc:
            raise FloatingPointError("Psi is exactly zero at this configuration")
        if with_scale:
            return dci, (dB0, dB1), (s0, s1)
        return dci, (dB0, dB1)


def vmc_replay(oracle: Oracle, R0: np.ndarray, eta: np.ndarray, u: np.ndarray, tau: float,
               n_steps: Optional[int] = None, jastrow: Optional[Dict] = None):
    """Metropolis trajectory: step t moves electron t mod n_tot (up electrons first).

    r' = r + tau * eta[t]; accept iff u[t] < |Psi(R') / Psi(R)|^2, with Psi multiplied by
    exp(J) when `jastrow` = dict(Z=..., b_ee=..., b_en=...) is given (``oracle.hamiltonian``).
    Returns per-step records (elec, rnew, ratio, grad, lap, absum, accept) and the final
    positions; `ratio` is that of Psi_MD alone, `ratio_T` that of the tested wavefunction.
    """
    from . import hamiltonian

    p = oracle.p
    R = np.array(R0, dtype=np.float64, copy=True)
    W = R.shape[0]
    cur = oracle.eval(R)
    steps = eta.shape[0] if n_steps is None else n_steps
    recs = []
    for t in range(steps):
        e = t % p.n_tot
        rnew = R[:, e, :] + tau * eta[t]
        ratio, new = oracle.ratio(R, e, rnew, cur)
        ratio_T = ratio
        if jastrow is not None:
            ratio_T = ratio * hamiltonian.jastrow_ratio(R, p.n_elec[0], e, rnew, p.nuc_xyz, np.asarray(jastrow["Z"]),
                                                        jastrow.get("b_ee", 0.0), jastrow.get("b_en", 0.0))
        acc = u[t] < ratio_T * ratio_T
        recs.append(dict(elec=e, rnew=rnew.copy(), ratio=ratio, ratio_T=ratio_T, grad=new["grad"].copy(),
                         lap=new["lap"].copy(), absum=new["absum"].copy(), accept=acc.copy(),
                         logabs_new=new["logabs"].copy()))
        R[acc, e, :] = rnew[acc]
        cur = dict(logabs=np.where(acc, new["logabs"], cur["logabs"]),
                   sign=np.where(acc, new["sign"], cur["sign"]))
    return recs, R
