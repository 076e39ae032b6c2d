"""Thin Python binding of libmsd (C ABI in ``include/msd.h``).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``libmsd.so``.  PyTorch provides device memory and the stream; tensors are passed to
the library as raw device pointers.  Importing this module loads the library and
raises if it has not been built; creating an :class:`MSD` raises without a GPU --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Tuple

import numpy as np
import torch

from .build import INCLUDE, library_path

MSD_FP64, MSD_MIXED, MSD_CANONICAL = 0, 1, 2
_STATUS = {0: "MSD_OK", 1: "MSD_ERR_ARG", 2: "MSD_ERR_CUDA", 3: "MSD_ERR_OOM", 4: "MSD_ERR_SINGULAR",
           5: "MSD_ERR_TIMEOUT", 6: "MSD_ERR_STATE"}
NCH = 5


class MSDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class _Problem(ctypes.Structure):
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
        ("n_walkers", ctypes.c_int32),
        ("prec", ctypes.c_int32),
        ("refresh_K", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
    ]


def header_functions():
    """Names of the functions declared in include/msd.h."""
    with open(os.path.join(INCLUDE, "msd.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msd_[a-z_0-9]+)\s*\(", src)))


_lib = None


class Jastrow(ctypes.Structure):
    """``msd_jastrow``: Pade parameters of the electron-electron and electron-nucleus terms
    (0 removes a term)."""
    _fields_ = [("b_ee", ctypes.c_double), ("b_en", ctypes.c_double)]


def load_library():
    """Load libmsd.so (built by ``paper_1106_2456_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libmsd is not built ({path}); run paper_1106_2456_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "msd_init": ([vp, i32, vp], i32),
        "msd_describe": ([vp, vp], i32),
        "msd_describe_records": ([vp, i32, vp, i64, vp, vp], i32),
        "msd_set_positions": ([vp, vp], i32),
        "msd_ratio": ([vp, i32, vp, vp, vp, vp], i32),
        "msd_accept": ([vp, i32, vp], i32),
        "msd_ratio_noalloc": ([vp, i32, vp, vp, vp, vp], i32),
        "msd_backward": ([vp, vp, vp, vp], i32),
        "msd_set_params": ([vp, vp, vp, vp], i32),
        "msd_grad_lap": ([vp, i32, vp, vp], i32),
        "msd_eval_batch": ([vp, vp, vp, vp, vp, vp], i32),
        "msd_get_state": ([vp, vp, vp, vp], i32),
        "msd_propose": ([vp, i32, vp, d, vp], i32),
        "msd_metropolis": ([vp, vp, vp, vp], i32),
        "msd_ratio_host": ([vp, i32, vp, vp, vp, vp], i32),
        "msd_accept_host": ([vp, i32, vp], i32),
        "msd_set_stream": ([vp, vp], i32),
        "msd_sync": ([vp], i32),
        "msd_last_error": ([vp], ctypes.c_char_p),
        "msd_exc_histogram": ([vp, i32, vp], i32),
        "msd_copy_state": ([vp, i32, i32, vp, vp], i32),
        "msd_timing_start": ([vp], i32),
        "msd_timing_stop": ([vp, vp, vp, vp], i32),
        "msd_timing_counts": ([vp, vp], i32),
        "msd_orbitals": ([vp, i32, i32, i32, vp, vp], i32),
        "msd_selftest_wait": ([vp, ctypes.c_int64], i32),
        "msd_set_rescue": ([vp, i32, ctypes.c_double, ctypes.c_double], i32),
        "msd_rescue_stats": ([vp, vp], i32),
        "msd_step": ([vp, i32, vp, ctypes.c_double, vp, vp, vp, vp, vp], i32),
        "msd_set_hamiltonian": ([vp, vp, vp], i32),
        "msd_jastrow_ratio": ([vp, i32, vp, vp], i32),
        "msd_local_energy": ([vp, vp, vp], i32),
        "msd_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _dptr(t: Optional[torch.Tensor], dtype: torch.dtype, shape=None, name: str = "") -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


def problem_struct(problem, n_walkers: int, precision: str, refresh_K: int = 1 << 30, stream_handle=None):
    """The msd_problem struct of a workloads.Problem, and the arrays it points into (keep them alive)."""
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(x, dtype=dt)
        if a.size == 0:
            a = np.zeros(1, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    s = _Problem()
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
    s.n_walkers = int(n_walkers)
    s.prec = {"fp64": MSD_FP64, "mixed": MSD_MIXED, "canonical": MSD_CANONICAL}[precision]
    s.refresh_K = int(min(refresh_K, 2 ** 31 - 1))
    s.cuda_stream = stream_handle
    return s, keep


def describe(problem, precision: str = "mixed") -> np.ndarray:
    """msd_describe: the device layout msd_init builds, [2 spins][16] (no GPU needed)."""
    lib = load_library()
    s, keep = problem_struct(problem, 1, precision)
    out = np.zeros(32, dtype=np.int64)
    rc = lib.msd_describe(ctypes.byref(s), out.ctypes.data)
    if rc != 0:
        raise MSDError(rc, lib.msd_last_error(None).decode())
    return out.reshape(2, 16)


class MSD:
    """One libmsd context: a multi-determinant wavefunction and W walkers on the current GPU."""

    def __init__(self, problem, n_walkers: int, precision: str = "fp64", refresh_K: int = 1 << 30,
                 stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise MSDError(2, "a CUDA GPU is required (libmsd has no CPU path)")
        self.lib = load_library()
        self.p = problem
        self.W = int(n_walkers)
        self.n_tot = problem.n_tot
        self.mixed = precision == "mixed"
        if precision not in ("fp64", "mixed", "canonical"):
            raise ValueError("precision must be 'fp64', 'mixed' or 'canonical' (FP64, per-determinant inverses)")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        s, self._keep = problem_struct(problem, self.W, precision, refresh_K, self.stream.cuda_stream)
        ctx = ctypes.c_void_p()
        rc = self.lib.msd_init(ctypes.byref(s), 1, ctypes.byref(ctx))
        if rc != 0:
            raise MSDError(rc, self.lib.msd_last_error(None).decode())
        self.ctx = ctx
        self.dev = torch.device("cuda", torch.cuda.current_device())

    # -- helpers -----------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise MSDError(rc, self.lib.msd_last_error(self.ctx).decode())

    def _empty(self, *shape, dtype=torch.float64):
        return torch.empty(shape, dtype=dtype, device=self.dev)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.msd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points --------------------------------------------------------------------
    def set_positions(self, R: torch.Tensor):
        self._check(self.lib.msd_set_positions(self.ctx, _dptr(R, torch.float64, (self.W, self.n_tot, 3), "R")))

    def ratio_into(self, elec: int, rnew: torch.Tensor, ratio: torch.Tensor, grad: Optional[torch.Tensor] = None,
                   lap: Optional[torch.Tensor] = None):
        W = self.W
        self._check(self.lib.msd_ratio(self.ctx, int(elec), _dptr(rnew, torch.float64, (W, 3), "rnew"),
                                       _dptr(ratio, torch.float64, (W,), "ratio"),
                                       _dptr(grad, torch.float64, (W, 3), "grad"),
                                       _dptr(lap, torch.float64, (W,), "lap")))

    def ratio_noalloc_into(self, elec: int, rnew: torch.Tensor, ratio: torch.Tensor,
                           grad: Optional[torch.Tensor] = None, lap: Optional[torch.Tensor] = None):
        """msd_ratio_noalloc: ratio (and grad/lap) at rnew with no device allocation and no
        proposal kept; a pending msd_ratio proposal stays valid."""
        W = self.W
        self._check(self.lib.msd_ratio_noalloc(self.ctx, int(elec), _dptr(rnew, torch.float64, (W, 3), "rnew"),
                                               _dptr(ratio, torch.float64, (W,), "ratio"),
                                               _dptr(grad, torch.float64, (W, 3), "grad"),
                                               _dptr(lap, torch.float64, (W,), "lap")))

    def set_params(self, ci: Optional[np.ndarray] = None, B: Optional[Tuple[np.ndarray, np.ndarray]] = None):
        """msd_set_params: new CI coefficients [n_det] and/or orbital coefficients (B_up, B_dn),
        host arrays; the state is rebuilt at the current positions."""
        c = None if ci is None else np.ascontiguousarray(ci, dtype=np.float64)
        if c is not None and c.shape != (self.p.n_det,):
            raise ValueError(f"ci: expected shape ({self.p.n_det},)")
        b0 = b1 = None
        if B is not None:
            b0 = np.ascontiguousarray(B[0], dtype=np.float64)
            b1 = np.ascontiguousarray(B[1], dtype=np.float64)
            if b0.shape != (self.p.n_basis, self.p.n_orb[0]) or b1.shape != (self.p.n_basis, self.p.n_orb[1]):
                raise ValueError("B: expected shapes (n_basis, n_orb[s])")
        self._check(self.lib.msd_set_params(self.ctx, None if c is None else c.ctypes.data,
                                            None if b0 is None else b0.ctypes.data,
                                            None if b1 is None else b1.ctypes.data))

    def backward(self, gbar: torch.Tensor):
        """msd_backward: (dci [n_det], (dB_up [n_basis, n_orb_up], dB_dn [n_basis, n_orb_dn])) of
        sum_w gbar[w] log|Psi_w| at the current positions."""
        nb, N0, N1 = self.p.n_basis, self.p.n_orb[0], self.p.n_orb[1]
        dci = self._empty(self.p.n_det)
        dB = self._empty(nb * (N0 + N1))
        self._check(self.lib.msd_backward(self.ctx, _dptr(gbar, torch.float64, (self.W,), "gbar"),
                                          dci.data_ptr(), dB.data_ptr()))
        return dci, (dB[:nb * N0].view(nb, N0), dB[nb * N0:].view(nb, N1))

    def ratio(self, elec: int, rnew: torch.Tensor, with_grad: bool = True):
        r = self._empty(self.W)
        g = self._empty(self.W, 3) if with_grad else None
        l = self._empty(self.W) if with_grad else None
        self.ratio_into(elec, rnew, r, g, l)
        return r, g, l

    def accept(self, elec: int, accept: torch.Tensor):
        self._check(self.lib.msd_accept(self.ctx, int(elec), _dptr(accept, torch.uint8, (self.W,), "accept")))

    def grad_lap(self, elec: int = -1):
        if elec >= 0:
            g, l = self._empty(self.W, 3), self._empty(self.W)
        else:
            g, l = self._empty(self.W, self.n_tot, 3), self._empty(self.W, self.n_tot)
        self._check(self.lib.msd_grad_lap(self.ctx, int(elec), g.data_ptr(), l.data_ptr()))
        return g, l

    def eval_batch(self, R: torch.Tensor, with_grad: bool = False):
        la, sg = self._empty(self.W), self._empty(self.W)
        g = self._empty(self.W, self.n_tot, 3) if with_grad else None
        l = self._empty(self.W, self.n_tot) if with_grad else None
        self._check(self.lib.msd_eval_batch(self.ctx, _dptr(R, torch.float64, (self.W, self.n_tot, 3), "R"),
                                            la.data_ptr(), sg.data_ptr(),
                                            g.data_ptr() if g is not None else None,
                                            l.data_ptr() if l is not None else None))
        return la, sg, g, l

    def get_state(self):
        R = self._empty(self.W, self.n_tot, 3)
        la, sg = self._empty(self.W), self._empty(self.W)
        self._check(self.lib.msd_get_state(self.ctx, R.data_ptr(), la.data_ptr(), sg.data_ptr()))
        return R, la, sg

    def propose(self, elec: int, eta: torch.Tensor, tau: float, out: torch.Tensor):
        self._check(self.lib.msd_propose(self.ctx, int(elec), _dptr(eta, torch.float64, (self.W, 3), "eta"),
                                         float(tau), _dptr(out, torch.float64, (self.W, 3), "out")))

    # -- VMC energy driver ----------------------------------------------------------------
    def set_hamiltonian(self, Z, b_ee: float = 0.0, b_en: float = 0.0):
        """msd_set_hamiltonian: nuclear charges Z [n_nuc] and the Pade-Jastrow parameters
        (0 removes a term; both 0 = no Jastrow)."""
        z = np.ascontiguousarray(Z, dtype=np.float64)
        if z.shape != (self.p.nuc_xyz.shape[0],):
            raise ValueError(f"Z: expected shape ({self.p.nuc_xyz.shape[0]},)")
        jas = Jastrow(float(b_ee), float(b_en))
        self._check(self.lib.msd_set_hamiltonian(self.ctx, z.ctypes.data, ctypes.byref(jas)))

    def jastrow_ratio_(self, elec: int, rnew: torch.Tensor, ratio: torch.Tensor):
        """msd_jastrow_ratio: ratio [W] *= exp(J(R') - J(R)) for the move of `elec` to rnew."""
        self._check(self.lib.msd_jastrow_ratio(self.ctx, int(elec), _dptr(rnew, torch.float64, (self.W, 3), "rnew"),
                                               _dptr(ratio, torch.float64, (self.W,), "ratio")))

    def local_energy_into(self, eloc: torch.Tensor, parts: Optional[torch.Tensor] = None):
        self._check(self.lib.msd_local_energy(self.ctx, _dptr(eloc, torch.float64, (self.W,), "eloc"),
                                              _dptr(parts, torch.float64, (self.W, 4), "parts")))

    def local_energy(self, with_parts: bool = False):
        """msd_local_energy: E_L [W] at the current positions and, if asked, the parts [W, 4]
        (kinetic, V_ee, V_en, V_nn)."""
        e = self._empty(self.W)
        parts = self._empty(self.W, 4) if with_parts else None
        self.local_energy_into(e, parts)
        return (e, parts) if with_parts else e

    def step(self, elec: int, eta: torch.Tensor, tau: float, u: torch.Tensor, ratio: torch.Tensor,
             grad: torch.Tensor, lap: torch.Tensor, accept: torch.Tensor):
        """msd_step: proposal, ratio/grad/lap, Metropolis decision and update of every walker."""
        W = self.W
        self._check(self.lib.msd_step(self.ctx, int(elec), _dptr(eta, torch.float64, (W, 3), "eta"), float(tau),
                                      _dptr(u, torch.float64, (W,), "u"), _dptr(ratio, torch.float64, (W,), "ratio"),
                                      _dptr(grad, torch.float64, (W, 3), "grad"), _dptr(lap, torch.float64, (W,), "lap"),
                                      _dptr(accept, torch.uint8, (W,), "accept")))

    def metropolis(self, u: torch.Tensor, ratio: torch.Tensor, out: torch.Tensor):
        self._check(self.lib.msd_metropolis(self.ctx, _dptr(u, torch.float64, (self.W,), "u"),
                                            _dptr(ratio, torch.float64, (self.W,), "ratio"),
                                            _dptr(out, torch.uint8, (self.W,), "out")))

    def ratio_host(self, elec: int, rnew: np.ndarray, ratio: np.ndarray, grad: Optional[np.ndarray] = None,
                   lap: Optional[np.ndarray] = None):
        """Host-buffer walker-move step (numpy arrays, ideally in pinned memory)."""
        self._check(self.lib.msd_ratio_host(self.ctx, int(elec), rnew.ctypes.data, ratio.ctypes.data,
                                            grad.ctypes.data if grad is not None else None,
                                            lap.ctypes.data if lap is not None else None))

    def accept_host(self, elec: int, accept: np.ndarray):
        self._check(self.lib.msd_accept_host(self.ctx, int(elec), accept.ctypes.data))

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self.lib.msd_set_stream(self.ctx, stream.cuda_stream))

    def sync(self):
        self._check(self.lib.msd_sync(self.ctx))

    _ITEMS = {"R": 0, "Ainv": 1, "T": 2, "logdet": 3, "sign": 4, "S": 5, "C": 6, "t": 7, "rho": 8, "num": 9,
              "y0": 10, "phi": 11}

    def copy_state(self, item: str, spin: int = 0) -> torch.Tensor:
        """A copy of one piece of the walker state (see msd_copy_state in include/msd.h)."""
        code = self._ITEMS[item]
        nbytes = ctypes.c_int64()
        self._check(self.lib.msd_copy_state(self.ctx, code, int(spin), None, ctypes.byref(nbytes)))
        small = self.mixed and item in ("T", "C", "t", "y0", "phi")
        dt = torch.float32 if small else torch.float64
        out = torch.empty(nbytes.value // (4 if small else 8), dtype=dt, device=self.dev)
        self._check(self.lib.msd_copy_state(self.ctx, code, int(spin), out.data_ptr(), None))
        return out.view(self.W, -1)

    def timing_start(self):
        self._check(self.lib.msd_timing_start(self.ctx))

    def timing_stop(self):
        """(summed excitation-sweep kernel time in ms, its launches, all kernel launches)."""
        ms = ctypes.c_double()
        n1 = ctypes.c_int64()
        n2 = ctypes.c_int64()
        self._check(self.lib.msd_timing_stop(self.ctx, ctypes.byref(ms), ctypes.byref(n1), ctypes.byref(n2)))
        return ms.value, n1.value, n2.value

    def orbitals(self, spin: int, pos: torch.Tensor, nch: int = 5) -> torch.Tensor:
        """msd_orbitals: [P][nch][N] orbitals (and derivatives) of one spin at pos [P][3]."""
        P = int(pos.shape[0])
        N = int(self.p.n_orb[spin])
        out = torch.empty(P, nch, N, dtype=torch.float32 if self.mixed else torch.float64, device=self.dev)
        self._check(self.lib.msd_orbitals(self.ctx, int(spin), int(nch), P, _dptr(pos, torch.float64, (P, 3), "pos"),
                                          out.data_ptr()))
        return out

    def set_rescue(self, slots: int, kappa_hold: float = 1e7, kappa_release: float = 1e5):
        """msd_set_rescue: walkers beyond kappa_hold are held in an FP64 context of `slots` walkers."""
        self._check(self.lib.msd_set_rescue(self.ctx, int(slots), float(kappa_hold), float(kappa_release)))

    def rescue_stats(self) -> dict:
        out = np.zeros(5, dtype=np.int64)
        self._check(self.lib.msd_rescue_stats(self.ctx, out.ctypes.data))
        return dict(held=int(out[0]), holds=int(out[1]), releases=int(out[2]), overflow=int(out[3]),
                    slots=int(out[4]))

    def selftest_wait(self, wait_ns: int):
        """msd_selftest_wait: a device wait that runs out; the next sync raises MSD_ERR_TIMEOUT."""
        self._check(self.lib.msd_selftest_wait(self.ctx, int(wait_ns)))

    def timing_counts(self):
        """(from-scratch refreshes of a spin, CI contractions) since timing_start."""
        out = np.zeros(2, dtype=np.int64)
        self._check(self.lib.msd_timing_counts(self.ctx, out.ctypes.data))
        return int(out[0]), int(out[1])

    def exc_histogram(self, spin: int) -> np.ndarray:
        out = np.zeros(1 + 9, dtype=np.int64)
        self._check(self.lib.msd_exc_histogram(self.ctx, int(spin), out.ctypes.data))
        return out


class MSDBatch:
    """A libmsd context over several independent systems (msd_init with n_systems > 1).

    Per-walker arrays are concatenations over systems; ``elec`` moves electron
    elec mod n_tot_s of system s.  Only the calls a Metropolis driver and the adjoint need are
    wrapped here; every other call of the C ABI works on the same context through ``lib``.
    """

    def __init__(self, problems, n_walkers, precision: str = "mixed", refresh_K=1 << 30,
                 stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise MSDError(2, "a CUDA GPU is required (libmsd has no CPU path)")
        self.lib = load_library()
        self.problems = list(problems)
        ns = len(self.problems)
        Ws = list(n_walkers) if hasattr(n_walkers, "__len__") else [int(n_walkers)] * ns
        Ks = list(refresh_K) if hasattr(refresh_K, "__len__") else [int(refresh_K)] * ns
        self.Ws = [int(w) for w in Ws]
        self.W = sum(self.Ws)
        self.R_len = 3 * sum(w * p.n_tot for w, p in zip(self.Ws, self.problems))
        self.n_det = sum(p.n_det for p in self.problems)
        self.n_B = sum(p.n_basis * (p.n_orb[0] + p.n_orb[1]) for p in self.problems)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (_Problem * ns)()
        self._keep = []
        for i, (p, w, k) in enumerate(zip(self.problems, self.Ws, Ks)):
            s, keep = problem_struct(p, w, precision, k, self.stream.cuda_stream)
            arr[i] = s
            self._keep.append(keep)
        self._arr = arr
        ctx = ctypes.c_void_p()
        rc = self.lib.msd_init(ctypes.cast(arr, ctypes.c_void_p), ns, ctypes.byref(ctx))
        if rc != 0:
            raise MSDError(rc, self.lib.msd_last_error(None).decode())
        self.ctx = ctx
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def _check(self, rc: int):
        if rc != 0:
            raise MSDError(rc, self.lib.msd_last_error(self.ctx).decode())

    def _empty(self, *shape, dtype=torch.float64):
        return torch.empty(shape, dtype=dtype, device=self.dev)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.msd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_positions(self, R: torch.Tensor):
        """R: the concatenation of every system's [W_s, n_tot_s, 3] positions, flattened."""
        self._check(self.lib.msd_set_positions(self.ctx, _dptr(R, torch.float64, (self.R_len,), "R")))

    def propose(self, elec: int, eta: torch.Tensor, tau: float, out: torch.Tensor):
        self._check(self.lib.msd_propose(self.ctx, int(elec), _dptr(eta, torch.float64, (self.W, 3), "eta"), float(tau),
                                         _dptr(out, torch.float64, (self.W, 3), "rnew")))

    def ratio_into(self, elec: int, rnew: torch.Tensor, ratio: torch.Tensor, grad: Optional[torch.Tensor] = None,
                   lap: Optional[torch.Tensor] = None):
        W = self.W
        self._check(self.lib.msd_ratio(self.ctx, int(elec), _dptr(rnew, torch.float64, (W, 3), "rnew"),
                                       _dptr(ratio, torch.float64, (W,), "ratio"),
                                       _dptr(grad, torch.float64, (W, 3), "grad"),
                                       _dptr(lap, torch.float64, (W,), "lap")))

    def ratio(self, elec: int, rnew: torch.Tensor, with_grad: bool = True):
        r = self._empty(self.W)
        g = self._empty(self.W, 3) if with_grad else None
        l = self._empty(self.W) if with_grad else None
        self.ratio_into(elec, rnew, r, g, l)
        return r, g, l

    def step(self, elec: int, eta: torch.Tensor, tau: float, u: torch.Tensor, ratio: torch.Tensor,
             grad: torch.Tensor, lap: torch.Tensor, accept: torch.Tensor):
        """msd_step: proposal, ratio/grad/lap, Metropolis decision and update of every walker."""
        W = self.W
        self._check(self.lib.msd_step(self.ctx, int(elec), _dptr(eta, torch.float64, (W, 3), "eta"), float(tau),
                                      _dptr(u, torch.float64, (W,), "u"), _dptr(ratio, torch.float64, (W,), "ratio"),
                                      _dptr(grad, torch.float64, (W, 3), "grad"), _dptr(lap, torch.float64, (W,), "lap"),
                                      _dptr(accept, torch.uint8, (W,), "accept")))

    def metropolis(self, u: torch.Tensor, ratio: torch.Tensor, out: torch.Tensor):
        self._check(self.lib.msd_metropolis(self.ctx, _dptr(u, torch.float64, (self.W,), "u"),
                                            _dptr(ratio, torch.float64, (self.W,), "ratio"),
                                            _dptr(out, torch.uint8, (self.W,), "accept")))

    def accept(self, elec: int, accept: torch.Tensor):
        self._check(self.lib.msd_accept(self.ctx, int(elec), _dptr(accept, torch.uint8, (self.W,), "accept")))

    def get_state(self):
        R, la, sg = self._empty(self.R_len), self._empty(self.W), self._empty(self.W)
        self._check(self.lib.msd_get_state(self.ctx, R.data_ptr(), la.data_ptr(), sg.data_ptr()))
        return R, la, sg

    def backward(self, gbar: torch.Tensor):
        dci, dB = self._empty(self.n_det), self._empty(self.n_B)
        self._check(self.lib.msd_backward(self.ctx, _dptr(gbar, torch.float64, (self.W,), "gbar"), dci.data_ptr(),
                                          dB.data_ptr()))
        return dci, dB

    def sync(self):
        self._check(self.lib.msd_sync(self.ctx))

    def timing_start(self):
        self._check(self.lib.msd_timing_start(self.ctx))

    def timing_stop(self):
        ms, n1, n2 = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.msd_timing_stop(self.ctx, ctypes.byref(ms), ctypes.byref(n1), ctypes.byref(n2)))
        return ms.value, n1.value, n2.value

    def timing_counts(self):
        out = np.zeros(2, dtype=np.int64)
        self._check(self.lib.msd_timing_counts(self.ctx, out.ctypes.data))
        return int(out[0]), int(out[1])

    def set_rescue(self, slots: int, kappa_hold: float = 1e7, kappa_release: float = 1e5):
        self._check(self.lib.msd_set_rescue(self.ctx, int(slots), float(kappa_hold), float(kappa_release)))

    def rescue_stats(self) -> dict:
        out = np.zeros(5, dtype=np.int64)
        self._check(self.lib.msd_rescue_stats(self.ctx, out.ctypes.data))
        return dict(held=int(out[0]), holds=int(out[1]), releases=int(out[2]), overflow=int(out[3]),
                    slots=int(out[4]))
