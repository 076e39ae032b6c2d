"""The excitation-determinant arithmetic of the CUDA kernels, built for the host and checked
against exact rational determinants (no GPU needed).

``paper_1106_2456_gb300/csrc/msd_smalldet.cuh`` holds the code that the excitation-sweep
kernel runs for every excitation of order k: det T_u and z = adj(T_u) x_u from a pivoted LU
of the first k-2 columns and a closed-form 2 x 2 Schur block (FMA-corrected 2 x 2
determinants); every bordered determinant of a move is det [[T_u, x_u], [-y^T, s]] =
det(T_u) s + y . z.
Here it is compiled by g++ through ``tests/native/smalldet_host.cpp``; the bordered values
it implies are compared with the exact determinant of the same floating-point inputs
(Python fractions).  The adversarial inputs give T a large
rank-1 component, as an ill-conditioned reference matrix A_0 does to T = A_0^{-1} Phi_virt;
closed-form cofactor expansions lose up to 1e-4 relative accuracy there (k = 3), which this
test would catch.
"""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def lib():
    out_dir = os.path.join(HERE, "native", "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "smalldet_host.so")
    src = os.path.join(HERE, "native", "smalldet_host.cpp")
    hdr = os.path.join(ROOT, "paper_1106_2456_gb300", "csrc", "msd_smalldet.cuh")
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(src), os.path.getmtime(hdr)):
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                        "-I" + os.path.join(ROOT, "paper_1106_2456_gb300", "csrc"), src, "-o", so + ".tmp"],
                       check=True)
        os.replace(so + ".tmp", so)
    L = ctypes.CDLL(so)
    vp, ci = ctypes.c_void_p, ctypes.c_int
    L.sd_det_f64.restype = ctypes.c_double
    L.sd_det_f64.argtypes = [ci, vp, ci, vp, vp]
    L.sd_det_f32.restype = ctypes.c_float
    L.sd_det_f32.argtypes = [ci, vp, ci, vp, vp]
    L.sd_adj_f64.restype = ctypes.c_double
    L.sd_adj_f64.argtypes = [ci, vp, ci, vp, vp, vp, vp]
    L.sd_adj_f32.restype = ctypes.c_float
    L.sd_adj_f32.argtypes = [ci, vp, ci, vp, vp, vp, vp]
    return L


def exact_det(M):
    A = [[Fraction(float(v)) for v in row] for row in M]
    n = len(A)
    det = Fraction(1)
    for k in range(n):
        piv = next((r for r in range(k, n) if A[r][k] != 0), None)
        if piv is None:
            return Fraction(0)
        if piv != k:
            A[k], A[piv] = A[piv], A[k]
            det = -det
        det *= A[k][k]
        for r in range(k + 1, n):
            f = A[r][k] / A[k][k]
            for j in range(k, n):
                A[r][j] -= f * A[k][j]
    return det


def case(rng, K, blowup, dtype):
    n, m = K + int(rng.integers(0, 4)), K + int(rng.integers(0, 5))
    T = rng.standard_normal((n, m)) + blowup * np.outer(rng.standard_normal(n), rng.standard_normal(m))
    x = rng.standard_normal(n) * (1 + blowup * abs(rng.standard_normal()))
    y = rng.standard_normal((5, m))
    s = rng.standard_normal(5)
    h = np.sort(rng.choice(n, K, replace=False)).astype(np.int32)
    p = np.sort(rng.choice(m, K, replace=False)).astype(np.int32)
    cast = lambda a: np.ascontiguousarray(a, dtype=dtype)
    return cast(T), cast(x), cast(y), cast(s), h, p, m


def run(lib, K, T, x, y, s, h, p, m, f32):
    """Bordered determinants det(T_u) s^a + y^a . z from the library's (det, z), and det T_u."""
    z = np.zeros(K, dtype=np.float32 if f32 else np.float64)
    fn = lib.sd_adj_f32 if f32 else lib.sd_adj_f64
    det = fn(K, T.ctypes.data, m, x.ctypes.data, h.ctypes.data, p.ctypes.data, z.ctypes.data)
    d = np.array([det * s[a] + np.dot(y[a, p], z) for a in range(5)], dtype=z.dtype)
    dt = (lib.sd_det_f32 if f32 else lib.sd_det_f64)(K, T.ctypes.data, m, h.ctypes.data, p.ctypes.data)
    return d, dt


def exact_results(K, T, x, y, s, h, p):
    Tu = T[np.ix_(h, p)].astype(np.float64)
    dets = []
    for a in range(5):
        Mb = np.zeros((K + 1, K + 1))
        Mb[:K, :K] = Tu
        Mb[:K, K] = x[h]
        Mb[K, :K] = -y[a, p]
        Mb[K, K] = s[a]
        dets.append(float(exact_det(Mb)))
    return np.array(dets), float(exact_det(Tu))


@pytest.mark.parametrize("K", range(1, 9))
@pytest.mark.parametrize("blowup", [0.0, 1e6])
def test_fp64_against_exact(lib, K, blowup):
    rng = np.random.default_rng(100 * K + int(blowup > 0))
    worst = 0.0
    for _ in range(12):
        T, x, y, s, h, p, m = case(rng, K, blowup, np.float64)
        d, dt = run(lib, K, T, x, y, s, h, p, m, False)
        ref, ref_t = exact_results(K, T, x, y, s, h, p)
        worst = max(worst, float(np.max(np.abs(d - ref) / np.abs(ref))), abs(dt - ref_t) / abs(ref_t))
    assert worst < 1e-8, worst


@pytest.mark.parametrize("K", range(1, 9))
def test_fp32_against_exact(lib, K):
    rng = np.random.default_rng(7 + K)
    worst = 0.0
    for _ in range(12):
        T, x, y, s, h, p, m = case(rng, K, 30.0, np.float32)
        d, dt = run(lib, K, T, x, y, s, h, p, m, True)
        ref, ref_t = exact_results(K, T, x, y, s, h, p)
        worst = max(worst, float(np.max(np.abs(d - ref) / np.abs(ref))), abs(dt - ref_t) / abs(ref_t))
    assert worst < 2e-3, worst


@pytest.mark.parametrize("K", [2, 3, 4, 6, 8])
def test_exactly_singular_table_block_uses_direct_bordered_lu(lib, K):
    rng = np.random.default_rng(K)
    T, x, y, s, h, p, m = case(rng, K, 0.0, np.float64)
    T[:, p[1]] = 0.0  # a zero column: det T_u = 0 exactly, the bordered determinants are not 0
    d, dt = run(lib, K, T, x, y, s, h, p, m, False)
    ref, ref_t = exact_results(K, T, x, y, s, h, p)
    assert dt == 0.0 and ref_t == 0.0
    assert np.max(np.abs(d - ref) / np.abs(ref)) < 1e-10
