"""The C ABI library without a GPU: it loads, exports every declared symbol, and rejects bad
problems on the host before any CUDA call (argument validation needs no device)."""
import ctypes

import numpy as np
import pytest

import __graft_entry__
from paper_1106_2456_gb300 import build as libbuild
from paper_1106_2456_gb300 import msd, workloads as wl


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return msd.load_library()


def test_exports_every_declared_function(lib):
    names = msd.header_functions()
    assert "msd_init" in names and "msd_ratio" in names and "msd_accept" in names
    assert "msd_grad_lap" in names and "msd_eval_batch" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def _struct(problem, W=4, prec=1, K=5):
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(x, dtype=dt)
        if a.size == 0:
            a = np.zeros(1, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    s = msd._Problem()
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
    s.n_walkers = W
    s.prec = prec
    s.refresh_K = K
    s.cuda_stream = None
    return s, keep


def _init_status(lib, s, n_systems=1):
    ctx = ctypes.c_void_p()
    rc = lib.msd_init(ctypes.byref(s), n_systems, ctypes.byref(ctx))
    return rc, lib.msd_last_error(None).decode()


@pytest.mark.parametrize("mutate,needle", [
    (lambda s, k: setattr(s, "n_walkers", 0), "n_walkers"),
    (lambda s, k: setattr(s, "refresh_K", 0), "refresh_K"),
    (lambda s, k: setattr(s, "prec", 7), "precision"),
    (lambda s, k: s.n_elec.__setitem__(0, 0), "n_elec"),
    (lambda s, k: s.n_orb.__setitem__(1, 3), "n_orb"),
    (lambda s, k: setattr(s, "n_det", 0), "term"),
])
def test_init_rejects_bad_arguments(lib, mutate, needle):
    w = wl.make_workload("water", n_walkers=4)
    s, keep = _struct(w.problem)
    mutate(s, keep)
    rc, msg = _init_status(lib, s)
    assert rc == 1 and needle in msg


def test_init_rejects_bad_strings(lib):
    w = wl.make_workload("water", n_walkers=4)
    p = w.problem
    # particle index beyond the virtuals
    bad = wl.dataclasses.replace(p, exc_parts=(p.exc_parts[0].copy(), p.exc_parts[1].copy()))
    bad.exc_parts[0][0] = 200
    s, keep = _struct(bad)
    rc, msg = _init_status(lib, s)
    assert rc == 1 and "out of range" in msg
    # holes not ascending
    off = p.exc_off[0]
    u = int(np.nonzero(np.diff(off) >= 2)[0][0])
    holes = p.exc_holes[0].copy()
    holes[off[u]], holes[off[u] + 1] = holes[off[u] + 1], holes[off[u]]
    bad = wl.dataclasses.replace(p, exc_holes=(holes, p.exc_holes[1]))
    s, keep = _struct(bad)
    rc, msg = _init_status(lib, s)
    assert rc == 1 and "ascending" in msg
    # a term pointing past the strings
    du = p.det_up.copy()
    du[3] = p.n_exc(0)
    s, keep = _struct(wl.dataclasses.replace(p, det_up=du))
    rc, msg = _init_status(lib, s)
    assert rc == 1 and "missing string" in msg
    # the reference must come first
    off2 = p.exc_off[1].copy()
    s, keep = _struct(p)
    fake = np.concatenate([[0], off2[1:] + 1]).astype(np.int32)
    keep.append(fake)
    s.exc_off[1] = fake.ctypes.data
    rc, msg = _init_status(lib, s)
    assert rc == 1


def test_init_batched_validation(lib):
    """n_systems > 1 reads an array of problems and validates each before any CUDA call."""
    w = wl.make_workload("water", n_walkers=4)
    rc, msg = _init_status(lib, _struct(w.problem)[0], n_systems=0)
    assert rc == 1 and "n_systems" in msg
    keep = []
    arr = (msd._Problem * 3)()
    for i in range(3):
        s, k = _struct(w.problem)
        keep.append(k)
        arr[i] = s
    arr[2].refresh_K = 0
    ctx = ctypes.c_void_p()
    rc = lib.msd_init(ctypes.cast(arr, ctypes.c_void_p), 3, ctypes.byref(ctx))
    msg = lib.msd_last_error(None).decode()
    assert rc == 1 and "system 2" in msg and "refresh_K" in msg and not ctx.value


def test_batched_workloads_shapes():
    ws = wl.batched_workloads(12, W=3, seed=5)
    for w in ws:
        p = w.problem
        n = p.n_elec[0]
        assert 4 <= n <= 96 and p.n_elec == (n, n) and p.n_orb == (3 * n, 3 * n)
        assert 1 <= p.n_det <= max(1, wl.feasible_terms(n, 2 * n, 1, 6) // 4)
        assert p.exc_orders(0).max() <= 6 and w.R0.shape == (3, 2 * n, 3)
    # the small-system cap: 4 electrons per spin, 8 virtuals
    assert wl.feasible_terms(4, 8, 1, 6) == 208764


def test_init_rejects_table_larger_than_shared_memory(lib):
    w = wl.make_workload("water", n_walkers=4)
    s, keep = _struct(w.problem)
    s.n_elec[0] = 200
    s.n_orb[0] = 400
    rc, msg = _init_status(lib, s)
    assert rc == 1


def test_null_arguments_are_rejected(lib):
    assert lib.msd_init(None, 1, None) == 1
    assert lib.msd_sync(None) == 1
    assert lib.msd_ratio(None, 0, None, None, None, None) == 1
    lib.msd_destroy(None)  # no-op


def test_graft_build_entry():
    __graft_entry__.build()


def _describe(lib, problem):
    s, keep = _struct(problem)
    out = np.zeros(32, dtype=np.int64)
    rc = lib.msd_describe(ctypes.byref(s), out.ctypes.data)
    assert rc == 0, lib.msd_last_error(None).decode()
    return out.reshape(2, 16)


@pytest.mark.parametrize("label,kw", [("water", {}), ("medium", {"n_walkers": 2}),
                                      ("large", {"n_walkers": 2, "n_det": 20000})])
def test_device_layout_plan(lib, label, kw):
    """The host-side plan of msd_init (string groups, dense singles, term lists), no GPU."""
    p = wl.make_workload(label, **kw).problem
    d = _describe(lib, p)
    for s in range(2):
        n, m = p.n_elec[s], p.n_orb[s] - p.n_elec[s]
        hist = np.bincount(p.exc_orders(s), minlength=9)
        dense = hist[1] > 0 and 4 * hist[1] >= n * m
        assert d[s, 1] == int(dense)
        goff = d[s, 5:15]
        assert goff[0] == 0 and np.all(np.diff(goff) >= 0)
        sizes = np.diff(goff)
        assert sizes[0] == hist[0]
        if dense:
            assert sizes[1] == n * m
        for k in range(2 if dense else 1, 9):
            assert sizes[k] % 32 == 0 and hist[k] <= sizes[k] and (sizes[k] > 0) == (hist[k] > 0)
        assert d[s, 0] == goff[-1]
        assert d[s, 2] == int(np.nonzero(hist)[0].max())
        assert d[s, 15] == p.n_det
        rb = {1: 2, 2: 4, 3: 8, 4: 8}
        want = 0
        for k in range(2 if dense else 1, 9):
            want = (want + 15) // 16 * 16 + int(sizes[k]) * rb.get(k, 16)
        assert d[s, 4] == (want + 15) // 16 * 16
        _check_records(lib, p, s, goff, dense)


@pytest.mark.parametrize("prec", [0, 2])
def test_device_layout_plan_fp64(prec):
    """FP64 tables and the canonical mode: batches filled in sorted order, padding only at
    the end of each order."""
    lib = msd.load_library()
    p = wl.make_workload("medium", n_walkers=2).problem
    s, keep = _struct(p, prec=prec)
    out = np.zeros(32, dtype=np.int64)
    assert lib.msd_describe(ctypes.byref(s), out.ctypes.data) == 0
    d = out.reshape(2, 16)
    for sp in range(2):
        hist = np.bincount(p.exc_orders(sp), minlength=9)
        sizes = np.diff(d[sp, 5:15])
        dense = bool(d[sp, 1])
        for k in range(2 if dense else 1, 9):
            assert sizes[k] == -(-hist[k] // 32) * 32
        _check_records(lib, p, sp, d[sp, 5:15], dense, conflict_free=False)


def _records(lib, problem, spin, prec=1):
    s, keep = _struct(problem, prec=prec)
    off = np.zeros(10, dtype=np.int64)
    nbytes = ctypes.c_int64()
    assert lib.msd_describe_records(ctypes.byref(s), spin, None, 0, off.ctypes.data, ctypes.byref(nbytes)) == 0
    out = np.zeros(max(nbytes.value, 1), dtype=np.uint8)
    assert lib.msd_describe_records(ctypes.byref(s), spin, out.ctypes.data, out.size, off.ctypes.data,
                                    ctypes.byref(nbytes)) == 0
    return out, off


def _perm_parity(a):
    a = list(a)
    inv = sum(1 for i in range(len(a)) for j in range(i + 1, len(a)) if a[i] > a[j])
    return inv & 1


def _check_records(lib, p, spin, goff, dense, conflict_free=True):
    """Every string of order k appears once in its group's records, holes and particles
    permuted with equal parity; slots of a batch hold distinct particle residues mod 32."""
    out, off = _records(lib, p, spin, prec=1 if conflict_free else 0)
    rb = {1: 2, 2: 4, 3: 8, 4: 8}
    offs = p.exc_off[spin]
    for k in range(2 if dense else 1, 9):
        size = goff[k + 1] - goff[k]
        if size == 0:
            continue
        r = out[off[k]:off[k] + size * rb.get(k, 16)].reshape(size, rb.get(k, 16))
        used = r[:, 0] != 0xFF
        holes, parts = r[used, :k].astype(int), r[used, k:2 * k].astype(int)
        # each string exactly once, with the same hole and particle sets
        want = sorted((tuple(p.exc_holes[spin][offs[u]:offs[u + 1]]), tuple(p.exc_parts[spin][offs[u]:offs[u + 1]]))
                      for u in range(p.n_exc(spin)) if offs[u + 1] - offs[u] == k)
        got = sorted((tuple(sorted(h)), tuple(sorted(q))) for h, q in zip(holes, parts))
        assert got == want
        for h, q in zip(holes, parts):
            assert _perm_parity(h) == _perm_parity(q)
        if not conflict_free:
            continue
        # distinct residues per slot within each batch of 32
        res = np.where(used[:, None], r[:, k:2 * k].astype(int) % 32, -1 - np.arange(size)[:, None])
        for b in range(size // 32):
            blk = res[32 * b:32 * b + 32]
            for l in range(k):
                assert len(set(blk[:, l].tolist())) == 32


def test_device_layout_plan_edge_cases(lib):
    # sparse singles (well under a quarter of the n m pairs) stay in per-excitation records
    w = wl.custom_workload((11, 9), (25, 26), 700, wl.uniform_orders(1, 8), W=3, n_nuc=4, seed=11)
    d = _describe(lib, w.problem)
    assert d[0, 2] == 8
    # one electron per spin, single determinant, no virtual orbitals
    base = wl.make_workload("water", n_walkers=2).problem
    B0 = (np.ascontiguousarray(base.B[0][:, :5]), np.ascontiguousarray(base.B[1][:, :5]))
    single = wl.explicit_problem(base.nuc_xyz, base.bas_center, base.bas_lm, base.bas_alpha, B0, base.n_elec,
                                 [((), ())], [((), ())], [0], [0], [1.0])
    d = _describe(lib, single)
    assert d[0, 0] == 1 and d[1, 0] == 1 and d[0, 15] == 1
    w = wl.custom_workload((1, 1), (6, 4), 9, wl.uniform_orders(1, 2), W=1, n_nuc=2, seed=3)
    d = _describe(lib, w.problem)
    assert d[0, 1] == 1 and d[0, 0] == 1 + 5  # dense singles: one hole, five virtuals
