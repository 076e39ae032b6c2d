"""Seeded synthetic multi-determinant problems (inputs only, no method arithmetic).

This module is the one piece shared by the FP64 oracle tests and the CUDA path:
it draws random numbers and arranges them into the problem format of the C ABI
(``include/msd.h``).  It evaluates no orbital, determinant, ratio or update.

Problem shape follows Section II of the paper:

* Psi = sum_I c_I det M_up,I det M_dn,I (Jastrow factor omitted, Section II).
* M_sigma,I(r, c) = phi_{col_I(c)}(r_r): rows are electrons, columns orbitals.
* Orbitals 0..n-1 of each spin form the reference determinant; n..N-1 are the
  m = N - n virtual orbitals.  A per-spin excitation string replaces the
  occupied columns h_1 < ... < h_k in place by virtuals p_1 < ... < p_k
  (particle-hole excitations, Section II).

Synthetic stand-ins (the paper's GAMESS ANO orbitals and SOCI/CSF expansion of
water are not available):

* basis: 12 Cartesian Gaussians per nucleus, 3 exponents drawn log-uniform in
  [0.1, 10] bohr^-2, each giving one s and one p shell (px, py, pz), unnormalised
  x^l exp(-alpha |r - R|^2);
* orbitals: B[mu, j] ~ N(0, 1) / sqrt(n_basis), one set shared by both spins;
* terms: total excitation order r from the config's distribution, split
  r_up uniform over its feasible range, holes/particles uniform without
  replacement, duplicate terms rejected, c_I = N(0,1) exp(-r/2), c_0 = 1;
* walkers: electron e starts at nucleus (e mod n_nuc) plus N(0, 1) bohr per axis;
  proposals r' = r + tau * N(0,1)^3, Metropolis uniforms U(0, 1).

Water geometry is the equilibrium one of Section VI (r_OH = 0.9572 A,
angle HOH = 104.52 deg).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
MAXK = 8  # largest per-spin excitation order the library accepts
_PAD = 32767  # padding of unused hole/particle slots in the draw arrays


@dataclasses.dataclass
class Problem:
    """One multi-determinant wavefunction, in the layout of ``msd_problem``."""

    n_elec: Tuple[int, int]
    n_orb: Tuple[int, int]
    nuc_xyz: np.ndarray            # [n_nuc, 3] f64, bohr
    bas_center: np.ndarray         # [n_basis] int32
    bas_lm: np.ndarray             # [n_basis] int8: 0 = s, 1..3 = px, py, pz
    bas_alpha: np.ndarray          # [n_basis] f64
    B: Tuple[np.ndarray, np.ndarray]  # per spin [n_basis, n_orb] f64
    exc_off: Tuple[np.ndarray, np.ndarray]    # per spin [n_exc + 1] int32 (CSR)
    exc_holes: Tuple[np.ndarray, np.ndarray]  # per spin uint8, occupied index
    exc_parts: Tuple[np.ndarray, np.ndarray]  # per spin uint8, virtual index 0..m-1
    det_up: np.ndarray             # [n_det] int32, index into spin-up strings
    det_dn: np.ndarray             # [n_det] int32
    ci: np.ndarray                 # [n_det] f64
    name: str = ""

    @property
    def n_basis(self) -> int:
        return int(self.bas_alpha.shape[0])

    @property
    def n_det(self) -> int:
        return int(self.ci.shape[0])

    @property
    def n_tot(self) -> int:
        return int(self.n_elec[0] + self.n_elec[1])

    def n_exc(self, s: int) -> int:
        return int(self.exc_off[s].shape[0] - 1)

    def exc_orders(self, s: int) -> np.ndarray:
        return np.diff(self.exc_off[s]).astype(np.int64)

    def spin_of(self, e: int) -> int:
        return 0 if e < self.n_elec[0] else 1


@dataclasses.dataclass
class Workload:
    """A problem plus walkers and the random streams of a Metropolis run."""

    problem: Problem
    R0: np.ndarray          # [W, n_tot, 3] f64 initial positions
    tau: float
    seed: int
    n_walkers: int
    refresh_K: int
    n_sweeps: int
    label: str

    def proposals(self, n_steps: int, seed_offset: int = 0) -> Tuple[np.ndarray, np.ndarray]:
        """Gaussian displacements eta [n_steps, W, 3] and uniforms u [n_steps, W]."""
        rng = np.random.default_rng(self.seed * 7919 + 17 + seed_offset)
        eta = rng.standard_normal((n_steps, self.n_walkers, 3))
        u = rng.random((n_steps, self.n_walkers))
        return eta, u


# ----------------------------------------------------------------------------
# geometry and basis
# ----------------------------------------------------------------------------

def water_nuclei() -> np.ndarray:
    """O at the origin, H at (+-0.757, 0, 0.586) A: r_OH 0.9572 A, angle 104.52 deg."""
    half = math.radians(104.52) / 2.0
    hx = 0.9572 * math.sin(half)
    hz = 0.9572 * math.cos(half)
    xyz = np.array([[0.0, 0.0, 0.0], [hx, 0.0, hz], [-hx, 0.0, hz]])
    return xyz * BOHR_PER_ANGSTROM


def chain_nuclei(rng: np.random.Generator, n_nuc: int) -> np.ndarray:
    """Random chain: consecutive spacing U(1.5, 3) bohr in a uniformly random direction."""
    xyz = np.zeros((n_nuc, 3))
    for a in range(1, n_nuc):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        xyz[a] = xyz[a - 1] + rng.uniform(1.5, 3.0) * v
    return xyz


def gaussian_basis(rng: np.random.Generator, n_nuc: int, n_exp: int = 3):
    """n_exp exponents per nucleus, each one s and one p shell: 4 * n_exp functions per nucleus."""
    centers, lms, alphas = [], [], []
    for a in range(n_nuc):
        ex = np.exp(rng.uniform(math.log(0.1), math.log(10.0), size=n_exp))
        for al in ex:
            for lm in range(4):
                centers.append(a)
                lms.append(lm)
                alphas.append(al)
    return (np.asarray(centers, np.int32), np.asarray(lms, np.int8), np.asarray(alphas, np.float64))


# ----------------------------------------------------------------------------
# excitation strings and CI terms
# ----------------------------------------------------------------------------

def _draw_subsets(rng: np.random.Generator, pool: int, counts: np.ndarray) -> np.ndarray:
    """Rows of sorted distinct draws from range(pool), padded with _PAD past counts[i]."""
    M = counts.shape[0]
    out = np.full((M, MAXK), _PAD, dtype=np.int16)
    chunk = 16384
    for s in range(0, M, chunk):
        c = counts[s:s + chunk]
        keys = rng.random((c.shape[0], pool))
        kk = min(MAXK, pool)
        idx = np.argpartition(keys, kk - 1, axis=1)[:, :kk] if pool > kk else np.argsort(keys, axis=1)
        # order the selected keys so the first c[i] are a uniform subset
        sel_keys = np.take_along_axis(keys, idx, axis=1)
        order = np.argsort(sel_keys, axis=1)
        idx = np.take_along_axis(idx, order, axis=1)
        blk = np.full((c.shape[0], MAXK), _PAD, dtype=np.int16)
        blk[:, :idx.shape[1]] = idx
        mask = np.arange(MAXK)[None, :] >= c[:, None]
        blk[mask] = _PAD
        blk.sort(axis=1)
        out[s:s + chunk] = blk
    return out


def draw_terms(rng: np.random.Generator, n: Tuple[int, int], m: Tuple[int, int], n_det: int,
               order_probs: Dict[int, float]):
    """Draw n_det distinct (up string, down string) terms; term 0 is (reference, reference).

    Returns per-spin padded hole/particle arrays [n_det, MAXK], per-spin orders and the
    total order r of each term.
    """
    kmax = (min(n[0], m[0], MAXK), min(n[1], m[1], MAXK))
    orders = np.array(sorted(order_probs), dtype=np.int64)
    probs = np.array([order_probs[k] for k in orders], dtype=np.float64)
    probs /= probs.sum()
    have_keys = set()
    H = [np.zeros((0, MAXK), np.int16), np.zeros((0, MAXK), np.int16)]
    P = [np.zeros((0, MAXK), np.int16), np.zeros((0, MAXK), np.int16)]
    K = [np.zeros(0, np.int64), np.zeros(0, np.int64)]
    R = np.zeros(0, np.int64)
    # reference term
    ref = np.full((1, MAXK), _PAD, np.int16)
    for s in range(2):
        H[s] = np.concatenate([H[s], ref])
        P[s] = np.concatenate([P[s], ref])
        K[s] = np.concatenate([K[s], np.zeros(1, np.int64)])
    R = np.concatenate([R, np.zeros(1, np.int64)])
    have_keys.add(np.concatenate([ref, ref, ref, ref], axis=1).tobytes())
    need = n_det - 1
    while need > 0:
        M = int(need * 1.25) + 64
        r = rng.choice(orders, size=M, p=probs)
        lo = np.maximum(0, r - kmax[1])
        hi = np.minimum(r, kmax[0])
        ok = lo <= hi
        r, lo, hi = r[ok], lo[ok], hi[ok]
        r_up = lo + (rng.random(r.shape[0]) * (hi - lo + 1)).astype(np.int64)
        r_up = np.minimum(r_up, hi)
        r_dn = r - r_up
        hu = _draw_subsets(rng, n[0], r_up)
        pu = _draw_subsets(rng, m[0], r_up)
        hd = _draw_subsets(rng, n[1], r_dn)
        pd = _draw_subsets(rng, m[1], r_dn)
        keys = np.concatenate([hu, pu, hd, pd], axis=1)
        take = []
        for i in range(keys.shape[0]):
            kb = keys[i].tobytes()
            if kb in have_keys:
                continue
            have_keys.add(kb)
            take.append(i)
            if len(take) == need:
                break
        take = np.asarray(take, dtype=np.int64)
        H[0] = np.concatenate([H[0], hu[take]]); P[0] = np.concatenate([P[0], pu[take]])
        H[1] = np.concatenate([H[1], hd[take]]); P[1] = np.concatenate([P[1], pd[take]])
        K[0] = np.concatenate([K[0], r_up[take]]); K[1] = np.concatenate([K[1], r_dn[take]])
        R = np.concatenate([R, r[take]])
        need -= take.shape[0]
    return H, P, K, R


def unique_strings(H: np.ndarray, P: np.ndarray, K: np.ndarray):
    """Deduplicate per-spin strings in order of first appearance (the reference comes first).

    Returns CSR (off, holes, parts) and the map term -> string index.
    """
    keys = np.concatenate([H, P], axis=1)
    _, first, inv = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    order = np.argsort(first, kind="stable")        # unique ids sorted by first appearance
    rank = np.empty_like(order)
    rank[order] = np.arange(order.shape[0])
    term_to_str = rank[inv].astype(np.int32)
    reps = first[order]
    k = K[reps]
    off = np.zeros(reps.shape[0] + 1, np.int32)
    off[1:] = np.cumsum(k)
    holes = np.concatenate([H[i, :K[i]] for i in reps]).astype(np.uint8) if off[-1] else np.zeros(0, np.uint8)
    parts = np.concatenate([P[i, :K[i]] for i in reps]).astype(np.uint8) if off[-1] else np.zeros(0, np.uint8)
    return off, holes, parts, term_to_str


def geometric_orders(kmin: int, kmax: int, p: float = 0.5) -> Dict[int, float]:
    """P(r) proportional to (1-p)^(r-kmin) on kmin..kmax (p = 0.5 gives 2^-r)."""
    return {k: (1.0 - p) ** (k - kmin) for k in range(kmin, kmax + 1)}


def uniform_orders(kmin: int, kmax: int) -> Dict[int, float]:
    return {k: 1.0 for k in range(kmin, kmax + 1)}


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------

def make_problem(seed: int, nuc_xyz: np.ndarray, n: Tuple[int, int], N: Tuple[int, int], n_det: int,
                 order_probs: Dict[int, float], rng: Optional[np.random.Generator] = None,
                 name: str = "") -> Problem:
    rng = np.random.default_rng(seed) if rng is None else rng
    n_nuc = nuc_xyz.shape[0]
    bc, blm, bal = gaussian_basis(rng, n_nuc)
    nb = bal.shape[0]
    if nb < max(n):
        raise ValueError("basis smaller than the electron count: reference determinant singular")
    Nmax = max(N)
    Bfull = rng.standard_normal((nb, Nmax)) / math.sqrt(nb)
    B = (np.ascontiguousarray(Bfull[:, :N[0]]), np.ascontiguousarray(Bfull[:, :N[1]]))
    m = (N[0] - n[0], N[1] - n[1])
    H, P, K, R = draw_terms(rng, n, m, n_det, order_probs)
    ci = rng.standard_normal(n_det) * np.exp(-0.5 * R)
    ci[0] = 1.0
    off_u, h_u, p_u, t_u = unique_strings(H[0], P[0], K[0])
    off_d, h_d, p_d, t_d = unique_strings(H[1], P[1], K[1])
    return Problem(n_elec=(int(n[0]), int(n[1])), n_orb=(int(N[0]), int(N[1])),
                   nuc_xyz=np.ascontiguousarray(nuc_xyz, dtype=np.float64),
                   bas_center=bc, bas_lm=blm, bas_alpha=bal, B=B,
                   exc_off=(off_u, off_d), exc_holes=(h_u, h_d), exc_parts=(p_u, p_d),
                   det_up=t_u, det_dn=t_d, ci=ci.astype(np.float64), name=name)


def initial_walkers(rng: np.random.Generator, nuc_xyz: np.ndarray, n_tot: int, W: int) -> np.ndarray:
    n_nuc = nuc_xyz.shape[0]
    centers = nuc_xyz[np.arange(n_tot) % n_nuc]
    return centers[None, :, :] + rng.standard_normal((W, n_tot, 3))


CONFIGS = {
    # Water-like toy system, plain FP64 (Section VI geometry).
    "water": dict(idx=1, n=(5, 5), N=(20, 20), n_det=200, orders=("uniform", 1, 4), W=64,
                  sweeps=50, nuclei="water", K=5),
    # Medium system, FP64 on the GPU.
    "medium": dict(idx=2, n=(32, 32), N=(120, 120), n_det=10_000, orders=("geom", 1, 6), W=1024,
                   sweeps=200, nuclei=6, K=32),
    # Mixed precision at scale: 64 + 64 electrons, 1e5 determinants, 4096 walkers.
    "large": dict(idx=3, n=(64, 64), N=(256, 256), n_det=100_000, orders=("geom", 1, 8), W=4096,
                  sweeps=1, nuclei=12, K=64),
    # Same as "large" with the uniform 1-8 order distribution (stress variant).
    "large_uniform": dict(idx=3, n=(64, 64), N=(256, 256), n_det=100_000, orders=("uniform", 1, 8),
                          W=4096, sweeps=1, nuclei=12, K=64),
    # Differentiation system: 32 + 32 electrons, 160 orbitals, 5e4 determinants.
    "diff": dict(idx=5, n=(32, 32), N=(160, 160), n_det=50_000, orders=("geom", 1, 6), W=4096,
                 sweeps=1, nuclei=6, K=32),
}


def make_workload(label: str, n_walkers: Optional[int] = None, n_det: Optional[int] = None,
                  seed: Optional[int] = None, tau: float = 0.5) -> Workload:
    """Build one of CONFIGS, optionally with fewer walkers or determinants for quick tests."""
    cfg = CONFIGS[label]
    seed = 1000 + cfg["idx"] if seed is None else seed
    rng = np.random.default_rng(seed)
    if cfg["nuclei"] == "water":
        nuc = water_nuclei()
    else:
        nuc = chain_nuclei(rng, int(cfg["nuclei"]))
    kind, k0, k1 = cfg["orders"]
    orders = uniform_orders(k0, k1) if kind == "uniform" else geometric_orders(k0, k1)
    nd = cfg["n_det"] if n_det is None else n_det
    prob = make_problem(seed, nuc, cfg["n"], cfg["N"], nd, orders, rng=rng, name=label)
    W = cfg["W"] if n_walkers is None else n_walkers
    R0 = initial_walkers(rng, nuc, prob.n_tot, W)
    return Workload(problem=prob, R0=R0, tau=tau, seed=seed, n_walkers=W, refresh_K=cfg["K"],
                    n_sweeps=cfg["sweeps"], label=label)


def nuclear_charges(problem: Problem) -> np.ndarray:
    """Charges Z_I for the local energy: water's (8, 1, 1) for the water system (10 electrons,
    neutral); otherwise the n_tot electrons shared over the nuclei as evenly as integers allow,
    the first nuclei taking the remainder, so that every synthetic system is neutral."""
    n_nuc = problem.nuc_xyz.shape[0]
    if problem.name == "water" and n_nuc == 3:
        return np.array([8.0, 1.0, 1.0])
    q, r = divmod(problem.n_tot, n_nuc)
    return np.array([q + (1 if I < r else 0) for I in range(n_nuc)], dtype=np.float64)


def feasible_terms(n: int, m: int, kmin: int, kmax: int) -> int:
    """Distinct (up string, down string) pairs of total excitation order kmin..kmax."""
    a = [math.comb(n, r) * math.comb(m, r) if r <= min(n, m, MAXK) else 0 for r in range(kmax + 1)]
    return sum(a[ru] * a[r - ru] for r in range(kmin, kmax + 1) for ru in range(r + 1))


def batched_workloads(n_systems: int = 256, W: int = 256, seed: int = 1004, n_range=(4, 96),
                      det_range=(1e2, 1e5), kmax: int = 6, K: int = 64, tau: float = 0.5) -> List[Workload]:
    """Independent systems of uneven size: n per spin uniform in n_range, N = 3 n orbitals,
    n_det log-uniform in det_range (capped at a quarter of the distinct terms that orders
    1..kmax allow, so small systems stay drawable), orders geometric on 1..kmax,
    max(3, ceil(n / 8)) nuclei on a chain, W walkers each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_systems):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        N = 3 * n
        nd = int(round(math.exp(rng.uniform(math.log(det_range[0]), math.log(det_range[1])))))
        nd = max(1, min(nd, feasible_terms(n, N - n, 1, kmax) // 4))
        sub_seed = int(rng.integers(1 << 30))
        srng = np.random.default_rng(sub_seed)
        nuc = chain_nuclei(srng, max(3, -(-n // 8)))
        prob = make_problem(sub_seed, nuc, (n, n), (N, N), nd, geometric_orders(1, kmax), rng=srng,
                            name=f"batch{i}")
        R0 = initial_walkers(srng, nuc, prob.n_tot, W)
        out.append(Workload(problem=prob, R0=R0, tau=tau, seed=sub_seed, n_walkers=W, refresh_K=K, n_sweeps=1,
                            label=f"batch{i}"))
    return out


def custom_workload(n: Tuple[int, int], N: Tuple[int, int], n_det: int, orders: Dict[int, float],
                    W: int, n_nuc: int = 3, seed: int = 7, tau: float = 0.5, K: int = 1 << 30,
                    label: str = "custom") -> Workload:
    """A small problem of arbitrary shape (tests: ragged tails, edge cases)."""
    rng = np.random.default_rng(seed)
    nuc = chain_nuclei(rng, n_nuc)
    prob = make_problem(seed, nuc, n, N, n_det, orders, rng=rng, name=label)
    R0 = initial_walkers(rng, nuc, prob.n_tot, W)
    return Workload(problem=prob, R0=R0, tau=tau, seed=seed, n_walkers=W, refresh_K=K,
                    n_sweeps=1, label=label)


def full_ci_strings(n: int, N: int) -> List[Tuple[Tuple[int, ...], Tuple[int, ...]]]:
    """Every n-subset of N orbitals as a (holes, particles) string, reference first.

    The string for a subset S keeps the occupied orbitals of S in place and fills the
    holes (occupied orbitals not in S, ascending) with the virtuals in S (ascending).
    """
    import itertools
    out = []
    for S in itertools.combinations(range(N), n):
        occ = set(S)
        holes = tuple(c for c in range(n) if c not in occ)
        parts = tuple(j - n for j in S if j >= n)
        out.append((holes, parts))
    out.sort(key=lambda hp: (len(hp[0]), hp))
    return out


def strings_to_csr(strings):
    off = np.zeros(len(strings) + 1, np.int32)
    hs, ps = [], []
    for i, (h, p) in enumerate(strings):
        off[i + 1] = off[i] + len(h)
        hs.extend(h)
        ps.extend(p)
    return off, np.asarray(hs, np.uint8), np.asarray(ps, np.uint8)


def explicit_problem(nuc_xyz, bas_center, bas_lm, bas_alpha, B, n, strings_up, strings_dn,
                     det_up, det_dn, ci, name="explicit") -> Problem:
    """Assemble a Problem from explicit per-spin strings and terms (test fixtures)."""
    ou, hu, pu = strings_to_csr(strings_up)
    od, hd, pd = strings_to_csr(strings_dn)
    return Problem(n_elec=(int(n[0]), int(n[1])), n_orb=(int(B[0].shape[1]), int(B[1].shape[1])),
                   nuc_xyz=np.ascontiguousarray(nuc_xyz, np.float64),
                   bas_center=np.asarray(bas_center, np.int32), bas_lm=np.asarray(bas_lm, np.int8),
                   bas_alpha=np.asarray(bas_alpha, np.float64),
                   B=(np.ascontiguousarray(B[0], np.float64), np.ascontiguousarray(B[1], np.float64)),
                   exc_off=(ou, od), exc_holes=(hu, hd), exc_parts=(pu, pd),
                   det_up=np.asarray(det_up, np.int32), det_dn=np.asarray(det_dn, np.int32),
                   ci=np.asarray(ci, np.float64), name=name)
