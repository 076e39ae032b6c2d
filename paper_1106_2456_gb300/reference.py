"""Reference-determinant switching (Section V).

The table method keeps A_0^{-1} of one reference determinant per spin.  Section V notes that
A_0 can become (nearly) singular while other determinants of the expansion keep Psi away
from zero, so such a move is accepted, and proposes switching, for a while, to another
determinant of the expansion as the reference.  The excitations relative to the new
reference may be larger (by the new reference's own excitation order).

:func:`switch_reference` rewrites a problem so that the determinants of term I become the
reference of each spin, with Psi unchanged:

* The orbitals of each spin are relabelled. The new reference's orbitals, in its column
  order, become orbitals 0..n-1; the remaining orbitals follow in ascending old index as the
  virtuals.  B's columns are permuted the same way.
* Every string's determinant is the same set of orbitals.  It is re-expressed in the
  library's convention: the holes h_1 < ... < h_k of the new reference are replaced in
  place by the particles p_1 < ... < p_k.  Reordering columns multiplies a determinant by
  the sign of the permutation.  That sign is folded into the CI coefficient of every term
  that uses the string.

The new problem goes to ``msd_init`` like any other.  Nothing here runs on the GPU.
The function is a host-side re-plan that a driver applies when ``msd_sync`` reports
MSD_ERR_SINGULAR or the reference becomes ill-conditioned.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from .workloads import MAXK, Problem, strings_to_csr


def string_columns(n: int, holes: Sequence[int], parts: Sequence[int]) -> List[int]:
    """Orbital held by each column c = 0..n-1 of a string's determinant: c itself, or
    n + p_q where c = h_q (in-place replacement, sorted holes paired with sorted particles)."""
    cols = list(range(n))
    for h, p in zip(holes, parts):
        cols[h] = n + p
    return cols


def permutation_sign(a: Sequence[int], b: Sequence[int]) -> int:
    """Sign of the permutation taking the sequence b to the sequence a (same elements)."""
    pos = {v: i for i, v in enumerate(b)}
    perm = [pos[v] for v in a]
    seen = [False] * len(perm)
    sign = 1
    for i in range(len(perm)):
        if seen[i]:
            continue
        j, length = i, 0
        while not seen[j]:
            seen[j] = True
            j = perm[j]
            length += 1
        if length % 2 == 0:
            sign = -sign
    return sign


def canonical_string(n: int, cols: Sequence[int]) -> Tuple[Tuple[int, ...], Tuple[int, ...], int]:
    """(holes, particles, sign) of the string whose in-place determinant holds the orbitals
    `cols` (a set of n distinct orbitals, any column order): det[cols] = sign det[canonical]."""
    occ = set(cols)
    holes = tuple(c for c in range(n) if c not in occ)
    parts = tuple(sorted(o - n for o in occ if o >= n))
    canon = string_columns(n, holes, parts)
    return holes, parts, permutation_sign(cols, canon)


def _strings(problem: Problem, s: int):
    off, H, P = problem.exc_off[s], problem.exc_holes[s], problem.exc_parts[s]
    return [(tuple(int(x) for x in H[off[u]:off[u + 1]]), tuple(int(x) for x in P[off[u]:off[u + 1]]))
            for u in range(len(off) - 1)]


def switch_reference(problem: Problem, term: int) -> Problem:
    """The same wavefunction with the determinants of `term` as the reference of each spin.

    Raises ValueError if a string's order relative to the new reference exceeds the
    library's largest order (8).
    """
    if not 0 <= term < problem.n_det:
        raise ValueError(f"term {term} out of range")
    ref = (int(problem.det_up[term]), int(problem.det_dn[term]))
    new_B, new_strings, signs = [], [], []
    for s in range(2):
        n, N = problem.n_elec[s], problem.n_orb[s]
        strings = _strings(problem, s)
        ref_cols = string_columns(n, *strings[ref[s]])
        rest = [o for o in range(N) if o not in set(ref_cols)]
        old_of_new = ref_cols + rest            # new orbital index -> old orbital index
        new_of_old = np.empty(N, dtype=np.int64)
        new_of_old[old_of_new] = np.arange(N)
        new_B.append(np.ascontiguousarray(problem.B[s][:, old_of_new]))
        out, sg = [], []
        for h, p in strings:
            cols = [int(new_of_old[o]) for o in string_columns(n, h, p)]
            hh, pp, sign = canonical_string(n, cols)
            if len(hh) > MAXK:
                raise ValueError(f"spin {s}: a string has order {len(hh)} > {MAXK} relative to the new reference")
            out.append((hh, pp))
            sg.append(sign)
        # the library wants string 0 to be the reference: swap it into place
        r = ref[s]
        order = list(range(len(out)))
        order[0], order[r] = order[r], order[0]
        remap = np.empty(len(out), dtype=np.int64)
        remap[order] = np.arange(len(out))
        new_strings.append(([out[u] for u in order], remap))
        signs.append(np.asarray(sg, dtype=np.float64))
    (su, mu), (sd, md) = new_strings
    ou, hu, pu = strings_to_csr(su)
    od, hd, pd = strings_to_csr(sd)
    up = problem.det_up.astype(np.int64)
    dn = problem.det_dn.astype(np.int64)
    ci = problem.ci * signs[0][up] * signs[1][dn]
    return Problem(n_elec=problem.n_elec, n_orb=problem.n_orb, nuc_xyz=problem.nuc_xyz,
                   bas_center=problem.bas_center, bas_lm=problem.bas_lm, bas_alpha=problem.bas_alpha,
                   B=(new_B[0], new_B[1]), exc_off=(ou, od), exc_holes=(hu, hd), exc_parts=(pu, pd),
                   det_up=mu[up].astype(np.int32), det_dn=md[dn].astype(np.int32), ci=ci.astype(np.float64),
                   name=f"{problem.name} (reference: term {term})")


def heaviest_term(problem: Problem) -> int:
    """The non-reference term with the largest |c_I|: a default choice of new reference (the
    paper does not say which determinant to switch to)."""
    w = np.abs(problem.ci).copy()
    w[(problem.det_up == 0) & (problem.det_dn == 0)] = -1.0
    return int(np.argmax(w))
