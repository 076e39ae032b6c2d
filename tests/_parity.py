"""Shared GPU-vs-oracle replay for the parity tests.

The CUDA path and the oracle see the same seeded proposals.  Accept decisions are the
Metropolis test u < ratio^2 on the GPU's ratio and are applied to both sides, so both
follow one trajectory ("replay").  Each reported result X (ratio, gradient component,
laplacian) is compared element by element:

    |X_gpu - X_oracle| <= tol * max(|X_oracle|, scale_X)

where scale_X = sum_I |c_I X_I| / |Psi| is the cancellation scale of the CI sum that forms
X (the oracle returns it), so a result that is a small difference of large terms is judged
against the size of the terms, as FP64 rounding of those terms allows nothing tighter.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

import oracle
from paper_1106_2456_gb300 import msd


def rel_err(x: np.ndarray, ref: np.ndarray, scale: np.ndarray) -> np.ndarray:
    return np.abs(x - ref) / np.maximum(np.abs(ref), scale)


U64 = 2.0 ** -53
U32 = 2.0 ** -24


def tol_fp64(kappa):
    """FP64 bar: 1e-10 while cond(A_0) <= 3e3; beyond that the table method's error grows
    with cond(A_0) (every quantity passes through A_0^{-1}; Section V), ~3e-14 * kappa."""
    return 1e-10 * np.maximum(1.0, np.asarray(kappa) / 3e3)


def tol_mixed(kappa):
    """Mixed bar: FP32 rounding amplified by cond(A_0): 1e3 * u_fp32 * max(kappa, 10)."""
    return 1e3 * U32 * np.maximum(np.asarray(kappa), 10.0)


def replay(wl, precision: str, n_steps: int, check: Optional[Sequence[int]] = None, refresh_K: Optional[int] = None,
           elec_order: Optional[Sequence[int]] = None, step_offset: int = 0) -> Dict[str, List[float]]:
    """Run n_steps single-electron moves on the GPU for all walkers; compare the walkers in
    `check` (default: all) with the oracle after every step.  Returns, per result kind and
    per step, the worst relative error and the worst ratio of error to the tolerance of the
    precision at that walker's conditioning (<= 1 passes)."""
    tol_fn = tol_mixed if precision == "mixed" else tol_fp64
    p = wl.problem
    W = wl.n_walkers
    idx = np.arange(W) if check is None else np.asarray(check)
    K = wl.refresh_K if refresh_K is None else refresh_K
    ctx = msd.MSD(p, W, precision, refresh_K=K)
    R = torch.tensor(wl.R0, device="cuda")
    ctx.set_positions(R)
    orc = oracle.Oracle(p)
    Rh = wl.R0.copy()
    cur = orc.eval(Rh[idx])
    # initial log|Psi| and sign
    _, la, sg = ctx.get_state()
    out = dict(ratio=[], grad=[], lap=[], logabs=[], sign_ok=[], accept=[], ratio_n=[], grad_n=[], lap_n=[],
               kappa=[])
    # |d log|Psi|| is the relative error of Psi: judged like the ratio, against the bar at the
    # walker's conditioning times the cancellation scale of the CI sum
    kap0 = np.array([orc.reference_condition(Rh[w_]) for w_ in idx])
    out["logabs0"] = float(np.max(np.abs(la.cpu().numpy()[idx] - cur["logabs"]) /
                                  (tol_fn(kap0) * np.maximum(1.0, cur["absum"][:, 0]))))
    out["sign0_ok"] = bool(np.all(sg.cpu().numpy()[idx] == cur["sign"]))
    eta, u = wl.proposals(n_steps + step_offset)
    eta, u = eta[step_offset:], u[step_offset:]
    order = list(range(p.n_tot)) if elec_order is None else list(elec_order)
    for t in range(n_steps):
        e = order[t % len(order)]
        rnew = Rh[:, e] + wl.tau * eta[t]
        ratio, grad, lap = ctx.ratio(e, torch.tensor(rnew, device="cuda"))
        g_r = ratio.cpu().numpy()
        g_g = grad.cpu().numpy()
        g_l = lap.cpu().numpy()
        r_or, new = orc.ratio(Rh[idx], e, rnew[idx], cur)
        ab = new["absum"]
        kap = np.array([orc.reference_condition(Rh[w_], e, rnew[w_]) for w_ in idx])
        tol = tol_fn(kap)
        er = rel_err(g_r[idx], r_or, ab[:, 0] * np.abs(r_or))
        eg = rel_err(g_g[idx], new["grad"], ab[:, 1:4]).max(axis=1)
        el = rel_err(g_l[idx], new["lap"], ab[:, 4])
        for key, v in (("ratio", er), ("grad", eg), ("lap", el)):
            out[key].append(float(v.max()))
            out[key + "_n"].append(float((v / tol).max()))
        out["kappa"].append(float(kap.max()))
        acc = u[t] < g_r * g_r
        out["accept"].append(float(acc.mean()))
        ctx.accept(e, torch.tensor(acc.astype(np.uint8), device="cuda"))
        Rh[acc, e] = rnew[acc]
        a_i = acc[idx]
        cur = dict(logabs=np.where(a_i, new["logabs"], cur["logabs"]), sign=np.where(a_i, new["sign"], cur["sign"]))
    ctx.sync()
    Rg, la, sg = ctx.get_state()
    out["R_final_err"] = float(np.max(np.abs(Rg.cpu().numpy() - Rh)))
    kapf = np.array([orc.reference_condition(Rh[w_]) for w_ in idx])
    fin = orc.eval(Rh[idx])
    out["logabs_final"] = float(np.max(np.abs(la.cpu().numpy()[idx] - cur["logabs"]) /
                                       (100 * tol_fn(kapf) * np.maximum(1.0, fin["absum"][:, 0]))))
    out["sign_final_ok"] = bool(np.all(sg.cpu().numpy()[idx] == cur["sign"]))
    ctx.close()
    return out
