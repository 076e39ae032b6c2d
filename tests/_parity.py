"""Shared GPU-vs-oracle replay for the parity tests.

The CUDA path and the oracle see the same seeded proposals.  Accept decisions are the
Metropolis test u < ratio^2 on the GPU's ratio and are applied to both sides, so both
follow one trajectory ("replay").  Each reported result X (ratio, gradient component,
laplacian) is compared element by element:

    |X_gpu - X_oracle| <= tol * max(|X_oracle|, scale_X)

where scale_X = sum_I |c_I X_I| / |Psi| is the cancellation scale of the CI sum that forms
X (the oracle returns it), so a result that is a small difference of large terms is judged
against the size of the terms, as FP64 rounding of those terms allows nothing tighter.

Every result is also classified (``bar_report``): whether it meets the flat bar (1e-10 for
FP64, i.e. the kappa-independent constant), whether it needed the kappa scaling to pass, and
its plain relative error |X_gpu - X_oracle| / |X_oracle|.  Setting MSD_PARITY_REPORT to a file
path appends one JSON line per replay with that classification.
"""
from __future__ import annotations

import json
import os
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
    """FP64 bar: 1e-10, the flat bar, while cond(A_0) <= 3e3; beyond that it may grow as
    1e-10 kappa / 3e3 (every quantity of the table method passes through A_0^{-1}; Section V
    names this instability), and the tests cap how many results may use that allowance
    (KAPPA_ONLY_SHARE).  Measured on the FP64 water walk the error does not grow with kappa
    (max 1e-11 up to kappa = 1e6); one result in about 1e5 of the GPU tests needs the allowance."""
    return 1e-10 * np.maximum(1.0, np.asarray(kappa) / 3e3)


def tol_mixed(kappa):
    """Mixed bar: 3e-3, the flat bar, or 10 u_fp32 kappa where that is larger (FP32 rounding of
    the orbitals and the table amplified by cond(A_0) through T = A_0^{-1} Phi_virt).  Measured
    on the mixed walks of the GPU tests the error stays below 1.3e-3 (gradients; 2.5e-4 for
    ratios and laplacians) at every kappa up to 1e6."""
    return np.maximum(3e-3, 10.0 * U32 * np.asarray(kappa))


FLAT = {"fp64": 1e-10, "mixed": 3e-3}
# Largest share of a test's results that may pass only through the kappa allowance of the bar.
KAPPA_ONLY_SHARE = {"fp64": 1e-3, "mixed": 2e-2}
KAPPA_EDGES = (0.0, 1e2, 1e3, 1e4, 1e5, 1e6, 1e7, 1e8, float("inf"))


def bar_report(out, precision: str, label: str = "") -> Dict:
    """Classify every compared result of a replay: how many meet the flat bar (FLAT), how many
    pass only through the kappa allowance, how many fail; the worst plain relative error overall
    and among well-conditioned results with little cancellation (kappa <= 3e3, scale_X <= 10 |X|),
    and the largest kappa seen."""
    flat = FLAT[precision]
    rep = {"label": label, "precision": precision}
    for key in ("ratio", "grad", "lap"):
        es = np.concatenate(out["rec"][key]["scaled"]) if out["rec"][key]["scaled"] else np.zeros(0)
        ep = np.concatenate(out["rec"][key]["plain"]) if out["rec"][key]["plain"] else np.zeros(0)
        kp = np.concatenate(out["rec"][key]["kappa"]) if out["rec"][key]["kappa"] else np.zeros(0)
        sc = np.concatenate(out["rec"][key]["canc"]) if out["rec"][key]["canc"] else np.zeros(0)
        tol = (tol_mixed if precision == "mixed" else tol_fp64)(kp)
        flat_ok = es <= flat
        ok = es <= tol
        plain_sel = (kp <= 3e3) & (sc <= 10.0)
        rep[key] = {"n": int(es.size), "flat_pass": int(flat_ok.sum()), "kappa_only": int((ok & ~flat_ok).sum()),
                    "fail": int((~ok).sum()), "max_scaled": float(es.max(initial=0.0)),
                    "max_plain": float(ep.max(initial=0.0)),
                    "n_plain_well": int(plain_sel.sum()),
                    "max_plain_well": float(ep[plain_sel].max(initial=0.0)),
                    "max_kappa": float(kp.max(initial=0.0)),
                    "by_kappa": [{"kappa_le": hi, "n": int(((kp > lo) & (kp <= hi)).sum()),
                                  "max_scaled": float(es[(kp > lo) & (kp <= hi)].max(initial=0.0))}
                                 for lo, hi in zip(KAPPA_EDGES[:-1], KAPPA_EDGES[1:])
                                 if ((kp > lo) & (kp <= hi)).any()]}
    path = os.environ.get("MSD_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rep) + "\n")
    return rep


def replay(wl, precision: str, n_steps: int, check: Optional[Sequence[int]] = None, refresh_K: Optional[int] = None,
           elec_order: Optional[Sequence[int]] = None, step_offset: int = 0, setup=None,
           bar: Optional[str] = None) -> Dict[str, List[float]]:
    """Run n_steps single-electron moves on the GPU for all walkers; compare the walkers in
    `check` (default: all) with the oracle after every step.  Returns, per result kind and
    per step, the worst relative error and the worst ratio of error to the tolerance of the
    precision at that walker's conditioning (<= 1 passes).  setup(ctx) runs before the positions
    are set; bar ("fp64" or "mixed") overrides the precision whose bar is applied."""
    tol_fn = tol_mixed if (bar or precision) == "mixed" else tol_fp64
    p = wl.problem
    W = wl.n_walkers
    idx = np.arange(W) if check is None else np.asarray(check)
    K = wl.refresh_K if refresh_K is None else refresh_K
    ctx = msd.MSD(p, W, precision, refresh_K=K)
    if setup is not None:
        setup(ctx)
    R = torch.tensor(wl.R0, device="cuda")
    ctx.set_positions(R)
    out_ctx_stats = ctx.rescue_stats() if precision == "mixed" else None
    orc = oracle.Oracle(p)
    Rh = wl.R0.copy()
    cur = orc.eval(Rh[idx])
    # initial log|Psi| and sign
    _, la, sg = ctx.get_state()
    out = dict(ratio=[], grad=[], lap=[], logabs=[], sign_ok=[], accept=[], ratio_n=[], grad_n=[], lap_n=[],
               kappa=[], rec={k: dict(scaled=[], plain=[], kappa=[], canc=[]) for k in ("ratio", "grad", "lap")})
    # |d log|Psi|| is the relative error of Psi: judged like the ratio, against the bar at the
    # walker's conditioning times the cancellation scale of the CI sum
    kap0 = np.array([orc.reference_condition(Rh[w_]) for w_ in idx])
    out["logabs0"] = float(np.max(np.abs(la.cpu().numpy()[idx] - cur["logabs"]) /
                                  (tol_fn(kap0) * np.maximum(1.0, cur["absum"][:, 0]))))
    out["sign0_ok"] = bool(np.all(sg.cpu().numpy()[idx] == cur["sign"]))
    out["rescue0"] = out_ctx_stats
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
        tiny = 1e-300
        plain = {"ratio": np.abs(g_r[idx] - r_or) / np.maximum(np.abs(r_or), tiny),
                 "grad": (np.abs(g_g[idx] - new["grad"]) / np.maximum(np.abs(new["grad"]), tiny)).max(axis=1),
                 "lap": np.abs(g_l[idx] - new["lap"]) / np.maximum(np.abs(new["lap"]), tiny)}
        canc = {"ratio": ab[:, 0],
                "grad": (ab[:, 1:4] / np.maximum(np.abs(new["grad"]), tiny)).max(axis=1),
                "lap": ab[:, 4] / np.maximum(np.abs(new["lap"]), tiny)}
        for key, v in (("ratio", er), ("grad", eg), ("lap", el)):
            out[key].append(float(v.max()))
            out[key + "_n"].append(float((v / tol).max()))
            out["rec"][key]["scaled"].append(v)
            out["rec"][key]["plain"].append(plain[key])
            out["rec"][key]["kappa"].append(kap)
            out["rec"][key]["canc"].append(canc[key])
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
