"""Metropolis VMC energy driver for Psi_T = exp(J) Psi_MD on one GPU.

Section II: a Metropolis step proposes moving one electron and accepts with probability
min(1, |Psi_T(R') / Psi_T(R)|^2); a sweep moves every electron once.  Section VI estimates
VMC energies of a Jastrow-multideterminant wavefunction.  Every step runs in libmsd kernels
(``msd_propose``, ``msd_ratio``, ``msd_jastrow_ratio``, ``msd_metropolis``, ``msd_accept``,
and ``msd_local_energy`` after each sweep); this module only orders the calls and supplies
the random numbers (a seeded torch generator on the device, or arrays the caller passes).
"""
from __future__ import annotations

from typing import Dict, Optional

import numpy as np
import torch

from .msd import MSD


def blocking_stderr(series, min_blocks: int = 16) -> float:
    """Standard error of the mean of a serially correlated series by blocking (Flyvbjerg and
    Petersen, J. Chem. Phys. 91, 461 (1989)).

    Neighbouring values are averaged in pairs, level after level.  The naive error of the
    blocked series grows until the blocks outlast the correlation time, then levels off.
    Returns the largest naive estimate over the levels that keep at least `min_blocks`
    blocks, and always includes level 0.  With fewer than 2 values the error is undefined
    (nan).
    """
    x = np.asarray(series, dtype=np.float64).ravel()
    if x.size < 2:
        return float("nan")
    best = float(x.std(ddof=1) / np.sqrt(x.size))
    while x.size // 2 >= min_blocks:
        h = x.size // 2
        x = 0.5 * (x[0:2 * h:2] + x[1:2 * h:2])
        best = max(best, float(x.std(ddof=1) / np.sqrt(x.size)))
    return best


def combine_replicas(sweep_sums: torch.Tensor, n_walkers: int, n_accepted: float, n_proposed: float):
    """Per-sweep mean energies over the walkers of every replica, and the overall acceptance.

    Each process runs its own walkers (independent Markov chains); when torch.distributed is
    initialised, one all-reduce of [per-sweep energy sums, walker count, accepted, proposed]
    per run combines them.  This is the only exchange of a replicated run, and it lies
    outside the moves.  The tensor must be on the device the process group uses.  Returns
    (means [n_sweeps], acceptance).
    """
    v = torch.cat([sweep_sums.to(torch.float64).ravel(),
                   torch.tensor([float(n_walkers), float(n_accepted), float(n_proposed)], dtype=torch.float64,
                                device=sweep_sums.device)])
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(v)
    k = sweep_sums.numel()
    means = v[:k] / v[k]
    acc = float(v[k + 1] / v[k + 2]) if float(v[k + 2]) > 0 else float("nan")
    return means, acc


class VMC:
    """Drive a walker population of an :class:`MSD` context.

    Z: nuclear charges [n_nuc] in the order of the problem's nuclei; b_ee, b_en: Pade-Jastrow
    parameters (0 removes a term); tau: Gaussian proposal width (bohr).  The context must
    hold positions (``set_positions``) before the first sweep.
    """

    def __init__(self, ctx: MSD, Z, b_ee: float = 0.0, b_en: float = 0.0, tau: float = 0.5, seed: int = 0):
        self.ctx = ctx
        self.tau = float(tau)
        self.jastrow = b_ee > 0.0 or b_en > 0.0
        ctx.set_hamiltonian(Z, b_ee, b_en)
        W, dev = ctx.W, ctx.dev
        self.rnew = torch.empty((W, 3), dtype=torch.float64, device=dev)
        self.ratio = torch.empty(W, dtype=torch.float64, device=dev)
        self.acc = torch.empty(W, dtype=torch.uint8, device=dev)
        self.n_acc = torch.zeros(W, dtype=torch.float64, device=dev)
        self.n_prop = 0
        self.eloc = torch.empty(W, dtype=torch.float64, device=dev)
        self.gen = torch.Generator(device=dev)
        self.gen.manual_seed(int(seed))

    def sweep(self, eta: Optional[torch.Tensor] = None, u: Optional[torch.Tensor] = None):
        """Move electrons 0 .. n_tot - 1 in order (up electrons first).  eta [n_tot, W, 3] and
        u [n_tot, W] on the device override the generator."""
        c = self.ctx
        W = c.W
        for e in range(c.n_tot):
            if eta is None:
                eta_e = torch.randn((W, 3), generator=self.gen, dtype=torch.float64, device=c.dev)
                u_e = torch.rand(W, generator=self.gen, dtype=torch.float64, device=c.dev)
            else:
                eta_e, u_e = eta[e], u[e]
            c.propose(e, eta_e, self.tau, self.rnew)
            c.ratio_into(e, self.rnew, self.ratio)
            if self.jastrow:
                c.jastrow_ratio_(e, self.rnew, self.ratio)
            c.metropolis(u_e, self.ratio, self.acc)
            c.accept(e, self.acc)
            self.n_acc += self.acc
        self.n_prop += c.n_tot

    def energy(self) -> torch.Tensor:
        """Local energies [W] at the current positions (a view of an internal buffer)."""
        self.ctx.local_energy_into(self.eloc)
        return self.eloc

    def run(self, n_sweeps: int, n_equil: int = 0) -> Dict[str, float]:
        """n_equil sweeps without measurement, then n_sweeps with E_L after each.  Returns the
        mean energy over all walkers (of every replica, when torch.distributed is initialised),
        its standard error by blocking the per-sweep means (successive sweeps are correlated),
        and the acceptance ratio of the measured sweeps."""
        for _ in range(n_equil):
            self.sweep()
        self.n_acc.zero_()
        self.n_prop = 0
        sums = []
        for _ in range(n_sweeps):
            self.sweep()
            sums.append(self.energy().sum())
        if not sums:
            return dict(energy=float("nan"), stderr=float("nan"), acceptance=float("nan"), sweeps=0)
        means, acc = combine_replicas(torch.stack(sums), self.ctx.W, float(self.n_acc.sum().item()),
                                      float(self.n_prop * self.ctx.W))
        m = means.cpu().numpy()
        return dict(energy=float(m.mean()), stderr=blocking_stderr(m), acceptance=acc, sweeps=int(n_sweeps))
