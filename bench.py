#!/usr/bin/env python
"""Throughput of the multi-determinant table method: walker-moves per second.

One step = one Metropolis sweep of every walker: each of the n_tot electrons in index order
is proposed r' = r + tau * eta, gets msd_ratio (ratio, gradient and laplacian at r'), the
Metropolis test and msd_accept (Sherman-Morrison update).  A sweep of the default workload
therefore holds 128 single-electron moves per walker, the from-scratch refresh of each spin
(every K = 64 of its moves) and the CI contraction at each of the two spin changes, so
every timed window, however many steps it spans, contains exactly the amortised share of
that work.  The line reports how many refreshes and CI contractions fell inside it.

Default workload (64 + 64 electrons, 256 orbitals per spin, 144 Gaussians, 1e5
determinants with excitation orders 1-8, 4096 walkers), synthetic and seeded.  The
headline value is the mixed-precision path; the same line reports the FP64 path, the
per-result difference between the two over a whole sweep, the excitation-sweep kernel's
roofline fraction, an end-to-end number through the host-buffer C ABI, and the FP64 CPU
oracle timed on a bounded sample (walker-moves of one walker) on this machine's cores.

--impl reference times the oracle alone (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "walker-moves/sec (ratio+grad+lap) at 128 e-, 1e5 dets; mixed vs FP64, % roofline"
UNIT = "walker-moves/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# FP32 ALU peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# FP64 ALU nominal rate of GB300 (no FP64 tensor path is used)
FP64_ALU_TFLOPS = 1.25


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


# ----------------------------------------------------------------------------------------
# work model of the excitation-sweep kernel (one launch = all walkers, one moved electron)
# ----------------------------------------------------------------------------------------
def exc_flops(k: int) -> float:
    """Flops of one excitation of order k in the sweep (FMA = 2): the pivoted elimination of
    k - 2 columns, three FMA-corrected 2 x 2 determinants (6 flops each), the back
    substitution of z = det T_u^{-1} x_u, and the accumulation C det into S_T and C z into G."""
    if k <= 1:
        return 4.0
    f = 18.0
    for j in range(k - 2):
        r = k - 1 - j
        f += r + 2.0 * r * r + 2.0 * r + 1.0   # multipliers, Schur update, right-hand side, 1/u_jj
    f += (k - 2) + 1 + 2                       # product of pivots, det, scaling of z_2
    for q in range(k - 2):
        f += 2 + 2.0 * (k - 1 - q)             # back substitution of z_1
    return f + 2.0 + 2.0 * k


def sweep_work(problem, spin: int, W: int, mixed: bool, n_exc_internal: int):
    """Algorithmic flops and HBM bytes of one excitation-sweep launch (all W walkers).

    Per walker: sum over strings of exc_flops(k) (dense singles: 4 per table entry), 2 n m for
    T G, 2 n m for the kept y^0 row, 10 (n + m) for the five channel dot products and 10 n for
    rho and s^a.  Bytes per walker: the C stream (one value per internal string, padding
    included), the table T, the column of A_0^{-1}, the five orbital rows at r' and the y^0 row
    written; the excitation records once per launch.
    """
    n, N = problem.n_elec[spin], problem.n_orb[spin]
    m = N - n
    hist = np.bincount(problem.exc_orders(spin), minlength=9)
    dense = hist[1] > 0 and 4 * hist[1] >= n * m
    f = 4.0 * n * m if dense else hist[1] * exc_flops(1)
    f += sum(int(hist[q]) * exc_flops(q) for q in range(2, 9))
    f += 4.0 * n * m + 10.0 * (n + m) + 10.0 * n
    b = 4 if mixed else 8
    per_walker = n_exc_internal * b + n * m * b + n * 8 + 5 * N * b + m * b + 6 * 8
    lists = sum(int(hist[q]) * (2 if q <= 1 else 4 if q == 2 else 8 if q <= 4 else 16) for q in range(1, 9))
    return f * W, per_walker * W + lists


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")
SWEEP_SOURCES = ("msd_smalldet.cuh", "msd_records.cuh")
SWEEP_SECTION = ("// A2-A5: reference ratio, excitation sweep", "// A6: accept")


def sweep_source_hash() -> str:
    """SHA-256 (first 16 hex digits) of the code the sweep kernel is compiled from: its section of
    msd_kernels.cu (from the A2-A5 banner to the A6 banner) and the headers it includes."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_1106_2456_gb300", "csrc")
    h = hashlib.sha256()
    with open(os.path.join(csrc, "msd_kernels.cu")) as f:
        text = f.read()
    a, b = text.index(SWEEP_SECTION[0]), text.index(SWEEP_SECTION[1])
    h.update(text[a:b].encode())
    for name in SWEEP_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(mixed: bool):
    """DRAM bytes per walker of one sweep-kernel launch from profiles/traffic.json (written from an
    ncu capture, with the capture's command), or None when there is none for this precision or
    the kernel's sources changed since the counters were taken."""
    if not os.path.exists(TRAFFIC_JSON):
        return None
    with open(TRAFFIC_JSON) as f:
        d = json.load(f)
    rec = d.get("k_ratio_mixed" if mixed else "k_ratio_fp64")
    if not rec or rec.get("source_hash") != sweep_source_hash():
        return None
    rec = dict(rec)
    rec["file"] = "profiles/traffic.json"
    return rec


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while running; summarised over a time window."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(device_index)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self, t0: float, t1: float):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                    rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[5:10]))
                except (ValueError, IndexError):
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if t0 - 0.25 <= r[0] <= t1 + 0.25]
        if not inside:
            inside = sorted(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))[:2]
        names = ("active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for r in inside:
            for nm, v in zip(names[1:], r[3][1:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_inputs(wl, rank: int, total: int):
    """Walker positions and Metropolis streams of one replica: rank 0 runs the workload's own
    seeds, rank r > 0 offset seeds and positions jittered by 0.01 bohr (independent chains)."""
    rng = np.random.default_rng(4242 + rank)
    R0 = wl.R0 + (0.01 * rng.standard_normal(wl.R0.shape) if rank else 0.0)
    eta, u = wl.proposals(total, seed_offset=rank)
    return R0, eta, u


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks (the job's time is its slowest replica's)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(walkers_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job walker-moves per second: every replica's walkers over the slowest time."""
    return walkers_per_rank * world * steps / seconds


# ----------------------------------------------------------------------------------------
# the oracle arm (CPU, FP64, every determinant by LU)
# ----------------------------------------------------------------------------------------
def oracle_rate(wl, n_moves: int, time_cap: float):
    """Walker-moves/s of the FP64 oracle on one walker: each move evaluates Psi, grad and
    lap at the proposed position from scratch and takes the ratio to the stored Psi."""
    import oracle as orc

    o = orc.Oracle(wl.problem)
    R = wl.R0[:1].copy()
    cur = o.eval(R)
    eta, u = wl.proposals(max(n_moves, 1), seed_offset=99)
    done = 0
    t0 = time.perf_counter()
    for t in range(n_moves):
        e = t % wl.problem.n_tot
        rnew = R[:, e] + wl.tau * eta[t, :1]
        ratio, new = o.ratio(R, e, rnew, cur)
        if u[t, 0] < ratio[0] ** 2:
            R[0, e] = rnew[0]
            cur = dict(logabs=new["logabs"], sign=new["sign"])
        done += 1
        if time.perf_counter() - t0 > time_cap:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt, orc.num_threads()


def workload_desc(name, wl):
    p = wl.problem
    return (f"{name}: {p.n_elec[0]}+{p.n_elec[1]} electrons, {p.n_orb[0]} orbitals per spin, {p.n_basis} "
            f"Gaussians, {p.n_det} determinants ({p.n_exc(0)}+{p.n_exc(1)} unique strings), {wl.n_walkers} walkers "
            f"per GPU, refresh every {wl.refresh_K} steps of a spin")


def batched_desc(systems, walkers_per_system):
    dets = sum(w.problem.n_det for w in systems)
    ns = [w.problem.n_elec[0] for w in systems]
    return (f"batched: {len(systems)} systems, n per spin {min(ns)}-{max(ns)}, N = 3n, {dets} determinants in total "
            f"(log-uniform 1e2-1e5 per system, orders 1-6), {walkers_per_system} walkers per system "
            f"({walkers_per_system * len(systems)} per GPU)")


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    from paper_1106_2456_gb300 import workloads

    if args.workload == "batched":
        # the oracle on the largest system of the batch (its slowest single-walker moves)
        systems = workloads.batched_workloads(args.systems, W=2, seed=1004)
        desc = batched_desc(systems, args.walkers or 256)
        wl = max(systems, key=lambda w: w.problem.n_det * w.problem.n_elec[0] ** 3)
    else:
        full = workloads.make_workload(args.workload, **({"n_walkers": args.walkers} if args.walkers else {}))
        desc = workload_desc(args.workload, full)
        wl = workloads.make_workload(args.workload, n_walkers=2)
    warm = min(args.warmup, 1)
    if warm:
        oracle_rate(wl, warm, 60.0)
    rate, done, dt, cores = oracle_rate(wl, args.steps, args.ref_time_cap)
    sample = (f"{done} single-walker moves (ratio + grad + lap, every determinant by LU) of the "
              f"{args.workload} workload, {dt:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws, "steps": done,
            "warmup": warm, "ms_per_step": 1e3 * dt / max(done, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "walkers_per_step": 1,
                       "precision": "fp64 (oracle: every determinant by LU)"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
# the CUDA arm
# ----------------------------------------------------------------------------------------
def run_batched(args):
    """Batched uneven systems (one context over many systems): walker-moves/s of all systems."""
    import torch

    from paper_1106_2456_gb300 import msd, workloads
    import __graft_entry__

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    msd.load_library()
    peaks, peak_kind = load_peaks()
    systems = workloads.batched_workloads(args.systems, W=args.walkers or 256, seed=1004)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    W = sum(w.n_walkers for w in systems)
    total = args.warmup + args.steps
    rng = np.random.default_rng(77 + rank)
    eta = torch.tensor(rng.standard_normal((total, W, 3)), device=dev)
    u = torch.tensor(rng.random((total, W)), device=dev)
    R0 = torch.tensor(np.concatenate([w.R0.reshape(-1) for w in systems]), device=dev)
    bufs = dict(rnew=torch.empty(W, 3, dtype=torch.float64, device=dev),
                ratio=torch.empty(W, dtype=torch.float64, device=dev),
                grad=torch.empty(W, 3, dtype=torch.float64, device=dev),
                lap=torch.empty(W, dtype=torch.float64, device=dev),
                acc=torch.empty(W, dtype=torch.uint8, device=dev))

    def run(prec, steps, rescue_slots=0):
        b = msd.MSDBatch([w.problem for w in systems], [w.n_walkers for w in systems], prec,
                         refresh_K=[w.refresh_K for w in systems], stream=stream)
        if rescue_slots:
            b.set_rescue(rescue_slots)
        b.set_positions(R0)

        def step(t):
            if args.separate:
                b.propose(t, eta[t], 0.5, bufs["rnew"])
                b.ratio_into(t, bufs["rnew"], bufs["ratio"], bufs["grad"], bufs["lap"])
                b.metropolis(u[t], bufs["ratio"], bufs["acc"])
                b.accept(t, bufs["acc"])
            else:  # msd_step: one persistent launch per group of systems (grid sizes tuned on warm-up)
                b.step(t, eta[t], 0.5, u[t], bufs["ratio"], bufs["grad"], bufs["lap"], bufs["acc"])

        for t in range(args.warmup):
            step(t)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clk = ClockSampler(local) if rank == 0 else None
        time.sleep(0.3 if clk else 0)
        b.timing_start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        e0.record(stream)
        for t in range(args.warmup, args.warmup + steps):
            step(t)
        e1.record(stream)
        torch.cuda.synchronize()
        w1 = time.time()
        sweep_ms, n_sweep, n_launch = b.timing_stop()
        if clk:
            clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        # a walker whose reference matrix becomes nearly singular (Section V) is held in FP64 on the
        # FP32 path; anything still non-finite is flagged by the library and reported here
        try:
            b.sync()
            flagged = None
        except msd.MSDError as ex:
            flagged = str(ex)
        rescue = b.rescue_stats() if rescue_slots else None
        b.close()
        # algorithmic work of every system's sweeps in these steps
        F = B = 0.0
        for w in systems:
            p = w.problem
            plan = msd.describe(p, prec)
            for t in range(args.warmup, args.warmup + steps):
                sp = p.spin_of(t % p.n_tot)
                f, by = sweep_work(p, sp, w.n_walkers, prec == "mixed", int(plan[sp][0]))
                F += f
                B += by
        return ms, sweep_ms, n_sweep, n_launch, F, B, (clk.summary(w0, w1) if clk else None), flagged, rescue

    ms, sweep_ms, n_sweep, n_launch, F, B, clocks, flagged, rescue = run("mixed", args.steps)
    sec = ms * 1e-3
    hbm_peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    hbm = {"achieved": B / sec / 1e9, "peak": hbm_peak, "unit": "GB/s", "frac": B / sec / 1e9 / hbm_peak,
           "peak_source": peak_kind}
    alu = {"achieved": F / sec / 1e12, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
           "frac": F / sec / 1e12 / FP32_ALU_TFLOPS, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    bound_alu = F / (FP32_ALU_TFLOPS * 1e12) >= B / (hbm_peak * 1e9)
    roof = dict(alu if bound_alu else hbm)
    roof.update(bound="alu" if bound_alu else "hbm", traffic=None,
                kernel="k_ratio of every system (launches of different systems overlap): sweep work per step / "
                       "step time",
                launches=int(n_sweep), other=hbm if bound_alu else alu)
    line = {"metric": METRIC, "value": job_rate(W, ws, args.steps, sec), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": batched_desc(systems, W // len(systems)),
                       "precision": "mixed", "parallelism": f"replicas x{ws}, systems on 8 streams",
                       "path": ("separate calls: proposal, orbitals, ratio, Metropolis, accept" if args.separate else
                                "msd_step: one persistent launch per shared-memory group of systems, device "
                                "work queue, grid size tuned on the warm-up steps"),
                       "l2": "inputs exceed L2"},
            "launches_per_step": n_launch / args.steps,
            "roofline": roof, "gpu_launches": int(n_launch), "clocks": clocks, "status": flagged or "ok"}
    if args.rescue_slots > 0:
        steps_r = min(args.steps, args.rescue_steps)
        ms_r, _, _, _, _, _, clk_r, flagged_r, rescue = run("mixed", steps_r, args.rescue_slots)
        line["rescue_on"] = {"value": job_rate(W, ws, steps_r, ms_r * 1e-3), "ms_per_step": ms_r / steps_r,
                             "steps": steps_r, "status": flagged_r or "ok", "stats": rescue,
                             "what": "ill-conditioned walkers held in FP64 (msd_set_rescue, up to "
                                     f"{args.rescue_slots} per system)"}
    if not args.skip_fp64:
        steps64 = min(args.steps, args.fp64_steps)
        ms64, _, _, _, _, _, clk64, flagged64, _ = run("fp64", steps64)
        line["fp64"] = {"value": job_rate(W, ws, steps64, ms64 * 1e-3), "ms_per_step": ms64 / steps64,
                        "steps": steps64, "clocks": clk64, "status": flagged64 or "ok"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_fig3(args):
    """Table method against the canonical method (every determinant's own inverse updated by
    Sherman-Morrison), both FP64 on the GPU: walker-moves/s of ratio + grad + lap + accept as the
    number of determinants grows, at an acceptance near 50% and near 100% (the two regimes of the
    paper's Fig. 3), on synthetic inputs."""
    import torch

    from paper_1106_2456_gb300 import msd, workloads
    import __graft_entry__

    __graft_entry__.build()
    msd.load_library()
    W = args.walkers or 256
    cases = []

    def run_method(method, wl, tau, eta, u, steps):
        p = wl.problem
        c = msd.MSD(p, W, method, refresh_K=wl.refresh_K)
        c.set_positions(torch.tensor(wl.R0, device="cuda"))
        rnew = torch.empty(W, 3, dtype=torch.float64, device="cuda")
        r = torch.empty(W, dtype=torch.float64, device="cuda")
        g = torch.empty(W, 3, dtype=torch.float64, device="cuda")
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        acc = torch.empty(W, dtype=torch.uint8, device="cuda")
        n_acc = torch.zeros((), dtype=torch.float64, device="cuda")

        def step(t, count):
            e = t % p.n_tot
            c.propose(e, eta[t], tau, rnew)
            c.ratio_into(e, rnew, r, g, lp)
            c.metropolis(u[t], r, acc)
            c.accept(e, acc)
            if count:
                n_acc.add_(acc.sum())

        for t in range(4):
            step(t, False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for t in range(4, 4 + steps):
            step(t, True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        c.sync()
        c.close()
        return ms, float(n_acc.item()) / (steps * W)

    def calibrate(wl, eta, u, target=0.5):
        """tau whose acceptance with the table method is closest to the target (short runs)."""
        best = None
        for tau in (0.15, 0.25, 0.4, 0.6, 0.9, 1.3):
            _, a = run_method("fp64", wl, tau, eta, u, wl.problem.n_tot)
            if best is None or abs(a - target) < abs(best[1] - target):
                best = (tau, a)
        return best[0]

    for n, N, dets in ((5, 20, (100, 300, 1000, 3000, 5000)), (16, 48, (100, 1000, 3000))):
        for nd in dets:
            wl = workloads.custom_workload((n, n), (N, N), nd, workloads.uniform_orders(1, 4), W=W,
                                           n_nuc=max(3, -(-N // 12)), seed=1000 + nd + n, K=n)
            p = wl.problem
            steps = 2 * p.n_tot
            eta_np, u_np = wl.proposals(steps + 4)
            eta = torch.tensor(eta_np, device="cuda")
            u = torch.tensor(u_np, device="cuda")
            for regime, tau in (("~50%", calibrate(wl, eta, u)), ("~100%", 0.005)):
                row = {"n": n, "N": N, "n_det": nd, "strings": [p.n_exc(0), p.n_exc(1)], "regime": regime,
                       "tau": tau}
                row["table_ms"], row["acceptance"] = run_method("fp64", wl, tau, eta, u, steps)
                row["canonical_ms"], acc_c = run_method("canonical", wl, tau, eta, u, steps)
                row["acceptance_canonical"] = acc_c
                row["speedup"] = row["canonical_ms"] / row["table_ms"]
                cases.append(row)
    best = max((r for r in cases if r["regime"] == "~50%"), key=lambda r: r["n_det"] * r["n"])
    line = {"metric": "table vs canonical method, walker-moves/s (ratio+grad+lap+accept), FP64", "value":
            W / (best["table_ms"] * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": None, "warmup": 4,
            "ms_per_step": best["table_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"fig3: n per spin 5 and 16, N = 4n or 3n, orders 1-4, {W} walkers, "
                                   "refresh every n steps of a spin; step size tuned to ~50% acceptance, and 0.005 "
                                   "bohr for ~100%"},
            "cases": cases}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_1106_2456_gb300 import msd, workloads
    import __graft_entry__

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build() if rank == 0 else None
    if dist is not None:
        dist.barrier()
    msd.load_library()
    peaks, peak_kind = load_peaks()
    wl = workloads.make_workload(args.workload, **({"n_walkers": args.walkers} if args.walkers else {}))
    p = wl.problem
    W = wl.n_walkers
    K = wl.refresh_K
    n_tot = p.n_tot
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sweeps_total = args.warmup + args.steps
    R0, eta_np, u_np = replica_inputs(wl, rank, sweeps_total * n_tot)
    eta = torch.tensor(eta_np, device=dev)
    u = torch.tensor(u_np, device=dev)

    def make(prec):
        c = msd.MSD(p, W, prec, refresh_K=K, stream=stream)
        c.set_positions(torch.tensor(R0, device=dev))
        return c

    bufs = dict(rnew=torch.empty(W, 3, dtype=torch.float64, device=dev),
                ratio=torch.empty(W, dtype=torch.float64, device=dev),
                grad=torch.empty(W, 3, dtype=torch.float64, device=dev),
                lap=torch.empty(W, dtype=torch.float64, device=dev),
                acc=torch.empty(W, dtype=torch.uint8, device=dev))

    def sweep(c, s):
        """Step s: every electron once, in index order (move t = s n_tot + e draws eta[t], u[t])."""
        for e in range(n_tot):
            t = s * n_tot + e
            c.propose(e, eta[t], wl.tau, bufs["rnew"])
            c.ratio_into(e, bufs["rnew"], bufs["ratio"], bufs["grad"], bufs["lap"])
            c.metropolis(u[t], bufs["ratio"], bufs["acc"])
            c.accept(e, bufs["acc"])

    def timed(c, steps):
        for s in range(args.warmup):
            sweep(c, s)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local) if rank == 0 else None
        time.sleep(0.3 if clk else 0)
        c.timing_start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        e0.record(stream)
        for s in range(args.warmup, args.warmup + steps):
            sweep(c, s)
        e1.record(stream)
        torch.cuda.synchronize()
        w1 = time.time()
        n_refresh, n_ci = c.timing_counts()
        sweep_ms, n_sweep, n_launch = c.timing_stop()
        if clk:
            clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        c.sync()
        window = {"sweeps": steps, "moves_per_walker": steps * n_tot, "refreshes": n_refresh,
                  "ci_contractions": n_ci}
        return ms, sweep_ms, n_sweep, n_launch, (clk.summary(w0, w1) if clk else None), window

    def roofline(prec, sweep_ms, steps):
        mixed = prec == "mixed"
        F = B = 0.0
        plan = msd.describe(p, prec)
        for e in range(n_tot):  # one sweep: every electron once
            s = p.spin_of(e)
            f, b = sweep_work(p, s, W, mixed, int(plan[s][0]))
            F += f * steps
            B += b * steps
        launches = steps * n_tot
        sec = sweep_ms * 1e-3
        hbm_peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
        alu_peak = FP32_ALU_TFLOPS if mixed else FP64_ALU_TFLOPS
        t_alu = F / (alu_peak * 1e12)
        t_hbm = B / (hbm_peak * 1e9)
        hbm = {"achieved": B / sec / 1e9, "peak": hbm_peak, "unit": "GB/s", "frac": B / sec / 1e9 / hbm_peak,
               "peak_source": peak_kind}
        alu = {"achieved": F / sec / 1e12, "peak": alu_peak, "unit": "TFLOP/s", "frac": F / sec / 1e12 / alu_peak,
               "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if mixed
               else "nominal GB300 FP64 rate"}
        main = dict(alu if t_alu >= t_hbm else hbm)
        main["bound"] = "alu" if t_alu >= t_hbm else "hbm"
        tb = profiled_traffic(mixed)
        main["traffic"] = None if tb is None else tb["dram_bytes_per_walker"] * W
        main["traffic_source"] = (None if tb is None else
                                  f"ncu dram__bytes_read.sum + dram__bytes_write.sum per walker of one launch "
                                  f"({tb['walkers']}-walker capture, {tb['file']}) x {W} walkers")
        main["kernel"] = "k_ratio (excitation sweep, steps A2-A5)"
        main["launches"] = launches
        main["avg_launch_us"] = 1e3 * sweep_ms / launches
        main["other"] = hbm if main["bound"] == "alu" else alu
        return main

    # ---- mixed precision (headline) ----
    cm = make("mixed")
    ms, sweep_ms, n_sweep, n_launch, clocks, window = timed(cm, args.steps)
    value = job_rate(W * n_tot, ws, args.steps, ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, wl),
                       "step": f"one Metropolis sweep: {n_tot} single-electron moves of every walker, with the "
                               f"refreshes and CI contractions they trigger",
                       "precision": "mixed: FP32 orbitals/table/excitation dets, FP64 inverse/SM/ratio sums",
                       "walkers_per_gpu": W, "parallelism": f"replicas x{ws}",
                       "l2": "inputs exceed L2 (per-walker tables and CI streams: >1 GB)"},
            "window": window,
            "roofline": roofline("mixed", sweep_ms, args.steps),
            "gpu_launches": int(n_launch), "clocks": clocks}
    # ---- the same with ill-conditioned walkers held in FP64 (msd_set_rescue) ----
    if args.rescue_slots > 0:
        cr = msd.MSD(p, W, "mixed", refresh_K=K, stream=stream)
        cr.set_rescue(args.rescue_slots)
        cr.set_positions(torch.tensor(R0, device=dev))
        ms_r, _, _, _, clk_r, win_r = timed(cr, min(args.steps, args.rescue_steps))
        line["rescue_on"] = {"value": job_rate(W * n_tot, ws, min(args.steps, args.rescue_steps), ms_r * 1e-3),
                             "ms_per_step": ms_r / min(args.steps, args.rescue_steps), "slots": args.rescue_slots,
                             "stats": cr.rescue_stats(), "window": win_r, "clocks": clk_r}
        cr.close()
    # ---- end to end through the host-buffer C ABI ----
    if args.e2e_steps > 0:
        e2e_steps = min(args.steps, args.e2e_steps)
        Rh, _, _ = cm.get_state()
        Rh = Rh.cpu().numpy()
        pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
        rnew_h, ratio_h = pin((W, 3), torch.float64), pin((W,), torch.float64)
        grad_h, lap_h, acc_h = pin((W, 3), torch.float64), pin((W,), torch.float64), pin((W,), torch.uint8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in range(e2e_steps * n_tot):
            t = q % (sweeps_total * n_tot)
            e = q % n_tot
            np.add(Rh[:, e], wl.tau * eta_np[t], out=rnew_h)
            cm.ratio_host(e, rnew_h, ratio_h, grad_h, lap_h)
            np.less(u_np[t], ratio_h * ratio_h, out=acc_h, casting="unsafe")
            cm.accept_host(e, acc_h)
            sel = acc_h.astype(bool)
            Rh[sel, e] = rnew_h[sel]
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        line["e2e"] = {"value": job_rate(W * n_tot, ws, e2e_steps, dt), "unit": UNIT, "steps": e2e_steps,
                       "h2d_bytes_per_step": (W * 3 * 8 + W) * n_tot, "d2h_bytes_per_step": W * 5 * 8 * n_tot,
                       "path": "msd_ratio_host + msd_accept_host per move (pinned host buffers, synchronous)"}
    # ---- VMC local energy (taken once per sweep in a VMC run) ----
    if args.eloc_calls > 0:
        cm.set_hamiltonian(workloads.nuclear_charges(p), 1.0, 1.0)
        eloc = torch.empty(W, dtype=torch.float64, device=dev)
        cm.local_energy_into(eloc)  # the first call allocates its workspace
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.eloc_calls):
            cm.local_energy_into(eloc)
        a1.record(stream)
        torch.cuda.synchronize()
        ms_le = max_over_ranks(a0.elapsed_time(a1), dist, dev) / args.eloc_calls
        line["local_energy"] = {
            "value": job_rate(W, ws, 1, ms_le * 1e-3), "unit": "walker local energies/s", "ms_per_call": ms_le,
            "calls": args.eloc_calls, "vs_sweep": ms_le / (ms / args.steps),
            "what": "msd_local_energy, mixed: all-electron grad/lap (one cofactor scatter per spin), "
                    "Pade-Jastrow (b_ee = b_en = 1) and Coulomb terms; vs_sweep = its time over one sweep"}
    def per_call_ms(fn, calls):
        fn()  # the first call allocates its workspace
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(calls):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(a0.elapsed_time(a1), dist, dev) / calls

    # ---- adjoint of log|Psi| (once per parameter update of an optimisation) ----
    gbar = torch.ones(W, dtype=torch.float64, device=dev)
    if args.adjoint_calls > 0:
        line["adjoint"] = {"unit": "ms per call", "calls": args.adjoint_calls,
                           "mixed": per_call_ms(lambda: cm.backward(gbar), args.adjoint_calls),
                           "what": "msd_backward: d log|Psi| / d c_I and d B of all walkers (refresh included)"}
    # ---- FP64 path on the same workload ----
    if not args.skip_fp64:
        cm.close()
        cd = make("fp64")
        steps64 = min(args.steps, args.fp64_steps)
        ms64, sweep64, _, _, clk64, win64 = timed(cd, steps64)
        line["fp64"] = {"value": job_rate(W * n_tot, ws, steps64, ms64 * 1e-3), "ms_per_step": ms64 / steps64,
                        "steps": steps64, "window": win64, "roofline": roofline("fp64", sweep64, steps64),
                        "clocks": clk64}
        if args.eloc_calls > 0:
            cd.set_hamiltonian(workloads.nuclear_charges(p), 1.0, 1.0)
            eloc64 = torch.empty(W, dtype=torch.float64, device=dev)
            line["fp64"]["local_energy_ms_per_call"] = per_call_ms(lambda: cd.local_energy_into(eloc64),
                                                                   min(args.eloc_calls, 2))
        if args.adjoint_calls > 0:
            line["adjoint"]["fp64"] = per_call_ms(lambda: cd.backward(gbar), min(args.adjoint_calls, 2))
        line["mixed_speedup_vs_fp64"] = value / line["fp64"]["value"]
        # per-result difference mixed vs FP64 on a common trajectory (FP64 accept decisions) over
        # whole sweeps, so the Sherman-Morrison drift between refreshes is in the sample
        def compare(rescue_slots):
            cd.set_positions(torch.tensor(R0, device=dev))
            cmx = msd.MSD(p, W, "mixed", refresh_K=K, stream=stream)
            if rescue_slots:
                cmx.set_rescue(rescue_slots)
            cmx.set_positions(torch.tensor(R0, device=dev))
            errs = {"ratio": [], "grad": [], "lap": []}
            big, same = [], []
            for t in range(args.cmp_steps):
                e = t % n_tot
                cd.propose(e, eta[t], wl.tau, bufs["rnew"])
                r64, g64, l64 = cd.ratio(e, bufs["rnew"])
                r32, g32, l32 = cmx.ratio(e, bufs["rnew"])
                for key, a, b in (("ratio", r32, r64), ("grad", g32, g64), ("lap", l32, l64)):
                    # per walker: |a - b| / |b|, the gradient by its Euclidean norm
                    d = (a - b).reshape(W, -1).norm(dim=1)
                    errs[key].append((d / b.reshape(W, -1).norm(dim=1).clamp_min(1e-300)).cpu().numpy())
                big.append((r64.abs() >= 0.1).cpu().numpy())
                same.append(((u[t] < r32 * r32) == (u[t] < r64 * r64)).cpu().numpy())
                cd.metropolis(u[t], r64, bufs["acc"])
                cd.accept(e, bufs["acc"])
                cmx.accept(e, bufs["acc"])
            big = np.concatenate(big)
            cmp = {}
            for k, v in errs.items():
                v = np.concatenate(v)
                cmp[k] = {"median_rel": float(np.median(v)), "p90_rel": float(np.percentile(v, 90)),
                          "p99_rel": float(np.percentile(v, 99)), "p999_rel": float(np.percentile(v, 99.9)),
                          "p99_rel_ratio_ge_0.1": float(np.percentile(v[big], 99))}
            cmp["moves"] = args.cmp_steps
            cmp["ratio_ge_0.1_share"] = float(big.mean())
            cmp["metropolis_decisions_equal"] = float(np.concatenate(same).mean())
            if rescue_slots:
                cmp["rescue"] = cmx.rescue_stats()
            cmx.close()
            return cmp

        cmp = compare(0)
        cmp["note"] = ("relative difference per walker-move (grad: Euclidean norm); the tail comes from moves "
                       "whose ratio is a small difference of large CI terms; p99_rel_ratio_ge_0.1 keeps the moves "
                       "with |ratio| >= 0.1; metropolis_decisions_equal: same accept decision from the same uniform")
        line["mixed_vs_fp64"] = cmp
        if args.rescue_slots > 0:
            line["mixed_vs_fp64_rescue"] = compare(args.rescue_slots)
        cd.close()
    cm.close()
    # ---- FP64 CPU oracle on a bounded sample ----
    if rank == 0 and ws == 1 and not args.skip_cpu:
        rate, done, dt, cores = oracle_rate(wl, args.cpu_moves, args.cpu_time_cap)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done} single-walker moves of this workload (every determinant and "
                                          f"derivative determinant by LU, FP64), {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4, help="timed steps (sweeps for the default workload)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed sweeps of the FP64 path")
    ap.add_argument("--e2e-steps", type=int, default=1, help="sweeps through the host-buffer entry points")
    ap.add_argument("--cmp-steps", type=int, default=128, help="moves of the mixed-vs-FP64 comparison")
    ap.add_argument("--eloc-calls", type=int, default=5)
    ap.add_argument("--adjoint-calls", type=int, default=2)
    ap.add_argument("--rescue-slots", type=int, default=32,
                    help="FP64 slots of the extra legs with ill-conditioned walkers held in FP64 (0: skip them)")
    ap.add_argument("--rescue-steps", type=int, default=4, help="timed sweeps of the rescue leg")
    ap.add_argument("--cpu-moves", type=int, default=30)
    ap.add_argument("--cpu-time-cap", type=float, default=25.0)
    ap.add_argument("--ref-time-cap", type=float, default=150.0)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--walkers", type=int, default=0, help="override the workload's walker count (profiling)")
    ap.add_argument("--systems", type=int, default=256, help="systems of the batched workload")
    ap.add_argument("--separate", action="store_true", help="batched workload: the separate calls instead of msd_step")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "fig3":
        return run_fig3(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
