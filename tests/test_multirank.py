"""The replicas-only multi-GPU path of bench.py, on CPU: two gloo ranks on 127.0.0.1.

Walkers are independent chains, so N GPUs run N replicas with no data-path collective; the
only exchanges are the barrier and the max-over-ranks timing.  Checked here: each rank gets
its own chains, the max reduction, the whole-job rate, and that under torchrun only rank 0
runs the reference arm.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    from paper_1106_2456_gb300 import workloads as wl

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = wl.make_workload("water", n_walkers=8)
    R0, eta, u = bench.replica_inputs(w, rank, 5)
    t_max = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    dist.barrier()
    # the reference arm: rank != 0 returns at once without output
    ref_rc = None
    if rank == 1:
        args = type("A", (), dict(workload="water", walkers=0, warmup=0, steps=1, ref_time_cap=1.0))()
        ref_rc = bench.run_reference(args)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), R0=R0, eta=eta, u=u, t_max=t_max,
             ref_rc=-1 if ref_rc is None else ref_rc)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path, capfd):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    assert float(r0["t_max"]) == 11.0 and float(r1["t_max"]) == 11.0
    assert not np.array_equal(r0["eta"], r1["eta"]) and not np.array_equal(r0["R0"], r1["R0"])
    assert np.max(np.abs(r0["R0"] - r1["R0"])) < 0.1  # same workload, jittered chains
    assert int(r1["ref_rc"]) == 0
    out = capfd.readouterr().out
    assert not any(line.startswith("{") for line in out.splitlines())  # rank 1 printed no JSON line


def test_job_rate_and_single_rank_max():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_rate(4096, 8, 512, 2.0) == 4096 * 8 * 512 / 2.0
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
