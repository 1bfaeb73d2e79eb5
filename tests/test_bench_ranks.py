"""The replicated multi-rank path of bench.py on CPU: two gloo ranks (one
process each, rendezvous on 127.0.0.1) time different amounts; every rank
gets the maximum, and the whole-job rate counts both replicas' work over it.
The reference arm under torchrun prints from rank 0 only."""
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")
        rate = bench.replica_rate(world, 1.0e9, ms * 1e-3)
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]           # both ranks see the slowest
    assert out[0][2] == pytest.approx(2 * 1.0e9 / 15e-3)  # two replicas' work over it


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_rate(1, 100.0, 2.0) == 50.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_summary_repeats_the_nested_results_as_one_flat_string():
    """The line's last key restates the step, batched and adjoint results,
    read from the nested objects (here a line as bench.py builds it)."""
    sys.path.insert(0, ROOT)
    import bench
    line = {"value": 1.52e11, "roofline": {"frac": 0.8}, "e2e": {"value": 1.36e11},
            "metric2": {"multigroup2d_256x256x128x64": {
                "fp32_s_per_step": 0.0293, "fp64_s_per_step": 0.471,
                "fp32_refined_s_per_step": 0.277, "refined_vs_fp64_T_rel": 1e-14,
                "fp32_vs_fp64_T_rel": 5.5e-8}},
            "batched": {"value": 1.076e11, "roofline": {"frac": 0.573}, "batched_speedup": 2.06,
                        "step": {"s_per_step": 0.548}},
            "adjoint_warm": {"fd_cells": 32, "fd_max_rel_err": 8.0e-7}}
    s = bench.summary_text(line)
    for part in ("152.0 G", "0.800 of HBM", "e2e 136.0 G", "FP32 29.30 ms", "FP64 471.00 ms",
                 "277.00 ms", "1.0e-14", "batched 107.6 G", "0.548 s", "32 cells",
                 "8.0e-07"):
        assert part in s, (part, s)
    assert bench.summary_text({"value": 1e9}) == "pass 1.0 G updates/s"
