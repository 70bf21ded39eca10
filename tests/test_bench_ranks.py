"""The N > 1 path of bench.py on the CPU (gloo, world size 2).

Several GPUs run independent replicas of the workload (weak scaling, no
data-path collective): the value is the units of all ranks over the slowest
rank's time, the time reduced by one all-reduce MAX.  The batched workload's
independent problems are sharded instead (largest first onto the least
loaded rank); "every rank converged" is the same MAX reduction.  The
reference arm runs on rank 0 only; the other ranks exit 0 without work or
output.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [0.5, 2.0][rank]           # rank 1 is the slow one
        tmax = bench.max_over_ranks(secs, world)
        q.put((rank, tmax, bench.replica_throughput(1000, 4, world, tmax)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, tmax, value in got:
        assert tmax == 2.0
        assert value == pytest.approx(2 * 4 * 1000 / 2.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.replica_throughput(10, 3, 1, 2.0) == 15.0


def test_reference_arm_two_ranks_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["steps"] == 1
    assert rec["value"] > 0 and rec["e2e"]["value"] == rec["value"]
    assert rec["cpu_baseline"]["kind"] == "oracle"


def test_shard_problems_largest_first():
    """Every problem on exactly one rank; the largest-first rule keeps the
    heaviest rank within one problem of the lightest; deterministic; one
    rank gets everything."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    m = np.random.default_rng(0).integers(127, 1024, size=64)
    sizes = [int(v) ** 2 * 32 for v in m]            # DOF x RHS of 64 problems, 32 RHS each
    assert bench.shard_problems(sizes, 1) == [list(range(64))]
    for world in (2, 3, 4, 8):
        parts = bench.shard_problems(sizes, world)
        assert parts == bench.shard_problems(sizes, world)
        assert sorted(i for part in parts for i in part) == list(range(64))
        loads = [sum(sizes[i] for i in part) for part in parts]
        assert max(loads) - min(loads) <= max(sizes)
    # by hand, sizes 3 5 2 4 3 onto two ranks (loads after each step):
    # #1 (5) -> r0 (5, 0); #3 (4) -> r1 (5, 4); #0 (3) -> r1 (5, 7);
    # #4 (3) -> r0 (8, 7); #2 (2) -> r1 (8, 9)
    assert bench.shard_problems([3, 5, 2, 4, 3], 2) == [[1, 4], [0, 2, 3]]


def test_batched_all_converged_reduction_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_conv_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, False), (1, False)]      # rank 1 did not converge: nobody reports converged


def _conv_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        conv = rank == 0
        q.put((rank, bench.max_over_ranks(0.0 if conv else 1.0, world) == 0.0))
    finally:
        dist.destroy_process_group()
