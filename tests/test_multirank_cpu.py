"""The benchmark's multi-rank path on the host (gloo, two ranks, no GPU).

With N GPUs the benchmark runs one process per GPU: every rank integrates
its own robot's sequence (the path shards by robot and has no collective
on the data path), and only the barrier and the max / sum of the timings
cross ranks.  The batched and served forms shard their robots and cameras
over the ranks the same way.  These tests run that plumbing as two gloo
ranks on the CPU: the reductions, that every rank gets its own robot, that
the ranks partition the robots and cameras, and that the reference arm
under torchrun prints one line from rank 0 while rank 1 exits cleanly.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    from synth import make
    d = bench.Dist(world, backend="gloo")
    d.barrier()
    # the job's time is the slowest rank's; its work is every rank's
    slowest = d.max(1.5 + rank)
    total = d.sum(10.0 * (rank + 1))
    w = make("seq", frames=1, seed=bench.rank_seed(rank))
    first_depth = float(w.frames[0].depth[::37, ::41].sum())
    # the batched and served forms: this rank's robots and cameras
    robots = bench.shard(range(64), rank, world)
    cams = bench.shard(range(256), rank, world)
    n_all = d.sum(len(robots)) + 1000 * d.sum(len(cams))
    d.barrier()
    d.close()
    out.put((rank, slowest, total, bench.rank_seed(rank), first_depth, robots, cams, n_all))


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reduce_timings_and_run_independent_robots():
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0, "rank process failed"
    res = sorted(out.get() for _ in range(world))
    for rank, slowest, total, _, _, _, _, n_all in res:
        assert slowest == 2.5          # max over ranks of 1.5 + rank
        assert total == 30.0           # sum over ranks of 10 * (rank + 1)
        assert n_all == 64 + 1000 * 256
    # the ranks partition the 64 robots and the 256 cameras: no unit twice, none left out
    for k, n in ((5, 64), (6, 256)):
        units = [u for r in res for u in r[k]]
        assert sorted(units) == list(range(n))
        assert all(len(r[k]) == n // world for r in res)
    seeds = [r[3] for r in res]
    assert len(set(seeds)) == world    # every rank its own robot
    assert res[0][4] != res[1][4]      # ... and so its own depth frames


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    saved = {k: os.environ.pop(k, None) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    try:
        d = bench.Dist(1, backend="gloo")
        assert d.pg is None and d.rank == 0
        assert d.max(3.0) == 3.0 and d.sum(4.0) == 4.0
        with pytest.raises(SystemExit):
            bench.Dist(2, backend="gloo")   # N > 1 without torchrun
    finally:
        for k, v in saved.items():
            if v is not None:
                os.environ[k] = v


@pytest.mark.timeout(300)
def test_reference_arm_under_torchrun_prints_once_from_rank0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--frames", "1", "--workload", "room"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
