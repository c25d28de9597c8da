"""The replicas-only multi-GPU path of bench.py, on CPU with gloo (world size 2).

Each rank solves its own copy, so the only cross-rank steps are the barrier
around the timed region and the max over ranks of the step time; both run
here on CPU processes.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        dist.barrier()
        mine = 10.0 + 7.5 * r            # rank-dependent step time (ms)
        got = bench.max_over_ranks(mine, "cpu")
        dist.barrier()
        q.put((r, w, local, got))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_max_step_time_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == world and o[2] == o[0] for o in out)
    assert all(o[3] == 17.5 for o in out)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the reference arm (the oracle on the host cores) is timed
    and printed by rank 0; every other rank exits 0 without work."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (1, 2, 1)
    assert bench.run_reference(None) == 0
