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


def _sharded_worker(rank, world, port, q):
    """One rank of the sharded SVRG solve with the oracle's FP64 primitives
    (test infrastructure standing in for the GPU kernels): the anchor on the
    rank's column slab, a gloo all-reduce, the inner loop on the whole X."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import lra_inputs as L
    from oracle import lra_oracle as O
    from paper_1607_02925_gb300 import dist as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, n, p = 64, 901, 3
        Xt, _, s = L.planted_numpy(d, n, L.sigma_small_gap(64), 13)
        c0, c1 = D.column_slab(n, rank, world)
        ctx = O.Context(Xt, 5, O.Options(tau=1e-8))
        lam1_up = s[0] ** 2 / 0.75
        lam = 2.0 * lam1_up
        mu = lam - lam1_up
        eta, m = ctx.step_params(lam, mu, lam1_up)
        rng = np.random.default_rng(2)
        B = rng.standard_normal((d, p))
        W0 = np.zeros((d, p))

        def allreduce(M):
            t = torch.from_numpy(np.ascontiguousarray(M))
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            return t.numpy()

        prim = D.Primitives(
            anchor_local=lambda Wt, Bb, lm: O.anchor(Xt[c0:c1], Wt, Bb, lm),
            allreduce=allreduce, zeros_like=np.zeros_like, sqnorm=lambda A: float(np.sum(A * A)),
            sample=lambda key, mm: O.sample_indices(ctx.table, key, mm),
            inner=lambda W, Wt, M, idx, mm, et, lm: O.svrg_epoch(Xt, W, Wt, M, idx, ctx.table.c, et, lm),
            copy=lambda A: np.array(A, copy=True))
        W, info = D.svrg_solve_sharded(prim, rank, B, W0, lam, eta, m, 1e-8,
                                       lambda e: O.stream_key(5, O.STREAM_SVRG, 0, e))
        q.put((rank, (c0, c1), W, info.epochs, info.status))
    finally:
        dist.destroy_process_group()


def test_sharded_anchor_solve_matches_the_single_process_oracle():
    """World size 2 on CPU: the column-sharded anchor with a d x p all-reduce
    per epoch and the replicated inner loop give the single-process oracle's
    SVRG solve (same samples, same epochs) to rounding."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import lra_inputs as L
    from oracle import lra_oracle as O
    from paper_1607_02925_gb300 import dist as D

    assert [D.column_slab(10, r, 3) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert out[0][1] == (0, 450) and out[1][1] == (450, 901)
    # the single-process oracle on the whole X
    d, n, p = 64, 901, 3
    Xt, _, s = L.planted_numpy(d, n, L.sigma_small_gap(64), 13)
    octx = O.Context(Xt, 5, O.Options(tau=1e-8))
    lam1_up = s[0] ** 2 / 0.75
    lam = 2.0 * lam1_up
    B = np.random.default_rng(2).standard_normal((d, p))
    Wref, st = octx.svrg_solve(B, np.zeros((d, p)), lam, lam - lam1_up, lam1_up)
    for rank, _, W, epochs, status in out:
        assert status == "ok" and epochs == st.epochs
        assert np.max(np.abs(W - Wref)) <= 1e-12 * np.max(np.abs(Wref))
    assert np.array_equal(out[0][2], out[1][2])
