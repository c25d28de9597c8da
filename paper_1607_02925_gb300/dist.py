"""The anchor pass sharded over ranks (one GPU per rank), inner loop replicated.

The anchor of an SVRG epoch (Sec. 2.3) is M = lambda W~ - X (X^T W~) - B, and
X (X^T W~) = sum over ranks g of X_g (X_g^T W~) for the column slabs X_g of X
(the sum over data points of the problem statement, Sec. 1).  Each rank runs
the anchor on its own slab with (lambda, B) on rank 0 and (0, 0) on the others,
and one all-reduce (sum) of the d x p block gives every rank the whole M.

The inner loop samples columns from all n, so every rank keeps the whole X
for it and draws the same index sequence (the streams are keyed by seed,
solve and epoch): the ranks' W stay identical with no communication per step.

Only the composition lives here.  The arithmetic is in the primitives the
caller passes: on GPUs, `gpu_primitives` binds the library's step entry points
(lra_anchor on the rank's slab, lra_gram for ||M||_F^2, lra_sample,
lra_svrg_inner) and an all-reduce from torch.distributed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Any, Callable


def column_slab(n: int, rank: int, world: int) -> tuple[int, int]:
    """Columns [c0, c1) of X owned by `rank`: contiguous slabs whose sizes
    differ by at most one."""
    if not (0 <= rank < world) or n < world:
        raise ValueError("need 0 <= rank < world <= n")
    return rank * n // world, (rank + 1) * n // world


@dataclass
class Primitives:
    """What one rank needs for the sharded solve.

    anchor_local(Wt, B, lam) -> M_g = lam Wt - X_g X_g^T Wt - B on the rank's slab
    allreduce(M) -> M summed over ranks (returns the reduced block)
    zeros_like(B) -> a zero block of B's shape and placement
    sqnorm(A) -> ||A||_F^2
    sample(key, m) -> m column indices of the whole X (importance sampling)
    inner(W, Wt, M, idx, m, eta, lam) -> W after the m inner steps on the whole X
    copy(A) -> a copy of A
    """
    anchor_local: Callable[..., Any]
    allreduce: Callable[[Any], Any]
    zeros_like: Callable[[Any], Any]
    sqnorm: Callable[[Any], float]
    sample: Callable[[int, int], Any]
    inner: Callable[..., Any]
    copy: Callable[[Any], Any]


def sharded_anchor(prim: Primitives, rank: int, Wt, B, lam: float):
    """M = lam Wt - X X^T Wt - B from the ranks' slabs: lam and B enter once,
    on rank 0, so the sum over ranks counts them once."""
    if rank == 0:
        Mg = prim.anchor_local(Wt, B, lam)
    else:
        Mg = prim.anchor_local(Wt, prim.zeros_like(B), 0.0)
    return prim.allreduce(Mg)


@dataclass
class ShardedSolveInfo:
    epochs: int = 0
    inner_steps: int = 0
    residual: float = float("nan")
    status: str = "ok"


def svrg_solve_sharded(prim: Primitives, rank: int, B, W0, lam: float, eta: float, m: int, tau: float,
                       key_of_epoch: Callable[[int], int], max_epochs: int = 60, fixed_epochs: int = 0):
    """SVRGsolve (Sec. 2.3) with the anchor sharded over ranks: epoch e takes
    W~ = W, M = lam W~ - X X^T W~ - B (sharded_anchor), stops when ||M||_F <=
    tau ||B||_F (or after `fixed_epochs` anchors), else runs m inner steps on
    the indices drawn from key_of_epoch(e), identical on every rank.  The stall
    and divergence rules are those of the single-GPU solve: after the fourth
    anchor a residual above 0.9 x the previous ends it; a non-finite residual,
    or one above 10 x the best, the first and 1e-3, is divergence."""
    info = ShardedSolveInfo()
    W = prim.copy(W0)
    nB = math.sqrt(prim.sqnorm(B))
    best = prev = res0 = float("inf")
    last = fixed_epochs if fixed_epochs > 0 else max_epochs
    for e in range(last):
        Wt = prim.copy(W)
        M = sharded_anchor(prim, rank, Wt, B, lam)
        res = math.sqrt(prim.sqnorm(M)) / nB if nB > 0 else 0.0
        info.epochs = e + 1
        info.residual = res
        if e == 0:
            res0 = res
        if not math.isfinite(res) or (res > 10.0 * best and res > max(res0, 1e-3)):
            info.status = "diverged"
            return W, info
        if fixed_epochs <= 0:
            if res <= tau:
                return W, info
            if e >= 3 and res > 0.9 * prev:
                return W, info
        if e == last - 1:
            if fixed_epochs <= 0:
                info.status = "notconv"
            return W, info
        best = min(best, res)
        prev = res
        idx = prim.sample(key_of_epoch(e), m)
        W = prim.inner(W, Wt, M, idx, m, eta, lam)
        info.inner_steps += m
    return W, info


def gpu_primitives(ctx, mat_full, mat_slab, d: int, n: int, p: int, group=None) -> Primitives:
    """Primitives on this rank's GPU: mat_full holds the whole X (d x n; inner
    loop, sampling table), mat_slab the rank's column slab (anchor).  Blocks
    are torch (p, d) CUDA tensors holding d x p column-major blocks."""
    import torch
    import torch.distributed as dist

    from . import lra_anchor, lra_colnorms, lra_gram, lra_sample, lra_sampling_table, lra_svrg_inner

    norm2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    lra_colnorms(mat_full, norm2)
    cum = torch.zeros(n, dtype=torch.int64, device="cuda")
    cvec = torch.zeros(n, dtype=torch.float32, device="cuda")
    total, _ = lra_sampling_table(ctx, n, norm2, 0, cum, cvec)
    gram = torch.zeros(p, p, dtype=torch.float64, device="cuda")

    def anchor_local(Wt, B, lam):
        M = torch.empty_like(Wt)
        lra_anchor(mat_slab, p, Wt, B, lam, M)
        return M

    def allreduce(M):
        torch.cuda.synchronize()
        dist.all_reduce(M, op=dist.ReduceOp.SUM, group=group)
        return M

    def sqnorm(A):
        lra_gram(ctx, d, p, A, d, gram)
        g = gram.cpu().numpy()
        return float(sum(g[j, j] for j in range(p)))

    def sample(key, m):
        idx = torch.zeros(max(m, 1), dtype=torch.int32, device="cuda")
        lra_sample(ctx, n, cum, total, key, m, idx)
        return idx

    def inner(W, Wt, M, idx, m, eta, lam):
        lra_svrg_inner(mat_full, p, W, Wt, M, idx, m, cvec, eta, lam)
        return W

    return Primitives(anchor_local=anchor_local, allreduce=allreduce, zeros_like=torch.zeros_like,
                      sqnorm=sqnorm, sample=sample, inner=inner, copy=lambda A: A.clone())
