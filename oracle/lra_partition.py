"""FP64 oracle of Algorithm 6's full loop: adaptive partitioning of {1..k} with
deflation (Gonen & Shalev-Shwartz, Sec. 3: Algorithms 3, 4, 5, 6, 7).

TEST INFRASTRUCTURE ONLY, like lra_oracle (imported by tests/, smoke() and the
CPU legs of bench.py; never by the library).

Stage t starts at index s with the columns U_1..U_{s-1} found so far and
works on the deflated matrix X_{-(s-1)} = (I - U U^T) X, formed explicitly as
Sec. 3 assumes ("we already applied the projection ... to the columns of X"):

  1. Algorithm 3 on A_{-(s-1)} with k - s + 1 vectors and eps' = 1/(9 p^2)
     gives lambda_hat_s..lambda_hat_k;
  2. Algorithm 4: the first q in {s..k-1} with lambda_hat_{q+1} <=
     lambda_hat_q (1 - p^-2); if there is one, Algorithm 1 on A_{-(s-1)} with
     q - s + 1 columns (no oversampling) gives u_s..u_q;
  3. otherwise Algorithm 7 on A_{-(s-1)} tunes the shift lambda, Algorithm 3 on
     D_{-(s-1)} (k - s + 1 vectors, eps' = 1/(9p)) estimates lambda - lambda_i,
     Algorithm 5 returns q (the first additive gap >= 5 Delta / 9, else k), and
     Algorithm 1 on D_{-(s-1)} with p' columns gives u_s..u_q;
  4. s = q + 1.
The columns are then orthonormalised together and Algorithm 2 with X X^T
returns U.

Readings:
  * D_{-(s-1)} = P (lambda I - A)^{-1} P (Eq. deflatedShift) is taken as
    P (lambda I - A_{-(s-1)})^{-1} P: the same operator when the u_i are exact
    eigenvectors, and the one SVRG can solve (lambda I - A is indefinite for
    lambda < lambda_1).  Its products are SVRG solves on X_{-(s-1)}.
  * Algorithm 3 runs L = ceil(eps'^-1 ln(d/eps')) iterations (the constant of
    the O() taken as 1, as for the lambda_1 estimate), capped at part_max_iters
    (default 2000; the bound is ~7e4 for p = 20 and eps' = 1/(9p^2)).  No early
    stop: block power Ritz values can rest at an inner eigenvalue until a
    weakly started direction emerges, which is what the gap-free count
    guards against.  Algorithm 1 on A (L = O(p^4 log(kd/eps)) in the paper)
    stops by the outer loop's rule on the block's Ritz error with the rate
    floor (lambda_hat_{q+1}/lambda_hat_q)^2.
  * Algorithm 4 returns "any" q: the smallest is taken.
  * Algorithm 6's p' line is garbled ("If q = k set p' = p. Otherwise, set
    p' = p"): p' = q - s + 1 when q < k (no oversampling, Sec. 3 item 2) and
    p' = p - (s - 1) when q = k, so that U is the d x p matrix the algorithm
    forms.  A stage with q = k keeps all p' Ritz vectors (its oversampling).
  * Each stage's randomness is keyed by a stage seed
    stream_key(seed, STREAM_PART, t, 0); the stage runs the hot path's streams
    (Gaussian starts, SVRG samples) under that seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import lra_oracle as O

STREAM_PART = 6          # per-stage seeds of Algorithm 6
STREAM_BLOCK = 7         # Gaussian start of Algorithm 3 / Algorithm 1 blocks within a stage


def deflate(Xt, Ut: np.ndarray) -> np.ndarray:
    """X_{-(s-1)} = (I - U U^T) X for orthonormal U (d x (s-1)); rows of Xt are the
    columns x_i, so the result's rows are (P x_i)^T (dense, FP64)."""
    X = O.as64(Xt)
    X = X.toarray() if hasattr(X, "toarray") else np.asarray(X)
    if Ut.shape[1] == 0:
        return X.copy()
    return X - (X @ Ut) @ Ut.T


def alg4(lam_hat: np.ndarray, p: int) -> int:
    """Algorithm 4 on lambda_hat_s..lambda_hat_k: the offset j of the first q = s + j
    in I \\ {k} with lambda_hat_{q+1} <= lambda_hat_q (1 - p^-2), or -1."""
    for j in range(len(lam_hat) - 1):
        if lam_hat[j + 1] <= lam_hat[j] * (1.0 - 1.0 / (p * p)):
            return j
    return -1


def alg5(inv_est: np.ndarray, delta: float) -> int:
    """Algorithm 5 on tilde-lambda^{-1}_s..tilde-lambda^{-1}_k (estimates of
    lambda - lambda_i, increasing): the offset of the first q in I \\ {k} with
    tilde-lambda^{-1}_{q+1} - tilde-lambda^{-1}_q >= 5 Delta / 9; else the offset of k."""
    for j in range(len(inv_est) - 1):
        if inv_est[j + 1] - inv_est[j] >= 5.0 * delta / 9.0:
            return j
    return len(inv_est) - 1


def _iters(eps: float, d: int, cap: int) -> int:
    return max(1, min(int(math.ceil((1.0 / eps) * math.log(d / eps))), cap))


def alg3_values(apply, S0: np.ndarray, eps: float, cap: int):
    """Algorithm 3 for a PSD operator C given by `apply` (S -> C S): Algorithm 1
    with the d x k' start S0 for L = min(ceil(eps^-1 ln(d/eps)), cap)
    iterations, then Algorithm 2 with C and the values z_i^T C z_i (the Ritz
    values).  Returns (theta descending, L)."""
    d = S0.shape[0]
    L = _iters(eps, d, cap)
    S = O.orth(S0)
    for _ in range(L):
        S = O.orth(apply(S))
    H = S.T @ apply(S)
    theta, _ = O.sym_eig_desc(0.5 * (H + H.T))
    return theta, L


@dataclass
class Stage:
    s: int                 # first index of the stage (1-based)
    q: int                 # last index found (1-based)
    kind: str              # "power" (Algorithm 4 found a gap) or "shift" (Algorithms 7, 5)
    lam_hat: np.ndarray    # Algorithm 3 on A_{-(s-1)}
    alg3_iters: int
    cols: int              # columns appended to U
    iters: int             # Algorithm 1 iterations of the block
    lam: float = float("nan")
    inv_est: np.ndarray | None = None
    d_iters: int = 0       # Algorithm 3 iterations on D
    shift_rounds: int = 0
    status: str = "ok"


@dataclass
class PartitionResult:
    U: np.ndarray
    ritz: np.ndarray
    stages: list = field(default_factory=list)
    status: str = "ok"
    delta: float = 0.0
    x_passes: int = 0
    solves: int = 0
    inner_steps: int = 0


def power_block(ctx: O.Context, b: int, eps: float, r_floor: float, seed: int):
    """Algorithm 1 on A (ctx's X) with b columns and no oversampling, then
    Algorithm 2 with the same A; stop by the outer loop's rule on
    E = ||X||_F^2 - sum of the b Ritz values."""
    o = ctx.opts
    S = O.orth(O.gaussian_block(seed, STREAM_BLOCK, 1, ctx.d, b))
    E: list[float] = []
    ell = 0
    while True:
        rho, Uh, _, _ = O.rayleigh_ritz(ctx.Xt, S)
        ctx.x_passes += 1
        E.append(ctx.fro2 - float(np.sum(rho)))
        if O.outer_stop(E, eps, ell, o.min_outer, r_floor) or ell >= o.max_outer:
            break
        S = O.orth(O.x_apply(ctx.Xt, S))
        ctx.x_passes += 2
        ell += 1
    return S @ Uh, rho, ell, ("ok" if ell < o.max_outer else "notconv")


def adaptive_solve(Xt, k: int, p: int, eps: float, seed: int, opts: O.Options | None = None,
                   delta: float = 0.0, part_max_iters: int = 2000) -> PartitionResult:
    """Algorithm 6 (all branches).  `delta` is the gap budget Delta (0: the
    hot path's estimate); `opts` sets the SVRG and outer-loop options of every
    stage (shift_policy is ignored: the shift-invert stages use Algorithm 7)."""
    opts = opts or O.Options()
    X64 = O.as64(Xt)
    d = X64.shape[1]
    if not (1 <= k < p < d):
        raise ValueError("need 1 <= k < p < d")
    if delta <= 0.0:
        delta = O.delta_estimate(O.Context(Xt, seed, opts), k, p)
    res = PartitionResult(U=np.zeros((d, 0)), ritz=np.zeros(0), delta=delta)
    Ucols = np.zeros((d, 0))
    s, t = 1, 0
    while s <= k:
        t += 1
        seed_t = O.stream_key(seed, STREAM_PART, t, 0)
        Xd = deflate(Xt, Ucols) if s > 1 else Xt
        ctx = O.Context(Xd, seed_t, opts)
        kk = k - s + 1

        def apply_a(S, c=ctx):
            c.x_passes += 2
            return O.x_apply(c.Xt, S)

        S0 = O.gaussian_block(seed_t, STREAM_BLOCK, 0, d, kk)
        lam_hat, it3 = alg3_values(apply_a, S0, 1.0 / (9.0 * p * p), part_max_iters)
        j = alg4(lam_hat, p)
        if j >= 0:
            q = s + j
            b = j + 1
            V, rho, ell, st = power_block(ctx, b, eps, (lam_hat[j + 1] / lam_hat[j]) ** 2, seed_t)
            stage = Stage(s=s, q=q, kind="power", lam_hat=lam_hat, alg3_iters=it3, cols=b, iters=ell,
                          status=st)
            new = V
        else:
            lam1_hat = O.lambda1_estimate(ctx)
            sh = O.shift_tune(ctx, lam1_hat, delta)
            if sh.status == "diverged":
                res.status = "diverged"
                break
            lam, mu = sh.lam, sh.mu_lb
            lam1_up = lam1_hat / (1.0 - 0.25)
            prev: dict = {}

            def apply_d(S, c=ctx):
                # warm start: the previous iteration's projection of D (Galerkin),
                # W0 = S C H C^T with H = S_prev^T D S_prev, C = S^T S_prev; the
                # first solve starts from S / (lambda - lambda_hat_s)
                if prev:
                    H = prev["S"].T @ prev["W"]
                    C = S.T @ prev["S"]
                    W0 = S @ (C @ (0.5 * (H + H.T)) @ C.T)
                else:
                    W0 = S / (lam - lam1_hat)
                W, st = c.solve_linear(S, W0, lam, mu, lam1_up)
                if st.status == "diverged":
                    raise RuntimeError("SVRG diverged")
                prev["S"], prev["W"] = S, W
                return W

            S0 = O.gaussian_block(seed_t, STREAM_BLOCK, 2, d, kk)
            theta, itd = alg3_values(apply_d, S0, 1.0 / (9.0 * p), part_max_iters)
            inv = 1.0 / theta
            jj = alg5(inv, delta)
            q = s + jj
            pp = p - (s - 1) if q == k else q - s + 1
            keep = pp if q == k else q - s + 1
            # rate floor of a block without oversampling: ((lambda - lambda_q) /
            # (lambda - lambda_{q+1}))^2 from Algorithm 3's estimates on D
            rf = None if q == k else (inv[jj] / inv[jj + 1]) ** 2
            r = O.subspace_on_d(ctx, q - s + 1, pp, eps, seed_t, lam, mu, lam1_up, rf)
            stage = Stage(s=s, q=q, kind="shift", lam_hat=lam_hat, alg3_iters=it3, cols=keep,
                          iters=r.outer_iters, lam=lam, inv_est=inv, d_iters=itd, shift_rounds=sh.rounds,
                          status=r.status)
            new = r.S @ r.Uh[:, :keep]
        res.stages.append(stage)
        res.x_passes += ctx.x_passes
        res.solves += ctx.solve_count
        res.inner_steps += ctx.inner_steps
        if stage.status != "ok":
            res.status = stage.status
        Ucols = O.orth(np.concatenate([Ucols, new], axis=1))
        s = q + 1
    # Algorithm 2 with X X^T on the orthonormalised columns (d x p)
    S = O.orth(Ucols)
    rho, Uh, _, _ = O.rayleigh_ritz(Xt, S)
    res.x_passes += 1
    res.U = S @ Uh[:, :k]
    res.ritz = rho[:k].copy()
    return res
