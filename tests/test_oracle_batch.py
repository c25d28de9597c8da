"""Pins of the oracle's minibatch inner step (a reading beyond the paper:
b samples per step, the stochastic term averaged; b = 1 is Sec. 2.3's step).

The batched step must be an unbiased estimate of the exact gradient step (by
enumeration of all ordered pairs for b = 2), reduce to the b = 1 step when the
batch repeats one index, agree between the dense and the sparse (factored)
oracle, and still solve the linear system to the stated residual.
"""
import itertools
import math

import numpy as np
import pytest

import lra_inputs as L
from oracle import lra_oracle as O


def _problem(seed=6, d=16, n=12, p=3):
    rng = np.random.default_rng(seed)
    Xt = rng.standard_normal((n, d)) / math.sqrt(n)
    A = Xt.T @ Xt                     # dense X X^T, formed explicitly
    lam1 = float(np.linalg.eigvalsh(A)[-1])
    lam = 1.3 * lam1
    B = rng.standard_normal((d, p))
    return rng, Xt, A, lam1, lam, B


def test_batched_step_is_unbiased_gradient_step():
    """E over two i.i.d. samples of one b = 2 step = W - eta grad F(W)."""
    rng, Xt, A, lam1, lam, B = _problem()
    n = Xt.shape[0]
    tab = O.sampling_table(O.colnorms(Xt)[0])
    q = tab.weights.astype(np.float64) / tab.total
    Wt = rng.standard_normal(B.shape)
    W = Wt + 0.3 * rng.standard_normal(B.shape)
    M = O.anchor(Xt, Wt, B, lam)
    eta = 0.01
    mean = np.zeros_like(W)
    for i, j in itertools.product(range(n), repeat=2):
        mean += q[i] * q[j] * O.svrg_epoch(Xt, W, Wt, M, np.array([i, j]), tab.c, eta, lam, batch=2)
    grad = (lam * np.eye(A.shape[0]) - A) @ W - B
    assert np.allclose(mean, W - eta * grad, rtol=1e-11, atol=1e-11)


def test_batch_of_one_repeated_index_is_the_single_step():
    rng, Xt, A, lam1, lam, B = _problem(seed=8)
    tab = O.sampling_table(O.colnorms(Xt)[0])
    Wt = rng.standard_normal(B.shape)
    W = Wt + 0.2 * rng.standard_normal(B.shape)
    M = O.anchor(Xt, Wt, B, lam)
    seq = np.array([3, 7, 1])
    one = O.svrg_epoch(Xt, W, Wt, M, seq, tab.c, 0.02, lam, batch=1)
    rep = O.svrg_epoch(Xt, W, Wt, M, np.repeat(seq, 4), tab.c, 0.02, lam, batch=4)
    assert np.allclose(rep, one, rtol=1e-13, atol=1e-13)


def test_step_size_and_epoch_length():
    rng, Xt, A, lam1, lam, B = _problem()
    ctx1 = O.Context(Xt, 0, O.Options())
    ctx4 = O.Context(Xt, 0, O.Options(batch=4))
    mu, l1u = lam - lam1, lam1 / 0.75
    eta1, m1 = ctx1.step_params(lam, mu, l1u)
    eta4, m4 = ctx4.step_params(lam, mu, l1u)
    kap = ctx1.table.kappa
    assert eta1 == pytest.approx(0.25 * mu / (lam ** 2 + kap * l1u), rel=1e-15)
    assert eta4 == pytest.approx(0.25 * mu / (lam ** 2 + kap * l1u / 4), rel=1e-15)
    assert m1 == math.ceil(2.0 / (eta1 * mu)) or m1 == 50 * Xt.shape[0]
    assert m4 == min(math.ceil(2.0 / (eta4 * mu)), 50 * Xt.shape[0] // 4)


def test_sparse_batched_epoch_equals_dense():
    sp = pytest.importorskip("scipy.sparse")
    rowptr, colidx, val = L.zipf_csr(300, 2000, 7, mean_nnz=10.0)
    X = sp.csr_matrix((val, colidx, rowptr), shape=(300, 2000))
    Xs, Xd = X.T.tocsr(), X.toarray().T.copy()
    rng = np.random.default_rng(2)
    tab = O.sampling_table(O.colnorms(Xd)[0])
    lam1 = float(np.linalg.eigvalsh(Xd.T.astype(np.float64) @ Xd)[-1])
    lam = 2.0 * lam1
    eta = 0.25 * lam1 / (lam * lam + tab.kappa * lam1 / 8)
    Wt = rng.standard_normal((300, 4))
    W = Wt + 0.1 * rng.standard_normal((300, 4))
    M = rng.standard_normal((300, 4))
    idx = O.sample_indices(tab, O.stream_key(5, O.STREAM_SVRG, 0, 0), 8 * 700)
    Wd = O.svrg_epoch(Xd, W, Wt, M, idx, tab.c, eta, lam, batch=8)
    Ws = O.svrg_epoch(Xs, W, Wt, M, idx, tab.c, eta, lam, batch=8)
    assert np.isfinite(Wd).all()
    assert np.linalg.norm(Ws - Wd) <= 1e-11 * np.linalg.norm(Wd)


@pytest.mark.parametrize("batch", [4, 16])
def test_batched_svrg_solve_matches_dense_solve(batch):
    rng, Xt, A, lam1, lam, B = _problem(seed=3, d=20, n=90, p=4)
    ctx = O.Context(Xt, 3, O.Options(tau=1e-10, batch=batch))
    W, st = ctx.svrg_solve(B, np.zeros_like(B), lam, lam - lam1, lam1)
    Wstar = np.linalg.solve(lam * np.eye(A.shape[0]) - A, B)
    assert st.status == "ok" and st.residual <= 1e-10
    assert np.linalg.norm(W - Wstar) <= 1e-10 * np.linalg.norm(B) / (lam - lam1) * 1.01


def test_batched_solve_meets_ratio():
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt, U, s = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    r = O.solve(Xt, wl.k, wl.p, 1e-3, 0, O.Options(shift_policy=O.SHIFT_FAR, batch=8))
    assert r.status == "ok"
    ratio = O.frobenius_error(Xt, r.U) / wl.opt()
    assert 1.0 - 1e-12 <= ratio <= 1.0 + 1e-3
