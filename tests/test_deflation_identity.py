"""The identities behind Algorithm 6's deflation applied on the fly.

A stage after the first works on X' = (I - U U^T) X for orthonormal U (d x c),
g_i = U^T x_i.  The library never forms X'; it uses

    X'^T W = X^T (W - U (U^T W)),   X' Y = (I - U U^T) X Y,
    ||x'_i||^2 = ||x_i||^2 - ||g_i||^2,   x'_i = x_i - U g_i,

and, for sparse X, an inner loop in factored form W - Wt = a (Z - U K) + b M
whose step is r = a (x_i^T Z - g_i^T L) + b (x_i^T M - g_i^T N) with L = U^T Z,
N = U^T M, both L and K advanced by (eta c / a') g_i r (so K = L - L0), and Z
rescaled with L and L0 when a falls below 2^-30.  Here those forms, written
out in FP64, must reproduce the oracle's operations on the materialised X'
(Sec. 3 assumes the projection applied to X's columns): the anchor, the column
norms and the SVRG epoch (Sec. 2.3), one sample and a batch per step.
"""
import math

import numpy as np
import pytest

from oracle import lra_oracle as O


def _problem(seed, d=40, n=90, c=3, p=4):
    rng = np.random.default_rng(seed)
    Xt = rng.standard_normal((n, d)) / math.sqrt(d)     # rows are the columns x_i
    U, _ = np.linalg.qr(rng.standard_normal((d, c)))
    Xd = Xt - (Xt @ U) @ U.T                            # rows (P x_i)^T
    return rng, Xt, U, Xd


def test_products_and_norms_of_the_deflated_matrix():
    rng, Xt, U, Xd = _problem(1)
    W = rng.standard_normal((Xt.shape[1], 5))
    B = rng.standard_normal(W.shape)
    lam = 2.5
    # X'^T W from the projected small operand; X' Y from the projected result
    Y = Xt @ (W - U @ (U.T @ W))
    assert np.allclose(Y, Xd @ W, rtol=0, atol=1e-12)
    G = Xt.T @ Y
    G = G - U @ (U.T @ G)
    M = lam * W - G - B
    assert np.allclose(M, O.anchor(Xd, W, B, lam), rtol=0, atol=1e-11)
    # deflated column norms
    g = Xt @ U
    n2 = O.colnorms(Xt)[0] - np.sum(g * g, axis=1)
    ref, fro2 = O.colnorms(Xd)
    assert np.allclose(n2, ref, rtol=0, atol=1e-13)
    assert abs(n2.sum() - fro2) <= 1e-12 * fro2


def factored_deflated_epoch(Xt, U, W, Wt, M, idx, c, eta, lam, batch=1):
    """The sparse kernels' deflated schedule in FP64."""
    X = np.asarray(Xt, dtype=np.float64).T              # d x n
    G = Xt @ U                                          # row i: g_i
    gam = 1.0 - eta * lam
    a, b = 1.0, 0.0
    Z = W - Wt
    L0 = U.T @ Z
    L = L0.copy()
    N = U.T @ M
    for t in range(len(idx) // batch):
        cols = idx[t * batch:(t + 1) * batch]
        # every r_u at the same state
        rs = [a * (X[:, i] @ Z - G[i] @ L) + b * (X[:, i] @ M - G[i] @ N) for i in cols]
        a1 = gam * a
        b = gam * b - eta
        for i, r in zip(cols, rs):
            coef = eta * c[i] / (a1 * batch)
            Z += coef * np.outer(X[:, i], r)
            L += coef * np.outer(G[i], r)
        a = a1
        if a < 2.0 ** -30:
            Z *= a
            L *= a
            L0 *= a
            a = 1.0
    return Wt + a * (Z - U @ (L - L0)) + b * M


@pytest.mark.parametrize("m,batch,eta_lam", [(0, 1, 0.05), (1, 1, 0.05), (57, 1, 0.05), (64, 1, 0.5),
                                             (40, 4, 0.05), (48, 2, 0.6)])
def test_factored_deflated_epoch_equals_the_epoch_on_the_deflated_matrix(m, batch, eta_lam):
    rng, Xt, U, Xd = _problem(10 + m + batch)
    d, p = Xt.shape[1], 4
    lam = 1.9
    eta = eta_lam / lam
    tab = O.sampling_table(O.colnorms(Xd)[0])
    idx = O.sample_indices(tab, O.stream_key(4, O.STREAM_SVRG, m, batch), m * batch)
    Wt = rng.standard_normal((d, p))
    W = Wt + 0.3 * rng.standard_normal((d, p))          # W != Wt: L0 != 0
    M = rng.standard_normal((d, p))
    ref = O.svrg_epoch(Xd, W, Wt, M, idx, tab.c, eta, lam, batch=batch)
    got = factored_deflated_epoch(Xt, U, W, Wt, M, idx, tab.c, eta, lam, batch)
    scale = max(1.0, float(np.abs(ref).max()))
    assert np.abs(got - ref).max() <= 1e-10 * scale


def test_a_wrong_deflation_term_is_caught():
    """Dropping the g_i^T L correction (stepping on x_i instead of x'_i in the
    product) must break the agreement above."""
    rng, Xt, U, Xd = _problem(7)
    d, p, m = Xt.shape[1], 4, 50
    lam, eta = 1.9, 0.05 / 1.9
    tab = O.sampling_table(O.colnorms(Xd)[0])
    idx = O.sample_indices(tab, O.stream_key(4, O.STREAM_SVRG, 1, 1), m)
    Wt = rng.standard_normal((d, p))
    W = Wt + 0.3 * rng.standard_normal((d, p))
    M = rng.standard_normal((d, p))
    ref = O.svrg_epoch(Xd, W, Wt, M, idx, tab.c, eta, lam)
    bad = factored_deflated_epoch(Xt, U * 0.0, W, Wt, M, idx, tab.c, eta, lam)
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()
