"""The first-order Cholesky factor behind CholeskyQR2's second pass.

After the first CholeskyQR pass the block Q has Gram G = Q^T Q = I + E with E
at the rounding level of that pass.  For ||E||_F <= 3e-5 the library takes
R = I + triu(E, 1) + diag(E) / 2 instead of the Cholesky factor of G.  Here, in
FP64: that R differs from the exact factor by at most ||E||_F^2, and Q R^-1 is
orthonormal to within a small multiple of ||E||_F^2, far below FP32 rounding;
a factor without the halved diagonal fails the same bound.
"""
import numpy as np
import pytest


def first_order_factor(G):
    E = G - np.eye(G.shape[0])
    return np.eye(G.shape[0]) + np.triu(E, 1) + np.diag(np.diag(E)) / 2.0


def _block(seed, d, p, size):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((d, p)))
    # perturb to a Gram I + E with ||E||_F about `size`
    P = rng.standard_normal((d, p))
    Q1 = Q + 0.5 * size / np.linalg.norm(Q.T @ P + P.T @ Q) * P
    return Q1


@pytest.mark.parametrize("p,size", [(10, 1e-6), (40, 1e-5), (100, 3e-5)])
def test_first_order_factor_is_the_cholesky_factor_to_second_order(p, size):
    Q1 = _block(p, 600, p, size)
    G = Q1.T @ Q1
    nE = np.linalg.norm(G - np.eye(p))
    assert nE <= 3e-5
    R_exact = np.linalg.cholesky(G).T            # upper, G = R^T R
    R = first_order_factor(G)
    assert np.linalg.norm(R - R_exact) <= nE ** 2
    Q2 = np.linalg.solve(R.T, Q1.T).T             # Q1 R^-1
    assert np.linalg.norm(Q2.T @ Q2 - np.eye(p)) <= 4.0 * nE ** 2


def test_a_factor_without_the_halved_diagonal_is_caught():
    p = 40
    Q1 = _block(3, 600, p, 1e-5)
    G = Q1.T @ Q1
    nE = np.linalg.norm(G - np.eye(p))
    E = G - np.eye(p)
    R_bad = np.eye(p) + np.triu(E, 0)             # full diagonal of E
    Q2 = np.linalg.solve(R_bad.T, Q1.T).T
    assert np.linalg.norm(Q2.T @ Q2 - np.eye(p)) > 10.0 * nE ** 2
