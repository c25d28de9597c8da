"""Pins of the oracle's sparse (compressed-column) path.

The sparse oracle reads the same X as its dense form: products go through
scipy.sparse, and the inner loop keeps W - Wt in the factored form a Z + b M so
a step costs O(nnz(x_i) p).  Each pin compares it with the dense definition
(dense oracle on X.toarray()) or with a brute-force SVD.
"""
import numpy as np
import pytest

sp = pytest.importorskip("scipy.sparse")

import lra_inputs as L
from oracle import lra_oracle as O


def _small(d=300, n=2000, mean=10.0, seed=7):
    rowptr, colidx, val = L.zipf_csr(d, n, seed, mean_nnz=mean)
    X = sp.csr_matrix((val, colidx, rowptr), shape=(d, n))
    return X.T.tocsr(), X.toarray().T.copy()       # X^T sparse (FP32), X^T dense (FP32)


def test_zipf_generator_properties():
    d, n, mean = 500, 4000, 12.0
    rowptr, colidx, val = L.zipf_csr(d, n, 3, mean_nnz=mean)
    assert rowptr.dtype == np.int64 and colidx.dtype == np.int32 and val.dtype == np.float32
    assert rowptr[0] == 0 and rowptr[-1] == colidx.size == val.size
    X = sp.csr_matrix((val, colidx, rowptr), shape=(d, n))
    # canonical CSR: strictly increasing column ids within each row (no duplicates)
    for r in range(d):
        seg = colidx[rowptr[r]:rowptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
    cnt = np.diff(X.tocsc().indptr)
    assert cnt.min() >= 1 and abs(cnt.mean() - mean) < 0.2
    nrm = np.asarray(X.multiply(X).sum(axis=0)).ravel()
    assert np.allclose(nrm, 1.0, atol=1e-5)
    # Zipf law: row 1 occurs more often than row 10, row 10 more than row 100
    occ = np.diff(rowptr)
    assert occ[0] > occ[9] > occ[99]
    # same arguments, same matrix
    r2, c2, v2 = L.zipf_csr(d, n, 3, mean_nnz=mean)
    assert np.array_equal(r2, rowptr) and np.array_equal(c2, colidx) and np.array_equal(v2, val)


def test_sparse_colnorms_and_apply_match_dense():
    Xs, Xd = _small()
    n2s, f2s = O.colnorms(Xs)
    n2d, f2d = O.colnorms(Xd)
    assert np.allclose(n2s, n2d, rtol=1e-14, atol=0)
    assert abs(f2s - f2d) <= 1e-12 * f2d
    W = np.random.default_rng(1).standard_normal((Xd.shape[1], 5))
    assert np.allclose(O.x_apply(Xs, W), O.x_apply(Xd, W), rtol=1e-12, atol=1e-12)
    rho_s, _, _, _ = O.rayleigh_ritz(Xs, np.linalg.qr(W)[0])
    rho_d, _, _, _ = O.rayleigh_ritz(Xd, np.linalg.qr(W)[0])
    assert np.allclose(rho_s, rho_d, rtol=1e-12)


@pytest.mark.parametrize("m", [200, 6000])  # (1 - eta lambda)^6000 < 2^-30: the factor is folded
def test_sparse_factored_epoch_equals_dense_epoch(m):
    Xs, Xd = _small()
    n, d = Xd.shape
    rng = np.random.default_rng(11)
    p = 4
    norm2, fro2 = O.colnorms(Xd)
    tab = O.sampling_table(norm2)
    lam1 = float(np.linalg.eigvalsh(Xd.T.astype(np.float64) @ Xd)[-1])
    lam = 2.0 * lam1
    eta = 0.25 * lam1 / (lam * lam + tab.kappa * lam1)   # the solver's step at mu = lambda_1
    if m == 6000:
        assert (1.0 - eta * lam) ** m < 2.0 ** -30
    Wt = rng.standard_normal((d, p))
    W = Wt + 0.1 * rng.standard_normal((d, p))      # Z starts at W - Wt != 0
    M = rng.standard_normal((d, p))
    idx = O.sample_indices(tab, O.stream_key(5, O.STREAM_SVRG, 0, 0), m)
    Wd = O.svrg_epoch(Xd, W, Wt, M, idx, tab.c, eta, lam)
    Ws = O.svrg_epoch(Xs, W, Wt, M, idx, tab.c, eta, lam)
    assert np.isfinite(Wd).all()
    assert np.linalg.norm(Ws - Wd) <= 1e-11 * np.linalg.norm(Wd)


def test_sparse_solve_meets_ratio_against_svd():
    Xs, Xd = _small(d=200, n=3000, mean=8.0, seed=9)
    k, p = 3, 6
    s = np.linalg.svd(Xd.astype(np.float64), compute_uv=False)
    opt = float(np.sum(s[k:] ** 2))
    r = O.solve(Xs, k, p, 1e-3, 0, O.Options(shift_policy=O.SHIFT_FAR))
    assert r.status == "ok"
    ratio = O.frobenius_error(Xs, r.U) / opt
    assert 1.0 - 1e-12 <= ratio <= 1.0 + 1e-3
    # the dense oracle on the same X and seeds gives the same subspace
    rd = O.solve(Xd, k, p, 1e-3, 0, O.Options(shift_policy=O.SHIFT_FAR))
    assert O.sin_angle(rd.U, r.U) < 1e-8
