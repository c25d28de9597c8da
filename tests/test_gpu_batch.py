"""Parity of the minibatch inner loop (lra_options.batch, lra_svrg_inner_batched)
with the FP64 oracle's batched step (needs a GPU).  Tolerances as for the
one-sample loop: relative 1e-5 on W - Wt (FP32 X), sin-angle 1e-4 on solves."""
import ctypes
import math

import numpy as np
import pytest

import lra_inputs as L
from oracle import lra_oracle as O

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1607_02925_gb300 as lra  # noqa: E402

DEV = "cuda"


from measures import elem_bound, elem_rms, rel  # noqa: E402,F401


def cm(t):
    return t.double().cpu().numpy().T


def dev_block(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T)).to(DEV)


@pytest.fixture(scope="module")
def ctx():
    c = lra.lra_init(0)
    yield c
    lra.lra_finalize(c)


def planted(d, n, k, seed):
    Xt, U, s = L.planted_numpy(d, n, L.sigma_serving(k, min(d, n)), seed)
    return np.ascontiguousarray(Xt.astype(np.float32))


@pytest.mark.parametrize("d,n,p,batch,storage", [(300, 3000, 13, 4, "f32"), (128, 777, 40, 16, "f32"),
                                                  (1024, 2000, 3, 2, "f32"), (512, 1500, 10, 8, "bf16")])
def test_dense_batched_inner_matches_oracle(ctx, d, n, p, batch, storage):
    Xt = planted(d, n, 5, 3 * d + batch)
    st = lra.LRA_F32 if storage == "f32" else lra.LRA_BF16
    if storage == "bf16":
        b = np.ascontiguousarray(Xt).view(np.uint32).astype(np.uint64)
        Xo = (((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32)
    else:
        Xo = Xt
    rng = np.random.default_rng(d + p + batch)
    tab = O.sampling_table(O.colnorms(Xo)[0])
    A = Xo.astype(np.float64).T @ Xo.astype(np.float64)
    lam1 = float(np.linalg.eigvalsh(A)[-1])
    lam = 2.0 * lam1
    eta = 0.25 * lam1 / (lam * lam + tab.kappa * lam1 / batch)
    steps = 300
    idx = O.sample_indices(tab, O.stream_key(4, O.STREAM_SVRG, 0, batch), steps * batch)
    Wt = rng.standard_normal((d, p)).astype(np.float32)
    M = (lam * rng.standard_normal((d, p))).astype(np.float32)
    W0 = (Wt + 0.5 * rng.standard_normal((d, p))).astype(np.float32)
    c = tab.c.astype(np.float32)
    m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, st)
    try:
        W = dev_block(W0)
        lra.lra_svrg_inner_batched(m, p, W, dev_block(Wt), dev_block(M), torch.from_numpy(idx.astype(np.int32)).to(DEV),
                                   steps, batch, torch.from_numpy(c).to(DEV), eta, lam)
        ref = O.svrg_epoch(Xo, W0.astype(np.float64), Wt.astype(np.float64), M.astype(np.float64), idx,
                           c.astype(np.float64), eta, lam, batch=batch)
        assert rel(cm(W) - Wt, ref - Wt) < 1e-5
        assert elem_rms(cm(W) - Wt, ref - Wt) < 1e-5
    finally:
        lra.lra_mat_destroy(m)


@pytest.mark.parametrize("batch,steps", [(4, 60), (8, 500)])   # 500 steps take the factor below 2^-30
def test_sparse_batched_inner_matches_oracle(ctx, batch, steps):
    d, n, p = 700, 5000, 13
    rowptr, colidx, val = L.zipf_csr(d, n, 2100, mean_nnz=20.0)
    Xs = sp.csr_matrix((val, colidx, rowptr), shape=(d, n)).T.tocsr()
    m = lra.lra_create_csr(ctx, d, n, int(rowptr[-1]), rowptr, colidx, val, False)
    try:
        rng = np.random.default_rng(batch)
        tab = O.sampling_table(O.colnorms(Xs)[0])
        A = O.as64(Xs).T @ O.as64(Xs)
        lam1 = float(sp.linalg.eigsh(A, k=1, return_eigenvectors=False)[0])
        lam = 2.0 * lam1
        eta = 0.25 * lam1 / (lam * lam + tab.kappa * lam1 / batch)
        idx = O.sample_indices(tab, O.stream_key(9, O.STREAM_SVRG, 1, batch), steps * batch)
        Wt = rng.standard_normal((d, p)).astype(np.float32)
        M = (lam * rng.standard_normal((d, p))).astype(np.float32)
        W0 = (Wt + 0.5 * rng.standard_normal((d, p))).astype(np.float32)
        c = tab.c.astype(np.float32)
        W = dev_block(W0)
        lra.lra_svrg_inner_batched(m, p, W, dev_block(Wt), dev_block(M), torch.from_numpy(idx.astype(np.int32)).to(DEV),
                                   steps, batch, torch.from_numpy(c).to(DEV), eta, lam)
        ref = O.svrg_epoch(Xs, W0.astype(np.float64), Wt.astype(np.float64), M.astype(np.float64), idx,
                           c.astype(np.float64), eta, lam, batch=batch)
        assert rel(cm(W) - Wt, ref - Wt) < 1e-5
        assert elem_rms(cm(W) - Wt, ref - Wt) < 1e-5
    finally:
        lra.lra_mat_destroy(m)


def test_batched_solve_matches_oracle_and_meets_eps(ctx):
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt64, _, _ = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    Xt = np.ascontiguousarray(Xt64.astype(np.float32))
    m = lra.lra_create_dense(ctx, wl.d, wl.n, lra.LRA_F64, Xt64, wl.d, False, lra.LRA_F32)
    try:
        U = torch.zeros(wl.k, wl.d, dtype=torch.float32, device=DEV)
        ritz = torch.zeros(wl.k, dtype=torch.float64, device=DEV)
        # fixed schedule: trajectory parity with the oracle at batch 8
        sched = dict(min_outer=10, max_outer=10, fixed_epochs=4)
        st = lra.lra_solve(m, wl.k, wl.p, 1e-3, 0, lra.options(shift_policy=lra.LRA_SHIFT_FAR, batch=8, **sched),
                           U, ritz)
        assert st in (0, 4)
        ref = O.solve(Xt, wl.k, wl.p, 1e-3, 0, O.Options(shift_policy=O.SHIFT_FAR, batch=8, **sched))
        assert O.sin_angle(ref.U, cm(U)) < 1e-4
        # default stop rule with the paper's shift policy and a batch of 16
        s = wl.sigma()
        delta = (s[wl.k - 1] ** 2 - s[wl.p] ** 2) / 1.5
        rep = lra.LraReport()
        st = lra.lra_solve(m, wl.k, wl.p, 1e-3, 0, lra.options(shift_policy=lra.LRA_SHIFT_PAPER, delta=delta,
                                                               batch=16), U, ritz, rep)
        assert st == 0
        ratio = O.frobenius_error(Xt64, cm(U)) / wl.opt()
        assert 1.0 - 1e-6 <= ratio <= 1.0 + 1e-3
    finally:
        lra.lra_mat_destroy(m)


def test_batch_errors(ctx):
    d, n = 4096, 600
    Xt = planted(d, n, 3, 1)
    m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, lra.LRA_F32)
    try:
        U = torch.zeros(3, d, device=DEV)
        r = torch.zeros(3, dtype=torch.float64, device=DEV)
        for b, code in [(3, 1), (32, 1), (0, 1)]:
            o = lra.options(shift_policy=lra.LRA_SHIFT_FAR, batch=b)
            assert lra.lib.lra_solve(m, 3, 6, 1e-3, 0, ctypes.byref(o), U.data_ptr(), r.data_ptr(), None) == code
        # d = 4096 FP32: a ring of 2 x 16 columns does not fit in shared memory
        o = lra.options(shift_policy=lra.LRA_SHIFT_FAR, batch=16)
        assert lra.lib.lra_solve(m, 3, 6, 1e-3, 0, ctypes.byref(o), U.data_ptr(), r.data_ptr(), None) == 11
    finally:
        lra.lra_mat_destroy(m)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_dense_input_returns_a_status(ctx, bad):
    """A NaN or Inf entry in a dense X makes ||X||_F^2 non-finite: the solve
    returns LRA_EINVAL before any iteration, and the context still solves the
    next matrix."""
    d, n = 256, 800
    Xt = planted(d, n, 3, 5)
    Xbad = Xt.copy()
    Xbad[17, 40] = bad
    U = torch.zeros(3, d, device=DEV)
    r = torch.zeros(3, dtype=torch.float64, device=DEV)
    o = lra.options(shift_policy=lra.LRA_SHIFT_FAR)
    m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xbad, d, False, lra.LRA_F32)
    try:
        st = lra.lib.lra_solve(m, 3, 6, 1e-3, 0, ctypes.byref(o), U.data_ptr(), r.data_ptr(), None)
        assert st == 1
    finally:
        lra.lra_mat_destroy(m)
    m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, lra.LRA_F32)
    try:
        assert lra.lib.lra_solve(m, 3, 6, 1e-3, 0, ctypes.byref(o), U.data_ptr(), r.data_ptr(), None) == 0
    finally:
        lra.lra_mat_destroy(m)
