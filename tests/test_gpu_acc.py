"""Parity of the accelerated solve (lra_options.acc) with the FP64 oracle's
acc_svrg_solve (needs a GPU).

Fixed schedules (every subproblem exactly `fixed_epochs` anchors, a fixed number
of subproblems) draw the same samples on both sides, so the iterates agree to
FP32 rounding: relative 2e-5 on W (FP32 X), as for the plain solve.  With the
residual stop, the solution must meet the dense system's residual bound and the
step counts must match the oracle's.
"""
import ctypes

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


def small_gap(d=256, n=2048, seed=31):
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt, _, s = L.planted_numpy(d, n, wl.sigma()[:d], seed)
    return np.ascontiguousarray(Xt.astype(np.float32)), s


@pytest.mark.parametrize("p,batch", [(6, 1), (1, 1), (16, 4)])
def test_fixed_schedule_matches_oracle(ctx, p, batch):
    Xt, s = small_gap()
    d = Xt.shape[1]
    rng = np.random.default_rng(p + batch)
    B = rng.standard_normal((d, p)).astype(np.float32)
    lam1 = float(s[0] ** 2)
    lam = 1.02 * lam1
    mu = lam - lam1
    seed, solve_id = 17, 3
    kw = dict(fixed_epochs=2, acc_max_outer=4, batch=batch)
    m = lra.lra_create_dense(ctx, d, Xt.shape[0], lra.LRA_F32, Xt, d, False, lra.LRA_F32)
    try:
        W = dev_block(np.zeros((d, p)))
        st, info = lra.lra_svrg_solve(m, p, dev_block(B), W, lam, mu, lam1, seed, solve_id,
                                      lra.options(acc=1, **kw))
        ctxo = O.Context(Xt, seed, O.Options(acc=1, **kw))
        ctxo.solve_count = solve_id
        g = ctxo.acc_gamma(lam, mu, lam1)
        assert g > 0.0
        Wo, sto = ctxo.acc_svrg_solve(B.astype(np.float64), np.zeros((d, p)), lam, mu, lam1)
        assert st == 0 and info.status == 0
        assert info.outer == sto.outer == 4 and ctxo.solve_count == solve_id + 4
        assert info.gamma == pytest.approx(g, rel=1e-12)
        assert info.inner_steps == sto.inner_steps and info.epochs == sto.epochs
        assert rel(cm(W), Wo) < 2e-5
        assert elem_rms(cm(W), Wo) < 2e-5
        assert info.residual == pytest.approx(sto.residual, rel=1e-3)
    finally:
        lra.lra_mat_destroy(m)


def test_residual_stop_meets_the_dense_bound(ctx):
    Xt, s = small_gap()
    n, d = Xt.shape
    p = 6
    rng = np.random.default_rng(2)
    B = rng.standard_normal((d, p)).astype(np.float32)
    lam1 = float(s[0] ** 2)
    lam = 1.01 * lam1
    mu = lam - lam1
    tau = 1e-5
    m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, lra.LRA_F32)
    try:
        W = dev_block(np.zeros((d, p)))
        st, info = lra.lra_svrg_solve(m, p, dev_block(B), W, lam, mu, lam1, 5, 0, lra.options(acc=1, tau=tau))
        assert st == 0 and info.status == 0 and info.outer > 1
        A = Xt.astype(np.float64).T @ Xt.astype(np.float64)
        r = np.linalg.norm((lam * np.eye(d) - A) @ cm(W) - B) / np.linalg.norm(B)
        assert r <= 2.0 * tau          # the anchor streams X as a BF16 pair (2^-17 relative)
        assert info.residual <= tau
        ctxo = O.Context(Xt, 5, O.Options(acc=1, tau=tau))
        Wo, sto = ctxo.acc_svrg_solve(B.astype(np.float64), np.zeros((d, p)), lam, mu, lam1)
        assert sto.status == "ok"
        Wstar = np.linalg.solve(lam * np.eye(d) - A, B.astype(np.float64))
        # ||(lam I - A)^{-1}|| = 1 / (lam - lambda_1) = 1 / mu here; at this shift
        # ||A W|| ~ 100 ||B||, so FP32 rounding of A W sits near tau itself
        bound = r * np.linalg.norm(B) / mu
        assert np.linalg.norm(cm(W) - Wstar) <= 1.05 * bound
        # same iteration within a subproblem or two (stops decided on FP32 vs FP64 norms)
        assert abs(info.outer - sto.outer) <= 2
        # and far fewer samples than the plain solve at the same shift
        Wp = dev_block(np.zeros((d, p)))
        stp, infop = lra.lra_svrg_solve(m, p, dev_block(B), Wp, lam, mu, lam1, 5, 0, lra.options(tau=tau))
        assert info.inner_steps < 0.5 * infop.inner_steps
    finally:
        lra.lra_mat_destroy(m)


def test_sparse_fixed_schedule_matches_oracle(ctx):
    d, n, p = 700, 5000, 5
    rowptr, colidx, val = L.zipf_csr(d, n, 77, mean_nnz=20.0)
    Xs = sp.csr_matrix((val, colidx, rowptr), shape=(d, n)).T.tocsr()
    A = O.as64(Xs).T @ O.as64(Xs)
    lam1 = float(sp.linalg.eigsh(A, k=1, return_eigenvectors=False)[0])
    lam = 1.05 * lam1
    mu = lam - lam1
    rng = np.random.default_rng(8)
    B = rng.standard_normal((d, p)).astype(np.float32)
    kw = dict(fixed_epochs=2, acc_max_outer=3)
    m = lra.lra_create_csr(ctx, d, n, int(rowptr[-1]), rowptr, colidx, val, False)
    try:
        W = dev_block(np.zeros((d, p)))
        st, info = lra.lra_svrg_solve(m, p, dev_block(B), W, lam, mu, lam1, 9, 0, lra.options(acc=1, **kw))
        ctxo = O.Context(Xs, 9, O.Options(acc=1, **kw))
        assert ctxo.acc_gamma(lam, mu, lam1) > 0.0
        Wo, sto = ctxo.acc_svrg_solve(B.astype(np.float64), np.zeros((d, p)), lam, mu, lam1)
        assert st == 0 and info.outer == 3 and info.inner_steps == sto.inner_steps
        assert rel(cm(W), Wo) < 2e-5
        assert elem_rms(cm(W), Wo) < 2e-5
    finally:
        lra.lra_mat_destroy(m)


def test_far_shift_is_the_plain_solve(ctx):
    """gamma = 0 (an epoch already within n samples): bit-identical to acc = 0."""
    Xt, s = small_gap()
    n, d = Xt.shape
    p = 4
    B = np.random.default_rng(4).standard_normal((d, p)).astype(np.float32)
    lam1_up = float(s[0] ** 2) / 0.75
    lam = 2.0 * lam1_up
    m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, lra.LRA_F32)
    try:
        Wa, Wb = dev_block(np.zeros((d, p))), dev_block(np.zeros((d, p)))
        _, ia = lra.lra_svrg_solve(m, p, dev_block(B), Wa, lam, lam - lam1_up, lam1_up, 1, 0, lra.options(acc=1))
        _, ib = lra.lra_svrg_solve(m, p, dev_block(B), Wb, lam, lam - lam1_up, lam1_up, 1, 0, lra.options())
        assert ia.gamma == 0.0 and ia.outer == 0
        assert torch.equal(Wa, Wb) and ia.inner_steps == ib.inner_steps
    finally:
        lra.lra_mat_destroy(m)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_accelerated_low_rank_solve_meets_eps(ctx, storage):
    """lra_solve with every solve accelerated, at a fixed shift close to
    lambda_1 (the regime where plain SVRG would need epochs of ~100 n)."""
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt64, _, s = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    k, p, eps = wl.k, wl.p, 1e-3
    lam1 = float(s[0] ** 2)
    st_ = lra.LRA_F32 if storage == "f32" else lra.LRA_BF16
    m = lra.lra_create_dense(ctx, wl.d, wl.n, lra.LRA_F64, Xt64, wl.d, False, st_)
    try:
        U = torch.zeros(k, wl.d, dtype=torch.float32, device=DEV)
        ritz = torch.zeros(k, dtype=torch.float64, device=DEV)
        rep = lra.LraReport()
        lam = 1.35 * lam1
        o = lra.options(shift_policy=lra.LRA_SHIFT_FIXED, lambda_=lam, lambda1_hat=lam1, acc=1)
        st = lra.lra_solve(m, k, p, eps, 0, o, U, ritz, rep)
        assert st == 0
        ratio = O.frobenius_error(Xt64, cm(U)) / wl.opt()
        assert 1.0 - 1e-6 <= ratio <= 1.0 + eps
        ctxo = O.Context(Xt64, 0, O.Options())
        assert ctxo.acc_gamma(lam, lam - lam1 / 0.75, lam1 / 0.75) > 0.0
        # one solve id per subproblem: more solves than outer iterations
        assert rep.solves > rep.outer_iters
    finally:
        lra.lra_mat_destroy(m)


def test_bad_acc_options_are_rejected(ctx):
    Xt, s = small_gap(d=64, n=256)
    n, d = Xt.shape
    m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, lra.LRA_F32)
    try:
        U = torch.zeros(2, d, dtype=torch.float32, device=DEV)
        ritz = torch.zeros(2, dtype=torch.float64, device=DEV)
        for bad in (dict(acc=2), dict(acc=1, acc_theta=0.0), dict(acc=1, acc_theta=1.5),
                    dict(acc=1, acc_max_outer=0), dict(acc=1, acc_target=-1)):
            o = lra.options(**bad)
            assert lra.lib.lra_solve(m, 2, 4, 1e-3, 0, ctypes.byref(o), U.data_ptr(), ritz.data_ptr(), None) == 1
    finally:
        lra.lra_mat_destroy(m)
