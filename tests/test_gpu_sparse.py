"""Parity of the sparse (CSR) CUDA path with the FP64 oracle (needs a GPU).

X is a seeded Zipf term-document matrix (lra_inputs.zipf_csr); the oracle
reads the same FP32 values through scipy.sparse and its factored inner loop
(itself pinned against the dense oracle).  Tolerances as for the dense FP32
path: relative 1e-5 for products, sums and the inner loop, sin-angle 1e-4 for
subspaces; the transposed structure and the column norms' inputs are exact.
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


class Csr:
    """A CSR X on the device plus the oracle's X^T (scipy, FP32 values)."""

    def __init__(self, ctx, d, n, seed, mean=20.0, on_device=False):
        self.d, self.n = d, n
        self.rowptr, self.colidx, self.val = L.zipf_csr(d, n, seed, mean_nnz=mean)
        X = sp.csr_matrix((self.val, self.colidx, self.rowptr), shape=(d, n))
        self.Xt = X.T.tocsr()
        nnz = int(self.rowptr[-1])
        if on_device:
            args = [torch.from_numpy(a).to(DEV) for a in (self.rowptr, self.colidx, self.val)]
        else:
            args = [self.rowptr, self.colidx, self.val]
        self.h = lra.lra_create_csr(ctx, d, n, nnz, *args, on_device)

    def close(self):
        lra.lra_mat_destroy(self.h)


@pytest.mark.parametrize("on_device", [False, True])
def test_create_and_colnorms(ctx, on_device):
    m = Csr(ctx, 700, 5000, 1, on_device=on_device)
    try:
        norm2 = torch.zeros(m.n, dtype=torch.float64, device=DEV)
        fro2 = lra.lra_colnorms(m.h, norm2)
        ref, fref = O.colnorms(m.Xt)
        assert rel(norm2.cpu().numpy(), ref) < 1e-13
        assert abs(fro2 / fref - 1) < 1e-13
        d, n, st, f = lra.lra_mat_info(m.h)
        assert (d, n) == (m.d, m.n) and abs(f / fref - 1) < 1e-13
    finally:
        m.close()


def test_invalid_csr_is_rejected(ctx):
    rowptr, colidx, val = L.zipf_csr(50, 400, 2, mean_nnz=5.0)
    nnz = int(rowptr[-1])

    def code(rp, ci, v, nz=nnz, n=400):
        out = ctypes.c_void_p()
        return lra.lib.lra_create_csr(ctx, 50, n, nz, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 0,
                                      ctypes.byref(out))

    ok = Csr.__new__(Csr)
    ok.h = lra.lra_create_csr(ctx, 50, 400, nnz, rowptr, colidx, val, False)   # the valid arrays pass
    ok.close()
    bad = rowptr.copy(); bad[10], bad[11] = bad[11], bad[10] - 1          # decreasing row pointer
    assert code(bad, colidx, val) == 1
    bad = colidx.copy(); bad[3] = 400                                    # column out of range
    assert code(rowptr, bad, val) == 1
    bad = colidx.copy(); bad[-1] = -1
    assert code(rowptr, bad, val) == 1
    r0 = int(np.argmax(np.diff(rowptr) >= 2))                            # duplicate column in a row
    bad = colidx.copy(); bad[rowptr[r0] + 1] = bad[rowptr[r0]]
    assert code(rowptr, bad, val) == 1
    bad = val.copy(); bad[7] = np.nan                                    # non-finite value
    assert code(rowptr, colidx, bad) == 1
    assert code(rowptr, colidx, val, nz=nnz - 1) == 1                    # rowptr[d] != nnz


@pytest.mark.parametrize("d,n,p", [(700, 5000, 13), (300, 2000, 40), (2000, 9000, 112), (129, 3000, 1)])
def test_anchor_and_products_match_oracle(ctx, d, n, p):
    m = Csr(ctx, d, n, d + p)
    try:
        rng = np.random.default_rng(p)
        Wt = rng.standard_normal((d, p)).astype(np.float32)
        B = rng.standard_normal((d, p)).astype(np.float32)
        lam = 1.7
        M = torch.zeros(p, d, dtype=torch.float32, device=DEV)
        nM2, nB2 = lra.lra_anchor(m.h, p, dev_block(Wt), dev_block(B), lam, M)
        W64, B64 = Wt.astype(np.float64), B.astype(np.float64)
        ref = O.anchor(m.Xt, W64, B64, lam)
        aX = abs(O.as64(m.Xt))                                   # |X|^T, sparse
        sY = np.asarray(aX @ np.abs(W64))
        sM = lam * np.abs(W64) + np.asarray(aX.T @ sY) + np.abs(B64)
        assert rel(cm(M), ref) < 1e-5
        assert elem_bound(cm(M), ref, sM) < 1e-5
        assert abs(nM2 / np.sum(ref ** 2) - 1) < 1e-5
        Y = torch.zeros(p, n, dtype=torch.float32, device=DEV)
        lra.lra_xt_mul(m.h, p, dev_block(Wt), Y)
        Yref = np.asarray(O.as64(m.Xt) @ W64)
        Yg = Y.double().cpu().numpy().T
        assert rel(Yg, Yref) < 1e-5
        assert elem_bound(Yg, Yref, sY) < 1e-5
        G = torch.zeros(p, d, dtype=torch.float32, device=DEV)
        lra.lra_x_mul(m.h, p, Y, G)
        Gref = np.asarray(O.as64(m.Xt).T @ Yg)
        assert rel(cm(G), Gref) < 1e-5
        assert elem_bound(cm(G), Gref, np.asarray(aX.T @ np.abs(Yg))) < 1e-5
    finally:
        m.close()


@pytest.mark.parametrize("d,n,p,steps", [(700, 5000, 13, 200), (700, 5000, 13, 3000), (300, 2000, 40, 3000)])
def test_inner_loop_matches_oracle(ctx, d, n, p, steps):
    """The solver's step size at lambda = 2 lambda_1; M scaled by lambda so that
    W - Wt stays O(1) (its fixed point is about -M/lambda); 3000 steps take the
    factor a below 2^-30, so the fold is exercised."""
    m = Csr(ctx, d, n, 3 * d)
    try:
        rng = np.random.default_rng(d + p)
        norm2, fro2 = O.colnorms(m.Xt)
        tab = O.sampling_table(norm2)
        lam1 = float(sp.linalg.eigsh(O.as64(m.Xt).T @ O.as64(m.Xt), k=1, return_eigenvectors=False)[0])
        lam = 2.0 * lam1
        Wt = rng.standard_normal((d, p)).astype(np.float32)
        M = (lam * rng.standard_normal((d, p))).astype(np.float32)
        W0 = (Wt + 0.5 * rng.standard_normal((d, p))).astype(np.float32)
        idx = O.sample_indices(tab, O.stream_key(9, O.STREAM_SVRG, 0, 0), steps)
        eta = 0.25 * lam1 / (lam * lam + tab.kappa * lam1)
        c = tab.c.astype(np.float32)
        W = dev_block(W0)
        lra.lra_svrg_inner(m.h, p, W, dev_block(Wt), dev_block(M), torch.from_numpy(idx.astype(np.int32)).to(DEV),
                           steps, torch.from_numpy(c).to(DEV), eta, lam)
        ref = O.svrg_epoch(m.Xt, W0.astype(np.float64), Wt.astype(np.float64), M.astype(np.float64),
                           idx, c.astype(np.float64), eta, lam)
        assert rel(cm(W) - Wt, ref - Wt) < 1e-5
        assert elem_rms(cm(W) - Wt, ref - Wt) < 1e-5
    finally:
        m.close()


@pytest.mark.parametrize("pol", ["far", "paper"])
def test_solve_matches_oracle_and_svd(ctx, pol):
    """k = 1: a Zipf X has one dominant direction (the head rows), so the q = k
    shift-and-invert iteration converges in a few outer steps; for k > 1 the
    rest of the spectrum is flat (lambda_2 ... lambda_21 within 12%), outside the
    method's regime without deflation."""
    d, n, k, p = 400, 6000, 1, 4
    m = Csr(ctx, d, n, 11, mean=15.0)
    try:
        U = torch.zeros(k, d, dtype=torch.float32, device=DEV)
        ritz = torch.zeros(k, dtype=torch.float64, device=DEV)
        rep = lra.LraReport()
        lp = lra.LRA_SHIFT_FAR if pol == "far" else lra.LRA_SHIFT_PAPER
        st = lra.lra_solve(m.h, k, p, 1e-3, 5, lra.options(shift_policy=lp), U, ritz, rep)
        assert st == 0
        Ug = cm(U)
        op = O.SHIFT_FAR if pol == "far" else O.SHIFT_PAPER
        ref = O.solve(m.Xt, k, p, 1e-3, 5, O.Options(shift_policy=op))
        Xd = O.as64(m.Xt).toarray()
        s = np.linalg.svd(Xd, compute_uv=False)
        opt = float(np.sum(s[k:] ** 2))
        ratio = O.frobenius_error(m.Xt, Ug) / opt
        assert 1.0 - 1e-6 <= ratio <= 1.0 + 1e-3
        assert np.max(np.abs(Ug.T @ Ug - np.eye(k))) < 1e-5
        assert O.sin_angle(ref.U, Ug) < 1e-4
        assert np.max(np.abs(ritz.cpu().numpy() - ref.ritz) / ref.ritz) < 1e-5
        assert rep.outer_iters == ref.outer_iters
    finally:
        m.close()


def test_fixed_schedule_matches_oracle_sparse(ctx):
    d, n, k, p = 300, 4000, 5, 10
    m = Csr(ctx, d, n, 21, mean=12.0)
    try:
        sched = dict(min_outer=8, max_outer=8, fixed_epochs=4)
        U = torch.zeros(k, d, dtype=torch.float32, device=DEV)
        ritz = torch.zeros(k, dtype=torch.float64, device=DEV)
        st = lra.lra_solve(m.h, k, p, 1e-3, 2, lra.options(shift_policy=lra.LRA_SHIFT_FAR, **sched), U, ritz)
        assert st in (0, 4)
        ref = O.solve(m.Xt, k, p, 1e-3, 2, O.Options(shift_policy=O.SHIFT_FAR, **sched))
        assert O.sin_angle(ref.U, cm(U)) < 1e-4
    finally:
        m.close()
