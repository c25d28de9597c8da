"""Parity of every step of the CUDA path with the FP64 oracle (needs a GPU).

All inputs are seeded and synthetic (lra_inputs, or a test-local numpy
generator for arbitrary step inputs); every expected value comes from
oracle/.  Tolerances:
  * integer / index work (sampling weights, prefix sums, sampled indices): exact;
  * FP32 arithmetic over sums of N terms: relative 1e-5 (the stated accuracy of the
    FP32 path; the observed error is ~1e-6);
  * subspaces: sin of the largest principal angle <= 1e-4 (FP32 X), 1e-3 (BF16 X).
"""
import math

import numpy as np
import pytest

import lra_inputs as L
from oracle import lra_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1607_02925_gb300 as lra  # noqa: E402

DEV = "cuda"


from measures import elem_bound, elem_rms, rel  # noqa: E402


def cm(t):
    """torch (p, d) row-major tensor holding a d x p column-major block -> numpy d x p."""
    return t.double().cpu().numpy().T


def dev_block(A):
    """numpy d x p -> device FP32 buffer laid out column-major (leading dim d)."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T)).to(DEV)


@pytest.fixture(scope="module")
def ctx():
    c = lra.lra_init(0)
    yield c
    lra.lra_finalize(c)


class Mat:
    def __init__(self, ctx, Xt, storage=lra.LRA_F32, src=None):
        self.Xt = Xt
        self.n, self.d = Xt.shape
        if src is None:
            src = np.ascontiguousarray(Xt.astype(np.float32))
        dt = {np.dtype(np.float32): lra.LRA_F32, np.dtype(np.float64): lra.LRA_F64}[src.dtype]
        self.h = lra.lra_create_dense(ctx, self.d, self.n, dt, src, self.d, False, storage)

    def close(self):
        lra.lra_mat_destroy(self.h)


def planted(d, n, k, seed, r=None):
    sig = L.sigma_serving(k, r or min(d, n))
    Xt, U, s = L.planted_numpy(d, n, sig, seed)
    return np.ascontiguousarray(Xt.astype(np.float32)), U, s


def bf16_values(x32):
    """Round-to-nearest-even FP32 -> BF16 values (as FP32), for the oracle's copy
    of a BF16-stored matrix."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def f16_values(x32):
    """The values an FP16-stored matrix holds: fp16(s x) / s with s the power of
    two that puts max |x| in [2^14, 2^15), rounded to nearest even."""
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    mx = float(np.max(np.abs(x32)))
    e = math.frexp(mx)[1]
    sc = math.ldexp(1.0, 15 - e)
    return ((x32.astype(np.float64) * sc).astype(np.float16).astype(np.float64) / sc)


def stored_values(Xt, storage):
    if storage == lra.LRA_BF16:
        return bf16_values(Xt)
    if storage == lra.LRA_F16:
        return f16_values(Xt)
    return Xt


# ragged d, n, p; p = 100 and 64 take the two-M-tile tensor-core kernels for BF16
# X (d = 520 -> 5 row tiles of 128: the last CTA's second tile lies past dpad)
SHAPES = [(300, 3000, 13), (256, 2048, 10), (128, 777, 40), (520, 1500, 48), (520, 1500, 100),
          (1100, 3001, 64)]


# ---------------------------------------------------------------------------
# a0: column norms, sampling table, sampler
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage", [lra.LRA_F32, lra.LRA_BF16, lra.LRA_F16])
def test_colnorms(ctx, storage):
    Xt, _, _ = planted(300, 3001, 5, 1)
    if storage == lra.LRA_BF16:
        Xt = bf16_values(Xt)
    m = Mat(ctx, Xt, storage)
    if storage == lra.LRA_F16:
        Xt = f16_values(Xt)
    try:
        n2 = torch.zeros(m.n, dtype=torch.float64, device=DEV)
        fro2 = lra.lra_colnorms(m.h, n2)
        ref, reff = O.colnorms(Xt)
        assert rel(n2.cpu().numpy(), ref) < 1e-13
        assert abs(fro2 / reff - 1) < 1e-13
    finally:
        m.close()


@pytest.mark.parametrize("mode", [lra.LRA_SAMPLE_IMPORTANCE, lra.LRA_SAMPLE_UNIFORM])
@pytest.mark.parametrize("n", [1, 1000, 5000, 70001])
def test_sampling_table_and_sampler_bit_exact(ctx, mode, n):
    rng = np.random.default_rng(n)
    norm2 = rng.gamma(1.5, 1.0, size=n)
    norm2[::13] = 0.0
    if n > 1:
        norm2[1] = 1e-300
    if not np.any(norm2 > 0):
        norm2[0] = 1.0
    tab = O.sampling_table(norm2, mode)
    nd = torch.from_numpy(norm2).to(DEV)
    cum = torch.zeros(n, dtype=torch.int64, device=DEV)
    c = torch.zeros(n, dtype=torch.float32, device=DEV)
    total, kappa = lra.lra_sampling_table(ctx, n, nd, mode, cum, c)
    assert total == tab.total
    assert kappa == tab.kappa
    assert np.array_equal(cum.cpu().numpy().view(np.uint64), tab.cum)
    assert np.array_equal(c.cpu().numpy(), tab.c.astype(np.float32))
    for key in [O.stream_key(3, O.STREAM_SVRG, 0, 0), O.stream_key(9, O.STREAM_SVRG, 17, 5)]:
        for mm in [0, 1, 1000, 65537]:
            idx = torch.zeros(max(mm, 1), dtype=torch.int32, device=DEV)
            lra.lra_sample(ctx, n, cum, total, key, mm, idx)
            ref = O.sample_indices(tab, key, mm)
            assert np.array_equal(idx.cpu().numpy()[:mm].astype(np.int64), ref)


def test_gaussian_block(ctx):
    for d, p, a in [(300, 13, 0), (4096, 1, 2), (97, 5, 3)]:
        out = torch.zeros(p, d, dtype=torch.float32, device=DEV)
        lra.lra_gaussian_block(ctx, 11, O.STREAM_INIT, a, d, p, out)
        ref = O.gaussian_block(11, O.STREAM_INIT, a, d, p)
        assert np.max(np.abs(cm(out) - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))


# ---------------------------------------------------------------------------
# a6 / a4: products with X and the anchor pass
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,n,p", SHAPES)
@pytest.mark.parametrize("storage", [lra.LRA_F32, lra.LRA_BF16, lra.LRA_F16])
def test_anchor_matches_oracle(ctx, d, n, p, storage):
    Xt, _, _ = planted(d, n, 5, d + n)
    if storage == lra.LRA_BF16:
        Xt = bf16_values(Xt)
    rng = np.random.default_rng(p)
    Wt = rng.standard_normal((d, p)).astype(np.float32)
    B = rng.standard_normal((d, p)).astype(np.float32)
    lam = 1.7
    m = Mat(ctx, Xt, storage)
    if storage == lra.LRA_F16:
        Xt = f16_values(Xt)
    try:
        M = torch.zeros(p, d, dtype=torch.float32, device=DEV)
        nM2, nB2 = lra.lra_anchor(m.h, p, dev_block(Wt), dev_block(B), lam, M)
        W64, B64 = Wt.astype(np.float64), B.astype(np.float64)
        ref = O.anchor(Xt, W64, B64, lam)
        aX = np.abs(np.asarray(Xt, dtype=np.float64))          # n x d = |X|^T
        sY = aX @ np.abs(W64)                                    # |X|^T |W|
        sM = lam * np.abs(W64) + aX.T @ sY + np.abs(B64)         # |lam W| + |X| |X|^T |W| + |B|
        assert rel(cm(M), ref) < 1e-5
        assert elem_bound(cm(M), ref, sM) < 1e-5
        assert abs(nM2 / np.sum(ref ** 2) - 1) < 1e-5
        assert abs(nB2 / np.sum(B64 ** 2) - 1) < 1e-12
        # the two passes separately
        Y = torch.zeros(p, n, dtype=torch.float32, device=DEV)
        lra.lra_xt_mul(m.h, p, dev_block(Wt), Y)
        Yref = np.asarray(Xt, dtype=np.float64) @ W64
        Yg = Y.double().cpu().numpy().T
        assert rel(Yg, Yref) < 1e-5
        assert elem_bound(Yg, Yref, sY) < 1e-5
        G = torch.zeros(p, d, dtype=torch.float32, device=DEV)
        lra.lra_x_mul(m.h, p, Y, G)
        Gref = np.asarray(Xt, dtype=np.float64).T @ Yg
        assert rel(cm(G), Gref) < 1e-5
        assert elem_bound(cm(G), Gref, aX.T @ np.abs(Yg)) < 1e-5
    finally:
        m.close()


# ---------------------------------------------------------------------------
# a7: inner loop and the whole SVRG solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,n,p", [(300, 3000, 13), (128, 777, 40), (1024, 2000, 3)])
def test_inner_loop_matches_oracle(ctx, d, n, p):
    Xt, _, _ = planted(d, n, 5, 3 * d)
    rng = np.random.default_rng(d + p)
    Wt = rng.standard_normal((d, p)).astype(np.float32)
    M = (0.1 * rng.standard_normal((d, p))).astype(np.float32)
    W0 = (Wt + 0.05 * rng.standard_normal((d, p))).astype(np.float32)
    steps = 700
    idx = rng.integers(0, n, size=steps).astype(np.int32)
    c = rng.uniform(0.5, 2.0, size=n).astype(np.float32) * n / 5
    eta, lam = 0.02, 1.3
    m = Mat(ctx, Xt)
    try:
        W = dev_block(W0)
        lra.lra_svrg_inner(m.h, p, W, dev_block(Wt), dev_block(M), torch.from_numpy(idx).to(DEV),
                           steps, torch.from_numpy(c).to(DEV), eta, lam)
        ref = O.svrg_epoch(Xt, W0.astype(np.float64), Wt.astype(np.float64), M.astype(np.float64),
                           idx.astype(np.int64), c.astype(np.float64), eta, lam)
        assert rel(cm(W) - Wt, ref - Wt) < 1e-5
        assert elem_rms(cm(W) - Wt, ref - Wt) < 1e-5
        # m = 0 leaves W unchanged
        W = dev_block(W0)
        lra.lra_svrg_inner(m.h, p, W, dev_block(Wt), dev_block(M), None, 0, None, eta, lam)
        assert np.array_equal(cm(W).astype(np.float32), W0)
    finally:
        m.close()


def test_svrg_solve_matches_oracle_and_dense_solve(ctx):
    d, n, p = 256, 2048, 6
    Xt, _, s = planted(d, n, 5, 77)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((d, p)).astype(np.float32)
    lam1 = float(s[0] ** 2)
    lam1_up = lam1 / 0.75
    lam = 2.0 * lam1_up
    mu = lam - lam1_up
    seed, solve_id = 123, 4
    opt = lra.options(tau=1e-5)
    m = Mat(ctx, Xt)
    try:
        W = dev_block(np.zeros((d, p)))
        st, info = lra.lra_svrg_solve(m.h, p, dev_block(B), W, lam, mu, lam1_up, seed, solve_id, opt)
        assert st == 0 and info.residual <= 1e-5
        ctxo = O.Context(Xt, seed, O.Options(tau=1e-5))
        ctxo.solve_count = solve_id
        Wo, sto = ctxo.svrg_solve(B.astype(np.float64), np.zeros((d, p)), lam, mu, lam1_up)
        A = np.asarray(Xt, np.float64).T @ np.asarray(Xt, np.float64)
        Wstar = np.linalg.solve(lam * np.eye(d) - A, B.astype(np.float64))
        bound = 1e-5 * np.linalg.norm(B) / (lam - lam1)
        assert np.linalg.norm(cm(W) - Wstar) <= 1.05 * bound
        assert info.m == math.ceil(2.0 / (0.25 * mu / (lam ** 2 + ctxo.table.kappa * lam1_up) * mu))
        assert info.epochs == sto.epochs
        assert rel(cm(W), Wo) < 2e-5
        assert elem_rms(cm(W), Wo) < 2e-5
    finally:
        m.close()


# ---------------------------------------------------------------------------
# a8: Gram and CholeskyQR2; a4: eigenproblem and Rayleigh-Ritz
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rows,p", [(300, 13), (4096, 40), (1000, 112), (64, 1)])
def test_gram_and_cholqr2(ctx, rows, p):
    rng = np.random.default_rng(rows + p)
    A = rng.standard_normal((rows, p)) @ np.diag(np.logspace(0, -2, p))
    A = A.astype(np.float32)
    G = torch.zeros(p, p, dtype=torch.float64, device=DEV)
    lra.lra_gram(ctx, rows, p, dev_block(A), rows, G)
    A64 = A.astype(np.float64)
    Gref = A64.T @ A64
    assert rel(G.cpu().numpy().T, Gref) < 1e-6
    assert elem_bound(G.cpu().numpy().T, Gref, np.abs(A64).T @ np.abs(A64)) < 1e-6
    W = dev_block(A)
    lra.lra_cholqr2(ctx, rows, p, W)
    Q = cm(W)
    assert np.max(np.abs(Q.T @ Q - np.eye(p))) < 2e-6
    Qref = O.orth(A64)
    assert rel(Q, Qref) < 1e-5
    assert elem_rms(Q, Qref) < 1e-5


def test_cholqr2_reports_rank_deficiency(ctx):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((200, 6)).astype(np.float32)
    A[:, 3] = A[:, 1]
    st = lra.lra_cholqr2(ctx, 200, 6, dev_block(A), allow=(6,))
    assert st == 6  # LRA_ENUMERIC


@pytest.mark.parametrize("p", [1, 2, 7, 40, 101, 112])
def test_sym_eig(ctx, p):
    rng = np.random.default_rng(p)
    V = O.orth(rng.standard_normal((p, p)))
    w = np.sort(rng.gamma(1.0, 1.0, size=p) + np.linspace(0, 0.5, p))[::-1]
    H = (V * w[None, :]) @ V.T
    Hd = torch.from_numpy(np.ascontiguousarray(H.T)).to(DEV)
    ev = torch.zeros(p, dtype=torch.float64, device=DEV)
    evec = torch.zeros(p, p, dtype=torch.float64, device=DEV)
    lra.lra_sym_eig(ctx, p, Hd, ev, evec)
    wr, Vr = O.sym_eig_desc(H)
    # FP64-refined eigenpairs
    assert np.max(np.abs(ev.cpu().numpy() - wr)) < 1e-12 * max(1.0, wr[0])
    Vg = evec.cpu().numpy().T
    gaps = np.abs(np.diff(wr))
    if p > 1 and gaps.min() > 1e-3:
        assert np.max(np.abs(Vg - Vr)) < 1e-9
    assert np.max(np.abs(Vg.T @ Vg - np.eye(p))) < 1e-12


@pytest.mark.parametrize("storage", [lra.LRA_F32, lra.LRA_BF16, lra.LRA_F16])
def test_rayleigh_ritz(ctx, storage):
    d, n, p = 300, 3000, 13
    Xt, U, s = planted(d, n, 5, 19)
    X_st = stored_values(Xt, storage)
    S = O.orth(np.random.default_rng(1).standard_normal((d, p)))
    m = Mat(ctx, Xt, storage)
    try:
        for use32 in (False, True):
            H = torch.zeros(p, p, dtype=torch.float64, device=DEV)
            ev = torch.zeros(p, dtype=torch.float64, device=DEV)
            evec = torch.zeros(p, p, dtype=torch.float64, device=DEV)
            lra.lra_ritz(m.h, p, dev_block(S), use32, H, ev, evec)
            Xref = Xt if (use32 or storage == lra.LRA_F32) else X_st
            rho, Uh, Q, Href = O.rayleigh_ritz(Xref, S.astype(np.float32).astype(np.float64))
            assert rel(H.cpu().numpy().T, Href) < 1e-5
            aQ = np.abs(np.asarray(Xref, dtype=np.float64)) @ np.abs(S)
            assert elem_bound(H.cpu().numpy().T, Href, aQ.T @ aQ) < 1e-5
            assert np.max(np.abs(ev.cpu().numpy() - rho)) < 1e-5 * rho[0]
    finally:
        m.close()


# ---------------------------------------------------------------------------
# a1 / a2: lambda_1 estimate and shift tuning
# ---------------------------------------------------------------------------

def test_lambda1_estimate(ctx):
    Xt, U, s = planted(256, 2048, 5, 4)
    m = Mat(ctx, Xt)
    try:
        lh = lra.lra_lambda1_estimate(m.h, 31)
        ref = O.lambda1_estimate(O.Context(Xt, 31, O.Options()))
        assert abs(lh / ref - 1) < 1e-5
        assert 0.75 * s[0] ** 2 <= lh <= s[0] ** 2 / 0.75
    finally:
        m.close()


def test_shift_tuning_matches_oracle(ctx):
    sig = L.sigma_small_gap(48)
    Xt, U, s = L.planted_numpy(48, 384, sig, 7)
    Xt = np.ascontiguousarray(Xt.astype(np.float32))
    k, p = 5, 10
    delta = (s[k - 1] ** 2 - s[p] ** 2) / 1.5
    octx = O.Context(Xt, 11, O.Options())
    lh = O.lambda1_estimate(octx)
    ref = O.shift_tune(octx, lh, delta)
    m = Mat(ctx, Xt)
    try:
        res = lra.lra_shift_tune(m.h, 11, lh, delta, lra.options())
        assert res["status"] == 0
        assert res["rounds"] == ref.rounds
        for (lg, ig), (lo, io) in zip(res["history"], ref.history):
            assert abs(lg / lo - 1) < 1e-6
            assert abs(ig / io - 1) < 1e-3
        assert abs(res["lam"] / ref.lam - 1) < 1e-6
        lam1 = s[0] ** 2
        assert delta / 30 <= res["lam"] - lam1 <= 2 * delta / 9
        assert res["solve_count"] == octx.solve_count
    finally:
        m.close()


def test_delta_estimate_matches_oracle(ctx):
    """Sec. 3's gap budget (no procedure printed; Algorithm 3 on A with p + 1
    vectors, eps' = 1/(9 p^2)): the GPU estimate equals the oracle's and lies in
    Theorem 4's interval around (lambda_k - lambda_{p+1}) / 1.5."""
    for d, n, k, p, seed, sig in [(48, 384, 5, 10, 11, L.sigma_small_gap(48)),
                                  (256, 2048, 5, 10, 0, L.sigma_small_gap(256)),
                                  (300, 3001, 20, 40, 3, L.sigma_steep_head(300))]:
        Xt, U, s = L.planted_numpy(d, n, sig, seed + 100)
        Xt = np.ascontiguousarray(Xt.astype(np.float32))
        m = Mat(ctx, Xt)
        try:
            dg = lra.lra_delta_estimate(m.h, k, p, seed)
        finally:
            m.close()
        do = O.delta_estimate(O.Context(Xt, seed, O.Options()), k, p)
        # each Ritz value within 1e-5 of rho_1 (the FP32 tolerance of the Ritz
        # step), so their difference over 1.5 within 2e-5 rho_1 / 1.5
        assert abs(dg - do) <= 2e-5 * s[0] ** 2 / 1.5, (d, dg, do)
        lam = s ** 2
        eps = 1.0 / (9.0 * p * p)
        assert ((1 - eps) * lam[k - 1] - lam[p]) / 1.5 * (1 - 1e-5) <= dg <= (lam[k - 1] - (1 - eps) * lam[p]) / 1.5 * (1 + 1e-5)


def test_solve_paper_shift_with_estimated_delta(ctx):
    """lra_solve under the PAPER policy with delta = 0 estimates the gap budget
    itself: the same Delta, shift and number of Algorithm 7 rounds as the
    oracle's run, and the returned U meets ratio <= 1 + eps."""
    sig = L.sigma_small_gap(48)
    Xt64, U, s = L.planted_numpy(48, 384, sig, 7)
    Xt = np.ascontiguousarray(Xt64.astype(np.float32))
    k, p = 5, 10
    st, Ug, rg, rep = run_solve(ctx, Xt, k, p, 11, src=Xt64, shift_policy=lra.LRA_SHIFT_PAPER, delta=0.0)
    assert st == 0
    ref = O.solve(Xt, k, p, 1e-3, 11, O.Options(shift_policy=O.SHIFT_PAPER, delta=0.0))
    assert abs(rep.delta / ref.delta - 1) < 1e-5
    assert rep.shift_rounds == ref.shift.rounds
    assert abs(rep.lambda_ / ref.lam - 1) < 1e-5
    ratio = O.frobenius_error(Xt64, Ug) / L.closed_form_opt(s, k)
    assert 1.0 - 1e-6 <= ratio <= 1.0 + 1e-3


# ---------------------------------------------------------------------------
# The whole path (Algorithm 6, q = k branch)
# ---------------------------------------------------------------------------

def run_solve(ctx, Xt, k, p, seed, storage=lra.LRA_F32, src=None, **kw):
    m = Mat(ctx, Xt, storage, src)
    try:
        d = Xt.shape[1]
        U = torch.zeros(k, d, dtype=torch.float32, device=DEV)
        ritz = torch.zeros(k, dtype=torch.float64, device=DEV)
        rep = lra.LraReport()
        st = lra.lra_solve(m.h, k, p, kw.pop("eps", 1e-3), seed, lra.options(**kw), U, ritz, rep)
        return st, cm(U), ritz.cpu().numpy(), rep
    finally:
        m.close()


def test_solve_fixed_schedule_matches_oracle_small_gap(ctx):
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt64, Uplant, s = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    Xt = np.ascontiguousarray(Xt64.astype(np.float32))
    sched = dict(min_outer=12, max_outer=12, fixed_epochs=5)
    st, Ug, rg, rep = run_solve(ctx, Xt, wl.k, wl.p, 0, src=Xt64, shift_policy=lra.LRA_SHIFT_FAR, **sched)
    ref = O.solve(Xt, wl.k, wl.p, 1e-3, 0, O.Options(shift_policy=O.SHIFT_FAR, **sched))
    assert O.sin_angle(ref.U, Ug) < 1e-4
    assert np.max(np.abs(rg - ref.ritz) / ref.ritz) < 1e-5
    assert rep.outer_iters == ref.outer_iters
    assert rep.kernel_launches > 0


def test_solve_default_stop_rule_meets_eps(ctx):
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt64, Uplant, s = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    for pol in (lra.LRA_SHIFT_FAR, lra.LRA_SHIFT_PAPER):
        delta = (s[wl.k - 1] ** 2 - s[wl.p] ** 2) / 1.5
        st, Ug, rg, rep = run_solve(ctx, Xt64, wl.k, wl.p, 0, src=Xt64, shift_policy=pol, delta=delta)
        assert st == 0
        ratio = O.frobenius_error(Xt64, Ug) / wl.opt()
        assert 1.0 - 1e-6 <= ratio <= 1.0 + 1e-3, (pol, ratio)
        assert np.max(np.abs(Ug.T @ Ug - np.eye(wl.k))) < 1e-5
        if pol == lra.LRA_SHIFT_PAPER:
            oo = O.solve(Xt64, wl.k, wl.p, 1e-3, 0, O.Options(shift_policy=O.SHIFT_PAPER, delta=delta))
            assert rep.shift_rounds == oo.shift.rounds
            assert abs(rep.lambda_ / oo.lam - 1) < 1e-5


def test_solve_bf16_storage_matches_oracle(ctx):
    Xt, U, s = planted(256, 2048, 5, 9)
    Xb = bf16_values(Xt)
    sched = dict(min_outer=10, max_outer=10, fixed_epochs=5)
    st, Ug, rg, rep = run_solve(ctx, Xt, 5, 10, 3, storage=lra.LRA_BF16, shift_policy=lra.LRA_SHIFT_FAR, **sched)
    ref = O.solve(Xb, 5, 10, 1e-3, 3, O.Options(shift_policy=O.SHIFT_FAR, **sched), Xt_final=Xt)
    assert O.sin_angle(ref.U, Ug) < 1e-3
    assert np.max(np.abs(rg - ref.ritz) / ref.ritz) < 1e-4


def test_solve_f16_storage_matches_oracle(ctx):
    """FP16 storage (fp16(s x), s a power of two) on a fixed schedule against the
    oracle run on the FP16-representable values, the final Rayleigh-Ritz step on
    the FP32 values; and the default stop rule meets the ratio."""
    Xt, U, s = planted(256, 2048, 5, 9)
    Xh = f16_values(Xt)
    sched = dict(min_outer=10, max_outer=10, fixed_epochs=5)
    st, Ug, rg, rep = run_solve(ctx, Xt, 5, 10, 3, storage=lra.LRA_F16, shift_policy=lra.LRA_SHIFT_FAR, **sched)
    ref = O.solve(Xh, 5, 10, 1e-3, 3, O.Options(shift_policy=O.SHIFT_FAR, **sched), Xt_final=Xt)
    assert O.sin_angle(ref.U, Ug) < 1e-4
    assert np.max(np.abs(rg - ref.ritz) / ref.ritz) < 1e-5
    st, Ug, rg, rep = run_solve(ctx, Xt, 5, 10, 3, storage=lra.LRA_F16, shift_policy=lra.LRA_SHIFT_FAR)
    assert st == 0
    ratio = O.frobenius_error(Xt, Ug) / L.closed_form_opt(s, 5)
    assert ratio <= 1.0 + 1e-3


def test_f16_storage_inner_loop_and_scale(ctx):
    """The inner loop on an FP16-stored X (stored as fp16(s x)) equals the
    oracle's epoch on the FP16-representable values, for a matrix whose entries
    lie far below FP16's normal range before the scale s."""
    d, n, p = 700, 2000, 6
    Xt, _, _ = planted(d, n, 5, 31)
    Xt = np.ascontiguousarray((Xt * 1e-4).astype(np.float32))   # entries ~1e-7: FP16 subnormal unscaled
    Xh = f16_values(Xt)
    rng = np.random.default_rng(3)
    Wt = rng.standard_normal((d, p)).astype(np.float32)
    M = (0.1 * rng.standard_normal((d, p))).astype(np.float32)
    W0 = (Wt + 0.05 * rng.standard_normal((d, p))).astype(np.float32)
    steps = 500
    idx = rng.integers(0, n, size=steps).astype(np.int32)
    c = (rng.uniform(0.5, 2.0, size=n) * n * 2e7).astype(np.float32)
    eta, lam = 0.02, 1.3
    m = Mat(ctx, Xt, lra.LRA_F16)
    try:
        W = dev_block(W0)
        lra.lra_svrg_inner(m.h, p, W, dev_block(Wt), dev_block(M), torch.from_numpy(idx).to(DEV),
                           steps, torch.from_numpy(c).to(DEV), eta, lam)
        ref = O.svrg_epoch(Xh, W0.astype(np.float64), Wt.astype(np.float64), M.astype(np.float64),
                           idx.astype(np.int64), c.astype(np.float64), eta, lam)
        assert rel(cm(W) - Wt, ref - Wt) < 1e-5
        assert elem_rms(cm(W) - Wt, ref - Wt) < 1e-5
        n2 = torch.zeros(n, dtype=torch.float64, device=DEV)
        lra.lra_colnorms(m.h, n2)
        assert rel(n2.cpu().numpy(), np.sum(Xh * Xh, axis=1)) < 1e-13
    finally:
        m.close()


def test_edge_cases_and_errors(ctx):
    Xt, U, s = planted(64, 300, 3, 2, r=64)
    # p = k + 1, d < 128 (row padding), ragged n
    st, Ug, rg, rep = run_solve(ctx, Xt, 3, 4, 1, shift_policy=lra.LRA_SHIFT_FAR)
    assert st in (0, 4)
    assert np.max(np.abs(Ug.T @ Ug - np.eye(3))) < 1e-5
    m = Mat(ctx, Xt)
    try:
        U = torch.zeros(3, 64, device=DEV)
        r = torch.zeros(3, dtype=torch.float64, device=DEV)
        for (k, p, eps) in [(3, 3, 1e-3), (0, 2, 1e-3), (3, 64, 1e-3), (3, 5, 0.0), (3, 5, 1.0)]:
            code = lra.lib.lra_solve(m.h, k, p, eps, 0, None, U.data_ptr(), r.data_ptr(), None)
            assert code == 1, (k, p, eps)
        # a FIXED shift below lambda_1 / (1 - 1/4) is rejected
        import ctypes
        o = lra.options(shift_policy=lra.LRA_SHIFT_FIXED, lambda_=0.1)
        code = lra.lib.lra_solve(m.h, 3, 5, 1e-3, 0, ctypes.byref(o), U.data_ptr(), r.data_ptr(), None)
        assert code == 1
    finally:
        m.close()


def test_full_size_steep_head_anchor_sampled_rows(ctx):
    """d = 4096, n = 262144 (the benchmark workload): sampled rows of the anchor
    gradient against FP64 products computed row by row."""
    wl = L.WORKLOADS["steep_head_4096x262144"]
    Xt, U = L.planted_torch(wl.d, wl.n, wl.sigma(), wl.seed, device=DEV)
    p = wl.p
    rng = np.random.default_rng(0)
    Wt = rng.standard_normal((wl.d, p)).astype(np.float32)
    B = rng.standard_normal((wl.d, p)).astype(np.float32)
    lam = 2.5
    ctx_mat = lra.lra_create_dense(ctx, wl.d, wl.n, lra.LRA_F32, Xt, wl.d, True, lra.LRA_F32)
    try:
        M = torch.zeros(p, wl.d, dtype=torch.float32, device=DEV)
        lra.lra_anchor(ctx_mat, p, dev_block(Wt), dev_block(B), lam, M)
        Xh = Xt.cpu().numpy()
        Y = Xh.astype(np.float64) @ Wt.astype(np.float64)   # n x p, FP64
        rows = rng.choice(wl.d, size=24, replace=False)
        Mg = cm(M)
        for r in rows:
            ref = lam * Wt[r].astype(np.float64) - Xh[:, r].astype(np.float64) @ Y - B[r]
            assert rel(Mg[r], ref) < 1e-4
        Mref_rows = np.stack([lam * Wt[r] - Xh[:, r].astype(np.float64) @ Y - B[r] for r in rows])
        assert rel(Mg[rows], Mref_rows) < 2e-5
    finally:
        lra.lra_mat_destroy(ctx_mat)
        del Xt
        torch.cuda.empty_cache()
