"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties one oracle function to something the paper or the mathematics
fixes: a published test vector, a closed form, an exact identity checked with an
independent formula (dense X X^T formed explicitly, a dense linear solve, an SVD),
an invariant the paper proves, or brute force on tiny inputs.  The mutation tests
at the end plant plausible mistakes in the oracle and check that a pin fails.
"""
import math
import os

import numpy as np
import pytest

import lra_inputs as L
from oracle import lra_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------------------
# Random numbers
# ----------------------------------------------------------------------------

def test_splitmix64_published_vector():
    rows = _read_golden("splitmix64.txt")
    seed = int(rows[0][1])
    expect = [int(r[0]) for r in rows[1:]]
    assert O.splitmix64_sequence(seed, len(expect)) == expect
    # the counter form u_t = mix(key + gamma (t+1)) is the same sequence
    assert [int(v) for v in O.uniforms_u64(seed, 0, len(expect))] == expect


def test_mulhi64_exact_against_bigint():
    rng = np.random.default_rng(1)
    u = rng.integers(0, 2**64, size=2000, dtype=np.uint64)
    u[:4] = [0, 1, 2**64 - 1, 2**63]
    for T in [1, 2, 3, 2**32 - 1, 2**32, 2**32 + 7, 123456789012345, 2**63 - 25, 2**64 - 1]:
        got = O.mulhi64(u, T)
        ref = [(int(x) * T) >> 64 for x in u]
        assert [int(g) for g in got] == ref


def test_gaussian_block_is_standard_normal():
    from scipy import stats
    z = O.gaussian_block(5, O.STREAM_INIT, 0, 1000, 60).ravel()
    assert abs(np.mean(z)) < 5.0 / math.sqrt(z.size)
    assert abs(np.var(z) - 1.0) < 5.0 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # distinct streams are not the same numbers
    z2 = O.gaussian_block(5, O.STREAM_INIT, 1, 1000, 60).ravel()
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.02


# ----------------------------------------------------------------------------
# Sampling distribution (Theorem 3 depends on sr(X): importance sampling)
# ----------------------------------------------------------------------------

def _random_norms(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.gamma(2.0, 1.0, size=n)
    v[::17] = 0.0          # zero columns are never drawn
    v[5] = 1e-30           # a tiny column keeps weight >= 1
    return v


def test_sampling_index_rule_by_definition():
    norm2 = _random_norms(300, 2)
    tab = O.sampling_table(norm2)
    key = O.stream_key(9, O.STREAM_SVRG, 3, 4)
    idx = O.sample_indices(tab, key, 5000)
    u = O.uniforms_u64(key, 0, 5000)
    for t in range(0, 5000, 37):
        r = (int(u[t]) * tab.total) >> 64
        i = int(idx[t])
        lo = 0 if i == 0 else int(tab.cum[i - 1])
        assert lo <= r < int(tab.cum[i])
        assert tab.weights[i] > 0
    assert np.all(norm2[idx] > 0)


def test_sampling_frequencies_chi_square():
    from scipy import stats
    norm2 = _random_norms(40, 3)
    tab = O.sampling_table(norm2)
    idx = O.sample_indices(tab, O.stream_key(1, O.STREAM_SVRG, 0, 0), 400000)
    counts = np.bincount(idx, minlength=40)
    q = tab.weights.astype(np.float64) / tab.total
    nz = q > 0
    assert counts[~nz].sum() == 0
    chi = stats.chisquare(counts[nz], 400000 * q[nz])
    assert chi.pvalue > 1e-4
    # importance weights follow ||x_i||^2 / ||X||_F^2 up to the quantisation
    # step 1/total (a non-zero column keeps weight >= 1)
    assert np.allclose(q[nz], norm2[nz] / norm2.sum(), rtol=1e-6, atol=2.0 / tab.total)


def test_importance_estimator_is_unbiased():
    """sum_i q_i c_i x_i x_i^T = X X^T exactly (c_i = 1/q_i), checked against
    the dense X X^T."""
    rng = np.random.default_rng(4)
    Xt = rng.standard_normal((70, 9)) * rng.gamma(1.0, 1.0, size=(70, 1))
    Xt[3] = 0.0
    norm2, _ = O.colnorms(Xt)
    for mode in (O.SAMPLE_IMPORTANCE, O.SAMPLE_UNIFORM):
        tab = O.sampling_table(norm2, mode)
        q = tab.weights.astype(np.float64) / tab.total
        est = sum(q[i] * tab.c[i] * np.outer(Xt[i], Xt[i]) for i in range(70))
        assert np.allclose(est, Xt.T @ Xt, rtol=1e-12, atol=1e-12)
    # kappa = max c_i ||x_i||^2 is ||X||_F^2 up to the floor quantisation:
    # fro2 - n/s <= kappa <= fro2 / (1 - 1/w_min), s = 2^32 / max ||x_i||^2
    tab = O.sampling_table(norm2)
    fro2 = norm2.sum()
    s = 4294967296.0 / norm2.max()
    wmin = float(tab.weights[tab.weights > 0].min())
    assert fro2 - 70 / s <= tab.kappa <= fro2 / (1.0 - 1.0 / wmin) * (1 + 1e-12)


def test_colnorms_against_definition():
    rng = np.random.default_rng(5)
    Xt = rng.standard_normal((33, 17)).astype(np.float32)
    norm2, fro2 = O.colnorms(Xt)
    for i in range(33):
        assert norm2[i] == pytest.approx(sum(float(x) ** 2 for x in Xt[i]), rel=1e-14)
    assert fro2 == pytest.approx(float(np.sum(Xt.astype(np.float64) ** 2)), rel=1e-14)


# ----------------------------------------------------------------------------
# Anchor and inner step (SVRGsolve)
# ----------------------------------------------------------------------------

def _problem(seed=6, d=20, n=90, p=3):
    rng = np.random.default_rng(seed)
    Xt = rng.standard_normal((n, d)) / math.sqrt(n)
    A = Xt.T @ Xt                     # dense X X^T, formed explicitly
    lam1 = float(np.linalg.eigvalsh(A)[-1])
    lam = 1.3 * lam1
    B = rng.standard_normal((d, p))
    return rng, Xt, A, lam1, lam, B


def test_anchor_vanishes_at_the_solution():
    rng, Xt, A, lam1, lam, B = _problem()
    Wstar = np.linalg.solve(lam * np.eye(A.shape[0]) - A, B)
    M = O.anchor(Xt, Wstar, B, lam)
    assert np.linalg.norm(M) < 1e-12 * np.linalg.norm(B)
    W = rng.standard_normal(B.shape)
    # and equals the gradient (lambda I - A) W - B elsewhere
    assert np.allclose(O.anchor(Xt, W, B, lam), (lam * np.eye(A.shape[0]) - A) @ W - B, atol=1e-12)


def test_inner_step_is_unbiased_gradient_step():
    """E_i[one step from W] = W - eta grad F(W), grad F(W) = (lambda I - A) W - B,
    checked by enumerating every column i with its probability q_i."""
    rng, Xt, A, lam1, lam, B = _problem()
    n = Xt.shape[0]
    norm2, _ = O.colnorms(Xt)
    tab = O.sampling_table(norm2)
    Wt = rng.standard_normal(B.shape)
    W = Wt + 0.3 * rng.standard_normal(B.shape)
    M = O.anchor(Xt, Wt, B, lam)
    eta = 0.01
    q = tab.weights.astype(np.float64) / tab.total
    mean = np.zeros_like(W)
    for i in range(n):
        Wi = O.svrg_epoch(Xt, W, Wt, M, np.array([i]), tab.c, eta, lam)
        mean += q[i] * Wi
    grad = (lam * np.eye(A.shape[0]) - A) @ W - B
    assert np.allclose(mean, W - eta * grad, rtol=1e-11, atol=1e-11)


def test_inner_loop_empty_and_anchor_fixed_point():
    rng, Xt, A, lam1, lam, B = _problem()
    tab = O.sampling_table(O.colnorms(Xt)[0])
    Wt = rng.standard_normal(B.shape)
    M = O.anchor(Xt, Wt, B, lam)
    W = O.svrg_epoch(Xt, Wt, Wt, M, np.zeros(0, dtype=np.int64), tab.c, 0.1, lam)
    assert np.array_equal(W, Wt)
    # at the exact solution M = 0 and W = Wt: every step leaves W unchanged
    Wstar = np.linalg.solve(lam * np.eye(A.shape[0]) - A, B)
    M0 = O.anchor(Xt, Wstar, B, lam)
    W1 = O.svrg_epoch(Xt, Wstar, Wstar, M0, np.array([0, 5, 7, 7, 3]), tab.c, 0.05, lam)
    assert np.allclose(W1, Wstar, atol=1e-12)


@pytest.mark.parametrize("mode", [O.SAMPLE_IMPORTANCE, O.SAMPLE_UNIFORM])
def test_svrg_solve_matches_dense_solve(mode):
    rng, Xt, A, lam1, lam, B = _problem(p=4)
    ctx = O.Context(Xt, 3, O.Options(tau=1e-10, sampling=mode))
    W, st = ctx.svrg_solve(B, np.zeros_like(B), lam, lam - lam1, lam1)
    Wstar = np.linalg.solve(lam * np.eye(A.shape[0]) - A, B)
    assert st.status == "ok" and st.residual <= 1e-10
    # ||W - W*|| <= ||(lambda I - A)^{-1}|| ||M|| <= tau ||B|| / (lambda - lambda_1)
    assert np.linalg.norm(W - Wstar) <= 1e-10 * np.linalg.norm(B) / (lam - lam1) * 1.01


# ----------------------------------------------------------------------------
# Orthonormalisation, eigen-decomposition, Rayleigh-Ritz
# ----------------------------------------------------------------------------

def test_orth_is_unique_positive_qr():
    rng = np.random.default_rng(8)
    W = rng.standard_normal((50, 7))
    Q = O.orth(W)
    assert np.allclose(Q.T @ Q, np.eye(7), atol=1e-13)
    R = Q.T @ W
    assert np.allclose(np.tril(R, -1), 0.0, atol=1e-12)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(Q @ R, W, atol=1e-12)


def test_sym_eig_desc_planted():
    rng = np.random.default_rng(9)
    V = O.orth(rng.standard_normal((12, 12)))
    w = np.linspace(5.0, -1.0, 12)
    H = (V * w[None, :]) @ V.T
    ev, U = O.sym_eig_desc(H)
    assert np.allclose(ev, w, atol=1e-12)
    for j in range(12):
        a = int(np.argmax(np.abs(U[:, j])))
        assert U[a, j] > 0
        assert abs(abs(U[:, j] @ V[:, j]) - 1.0) < 1e-10


def test_rayleigh_ritz_planted_closed_form():
    w = L.WORKLOADS["small_gap_256x2048"]
    Xt, U, s = L.planted_numpy(w.d, w.n, w.sigma(), w.seed)
    rho, Uh, Q, H = O.rayleigh_ritz(Xt, U[:, : w.p])
    assert np.allclose(rho, s[: w.p] ** 2, rtol=1e-12)
    norm2, fro2 = O.colnorms(Xt)
    E = fro2 - float(np.sum(rho[: w.k]))
    assert E == pytest.approx(w.opt(), rel=1e-12)
    # E_l equals the Frobenius error of the Ritz projector (Alg. 2 output)
    Uk = U[:, : w.p] @ Uh[:, : w.k]
    assert O.frobenius_error(Xt, Uk) == pytest.approx(E, rel=1e-12)


def test_golden_optima_match_planted_spectra():
    rows = {r[0]: (int(r[1]), float(r[2]), float(r[3])) for r in _read_golden("planted_optima.txt")}
    for name, (k, opt, fro2) in rows.items():
        wl = L.WORKLOADS[name]
        s = wl.sigma()
        assert wl.k == k
        assert L.closed_form_opt(s, k) == pytest.approx(opt, abs=2e-10)
        assert float(np.sum(s ** 2)) == pytest.approx(fro2, abs=2e-10)


def test_metrics_against_svd():
    rng = np.random.default_rng(10)
    Xt = rng.standard_normal((40, 15))
    Ufull, sv, _ = np.linalg.svd(Xt.T, full_matrices=False)
    Uk = Ufull[:, :4]
    assert O.frobenius_error(Xt, Uk) == pytest.approx(float(np.sum(sv[4:] ** 2)), rel=1e-12)
    assert O.sin_angle(Uk, Uk) < 1e-14
    # a rotation inside the span leaves the angle 0; one foreign direction gives 1
    Rot = O.orth(rng.standard_normal((4, 4)))
    assert O.sin_angle(Uk, Uk @ Rot) < 1e-13
    V = Uk.copy()
    V[:, 3] = Ufull[:, 6]
    assert O.sin_angle(Uk, V) == pytest.approx(1.0, abs=1e-12)


# ----------------------------------------------------------------------------
# Algorithm 3, Algorithm 7 and the whole path
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_planted():
    s = L.sigma_small_gap(48)
    Xt, U, s = L.planted_numpy(48, 384, s, 7)
    return Xt, U, s


def test_lambda1_estimate_sandwich(small_planted):
    Xt, U, s = small_planted
    ctx = O.Context(Xt, 11, O.Options())
    lh = O.lambda1_estimate(ctx)
    lam1 = s[0] ** 2
    assert 0.75 * lam1 <= lh <= lam1 / 0.75   # Theorem 4 with eps = 1/4
    rng = np.random.default_rng(12)
    Xr = rng.standard_normal((300, 40))
    lam1r = float(np.linalg.svd(Xr, compute_uv=False)[0] ** 2)
    lhr = O.lambda1_estimate(O.Context(Xr, 1, O.Options()))
    assert 0.75 * lam1r <= lhr <= lam1r / 0.75


def test_shift_tuning_invariants(small_planted):
    """Lemma 10: each round keeps lambda - lambda_1 positive and shrinks it into
    [1/2, 3/4] of its value; on return the estimate lies in [Delta/27, Delta/5]
    and lambda - lambda_1 in [Delta/30, 2 Delta/9] (Eq. shiftClose); every
    estimate is within (1-eps')^{+-1} of lambda - lambda_1 (Eq. approxShiftGap)."""
    Xt, U, s = small_planted
    lam1 = s[0] ** 2
    k, p = 5, 10
    delta = (s[k - 1] ** 2 - s[p] ** 2) / 1.5
    ctx = O.Context(Xt, 11, O.Options())
    lh = O.lambda1_estimate(ctx)
    sh = O.shift_tune(ctx, lh, delta)
    assert sh.status == "ok"
    assert sh.rounds <= 2 + math.ceil(math.log(lam1 / delta) / math.log(4.0 / 3.0))
    eps = 1.0 / 9.0
    gaps = [lam - lam1 for lam, _ in sh.history]
    for (lam, inv), g in zip(sh.history, gaps):
        assert g > 0
        assert (1 - eps) * g <= inv <= g / (1 - eps)
    for g0, g1 in zip(gaps, gaps[1:]):
        assert 0.5 * g0 <= g1 <= 0.75 * g0
    assert delta / 27 <= sh.inv_est <= delta / 5
    assert delta / 30 <= sh.lam - lam1 <= 2 * delta / 9
    assert 0 < sh.mu_lb <= sh.lam - lam1



def _slow_tail_planted():
    """lambda = 10, 9, 8 | 5, 4.9, 4.8 | 4.0, then 89 eigenvalues just below
    0.97 * 4.0: with k = 3, p = 6 the (p+1)-th Ritz value converges at the slow
    ratio ~0.97 per power step against a heavy tail, so Theorem 4's accuracy
    eps' = 1/(9 p^2) is reached only after many steps (20 are too few)."""
    lam = np.array([10.0, 9.0, 8.0, 5.0, 4.9, 4.8, 4.0] + [4.0 * 0.97 * (1 - 0.001 * j) for j in range(89)])
    Xt, U, s = L.planted_numpy(96, 600, np.sqrt(lam), 21)
    return Xt, s


def _check_delta_estimate(delta_fn):
    """Sec. 3's gap budget: Delta <= lambda_k - lambda_{p+1} <= 2 Delta.  The
    estimate is (rho_k - rho_{p+1}) / 1.5 with rho from Algorithm 3 at
    eps' = 1/(9 p^2); Theorem 4 gives (1 - eps') lambda_i <= rho_i and
    Rayleigh-Ritz values never exceed the eigenvalues (Cauchy interlacing), so
    the estimate lies in [((1-eps') l_k - l_{p+1}) / 1.5, (l_k - (1-eps') l_{p+1}) / 1.5]."""
    cases = [(L.planted_numpy(48, 384, L.sigma_small_gap(48), 7)[0], L.sigma_small_gap(48), 5, 10, 11)]
    Xs, ss = _slow_tail_planted()
    cases.append((Xs, ss, 3, 6, 4))
    for Xt, s, k, p, seed in cases:
        lam = np.asarray(s, dtype=np.float64) ** 2
        eps = 1.0 / (9.0 * p * p)
        lk, lp1 = lam[k - 1], lam[p]
        dh = delta_fn(O.Context(Xt, seed, O.Options()), k, p)
        lo = ((1.0 - eps) * lk - lp1) / 1.5
        hi = (lk - (1.0 - eps) * lp1) / 1.5
        assert lo * (1 - 1e-12) <= dh <= hi * (1 + 1e-12), (k, p, dh, lo, hi)
        assert dh <= lk - lp1 <= 2.0 * dh


def test_delta_estimate_theorem4_interval():
    _check_delta_estimate(O.delta_estimate)


def test_subspace_iteration_rate_matches_theory(small_planted):
    """Algorithm 1 on D = (lambda I - A)^{-1}: the top-k directions converge at
    the ratio of D's eigenvalues, (lambda - lambda_j)/(lambda - lambda_{p+1}) for
    j <= k (Theorem 'zhang' bounds the slowest, j = k).  The averaged decay of
    sin theta_k(U_k, S_l) must lie between the fastest (j = 1) and slowest (j = k)
    of these; A in place of D (0.43 here) or a wrong-signed shift (0.87) falls
    outside."""
    Xt, U, s = small_planted
    k, p = 5, 10
    lam1 = s[0] ** 2
    lam = 3.0 * lam1
    ctx = O.Context(Xt, 2, O.Options(tau=1e-13))
    S = O.orth(O.gaussian_block(2, O.STREAM_INIT, 0, Xt.shape[1], p))
    Uk = U[:, :k]
    sins = []
    for _ in range(32):
        W, st = ctx.svrg_solve(S, np.zeros_like(S), lam, lam - lam1, lam1)
        S = O.orth(W)
        sins.append(float(np.linalg.norm(Uk - S @ (S.T @ Uk), 2)))
    slow = (lam - s[k - 1] ** 2) / (lam - s[p] ** 2)
    fast = (lam - s[0] ** 2) / (lam - s[p] ** 2)
    obs = (sins[31] / sins[15]) ** (1.0 / 16.0)
    assert fast - 0.01 <= obs <= slow + 0.01


def test_solve_small_gap_far_shift_meets_ratio():
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt, U, s = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    r = O.solve(Xt, wl.k, wl.p, 1e-3, 0, O.Options(shift_policy=O.SHIFT_FAR))
    assert r.status == "ok"
    assert np.allclose(r.U.T @ r.U, np.eye(wl.k), atol=1e-12)
    ratio = O.frobenius_error(Xt, r.U) / wl.opt()
    assert 1.0 - 1e-12 <= ratio <= 1.0 + 1e-3
    # the returned Ritz values are Rayleigh quotients of U's columns
    AU = O.x_apply(Xt, r.U)
    assert np.allclose(np.sum(r.U * AU, axis=0), r.ritz, rtol=1e-12)


def test_solve_tiny_brute_force_svd():
    """On a tiny X with a clear gap the method recovers the SVD's U_k."""
    rng = np.random.default_rng(13)
    d, n, k, p = 16, 64, 3, 6
    s = np.array([3.0, 2.5, 2.0] + [1.0 * 0.8 ** i for i in range(13)])
    Xt, U, s = L.planted_numpy(d, n, s, 14)
    Usvd = np.linalg.svd(Xt.T, full_matrices=False)[0][:, :k]
    r = O.solve(Xt, k, p, 1e-12, 5, O.Options(shift_policy=O.SHIFT_FAR, tau=1e-13, max_outer=300))
    assert O.sin_angle(Usvd, r.U) < 1e-6
    assert np.allclose(r.ritz, s[:k] ** 2, rtol=1e-10)


# ----------------------------------------------------------------------------
# Planted mistakes: a pin must fail for each
# ----------------------------------------------------------------------------

def _pin_raises(fn):
    try:
        fn()
    except AssertionError:
        return True
    return False


def test_planted_mistakes_are_caught(monkeypatch):
    # c_i = q_i instead of 1/q_i
    real_table = O.sampling_table

    def bad_table(norm2, mode=O.SAMPLE_IMPORTANCE):
        t = real_table(norm2, mode)
        q = t.weights.astype(np.float64) / max(t.total, 1)
        return O.SamplingTable(t.weights, t.cum, t.total, q, t.kappa)

    monkeypatch.setattr(O, "sampling_table", bad_table)
    assert _pin_raises(test_importance_estimator_is_unbiased)
    monkeypatch.setattr(O, "sampling_table", real_table)

    # wrong sign of the A W term in the anchor
    real_anchor = O.anchor
    monkeypatch.setattr(O, "anchor", lambda Xt, Wt, B, lam: lam * Wt + O.x_apply(Xt, Wt) - B)
    assert _pin_raises(test_anchor_vanishes_at_the_solution)
    monkeypatch.setattr(O, "anchor", real_anchor)

    # Ritz on X instead of X^T (transposed operand)
    real_rr = O.rayleigh_ritz

    def bad_rr(Xt, S):
        Q = np.asarray(Xt, dtype=np.float64)[: S.shape[0]] @ S
        H = Q.T @ Q
        rho, Uh = O.sym_eig_desc(H)
        return rho, Uh, Q, H

    monkeypatch.setattr(O, "rayleigh_ritz", bad_rr)
    assert _pin_raises(test_rayleigh_ritz_planted_closed_form)
    monkeypatch.setattr(O, "rayleigh_ritz", real_rr)

    # dropped lambda (W - Wt) term of the inner step: the unbiasedness pin fails
    real_epoch = O.svrg_epoch

    def bad_epoch(Xt, W, Wt, M, idx, c, eta, lam):
        return real_epoch(Xt, W, Wt, M, idx, c, eta, 0.0) - eta * 0.0

    monkeypatch.setattr(O, "svrg_epoch", bad_epoch)
    assert _pin_raises(test_inner_step_is_unbiased_gradient_step)
    monkeypatch.setattr(O, "svrg_epoch", real_epoch)


    # gap budget: rho_p in place of rho_{p+1}, a second division by 1.5, and
    # too few power steps (L = 20) each leave Theorem 4's interval
    def delta_variant(rho_index_shift=0, div=1.5, steps=None):
        def fn(ctx, k, p):
            d = ctx.d
            eps = 1.0 / (9.0 * p * p)
            Lsteps = steps or min(200, int(math.ceil((1.0 / eps) * math.log(d / eps))))
            S = O.orth(O.gaussian_block(ctx.seed, O.STREAM_DELTA, 0, d, p + 1))
            for _ in range(Lsteps):
                S = O.orth(O.x_apply(ctx.Xt, S))
            rho = O.rayleigh_ritz(ctx.Xt, S)[0]
            return float(rho[k - 1] - rho[p - rho_index_shift]) / div
        return fn

    _check_delta_estimate(delta_variant())          # the restatement itself passes
    assert _pin_raises(lambda: _check_delta_estimate(delta_variant(rho_index_shift=1)))
    assert _pin_raises(lambda: _check_delta_estimate(delta_variant(div=1.5 * 1.5)))
    assert _pin_raises(lambda: _check_delta_estimate(delta_variant(steps=20)))
