"""Pins of the oracle's accelerated SVRG solve (AccSVRGsolve, Sec. 1 and
Cor. mainCond; the acceleration itself is not printed in the paper, so the
reading is an accelerated proximal-point loop around SVRG).

What fixes it independently of its own code:
  * the proximal weight gamma solves the epoch-length equation it states
    (checked by evaluating the uncapped epoch length at gamma);
  * the outer residual read off the subproblem's first anchor equals
    (lambda I - A) W - B formed from the dense matrix;
  * with exact subproblem solves the loop is Nesterov's method on a quadratic,
    whose error contracts as (s + 1)(1 - sqrt q)^s (a double root of the
    two-step recurrence at the slowest eigen-direction), while plain proximal
    point (beta = 0) only contracts as (1 - q)^s;
  * the solve reaches the stated residual on the dense system and, at gamma = 0,
    is the plain SVRG solve bit for bit.
"""
import math

import numpy as np
import pytest

import lra_inputs as L
from oracle import lra_oracle as O


def _problem(seed=3, d=24, n=400, p=2):
    rng = np.random.default_rng(seed)
    # a steep head so that lambda_1 dominates ||X||_F^2 only moderately
    sig = np.concatenate([[3.0, 1.5], np.linspace(1.0, 0.2, d - 2)])
    Xt, _, s = L.planted_numpy(d, n, sig, seed)
    A = Xt.T @ Xt
    lam1 = float(np.linalg.eigvalsh(A)[-1])
    B = rng.standard_normal((d, p))
    return rng, Xt, A, lam1, B


def _epoch_samples(ctx, lam, mu, lam1_up):
    """Uncapped samples per epoch, b * theta_m / (eta mu), at (lam, mu)."""
    o = ctx.opts
    b = max(1, int(o.batch))
    eta = o.theta_eta * mu / (lam * lam + ctx.table.kappa * lam1_up / b)
    return b * o.theta_m / (eta * mu)


@pytest.mark.parametrize("batch,target", [(1, 0), (4, 0), (1, 150)])
def test_gamma_balances_the_epoch(batch, target):
    rng, Xt, A, lam1, B = _problem()
    ctx = O.Context(Xt, 0, O.Options(batch=batch, acc_target=target))
    T = target if target > 0 else Xt.shape[0]
    for frac in (0.002, 0.01, 0.05):
        lam = lam1 * (1.0 + frac)
        mu = lam - lam1
        g = ctx.acc_gamma(lam, mu, lam1)
        assert g > 0.0
        # at the target (from below, by the 1e-9 relative nudge of gamma)
        e = _epoch_samples(ctx, lam + g, mu + g, lam1)
        assert e == pytest.approx(T, rel=1e-8) and e < T
        step = ctx.step_params(lam + g, mu + g, lam1)[1]
        assert step == math.ceil(T / batch)
        # the smallest such gamma: a little less is over the target
        assert _epoch_samples(ctx, lam + 0.99 * g, mu + 0.99 * g, lam1) > T
    # an epoch already within the target: no proximal term
    lam = 3.0 * lam1
    assert _epoch_samples(ctx, lam, lam - lam1, lam1) < T
    assert ctx.acc_gamma(lam, lam - lam1, lam1) == 0.0


def test_outer_residual_from_the_first_anchor():
    rng, Xt, A, lam1, B = _problem(seed=5)
    d, p = B.shape
    lam = 1.05 * lam1
    gamma = 0.7 * lam1
    Z = rng.standard_normal((d, p))
    W0 = rng.standard_normal((d, p))
    ctx = O.Context(Xt, 0, O.Options(fixed_epochs=1))
    acc = O.AccStep(gamma=gamma, Z=Z, nB=float(np.linalg.norm(B)), sq=0.5)
    _, st = ctx.svrg_solve(B + gamma * Z, W0, lam + gamma, 0.05 * lam1, lam1, acc=acc)
    direct = np.linalg.norm((lam * np.eye(d) - A) @ W0 - B)
    assert st.outer_res == pytest.approx(direct, rel=1e-12)


def _exact_run(Xt, A, B, lam, mu, gamma_target, S, beta_zero=False):
    """acc_svrg_solve with exact subproblem solves and exactly S iterations
    (fixed_epochs > 0 turns the residual and stall stops off)."""
    d = A.shape[0]
    ctx = O.Context(Xt, 0, O.Options(tau=0.0, acc_max_outer=S, acc_target=gamma_target, fixed_epochs=1))

    def exact(R, W, lam_p, mu_p):
        return np.linalg.solve(lam_p * np.eye(d) - A, R)

    if beta_zero:
        # plain proximal point: the same loop with Z = W (no momentum)
        g = ctx.acc_gamma(lam, mu, lam / 1.0)
        W = np.zeros_like(B)
        for _ in range(S):
            W = exact(B + g * W, W, lam + g, mu + g)
        return W, g
    W, st = ctx.acc_svrg_solve(B, np.zeros_like(B), lam, mu, lam / 1.0, inner=exact)
    assert st.outer == S
    return W, ctx.acc_gamma(lam, mu, lam / 1.0)


def test_exact_inner_contracts_at_the_accelerated_rate():
    rng, Xt, A, lam1, B = _problem(seed=9)
    d = A.shape[0]
    lam = 1.01 * lam1
    mu = lam - lam1                      # exact strong-convexity modulus
    Wstar = np.linalg.solve(lam * np.eye(d) - A, B)
    e0 = np.linalg.norm(Wstar)
    _, g = _exact_run(Xt, A, B, lam, mu, 40, 1)
    q = mu / (mu + g)
    assert 1e-3 < q < 0.2
    errs = {}
    for S in (25, 60, 120):
        W, _ = _exact_run(Xt, A, B, lam, mu, 40, S)
        err = np.linalg.norm(W - Wstar) / e0
        errs[S] = err
        bound = 2.0 * (S + 1) * (1.0 - math.sqrt(q)) ** S
        assert err <= bound, (S, err, bound)
        Wp, _ = _exact_run(Xt, A, B, lam, mu, 40, S, beta_zero=True)
        errp = np.linalg.norm(Wp - Wstar) / e0
        # plain proximal point sits near (1 - q)^S at the slowest direction
        assert errp > 0.1 * (1.0 - q) ** S
        assert err < 0.5 * errp
    # the observed rate between 60 and 120 iterations: (1 - sqrt q) times the
    # polynomial factor of the double root, (121/61)^(1/60) < 1.012
    rate = (errs[120] / errs[60]) ** (1.0 / 60.0)
    assert rate <= 1.03 * (1.0 - math.sqrt(q))
    assert rate < 1.0 - 4.0 * q


def test_wrong_momentum_is_caught(monkeypatch):
    """A planted sign error in beta breaks the rate bound above."""
    rng, Xt, A, lam1, B = _problem(seed=9)
    d = A.shape[0]
    lam = 1.01 * lam1
    mu = lam - lam1
    Wstar = np.linalg.solve(lam * np.eye(d) - A, B)
    real_sqrt = math.sqrt

    class FlippedMath:
        def __getattr__(self, name):
            return getattr(math, name)

        @staticmethod
        def sqrt(x):
            return -real_sqrt(x) if x < 1.0 else real_sqrt(x)   # beta -> (1 + sqrt q)/(1 - sqrt q)

    monkeypatch.setattr(O, "math", FlippedMath())
    _, g = _exact_run(Xt, A, B, lam, mu, 40, 1)
    q = mu / (mu + g)
    # 25 iterations exactly, as in the rate test above
    W, _ = _exact_run(Xt, A, B, lam, mu, 40, 25)
    err = np.linalg.norm(W - Wstar) / np.linalg.norm(Wstar)
    assert not err <= 2.0 * 26 * (1.0 - real_sqrt(q)) ** 25


def test_accelerated_solve_reaches_the_residual():
    rng, Xt, A, lam1, B = _problem(seed=11, n=600)
    d = A.shape[0]
    lam = 1.01 * lam1
    mu = lam - lam1
    ctx = O.Context(Xt, 0, O.Options(tau=1e-6, acc=1))
    assert ctx.acc_gamma(lam, mu, lam1) > 0.0
    W, st = ctx.acc_svrg_solve(B, np.zeros_like(B), lam, mu, lam1)
    assert st.status == "ok" and st.outer_done
    r = np.linalg.norm((lam * np.eye(d) - A) @ W - B) / np.linalg.norm(B)
    assert r <= 1e-6
    assert st.residual == pytest.approx(r, rel=1e-9)
    # fewer samples than the plain solve, which hits its epoch cap here
    plain = O.Context(Xt, 0, O.Options(tau=1e-6))
    _, sp = plain.svrg_solve(B, np.zeros_like(B), lam, mu, lam1)
    assert st.inner_steps < 0.5 * sp.inner_steps


def test_gamma_zero_is_the_plain_solve():
    rng, Xt, A, lam1, B = _problem(seed=13)
    lam = 2.0 * lam1 / 0.75
    mu = lam - lam1 / 0.75
    a = O.Context(Xt, 7, O.Options(acc=1))
    b = O.Context(Xt, 7, O.Options())
    assert a.acc_gamma(lam, mu, lam1 / 0.75) == 0.0
    Wa, sa = a.solve_linear(B, np.zeros_like(B), lam, mu, lam1 / 0.75)
    Wb, sb = b.solve_linear(B, np.zeros_like(B), lam, mu, lam1 / 0.75)
    assert np.array_equal(Wa, Wb) and sa.inner_steps == sb.inner_steps


def test_accelerated_low_rank_solve_meets_eps():
    """Algorithm 6's q = k branch with every solve accelerated, at a shift
    close enough to lambda_1 that SVRG needs the proximal term."""
    wl = L.WORKLOADS["small_gap_256x2048"]
    Xt, U, s = L.planted_numpy(128, 1024, wl.sigma()[:128], 21)
    k, p, eps = 4, 8, 1e-3
    lam1 = float(s[0] ** 2)
    opt = float(np.sum(s[k:] ** 2))
    o = O.Options(shift_policy=O.SHIFT_FIXED, lam=1.35 * lam1, acc=1, tau=1e-6)
    res = O.solve(Xt, k, p, eps, seed=2, opts=o, lam1_hat=lam1)
    assert res.status == "ok"
    ctx = O.Context(Xt, 0, o)
    assert ctx.acc_gamma(o.lam, o.lam - lam1 / 0.75, lam1 / 0.75) > 0.0
    assert O.frobenius_error(Xt, res.U) <= (1.0 + eps) * opt
