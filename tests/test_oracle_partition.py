"""Pins of the oracle's Algorithm 6 loop (adaptive partitioning and deflation,
Sec. 3: Algorithms 3, 4, 5, 6, 7), on planted spectra whose eigenvalues and
eigenvectors are known in closed form.

  * Algorithms 4 and 5 against their definitions on hand-made sequences;
  * deflation: P x_i is orthogonal to U, and with the planted top eigenvectors
    the deflated spectrum is the planted one without them;
  * Algorithm 3's values inside Theorem 4's sandwich (1-eps) lambda_i <=
    lambda_hat_i <= lambda_i / (1-eps), for A and for D at a shift;
  * Lemma deltaSound (a returned q < k has lambda_q - lambda_{q+1} >= Delta/9) and
    the multiplicative-gap lemma on the planted partition workload;
  * the full loop meets the ratio 1 + eps, spans the planted subspace, takes the
    designed partition, and fails when a planted mistake drops the deflation.
"""
import math

import numpy as np
import pytest

import lra_inputs as L
from oracle import lra_oracle as O
from oracle import lra_partition as P


def test_alg4_definition():
    p = 4                                    # threshold 1 - 1/16
    assert P.alg4(np.array([10.0, 9.5, 9.0]), p) == -1
    assert P.alg4(np.array([10.0, 9.3, 9.0]), p) == 0          # 9.3 <= 9.375
    assert P.alg4(np.array([10.0, 9.9, 9.0]), p) == 1          # first such q
    assert P.alg4(np.array([10.0, 9.0, 8.0]), p) == 0          # smallest, not any
    assert P.alg4(np.array([10.0]), p) == -1                   # I \ {k} empty


def test_alg5_definition():
    delta = 0.9                              # 5 Delta / 9 = 0.5
    assert P.alg5(np.array([0.1, 0.3, 0.7]), delta) == 2        # no gap: q = k
    assert P.alg5(np.array([0.1, 0.6, 0.7]), delta) == 0        # 0.5 >= 0.5
    assert P.alg5(np.array([0.1, 0.3, 0.9, 1.6]), delta) == 1   # the first one
    assert P.alg5(np.array([0.2]), delta) == 0                  # single index: k


def test_deflation_removes_the_planted_directions():
    d, n = 40, 300
    Xt, U, s = L.planted_numpy(d, n, L.sigma_partition(d), 2)
    Xd = P.deflate(Xt, U[:, :2])
    assert np.abs(Xd @ U[:, :2]).max() < 1e-12
    lam = np.sort(np.linalg.eigvalsh(Xd.T @ Xd))[::-1]
    expect = np.sort(np.concatenate([s[2:] ** 2, [0.0, 0.0]]))[::-1]
    assert np.allclose(lam, expect[:d], atol=1e-10)
    # no columns: X itself
    assert np.array_equal(P.deflate(Xt, np.zeros((d, 0))), Xt)


def test_alg3_sandwich_on_a_and_d():
    d, n = 48, 400
    Xt, U, s = L.planted_numpy(d, n, L.sigma_partition(d), 3)
    lam = s ** 2
    A = Xt.T @ Xt
    S0 = O.gaussian_block(11, P.STREAM_BLOCK, 0, d, 3)
    eps = 1.0 / 144.0
    th, it = P.alg3_values(lambda S: A @ S, S0, eps, 5000)
    assert it == math.ceil(144.0 * math.log(d * 144.0))
    assert np.all((1 - eps) * lam[:3] <= th) and np.all(th <= lam[:3] / (1 - eps))
    # D at a shift just above lambda_2 of the matrix deflated of u_1
    Xd = P.deflate(Xt, U[:, :1])
    Ad = Xd.T @ Xd
    shift = lam[1] + 0.08
    Dm = np.linalg.inv(shift * np.eye(d) - Ad)
    eps_d = 1.0 / 36.0
    th, _ = P.alg3_values(lambda S: Dm @ S, O.gaussian_block(12, P.STREAM_BLOCK, 2, d, 2), eps_d, 5000)
    true = 1.0 / (shift - lam[1:3])
    assert np.all((1 - eps_d) * true <= th) and np.all(th <= true / (1 - eps_d))


@pytest.fixture(scope="module")
def partition_run():
    wl = L.WORKLOADS["partition_64x800"]
    Xt, U, s = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    res = P.adaptive_solve(Xt, wl.k, wl.p, 1e-3, 0, O.Options(acc=1), delta=0.5)
    return wl, Xt, U, s, res


def test_partition_takes_the_designed_stages(partition_run):
    wl, Xt, U, s, res = partition_run
    lam = s ** 2
    kinds = [(st.s, st.q, st.kind) for st in res.stages]
    # lambda_1 / lambda_2 = 4: a multiplicative gap; then the additive gap
    # lambda_2 - lambda_3 = 0.4 >= 5 Delta / 9; then q = k with oversampling
    assert kinds == [(1, 1, "power"), (2, 2, "shift"), (3, 3, "shift")]
    assert [st.cols for st in res.stages] == [1, 1, 2]
    # Lemma deltaSound: the additive gap returned is >= Delta / 9
    st = res.stages[1]
    assert lam[st.q - 1] - lam[st.q] >= res.delta / 9.0
    # Eq. shiftClose on return of Algorithm 7: Delta/30 <= lambda - lambda_s <= 2 Delta/9
    for st in res.stages[1:]:
        gap = st.lam - lam[st.s - 1]
        assert res.delta / 30.0 <= gap <= 2.0 * res.delta / 9.0
        # Algorithm 3 on D: estimates of lambda - lambda_i within (1 -+ 1/(9p))
        e = 1.0 / (9.0 * wl.p)
        true = st.lam - lam[st.s - 1: wl.k]
        assert np.all((1 - e) * true <= st.inv_est * (1 + 1e-12))
        assert np.all(st.inv_est <= true / (1 - e))
    # Algorithm 3 on A at every stage inside Theorem 4's sandwich
    e = 1.0 / (9.0 * wl.p ** 2)
    for st in res.stages:
        true = lam[st.s - 1: wl.k]
        assert np.all((1 - e) * true <= st.lam_hat) and np.all(st.lam_hat <= true / (1 - e))


def test_partition_meets_eps_and_spans_the_planted_subspace(partition_run):
    wl, Xt, U, s, res = partition_run
    assert res.status == "ok"
    ratio = O.frobenius_error(Xt, res.U) / wl.opt()
    assert 1.0 - 1e-9 <= ratio <= 1.0 + 1e-3
    assert O.sin_angle(res.U, U[:, :wl.k]) < 1e-2
    assert np.allclose(res.ritz, (s ** 2)[:wl.k], rtol=1e-4)


def test_dropped_deflation_is_caught(monkeypatch):
    """A planted mistake: stages see X instead of X_{-(s-1)}."""
    wl = L.WORKLOADS["partition_64x800"]
    Xt, U, s = L.planted_numpy(wl.d, wl.n, wl.sigma(), wl.seed)
    monkeypatch.setattr(P, "deflate", lambda X, Ut: O.as64(X).copy())
    res = P.adaptive_solve(Xt, wl.k, wl.p, 1e-3, 0, O.Options(acc=1), delta=0.5, part_max_iters=300)
    kinds = [(st.s, st.q, st.kind) for st in res.stages]
    ok = kinds == [(1, 1, "power"), (2, 2, "shift"), (3, 3, "shift")]
    ratio = O.frobenius_error(Xt, res.U) / wl.opt()
    assert not (ok and ratio <= 1.0 + 1e-3)
