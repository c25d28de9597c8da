"""The look-ahead identity behind the paired one-sample inner kernel (d <= 512).

With Delta_{t+1} = a Delta_t + c_t x_t - eta M (a = 1 - eta lambda and
c_t = eta c_{i_t} x_{i_t}^T Delta_t, the step of Sec. 2.3 as the oracle's
svrg_epoch takes it), the next step's product is

    r_{t+1} = a x_{t+1}^T Delta_t + c_t x_{t+1}^T x_t - x_{t+1}^T (eta M).

The kernel takes two steps per iteration on that identity.  Here the same
schedule, written out in FP64, must reproduce the oracle's epoch on the same
sample sequence (even and odd m, m = 0 and 1), so the GPU parity tolerance
only has to absorb FP32 rounding.
"""
import math

import numpy as np
import pytest

from oracle import lra_oracle as O


def paired_epoch(Xt, W, Wt, M, idx, c, eta, lam):
    """The paired kernel's schedule in FP64 (columns of W at once)."""
    X = np.asarray(Xt, dtype=np.float64).T        # d x n
    m = len(idx)
    a = 1.0 - eta * lam
    mm = eta * M
    dl = W - Wt

    def col(t):
        return X[:, idx[t]] if t < m else np.zeros(X.shape[0])

    x0 = col(0)
    r = x0 @ dl
    t = 0
    while t < m:
        x1, x2 = col(t + 1), col(t + 2)
        ct = eta * c[idx[t]] * r
        uA, wA, vA = x1 @ dl, x1 @ mm, x1 @ x0          # for r_{t+1}, on Delta_t
        dl = a * dl + np.outer(x0, ct) - mm             # step t
        uB, wB, vB = x2 @ dl, x2 @ mm, x2 @ x1          # for r_{t+2}, on Delta_{t+1}
        if t + 1 < m:
            c1 = eta * c[idx[t + 1]] * (a * uA + ct * vA - wA)
            dl = a * dl + np.outer(x1, c1) - mm         # step t + 1
            r = a * uB + c1 * vB - wB
        x0 = x2
        t += 2
    return Wt + dl


@pytest.mark.parametrize("m", [0, 1, 2, 7, 64, 301])
def test_paired_schedule_equals_the_sequential_epoch(m):
    rng = np.random.default_rng(m + 3)
    d, n, p = 48, 120, 3
    Xt = rng.standard_normal((n, d)) / math.sqrt(d)
    tab = O.sampling_table(O.colnorms(Xt)[0])
    idx = O.sample_indices(tab, O.stream_key(2, O.STREAM_SVRG, 0, m), m)
    lam = 1.7
    eta = 0.02
    Wt = rng.standard_normal((d, p))
    W = Wt + 0.4 * rng.standard_normal((d, p))
    M = rng.standard_normal((d, p))
    ref = O.svrg_epoch(Xt, W, Wt, M, idx, tab.c, eta, lam)
    got = paired_epoch(Xt, W, Wt, M, idx, tab.c, eta, lam)
    scale = max(1.0, float(np.abs(ref).max()))
    assert np.abs(got - ref).max() <= 1e-11 * scale
