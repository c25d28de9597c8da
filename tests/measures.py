"""Error measures shared by the GPU parity tests.

Every comparison of a CUDA result with the oracle reports two numbers:

* ``rel``: the relative Frobenius error over the whole block;
* an element-by-element maximum, so that a wrong tile, a wrong padded region or
  a transposed operand cannot hide under a block norm.

Element by element, a floating-point product is held to the classical
componentwise bound of a sum of K terms, |fl(sum_k a_k b_k) - sum_k a_k b_k| <=
gamma_K sum_k |a_k| |b_k|: ``elem_bound`` divides each element's error by its own
value plus that scale (|A| |B| for the product A B), so an element that is the
small difference of large terms is judged against the terms it was summed
from.  Results of recurrences and solves (an inner loop, a linear solve) have no
such per-element scale; ``elem_rms`` divides by the element's value plus the
block's root-mean-square value.
"""
import numpy as np


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def elem_bound(a, b, scale) -> float:
    """max |a - b| / (|b| + scale), elementwise; scale >= 0 of b's shape."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.abs(b) + np.asarray(scale, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(s, 1e-300)))


def elem_rms(a, b) -> float:
    """max |a - b| / (|b| + rms(b)) over the N elements, divided by
    sqrt(2 ln N): independent rounding errors of relative size t (Frobenius)
    reach about t sqrt(2 ln N) at their largest element, so this measure is
    about t for them, while a localized error (a wrong tile or row) keeps its
    full size."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if not b.size:
        return 0.0
    rms = float(np.sqrt(np.mean(b * b)))
    worst = float(np.max(np.abs(a - b) / np.maximum(np.abs(b) + rms, 1e-300)))
    return worst / np.sqrt(2.0 * np.log(max(b.size, 3)))
