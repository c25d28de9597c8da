"""FP64 CPU oracle for shift-and-invert block power iteration with SVRG solves.

TEST INFRASTRUCTURE ONLY.  This module may be imported by tests/, by
__graft_entry__.smoke() and by the CPU-baseline leg of bench.py, and by nothing
else.  The library (paper_1607_02925_gb300) never imports, links or calls it, and
it shares no code with the library: the two meet only through the seeded inputs
of the separate `lra_inputs` module.

It follows Gonen & Shalev-Shwartz, "Faster Low-rank Approximation using Adaptive
Gap-based Preconditioning", on the branch of Algorithm 6 where no gap is found
(q = k, s = 1, no deflation):

  1. estimate lambda_1 (Algorithm 3 with C = A = X X^T, k = 1, eps = 1/4),
  2. tune the shift lambda (Algorithm 7, Appendix B), or take a fixed policy,
  3. subspace iteration (Algorithm 1) on D = (lambda I - A)^{-1} with p columns,
     every product D S solved by SVRG (Sec. 2.3, Theorem 3),
  4. Rayleigh-Ritz with C = A (Algorithm 2), returning U = S U_hat_k.

Everything is plain FP64 numpy (library primitives: matmul, QR, eigh,
searchsorted) except the SVRG inner loop, which is the plain C in svrg_inner.c.
X is read exactly as stored (FP64 or FP32 values widened).

Readings where the paper is silent or garbled:
  * SVRGsolve's update is not printed; the step used is the variance-reduced
    gradient of the quadratic F(W) = 1/2 tr W^T(lambda I - A)W - tr B^T W with
    importance sampling q_i ~ ||x_i||^2 and c_i = 1/q_i (svrg_epoch).
  * Step size eta = theta_eta mu/(lambda^2 + kappa lambda1_up) and epoch length
    m = ceil(theta_m/(eta mu)), mu a lower bound on lambda - lambda_1 and
    kappa = max_i c_i ||x_i||^2 (= ||X||_F^2 for exact importance sampling).
  * Alg. 7 prints the target interval as [Delta/27, Delta/25]; Eq. (shiftClose),
    the text and the proof use [Delta/27, Delta/5], which is taken here.  The
    loop returns the shift whose estimate fell in the interval (no update after
    the last estimate), as the lemma's conclusion states.
  * The number of subspace iterations is not fixed by the paper (only
    O(k log(kd/eps))); the loop stops on the predicted remaining decrease of the
    Ritz error E_l = ||X||_F^2 - sum_{j<=k} rho_j.
  * The only randomness in the paper is the Gaussian start of Algorithm 1
    (Sec. 2.4); the SVRG sample streams are a second, separately keyed stream.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64, Steele/Lea/Flood 2014)
# ----------------------------------------------------------------------------
MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15

STREAM_INIT = 1       # Gaussian start S0 of the main subspace iteration
STREAM_POWER_A = 2    # start vector of the lambda_1 estimate (Alg. 3 on A)
STREAM_POWER_D = 3    # start vector of each shift-tuning round (Alg. 3 on D)
STREAM_SVRG = 4       # SVRG sample sequence of (solve, epoch)
STREAM_DELTA = 5      # start block of the gap-budget estimate

SHIFT_PAPER, SHIFT_FAR, SHIFT_FIXED = 0, 1, 2
SAMPLE_IMPORTANCE, SAMPLE_UNIFORM = 0, 1


def mix64(z: int) -> int:
    """SplitMix64 output function applied to a 64-bit state (Python ints)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_sequence(seed: int, count: int) -> list[int]:
    """The first `count` outputs of the SplitMix64 generator seeded with `seed`:
    state += gamma; output mix64(state)."""
    out, s = [], seed & MASK64
    for _ in range(count):
        s = (s + GAMMA) & MASK64
        out.append(mix64(s))
    return out


def stream_key(seed: int, stream: int, a: int = 0, b: int = 0) -> int:
    """Key of the counter stream (seed, stream, a, b): three chained SplitMix64
    steps, each absorbing one word."""
    h = mix64((seed + GAMMA * (stream + 1)) & MASK64)
    h = mix64((h + GAMMA * (a + 1)) & MASK64)
    h = mix64((h + GAMMA * (b + 1)) & MASK64)
    return h


def _mix64_vec(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def uniforms_u64(key: int, t0: int, count: int) -> np.ndarray:
    """u_t = mix64(key + gamma (t + 1)) for t = t0 .. t0+count-1 (uint64)."""
    t = np.arange(t0 + 1, t0 + count + 1, dtype=np.uint64)
    z = np.uint64(key) + t * np.uint64(GAMMA)
    return _mix64_vec(z)


def mulhi64(u: np.ndarray, T: int) -> np.ndarray:
    """floor(u * T / 2^64) for uint64 arrays u and a scalar T < 2^64, built from
    32-bit halves (exact)."""
    u = np.asarray(u, dtype=np.uint64)
    lo32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    ul, uh = u & lo32, u >> s32
    Tl, Th = np.uint64(T & 0xFFFFFFFF), np.uint64(T >> 32)
    ll, lh, hl, hh = ul * Tl, ul * Th, uh * Tl, uh * Th
    mid = (ll >> s32) + (lh & lo32) + (hl & lo32)
    return hh + (lh >> s32) + (hl >> s32) + (mid >> s32)


def gaussian_block(seed: int, stream: int, a: int, d: int, p: int) -> np.ndarray:
    """d x p N(0,1) block (FP64) for Algorithm 1's S0 ~ N(0,1)^{d x p}.

    Element e = row + d*col (column-major) takes the Box-Muller pair
    q = e // 2 built from u_{2q}, u_{2q+1} of stream (seed, stream, a, 0):
    U1 = ((u_{2q} >> 11) + 1) 2^-53 in (0,1], U2 = (u_{2q+1} >> 11) 2^-53,
    z = sqrt(-2 ln U1) cos(2 pi U2) for even e, sin(...) for odd e.
    """
    key = stream_key(seed, stream, a, 0)
    count = d * p
    npairs = (count + 1) // 2
    u = uniforms_u64(key, 0, 2 * npairs)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (u[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count].reshape(p, d).T.copy()


# ----------------------------------------------------------------------------
# Setup: column norms and the sampling distribution q_i (a reading of Thm. 3)
# ----------------------------------------------------------------------------

def is_sparse(Xt) -> bool:
    """True for a scipy.sparse X^T (row i = column x_i of X)."""
    try:
        import scipy.sparse as sp
    except ImportError:  # pragma: no cover
        return False
    return sp.issparse(Xt)


def as64(Xt):
    """X^T with its stored values widened exactly to FP64 (dense or CSR)."""
    if is_sparse(Xt):
        return Xt.tocsr().astype(np.float64, copy=False)
    return np.asarray(Xt, dtype=np.float64)


def colnorms(Xt) -> tuple[np.ndarray, float]:
    """||x_i||^2 for every column of X and ||X||_F^2, in FP64 (Xt is (n, d))."""
    X64 = as64(Xt)
    if is_sparse(X64):
        norm2 = np.asarray(X64.multiply(X64).sum(axis=1)).ravel()
    else:
        norm2 = np.einsum("ij,ij->i", X64, X64)
    return norm2, float(np.sum(norm2))


@dataclass
class SamplingTable:
    weights: np.ndarray   # uint64 integer weights w_i
    cum: np.ndarray       # inclusive prefix sums of w (uint64)
    total: int            # sum of w
    c: np.ndarray         # c_i = total / w_i  (0 where w_i = 0)
    kappa: float          # max_i c_i ||x_i||^2


def sampling_table(norm2: np.ndarray, mode: int = SAMPLE_IMPORTANCE) -> SamplingTable:
    """Integer sampling weights, q_i = w_i / sum w, and c_i = 1/q_i.

    Importance sampling: w_i = max(1, floor(||x_i||^2 * (2^32 / max_j ||x_j||^2)))
    for non-zero columns, 0 for zero columns, so q_i is ||x_i||^2/||X||_F^2 up to
    the quantisation and zero columns are never drawn.  Uniform: w_i = 1.
    With c_i = 1/q_i the stochastic term c_i x_i x_i^T is an unbiased estimate of
    X X^T whatever the quantisation.
    """
    norm2 = np.asarray(norm2, dtype=np.float64)
    n = norm2.shape[0]
    if mode == SAMPLE_UNIFORM:
        w = np.ones(n, dtype=np.uint64)
    else:
        mx = float(np.max(norm2)) if n else 0.0
        if mx <= 0.0:
            w = np.zeros(n, dtype=np.uint64)
        else:
            scale = 4294967296.0 / mx
            f = np.floor(norm2 * scale)
            w = f.astype(np.uint64)
            w[(norm2 > 0) & (w == 0)] = 1
            w[norm2 <= 0] = 0
    cum = np.cumsum(w, dtype=np.uint64)
    total = int(cum[-1]) if n else 0
    c = np.zeros(n)
    nz = w > 0
    c[nz] = float(total) / w[nz].astype(np.float64)
    kappa = float(np.max(c[nz] * norm2[nz])) if np.any(nz) else 0.0
    return SamplingTable(w, cum, total, c, kappa)


def sample_indices(table: SamplingTable, key: int, m: int) -> np.ndarray:
    """m column indices i_t ~ q: r_t = floor(u_t * total / 2^64), and i_t is the
    first index whose inclusive prefix sum exceeds r_t."""
    if m == 0:
        return np.zeros(0, dtype=np.int64)
    u = uniforms_u64(key, 0, m)
    r = mulhi64(u, table.total)
    return np.searchsorted(table.cum, r, side="right").astype(np.int64)


# ----------------------------------------------------------------------------
# The anchor pass and the inner loop (SVRGsolve)
# ----------------------------------------------------------------------------

def x_apply(Xt, W: np.ndarray) -> np.ndarray:
    """A W = X (X^T W) with X read as stored, in FP64 (Xt is (n, d))."""
    X64 = as64(Xt)
    return np.asarray(X64.T @ np.asarray(X64 @ W))


def anchor(Xt: np.ndarray, Wt: np.ndarray, B: np.ndarray, lam: float) -> np.ndarray:
    """Anchor gradient M = grad F(Wt) = lambda Wt - X (X^T Wt) - B."""
    return lam * Wt - x_apply(Xt, Wt) - B


_CLIB = None


def _clib():
    """Load (building it with gcc on first use if needed) the plain-C inner loop."""
    global _CLIB
    if _CLIB is not None:
        return _CLIB
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "svrg_inner.c")
    so = os.path.join(here, "_svrg_inner.so")
    if (not os.path.exists(so)) or os.path.getmtime(so) < os.path.getmtime(src):
        build_c()
    lib = ctypes.CDLL(so)
    i64, dbl = ctypes.c_int64, ctypes.c_double
    vp = ctypes.c_void_p
    for name in ("oracle_svrg_inner_f64", "oracle_svrg_inner_f32"):
        fn = getattr(lib, name)
        fn.argtypes = [i64, i64, vp, i64, vp, i64, i64, vp, dbl, dbl, vp, vp, vp]
        fn.restype = None
    fn = lib.oracle_svrg_inner_csc
    fn.argtypes = [i64, i64, vp, vp, vp, vp, i64, i64, vp, dbl, dbl, vp, vp, vp]
    fn.restype = None
    _CLIB = lib
    return lib


def build_c() -> str:
    """Compile svrg_inner.c into oracle/_svrg_inner.so (plain gcc, -O2)."""
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "svrg_inner.c")
    so = os.path.join(here, "_svrg_inner.so")
    tmp = so + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src])
    os.replace(tmp, so)
    return so


def svrg_epoch(Xt: np.ndarray, W: np.ndarray, Wt: np.ndarray, M: np.ndarray,
               idx: np.ndarray, c: np.ndarray, eta: float, lam: float, batch: int = 1) -> np.ndarray:
    """len(idx) / batch variance-reduced steps from W; returns the new W.

    Step (batch b, samples i_1..i_b): r_u = x_{i_u}^T (W - Wt) for every u at the
    same W; W <- W - eta [lambda (W - Wt) - (1/b) sum_u c_{i_u} x_{i_u} r_u + M].
    b = 1 is the step of Sec. 2.3's SVRGsolve.
    """
    if len(idx) % batch:
        raise ValueError("index sequence is not a whole number of batches")
    m = len(idx) // batch
    lib = _clib()
    d, p = W.shape
    Wc = np.array(W, dtype=np.float64, order="F", copy=True)
    Wtc = np.asfortranarray(Wt, dtype=np.float64)
    Mc = np.asfortranarray(M, dtype=np.float64)
    idx64 = np.ascontiguousarray(idx, dtype=np.int64)
    c64 = np.ascontiguousarray(c, dtype=np.float64)
    if is_sparse(Xt):
        # rows of X^T = columns of X, in compressed form (factored update, C7b reading)
        Xr = Xt.tocsr()
        colptr = np.ascontiguousarray(Xr.indptr, dtype=np.int64)
        rowidx = np.ascontiguousarray(Xr.indices, dtype=np.int32)
        val = np.ascontiguousarray(Xr.data, dtype=np.float32)
        lib.oracle_svrg_inner_csc(d, p, colptr.ctypes.data, rowidx.ctypes.data, val.ctypes.data,
                                  idx64.ctypes.data, m, batch, c64.ctypes.data, float(eta),
                                  float(lam), Wtc.ctypes.data, Mc.ctypes.data, Wc.ctypes.data)
        return np.array(Wc)
    Xc = np.ascontiguousarray(Xt)
    if Xc.dtype == np.float64:
        fn = lib.oracle_svrg_inner_f64
    elif Xc.dtype == np.float32:
        fn = lib.oracle_svrg_inner_f32
    else:
        Xc = Xc.astype(np.float64)
        fn = lib.oracle_svrg_inner_f64
    fn(d, p, Xc.ctypes.data, Xc.shape[1], idx64.ctypes.data, m, batch,
       c64.ctypes.data, float(eta), float(lam), Wtc.ctypes.data, Mc.ctypes.data,
       Wc.ctypes.data)
    return np.array(Wc)


@dataclass
class Options:
    shift_policy: int = SHIFT_PAPER
    lam: float = 0.0            # FIXED policy shift
    delta: float = 0.0          # gap budget; 0 = estimate it
    theta_eta: float = 0.25
    theta_m: float = 2.0
    tau: float = 1e-6
    max_epochs: int = 60
    m_max: int = 0              # 0 = 50 n
    min_outer: int = 3
    max_outer: int = 2000
    fixed_epochs: int = 0       # > 0: exactly this many anchors per solve
    sampling: int = SAMPLE_IMPORTANCE
    warm_start: int = 1
    max_shift_rounds: int = 30
    batch: int = 1              # samples per inner step (minibatch reading; 1 = Sec. 2.3)
    acc: int = 0                # 1: accelerated SVRG (AccSVRGsolve reading, acc_svrg_solve)
    acc_theta: float = 0.5      # inner accuracy: ||grad|| <= max(tau ||B||, theta sqrt(q) ||r_s||)
    acc_max_outer: int = 200    # proximal-point iterations per accelerated solve
    acc_target: int = 0         # samples per epoch the proximal term aims for; 0 = n


@dataclass
class SolveStats:
    epochs: int = 0
    inner_steps: int = 0
    residual: float = float("nan")
    status: str = "ok"            # ok | notconv | diverged
    outer: int = 0                # proximal-point iterations (accelerated solves)
    outer_res: float = float("nan")  # ||(lambda I - A) W - B|| at the epoch-0 anchor (accelerated)
    outer_done: bool = False


@dataclass
class AccStep:
    """One proximal subproblem of the accelerated solve: the epoch-0 anchor of
    the inner solve also yields the residual of the original system,
    (lambda I - A) W - B = M' - gamma (W - Z), where M' is that anchor's
    gradient of the subproblem.  The inner solve stops at ||M'|| <= tol (set
    from that residual) instead of at tau ||R||."""
    gamma: float
    Z: np.ndarray
    nB: float                     # ||B||_F of the original system
    sq: float                     # sqrt(q), q = mu / (mu + gamma)


class Context:
    """Per-matrix state of one oracle run: X, the sampling table, the counters."""

    def __init__(self, Xt: np.ndarray, seed: int, opts: Options):
        self.Xt = Xt
        self.d = Xt.shape[1]
        self.n = Xt.shape[0]
        self.seed = int(seed)
        self.opts = opts
        self.norm2, self.fro2 = colnorms(Xt)
        self.table = sampling_table(self.norm2, opts.sampling)
        self.solve_count = 0
        self.epochs = 0
        self.inner_steps = 0
        self.x_passes = 0

    def step_params(self, lam: float, mu: float, lam1_up: float) -> tuple[float, int]:
        """eta = theta_eta mu/(lambda^2 + kappa lambda1_up / b), m = ceil(theta_m/(eta mu))
        steps of b samples (b = 1: the step size and epoch length of Theorem 3's
        SVRG; a batch of b averages the stochastic term, dividing its variance,
        the kappa lambda1_up term, by b).  At most m_max samples per epoch."""
        o = self.opts
        b = max(1, int(o.batch))
        eta = o.theta_eta * mu / (lam * lam + self.table.kappa * lam1_up / b)
        m = int(math.ceil(o.theta_m / (eta * mu)))
        m_max = o.m_max if o.m_max > 0 else 50 * self.n
        return eta, min(m, max(1, m_max // b))

    def svrg_solve(self, B: np.ndarray, W0: np.ndarray, lam: float, mu: float,
                   lam1_up: float, Y0: np.ndarray | None = None, acc: AccStep | None = None):
        """Approximate (lambda I - X X^T)^{-1} B by SVRG epochs (Thm. 3).

        Epoch e: Wt = W; M = lambda Wt - X X^T Wt - B; stop when
        ||M||_F <= tau ||B||_F (or after `fixed_epochs` anchors); otherwise m
        inner steps on the stream (seed, SVRG, solve, e).  Stalls (an epoch that
        shrinks the residual by less than 10% after the third) end the solve at
        its floor; a residual above 10x the best, above the first one and above
        1e-3 is divergence (a rebound at the rounding floor, below the start or
        below 1e-3 ||B||, is left to the stall rule).

        With `acc` (one subproblem of acc_svrg_solve) the solve first checks the
        original system's residual at the epoch-0 anchor and returns at once
        (outer_done) when it is below tau ||B_orig||; its own stop is then
        ||M|| <= max(tau ||B_orig||, acc_theta sqrt(q) ||r||).
        """
        o = self.opts
        eta, m = self.step_params(lam, mu, lam1_up)
        solve_id = self.solve_count
        self.solve_count += 1
        W = np.array(W0, dtype=np.float64, copy=True)
        nB = float(np.linalg.norm(B))
        st = SolveStats()
        best = float("inf")
        prev = float("inf")
        res0 = float("inf")
        max_e = o.fixed_epochs if o.fixed_epochs > 0 else o.max_epochs
        for e in range(max_e):
            Wt = W
            M = anchor(self.Xt, Wt, B, lam)
            self.x_passes += 2
            res = float(np.linalg.norm(M)) / nB if nB > 0 else 0.0
            st.epochs = e + 1
            st.residual = res
            self.epochs += 1
            if e == 0:
                res0 = res
            if not np.isfinite(res) or (res > 10.0 * best and res > max(res0, 1e-3)):
                st.status = "diverged"
                return W, st
            tol = o.tau
            if acc is not None:
                if e == 0:
                    st.outer_res = float(np.linalg.norm(M - acc.gamma * (Wt - acc.Z)))
                    if o.fixed_epochs <= 0 and st.outer_res <= o.tau * acc.nB:
                        st.outer_done = True
                        return W, st
                tol = max(o.tau * acc.nB, o.acc_theta * acc.sq * st.outer_res) / nB if nB > 0 else 0.0
            if o.fixed_epochs <= 0:
                if res <= tol:
                    return W, st
                if e >= 3 and res > 0.9 * prev:
                    return W, st
            if e == max_e - 1:
                if o.fixed_epochs <= 0:
                    st.status = "notconv"
                return W, st
            best = min(best, res)
            prev = res
            key = stream_key(self.seed, STREAM_SVRG, solve_id, e)
            b = max(1, int(o.batch))
            idx = sample_indices(self.table, key, m * b)
            W = svrg_epoch(self.Xt, Wt, Wt, M, idx, self.table.c, eta, lam, b)
            st.inner_steps += m
            self.inner_steps += m
        return W, st

    def acc_gamma(self, lam: float, mu: float, lam1_up: float) -> float:
        """Proximal weight gamma of the accelerated solve: 0 when an SVRG epoch
        already draws at most `acc_target` samples (n by default), else the
        gamma at which it draws exactly that many.  With lambda' = lambda + gamma,
        mu' = mu + gamma, K = kappa lambda1_up / b and c = theta_m / theta_eta,
        the uncapped epoch length is m b = b c (lambda'^2 + K) / mu'^2; setting it
        to the target T gives (1 - a) g^2 + 2 (lambda - a mu) g + lambda^2 + K
        - a mu^2 = 0 with a = T / (b c), whose positive root is taken, raised by
        1e-9 relative so that the epoch length ceil(...) is not decided by the
        last bit of a value that sits exactly on the integer T / b."""
        o = self.opts
        b = max(1, int(o.batch))
        T = float(o.acc_target if o.acc_target > 0 else self.n)
        K = self.table.kappa * lam1_up / b
        a = T * o.theta_eta / (b * o.theta_m)
        C = lam * lam + K - a * mu * mu
        if C <= 0.0 or a <= 1.0:
            return 0.0
        h = lam - a * mu
        return (h + math.sqrt(h * h + (a - 1.0) * C)) / (a - 1.0) * (1.0 + 1e-9)

    def solve_linear(self, B: np.ndarray, W0: np.ndarray, lam: float, mu: float,
                     lam1_up: float):
        """(lambda I - A)^{-1} B by SVRG, accelerated when opts.acc is set."""
        if self.opts.acc:
            return self.acc_svrg_solve(B, W0, lam, mu, lam1_up)
        return self.svrg_solve(B, W0, lam, mu, lam1_up)

    def acc_svrg_solve(self, B: np.ndarray, W0: np.ndarray, lam: float, mu: float,
                       lam1_up: float, inner=None):
        """AccSVRGsolve (Sec. 1, Sec. 3, Cor. mainCond): the paper takes the
        acceleration of Frostig et al. 2015 and does not print it.  Reading: an
        accelerated proximal-point loop on F(W) = 1/2 tr W^T (lambda I - A) W
        - tr B^T W, strongly convex with modulus mu.  Iteration s solves the
        subproblem F(W) + gamma/2 ||W - Z_s||^2, i.e. the shifted system
        ((lambda + gamma) I - A) W = B + gamma Z_s, by SVRG warm-started at W_s,
        then extrapolates Z_{s+1} = W_{s+1} + beta (W_{s+1} - W_s) with
        beta = (1 - sqrt q)/(1 + sqrt q), q = mu/(mu + gamma) (Nesterov's
        constant momentum for a strongly convex objective).  gamma balances an
        epoch at about n samples (acc_gamma); gamma = 0 is plain svrg_solve.
        The loop ends when ||(lambda I - A) W_s - B|| <= tau ||B||, read off the
        subproblem's first anchor, or at a stall: after w = max(3, ceil(2/sqrt q))
        subproblems (an expected contraction of e^-2), a residual above half the
        one w subproblems before (the rounding floor of the path).
        `inner(R, W, lam', mu')`, if given, replaces the SVRG subproblem solve
        (tests use an exact solve)."""
        o = self.opts
        gamma = self.acc_gamma(lam, mu, lam1_up)
        if gamma <= 0.0 and inner is None:
            return self.svrg_solve(B, W0, lam, mu, lam1_up)
        q = mu / (mu + gamma)
        sq = math.sqrt(q)
        beta = (1.0 - sq) / (1.0 + sq)
        nB = float(np.linalg.norm(B))
        W = np.array(W0, dtype=np.float64, copy=True)
        Z = W.copy()
        st = SolveStats(status="notconv" if o.fixed_epochs <= 0 else "ok")
        w = max(3, int(math.ceil(2.0 / sq)))
        hist: list[float] = []
        for s in range(o.acc_max_outer):
            R = B + gamma * Z
            if inner is not None:
                Wn = inner(R, W, lam + gamma, mu + gamma)
                sub = SolveStats(outer_res=float(np.linalg.norm(anchor(self.Xt, W, B, lam))))
                sub.outer_done = o.fixed_epochs <= 0 and sub.outer_res <= o.tau * nB
            else:
                Wn, sub = self.svrg_solve(R, W, lam + gamma, mu + gamma, lam1_up,
                                          acc=AccStep(gamma=gamma, Z=Z, nB=nB, sq=sq))
            st.epochs += sub.epochs
            st.inner_steps += sub.inner_steps
            st.outer = s + 1
            st.outer_res = sub.outer_res
            st.residual = sub.outer_res / nB if nB > 0 else 0.0
            if sub.status == "diverged":
                st.status = "diverged"
                return W, st
            if sub.outer_done:
                st.status = "ok"
                st.outer_done = True
                return W, st
            hist.append(sub.outer_res)
            if o.fixed_epochs <= 0 and len(hist) > w and hist[-1] > 0.5 * hist[-1 - w]:
                st.status = "ok"
                return W, st
            Z = Wn + beta * (Wn - W)
            W = Wn
        return W, st


# ----------------------------------------------------------------------------
# Orthonormalisation, Rayleigh-Ritz (Algorithms 1 and 2)
# ----------------------------------------------------------------------------

def orth(W: np.ndarray) -> np.ndarray:
    """Q of W = Q R with diag(R) > 0 (Householder QR; unique for full rank)."""
    q, r = np.linalg.qr(W)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def sym_eig_desc(H: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Eigenpairs of a symmetric H, eigenvalues descending, each eigenvector
    signed so that its largest-magnitude entry is positive."""
    w, V = np.linalg.eigh((H + H.T) * 0.5)
    order = np.argsort(-w, kind="stable")
    w, V = w[order], V[:, order]
    for j in range(V.shape[1]):
        a = int(np.argmax(np.abs(V[:, j])))
        if V[a, j] < 0:
            V[:, j] = -V[:, j]
    return w, V


def rayleigh_ritz(Xt: np.ndarray, S: np.ndarray):
    """Algorithm 2 with C = X X^T: eigendecomposition of S^T C S = (X^T S)^T (X^T S).

    Returns (rho descending, U_hat, Q = X^T S, H)."""
    Q = np.asarray(as64(Xt) @ S)
    H = Q.T @ Q
    rho, Uh = sym_eig_desc(H)
    return rho, Uh, Q, H


# ----------------------------------------------------------------------------
# lambda_1 estimate (Alg. 3 on A), shift tuning (Alg. 7), gap budget
# ----------------------------------------------------------------------------

def lambda1_estimate(ctx: Context, eps: float = 0.25) -> float:
    """Algorithm 3 with C = X X^T, k = 1: L = ceil(eps^-1 ln(d/eps)) power steps
    from z0 ~ N(0, I), then lambda_hat = z^T C z (Theorem 4 sandwich:
    (1-eps) lambda_1 <= lambda_hat <= lambda_1/(1-eps))."""
    d = ctx.d
    L = int(math.ceil((1.0 / eps) * math.log(d / eps)))
    z = gaussian_block(ctx.seed, STREAM_POWER_A, 0, d, 1)
    z /= np.linalg.norm(z)
    for _ in range(L):
        y = x_apply(ctx.Xt, z)
        ctx.x_passes += 2
        z = y / np.linalg.norm(y)
    q = np.asarray(as64(ctx.Xt) @ z)
    ctx.x_passes += 1
    return float(np.sum(q * q))


@dataclass
class ShiftResult:
    lam: float
    inv_est: float           # tilde-lambda^{-1}, ~ lambda - lambda_1
    mu_lb: float             # lower bound on lambda - lambda_1 used for eta, m
    rounds: int
    history: list = field(default_factory=list)   # (lambda, inv_est) per round
    status: str = "ok"


def d_top_eig_inverse(ctx: Context, lam: float, mu: float, lam1_up: float, rnd: int,
                      eps: float = 1.0 / 9.0):
    """Algorithm 3 applied to D = (lambda I - A)^{-1} with k = 1 and accuracy eps:
    L = ceil(eps^-1 ln(d/eps)) power steps, each product D z an SVRG solve, then
    lambda_tilde = z^T D z.  Returns (1/lambda_tilde, status)."""
    d = ctx.d
    L = int(math.ceil((1.0 / eps) * math.log(d / eps)))
    z = gaussian_block(ctx.seed, STREAM_POWER_D, rnd, d, 1)
    z /= np.linalg.norm(z)
    scale = 1.0 / lam
    status = "ok"
    for _ in range(L):
        w, st = ctx.solve_linear(z, scale * z, lam, mu, lam1_up)
        if st.status == "diverged":
            return float("nan"), "diverged"
        nw = float(np.linalg.norm(w))
        scale = nw
        z = w / nw
    w, st = ctx.solve_linear(z, scale * z, lam, mu, lam1_up)
    if st.status == "diverged":
        return float("nan"), "diverged"
    lt = float(z[:, 0] @ w[:, 0])
    if not (lt > 0):
        return float("nan"), "diverged"
    return 1.0 / lt, status


def shift_tune(ctx: Context, lam1_hat: float, delta: float, eps_d: float = 1.0 / 9.0) -> ShiftResult:
    """Algorithm 7: lambda = 1.5 lambda_hat_1, then while the estimate of
    lambda - lambda_1 lies outside [Delta/27, Delta/5], move
    lambda <- lambda - (1 - eps')/2 * estimate.

    mu_lb (for the SVRG step size) starts at lambda - lambda_hat_1/(1-1/4) and is
    then (1-eps')/2 * previous estimate, a lower bound on the new gap by the
    contraction argument of Lemma 10; on return it is (1-eps') * estimate."""
    lam1_up = lam1_hat / (1.0 - 0.25)
    lam = 1.5 * lam1_hat
    mu = lam - lam1_up
    res = ShiftResult(lam=lam, inv_est=float("inf"), mu_lb=mu, rounds=0)
    for rnd in range(ctx.opts.max_shift_rounds):
        inv, status = d_top_eig_inverse(ctx, lam, mu, lam1_up, rnd, eps_d)
        res.rounds = rnd + 1
        res.history.append((lam, inv))
        if status != "ok":
            res.status = status
            return res
        res.lam, res.inv_est = lam, inv
        if delta / 27.0 <= inv <= delta / 5.0:
            res.mu_lb = (1.0 - eps_d) * inv
            return res
        lam = lam - 0.5 * (1.0 - eps_d) * inv
        mu = 0.5 * (1.0 - eps_d) * inv
        res.mu_lb = mu
    res.lam = lam
    res.status = "notconv"
    return res


def delta_estimate(ctx: Context, k: int, p: int) -> float:
    """Gap budget Delta with Delta <= lambda_k - lambda_{p+1} <= 2 Delta
    (Sec. 3; the paper gives no procedure): Algorithm 3 on A with p+1 vectors,
    eps' = 1/(9 p^2), L = min(200, ceil(eps'^-1 ln(d/eps'))) steps, Ritz values
    rho, Delta = (rho_k - rho_{p+1}) / 1.5."""
    d = ctx.d
    eps = 1.0 / (9.0 * p * p)
    L = min(200, int(math.ceil((1.0 / eps) * math.log(d / eps))))
    S = orth(gaussian_block(ctx.seed, STREAM_DELTA, 0, d, p + 1))
    for _ in range(L):
        S = orth(x_apply(ctx.Xt, S))
        ctx.x_passes += 2
    rho, _, _, _ = rayleigh_ritz(ctx.Xt, S)
    ctx.x_passes += 1
    return float(rho[k - 1] - rho[p]) / 1.5


# ----------------------------------------------------------------------------
# The whole path
# ----------------------------------------------------------------------------

@dataclass
class Result:
    U: np.ndarray
    ritz: np.ndarray
    lam: float
    lam1_hat: float
    delta: float
    outer_iters: int
    E_trace: list
    shift: ShiftResult | None
    status: str
    solves: int
    epochs: int
    inner_steps: int
    x_passes: int
    S: np.ndarray


def outer_stop(E: list, eps: float, ell: int, min_outer: int, r_floor: float = 0.0) -> bool:
    """Stop when the predicted remaining decrease of E is <= (eps/4) E_l.

    With differences D_j = E_{j-1} - E_j, the observed rate is the geometric
    mean over the last w <= 4 of them, (D_l / D_{l-w})^(1/w) (R when D_{l-w} is
    not positive), raised to at least r_floor, the rate Theorem 2 predicts for
    the slowest direction; r is clamped to [0, R], R = 1 - 1e-6, and remaining
    = max(D_l, 0) r / (1 - r).  Fast early components cannot end a slow
    iteration, and a non-positive last difference (E at its rounding floor)
    stops."""
    if ell + 1 < max(3, min_outer):
        return False
    w = min(4, len(E) - 2)
    d1 = E[-2] - E[-1]
    d0 = E[-2 - w] - E[-1 - w]
    if d0 > 0 and d1 > 0:
        r = (d1 / d0) ** (1.0 / w)
    elif d0 > 0:
        r = 0.0
    else:
        r = RATE_MAX
    r = min(max(r, r_floor, 0.0), RATE_MAX)
    remaining = max(d1, 0.0) * r / (1.0 - r)
    return remaining <= 0.25 * eps * E[-1]


RATE_MAX = 1.0 - 1e-6


def theory_rate(lam: float, rho: np.ndarray, k: int, p: int) -> float:
    """Per-iteration decrease factor of E from Theorem 2 on D: tan theta_k
    contracts by (lambda - lambda_k)/(lambda - lambda_{p+1}) per step and E's
    excess by its square; estimated with the current Ritz values rho_k and
    rho_p (rho_p <= lambda_p, which overestimates the factor once rho_p has
    passed lambda_{p+1})."""
    den = lam - float(rho[p - 1])
    if den <= 0.0:
        return RATE_MAX
    return min(max((lam - float(rho[k - 1])) / den, 0.0), 1.0) ** 2


def solve(Xt: np.ndarray, k: int, p: int, eps: float, seed: int, opts: Options | None = None,
          Xt_final: np.ndarray | None = None, lam1_hat: float | None = None) -> Result:
    """Rank-k approximation U (d x k) of X by the q = k branch of Algorithm 6.

    Xt_final, if given, is the FP32 copy of a BF16-stored X used for the final
    Rayleigh-Ritz step (the method runs on the stored values, the answer is
    measured on the FP32 ones)."""
    opts = opts or Options()
    ctx = Context(Xt, seed, opts)
    d = ctx.d
    if not (1 <= k < p < d):
        raise ValueError("need 1 <= k < p < d")
    if lam1_hat is None:
        lam1_hat = lambda1_estimate(ctx)
    lam1_up = lam1_hat / (1.0 - 0.25)
    shift = None
    delta = opts.delta
    if opts.shift_policy == SHIFT_PAPER:
        if delta <= 0:
            delta = delta_estimate(ctx, k, p)
        shift = shift_tune(ctx, lam1_hat, delta)
        lam, mu = shift.lam, shift.mu_lb
        if shift.status == "diverged":
            raise RuntimeError("shift tuning diverged")
    elif opts.shift_policy == SHIFT_FAR:
        lam = 2.0 * lam1_up
        mu = lam - lam1_up
    else:
        lam = float(opts.lam)
        mu = lam - lam1_up
        if not mu > 0:
            raise ValueError("fixed shift must exceed lambda_1 / (1 - 1/4)")

    sub = subspace_on_d(ctx, k, p, eps, seed, lam, mu, lam1_up)
    S, rho, Uh = sub.S, sub.rho, sub.Uh
    if Xt_final is not None:
        rho, Uh, Q, H = rayleigh_ritz(Xt_final, S)
        ctx.x_passes += 1
    U = S @ Uh[:, :k]
    return Result(U=U, ritz=rho[:k].copy(), lam=lam, lam1_hat=lam1_hat, delta=delta,
                  outer_iters=sub.outer_iters, E_trace=sub.E_trace, shift=shift, status=sub.status,
                  solves=ctx.solve_count, epochs=ctx.epochs, inner_steps=ctx.inner_steps,
                  x_passes=ctx.x_passes, S=S)


@dataclass
class SubspaceResult:
    S: np.ndarray           # final orthonormal basis (d x p)
    rho: np.ndarray         # its Ritz values with C = A, descending
    Uh: np.ndarray          # Ritz vectors in the basis (p x p)
    outer_iters: int
    E_trace: list
    status: str


def subspace_on_d(ctx: Context, k: int, p: int, eps: float, seed: int, lam: float, mu: float,
                  lam1_up: float, r_floor: float | None = None) -> SubspaceResult:
    """Algorithm 1 on D = (lambda I - A)^{-1} (A of ctx's X) with p columns from
    the Gaussian start (seed, INIT), Rayleigh-Ritz with C = A every iteration
    (Algorithm 2), stopped by outer_stop on E_l = ||X||_F^2 - sum_{j<=k} rho_j
    with the rate floor r_floor (default: theory_rate from rho_k and rho_p;
    without oversampling, p = k, the caller supplies it)."""
    opts = ctx.opts
    d = ctx.d
    S = orth(gaussian_block(seed, STREAM_INIT, 0, d, p))
    E: list[float] = []
    status = "ok"
    ell = 0
    while True:
        rho, Uh, Q, H = rayleigh_ritz(ctx.Xt, S)
        ctx.x_passes += 1
        E.append(ctx.fro2 - float(np.sum(rho[:k])))
        rf = theory_rate(lam, rho, k, p) if r_floor is None else r_floor
        if outer_stop(E, eps, ell, opts.min_outer, rf):
            break
        if ell >= opts.max_outer:
            status = "notconv"
            break
        if opts.warm_start:
            P = (Uh / (lam - rho)[None, :]) @ Uh.T
            W0 = S @ P
        else:
            W0 = np.zeros_like(S)
        W, st = ctx.solve_linear(S, W0, lam, mu, lam1_up)
        if st.status == "diverged":
            status = "diverged"
            break
        S = orth(W)
        ell += 1
    return SubspaceResult(S=S, rho=rho, Uh=Uh, outer_iters=ell, E_trace=E, status=status)


# ----------------------------------------------------------------------------
# Reference optimum of an X without a planted spectrum
# ----------------------------------------------------------------------------

def top_eigs_lanczos(Xt, q: int, tol: float = 1e-13) -> np.ndarray:
    """The q largest eigenvalues of A = X X^T (descending) by ARPACK's implicitly
    restarted Lanczos on the operator v -> X (X^T v), in FP64 (library routine)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    X64 = as64(Xt)
    d = X64.shape[1]
    op = LinearOperator((d, d), matvec=lambda v: np.asarray(X64.T @ np.asarray(X64 @ v)).ravel(),
                        dtype=np.float64)
    w = eigsh(op, k=q, which="LA", tol=tol, return_eigenvectors=False, v0=np.ones(d) / math.sqrt(d))
    return np.sort(w)[::-1]


def plain_subspace_iteration(Xt, k: int, p: int, iters: int, seed: int = 0):
    """Algorithm 1 on A itself (no shift, exact products): S <- orth(A S) from a
    Gaussian start, then Algorithm 2; returns the Ritz values rho_1..rho_p."""
    S = orth(gaussian_block(seed, STREAM_INIT, 0, Xt.shape[1], p))
    for _ in range(iters):
        S = orth(x_apply(Xt, S))
    rho, _, _, _ = rayleigh_ritz(Xt, S)
    return rho


def reference_optimum(Xt, k: int, tol: float = 1e-13) -> float:
    """opt = ||X - X_k||_F^2 = ||X||_F^2 - sum_{j<=k} lambda_j(X X^T)."""
    fro2 = colnorms(Xt)[1]
    return fro2 - float(np.sum(top_eigs_lanczos(Xt, k, tol)[:k]))


# ----------------------------------------------------------------------------
# Metrics (Sec. 1 and Appendix C)
# ----------------------------------------------------------------------------

def frobenius_error(Xt: np.ndarray, U: np.ndarray) -> float:
    """||X - U U^T X||_F^2 = ||X||_F^2 - ||U^T X||_F^2 for orthonormal U."""
    X64 = as64(Xt)
    fro2 = colnorms(X64)[1]
    P = np.asarray(X64 @ U)
    return fro2 - float(np.sum(P * P))


def sin_angle(U1: np.ndarray, U2: np.ndarray) -> float:
    """Largest principal-angle sine between span(U1) and span(U2) (orthonormal
    columns, same count): || U2 - U1 (U1^T U2) ||_2."""
    R = U2 - U1 @ (U1.T @ U2)
    return float(np.linalg.norm(R, 2))
