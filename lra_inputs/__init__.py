"""Seeded synthetic inputs for rank-k approximation workloads.

This module only *generates data*: planted-spectrum dense matrices
X = U diag(sigma) V^T with Haar-distributed U, V, and Zipf-row sparse matrices.
It holds none of the method's arithmetic (no power iteration, no solver, no
sampling rule), so both the FP64 oracle and the CUDA path may draw their inputs
from it.

The paper (Gonen & Shalev-Shwartz, "Faster Low-rank Approximation using Adaptive
Gap-based Preconditioning", Sec. 1) works with X in R^{d x n}, columns x_i being
data points, and the optimum Pi* = sum_{i<=k} u_i u_i^T with
||X - X_k||_F^2 = sum_{i>k} sigma_i^2.  Planting sigma therefore fixes the optimum
in closed form, which is what the tests pin against.

Layout convention: X is column-major d x n with leading dimension d (a column,
i.e. one data point, is contiguous), which is the same memory as a C-contiguous
(n, d) array.  Every generator here returns that (n, d) C-contiguous array
`Xt`, so `Xt.T` is the d x n matrix X.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "sigma_small_gap", "sigma_steep_head", "sigma_exp_two_gaps",
    "sigma_serving", "haar_numpy", "planted_numpy", "planted_torch", "zipf_csr",
    "closed_form_opt",
]


# ----------------------------------------------------------------------------
# Planted spectra (sigma_1 >= sigma_2 >= ...), 1-based descriptions in docstrings
# ----------------------------------------------------------------------------

def sigma_small_gap(r: int = 256) -> np.ndarray:
    """Spectrum with a tiny consecutive gap at k=5 and a large one at p+1=11.

    sigma_1..5 = 1.00 .98 .96 .94 .92, sigma_6..10 = .915 .90 .88 .86 .84,
    sigma_11 = .60 and sigma_i = .60 (i/11)^-1 for i > 11.  With k=5, p=10 the
    multiplicative gaps are G_{k,k+1} ~ 0.005 and G_{k,p+1} ~ 0.35 (Eq. 1 of the
    paper defines G_{i,j} = (sigma_i - sigma_j)/sigma_i).
    """
    s = np.zeros(r)
    head = [1.00, 0.98, 0.96, 0.94, 0.92, 0.915, 0.90, 0.88, 0.86, 0.84, 0.60]
    s[: len(head)] = head
    i = np.arange(len(head) + 1, r + 1, dtype=np.float64)
    s[len(head):] = 0.60 * (i / 11.0) ** -1
    return s


def sigma_steep_head(r: int = 4096) -> np.ndarray:
    """sigma_i = i^-1/2 (i <= 20), sigma_21 = .98 sigma_20, sigma_22..40 linear
    from sigma_21 down to sigma_40 = .6 sigma_20 (endpoint included), and
    sigma_i = .6 sigma_20 (i - 39)^-1/2 for i > 40."""
    s = np.zeros(r)
    i = np.arange(1, r + 1, dtype=np.float64)
    s[:20] = i[:20] ** -0.5
    s20 = s[19]
    s[20] = 0.98 * s20
    for ii in range(22, 41):
        s[ii - 1] = s[20] + (ii - 21) / (40 - 21) * (0.6 * s20 - s[20])
    s[40:] = 0.6 * s20 * (i[40:] - 39.0) ** -0.5
    return s


def sigma_exp_two_gaps(r: int = 640) -> np.ndarray:
    """sigma_i = exp(-i/30), times .95 for i > 50 and a further .6 for i > 100
    (a 5% gap between sigma_50 and sigma_51, a 40% gap between sigma_100 and
    sigma_101).  Truncated at r = 640, where sigma ~ 3e-10."""
    i = np.arange(1, r + 1, dtype=np.float64)
    s = np.exp(-i / 30.0)
    s[i > 50] *= 0.95
    s[i > 100] *= 0.6
    return s


def sigma_partition(r: int = 64) -> np.ndarray:
    """Spectrum for Algorithm 6's branches with k = 3, p = 4 (lambda = sigma^2):
    lambda_1 = 40 (a multiplicative gap to lambda_2 = 10), lambda_2..4 = 10, 9.6,
    9.3 (relative steps 4% and 3%, below p^-2 = 6.25%), lambda_5 = 8.85
    (lambda_3 - lambda_5 = 0.75 = 1.5 Delta with Delta = 0.5, so the 0.4 gap after
    lambda_2 exceeds 5 Delta / 9 and the 0.3 one after lambda_3 does not), then
    lambda_i = 2 (i / 6)^-1 for i >= 6."""
    lam = np.zeros(r)
    head = [40.0, 10.0, 9.6, 9.3, 8.85]
    lam[: len(head)] = head
    i = np.arange(len(head) + 1, r + 1, dtype=np.float64)
    lam[len(head):] = 2.0 * (i / 6.0) ** -1
    return np.sqrt(lam)


def sigma_serving(k: int, r: int) -> np.ndarray:
    """Small-gap spectrum rescaled to rank k (p = 2k): k=5 gives sigma_small_gap.

    Otherwise sigma_1..k linear 1.00 -> .92, sigma_{k+1} = .915, sigma_{k+2..2k}
    linear down to .84, sigma_{2k+1} = .6 and sigma_i = .6 (2k+1)/i beyond.
    """
    if k == 5:
        return sigma_small_gap(r)
    s = np.zeros(r)
    s[:k] = np.linspace(1.00, 0.92, k)
    s[k] = 0.915
    s[k + 1: 2 * k] = np.linspace(0.915, 0.84, k)[1:]
    s[2 * k] = 0.60
    i = np.arange(2 * k + 2, r + 1, dtype=np.float64)
    s[2 * k + 1:] = 0.60 * (2 * k + 1) / i
    return s


def closed_form_opt(sigma: np.ndarray, k: int) -> float:
    """||X - X_k||_F^2 = sum_{i>k} sigma_i^2 (Sec. 1 / Sec. 2.1 of the paper)."""
    return float(np.sum(np.asarray(sigma, dtype=np.float64)[k:] ** 2))


# ----------------------------------------------------------------------------
# Haar-distributed orthonormal factors
# ----------------------------------------------------------------------------

def haar_numpy(rows: int, r: int, rng: np.random.Generator) -> np.ndarray:
    """rows x r matrix with orthonormal columns, Haar distributed.

    Q factor of an N(0,1) matrix with the signs of diag(R) made positive
    (Mezzadri's correction), FP64.
    """
    g = rng.standard_normal((rows, r))
    q, rr = np.linalg.qr(g)
    q *= np.sign(np.diag(rr))[None, :]
    return q


def planted_numpy(d: int, n: int, sigma: np.ndarray, seed: int):
    """FP64 X = U diag(sigma) V^T (d x n) on the host.

    Returns (Xt, U, sigma) where Xt is the C-contiguous (n, d) array holding X
    column-major, and U (d x r) the planted left singular vectors.
    """
    r = len(sigma)
    assert r <= min(d, n)
    rng = np.random.default_rng(seed)
    U = haar_numpy(d, r, rng)
    V = haar_numpy(n, r, rng)
    Xt = np.ascontiguousarray((V * sigma[None, :]) @ U.T)  # (n, d) = X^T
    return Xt, U, np.asarray(sigma, dtype=np.float64)


def _qr(a):
    """QR of a torch matrix on its device; on the host when the device's linear
    algebra library cannot be loaded (as under a profiler), moved back after."""
    import torch
    try:
        return torch.linalg.qr(a)
    except RuntimeError:
        q, r = torch.linalg.qr(a.cpu())
        return q.to(a.device), r.to(a.device)


def planted_torch(d: int, n: int, sigma: np.ndarray, seed: int, device="cpu",
                  dtype=None, chunk: int = 1 << 16):
    """X = U diag(sigma) V^T generated with torch (for sizes that need a GPU).

    Computed in FP32 with TF32 disabled; returns (Xt, U) with Xt an (n, d)
    tensor of `dtype` (default float32) on `device` holding X column-major, and U
    (d x r, float64 on the host).  V is only ever materialised chunk by chunk of
    rows after its QR: the Haar V of size n x r is the Q factor of an N(0,1)
    n x r matrix, whose QR needs the whole matrix, so it is formed once.
    """
    import torch
    if dtype is None:
        dtype = torch.float32
    r = len(sigma)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        gu = torch.randn(d, r, generator=gen, device=device, dtype=torch.float32)
        qu, ru = _qr(gu)
        qu = qu * torch.sign(torch.diagonal(ru))[None, :]
        del gu, ru
        gv = torch.randn(n, r, generator=gen, device=device, dtype=torch.float32)
        qv, rv = _qr(gv)
        qv = qv * torch.sign(torch.diagonal(rv))[None, :]
        del gv, rv
        sig = torch.as_tensor(np.asarray(sigma), device=device, dtype=torch.float32)
        us = (qu * sig[None, :]).T.contiguous()          # r x d
        Xt = torch.empty(n, d, device=device, dtype=dtype)
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            Xt[s:e] = (qv[s:e] @ us).to(dtype)
        U = qu.double().cpu().numpy()
        del qv, us, qu
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev_tf32
    return Xt, U


# ----------------------------------------------------------------------------
# Sparse term-document-like matrix
# ----------------------------------------------------------------------------

def zipf_csr(d: int, n: int, seed: int, mean_nnz: float = 100.0, zipf_s: float = 1.1,
             chunk: int = 16384):
    """Sparse X (d x n) with Zipf(s) row ids, returned in CSR of X (d rows).

    Column j holds c_j = 1 + Poisson(mean_nnz - 1) distinct rows (at most d),
    drawn from a Zipf(s) law over 1..d one after another with repeats rejected
    (no row permutation): the column keeps the first c_j distinct rows of its
    draw sequence.  Its values are ln(2 + Poisson(2)) and the column is then
    L2-normalised.  Columns are generated in chunks of `chunk`, each from one
    draw block of the seeded generator, so the output depends only on the
    arguments.  Returns (rowptr int64[d+1], colidx int32[nnz], val float32[nnz])
    with column indices sorted within each row.
    """
    rng = np.random.default_rng(seed)
    ranks = np.arange(1, d + 1, dtype=np.float64)
    pmf = ranks ** (-zipf_s)
    pmf /= pmf.sum()
    cdf = np.cumsum(pmf)
    cdf[-1] = 1.0
    cnt = np.minimum(1 + rng.poisson(mean_nnz - 1.0, size=n), d).astype(np.int64)
    rows_parts, cols_parts = [], []
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        need = cnt[c0:c1]
        got_rows = [None] * (c1 - c0)
        todo = np.arange(c1 - c0)
        budget = 2 * need + 16
        while todo.size:
            nd = budget[todo]
            col = np.repeat(todo, nd)
            row = np.minimum(np.searchsorted(cdf, rng.random(int(nd.sum())), side="right"), d - 1)
            # first occurrence of each (column, row) in draw order
            key = col.astype(np.int64) * d + row
            _, first = np.unique(key, return_index=True)
            first.sort()
            col_f, row_f = col[first], row[first]
            # rank of each distinct draw within its column, in draw order
            starts = np.searchsorted(col_f, todo)
            rank = np.arange(col_f.size) - np.repeat(starts, np.diff(np.append(starts, col_f.size)))
            have = np.diff(np.append(starts, col_f.size))
            ok = have >= need[todo]
            keep = rank < need[col_f]
            sel = keep & ok[np.searchsorted(todo, col_f)]
            rr, cc = row_f[sel], col_f[sel]
            bounds = np.searchsorted(cc, todo[ok])
            ends = np.append(bounds[1:], cc.size)
            for t, b, e in zip(todo[ok], bounds, ends):
                got_rows[t] = rr[b:e]
            todo = todo[~ok]
            budget[todo] *= 2
        for t in range(c1 - c0):
            rows_parts.append(got_rows[t])
            cols_parts.append(np.full(got_rows[t].size, c0 + t, dtype=np.int32))
    rows_all = np.concatenate(rows_parts).astype(np.int32)
    cols_all = np.concatenate(cols_parts)
    v = np.log(2.0 + rng.poisson(2.0, size=rows_all.size))
    colptr = np.concatenate(([0], np.cumsum(cnt)))
    nrm = np.sqrt(np.add.reduceat(v * v, colptr[:-1]))
    vals_all = (v / np.repeat(nrm, cnt)).astype(np.float32)
    order = np.lexsort((cols_all, rows_all))
    rows_s = rows_all[order]
    colidx = cols_all[order]
    val = vals_all[order]
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.add.at(rowptr, rows_s.astype(np.int64) + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, colidx, val


# ----------------------------------------------------------------------------
# Named workloads (shapes and spectra of the benchmark configurations)
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    d: int
    n: int
    k: int
    p: int
    r: int
    seed: int
    storage: str          # "f64", "f32", "bf16", "csr"

    def sigma(self) -> np.ndarray:
        if self.name.startswith("small_gap"):
            return sigma_small_gap(self.r)
        if self.name.startswith("steep_head"):
            return sigma_steep_head(self.r)
        if self.name.startswith("exp_two_gaps"):
            return sigma_exp_two_gaps(self.r)
        if self.name.startswith("partition"):
            return sigma_partition(self.r)
        raise ValueError(f"{self.name} has no planted spectrum")

    def csr(self):
        """(rowptr, colidx, val) of a sparse workload."""
        return zipf_csr(self.d, self.n, self.seed)

    def opt(self) -> float:
        return closed_form_opt(self.sigma(), self.k)


WORKLOADS = {
    # FP64 dense, d=256, n=2048, k=5, p=10: the oracle finishes in seconds
    "small_gap_256x2048": Workload("small_gap_256x2048", 256, 2048, 5, 10, 256, 0, "f64"),
    # FP32 dense, d=4096, n=262144, k=20, p=40
    "steep_head_4096x262144": Workload("steep_head_4096x262144", 4096, 262144, 20, 40, 4096, 2, "f32"),
    # the same spectrum and d with n = 65536 (X = 1 GB): profiling captures
    "steep_head_4096x65536": Workload("steep_head_4096x65536", 4096, 65536, 20, 40, 4096, 2, "f32"),
    # BF16 (and FP32) dense, d=8192, n=1048576, k=50, p=100
    "exp_two_gaps_8192x1048576": Workload("exp_two_gaps_8192x1048576", 8192, 1048576, 50, 100, 640, 3, "bf16"),
    # the same spectrum and d with n = 65536 (X = 1.07 GB BF16): profiling captures
    "exp_two_gaps_8192x65536": Workload("exp_two_gaps_8192x65536", 8192, 65536, 50, 100, 640, 3, "bf16"),
    # Algorithm 6's branches (a multiplicative gap, then an additive one): FP64,
    # d=64, n=800, k=3, p=4, Delta = 0.5
    "partition_64x800": Workload("partition_64x800", 64, 800, 3, 4, 64, 5, "f64"),
    # sparse CSR (Zipf term-document), d=50000, n=500000, ~100 non-zeros per column
    "zipf_csr_50000x500000": Workload("zipf_csr_50000x500000", 50000, 500000, 10, 20, 0, 4, "csr"),
    # the same law at d=2000, n=20000 (tests and the reference optimum's cross-check)
    "zipf_csr_2000x20000": Workload("zipf_csr_2000x20000", 2000, 20000, 10, 20, 0, 4, "csr"),
}
