"""Thin Python binding of liblra.so (C ABI in include/lra.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Functions keep the C names; device buffers are passed as raw
pointers (e.g. a torch CUDA tensor's data_ptr()).  Importing this package
loads the compiled library and fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

from ._ffi import (LRA_BF16, LRA_F16, LRA_F32, LRA_F64, LRA_MAX_P, LRA_NOALLOC_MAX_N,
                   LRA_SAMPLE_IMPORTANCE,
                   LRA_SAMPLE_UNIFORM, LRA_SHIFT_FAR, LRA_SHIFT_FIXED, LRA_SHIFT_PAPER,
                   LRA_STREAM_DELTA, LRA_STREAM_INIT, LRA_STREAM_POWER_A, LRA_STREAM_POWER_D,
                   LRA_STREAM_BLOCK, LRA_STREAM_PART, LRA_STREAM_SVRG, STATUS, LraError, LraOptions,
                   LraReport, LraSolveInfo,
                   declared_symbols, lib, library_path)

__all__ = [n for n in dir() if n.startswith(("LRA_", "Lra", "lra_"))] + [
    "lib", "library_path", "declared_symbols", "STATUS", "options"]


def _check(st: int, allow=()) -> int:
    if st != 0 and st not in allow:
        raise LraError(st, lib.lra_last_error().decode(errors="replace"))
    return st


def _p(x) -> int:
    """Raw pointer of a torch tensor, ctypes buffer, int, or None."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    return C.addressof(x)


def options(**kw) -> LraOptions:
    """lra_options_default() with fields overridden by keyword."""
    o = LraOptions()
    lib.lra_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def lra_stream_key(seed: int, stream: int, a: int = 0, b: int = 0) -> int:
    return int(lib.lra_stream_key(seed, stream, a, b))


def lra_status_str(st: int) -> str:
    return lib.lra_status_str(st).decode()


def lra_init(device: int = 0, hbm_budget_bytes: int = 0):
    ctx = C.c_void_p()
    _check(lib.lra_init(device, hbm_budget_bytes, C.byref(ctx)))
    return ctx


def lra_ctx_stream(ctx) -> int:
    return int(lib.lra_ctx_stream(ctx) or 0)


def lra_finalize(ctx) -> None:
    _check(lib.lra_finalize(ctx))


def lra_create_dense(ctx, d: int, n: int, src_dtype: int, X, ld: int, src_on_device: bool,
                     storage: int):
    m = C.c_void_p()
    _check(lib.lra_create_dense(ctx, d, n, src_dtype, _p(X), ld, int(bool(src_on_device)), storage,
                                C.byref(m)))
    return m


def lra_create_csr(ctx, d, n, nnz, rowptr, colidx, val, src_on_device):
    m = C.c_void_p()
    _check(lib.lra_create_csr(ctx, d, n, nnz, _p(rowptr), _p(colidx), _p(val),
                              int(bool(src_on_device)), C.byref(m)))
    return m


def lra_mat_destroy(m) -> None:
    _check(lib.lra_mat_destroy(m))


def lra_mat_info(m):
    d, n, st, f = C.c_int64(), C.c_int64(), C.c_int(), C.c_double()
    _check(lib.lra_mat_info(m, C.byref(d), C.byref(n), C.byref(st), C.byref(f)))
    return d.value, n.value, st.value, f.value


def lra_solve(m, k, p, eps, seed, opt, U, ritz, rep=None, allow=(4,)) -> int:
    return _check(lib.lra_solve(m, k, p, eps, seed, C.byref(opt) if opt is not None else None,
                                _p(U), _p(ritz), C.byref(rep) if rep is not None else None),
                  allow=allow)


def lra_submit(ctx, m, k, p, eps, seed, opt=None) -> int:
    job = C.c_uint64()
    _check(lib.lra_submit(ctx, m, k, p, eps, seed, C.byref(opt) if opt is not None else None,
                          C.byref(job)))
    return job.value


def lra_poll(ctx, job, timeout_ms, U=None, ritz=None, rep=None, allow=(4, 7, 8)) -> int:
    return _check(lib.lra_poll(ctx, job, timeout_ms, _p(U), _p(ritz),
                               C.byref(rep) if rep is not None else None), allow=allow)


def lra_cancel(ctx, job) -> None:
    _check(lib.lra_cancel(ctx, job))


def lra_colnorms(m, norm2) -> float:
    f = C.c_double()
    _check(lib.lra_colnorms(m, _p(norm2), C.byref(f)))
    return f.value


def lra_sampling_table(ctx, n, norm2, mode, cum, c):
    tot, kap = C.c_uint64(), C.c_double()
    _check(lib.lra_sampling_table(ctx, n, _p(norm2), mode, _p(cum), _p(c), C.byref(tot),
                                  C.byref(kap)))
    return tot.value, kap.value


def lra_sampling_table_noalloc(ctx, n, norm2, mode, cum, c):
    tot, kap = C.c_uint64(), C.c_double()
    _check(lib.lra_sampling_table_noalloc(ctx, n, _p(norm2), mode, _p(cum), _p(c), C.byref(tot),
                                          C.byref(kap)))
    return tot.value, kap.value


def lra_sample(ctx, n, cum, total, key, m, idx) -> None:
    _check(lib.lra_sample(ctx, n, _p(cum), total, key, m, _p(idx)))


def lra_gaussian_block(ctx, seed, stream, a, d, p, out) -> None:
    _check(lib.lra_gaussian_block(ctx, seed, stream, a, d, p, _p(out)))


def lra_anchor(m, p, Wt, B, lam, M):
    a, b = C.c_double(), C.c_double()
    _check(lib.lra_anchor(m, p, _p(Wt), _p(B), lam, _p(M), C.byref(a), C.byref(b)))
    return a.value, b.value


def lra_xt_mul(m, p, W, Y, use_f32_copy=False) -> None:
    _check(lib.lra_xt_mul(m, p, _p(W), _p(Y), int(bool(use_f32_copy))))


def lra_x_mul(m, p, Y, G, use_f32_copy=False) -> None:
    _check(lib.lra_x_mul(m, p, _p(Y), _p(G), int(bool(use_f32_copy))))


def lra_svrg_inner(m, p, W, Wt, M, idx, steps, c, eta, lam) -> None:
    _check(lib.lra_svrg_inner(m, p, _p(W), _p(Wt), _p(M), _p(idx), steps, _p(c), eta, lam))


def lra_svrg_inner_batched(m, p, W, Wt, M, idx, steps, batch, c, eta, lam) -> None:
    _check(lib.lra_svrg_inner_batched(m, p, _p(W), _p(Wt), _p(M), _p(idx), steps, batch, _p(c), eta, lam))


def lra_svrg_solve(m, p, B, W, lam, mu, lam1_up, seed, solve_id, opt=None):
    info = LraSolveInfo()
    st = _check(lib.lra_svrg_solve(m, p, _p(B), _p(W), lam, mu, lam1_up, seed, solve_id,
                                   C.byref(opt) if opt is not None else None, C.byref(info)),
                allow=(4, 5))
    return st, info


def lra_gram(ctx, rows, p, A, lda, G) -> None:
    _check(lib.lra_gram(ctx, rows, p, _p(A), lda, _p(G)))


def lra_cholqr2(ctx, d, p, W, allow=()) -> int:
    return _check(lib.lra_cholqr2(ctx, d, p, _p(W)), allow=allow)


def lra_sym_eig(ctx, p, H, evals, evecs) -> None:
    _check(lib.lra_sym_eig(ctx, p, _p(H), _p(evals), _p(evecs)))


def lra_ritz(m, p, S, use_f32_copy, H, evals, evecs) -> None:
    _check(lib.lra_ritz(m, p, _p(S), int(bool(use_f32_copy)), _p(H), _p(evals), _p(evecs)))


def lra_lambda1_estimate(m, seed) -> float:
    v = C.c_double()
    _check(lib.lra_lambda1_estimate(m, seed, C.byref(v)))
    return v.value


def lra_shift_tune(m, seed, lam1_hat, delta, opt=None, solve_count=0, max_rounds=30):
    sc = C.c_int64(solve_count)
    lam, inv, mu = C.c_double(), C.c_double(), C.c_double()
    rounds = C.c_int()
    hist = (C.c_double * (2 * max_rounds))()
    st = _check(lib.lra_shift_tune(m, seed, lam1_hat, delta,
                                   C.byref(opt) if opt is not None else None, C.byref(sc),
                                   C.byref(lam), C.byref(inv), C.byref(mu), C.byref(rounds), hist),
                allow=(4,))
    h = [(hist[2 * i], hist[2 * i + 1]) for i in range(rounds.value)]
    return dict(status=st, lam=lam.value, inv_est=inv.value, mu_lb=mu.value, rounds=rounds.value,
                history=h, solve_count=sc.value)


def lra_delta_estimate(m, k, p, seed) -> float:
    v = C.c_double()
    _check(lib.lra_delta_estimate(m, k, p, seed, C.byref(v)))
    return v.value
