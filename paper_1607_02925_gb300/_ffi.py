"""ctypes declarations of include/lra.h (structs, constants, prototypes)."""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "lra.h")
_LIBDIR = os.path.join(HERE, "_lib")


def library_path() -> str:
    return os.path.join(_LIBDIR, "liblra.so")


LRA_F32, LRA_BF16, LRA_F16, LRA_F64 = 0, 1, 2, 3
LRA_SHIFT_PAPER, LRA_SHIFT_FAR, LRA_SHIFT_FIXED = 0, 1, 2
LRA_SAMPLE_IMPORTANCE, LRA_SAMPLE_UNIFORM = 0, 1
LRA_STREAM_INIT, LRA_STREAM_POWER_A, LRA_STREAM_POWER_D, LRA_STREAM_SVRG, LRA_STREAM_DELTA = 1, 2, 3, 4, 5
LRA_STREAM_PART, LRA_STREAM_BLOCK = 6, 7
LRA_MAX_P = 112
LRA_NOALLOC_MAX_N = 1 << 24
STATUS = ["LRA_OK", "LRA_EINVAL", "LRA_ENOMEM", "LRA_ECUDA", "LRA_ENOTCONV", "LRA_EDIVERGED",
          "LRA_ENUMERIC", "LRA_ETIMEOUT", "LRA_EAGAIN", "LRA_EBUSY", "LRA_ECANCELLED",
          "LRA_EUNSUPPORTED"]


class LraError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}")


class LraOptions(C.Structure):
    _fields_ = [
        ("struct_size", C.c_size_t),
        ("shift_policy", C.c_int),
        ("lambda_", C.c_double),
        ("delta", C.c_double),
        ("theta_eta", C.c_double),
        ("theta_m", C.c_double),
        ("tau", C.c_double),
        ("max_epochs", C.c_int),
        ("m_max", C.c_int64),
        ("min_outer", C.c_int),
        ("max_outer", C.c_int),
        ("fixed_epochs", C.c_int),
        ("sampling", C.c_int),
        ("warm_start", C.c_int),
        ("max_shift_rounds", C.c_int),
        ("lambda1_hat", C.c_double),
        ("trace_E", C.POINTER(C.c_double)),
        ("trace_cap", C.c_int),
        ("profile", C.c_int),
        ("batch", C.c_int),
        ("acc", C.c_int),
        ("acc_theta", C.c_double),
        ("acc_max_outer", C.c_int),
        ("acc_target", C.c_int64),
        ("partition", C.c_int),
        ("part_max_iters", C.c_int),
        ("wait_cycles", C.c_int64),
    ]


class LraReport(C.Structure):
    _fields_ = [
        ("struct_size", C.c_size_t),
        ("status", C.c_int),
        ("outer_iters", C.c_int),
        ("shift_rounds", C.c_int),
        ("solves", C.c_int64),
        ("epochs", C.c_int64),
        ("inner_steps", C.c_int64),
        ("x_passes", C.c_int64),
        ("kernel_launches", C.c_int64),
        ("lambda_", C.c_double),
        ("lambda1_hat", C.c_double),
        ("delta", C.c_double),
        ("mu_lb", C.c_double),
        ("eta", C.c_double),
        ("m", C.c_int64),
        ("fro2", C.c_double),
        ("err_est", C.c_double),
        ("last_residual", C.c_double),
        ("ms_setup", C.c_double),
        ("ms_shift", C.c_double),
        ("ms_outer", C.c_double),
        ("ms_final", C.c_double),
        ("ms_total", C.c_double),
        ("xtw_ms", C.c_double),
        ("xy_ms", C.c_double),
        ("inner_ms", C.c_double),
        ("xtw_launches", C.c_int64),
        ("xy_launches", C.c_int64),
        ("inner_launches", C.c_int64),
        ("xtw_cols", C.c_int64),
        ("xy_cols", C.c_int64),
        ("phase_ms", C.c_double * 8),
        ("part_stages", C.c_int),
        ("part_q", C.c_int * LRA_MAX_P),
        ("part_kind", C.c_int * LRA_MAX_P),
    ]

    def __init__(self):
        super().__init__()
        self.struct_size = C.sizeof(LraReport)

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "struct_size"}


class LraSolveInfo(C.Structure):
    _fields_ = [
        ("epochs", C.c_int),
        ("inner_steps", C.c_int64),
        ("m", C.c_int64),
        ("eta", C.c_double),
        ("residual", C.c_double),
        ("status", C.c_int),
        ("outer", C.c_int),
        ("gamma", C.c_double),
    ]


vp, i64, u64, dbl, ci = C.c_void_p, C.c_int64, C.c_uint64, C.c_double, C.c_int
_PROTOS = {
    "lra_options_default": (None, [vp]),
    "lra_init": (ci, [ci, C.c_size_t, vp]),
    "lra_finalize": (ci, [vp]),
    "lra_ctx_stream": (vp, [vp]),
    "lra_create_dense": (ci, [vp, i64, i64, ci, vp, i64, ci, ci, vp]),
    "lra_create_csr": (ci, [vp, i64, i64, i64, vp, vp, vp, ci, vp]),
    "lra_mat_destroy": (ci, [vp]),
    "lra_mat_info": (ci, [vp, vp, vp, vp, vp]),
    "lra_solve": (ci, [vp, ci, ci, dbl, u64, vp, vp, vp, vp]),
    "lra_submit": (ci, [vp, vp, ci, ci, dbl, u64, vp, vp]),
    "lra_poll": (ci, [vp, u64, ci, vp, vp, vp]),
    "lra_cancel": (ci, [vp, u64]),
    "lra_status_str": (C.c_char_p, [ci]),
    "lra_last_error": (C.c_char_p, []),
    "lra_stream_key": (u64, [u64, u64, u64, u64]),
    "lra_colnorms": (ci, [vp, vp, vp]),
    "lra_sampling_table": (ci, [vp, i64, vp, ci, vp, vp, vp, vp]),
    "lra_sampling_table_noalloc": (ci, [vp, i64, vp, ci, vp, vp, vp, vp]),
    "lra_sample": (ci, [vp, i64, vp, u64, u64, i64, vp]),
    "lra_gaussian_block": (ci, [vp, u64, u64, u64, i64, ci, vp]),
    "lra_anchor": (ci, [vp, ci, vp, vp, dbl, vp, vp, vp]),
    "lra_xt_mul": (ci, [vp, ci, vp, vp, ci]),
    "lra_x_mul": (ci, [vp, ci, vp, vp, ci]),
    "lra_svrg_inner": (ci, [vp, ci, vp, vp, vp, vp, i64, vp, dbl, dbl]),
    "lra_svrg_inner_batched": (ci, [vp, ci, vp, vp, vp, vp, i64, ci, vp, dbl, dbl]),
    "lra_svrg_solve": (ci, [vp, ci, vp, vp, dbl, dbl, dbl, u64, i64, vp, vp]),
    "lra_gram": (ci, [vp, i64, ci, vp, i64, vp]),
    "lra_cholqr2": (ci, [vp, i64, ci, vp]),
    "lra_sym_eig": (ci, [vp, ci, vp, vp, vp]),
    "lra_ritz": (ci, [vp, ci, vp, ci, vp, vp, vp]),
    "lra_lambda1_estimate": (ci, [vp, u64, vp]),
    "lra_shift_tune": (ci, [vp, u64, dbl, dbl, vp, vp, vp, vp, vp, vp, vp]),
    "lra_delta_estimate": (ci, [vp, ci, ci, u64, vp]),
}


def declared_symbols() -> list[str]:
    """Names of the functions include/lra.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lra_[a-z0-9_]+)\s*\(", txt)))


def _load():
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(
            "liblra.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"`"
            % path)
    L = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()
