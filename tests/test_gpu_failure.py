"""Failure handling on the GPU without faulting it (needs a GPU).

* A tensor-core pipeline wait that runs out: lra_options.wait_cycles = 1 makes
  the first wait of the X passes give up; the kernels record the timeout,
  wait (with the default limit) for their own copies and MMAs in flight, free
  their tensor memory and return, and the solve returns LRA_ETIMEOUT.  The same
  context then solves the same matrix normally.
* Cancelling a job of the request loop while it runs: the solve stops between
  outer iterations with LRA_ECANCELLED, and the loop serves the next job.
"""
import ctypes
import os
import time

import numpy as np
import pytest

import lra_inputs as L
from oracle import lra_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1607_02925_gb300 as lra  # noqa: E402

LRA_EAGAIN, LRA_ETIMEOUT, LRA_ECANCELLED = 8, 7, 10


def _planted(d, n, k, seed):
    Xt, _, s = L.planted_numpy(d, n, L.sigma_serving(k, min(d, n)), seed)
    return np.ascontiguousarray(Xt.astype(np.float32)), s


@pytest.mark.parametrize("storage", [lra.LRA_F32, lra.LRA_BF16])
def test_pipeline_wait_timeout_returns_status_and_context_recovers(storage):
    d, n, k, p = 512, 8192, 5, 10
    Xt, s = _planted(d, n, k, 3)
    ctx = lra.lra_init(0)
    try:
        m = lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, storage)
        try:
            U = torch.zeros(k, d, device="cuda")
            r = torch.zeros(k, dtype=torch.float64, device="cuda")
            o = lra.options(shift_policy=lra.LRA_SHIFT_FAR, wait_cycles=1)
            st = lra.lib.lra_solve(m, k, p, 1e-3, 0, ctypes.byref(o), U.data_ptr(), r.data_ptr(), None)
            assert st == LRA_ETIMEOUT, lra.lra_status_str(st)
            assert "timed out" in lra.lib.lra_last_error().decode()
            # the context and the matrix are still usable at the default limit
            o = lra.options(shift_policy=lra.LRA_SHIFT_FAR)
            st = lra.lib.lra_solve(m, k, p, 1e-3, 0, ctypes.byref(o), U.data_ptr(), r.data_ptr(), None)
            assert st == 0, lra.lra_status_str(st)
            ratio = O.frobenius_error(Xt, U.double().cpu().numpy().T) / L.closed_form_opt(s, k)
            assert ratio <= 1.0 + 1e-3
        finally:
            lra.lra_mat_destroy(m)
    finally:
        lra.lra_finalize(ctx)


def test_cancel_running_job():
    os.environ["LRA_SERVE_SLOTS"] = "1"
    ctx = lra.lra_init(0)
    try:
        Xt, s = _planted(1024, 16384, 10, 5)
        m = lra.lra_create_dense(ctx, 1024, 16384, lra.LRA_F32, Xt, 1024, False, lra.LRA_F32)
        # a long fixed schedule: 20000 outer iterations with 4 anchors each (tens of seconds)
        slow = lra.options(shift_policy=lra.LRA_SHIFT_FAR, min_outer=20000, max_outer=20000, fixed_epochs=4)
        job = lra.lra_submit(ctx, m, 10, 20, 1e-3, 1, slow)
        time.sleep(0.5)   # one slot, one job: it is running by now
        assert lra.lra_poll(ctx, job, 0) == LRA_EAGAIN
        t0 = time.perf_counter()
        lra.lra_cancel(ctx, job)
        st = lra.lra_poll(ctx, job, 60000, allow=(LRA_ECANCELLED,))
        assert st == LRA_ECANCELLED
        assert time.perf_counter() - t0 < 30.0
        # the loop serves the next job normally
        fast = lra.options(shift_policy=lra.LRA_SHIFT_FAR)
        job2 = lra.lra_submit(ctx, m, 10, 20, 1e-3, 2, fast)
        U = torch.zeros(10, 1024, device="cuda")
        r = torch.zeros(10, dtype=torch.float64, device="cuda")
        assert lra.lra_poll(ctx, job2, -1, U, r) == 0
        ratio = O.frobenius_error(Xt, U.double().cpu().numpy().T) / L.closed_form_opt(s, 10)
        assert ratio <= 1.0 + 1e-3
        lra.lra_mat_destroy(m)
    finally:
        os.environ.pop("LRA_SERVE_SLOTS", None)
        lra.lra_finalize(ctx)
