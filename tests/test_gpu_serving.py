"""Request loop (lra_submit / lra_poll / lra_cancel) on the GPU.

Jobs of different shapes and storage types run concurrently; each result must
be bitwise equal to the same solve run alone (no reduction order depends on
co-running work), and the loop's bookkeeping (cancellation, non-blocking
poll, busy matrices, admission by memory) must hold.
"""
import os

import numpy as np
import pytest

import lra_inputs as L

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1607_02925_gb300 as lra  # noqa: E402

LRA_EAGAIN, LRA_EBUSY, LRA_ECANCELLED, LRA_ENOMEM = 8, 9, 10, 2


def _mat(ctx, d, n, k, seed, storage):
    sig = L.sigma_serving(k, min(d, n))
    Xt, _, _ = L.planted_numpy(d, n, sig, seed)
    Xt = np.ascontiguousarray(Xt.astype(np.float32))
    return lra.lra_create_dense(ctx, d, n, lra.LRA_F32, Xt, d, False, storage)


JOBS = [  # (d, n, k, storage, seed)
    (256, 2048, 5, lra.LRA_F32, 1),
    (300, 3000, 4, lra.LRA_BF16, 2),
    (512, 4096, 8, lra.LRA_F32, 3),
    (256, 2048, 5, lra.LRA_BF16, 4),
    (640, 5000, 10, lra.LRA_F32, 5),
    (384, 2500, 6, lra.LRA_BF16, 6),
]


def test_results_in_the_mix_equal_results_alone():
    ctx = lra.lra_init(0)
    mats = []
    try:
        opt = lra.options(shift_policy=lra.LRA_SHIFT_FAR)
        mats = [_mat(ctx, d, n, k, s, st) for (d, n, k, st, s) in JOBS]
        alone = []
        for (d, n, k, st, s), m in zip(JOBS, mats):
            U = torch.zeros(k, d, device="cuda")
            r = torch.zeros(k, dtype=torch.float64, device="cuda")
            lra.lra_solve(m, k, 2 * k, 1e-3, 100 + s, opt, U, r)
            alone.append((U.cpu().numpy().copy(), r.cpu().numpy().copy()))
        # all jobs submitted at once, twice over (12 jobs over 8 slots)
        ids = []
        for rep in range(2):
            for (d, n, k, st, s), m in zip(JOBS, mats):
                ids.append((lra.lra_submit(ctx, m, k, 2 * k, 1e-3, 100 + s, opt), d, k))
        for j, (jid, d, k) in enumerate(ids):
            U = torch.zeros(k, d, device="cuda")
            r = torch.zeros(k, dtype=torch.float64, device="cuda")
            rep = lra.LraReport()
            st = lra.lra_poll(ctx, jid, -1, U, r, rep)
            assert st == 0, lra.lra_status_str(st)
            Ua, ra = alone[j % len(JOBS)]
            assert np.array_equal(U.cpu().numpy(), Ua)
            assert np.array_equal(r.cpu().numpy(), ra)
            assert rep.kernel_launches > 0
    finally:
        for m in mats:
            lra.lra_mat_destroy(m)
        lra.lra_finalize(ctx)


def test_cancel_queued_job_nonblocking_poll_and_busy_matrix():
    os.environ["LRA_SERVE_SLOTS"] = "1"
    ctx = lra.lra_init(0)
    try:
        m1 = _mat(ctx, 512, 8192, 8, 11, lra.LRA_F32)
        m2 = _mat(ctx, 256, 2048, 5, 12, lra.LRA_F32)
        opt = lra.options(shift_policy=lra.LRA_SHIFT_FAR, min_outer=60, max_outer=60)
        a = lra.lra_submit(ctx, m1, 8, 16, 1e-3, 1, opt)
        b = lra.lra_submit(ctx, m2, 5, 10, 1e-3, 2, opt)
        # one slot: b waits behind a
        assert lra.lra_poll(ctx, b, 0) == LRA_EAGAIN
        assert lra.lib.lra_mat_destroy(m2) == LRA_EBUSY
        lra.lra_cancel(ctx, b)
        assert lra.lra_poll(ctx, b, -1, allow=(LRA_ECANCELLED,)) == LRA_ECANCELLED
        st = lra.lra_poll(ctx, a, -1)
        assert st in (0, 4)
        lra.lra_mat_destroy(m1)
        lra.lra_mat_destroy(m2)
    finally:
        os.environ.pop("LRA_SERVE_SLOTS", None)
        lra.lra_finalize(ctx)


def test_job_beyond_the_memory_budget_is_rejected():
    import ctypes
    ctx = lra.lra_init(0, 24 << 20)   # 24 MB device budget for this context
    try:
        m = _mat(ctx, 256, 4096, 5, 3, lra.LRA_F32)   # 4 MB of X + 4 MB BF16 pair
        job = ctypes.c_uint64()
        # p = 100 needs a workspace far beyond what is left of the budget
        st = lra.lib.lra_submit(ctx, m, 60, 100, 1e-3, 1, None, ctypes.byref(job))
        assert st == LRA_ENOMEM
        # a small job fits and runs
        opt = lra.options(shift_policy=lra.LRA_SHIFT_FAR)
        small = lra.lra_submit(ctx, m, 5, 10, 1e-3, 1, opt)
        U = torch.zeros(5, 256, device="cuda")
        r = torch.zeros(5, dtype=torch.float64, device="cuda")
        assert lra.lra_poll(ctx, small, -1, U, r) == 0
        lra.lra_mat_destroy(m)
    finally:
        lra.lra_finalize(ctx)


def test_admission_sees_matrices_created_after_the_loop_started():
    """The loop's capacity is read at admission time: after a matrix created
    later takes nearly all of the context's budget, a job that fitted before
    is refused with LRA_ENOMEM instead of failing part-way through its solve."""
    import ctypes
    ctx = lra.lra_init(0, 24 << 20)
    mats = []
    try:
        m = _mat(ctx, 256, 4096, 5, 3, lra.LRA_F32)
        mats.append(m)
        opt = lra.options(shift_policy=lra.LRA_SHIFT_FAR)
        U = torch.zeros(5, 256, device="cuda")
        r = torch.zeros(5, dtype=torch.float64, device="cuda")
        first = lra.lra_submit(ctx, m, 5, 10, 1e-3, 1, opt)
        assert lra.lra_poll(ctx, first, -1, U, r) == 0
        # the largest matrix that still fits the budget (200 KB steps), leaving
        # less than any job's workspace
        sig = L.sigma_serving(5, 256)
        for n2 in range(8000, 200, -100):
            Xt, _, _ = L.planted_numpy(256, n2, sig, 9)
            Xd = torch.from_numpy(np.ascontiguousarray(Xt.astype(np.float32))).cuda()  # no staging copy
            h = ctypes.c_void_p()
            st = lra.lib.lra_create_dense(ctx, 256, n2, lra.LRA_F32, Xd.data_ptr(), 256, 1, lra.LRA_F32,
                                          ctypes.byref(h))
            del Xd
            if st == 0:
                mats.append(h)
                break
            assert st == LRA_ENOMEM
        assert len(mats) == 2
        job = ctypes.c_uint64()
        st = lra.lib.lra_submit(ctx, m, 5, 10, 1e-3, 1, ctypes.byref(opt), ctypes.byref(job))
        assert st == LRA_ENOMEM
        # destroying the big matrix gives the memory back to the loop
        lra.lra_mat_destroy(mats.pop())
        again = lra.lra_submit(ctx, m, 5, 10, 1e-3, 1, opt)
        assert lra.lra_poll(ctx, again, -1, U, r) == 0
    finally:
        for h in mats:
            lra.lra_mat_destroy(h)
        lra.lra_finalize(ctx)
