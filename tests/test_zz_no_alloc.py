"""The sampling table built without allocating (lra_sampling_table_noalloc).

Some callers cannot call cudaMalloc/cudaFree when they build the table: their
framework has reserved the GPU's memory for its own pool allocator, or they
cannot afford the device-wide synchronisation of cudaFree in the middle of
their stream work.  For them the library offers a variant whose scratch lives
in a fixed device array.  Its results must equal those of the allocating entry
point; two calls in a row (a larger input after a smaller one, then a
different mode) check that the shared array's leftover contents never leak into
a result.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1607_02925_gb300 as lra  # noqa: E402


def _norms(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.gamma(1.5, 1.0, size=n)
    v[::11] = 0.0
    v[0] = 3.0
    return v


def _table(fn, ctx, norm2, mode):
    n = norm2.shape[0]
    nd = torch.from_numpy(norm2).cuda()
    cum = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    c = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    total, kappa = fn(ctx, n, nd, mode, cum, c)
    return total, kappa, cum.cpu().numpy(), c.cpu().numpy()


def test_noalloc_table_equals_allocating_table_on_consecutive_calls():
    ctx = lra.lra_init(0)
    try:
        calls = [(70001, lra.LRA_SAMPLE_IMPORTANCE, 1), (1_000_003, lra.LRA_SAMPLE_IMPORTANCE, 2),
                 (4099, lra.LRA_SAMPLE_UNIFORM, 3)]
        for n, mode, seed in calls:
            norm2 = _norms(n, seed)
            ref = _table(lra.lra_sampling_table, ctx, norm2, mode)
            got = _table(lra.lra_sampling_table_noalloc, ctx, norm2, mode)
            # integer and index work is compared bit for bit, as in the other tests
            assert got[0] == ref[0]
            assert got[1] == ref[1]
            assert np.array_equal(got[2], ref[2])
            assert np.array_equal(got[3], ref[3])
    finally:
        lra.lra_finalize(ctx)


def test_noalloc_table_allocates_nothing():
    """On a context whose device-memory budget is one byte every allocation of
    the library fails with LRA_ENOMEM (the allocating builder shows it); the
    no-allocation builder still succeeds there, on two calls in a row, with the
    allocating builder's results from an unconstrained context."""
    ref_ctx = lra.lra_init(0)
    tiny = lra.lra_init(0, 1)
    try:
        for n, mode, seed in [(5000, lra.LRA_SAMPLE_IMPORTANCE, 7), (123457, lra.LRA_SAMPLE_IMPORTANCE, 8)]:
            norm2 = _norms(n, seed)
            nd = torch.from_numpy(norm2).cuda()
            cum = torch.zeros(n, dtype=torch.int64, device="cuda")
            c = torch.zeros(n, dtype=torch.float32, device="cuda")
            st = lra.lib.lra_sampling_table(tiny, n, nd.data_ptr(), mode, cum.data_ptr(), c.data_ptr(), None, None)
            assert st == 2  # LRA_ENOMEM: the budget refuses any allocation
            ref = _table(lra.lra_sampling_table, ref_ctx, norm2, mode)
            got = _table(lra.lra_sampling_table_noalloc, tiny, norm2, mode)
            assert got[0] == ref[0] and got[1] == ref[1]
            assert np.array_equal(got[2], ref[2]) and np.array_equal(got[3], ref[3])
    finally:
        lra.lra_finalize(tiny)
        lra.lra_finalize(ref_ctx)


def test_noalloc_table_rejects_sizes_beyond_its_array():
    ctx = lra.lra_init(0)
    try:
        dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
        st = lra.lib.lra_sampling_table_noalloc(ctx, lra.LRA_NOALLOC_MAX_N + 1, dummy.data_ptr(), 0,
                                                dummy.data_ptr(), dummy.data_ptr(), None, None)
        assert st == 1  # LRA_EINVAL, before any device work
    finally:
        lra.lra_finalize(ctx)
