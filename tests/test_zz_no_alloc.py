"""collide_batch_noalloc: the allocation-free variant of collide_batch.

It serves callers that cannot allocate device memory while they run (device
memory owned by another allocator, real-time loops that must not meet an
allocation's latency or failure).  Its scratch is one static device array, and
it launches exactly the kernels of collide_batch, so every result must equal
collide_batch's bit for bit: on two calls in a row (different inputs and sizes,
the second smaller, so stale scratch from the first would show), on a 48^2
grid (16-cell tiles, a larger spectrum per cell), with the conservation
projection, and at the size limits (the largest batch accepted; one more cell
refused) in FP32 and FP64.  This file is collected last so that a run stopping
at the first failure has run every other test already."""
import ctypes

import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import bz_module, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bz():
    return bz_module()


def _noalloc_raw(bz, m, f, precision, flags=0):
    """One call through the C ABI (ctypes), output pre-filled with NaN."""
    import torch
    lib = bz.load()
    got = torch.full_like(f, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    n = f.shape[0]
    rc = lib.collide_batch_noalloc(m._h, bz.PRECISION[precision], flags, ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(got.data_ptr()), n, ctypes.c_void_p(stream))
    assert rc == bz.OK, lib.bz_last_error()
    bz.check()
    return got


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_collide_batch_twice(bz, precision):
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    for seed, n in ((41, 1000), (42, 77)):          # second call smaller: stale scratch must not leak
        f = to_dev(workloads.shifted_maxwellians(n, 2, 32, 10.0, seed=seed), precision)
        want = bz.collide_batch(m, f, precision=precision)
        got = _noalloc_raw(bz, m, f, precision)
        g, w = got.cpu().numpy(), want.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.array_equal(g, w)


def test_noalloc_48_grid_twice(bz):
    """48^2 grid: the mode sum runs on 16-cell tiles; 100 then 45 cells."""
    m = bz.Modes(bz.Grid(2, 48, 10.0), 1.0)
    for seed, n in ((44, 100), (45, 45)):
        f = to_dev(workloads.bi_maxwellian(n, 2, 48, 10.0, seed=seed), "fp32")
        want = bz.collide_batch(m, f, precision="fp32")
        got = _noalloc_raw(bz, m, f, "fp32")
        assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())


@pytest.mark.parametrize("precision,N,limit", [("fp32", 32, 4224), ("fp64", 32, 2112), ("fp32", 48, 1856)])
def test_noalloc_size_limits(bz, precision, N, limit):
    """The largest batch the 32 MiB array holds is accepted and equals
    collide_batch; one more cell is refused with the limit in the message."""
    import torch
    m = bz.Modes(bz.Grid(2, N, 10.0), 1.0)
    dt = torch.float32 if precision == "fp32" else torch.float64
    over = torch.zeros((limit + 1, N * N), dtype=dt, device="cuda")
    with pytest.raises(bz.BzError) as e:
        bz.collide_batch_noalloc(m, over, precision=precision)
    assert e.value.code == bz.EINVAL and str(limit) in str(e.value)
    f = to_dev(workloads.bi_maxwellian(limit, 2, N, 10.0, seed=46), precision)
    want = bz.collide_batch(m, f, precision=precision)
    got = _noalloc_raw(bz, m, f, precision)
    assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())


def test_noalloc_conserve_and_flags(bz):
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    f = to_dev(workloads.bi_maxwellian(64, 2, 32, 10.0, seed=43), "fp32")
    want = bz.collide_batch(m, f, precision="fp32", conserve=True)
    got = _noalloc_raw(bz, m, f, "fp32", flags=bz.CONSERVE)
    assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())
    # BZ_CHECK_INPUT would need an allocated error word: refused
    lib = bz.load()
    rc = lib.collide_batch_noalloc(m._h, bz.PRECISION["fp32"], bz.CHECK_INPUT, ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(got.data_ptr()), 64, None)
    assert rc == bz.EINVAL
