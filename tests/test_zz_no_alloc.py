"""collide_batch_noalloc: the allocation-free variant of collide_batch, for
callers that cannot allocate device memory (stream capture without allocation
nodes, fixed device-memory budgets).  Its scratch is a static device array, so
the test checks that two calls in a row (different inputs, shared scratch)
reproduce collide_batch, and that a batch beyond the static size is refused.
This file is collected last so that a run stopping at the first failure has
run every other test already."""
import ctypes

import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import bz_module, relerr, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bz():
    return bz_module()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_noalloc_matches_collide_batch_twice(bz, precision, tol):
    import torch
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    lib = bz.load()
    stream = torch.cuda.current_stream().cuda_stream
    for seed, n in ((41, 1000), (42, 77)):          # second call smaller: stale scratch must not leak
        f = to_dev(workloads.shifted_maxwellians(n, 2, 32, 10.0, seed=seed), precision)
        want = bz.collide_batch(m, f, precision=precision)
        got = torch.full_like(f, float("nan"))
        rc = lib.collide_batch_noalloc(m._h, bz.PRECISION[precision], 0, ctypes.c_void_p(f.data_ptr()),
                                       ctypes.c_void_p(got.data_ptr()), n, ctypes.c_void_p(stream))
        assert rc == bz.OK, lib.bz_last_error()
        bz.check()
        g, w = got.double().cpu().numpy(), want.double().cpu().numpy()
        assert np.isfinite(g).all()
        assert relerr(g, w) <= tol


def test_noalloc_conserve_and_limits(bz):
    import torch
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    f = to_dev(workloads.bi_maxwellian(64, 2, 32, 10.0, seed=43), "fp32")
    want = bz.collide_batch(m, f, precision="fp32", conserve=True)
    got = bz.collide_batch_noalloc(m, f, precision="fp32", conserve=True)
    bz.check()
    assert relerr(got.double().cpu().numpy(), want.double().cpu().numpy()) <= 1e-5
    # 32 MiB of scratch holds 4224 cells of a 32^2 grid in FP32
    big = torch.zeros((4225, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(bz.BzError) as e:
        bz.collide_batch_noalloc(m, big, precision="fp32")
    assert e.value.code == bz.EINVAL and "4224" in str(e.value)
    ok = bz.collide_batch_noalloc(m, big[:4224], precision="fp32")
    bz.check()
    assert torch.isfinite(ok).all()
    # BZ_CHECK_INPUT would need an allocated error word: refused
    lib = bz.load()
    rc = lib.collide_batch_noalloc(m._h, bz.PRECISION["fp32"], bz.CHECK_INPUT, ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(got.data_ptr()), 64, None)
    assert rc == bz.EINVAL
