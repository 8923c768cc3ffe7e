"""collide_batch_host: the pipelined host-buffer entry point must give exactly
the device entry point's result (same kernels per chunk), for pinned and
pageable buffers, ragged chunk counts and both precisions."""
import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import bz_module, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bz():
    return bz_module()


@pytest.mark.parametrize("n", [1, 4864, 7296, 20000, 40000])
def test_host_pinned_equals_device(bz, n):
    """A chunk is one full wave of the grid's mode-sum kernel (4864 cells for a
    one-CTA-per-SM 32-cell kernel on 152 SMs, 7296 for three 16-cell CTAs per
    SM): one cell, one exact chunk of either size, and batches of several
    chunks with quarter-size first and last chunks and a ragged one."""
    import torch
    N, L = 16, 8.0
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    f = workloads.bi_maxwellian(n, 2, N, L, seed=77).astype(np.float32)
    fh = torch.from_numpy(f).pin_memory()
    Qh = bz.collide_batch_host(m, fh, precision="fp32")
    torch.cuda.current_stream().synchronize()
    bz.check()
    Qd = bz.collide_batch(m, to_dev(f, "fp32"), precision="fp32").cpu().numpy()
    assert np.array_equal(Qh.numpy(), Qd)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_host_pageable_numpy(bz, precision):
    import torch
    N, L, n = 32, 10.0, 9000
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    f = workloads.bi_maxwellian(n, 2, N, L, seed=78)
    f = f.astype(np.float32) if precision == "fp32" else f
    Q = np.full_like(f, np.nan)
    bz.collide_batch_host(m, f, Q, precision=precision, conserve=True)
    torch.cuda.current_stream().synchronize()
    bz.check()
    Qd = bz.collide_batch(m, to_dev(f, precision), precision=precision, conserve=True).cpu().numpy()
    assert np.array_equal(Q, Qd)


def test_host_rejects_device_tensor_and_capture(bz):
    import torch
    m = bz.Modes(bz.Grid(2, 16, 8.0), 1.0)
    fd = torch.zeros((4, 256), dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        bz.collide_batch_host(m, fd)
    fh = torch.zeros((4, 256), dtype=torch.float32).pin_memory()
    qh = torch.empty_like(fh).pin_memory()            # no host allocation inside the capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(bz.BzError):
        with torch.cuda.graph(g, stream=s):
            bz.collide_batch_host(m, fh, qh, stream=s)
