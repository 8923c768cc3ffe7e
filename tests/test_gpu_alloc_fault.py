"""Host-side allocation failure injection (bz_inject_alloc_failure).

Every entry point that takes device memory is run with its k-th allocation
failing, k = 0, 1, 2, ... until an attempt meets no failure.  Each failing
attempt must return BZ_ENOMEM, hand back everything it took (the library's
live blocks and pool bytes equal their values before the attempt once the
device is idle), and leave every handle usable: the attempt that finally
succeeds gives the result of a call made without injection, bit for bit.  The
failure is made on the host (the allocation is not attempted); no GPU fault is
involved."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import bz_module, to_dev

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bz():
    return bz_module()


def _idle():
    import torch
    torch.cuda.synchronize()


def _sweep(bz, call, limit=200):
    """Run call() with the k-th allocation failing for k = 0, 1, ...; returns
    (number of allocations the call makes, result of the first clean run)."""
    for k in range(limit):
        _idle()
        base = bz.alloc_stats()
        bz.inject_alloc_failure(k)
        try:
            out = call()
        except bz.BzError as e:
            bz.inject_alloc_failure(None)
            assert e.code == bz.ENOMEM, (k, e.code, str(e))
            _idle()
            assert bz.alloc_stats() == base, ("attempt %d kept memory" % k, base, bz.alloc_stats())
            continue
        bz.inject_alloc_failure(None)
        bz.check()
        return k, out
    raise AssertionError("no clean run within %d allocations" % limit)


def _f(n, N=32, seed=5, precision="fp32"):
    return to_dev(workloads.bi_maxwellian(n, 2, N, 10.0, seed=seed), precision)


def test_handles(bz):
    """init_velocity_grid, build_kernel_modes (variant tables, split tables,
    FP64 tables; on a 28^2 grid the autotuner's timing batch too, the first
    time that grid is tuned in the process), build_fast_modes: each failing
    attempt frees its partial tables; the handle of the clean run computes what
    a handle built without injection computes."""
    import gc
    import torch
    bz.check()                                       # the error word exists from here on
    gc.collect()                                     # handles that earlier tests dropped are freed first
    _idle()
    live0 = bz.alloc_stats()[0]
    ng, g = _sweep(bz, lambda: bz.Grid(2, 28, 10.0))
    assert ng == 2                                   # the FP64 and FP32 DFT tables
    nm, m = _sweep(bz, lambda: bz.Modes(g, 1.0))
    assert nm >= 6
    g24 = bz.Grid(2, 24, 10.0)
    nf, fm = _sweep(bz, lambda: bz.FastModes(g24, 8))
    assert nf >= 2
    f, f24 = _f(100, N=28, seed=7), _f(100, N=24, seed=8)
    got = [bz.collide_batch(m, f), bz.collide_batch(fm, f24)]
    want = [bz.collide_batch(bz.Modes(bz.Grid(2, 28, 10.0), 1.0), f),
            bz.collide_batch(bz.FastModes(bz.Grid(2, 24, 10.0), 8), f24)]
    bz.check()
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    print("allocations: grid %d, modes %d, fast modes %d" % (ng, nm, nf))
    del m, fm, g, g24
    gc.collect()
    _idle()
    assert bz.alloc_stats()[0] == live0


@pytest.mark.parametrize("precision,conserve", [("fp32", False), ("fp64", True), ("fp32x2", False)])
def test_collide_batch(bz, precision, conserve):
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    f = _f(333, precision="fp64" if precision == "fp64" else "fp32")
    want = bz.collide_batch(m, f, precision=precision, conserve=conserve)
    n, got = _sweep(bz, lambda: bz.collide_batch(m, f, precision=precision, conserve=conserve))
    assert n == 1                                    # one scratch block per call
    assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())


def test_collide_batch_host(bz):
    """One block for both pipeline slots (f, Q and the Fourier scratch of a
    chunk each), taken before anything is queued; a batch of several chunks."""
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    f = workloads.bi_maxwellian(20000, 2, 32, 10.0, seed=9).astype(np.float32)
    want = bz.collide_batch_host(m, f)
    bz.check()
    n, got = _sweep(bz, lambda: bz.collide_batch_host(m, f))
    assert n == 1
    assert np.array_equal(got, want)


def test_group_collide(bz):
    import torch
    items = []
    for (d, N, n) in ((2, 16, 40), (2, 32, 70), (3, 8, 9)):
        m = bz.Modes(bz.Grid(d, N, 10.0), 1.0)
        f = to_dev(workloads.bi_maxwellian(n, d, N, 10.0, seed=N), "fp32")
        items.append((m, f, bz.collide_batch(m, f)))

    def run():
        entries = [(m, f, torch.full_like(f, float("nan"))) for m, f, _ in items]
        bz.group_collide(entries)
        return entries
    n, entries = _sweep(bz, run)
    assert n == 1
    for (_, _, Q), (_, _, want) in zip(entries, items):
        assert torch.equal(Q, want)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_imex_step_direct_and_graph(bz, precision):
    """The legacy stream (pool scratch) and a side stream (the cached graph's
    scratch block: a failing capture keeps nothing; the clean run adds one
    cached graph)."""
    import torch
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    f = _f(90, seed=11, precision=precision)
    want = bz.imex_step(m, f, 2.5e-4, 5e-3, precision=precision)
    n, got = _sweep(bz, lambda: bz.imex_step(m, f, 2.5e-4, 5e-3, precision=precision))
    assert n == 1
    assert torch.equal(got, want)
    s = torch.cuda.Stream()
    dt = 1.25e-4                                     # a graph not cached by any earlier call
    want = bz.imex_step(m, f, dt, 5e-3, precision=precision)

    def side():
        with torch.cuda.stream(s):
            out = bz.imex_step(m, f, dt, 5e-3, precision=precision, stream=s)
            s.synchronize()
            return out
    n, got = _sweep(bz, side)
    assert n == 1
    assert torch.equal(got, want)


def _square(n_side, seed=3):
    pts, tri = workloads.sod_triangulation(n_side, seed)
    cnt = {}
    for t in tri:
        for q in range(3):
            e = tuple(sorted((int(t[q]), int(t[(q + 1) % 3]))))
            cnt[e] = cnt.get(e, 0) + 1
    edges = np.array([e for e, c in cnt.items() if c == 1], dtype=np.int64)
    params = np.tile([1.1, 0.1, -0.1], (len(edges), 1))
    return pts, tri, edges, params


def test_mesh_transport_and_fv_step(bz):
    """build_fv_mesh (orders 2 and 3), fv_mesh_set_walls (a failing call keeps
    the mesh's walls off), transport_residual and imex_step_fv."""
    import torch
    pts, tri, edges, params = _square(10)
    for order in (2, 3):
        n, mesh = _sweep(bz, lambda: bz.Mesh(pts, tri, order=order))
        assert n >= 9
        ref = bz.Mesh(pts, tri, order=order)
        ref.set_walls(edges, params)
        n, _ = _sweep(bz, lambda: mesh.set_walls(edges, params))
        assert n == 3
        g = bz.Grid(2, 16, 8.0)
        f = to_dev(workloads.mesh_states(pts[tri].mean(axis=1), 16, 8.0, jump=True), "fp32")
        want = bz.transport_residual(ref, g, f)
        n, got = _sweep(bz, lambda: bz.transport_residual(mesh, g, f))
        assert torch.equal(got, want)
    m = bz.Modes(g, 0.0)
    want = bz.imex_step_fv(m, ref, f, 1e-3, 1e-2)
    n, got = _sweep(bz, lambda: bz.imex_step_fv(m, mesh, f, 1e-3, 1e-2))
    assert n == 1
    assert torch.equal(got, want)


_ERROR_WORD_CHILD = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2103_14890_gb300 import binding as bz
torch.zeros(1, device="cuda")
bz.inject_alloc_failure(0)
try:
    bz.check()
    print("no failure")
    sys.exit(1)
except bz.BzError as e:
    assert e.code == bz.ENOMEM, e.code
bz.inject_alloc_failure(None)
m = bz.Modes(bz.Grid(2, 16, 8.0), 1.0)
f = torch.rand(5, 256, device="cuda")
bz.collide_batch(m, f, check_input=True)
bz.check()
print("ok")
"""


def test_error_word_first_use():
    """The device error word is allocated on first use (once per device and
    process), so a fresh process: bz_check meeting the failure returns
    BZ_ENOMEM, and the next call allocates it and works."""
    r = subprocess.run([sys.executable, "-c", _ERROR_WORD_CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
