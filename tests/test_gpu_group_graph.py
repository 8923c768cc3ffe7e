"""Grouped heterogeneous launch (group_collide) and the graph-captured IMEX
step: both must reproduce the per-instance / direct-launch results."""
import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import as_input, bz_module, relerr, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bz():
    return bz_module()


def _instances():
    # (dim, N, L, n_cells): 2-D grids of every size class, a ragged tail, a
    # grid above the register-blocked limit (48) and a 3-D grid
    return [(2, 16, 8.0, 300), (2, 24, 10.0, 45), (2, 32, 10.0, 97), (2, 48, 10.0, 5), (3, 8, 8.0, 33),
            (2, 32, 10.0, 1)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_group_collide_matches_per_instance(bz, precision):
    import torch
    entries, refs = [], []
    for i, (dim, N, L, n) in enumerate(_instances()):
        m = bz.Modes(bz.Grid(dim, N, L), 1.0)
        f = to_dev(workloads.bi_maxwellian(n, dim, N, L, seed=60 + i), precision)
        refs.append(bz.collide_batch(m, f, precision=precision).cpu().numpy())
        entries.append((m, f, torch.full_like(f, float("nan"))))
    bz.group_collide(entries, precision=precision)
    bz.check()
    for (m, f, Q), ref in zip(entries, refs):
        got = Q.cpu().numpy()
        assert np.array_equal(got, ref)            # same kernels, same arithmetic


def test_group_collide_mixed_variants(bz, monkeypatch):
    """Instances on different register-blocked variants in one call (one grouped
    launch per variant), results equal to per-instance calls."""
    import torch
    entries, refs = [], []
    for i, (d, N, var, n) in enumerate([(2, 32, 1, 80), (2, 24, 2, 50), (2, 32, 3, 33), (2, 16, 1, 70),
                                        (2, 48, 3, 21), (2, 24, 3, 40), (3, 16, 4, 11), (2, 16, 4, 9),
                                        (2, 32, 5, 45), (2, 24, 5, 70), (2, 32, 6, 45), (2, 24, 6, 70),
                                        (2, 16, 6, 33), (2, 32, 7, 40), (3, 8, 7, 20), (2, 48, 8, 21),
                                        (2, 32, 8, 40), (2, 32, 9, 37), (2, 48, 9, 19), (2, 32, 10, 39),
                                        (2, 48, 10, 23), (2, 16, 10, 41)]):
        monkeypatch.setenv("BZ_MODESUM_VARIANT", str(var))
        m = bz.Modes(bz.Grid(d, N, 10.0), 1.0)
        assert m.modesum_variant == var
        f = to_dev(workloads.bi_maxwellian(n, d, N, 10.0, seed=90 + i), "fp32")
        refs.append(bz.collide_batch(m, f, precision="fp32").cpu().numpy())
        entries.append((m, f, torch.full_like(f, float("nan"))))
    bz.group_collide(entries, precision="fp32")
    bz.check()
    for (m, f, Q), ref in zip(entries, refs):
        assert np.array_equal(Q.cpu().numpy(), ref)


def test_group_collide_matches_oracle(bz):
    import oracle
    dim, N, L, n = 2, 24, 10.0, 40
    m = bz.Modes(bz.Grid(dim, N, L), 1.0)
    f = workloads.bi_maxwellian(n, dim, N, L, seed=70)
    Q = to_dev(np.zeros_like(f), "fp32")
    bz.group_collide([(m, to_dev(f, "fp32"), Q)], precision="fp32")
    want = oracle.Kernel(dim, N, L, 1.0).collide(as_input(f, "fp32"))
    assert relerr(Q.double().cpu().numpy(), want) < 1e-5


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_graph_step_equals_direct_launches(bz, precision):
    import torch
    N, L, n = 32, 10.0, 70
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    f = to_dev(workloads.bi_maxwellian(n, 2, N, L, seed=71), precision)
    direct = bz.imex_step(m, f, 2.5e-4, 5e-3, precision=precision)       # legacy stream: direct launches
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    out = torch.empty_like(f)
    with torch.cuda.stream(s):
        for _ in range(3):                                               # capture, then two replays
            out.fill_(float("nan"))
            bz.imex_step(m, f, 2.5e-4, 5e-3, f_out=out, precision=precision, stream=s)
            bz.check(s)
            assert torch.equal(out, direct)
    # a different dt is a different graph
    with torch.cuda.stream(s):
        o2 = bz.imex_step(m, f, 1e-4, 5e-3, precision=precision, stream=s)
        bz.check(s)
    d2 = bz.imex_step(m, f, 1e-4, 5e-3, precision=precision)
    torch.cuda.synchronize()
    assert torch.equal(o2, d2)
