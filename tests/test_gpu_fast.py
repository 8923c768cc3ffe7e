"""Parity of the CUDA fast spectral form (Sec. 3.3, Carleman representation,
eq. ode with the direction decomposition of eq. FKM) with the FP64 oracle's
fast kernel modes, through the C ABI.

The CUDA path evaluates eq. ode by FFT convolutions on a zero-padded grid;
the oracle sums eq. ode pair by pair with the same direction factors, so the
two share nothing but the definition.  FP64: <= 1e-12 relative L2.

FP32 budget.  The FFT pipeline rounds relative to the size of the gain and
loss terms it carries, not to their difference Q, so the FP32 error is
bounded on the loss scale: with u = 2^-24, the forward DFT of f (log2 N^2 = 10
stages), the direction factor (2 roundings), the inverse P x P transform
(log2 P^2 <= 11.2 stages), the product and the sum over A + 1 terms, the
forward P x P transform of the sum and the inverse DFT to the grid add up to
about 54 u normwise for A = 8, so the test bound is
  ||Q_32 - Q_64|| <= 64 u ||nu f||,   nu = 2 pi b0 rho (the loss frequency),
which the relative error ||Q_32 - Q_64|| / ||Q_64|| exceeds only by the
cancellation factor ||nu f|| / ||Q_64|| of the input.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import as_input, bz_module, relerr, to_dev

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_LOSS = 64 * 2.0 ** -24
L = 10.0


def loss_scaled(Q, Qr, f, N, Lb=L):
    """||Q - Qr|| / ||nu f|| with nu = rho for b0 = 1/(2 pi) (rho = sum f dv^2)."""
    f = np.asarray(f, dtype=np.float64).reshape(Qr.shape)
    rho = f.sum(axis=1) * (2 * Lb / N) ** 2
    return float(np.linalg.norm(Q - Qr) / np.linalg.norm(rho[:, None] * f))


@pytest.fixture(scope="module")
def bz():
    return bz_module()


@pytest.fixture(scope="module")
def okf():
    import oracle
    cache = {}

    def get(N, ndirs, Lb=L):
        key = (N, ndirs, Lb)
        if key not in cache:
            cache[key] = oracle.FastKernel(N, Lb, ndirs)
        return cache[key]
    return get


def _modes(bz, N, ndirs, Lb=L):
    return bz.FastModes(bz.Grid(2, N, Lb), ndirs)


@pytest.mark.parametrize("N,ndirs", [(8, 1), (8, 3), (16, 8)])
def test_fast_weights_match_oracle(bz, okf, N, ndirs):
    m = _modes(bz, N, ndirs)
    assert (m.method, m.ndirs) == (1, ndirs)
    got = m.beta_table()
    want = okf(N, ndirs).beta_table()
    mask = got != 0
    assert np.abs(got - want)[mask].max() < 1e-13 * np.abs(want).max()


def test_fast_shapes(bz):
    """Padded length P >= 3h + 1 (no aliasing into K_h); C * P = 96 threads per
    CTA, 144 for the P = 72 of 48^2."""
    for N, P in [(8, 12), (16, 24), (24, 48), (32, 48), (48, 72)]:
        m = _modes(bz, N, 4)
        assert m.pad == P and P >= 3 * (N // 2 - 1) + 1
        assert m.fast_cells * m.pad == (96 if P <= 48 else 144)


@pytest.mark.parametrize("N,ndirs,n", [(8, 1, 70), (16, 4, 70), (24, 8, 37), (32, 8, 70), (32, 3, 5),
                                       (48, 8, 3), (48, 5, 2)])
def test_fast_fp64_matches_oracle(bz, okf, N, ndirs, n):
    f = workloads.bi_maxwellian(n, 2, N, L, seed=2100 + N + ndirs)
    m = _modes(bz, N, ndirs)
    Q = bz.collide_batch(m, to_dev(f, "fp64"), precision="fp64")
    bz.check()
    Qr = okf(N, ndirs).collide(f)
    assert relerr(Q.cpu().numpy(), Qr) < TOL64


@pytest.mark.parametrize("N,ndirs,n", [(8, 2, 70), (16, 8, 70), (24, 8, 37), (32, 8, 70), (32, 16, 33),
                                       (48, 8, 5)])
def test_fast_fp32_matches_oracle(bz, okf, N, ndirs, n):
    f = workloads.shifted_maxwellians(n, 2, N, L, seed=2200 + N + ndirs)
    m = _modes(bz, N, ndirs)
    Q = bz.collide_batch(m, to_dev(f, "fp32"), precision="fp32")
    bz.check()
    fin = as_input(f, "fp32")
    Qr = okf(N, ndirs).collide(fin)
    assert loss_scaled(Q.double().cpu().numpy(), Qr, fin, N) < TOL32_LOSS


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fast_edge_sizes(bz, okf, precision):
    """No cells, one cell, one short of a CTA pair, a ragged 32-cell tile."""
    m = _modes(bz, 32, 8)
    for n in (0, 1, 3, 33):
        f = workloads.bi_maxwellian(max(n, 1), 2, 32, L, seed=2300 + n)[:n]
        Q = bz.collide_batch(m, to_dev(f, precision), precision=precision)
        bz.check()
        assert Q.shape == (n, 32 * 32)
        if n:
            fin = as_input(f, precision)
            Qr = okf(32, 8).collide(fin)
            if precision == "fp64":
                assert relerr(Q.cpu().numpy(), Qr) < TOL64
            else:
                assert loss_scaled(Q.double().cpu().numpy(), Qr, fin, 32) < TOL32_LOSS


def test_fast_conservation_fix(bz, okf):
    f = workloads.bi_maxwellian(20, 2, 16, L, seed=2400)
    m = _modes(bz, 16, 8)
    Q = bz.collide_batch(m, to_dev(f, "fp64"), precision="fp64", conserve=True)
    bz.check()
    Qr = okf(16, 8).collide(f, conserve=True)
    assert relerr(Q.cpu().numpy(), Qr) < TOL64


def test_fast_deterministic_and_mass_conserving(bz):
    import torch
    m = _modes(bz, 32, 8)
    f = to_dev(workloads.shifted_maxwellians(300, 2, 32, L, seed=2500), "fp32")
    Q1 = bz.collide_batch(m, f, precision="fp32")
    Q2 = bz.collide_batch(m, f, precision="fp32")
    bz.check()
    assert torch.equal(Q1, Q2)
    mass = Q1.double().sum(dim=1).abs()
    assert float(mass.max()) < 1e-5 * float(Q1.double().abs().sum(dim=1).max())


def test_fast_imex_step_matches_oracle(bz, okf):
    """One ARS(2,2,2) step of the penalised IMEX scheme with the fast operator."""
    N, ndirs, n = 16, 8, 20
    f = workloads.bi_maxwellian(n, 2, N, L, seed=2600)
    m = _modes(bz, N, ndirs)
    out = bz.imex_step(m, to_dev(f, "fp64"), 1e-3, 5e-3, precision="fp64")
    bz.check()
    want = okf(N, ndirs).imex_step(f, 1e-3, 5e-3)
    assert relerr(out.cpu().numpy(), want) < TOL64


@pytest.mark.parametrize("eps", [1.0, 5e-3])
def test_fast_imex_step_fp32_within_budget(bz, okf, eps):
    """FP32 step with the fast operator: the FP32 rounding of the state plus the
    FP32 collision error entering every stage through dt G / eps (amplified by at
    most ~2 dt/eps (1 + dt rho / eps) by the ARS(2,2,2) coefficients)."""
    N, ndirs, n, dt = 32, 8, 40, 2.5e-4
    f = workloads.bi_maxwellian(n, 2, N, L, seed=2650)
    fin = as_input(f, "fp32")
    k = okf(N, ndirs)
    want = k.imex_step(fin, dt, eps)
    m = _modes(bz, N, ndirs)
    got = bz.imex_step(m, to_dev(f, "fp32"), dt, eps, precision="fp32").double().cpu().numpy()
    q_err = np.linalg.norm(bz.collide_batch(m, to_dev(f, "fp32"), precision="fp32").double().cpu().numpy()
                           - k.collide(fin))
    bz.check()
    rho = fin.sum(axis=1).max() * (2 * L / N) ** 2
    budget = 8 * 2.0 ** -24 * np.linalg.norm(fin) + 4 * (dt / eps) * (1 + dt * rho / eps) * q_err
    assert np.linalg.norm(got - want) < budget


def test_fast_group_noalloc_and_host_paths_agree(bz):
    """A fast instance inside group_collide (next to a direct one), the
    allocation-free entry and the host pipeline all give collide_batch's bits."""
    import torch
    mf = _modes(bz, 32, 8)
    md = bz.Modes(bz.Grid(2, 16, L), 1.0)
    ff = to_dev(workloads.shifted_maxwellians(90, 2, 32, L, seed=2700), "fp32")
    fd = to_dev(workloads.bi_maxwellian(40, 2, 16, L, seed=2701), "fp32")
    Qf = bz.collide_batch(mf, ff, precision="fp32")
    Qd = bz.collide_batch(md, fd, precision="fp32")
    Gf, Gd = torch.empty_like(ff), torch.empty_like(fd)
    bz.group_collide([(mf, ff, Gf), (md, fd, Gd)], precision="fp32")
    Qn = bz.collide_batch_noalloc(mf, ff, precision="fp32")
    Qh = bz.collide_batch_host(mf, ff.cpu(), precision="fp32")
    bz.check()
    assert torch.equal(Gf, Qf) and torch.equal(Gd, Qd)
    assert torch.equal(Qn, Qf)
    assert torch.equal(Qh, Qf.cpu())


def test_fast_full_size_fp32_sampled(bz, okf):
    """65536 cells in one launch (the measured configuration): sampled cells
    against the oracle."""
    n, N, ndirs = 65536, 32, 8
    f = workloads.shifted_maxwellians(n, 2, N, L, seed=2800)
    m = _modes(bz, N, ndirs)
    Q = bz.collide_batch(m, to_dev(f, "fp32"), precision="fp32")
    bz.check()
    idx = np.random.default_rng(2801).choice(n, 24, replace=False)
    idx = np.concatenate([idx, [0, 1, n - 2, n - 1]])
    fin = as_input(f[idx], "fp32")
    Qr = okf(N, ndirs).collide(fin)
    assert loss_scaled(Q.double().cpu().numpy()[idx], Qr, fin, N) < TOL32_LOSS


def test_fast_argument_errors(bz):
    lib = bz.load()
    out = ctypes.c_void_p()
    g3 = bz.Grid(3, 8, L)
    assert lib.build_fast_modes(g3._h, 0.0, 8, ctypes.byref(out)) == bz.ENOTSUP
    g64 = bz.Grid(2, 64, L)
    assert lib.build_fast_modes(g64._h, 0.0, 8, ctypes.byref(out)) == bz.ENOTSUP
    g12 = bz.Grid(2, 12, L)
    assert lib.build_fast_modes(g12._h, 0.0, 8, ctypes.byref(out)) == bz.ENOTSUP
    g = bz.Grid(2, 32, L)
    assert lib.build_fast_modes(g._h, 0.0, 0, ctypes.byref(out)) == bz.EINVAL
    assert lib.build_fast_modes(g._h, 0.0, 8, None) == bz.EINVAL
    md = bz.Modes(bz.Grid(2, 16, L), 1.0)
    assert (md.method, md.ndirs, md.pad) == (0, 0, 0)
