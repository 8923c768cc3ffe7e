"""Parity of the CUDA IMEX stage/step (Sec. 3.4) with the FP64 oracle."""
import math

import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import AbsModeSum, as_input, bz_module, fp32_cell_bounds, relerr, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bz():
    return bz_module()


@pytest.mark.parametrize("scheme", ["ars222", "bpr343", "euler"])
@pytest.mark.parametrize("model", ["boltzmann", "bgk"])
def test_stages_fp64_match_oracle(bz, scheme, model):
    import oracle
    import torch
    N, L, n = 16, 8.0, 40
    f = workloads.bi_maxwellian(n, 2, N, L, seed=31, noise=0.05)
    k = oracle.Kernel(2, N, L, 1.0)
    dt, eps = 0.02, 0.05
    out_r, Fr, Gr, Pr = k.imex_step(f, dt, eps, scheme=scheme, model=model, stages=True)
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    s = bz.STAGES[scheme]
    fd = to_dev(f, "fp64")
    F = torch.zeros((s, n, N * N), dtype=torch.float64, device="cuda")
    G = torch.zeros_like(F)
    P = torch.zeros_like(F)
    for l in range(1, s + 1):
        bz.imex_stage_local(m, l, fd, F, G, P, dt, eps, scheme=scheme, model=model, precision="fp64")
    bz.check()
    scale = np.abs(f).max()
    for name, a, b in (("F", F, Fr), ("G", G, Gr), ("P", P, Pr)):
        a = a.cpu().numpy()
        assert np.abs(a - b).max() < 1e-12 * max(scale, np.abs(b).max()), name
    fo = bz.imex_step(m, fd, dt, eps, scheme=scheme, model=model, precision="fp64").cpu().numpy()
    assert np.abs(fo - out_r).max() < 1e-12 * scale


def test_transport_residual_and_conserve_fp64(bz):
    import oracle
    N, L, n = 16, 8.0, 33
    f = workloads.bi_maxwellian(n, 2, N, L, seed=32)
    rng = np.random.default_rng(5)
    Lres = 0.01 * rng.normal(size=(3, n, N * N))
    k = oracle.Kernel(2, N, L, 0.0)
    want = k.imex_step(f, 0.01, 0.1, Lres=Lres, conserve=True)
    m = bz.Modes(bz.Grid(2, N, L), 0.0)
    got = bz.imex_step(m, to_dev(f, "fp64"), 0.01, 0.1, L_res=to_dev(Lres, "fp64"), conserve=True,
                       precision="fp64").cpu().numpy()
    assert np.abs(got - want).max() < 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("scheme", ["ars222", "bpr343", "euler"])
def test_stiff_step_fp64_matches_oracle(bz, scheme):
    """dt/eps = 5 (eps = 5e-5): the plain form still reproduces the oracle."""
    import oracle
    N, L, n = 32, 10.0, 20
    f = workloads.bi_maxwellian(n, 2, N, L, seed=34)
    k = oracle.Kernel(2, N, L, 1.0)
    want = k.imex_step(f, 2.5e-4, 5e-5, scheme=scheme)
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    got = bz.imex_step(m, to_dev(f, "fp64"), 2.5e-4, 5e-5, scheme=scheme, precision="fp64").cpu().numpy()
    # rounding re-enters later stages multiplied by dt rho / eps (here ~ 5 rho)
    rho = f.sum(axis=1).max() * (2 * L / N) ** 2
    assert np.abs(got - want).max() < 1e-12 * (1 + 5 * rho) * np.abs(f).max()


@pytest.mark.parametrize("eps", [1.0, 5e-3, 5e-5])
def test_step_fp32_matches_oracle(bz, eps):
    """FP32 form: the error budget is the FP32 rounding of the state (a few u |f|)
    plus the FP32 collision error at the two stage values that enter the step,
    bounded per cell by the rounding count of the operator
    (gpu_util.fp32_cell_bounds, from the oracle's stage values and kernel modes
    only); it enters the later stages through dt G / eps, multiplied by up to
    ~2 dt/eps by the ARS(2,2,2) coefficients and by the implicit BGK factor
    (1 + dt rho / eps)."""
    import oracle
    N, L, n = 32, 10.0, 40
    f = workloads.bi_maxwellian(n, 2, N, L, seed=33)
    dt = 2.5e-4
    fin = as_input(f, "fp32")
    k = oracle.Kernel(2, N, L, 1.0)
    want, F, _, _ = k.imex_step(fin, dt, eps, stages=True)
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    got = bz.imex_step(m, to_dev(f, "fp32"), dt, eps, precision="fp32").double().cpu().numpy()
    A = AbsModeSum(k)
    q_bound = 0.0
    for Fl in F[:2]:
        b2, _ = fp32_cell_bounds(k, A(Fl), k.collide(Fl))
        q_bound = max(q_bound, float(np.linalg.norm(b2)))
    rho = fin.sum(axis=1).max() * (2 * L / N) ** 2
    budget = 8 * 2.0 ** -24 * np.linalg.norm(fin) + 4 * (dt / eps) * (1 + dt * rho / eps) * q_bound
    err = np.linalg.norm(got - want)
    print("fp32 imex eps=%g: err %.3e budget %.3e (rel %.3e)" % (eps, err, budget, err / np.linalg.norm(want)))
    assert err < budget


def test_sod_mesh_step_sampled(bz):
    """~19.6k triangle cells with the density/temperature jump across x = 0.5,
    32^2 grid on [-10,10]^2, hard spheres, eps = 5e-3, dt = h / (2 max|v|):
    one ARS(2,2,2) step in FP32, sampled cells against the oracle."""
    import oracle
    N, L = 32, 10.0
    f, hmesh = workloads.sod_cells(N, L)
    vmax = math.sqrt(2) * L
    dt = 0.5 * hmesh / vmax
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    got = bz.imex_step(m, to_dev(f, "fp32"), dt, 5e-3, precision="fp32").double().cpu().numpy()
    n = f.shape[0]
    idx = np.array([0, 1, n // 3, n // 2, n - 1])
    k = oracle.Kernel(2, N, L, 1.0)
    want = k.imex_step(as_input(f[idx], "fp32"), dt, 5e-3)
    assert relerr(got[idx], want) < 1e-6


def test_penalty_factor_matches_oracle_and_drops_graphs(bz):
    """nu = c rho with c = 3 for the Boltzmann model (bz_modes_set_penalty):
    FP64 stages and step against the oracle with the same c; a step captured in
    a CUDA graph before the change is not replayed with the old rate; the BGK
    model ignores c."""
    import oracle
    import torch
    N, L, n = 16, 8.0, 24
    f = workloads.bi_maxwellian(n, 2, N, L, seed=35, noise=0.05)
    k = oracle.Kernel(2, N, L, 0.0)
    dt, eps = 0.01, 2e-3
    m = bz.Modes(bz.Grid(2, N, L), 0.0)
    fd = to_dev(f, "fp64")
    s = torch.cuda.Stream()
    out = torch.empty_like(fd)
    scale = np.abs(f).max()
    for c in (1.0, 3.0, 1.0):
        m.set_penalty(c)
        want = k.imex_step(f, dt, eps, conserve=True, penalty=c)
        with torch.cuda.stream(s):
            for _ in range(2):                       # capture, then a replay
                out.fill_(float("nan"))
                bz.imex_step(m, fd, dt, eps, f_out=out, conserve=True, precision="fp64", stream=s)
                bz.check(s)
                assert np.abs(out.cpu().numpy() - want).max() < 1e-12 * (1 + dt * c / eps) * scale, c
    m.set_penalty(3.0)
    _, Fr, Gr, Pr = k.imex_step(f, dt, eps, penalty=3.0, stages=True)
    F = torch.zeros((3, n, N * N), dtype=torch.float64, device="cuda")
    G = torch.zeros_like(F)
    P = torch.zeros_like(F)
    for l in (1, 2, 3):
        bz.imex_stage_local(m, l, fd, F, G, P, dt, eps, precision="fp64")
    bz.check()
    for a, b in ((F, Fr), (G, Gr), (P, Pr)):
        assert np.abs(a.cpu().numpy() - b).max() < 1e-12 * (1 + dt * 3 / eps) * max(scale, np.abs(b).max())
    bgk = bz.imex_step(m, fd, dt, eps, model="bgk", precision="fp64").cpu().numpy()
    assert np.abs(bgk - k.imex_step(f, dt, eps, model="bgk")).max() < 1e-12 * (1 + dt / eps) * scale
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(bz.BzError):
            m.set_penalty(bad)


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("scheme", ["ars222", "euler"])
@pytest.mark.parametrize("conserve,with_L", [(False, False), (True, True)])
def test_step_equals_stage_chain(bz, N, scheme, conserve, with_L):
    """imex_step (FP32, 16^2 / 32^2) runs the arithmetic of the per-stage chain
    of imex_stage_local in the same order, so f^{n+1} must equal the chain's
    last stage value bit for bit: on the legacy stream (direct launches), in a
    captured graph and its replay; 70 cells (a ragged tile)."""
    import torch
    L, n = 10.0, 70
    f = to_dev(workloads.bi_maxwellian(n, 2, N, L, seed=40 + N, noise=0.05), "fp32")
    s = bz.STAGES[scheme]
    Lres = None
    if with_L:
        rng = np.random.default_rng(N)
        Lres = to_dev(0.01 * rng.normal(size=(s, n, N * N)), "fp32")
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    dt, eps = 2.5e-4, 5e-3
    F = torch.zeros((s, n, N * N), dtype=torch.float32, device="cuda")
    G = torch.zeros_like(F)
    P = torch.zeros_like(F)
    for l in range(1, s + 1):
        bz.imex_stage_local(m, l, f, F, G, P, dt, eps, scheme=scheme, L_res=Lres, conserve=conserve, precision="fp32")
    bz.check()
    want = F[s - 1].cpu().numpy()
    got = bz.imex_step(m, f, dt, eps, scheme=scheme, L_res=Lres, conserve=conserve, precision="fp32")
    bz.check()
    assert np.array_equal(got.cpu().numpy(), want)
    st = torch.cuda.Stream()
    out = torch.full_like(f, float("nan"))
    with torch.cuda.stream(st):
        for _ in range(2):              # capture, then a replay
            bz.imex_step(m, f, dt, eps, f_out=out, scheme=scheme, L_res=Lres, conserve=conserve, precision="fp32",
                         stream=st)
            bz.check(st)
            assert np.array_equal(out.cpu().numpy(), want)


def test_step_fast_form_equals_stage_chain(bz):
    """The step with the fast (Carleman) operator equals its stage chain."""
    import torch
    N, L, n = 32, 10.0, 40
    f = to_dev(workloads.bi_maxwellian(n, 2, N, L, seed=48), "fp32")
    m = bz.FastModes(bz.Grid(2, N, L), 8)
    F = torch.zeros((3, n, N * N), dtype=torch.float32, device="cuda")
    G = torch.zeros_like(F)
    P = torch.zeros_like(F)
    for l in (1, 2, 3):
        bz.imex_stage_local(m, l, f, F, G, P, 2.5e-4, 5e-3, precision="fp32")
    got = bz.imex_step(m, f, 2.5e-4, 5e-3, precision="fp32")
    bz.check()
    assert np.array_equal(got.cpu().numpy(), F[2].cpu().numpy())
