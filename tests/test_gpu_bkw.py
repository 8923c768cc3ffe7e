"""The homogeneous BKW relaxation (Sec. 4.1) marched with the CUDA operator.

The closed-form BKW solution of the space-homogeneous equation for 2-D Maxwell
molecules, f(t, v) = exp(-|v|^2 / (2S)) / (2 pi S^2) (2S - 1 + (1 - S) |v|^2 /
(2S)), S = 1 - exp(-t/8)/2, is integrated from t = 0 to t = 1 with dt = 0.01
by classic RK4 (the time integrator the paper leaves unstated) with every
Q(f, f) evaluated by collide_batch through the C ABI, in FP64 and FP32, on the
16^2 grid of [-8,8]^2 (the small configuration) and on a 32^2 grid:

  * against the oracle's own RK4 run with the FP64 oracle operator: element by
    element to 1e-12 in FP64; in FP32 within the bound derived from the
    rounding count (per evaluation the FP32 operator bound of gpu_util, plus
    the FP32 rounding of the RK4 combinations, amplified by at most e^(2t)
    over the march: the linearised operator of Maxwell molecules has rate
    at most 2 rho = 2 here);
  * against the closed form: the same error the oracle reaches (the spectral
    and time error of the discretisation, not of the arithmetic).

ARS(2,2,2) with eps = 1 on the same problem converges at second order in time
on the GPU (self-convergence under dt halving)."""
import math
import os
import sys

import numpy as np
import pytest

from gpu_util import U32, AbsModeSum, bz_module, fp32_cell_bounds, to_dev

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_oracle_collision import _bkw  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bz():
    return bz_module()


def _r2(k):
    v = k.velocities()
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    return (V1 ** 2 + V2 ** 2).ravel()


def _rk4_oracle(k, f, dt, steps, scale_fn=None):
    """Oracle RK4; scale_fn(state) is called on every state the operator sees."""
    for _ in range(steps):
        k1 = k.collide(f)
        if scale_fn:
            scale_fn(f, k1)
        y = f + 0.5 * dt * k1
        k2 = k.collide(y)
        if scale_fn:
            scale_fn(y, k2)
        y = f + 0.5 * dt * k2
        k3 = k.collide(y)
        if scale_fn:
            scale_fn(y, k3)
        y = f + dt * k3
        k4 = k.collide(y)
        if scale_fn:
            scale_fn(y, k4)
        f = f + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return f


def _rk4_gpu(bz, m, f, dt, steps, precision):
    for _ in range(steps):
        k1 = bz.collide_batch(m, f, precision=precision)
        k2 = bz.collide_batch(m, f + 0.5 * dt * k1, precision=precision)
        k3 = bz.collide_batch(m, f + 0.5 * dt * k2, precision=precision)
        k4 = bz.collide_batch(m, f + dt * k3, precision=precision)
        f = f + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    bz.check()
    return f


@pytest.mark.parametrize("N,L", [(16, 8.0), (32, 8.0)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bkw_rk4_to_t1(bz, N, L, precision):
    import oracle
    dt, steps = 0.01, 100
    k = oracle.Kernel(2, N, L, 0.0)
    r2 = _r2(k)
    f0 = _bkw(r2, 0.0)[None]
    f0_in = f0 if precision == "fp64" else f0.astype(np.float32).astype(np.float64)
    # the oracle's march, with the FP32 error scale of every evaluation
    A = AbsModeSum(k)
    per_eval = []

    def scale(y, q):
        b2, _ = fp32_cell_bounds(k, A(y), q)
        per_eval.append(float(b2[0]))
    want = _rk4_oracle(k, f0_in, dt, steps, scale if precision == "fp32" else None)
    m = bz.Modes(bz.Grid(2, N, L), 0.0)
    got = _rk4_gpu(bz, m, to_dev(f0, precision), dt, steps, precision).double().cpu().numpy()
    exact = _bkw(r2, 1.0)
    e_or = np.abs(want[0] - exact).sum() / np.abs(exact).sum()
    e_gpu = np.abs(got[0] - exact).sum() / np.abs(exact).sum()
    diff = np.abs(got - want).max()
    print("BKW %s N=%d: L1 vs closed form gpu %.4e oracle %.4e; max |gpu - oracle| %.3e"
          % (precision, N, e_gpu, e_or, diff))
    if precision == "fp64":
        assert diff < 1e-12 * np.abs(want).max()
    else:
        # per step: dt/6 (b1 + 2 b2 + 2 b3 + b4) <= dt max b, plus ~8 FP32
        # roundings of the state in the stage and step combinations
        b = np.array(per_eval).reshape(steps, 4).max(axis=1)
        budget = math.exp(2.0 * dt * steps) * (dt * b.sum() + 8 * steps * U32 * np.linalg.norm(want))
        assert np.linalg.norm(got - want) < budget, (np.linalg.norm(got - want), budget)
    # the discretisation error against the closed form is the oracle's
    assert abs(e_gpu - e_or) < (1e-9 * e_or if precision == "fp64" else 1e-2 * e_or + 1e-5)
    assert e_gpu < (0.3 if N == 16 else 2e-3)


def test_bkw_ars222_second_order_in_time(bz):
    """ARS(2,2,2), eps = 1, Boltzmann model (BGK penalty implicit), FP64:
    f(t = 0.8) at dt = 0.2, 0.1, 0.05, 0.025, 0.0125; the differences of
    successive runs shrink by a factor approaching 4 (second order).  The
    dt = 0.1 march also equals the oracle's step by step to 1e-12."""
    import oracle
    N, L = 32, 8.0
    k = oracle.Kernel(2, N, L, 0.0)
    r2 = _r2(k)
    f0 = _bkw(r2, 0.0)[None]
    m = bz.Modes(bz.Grid(2, N, L), 0.0)

    def march(dt):
        f = to_dev(f0, "fp64")
        for _ in range(int(round(0.8 / dt))):
            f = bz.imex_step(m, f, dt, 1.0, precision="fp64")
        bz.check()
        return f.cpu().numpy()
    runs = [march(dt) for dt in (0.2, 0.1, 0.05, 0.025, 0.0125)]
    diffs = [np.linalg.norm(runs[i] - runs[i + 1]) for i in range(4)]
    ratios = [diffs[i] / diffs[i + 1] for i in range(3)]
    print("ARS(2,2,2) BKW successive differences", diffs, "ratios", ratios)
    assert all(3.5 < r < 4.5 for r in ratios[1:]), ratios
    fo = f0
    for _ in range(8):
        fo = k.imex_step(fo, 0.1, 1.0)
    assert np.abs(march(0.1) - fo).max() < 1e-12 * np.abs(f0).max()
