"""Pins for the oracle's penalised IMEX step (Sec. 3.4).

- BGK-only model: the step is the implicit Runge-Kutta method applied to the
  linear relaxation, so f^{n+1} - M = R(z) (f^n - M) with z = -dt rho/eps and
  R the stability function of the implicit tableau (closed form for ARS(2,2,2)
  and for IMEX Euler, R(z) = 1/(1 - z); numpy linear algebra for BPR(3,4,3);
  tableaux typed from the paper);
- Boltzmann model: moments are conserved by the step when Q is conserving;
  the stiff limit keeps a Maxwellian a Maxwellian (asymptotic preservation);
  the global error falls at the order of the scheme.
"""
import math

import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads

G = 1.0 - 1.0 / math.sqrt(2.0)


def _A_impl(scheme):
    if scheme == "euler":
        return np.array([[0, 0], [0, 1]], float)
    if scheme == "ars222":
        return np.array([[0, 0, 0], [0, G, 0], [0, 1 - G, G]], float)
    return np.array([[0, 0, 0, 0, 0],
                     [1 / 2, 1 / 2, 0, 0, 0],
                     [5 / 18, -1 / 9, 1 / 2, 0, 0],
                     [1 / 2, 0, 0, 1 / 2, 0],
                     [1 / 4, 0, 3 / 4, -1 / 2, 1 / 2]], float)


def _stability(scheme, z):
    A = _A_impl(scheme)
    s = A.shape[0]
    e = np.zeros(s)
    e[-1] = 1.0                                  # stiffly accurate: last row = weights
    return e @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


def test_ars_closed_form_matches_linear_algebra():
    for z in (-0.1, -3.0, -1e4):
        closed = (1 + (1 - 2 * G) * z) / (1 - G * z) ** 2
        assert abs(closed - _stability("ars222", z)) < 1e-14 * max(1, abs(closed))
        assert abs(1 / (1 - z) - _stability("euler", z)) < 1e-15


def test_euler_bgk_step_closed_form(oracle_mod):
    """IMEX Euler on the BGK model: f^{n+1} = (f^n + c M)/(1 + c), c = dt rho/eps,
    with M the Maxwellian of f^n (backward Euler of the linear relaxation)."""
    k = oracle_mod.Kernel(2, 16, 8.0, 0.0)
    f = workloads.bi_maxwellian(2, 2, 16, 8.0, seed=24)
    dt, eps = 0.03, 0.01
    out = k.imex_step(f, dt, eps, scheme="euler", model="bgk")
    for fn, fo in zip(f, out):
        U = k.moments(fn)
        c = dt * U[0] / eps
        want = (fn + c * k.maxwellian(U).ravel()) / (1 + c)
        assert np.abs(fo - want).max() < 1e-14 * np.abs(fn).max()


def test_euler_boltzmann_step_is_explicit_plus_penalty(oracle_mod):
    """IMEX Euler on the Boltzmann model, written out: G = Q(f) - rho (M - f),
    R = f + dt G/eps, then the backward-Euler penalty with the moments of R."""
    k = oracle_mod.Kernel(2, 16, 8.0, 1.0)
    f = workloads.bi_maxwellian(2, 2, 16, 8.0, seed=25)
    dt, eps = 0.02, 0.1
    out = k.imex_step(f, dt, eps, scheme="euler")
    Q = k.collide(f)
    for i, fn in enumerate(f):
        U = k.moments(fn)
        G1 = Q[i] - U[0] * (k.maxwellian(U).ravel() - fn)
        R = fn + dt * G1 / eps
        U2 = k.moments(R)
        c = dt * U2[0] / eps
        want = (R + c * k.maxwellian(U2).ravel()) / (1 + c)
        assert np.abs(out[i] - want).max() < 1e-13 * np.abs(fn).max()


@pytest.mark.parametrize("scheme", ["ars222", "bpr343", "euler"])
@pytest.mark.parametrize("dt_over_eps", [0.05, 1.0, 40.0, 1e6])
def test_bgk_model_amplification(oracle_mod, scheme, dt_over_eps):
    N, L = 32, 10.0
    k = oracle_mod.Kernel(2, N, L, 1.0)
    f = workloads.bi_maxwellian(3, 2, N, L, seed=21)
    eps = 1e-2
    dt = dt_over_eps * eps
    out = k.imex_step(f, dt, eps, scheme=scheme, model="bgk")
    for fn, fo in zip(f, out):
        U = k.moments(fn)
        M = k.maxwellian(U).ravel()
        z = -dt * U[0] / eps
        want = M + _stability(scheme, z) * (fn - M)
        # rounding of a stage value is multiplied by |z| when it re-enters the
        # next stage through dt * P / eps, so the bound grows with |z|
        tol = max(1e-13, 5e-15 * (1 + abs(z))) * np.abs(fn).max()
        assert np.abs(fo - want).max() < tol


def test_bgk_stage_outputs(oracle_mod):
    """BGK model: G = 0 in every stage and P_l = rho (M - F_l)."""
    k = oracle_mod.Kernel(2, 16, 8.0, 0.0)
    f = workloads.bi_maxwellian(2, 2, 16, 8.0, seed=22)
    out, F, Gs, P = k.imex_step(f, 0.01, 0.01, model="bgk", stages=True)
    assert np.all(Gs == 0)
    assert np.array_equal(F[0], f)
    assert np.array_equal(out, F[-1])
    for c in range(2):
        U = k.moments(f[c])
        M = k.maxwellian(U).ravel()
        assert np.abs(P[0, c] - U[0] * (M - f[c])).max() < 1e-14 * np.abs(f[c]).max()


@pytest.mark.parametrize("scheme", ["ars222", "bpr343"])
def test_boltzmann_step_conserves_moments(oracle_mod, scheme):
    k = oracle_mod.Kernel(2, 32, 10.0, 1.0)
    f = workloads.bi_maxwellian(2, 2, 32, 10.0, seed=23)
    out = k.imex_step(f, 0.02, 0.05, scheme=scheme, conserve=True)
    for fn, fo in zip(f, out):
        Un, Uo = k.moments(fn), k.moments(fo)
        assert np.abs(Un - Uo).max() < 1e-12 * np.abs(Un).max()
        assert np.linalg.norm(fo - fn) > 1e-3 * np.linalg.norm(fn)     # it did relax


@pytest.mark.parametrize("scheme", ["ars222", "bpr343"])
def test_stiff_limit_keeps_maxwellian(oracle_mod, scheme):
    """Asymptotic preservation: with eps -> 0 a (well-prepared) Maxwellian stays
    the Maxwellian of its moments, to the level of Q(M) on the grid."""
    N, L = 32, 8.0
    k = oracle_mod.Kernel(2, N, L, 1.0)
    M = k.maxwellian(np.array([1.3, 1.3 * 0.3, -1.3 * 0.2, 0.5 * 1.3 * (2 * 0.9 + 0.13)])).ravel()
    want = k.maxwellian(k.moments(M)).ravel()
    qm = np.abs(k.collide(M[None], conserve=True)).max()
    # dt/eps up to 1e5: beyond that the stage form multiplies rounding by dt/eps
    for eps in (1e-6, 1e-8):
        out = k.imex_step(M[None], 1e-3, eps, scheme=scheme, conserve=True)[0]
        assert np.abs(out - want).max() < 100 * qm + 1e-13 * np.abs(M).max()


def test_moments_of_sampled_gaussian(oracle_mod):
    """Eq. Mo on the grid: for a Gaussian well inside the box the discrete
    moments equal the continuous ones (rho, rho u, E) to rounding, and the
    Maxwellian rebuilt from them reproduces them."""
    for dim, N, L in [(2, 32, 10.0), (3, 32, 10.0)]:
        k = oracle_mod.Kernel(dim, N, L, 1.0)
        rho, th = 1.7, 1.1
        u = np.array([0.4, -0.3, 0.2][:dim])
        f = workloads._gaussian(dim, N, L, np.array([rho]), u[None], np.array([th]))[0]
        U = k.moments(f)
        E = 0.5 * rho * (dim * th + u @ u)
        want = np.concatenate([[rho], rho * u, [E]])
        assert np.abs(U - want).max() < 1e-12 * E
        assert np.abs(k.maxwellian(U).ravel() - f).max() < 1e-12 * f.max()


def _bkw(r2, t):
    S = 1 - math.exp(-t / 8) / 2
    return np.exp(-r2 / (2 * S)) / (2 * math.pi * S ** 2) * (2 * S - 1 + (1 - S) / (2 * S) * r2)


@pytest.mark.parametrize("scheme,order", [("euler", 1), ("ars222", 2), ("bpr343", 3)])
def test_time_order_on_bkw(oracle_mod, scheme, order):
    """eps = 1, Maxwell molecules: error against a fine-step run of the same
    scheme on the same grid falls as dt^order."""
    k = oracle_mod.Kernel(2, 24, 8.0, 0.0)
    v = k.velocities()
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    f0 = _bkw((V1 ** 2 + V2 ** 2).ravel(), 0.0)[None]
    T = 0.8

    def run(dt):
        f = f0.copy()
        for _ in range(int(round(T / dt))):
            f = k.imex_step(f, dt, 1.0, scheme=scheme)
        return f

    ref = run(T / 64)
    errs = [np.linalg.norm(run(T / n) - ref) for n in (2, 4, 8)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > order - 0.35, (errs, rates)
