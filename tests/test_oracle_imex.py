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


def test_euler_boltzmann_step_with_penalty_factor(oracle_mod):
    """The same written-out step with the penalty rate nu = c rho, c = 3; the
    BGK model ignores c (its rate is its collision frequency)."""
    k = oracle_mod.Kernel(2, 16, 8.0, 1.0)
    f = workloads.bi_maxwellian(2, 2, 16, 8.0, seed=26)
    dt, eps, c = 0.02, 0.1, 3.0
    out = k.imex_step(f, dt, eps, scheme="euler", penalty=c)
    Q = k.collide(f)
    for i, fn in enumerate(f):
        U = k.moments(fn)
        G1 = Q[i] - c * U[0] * (k.maxwellian(U).ravel() - fn)
        R = fn + dt * G1 / eps
        U2 = k.moments(R)
        cc = dt * c * U2[0] / eps
        want = (R + cc * k.maxwellian(U2).ravel()) / (1 + cc)
        assert np.abs(out[i] - want).max() < 1e-13 * np.abs(fn).max()
    bgk = k.imex_step(f, dt, eps, scheme="ars222", model="bgk", penalty=c)
    assert np.array_equal(bgk, k.imex_step(f, dt, eps, scheme="ars222", model="bgk"))


def _jacobian(k, M):
    """Linearised conservative Q at M by central differences (exact for the
    bilinear Q up to rounding)."""
    n = M.size
    h = 1e-6 * np.abs(M).max()
    E = np.eye(n) * h
    return ((k.collide(M[None] + E, conserve=True) - k.collide(M[None] - E, conserve=True)) / (2 * h)).T


def _zero_moments(k, x):
    """x minus its projection on the collision invariants (1, v, |v|^2) in the
    discrete inner product: a perturbation that leaves the moments alone."""
    v = k.velocities()
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    B = np.stack([np.ones(V1.size), V1.ravel(), V2.ravel(), (V1 ** 2 + V2 ** 2).ravel()], axis=1)
    return x - B @ np.linalg.solve(B.T @ B, B.T @ x)


@pytest.mark.parametrize("c", [1.0, 3.0])
def test_ars222_linear_response_near_equilibrium(oracle_mod, c):
    """Near a Maxwellian M the step acts linearly on a perturbation d with zero
    moments (the moments, hence nu and the stage Maxwellians, do not move):
    with J_l the linearised Q at the unperturbed stage value F_l (Q of a
    Maxwellian is not zero on the grid, so F_2 is not M), a = dt gamma nu/eps,
    and the ARS(2,2,2) tableau,
      F_1' = d, G_1' = (J_1 + nu) d,
      F_2' = (d + (dt gamma/eps) G_1') / (1 + a), G_2' = (J_2 + nu) F_2', P_2' = -nu F_2',
      F_3' = (d + (dt/eps)(dl G_1' + (1 - dl) G_2' + (1 - gamma) P_2')) / (1 + a),
    dl = 1 - 1/(2 gamma).  The step's odd part in the amplitude matches F_3'
    (Q is bilinear, so the even part holds the quadratic terms)."""
    N, L = 16, 8.0
    k = oracle_mod.Kernel(2, N, L, 0.0)
    rho = 0.7      # theta = 1.2: the grid resolves M (the sampled Maxwellian of its own
    # discrete moments then has those moments to 1e-10, so nu and M_l hold still)
    M = k.maxwellian(np.array([rho, rho * 0.3, -rho * 0.2, 0.5 * rho * (2 * 1.2 + 0.13)])).ravel()
    d = _zero_moments(k, np.random.default_rng(4).standard_normal(M.size) * M)
    dt, eps, eta = 0.01, 1e-3, 1e-4
    _, F0, _, _ = k.imex_step(M[None], dt, eps, conserve=True, penalty=c, stages=True)
    J1, J2 = _jacobian(k, F0[0, 0]), _jacobian(k, F0[1, 0])
    nu = c * k.moments(M)[0]
    a = dt * G * nu / eps
    dl = 1 - 1 / (2 * G)
    G1 = (J1 + nu * np.eye(M.size)) @ d
    F2 = (d + dt * G / eps * G1) / (1 + a)
    G2 = (J2 + nu * np.eye(M.size)) @ F2
    F3 = (d + dt / eps * (dl * G1 + (1 - dl) * G2 - (1 - G) * nu * F2)) / (1 + a)
    up = k.imex_step((M + eta * d)[None], dt, eps, conserve=True, penalty=c)[0]
    dn = k.imex_step((M - eta * d)[None], dt, eps, conserve=True, penalty=c)[0]
    odd = (up - dn) / (2 * eta)
    assert np.abs(odd - F3).max() < 1e-6 * np.abs(F3).max()


def test_fluid_limit_amplification_and_penalty():
    """Why the penalty factor exists: as eps -> 0 the recursion above multiplies
    an eigenvector of J (eigenvalue lam) by g(K) = ((1 - dl) K^2 + (dl - 1 +
    gamma) K)/gamma, K = 1 + lam/nu.  For complex K near 0.41, |g| > 1.  The
    closed form is checked against the limit of the recursion, and on the
    spectrum of the spectral Q at the coldest state of the isentropic vortex
    (rho = theta = 0.596, 30^2 grid on [-10,10]^2) c = 1 gives |g| = 1.30 (the
    growth per step seen when the vortex is marched at eps = 1e-6) while c = 3
    keeps |g| <= 1."""
    import oracle
    dl = 1 - 1 / (2 * G)

    def g(K):
        return ((1 - dl) * K * K + (dl - 1 + G) * K) / G

    for K in (0.3 + 0.1j, 0.9, -0.02 + 0.2j):       # the limit of the recursion, written per mode
        nu, lam = 1.0, K - 1.0
        G1 = lam + nu
        F2 = G1 / nu
        F3 = (dl * G1 + (1 - dl) * (lam + nu) * F2 - (1 - G) * nu * F2) / (G * nu)
        assert abs(F3 - g(K)) < 1e-12
    assert abs(g(0.4142 + 0.2j)) > 1.2 and abs(g(0.4142)) <= 1.0 + 1e-4
    N, L, rho = 30, 10.0, 0.596
    k = oracle.Kernel(2, N, L, 0.0)
    M = workloads._gaussian(2, N, L, np.array([rho]), np.array([[1.0, 1.0]]), np.array([rho]))[0]
    lam = np.linalg.eigvals(_jacobian(k, M))
    lam = lam[np.abs(lam) > 1e-8 * np.abs(lam).max()]          # drop the conserved directions
    amp = {c: float(np.abs(g(1 + lam / (c * rho))).max()) for c in (1.0, 3.0)}
    assert amp[1.0] > 1.25 and amp[3.0] <= 1.0 + 1e-6, amp


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


@pytest.mark.parametrize("scheme,order,penalty", [("euler", 1, 1.0), ("ars222", 2, 1.0), ("bpr343", 3, 1.0),
                                                   ("ars222", 2, 3.0)])
def test_time_order_on_bkw(oracle_mod, scheme, order, penalty):
    """eps = 1, Maxwell molecules: error against a fine-step run of the same
    scheme on the same grid falls as dt^order (with the penalty rate nu = c rho
    for c = 1 and 3: the penalty changes the splitting, not the limit)."""
    k = oracle_mod.Kernel(2, 24, 8.0, 0.0)
    v = k.velocities()
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    f0 = _bkw((V1 ** 2 + V2 ** 2).ravel(), 0.0)[None]
    T = 0.8

    def run(dt):
        f = f0.copy()
        for _ in range(int(round(T / dt))):
            f = k.imex_step(f, dt, 1.0, scheme=scheme, penalty=penalty)
        return f

    ref = run(T / 64)
    errs = [np.linalg.norm(run(T / n) - ref) for n in (2, 4, 8)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > order - 0.35, (errs, rates)
