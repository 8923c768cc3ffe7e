"""Pins for the oracle's fast spectral method (Sec. 3.3, Carleman form:
eq. defQBCarleman, eq. Btilde, eq. FKM, eq. ode), 2-D Maxwell molecules.

The oracle's kernel modes B_F(l,m) = sum_p alpha_p(l) alpha'_p(m) are checked
against things other than themselves:
  - a Gauss cubature of eq. FKM itself (square truncation |x|, |y| <= R),
    written here with no closed form for the inner integrals;
  - the same cubature over the disk |x|^2 + |y|^2 <= R^2, which is the
    Carleman form of the classical truncation |q| <= R and must reproduce the
    classical kernel modes of eq. KM in their Lommel closed form (this pins
    the change of variables: the weight 2 b0, theta over [0, pi), rho and
    rho' over [-R, R]);
  - the BKW closed form (Sec. 4.1): Q_F(f_BKW(t)) = d/dt f_BKW(t);
  - invariants: exact mass conservation, D4 and shift equivariance.
"""
import math

import numpy as np
import pytest
from scipy import special

LAM = 2.0 / (3.0 + math.sqrt(2.0))
RCUT = 2.0 * LAM * math.pi          # truncation radius in the computational box
B0_2D = 1.0 / (2.0 * math.pi)


def _carleman_cubature(l, m, region, b0=B0_2D, nth=240, nr=120):
    """2 b0 int_0^pi dtheta int int e^{i(rho l.e + rho' m.e_perp)} drho drho'
    over the square [-R,R]^2 or the disk rho^2 + rho'^2 <= R^2, all three
    integrals by Gauss-Legendre (the imaginary part vanishes by symmetry)."""
    xt, wt = np.polynomial.legendre.leggauss(nth)
    th, wth = 0.5 * math.pi * (xt + 1), 0.5 * math.pi * wt
    x, w = np.polynomial.legendre.leggauss(nr)
    if region == "square":
        rho, wr, Y = RCUT * x, RCUT * w, np.full(nr, RCUT)
    else:                       # rho = R sin s keeps the disk's edge smooth
        s = 0.5 * math.pi * x
        rho, wr, Y = RCUT * np.sin(s), RCUT * np.cos(s) * 0.5 * math.pi * w, RCUT * np.cos(s)
    tot = 0.0
    for t, wtt in zip(th, wth):
        a = l[0] * math.cos(t) + l[1] * math.sin(t)
        b = -m[0] * math.sin(t) + m[1] * math.cos(t)
        inner = (Y[:, None] * w[None, :] * np.cos(Y[:, None] * x[None, :] * b)).sum(axis=1)
        tot += wtt * np.dot(wr, np.cos(rho * a) * inner)
    return 2.0 * b0 * tot


def _lommel_bhat(l, m):
    """Classical B-hat(l,m) of eq. KM for 2-D Maxwell molecules in closed form:
    b0 (2 pi)^2 int_0^R rho J0(rho |l+m|/2) J0(rho |l-m|/2) drho."""
    al = np.linalg.norm(np.add(l, m)) / 2
    be = np.linalg.norm(np.subtract(l, m)) / 2
    j0, j1, R = special.j0, special.j1, RCUT
    if al == 0 and be == 0:
        v = R * R / 2
    elif be == 0:
        v = R * j1(al * R) / al
    elif al == 0:
        v = R * j1(be * R) / be
    elif abs(al - be) < 1e-15:
        v = R * R / 2 * (j0(al * R) ** 2 + j1(al * R) ** 2)
    else:
        v = R * (al * j1(al * R) * j0(be * R) - be * j0(al * R) * j1(be * R)) / (al ** 2 - be ** 2)
    return B0_2D * (2 * math.pi) ** 2 * v


PAIRS = [((0, 0), (0, 0)), ((1, 2), (0, -1)), ((3, -1), (2, 2)), ((7, 0), (-3, 5)),
         ((5, 5), (-6, 2)), ((-4, 7), (7, -7))]


@pytest.mark.parametrize("l,m", PAIRS)
def test_direction_sum_matches_cubature_of_eq_FKM(oracle_mod, l, m):
    """Many directions: the oracle's rectangle rule in theta converges to the
    cubature of eq. FKM (which uses no closed form for phi)."""
    k = oracle_mod.FastKernel(16, 8.0, 512)
    got = k.bhat(l, m)
    want = _carleman_cubature(l, m, "square")
    assert abs(got - want) <= 1e-11 * max(1.0, abs(want))


@pytest.mark.parametrize("l,m", PAIRS)
def test_carleman_variables_reproduce_classical_modes(oracle_mod, l, m):
    """Over the disk |x|^2 + |y|^2 <= R^2 the Carleman integral is the
    classical eq. KM with |q| <= R: it must equal the Lommel closed form."""
    want = _lommel_bhat(l, m)
    got = _carleman_cubature(l, m, "disk")
    assert abs(got - want) <= 1e-11 * max(1.0, abs(want))
    # and the oracle's classical table agrees (same closed form)
    assert abs(oracle_mod.Kernel(2, 16, 8.0, 0.0).bhat(l, m) - want) <= 1e-12 * max(1.0, abs(want))


def test_direction_factors_on_the_axes(oracle_mod):
    """theta_0 = 0: alpha_0(k) alpha'_0(m) = (2 b0 pi / A) phi(k_1) phi(m_2)
    with phi(xi) = 2 sin(R xi)/xi; one direction isolates that term."""
    k = oracle_mod.FastKernel(8, 8.0, 1)
    phi = lambda xi: 2 * RCUT if xi == 0 else 2 * math.sin(RCUT * xi) / xi
    for l, m in [((1, 2), (3, -1)), ((0, 0), (2, 1)), ((-3, 1), (0, 0))]:
        want = 2 * B0_2D * math.pi * phi(l[0]) * phi(m[1])
        assert abs(k.bhat(l, m) - want) <= 1e-13 * max(1.0, abs(want))


def _bkw(r2, t):
    S = 1 - math.exp(-t / 8) / 2
    return np.exp(-r2 / (2 * S)) / (2 * math.pi * S ** 2) * (2 * S - 1 + (1 - S) / (2 * S) * r2)


def _bkw_dt(r2, t):
    S = 1 - math.exp(-t / 8) / 2
    A = np.exp(-r2 / (2 * S)) / (2 * math.pi * S ** 2)
    B = 2 * S - 1 + (1 - S) / (2 * S) * r2
    dA = A * (r2 / (2 * S ** 2) - 2 / S)
    dB = 2 - r2 / (2 * S ** 2)
    return (dA * B + A * dB) * (1 - S) / 8


@pytest.mark.parametrize("ndirs", [8, 16])
def test_fast_bkw_time_derivative(oracle_mod, ndirs):
    """Q_F(f_BKW(t)) = d/dt f_BKW(t): pins b0, the Carleman weight, the loss
    term's sign and the s^d scale of the fast form at O(1)."""
    k = oracle_mod.FastKernel(64, 12.0, ndirs)
    v = k.velocities()
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    r2 = (V1 ** 2 + V2 ** 2).ravel()
    for t in (0.5, 2.0):
        Q = k.collide(_bkw(r2, t)[None])[0]
        d = _bkw_dt(r2, t)
        assert np.linalg.norm(Q - d) / np.linalg.norm(d) < 1e-5


def _two_maxwellians(k, rng):
    v = k.velocities()
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    f = np.zeros_like(V1)
    for _ in range(2):
        rho, th = rng.uniform(0.5, 2.0), rng.uniform(0.5, 1.5)
        u = rng.uniform(-1.5, 1.5, 2)
        f += rho / (2 * math.pi * th) * np.exp(-((V1 - u[0]) ** 2 + (V2 - u[1]) ** 2) / (2 * th))
    return f


def test_fast_mass_and_equivariance(oracle_mod):
    rng = np.random.default_rng(11)
    k = oracle_mod.FastKernel(16, 8.0, 8)
    f = _two_maxwellians(k, rng) * (1 + 0.1 * rng.uniform(-1, 1, (16, 16)))
    Q = k.collide(f[None])[0].reshape(16, 16)
    assert abs(Q.sum()) < 1e-14 * np.abs(Q).sum()
    # D4 about the grid's centre node v = 0 (index N/2): a quarter turn maps
    # B_F(l,m) to B_F(m,l) and the gain sees only B_F(l,m) + B_F(m,l), so it
    # holds for any number of directions; likewise a reflection
    rot = lambda a: np.roll(np.rot90(np.roll(a, -8, (0, 1))), 8, (0, 1))
    ref = lambda a: np.roll(np.roll(a, -8, 0)[::-1], 9, 0)
    for op in (rot, ref):
        Qo = k.collide(op(f)[None])[0].reshape(16, 16)
        assert np.abs(Qo - op(Q)).max() < 1e-12 * np.abs(Q).max()
    # cyclic shift by whole grid steps
    Qs = k.collide(np.roll(f, (3, -5), (0, 1))[None])[0].reshape(16, 16)
    assert np.abs(Qs - np.roll(Q, (3, -5), (0, 1))).max() < 1e-12 * np.abs(Q).max()


def test_fast_and_classical_forms_agree_for_resolved_f(oracle_mod):
    """Both truncations reproduce the collision integral for f supported in
    the ball of radius lambda*pi (computational box): for two Maxwellians well
    inside a wide box the two discrete operators agree to the spectral error."""
    diffs = {}
    for N in (48, 64):
        rng = np.random.default_rng(5)
        kf = oracle_mod.FastKernel(N, 14.0, 16)
        kc = oracle_mod.Kernel(2, N, 14.0, 0.0)
        f = _two_maxwellians(kf, rng)
        Qf = kf.collide(f[None])[0]
        Qc = kc.collide(f[None])[0]
        diffs[N] = np.linalg.norm(Qf - Qc) / np.linalg.norm(Qc)
    assert diffs[48] < 1e-5 and diffs[64] < 1e-8
