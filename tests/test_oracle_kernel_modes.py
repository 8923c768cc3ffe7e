"""Pins for the oracle's kernel modes B-hat(l,m) (eq. KM) and its quadrature.

Each check compares the oracle with something other than itself: numpy's
Gauss-Legendre rule, closed-form Lommel / sine integrals, and brute-force
cubature of eq. KM over q and omega with no Bessel reduction.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import special

LAM = 2.0 / (3.0 + math.sqrt(2.0))
RCUT = 2.0 * LAM * math.pi          # |q| cut-off of eq. KM in the computational box
B0_2D = 1.0 / (2.0 * math.pi)


def test_gauss_legendre_matches_numpy(oracle_mod):
    for n in (2, 5, 17, 64, 150):
        x, w = oracle_mod.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        order = np.argsort(x)
        assert np.allclose(x[order], xr, atol=1e-14, rtol=0)
        assert np.allclose(w[order], wr, atol=1e-14, rtol=0)
        # exactness on monomials up to degree 2n-1
        for p in range(0, 2 * n, max(1, n // 3)):
            exact = 0.0 if p % 2 else 2.0 / (p + 1)
            assert abs(np.dot(w, x ** p) - exact) < 1e-13


def _lommel(alpha, beta, R):
    """int_0^R rho J0(alpha rho) J0(beta rho) drho in closed form."""
    j0, j1 = special.j0, special.j1
    if alpha == 0 and beta == 0:
        return R * R / 2
    if beta == 0:
        return R * j1(alpha * R) / alpha
    if alpha == 0:
        return R * j1(beta * R) / beta
    if abs(alpha - beta) < 1e-15:
        return R * R / 2 * (j0(alpha * R) ** 2 + j1(alpha * R) ** 2)
    return R * (alpha * j1(alpha * R) * j0(beta * R) - beta * j0(alpha * R) * j1(beta * R)) / (
        alpha ** 2 - beta ** 2)


def _sine_integral(alpha, beta, R):
    """int_0^R rho^2 sinc(alpha rho) sinc(beta rho) drho in closed form."""
    if alpha == 0 and beta == 0:
        return R ** 3 / 3
    if beta == 0 or alpha == 0:
        a = alpha or beta
        return (math.sin(a * R) / a ** 2 - R * math.cos(a * R) / a) / a
    if abs(alpha - beta) < 1e-15:
        return (R / 2 - math.sin(2 * alpha * R) / (4 * alpha)) / alpha ** 2
    return (math.sin((alpha - beta) * R) / (2 * (alpha - beta))
            - math.sin((alpha + beta) * R) / (2 * (alpha + beta))) / (alpha * beta)


@pytest.mark.parametrize("a,b", [(0, 0), (0, 3), (2, 0), (1.5, 1.5), (3, 7.2), (21.2, 42.4),
                                 (math.sqrt(5), math.sqrt(13)), (10, 10)])
def test_maxwell_2d_matches_lommel(oracle_mod, a, b):
    got = oracle_mod.radial_bhat(2, 0.0, B0_2D, 160, a, b)
    want = B0_2D * (2 * math.pi) ** 2 * _lommel(a / 2, b / 2, RCUT)
    assert abs(got - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("a,b", [(0, 0), (0, 3), (2, 0), (1.5, 1.5), (3, 7.2), (12, 24)])
def test_maxwell_3d_matches_sine_integral(oracle_mod, a, b):
    b0 = 1.0 / (4 * math.pi)
    got = oracle_mod.radial_bhat(3, 0.0, b0, 160, a, b)
    want = b0 * (4 * math.pi) ** 2 * _sine_integral(a / 2, b / 2, RCUT)
    assert abs(got - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("dim,N", [(2, 16), (2, 32), (2, 48), (3, 16)])
def test_default_nodes_self_converged(oracle_mod, dim, N):
    """Hard spheres (gamma = 1) have no closed form: the default node count must
    agree with twice as many nodes over the full range of norms."""
    k = oracle_mod.Kernel(dim, N, 10.0, 1.0)
    h = k.h
    amax = h * math.sqrt(dim)
    bmax = 2 * h * math.sqrt(dim)
    scale = abs(oracle_mod.radial_bhat(dim, 1.0, k.b0, k.nq, 0, 0))
    for a in np.linspace(0, amax, 7):
        for b in np.linspace(0, bmax, 7):
            r1 = oracle_mod.radial_bhat(dim, 1.0, k.b0, k.nq, a, b)
            r2 = oracle_mod.radial_bhat(dim, 1.0, k.b0, 2 * k.nq, a, b)
            assert abs(r1 - r2) <= 2e-14 * scale


def _bhat_bruteforce_2d(l, m, gamma, b0, nr=40, nphi=64, npsi=64):
    """Eq. KM by direct cubature: q = rho (cos phi, sin phi) over the disc of
    radius RCUT (Gauss-Legendre in rho, trapezoid in phi), omega = (cos psi,
    sin psi) (trapezoid), integrand b0 |q|^gamma exp(-i (l.q+ + m.q-))."""
    x, w = np.polynomial.legendre.leggauss(nr)
    rho = 0.5 * RCUT * (x + 1)
    wr = 0.5 * RCUT * w
    phi = 2 * math.pi * np.arange(nphi) / nphi
    psi = 2 * math.pi * np.arange(npsi) / npsi
    R, PHI, PSI = np.meshgrid(rho, phi, psi, indexing="ij")
    q1, q2 = R * np.cos(PHI), R * np.sin(PHI)
    o1, o2 = np.cos(PSI), np.sin(PSI)
    qp1, qp2 = 0.5 * (q1 + R * o1), 0.5 * (q2 + R * o2)
    qm1, qm2 = 0.5 * (q1 - R * o1), 0.5 * (q2 - R * o2)
    phase = l[0] * qp1 + l[1] * qp2 + m[0] * qm1 + m[1] * qm2
    integrand = b0 * R ** gamma * np.exp(-1j * phase) * R          # R: polar Jacobian
    val = (integrand * wr[:, None, None]).sum() * (2 * math.pi / nphi) * (2 * math.pi / npsi)
    return val


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_bhat_2d_matches_bruteforce_eq_KM(oracle_mod, gamma):
    k = oracle_mod.Kernel(2, 4, 5.0, gamma)
    modes = list(itertools.product(range(-k.h, k.h + 1), repeat=2))
    for l in modes:
        for m in modes:
            want = _bhat_bruteforce_2d(l, m, gamma, k.b0)
            got = k.bhat(l, m)
            assert abs(want.imag) < 1e-12          # B-hat is real (q -> -q symmetry)
            assert abs(got - want.real) < 1e-12 * max(1.0, abs(want.real)), (l, m, got, want)


def test_bhat_2d_bruteforce_larger_modes(oracle_mod):
    """N = 6 (h = 2), a sample of pairs including ones with |l+m| off-lattice-axis."""
    k = oracle_mod.Kernel(2, 6, 5.0, 1.0)
    rng = np.random.default_rng(7)
    for _ in range(12):
        l = tuple(int(v) for v in rng.integers(-2, 3, 2))
        m = tuple(int(v) for v in rng.integers(-2, 3, 2))
        want = _bhat_bruteforce_2d(l, m, 1.0, k.b0, nr=48, nphi=80, npsi=80)
        assert abs(k.bhat(l, m) - want.real) < 1e-11 * max(1.0, abs(want.real))


def test_bhat_3d_matches_bruteforce_eq_KM(oracle_mod):
    """3-D: q in spherical coordinates, omega on S^2, no sinc reduction."""
    k = oracle_mod.Kernel(3, 4, 5.0, 1.0)
    nr, nt, nph = 24, 20, 32
    x, w = np.polynomial.legendre.leggauss(nr)
    rho = 0.5 * RCUT * (x + 1); wr = 0.5 * RCUT * w
    ct, wt = np.polynomial.legendre.leggauss(nt)         # cos(theta) nodes
    ph = 2 * math.pi * np.arange(nph) / nph
    st = np.sqrt(1 - ct ** 2)
    # unit vectors on the sphere (nt*nph) with weights
    U = np.stack([np.outer(st, np.cos(ph)).ravel(), np.outer(st, np.sin(ph)).ravel(),
                  np.repeat(ct, nph)], axis=1)
    WU = np.repeat(wt, nph) * (2 * math.pi / nph)
    for (l, m) in [((0, 0, 0), (1, 0, 0)), ((1, -1, 0), (0, 1, 1)), ((1, 1, 1), (-1, 1, 0)),
                   ((1, 0, -1), (1, 0, -1))]:
        l = np.array(l, float); m = np.array(m, float)
        total = 0.0 + 0.0j
        for ir in range(nr):
            q = rho[ir] * U                                   # (nu, 3)
            qp = 0.5 * (q[:, None, :] + rho[ir] * U[None, :, :])
            qm = 0.5 * (q[:, None, :] - rho[ir] * U[None, :, :])
            phase = qp @ l + qm @ m
            val = (np.exp(-1j * phase) * WU[:, None] * WU[None, :]).sum()
            total += wr[ir] * k.b0 * rho[ir] ** 1.0 * rho[ir] ** 2 * val
        assert abs(total.imag) < 1e-11
        got = k.bhat(l.astype(int), m.astype(int))
        assert abs(got - total.real) < 1e-10 * max(1.0, abs(total.real)), (l, m, got, total)


def test_bhat_symmetries(oracle_mod):
    k = oracle_mod.Kernel(2, 16, 8.0, 1.0)
    rng = np.random.default_rng(3)
    h = k.h
    for _ in range(200):
        l = rng.integers(-h, h + 1, 2)
        m = rng.integers(-h, h + 1, 2)
        b = k.bhat(l, m)
        assert b == k.bhat(m, l)                                   # exchange l <-> m
        assert b == k.bhat(-l, -m)                                 # q -> -q
        rot = lambda v: np.array([-v[1], v[0]])                    # lattice rotation
        assert b == k.bhat(rot(l), rot(m))
        assert b == k.bhat(l[::-1].copy(), m[::-1].copy())         # reflection
        assert k.beta(l, -l) == 0.0                                # beta(l,-l) = 0 bitwise


def test_cached_table_equals_direct_quadrature(oracle_mod):
    for dim, N, gamma in [(2, 16, 0.0), (2, 32, 1.0), (3, 8, 1.0)]:
        k = oracle_mod.Kernel(dim, N, 10.0, gamma)
        rng = np.random.default_rng(11)
        for _ in range(40):
            l = rng.integers(-k.h, k.h + 1, dim)
            m = rng.integers(-k.h, k.h + 1, dim)
            a = float(np.linalg.norm(l + m)); b = float(np.linalg.norm(l - m))
            direct = oracle_mod.radial_bhat(dim, gamma, k.b0, k.nq, a, b)
            assert abs(k.bhat(l, m) - direct) <= 1e-14 * max(1.0, abs(direct)) * 50
