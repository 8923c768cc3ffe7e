"""Pins for the oracle's forward/inverse transforms (eq. FC, eq. FU on the grid).

Checks against exact trigonometric polynomials evaluated directly and against
numpy's FFT (an independent library routine).
"""
import math

import numpy as np
import pytest


def _grid_u(N):
    return -math.pi + 2 * math.pi * np.arange(N) / N


def _random_hermitian(rng, dim, h):
    """Random coefficients c_k on K_h with c_{-k} = conj(c_k) (real function)."""
    M = 2 * h + 1
    c = rng.normal(size=(M,) * dim) + 1j * rng.normal(size=(M,) * dim)
    flip = c[(slice(None, None, -1),) * dim]
    return 0.5 * (c + np.conj(flip))


def _eval_trig(c, h, pts_axes):
    """sum_k c_k exp(i k.u) on the tensor grid given by the 1-D axes."""
    dim = c.ndim
    ks = np.arange(-h, h + 1)
    out = c
    for i in range(dim):
        E = np.exp(1j * np.outer(ks, pts_axes[i]))      # (M, P)
        out = np.tensordot(out, E, axes=([0], [0]))     # contracts the leading mode axis
    return out


@pytest.mark.parametrize("dim,N", [(2, 8), (2, 16), (3, 6)])
def test_forward_recovers_trig_polynomial(oracle_mod, dim, N):
    k = oracle_mod.Kernel(dim, N, 3.0, 0.0)
    rng = np.random.default_rng(1)
    c = _random_hermitian(rng, dim, k.h)
    u = _grid_u(N)
    f = _eval_trig(c, k.h, [u] * dim)
    assert np.abs(f.imag).max() < 1e-12
    fhat = k.dft_forward(f.real)
    assert np.abs(fhat - c).max() < 1e-13 * np.abs(c).max()
    back = k.dft_inverse(fhat, scale=1.0)
    assert np.abs(back - f.real).max() < 1e-12 * np.abs(f).max()


def test_forward_matches_numpy_fft(oracle_mod):
    """f-hat_k = N^-d (-1)^(k_1+..+k_d) FFT(f)[k mod N] because u_0 = -pi."""
    for dim, N in [(2, 16), (2, 32), (3, 8)]:
        k = oracle_mod.Kernel(dim, N, 5.0, 1.0)
        rng = np.random.default_rng(2)
        f = rng.uniform(size=(N,) * dim)
        F = np.fft.fftn(f) / N ** dim
        ks = np.arange(-k.h, k.h + 1)
        idx = np.ix_(*([ks % N] * dim))
        sign = np.ones((k.M,) * dim)
        for i in range(dim):
            shape = [1] * dim
            shape[i] = k.M
            sign = sign * ((-1.0) ** ks).reshape(shape)
        want = F[idx] * sign
        got = k.dft_forward(f)
        assert np.abs(got - want).max() < 1e-15 * N ** dim * np.abs(f).max()


def test_single_modes(oracle_mod):
    """cos(u_1) -> 1/2 at k = (+-1, 0); sin(2 u_2) -> -+ i/2 at k = (0, +-2)."""
    k = oracle_mod.Kernel(2, 8, 3.0, 0.0)
    u = _grid_u(8)
    U1, U2 = np.meshgrid(u, u, indexing="ij")
    h = k.h
    fh = k.dft_forward(np.cos(U1))
    want = np.zeros((k.M, k.M), complex)
    want[h + 1, h] = want[h - 1, h] = 0.5
    assert np.abs(fh - want).max() < 1e-15
    fh = k.dft_forward(np.sin(2 * U2))
    want = np.zeros((k.M, k.M), complex)
    want[h, h + 2] = -0.5j
    want[h, h - 2] = 0.5j
    assert np.abs(fh - want).max() < 1e-15


def test_inverse_scale_and_nyquist_drop(oracle_mod):
    """The Nyquist mode is not in K_h: cos(N u/2) has no retained coefficient."""
    k = oracle_mod.Kernel(2, 8, 3.0, 0.0)
    u = _grid_u(8)
    U1, _ = np.meshgrid(u, u, indexing="ij")
    assert np.abs(k.dft_forward(np.cos(4 * U1))).max() < 1e-15
    qh = np.zeros((k.M, k.M), complex)
    qh[k.h, k.h] = 2.0
    assert np.allclose(k.dft_inverse(qh, scale=3.5), 7.0, atol=1e-15, rtol=0)
