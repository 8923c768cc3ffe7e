"""Host arithmetic of the vortex study (moments, geometry, time step) against
closed forms; the march itself runs on the GPU (test_gpu_transport.py)."""
import math

import numpy as np

from paper_2103_14890_gb300 import convergence, workloads


def test_moments_of_vortex_maxwellians():
    """The sampled Maxwellians of the vortex carry its density and temperature
    (rectangle rule on a periodic-like grid: exponentially accurate for a
    Gaussian well inside [-10,10]^2)."""
    pts, tri = workloads.periodic_triangulation(6)
    _, bary, _ = convergence.mesh_geometry(pts, tri)
    f, rho, T = workloads.vortex_states(bary, 30, 10.0)
    r, t = convergence.moments(f, 30, 10.0)
    assert np.abs(r - rho).max() < 1e-10 and np.abs(t - T).max() < 1e-10
    assert T.min() < 0.9 and rho.min() < 0.9         # the vortex core is resolved


def test_geometry_and_time_step():
    pts, tri = workloads.periodic_triangulation(10, jitter=0.0)
    area, bary, per = convergence.mesh_geometry(pts, tri)
    assert abs(area.sum() - 100.0) < 1e-9                      # the box [0,10]^2
    assert np.allclose(per, 1.0 * (2 + math.sqrt(2)))          # right triangles with legs 1
    assert (bary > 0).all() and (bary < 10).all()
    dt = convergence.time_step(area, per, 30, 10.0, 0.4)
    assert abs(dt - 0.4 * (0.5 / (2 + math.sqrt(2))) / (10 * math.sqrt(2))) < 1e-15


def test_orders_and_errors():
    rows = [{"h": 0.4, "e": 1.6e-2}, {"h": 0.2, "e": 4e-3}, {"h": 0.1, "e": 1e-3}]
    assert np.allclose(convergence.orders(rows, "e"), [2.0, 2.0])
    rows = [{"dt": 1e-3, "e": 8e-6}, {"dt": 5e-4, "e": 1e-6}]
    assert np.allclose(convergence.orders(rows, "e", by="dt"), [3.0])
    e = convergence.errors(np.array([2.0, 3.0]), np.array([1.0, 1.5]), np.array([1.0, 1.0]),
                           np.array([1.0, 1.0]), np.array([0.5, 1.0]))
    assert np.isclose(e["rho_L1"], 1.5) and np.isclose(e["rho_L2"], np.sqrt(0.75))
    assert np.isclose(e["T_L1"], 1.0) and np.isclose(e["T_L2"], np.sqrt(0.5))


def test_vortex_is_a_steady_isentropic_euler_solution():
    """The vortex states (T = 1 + dT, rho = (1 + dT)^(1/(gamma-1)), gamma = 2,
    the velocity perturbation of Sec. 4.1) satisfy, in the frame moving with
    (1, 1), p / rho^gamma = const and the radial balance dp/dr = rho u_th^2 / r
    of a steady rotating flow of the Euler equations: checked by central
    differences of the states' own moments along a ray."""
    N, L = 48, 10.0
    r = np.linspace(0.2, 3.0, 15)
    dr = 1e-4
    pts = np.stack([5.0 + r, np.full_like(r, 5.0)], axis=1)                   # a ray along +x from the centre
    _, rho, T = workloads.vortex_states(pts, N, L)
    p = rho * T
    assert np.abs(p / rho ** 2 - 1.0).max() < 1e-12                        # isentropic, gamma = 2
    rp = np.stack([5.0 + r + dr, np.full_like(r, 5.0)], axis=1)
    rm = np.stack([5.0 + r - dr, np.full_like(r, 5.0)], axis=1)
    _, rho_p, T_p = workloads.vortex_states(rp, N, L)
    _, rho_m, T_m = workloads.vortex_states(rm, N, L)
    dpdr = (rho_p * T_p - rho_m * T_m) / (2 * dr)
    # azimuthal velocity from the moments of the sampled Maxwellians (minus the mean flow)
    f, _, _ = workloads.vortex_states(pts, N, L)
    v = -L + (2.0 * L / N) * np.arange(N)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    w = (2.0 * L / N) ** 2
    u2 = (f * V2.ravel()).sum(axis=1) * w / (f.sum(axis=1) * w) - 1.0       # on the +x ray u_theta = u_y - 1
    assert np.abs(dpdr - rho * u2 ** 2 / r).max() < 1e-6 * np.abs(dpdr).max()
