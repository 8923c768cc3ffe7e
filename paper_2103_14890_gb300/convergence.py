"""Isentropic-vortex convergence study of Sec. 4.1 (Table conv_0): the full
scheme of Sec. 3.4 (CWENO transport of Sec. 3.2 with the penalised IMEX
stages and the spectral collision operator) on periodic triangulations of the
box [0,10]^2, in the fluid limit (a small Knudsen number), against the exact
solution of the Euler equations, the vortex advected by the mean flow (1, 1).

Errors as in Sec. 4.1: the density in the L1 norm and the temperature in the
L2 norm over the box, cell averages of the scheme against the exact fields at
the cell barycentres (which differ from the cell averages by O(h^2), inside
the error of a second-order scheme); the mesh size is the mean of
sqrt(|P_i|).  Every time step runs on the device through imex_step_fv; the
host forms only the moments of the final state and the norms."""
import math

import numpy as np

from . import binding as bz
from . import workloads

BOX = 10.0


def mesh_geometry(pts, cells):
    """Areas, barycentres and perimeters of triangles (n, 3) given
    counter-clockwise or clockwise."""
    P = np.asarray(pts, dtype=np.float64)[np.asarray(cells)]
    e1, e2 = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]
    area = 0.5 * np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    per = sum(np.hypot(*(P[:, (q + 1) % 3] - P[:, q]).T) for q in range(3))
    return area, P.mean(axis=1), per


def moments(f, N, L):
    """Density and temperature (2-D: |v - u|^2 f integrates to 2 rho T) of
    f (n, N^2) on the velocity grid v = -L + (2L/N) k."""
    f = np.asarray(f, dtype=np.float64)
    v = -L + (2.0 * L / N) * np.arange(N)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    V1, V2 = V1.ravel(), V2.ravel()
    w = (2.0 * L / N) ** 2
    rho = f.sum(axis=1) * w
    u1 = (f * V1).sum(axis=1) * w / rho
    u2 = (f * V2).sum(axis=1) * w / rho
    e = (f * (V1 * V1 + V2 * V2)).sum(axis=1) * w / rho
    return rho, 0.5 * (e - u1 * u1 - u2 * u2)


def time_step(area, perimeter, N, L, cfl):
    """The largest step with dt |v|_max perimeter_i / |P_i| <= cfl for every
    cell (the Rusanov flux moves at most |v . n| <= |v| per unit of face)."""
    v = np.abs(-L + (2.0 * L / N) * np.arange(N))
    vmax = math.sqrt(2.0) * v.max()
    return cfl * float((area / perimeter).min()) / vmax


def vortex_run(n_side, N=30, L=10.0, t_final=0.1, eps=1e-6, cfl=0.4, order=2, precision="fp64",
               scheme="ars222", seed=1006, modes=None):
    """March the vortex to t_final on the periodic n_side x n_side
    triangulation; returns a dict with the mesh size h, the step count, dt and
    the errors rho_L1, rho_L2, T_L1, T_L2."""
    import torch
    pts, tri = workloads.periodic_triangulation(n_side, BOX, BOX, seed=seed)
    area, bary, per = mesh_geometry(pts, tri)
    mesh = bz.Mesh(pts, tri, order=order, periodic=(BOX, BOX))
    if modes is None:
        modes = bz.Modes(bz.Grid(2, N, L), 0.0)
    f0, _, _ = workloads.vortex_states(bary, N, L, 0.0, BOX, BOX)
    dt0 = time_step(area, per, N, L, cfl)
    steps = max(1, math.ceil(t_final / dt0 - 1e-12))
    dt = t_final / steps
    ty = torch.float64 if precision == "fp64" else torch.float32
    a = torch.from_numpy(f0).to(device="cuda", dtype=ty).contiguous()
    b = torch.empty_like(a)
    for _ in range(steps):
        bz.imex_step_fv(modes, mesh, a, dt, eps, f_out=b, scheme=scheme, precision=precision)
        a, b = b, a
    bz.check()
    rho, T = moments(a.double().cpu().numpy(), N, L)
    _, rho_x, T_x = workloads.vortex_states(bary, N, L, t_final, BOX, BOX)
    dr, dT = rho - rho_x, T - T_x
    return {"n_side": n_side, "cells": len(tri), "h": float(np.sqrt(area).mean()), "steps": steps, "dt": dt,
            "rho_L1": float((area * np.abs(dr)).sum()), "rho_L2": float(np.sqrt((area * dr * dr).sum())),
            "T_L1": float((area * np.abs(dT)).sum()), "T_L2": float(np.sqrt((area * dT * dT).sum()))}


def orders(rows, key):
    """Observed orders log(e_k / e_{k+1}) / log(h_k / h_{k+1}) between
    consecutive meshes."""
    return [math.log(r0[key] / r1[key]) / math.log(r0["h"] / r1["h"]) for r0, r1 in zip(rows, rows[1:])]


def main(argv=None):
    """Print the convergence table (one row per mesh, then the observed
    orders) as JSON lines."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sides", type=int, nargs="+", default=[18, 36, 54, 72])
    ap.add_argument("--N", type=int, default=30)
    ap.add_argument("--L", type=float, default=10.0)
    ap.add_argument("--t-final", type=float, default=0.1)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    a = ap.parse_args(argv)
    modes = bz.Modes(bz.Grid(2, a.N, a.L), 0.0)
    rows = []
    for n in a.sides:
        rows.append(vortex_run(n, a.N, a.L, a.t_final, a.eps, a.cfl, a.order, a.precision, modes=modes))
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({k: orders(rows, k) for k in ("rho_L1", "rho_L2", "T_L1", "T_L2")}))


if __name__ == "__main__":
    main()
