"""Isentropic-vortex convergence studies of Sec. 4.1 (Tables conv_0,
conv_1e-3, conv_1e-2 and conv_1): the full scheme of Sec. 3.4 (CWENO
transport of Sec. 3.2 with the penalised IMEX stages and the spectral
collision operator) on periodic triangulations or Voronoi tessellations of
the box [0,10]^2, 30^2 velocities on [-10,10]^2, every time step on the
device through imex_step_fv; the host forms only the moments of the final
states and the norms.

- Space-time study (eps -> 0, Table conv_0): errors against the exact
  solution of the Euler equations, the vortex advected by the mean flow
  (1, 1), on a sequence of meshes with the time step tied to the mesh.  In
  the limit the collision operator enters only through its equilibria, the
  Maxwellians of the stage moments, which the Boltzmann and BGK models share;
  the study takes the limit through the BGK relaxation at eps = 1e-8.  The
  penalised Boltzmann step at eps << dt leaves the non-equilibrium part of f
  that lies in the near-null directions of the linearised spectral Q
  unrelaxed (at the vortex core, 191 of the 900 eigenvalues of the 30^2
  operator are below 0.05 rho in size), and the temperature error then grows
  with the number of steps; that run is kept as an option (model="boltzmann").
- Time study (eps = 1e-3, 1e-2, 1; Tables conv_1e-3 to conv_1): the
  Boltzmann model on one mesh with h = 1/3, errors at t_f = 9e-3 against a
  run with a 32 times smaller step on the same mesh.

Errors as in Sec. 4.1: the density and the temperature in the L1 and L2 norms
over the box; the space study compares cell averages with the exact fields
at the barycentres (they differ by O(h^2), inside the error of a
second-order scheme); the mesh size is the mean of sqrt(|P_i|)."""
import math

import numpy as np

from . import binding as bz
from . import workloads

BOX = 10.0


def mesh_geometry(pts, cells):
    """Areas, barycentres and perimeters of polygons given counter-clockwise
    or clockwise (an (n, k) array or a list of vertex lists)."""
    pts = np.asarray(pts, dtype=np.float64)
    area, bary, per = np.zeros(len(cells)), np.zeros((len(cells), 2)), np.zeros(len(cells))
    for i, c in enumerate(cells):
        P = pts[list(c)] - pts[c[0]]
        x, y = P[:, 0], P[:, 1]
        xn, yn = np.roll(x, -1), np.roll(y, -1)
        cr = x * yn - xn * y
        a = 0.5 * cr.sum()
        area[i] = abs(a)
        bary[i] = pts[c[0]] + np.array([((x + xn) * cr).sum(), ((y + yn) * cr).sum()]) / (6.0 * a)
        per[i] = np.hypot(xn - x, yn - y).sum()
    return area, bary, per


def vortex_mesh(n, kind="tri", seed=None):
    """The periodic meshes of the study: kind "tri", an n x n jittered
    triangulation (2 n^2 cells); kind "voronoi", a Voronoi tessellation with
    n cells (the polygonal meshes of Table conv_0)."""
    if kind == "tri":
        return workloads.periodic_triangulation(n, BOX, BOX, seed=1006 if seed is None else seed)
    return workloads.periodic_voronoi(n, BOX, BOX, seed=1007 if seed is None else seed)


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


def errors(area, rho, T, rho_ref, T_ref):
    dr, dT = rho - rho_ref, T - T_ref
    return {"rho_L1": float((area * np.abs(dr)).sum()), "rho_L2": float(np.sqrt((area * dr * dr).sum())),
            "T_L1": float((area * np.abs(dT)).sum()), "T_L2": float(np.sqrt((area * dT * dT).sum()))}


def vortex_march(n, N=30, L=10.0, t_final=0.1, eps=1e-8, model="bgk", steps=None, cfl=0.4, order=2,
                 precision="fp64", scheme="ars222", seed=None, modes=None, conserve=True, penalty=1.0, mesh="tri"):
    """March the vortex to t_final on the periodic mesh vortex_mesh(n, mesh)
    with `steps` steps (default: the CFL step).  Returns (moments (rho, T) of
    the final state, area, barycentres, steps)."""
    import torch
    pts, tri = vortex_mesh(n, mesh, seed)
    area, bary, per = mesh_geometry(pts, tri)
    fvm = bz.Mesh(pts, tri, order=order, periodic=(BOX, BOX))
    if modes is None:
        modes = bz.Modes(bz.Grid(2, N, L), 0.0)
    modes.set_penalty(penalty)
    f0, _, _ = workloads.vortex_states(bary, N, L, 0.0, BOX, BOX)
    if steps is None:
        steps = max(1, math.ceil(t_final / time_step(area, per, N, L, cfl) - 1e-12))
    dt = t_final / steps
    ty = torch.float64 if precision == "fp64" else torch.float32
    a = torch.from_numpy(f0).to(device="cuda", dtype=ty).contiguous()
    b = torch.empty_like(a)
    for _ in range(steps):
        bz.imex_step_fv(modes, fvm, a, dt, eps, f_out=b, scheme=scheme, model=model, precision=precision,
                        conserve=conserve)
        a, b = b, a
    bz.check()
    return moments(a.double().cpu().numpy(), N, L), area, bary, steps


def space_study(sizes=(18, 36, 54, 72), N=30, L=10.0, t_final=0.1, eps=1e-8, model="bgk", **kw):
    """Table conv_0: one row per mesh (vortex_mesh(n, kw["mesh"]) for n in
    sizes), errors against the exact vortex."""
    rows = []
    for n in sizes:
        (rho, T), area, bary, steps = vortex_march(n, N, L, t_final, eps, model, **kw)
        _, rho_x, T_x = workloads.vortex_states(bary, N, L, t_final, BOX, BOX)
        rows.append({"n": n, "mesh": kw.get("mesh", "tri"), "cells": len(area), "h": float(np.sqrt(area).mean()),
                     "steps": steps, "dt": t_final / steps, **errors(area, rho, T, rho_x, T_x)})
    return rows


def time_study(eps, n_side=21, N=30, L=10.0, t_final=9e-3, dts=(1.8e-3, 9e-4, 4.5e-4, 2.25e-4), refine=32,
               model="boltzmann", **kw):
    """Tables conv_1e-3 to conv_1: one row per time step on one mesh
    (vortex_mesh(n_side, kw["mesh"])), errors against the run with a step
    `refine` times smaller than the smallest."""
    modes = kw.pop("modes", None) or bz.Modes(bz.Grid(2, N, L), 0.0)
    ref_steps = int(round(t_final / (min(dts) / refine)))
    (rho_r, T_r), area, _, _ = vortex_march(n_side, N, L, t_final, eps, model, steps=ref_steps, modes=modes, **kw)
    rows = []
    for dt in dts:
        steps = int(round(t_final / dt))
        (rho, T), _, _, _ = vortex_march(n_side, N, L, t_final, eps, model, steps=steps, modes=modes, **kw)
        rows.append({"eps": eps, "dt": t_final / steps, "steps": steps, "h": float(np.sqrt(area).mean()),
                     **errors(area, rho, T, rho_r, T_r)})
    return rows


def orders(rows, key, by="h"):
    """Observed orders log(e_k / e_{k+1}) / log(s_k / s_{k+1}) between
    consecutive rows, s the mesh size (by="h") or the time step (by="dt")."""
    return [math.log(r0[key] / r1[key]) / math.log(r0[by] / r1[by]) for r0, r1 in zip(rows, rows[1:])]


def main(argv=None):
    """Print a study as JSON lines: one per row, then the observed orders."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--study", choices=["space", "time"], default="space")
    ap.add_argument("--sizes", type=int, nargs="+", default=None,
                    help="triangulation sides (default 18 36 54 72) or Voronoi cell counts (678 2603 5739 10203)")
    ap.add_argument("--mesh", choices=["tri", "voronoi"], default="tri")
    ap.add_argument("--eps", type=float, nargs="+", default=None)
    ap.add_argument("--model", choices=["bgk", "boltzmann"], default=None)
    ap.add_argument("--order", type=int, default=2, help="1, 2 or 3 (CWENO of degree 0, 1, 2)")
    ap.add_argument("--scheme", choices=["ars222", "bpr343", "euler"], default=None,
                    help="IMEX scheme (default: bpr343 with --order 3, else ars222)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--penalty", type=float, default=1.0)
    a = ap.parse_args(argv)
    modes = bz.Modes(bz.Grid(2, 30, 10.0), 0.0)
    kw = dict(order=a.order, precision=a.precision, penalty=a.penalty, modes=modes, mesh=a.mesh,
              scheme=a.scheme or ("bpr343" if a.order == 3 else "ars222"))
    keys = ("rho_L1", "rho_L2", "T_L1", "T_L2")
    if a.study == "space":
        for eps in a.eps or [1e-8]:
            sizes = a.sizes or ([18, 36, 54, 72] if a.mesh == "tri" else [678, 2603, 5739, 10203])
            rows = space_study(sizes, eps=eps, model=a.model or "bgk", **kw)
            for r in rows:
                print(json.dumps(r), flush=True)
            print(json.dumps({"orders": {k: orders(rows, k) for k in keys}}), flush=True)
    else:
        for eps in a.eps or [1e-3, 1e-2, 1.0]:
            rows = time_study(eps, model=a.model or "boltzmann", **kw)
            for r in rows:
                print(json.dumps(r), flush=True)
            print(json.dumps({"eps": eps, "orders": {k: orders(rows, k, by="dt") for k in keys}}), flush=True)


if __name__ == "__main__":
    main()
