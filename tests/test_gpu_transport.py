"""Parity of the CUDA transport step (Sec. 3.2: CWENO reconstruction, Rusanov
fluxes; Sec. 3.4: the step coupled to the IMEX stages) with the FP64 oracle
(`oracle/fv.py`), through the C ABI.

Tolerance: a running-error bound of the residual.  L is a sum of face fluxes
scaled by 1/|P_i|; on a sliver cell the fluxes cancel to a small L, so its
rounding is set by the magnitudes summed, not by L.  The test evaluates the
residual once more with every quantity replaced by its magnitude,
  M_ik = (1/|P_i|) sum_e |e| ((|v_1| + L/4)|n_1| + (|v_2| + L/4)|n_2|) (|f_L| + |f_R|),
  |f_L| <= |f_i| + |x_f - x_b,i|_1 G_i,
with G_i the largest gradient any CWENO polynomial of the cell can take from
the magnitudes of its stencil (|R| applied to |f_j| + |f_i|; the weighted
combination is convex), and requires |L_gpu - L_oracle| <= 64 u M_ik
element by element, u = 2^-53 for BZ_FP64 and 2^-24 for BZ_FP32 (about 40
roundings lie on the path from the averages to L), plus the same sums of the
absolute rounding error of subnormal values (the Maxwellian tails of f fall
below the FP32 normal range).  The nodes v = -L + j dv carry an absolute
rounding error of a few u L (dv = 2L/N is inexact, and the two sides may
round the product differently; the node that is 0 in exact arithmetic need
not be 0 on either side), so the magnitude of a velocity component in M is
|v_c| + L/4, which leaves 16 u L for it inside 64 u M.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import as_input, bz_module, relerr, to_dev

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
U64, ETA64 = 2.0 ** -53, 2.0 ** -1075
U32, ETA32 = 2.0 ** -24, 2.0 ** -150


@pytest.fixture(scope="module")
def bz():
    return bz_module()


@pytest.fixture(scope="module")
def fvo():
    from oracle import fv
    return fv


def _tri(n_side, seed=7):
    return workloads.sod_triangulation(n_side=n_side, seed=seed)


def _mixed():
    n = 8
    g = np.linspace(0, 1, n + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    rng = np.random.default_rng(3)
    X[1:-1, 1:-1] += rng.uniform(-0.2, 0.2, (n - 1, n - 1)) / n
    Y[1:-1, 1:-1] += rng.uniform(-0.2, 0.2, (n - 1, n - 1)) / n
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    idx = np.arange((n + 1) ** 2).reshape(n + 1, n + 1)
    cells = []
    for a in range(n):
        for b in range(n):
            q = [idx[a, b], idx[a + 1, b], idx[a + 1, b + 1], idx[a, b + 1]]
            if (a + b) % 3 == 0:
                cells += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
            else:
                cells.append(q[::-1] if (a * b) % 2 else q)      # both orientations
    return pts, cells


def _magnitude(om, f, N, L, order, fvo, walls=None):
    """M_ik of the module docstring (at a wall face the inner state bounds the
    outgoing half and mu_mag M_w the incoming one, mu_mag formed from the
    magnitudes)."""
    v1, v2 = fvo.velocity_grid(N, L)
    af = np.abs(np.asarray(f, dtype=np.float64))
    n = len(om.cells)
    G = np.zeros_like(af)
    if order == 2:
        for i in range(n):
            sts = om.central_stencil_shifted(i)
            st = [j for j, _ in sts]
            A = np.array([om.bary[j] + s - om.bary[i] for j, s in sts])
            R = np.abs(np.linalg.inv(A.T @ A) @ A.T)
            gc = (R @ (af[st] + af[i])).max(axis=0)
            gs = []
            for a, sa, b, sb in om.sectors_shifted(i):
                Rs = np.abs(np.linalg.inv(np.array([om.bary[a] + sa - om.bary[i], om.bary[b] + sb - om.bary[i]])))
                gs.append((Rs @ np.stack([af[a] + af[i], af[b] + af[i]])).max(axis=0))
            cand = [gc] + gs
            if gs:
                cand.append((gc + 0.25 * sum(gs) / len(gs)) / 0.75)
            G[i] = np.max(cand, axis=0)
    M = np.zeros_like(af)
    for i, fl in enumerate(om.faces):
        for q, (j, ln, nx, ny, mx, my) in enumerate(fl):
            avn = ln * ((np.abs(v1) + 0.25 * L) * abs(nx) + (np.abs(v2) + 0.25 * L) * abs(ny))
            fl_ = af[i] + G[i] * (abs(mx - om.bary[i, 0]) + abs(my - om.bary[i, 1]))
            sh = om.face_shift[i][q]
            fr_ = fl_ if j < 0 else af[j] + G[j] * (abs(mx - sh[0] - om.bary[j, 0]) + abs(my - sh[1] - om.bary[j, 1]))
            wall = None if (walls is None or j >= 0) else walls.get(frozenset(om.face_vertices[i][q]))
            if wall is not None:
                vn = v1 * nx + v2 * ny
                mw = fvo.wall_maxwellian(v1, v2, *wall)
                mu = (fl_ * np.abs(vn))[vn > 0].sum() / (mw * np.abs(vn))[vn < 0].sum()
                fr_ = fl_ + mu * mw
            M[i] += avn * (fl_ + fr_)
        M[i] /= om.area[i]
    return M


def _check(got, want, om, fin, N, L, order, fvo, u, eta, walls=None):
    """err <= C (u M(|f|) + eta M(1)): eta is the absolute error of a rounding
    in the subnormal range (2^-150 in FP32), which the tails of f reach; M(1)
    carries it through the same sums.  C = 64; with walls, the mass balance of
    a wall face adds two sums over the N^2 velocities and a division (up to
    2 log2 N^2 + 8 roundings, in the incoming half of the face state), so
    C = 64 + 4 log2 N^2 + 16."""
    err = np.abs(got - want)
    C = 64 if walls is None else 64 + 4 * np.log2(N * N) + 16
    bound = C * (u * _magnitude(om, fin, N, L, order, fvo, walls) +
                 eta * _magnitude(om, np.ones_like(fin), N, L, order, fvo, walls))
    bad = [int((~np.isfinite(a)).sum()) for a in (got, want, bound)]
    assert bad == [0, 0, 0], ("non-finite values in got, want, bound", bad, np.argwhere(~np.isfinite(got))[:8])
    assert (err <= bound).all(), float((err / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("mesh_kind,N,jump", [("tri", 8, False), ("tri", 8, True), ("mixed", 8, False),
                                              ("tri", 32, False)])
def test_transport_fp64_matches_oracle(bz, fvo, order, mesh_kind, N, jump):
    Lv = 8.0
    pts, cells = _tri(10 if N == 32 else 16) if mesh_kind == "tri" else _mixed()
    om = fvo.Mesh(pts, cells)
    f = workloads.mesh_states(om.bary, N, Lv, jump=jump)
    m = bz.Mesh(pts, cells, order=order)
    assert m.n_cells == len(om.cells)
    g = bz.Grid(2, N, Lv)
    Lr = bz.transport_residual(m, g, to_dev(f, "fp64"), precision="fp64")
    bz.check()
    want = fvo.transport_residual(om, f, N, Lv, order=order)
    _check(Lr.cpu().numpy(), want, om, f, N, Lv, order, fvo, U64, ETA64)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("jump,N", [(False, 16), (True, 16), (False, 48)])
def test_transport_fp32_within_bound(bz, fvo, order, jump, N):
    """Triangles in FP32: at N = 16 (order 2) the persistent face-value passes
    with one block per cell (fewer cells than blocks of the grid); at N = 48
    the 2304 velocities span three velocity blocks per cell."""
    Lv = 8.0
    pts, cells = _tri(14)
    om = fvo.Mesh(pts, cells)
    f = workloads.mesh_states(om.bary, N, Lv, jump=jump)
    fin = as_input(f, "fp32")
    m = bz.Mesh(pts, cells, order=order)
    Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, "fp32"), precision="fp32")
    bz.check()
    want = fvo.transport_residual(om, fin, N, Lv, order=order)
    _check(Lr.double().cpu().numpy(), want, om, fin, N, Lv, order, fvo, U32, ETA32)


def test_transport_scalar_paths(bz, fvo):
    """N = 6 (4 does not divide N: one velocity per thread in the flux pass) and
    rows that start off a 16-byte boundary (one velocity per thread in both
    passes) give the oracle's result too."""
    import torch
    pts, cells = _tri(12)
    om = fvo.Mesh(pts, cells)
    m = bz.Mesh(pts, cells, order=2)
    for N in (6, 8):
        Lv = 6.0
        f = workloads.mesh_states(om.bary, N, Lv, jump=True)
        want = fvo.transport_residual(om, f, N, Lv, order=2)
        g = bz.Grid(2, N, Lv)
        buf = torch.zeros(f.size + 1, dtype=torch.float64, device="cuda")
        fd = buf[1:].view(f.shape)                        # 8-byte but not 16-byte aligned
        fd.copy_(torch.from_numpy(f))
        out = torch.zeros(f.size + 1, dtype=torch.float64, device="cuda")[1:].view(f.shape)
        for src, dst in ((to_dev(f, "fp64"), None), (fd, out)):
            Lr = bz.transport_residual(m, g, src, dst, precision="fp64")
            bz.check()
            _check(Lr.cpu().numpy(), want, om, f, N, Lv, 2, fvo, U64, ETA64)


def test_mesh_info_and_errors(bz):
    pts, cells = _tri(12)
    m = bz.Mesh(pts, cells, order=2)
    assert m.max_faces == 3 and m.order == 2
    assert 3 * m.n_cells == 2 * m.n_faces_interior + m.n_faces_boundary
    lib = bz.load()
    out = ctypes.c_void_p()
    xy = np.ascontiguousarray(pts, dtype=np.float64)
    ptr = np.array([0, 3], dtype=np.int64)
    bad = np.array([0, 1, len(pts)], dtype=np.int64)              # vertex out of range
    assert lib.build_fv_mesh(len(pts), xy.ctypes.data_as(ctypes.c_void_p), 1, ptr.ctypes.data_as(ctypes.c_void_p),
                             bad.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(out)) == bz.EINVAL
    flat = np.array([0, 1, 2], dtype=np.int64)
    line = np.ascontiguousarray([[0, 0], [1, 0], [2, 0]], dtype=np.float64)   # zero area
    assert lib.build_fv_mesh(3, line.ctypes.data_as(ctypes.c_void_p), 1, ptr.ctypes.data_as(ctypes.c_void_p),
                             flat.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(out)) == bz.EINVAL
    g3 = bz.Grid(3, 8, 8.0)
    import torch
    f = torch.zeros((m.n_cells, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(bz.BzError):
        bz.transport_residual(m, g3, f, precision="fp32")


def test_imex_step_fv_matches_oracle(bz, fvo):
    """ARS(2,2,2) with transport: the oracle composes the stages, stage l taking
    the residuals of the stage values 0..l-1 (each computed by oracle/fv.py)."""
    import oracle
    N, Lv, dt, eps = 8, 6.0, 2e-3, 5e-2
    pts, cells = _tri(10)
    om = fvo.Mesh(pts, cells)
    f = workloads.mesh_states(om.bary, N, Lv, jump=True)
    k = oracle.Kernel(2, N, Lv, 0.0)
    Lres = np.zeros((3,) + f.shape)
    for l in range(2):
        _, F, _, _ = k.imex_step(f, dt, eps, Lres=Lres, stages=True)
        Lres[l] = fvo.transport_residual(om, F[l], N, Lv, order=2)
    want = k.imex_step(f, dt, eps, Lres=Lres)
    m = bz.Mesh(pts, cells, order=2)
    md = bz.Modes(bz.Grid(2, N, Lv), 0.0)
    got = bz.imex_step_fv(md, m, to_dev(f, "fp64"), dt, eps, precision="fp64")
    bz.check()
    assert relerr(got.cpu().numpy(), want) < TOL64
    # and the fast collision form inside the same step
    kf = oracle.FastKernel(N, Lv, 8)
    Lres[:] = 0
    for l in range(2):
        _, F, _, _ = kf.imex_step(f, dt, eps, Lres=Lres, stages=True)
        Lres[l] = fvo.transport_residual(om, F[l], N, Lv, order=2)
    want_f = kf.imex_step(f, dt, eps, Lres=Lres)
    got_f = bz.imex_step_fv(bz.FastModes(bz.Grid(2, N, Lv), 8), m, to_dev(f, "fp64"), dt, eps, precision="fp64")
    bz.check()
    assert relerr(got_f.cpu().numpy(), want_f) < TOL64


def test_full_mesh_fp32_sampled(bz, fvo):
    """The 19802-triangle mesh with the 32^2 grid (the measured configuration):
    every cell against the oracle within the FP32 bound."""
    N, Lv = 32, 10.0
    pts, cells = workloads.sod_triangulation()
    om = fvo.Mesh(pts, cells)
    f = workloads.mesh_states(om.bary, N, Lv, jump=True)
    fin = as_input(f, "fp32")
    m = bz.Mesh(pts, cells, order=2)
    Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, "fp32"), precision="fp32")
    bz.check()
    want = fvo.transport_residual(om, fin, N, Lv, order=2)
    _check(Lr.double().cpu().numpy(), want, om, fin, N, Lv, 2, fvo, U32, ETA32)


def _walls(om, rng=None):
    """Every boundary edge a wall: temperatures and velocities vary by edge."""
    rng = rng or np.random.default_rng(0)
    edges, params, walls = [], [], {}
    for i, fl in enumerate(om.faces):
        for q, fc in enumerate(fl):
            if fc[0] < 0:
                a, b = om.face_vertices[i][q]
                p = (float(rng.uniform(0.6, 1.4)), float(rng.uniform(-0.3, 0.3)), float(rng.uniform(-0.3, 0.3)))
                edges.append((a, b))
                params.append(p)
                walls[frozenset((a, b))] = p
    return np.array(edges), np.array(params), walls


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [1, 2])
def test_walls_match_oracle(bz, fvo, precision, order):
    N, Lv = 8, 6.0
    pts, cells = _tri(12)
    om = fvo.Mesh(pts, cells)
    edges, params, walls = _walls(om)
    f = workloads.mesh_states(om.bary, N, Lv, jump=True)
    fin = as_input(f, precision)
    m = bz.Mesh(pts, cells, order=order)
    m.set_walls(edges, params)
    Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, precision), precision=precision)
    bz.check()
    want = fvo.transport_residual(om, fin, N, Lv, order=order, walls=walls)
    u, eta = (U64, ETA64) if precision == "fp64" else (U32, ETA32)
    _check(Lr.double().cpu().numpy(), want, om, fin, N, Lv, order, fvo, u, eta, walls)
    if precision == "fp64":     # a closed box: no mass crosses the walls
        tot = (om.area[:, None] * Lr.cpu().numpy()).sum()
        assert abs(tot) < 1e-12 * (om.area[:, None] * np.abs(want)).sum()


def test_walls_imex_step_and_limits(bz, fvo):
    """The coupled step with walls against the oracle's composed stages; walls
    removed again give the transmissive result; unsupported grids and edges
    that are not boundary edges are refused."""
    import oracle
    N, Lv, dt, eps = 8, 6.0, 2e-3, 5e-2
    pts, cells = _tri(10)
    om = fvo.Mesh(pts, cells)
    edges, params, walls = _walls(om, np.random.default_rng(5))
    f = workloads.mesh_states(om.bary, N, Lv, jump=True)
    k = oracle.Kernel(2, N, Lv, 0.0)
    Lres = np.zeros((3,) + f.shape)
    for l in range(2):
        _, F, _, _ = k.imex_step(f, dt, eps, Lres=Lres, stages=True)
        Lres[l] = fvo.transport_residual(om, F[l], N, Lv, order=2, walls=walls)
    want = k.imex_step(f, dt, eps, Lres=Lres)
    m = bz.Mesh(pts, cells, order=2)
    m.set_walls(edges, params)
    got = bz.imex_step_fv(bz.Modes(bz.Grid(2, N, Lv), 0.0), m, to_dev(f, "fp64"), dt, eps, precision="fp64")
    bz.check()
    assert relerr(got.cpu().numpy(), want) < TOL64
    m.set_walls([], [])
    L0 = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, "fp64"), precision="fp64").cpu().numpy()
    _check(L0, fvo.transport_residual(om, f, N, Lv, order=2), om, f, N, Lv, 2, fvo, U64, ETA64)
    m.set_walls(edges, params)
    import torch
    with pytest.raises(bz.BzError):          # 4 does not divide N
        bz.transport_residual(m, bz.Grid(2, 6, Lv), torch.zeros((m.n_cells, 36), dtype=torch.float64,
                                                                 device="cuda"), precision="fp64")
    inner = next((om.face_vertices[i][q] for i, fl in enumerate(om.faces) for q, fc in enumerate(fl) if fc[0] >= 0))
    with pytest.raises(bz.BzError):
        m.set_walls([inner], [(1.0, 0.0, 0.0)])


def _periodic(n_side, seed=1006):
    return workloads.periodic_triangulation(n_side, 10.0, 10.0, seed=seed)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("n_side,per", [(8, (10.0, 10.0)), (8, (10.0, 0.0)), (8, (0.0, 10.0)), (3, (10.0, 10.0))])
def test_periodic_fp64_matches_oracle(bz, fvo, order, n_side, per):
    """Periodic in both directions, in one direction (the other boundary
    transmissive) and a torus 3 cells wide, where a stencil holds several
    copies of one cell; the isentropic-vortex states."""
    N, Lv = 8, 8.0
    pts, tri = _periodic(n_side)
    om = fvo.Mesh(pts, tri, periodic=per)
    f, _, _ = workloads.vortex_states(om.bary, N, Lv)
    m = bz.Mesh(pts, tri, order=order, periodic=per)
    nb = sum(1 for fl in om.faces for fc in fl if fc[0] < 0)
    assert m.n_faces_boundary == nb and 3 * m.n_cells == 2 * m.n_faces_interior + nb
    if per == (10.0, 10.0):
        assert nb == 0
    import torch
    out = torch.full(f.shape, float("nan"), dtype=torch.float64, device="cuda")   # every element is written
    Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, "fp64"), out, precision="fp64")
    bz.check()
    want = fvo.transport_residual(om, f, N, Lv, order=order)
    _check(Lr.cpu().numpy(), want, om, f, N, Lv, order, fvo, U64, ETA64)


@pytest.mark.parametrize("order", [1, 2])
def test_periodic_fp32_within_bound(bz, fvo, order):
    N, Lv = 16, 8.0
    pts, tri = _periodic(12, seed=11)
    om = fvo.Mesh(pts, tri, periodic=(10.0, 10.0))
    f, _, _ = workloads.vortex_states(om.bary, N, Lv, t=3.3)
    fin = as_input(f, "fp32")
    m = bz.Mesh(pts, tri, order=order, periodic=(10.0, 10.0))
    import torch
    out = torch.full(f.shape, float("nan"), dtype=torch.float32, device="cuda")
    Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, "fp32"), out, precision="fp32")
    bz.check()
    want = fvo.transport_residual(om, fin, N, Lv, order=order)
    _check(Lr.double().cpu().numpy(), want, om, fin, N, Lv, order, fvo, U32, ETA32)


def test_periodic_conserves_mass_at_scale(bz, fvo):
    """On the torus no mass leaves the box: sum_i |P_i| L_ik vanishes for every
    velocity up to rounding, bounded by the same sums of magnitudes as one
    element (48 x 48 periodic triangulation, 4608 cells, the 30^2 grid of the
    vortex study, both precisions); in FP64 every cell against the oracle at
    that size."""
    N, Lv = 30, 10.0
    pts, tri = _periodic(48)
    m = bz.Mesh(pts, tri, order=2, periodic=(10.0, 10.0))
    om = fvo.Mesh(pts, tri, periodic=(10.0, 10.0))
    f, _, _ = workloads.vortex_states(om.bary, N, Lv)
    M1 = _magnitude(om, np.ones_like(f), N, Lv, 2, fvo)
    for precision, u, eta in (("fp64", U64, ETA64), ("fp32", U32, ETA32)):
        fin = as_input(f, precision)
        Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, precision), precision=precision)
        bz.check()
        got = Lr.double().cpu().numpy()
        Mf = _magnitude(om, fin, N, Lv, 2, fvo)
        bound = 64 * (u * Mf + eta * M1)
        assert (np.abs(om.area @ got) <= om.area @ bound).all()
        if precision == "fp64":
            err = np.abs(got - fvo.transport_residual(om, fin, N, Lv, order=2))
            assert (err <= bound).all(), float((err / np.maximum(bound, 1e-300)).max())


def test_periodic_imex_step_fv_matches_oracle(bz, fvo):
    import oracle
    N, Lv, dt, eps = 16, 8.0, 2e-3, 5e-2
    pts, tri = _periodic(5)
    om = fvo.Mesh(pts, tri, periodic=(10.0, 10.0))
    f, _, _ = workloads.vortex_states(om.bary, N, Lv)
    k = oracle.Kernel(2, N, Lv, 0.0)
    Lres = np.zeros((3,) + f.shape)
    for l in range(2):
        _, F, _, _ = k.imex_step(f, dt, eps, Lres=Lres, stages=True)
        Lres[l] = fvo.transport_residual(om, F[l], N, Lv, order=2)
    want = k.imex_step(f, dt, eps, Lres=Lres)
    m = bz.Mesh(pts, tri, order=2, periodic=(10.0, 10.0))
    got = bz.imex_step_fv(bz.Modes(bz.Grid(2, N, Lv), 0.0), m, to_dev(f, "fp64"), dt, eps, precision="fp64")
    bz.check()
    assert relerr(got.cpu().numpy(), want) < TOL64


def test_periodic_mesh_errors(bz):
    pts, tri = _periodic(4)
    lib = bz.load()
    out = ctypes.c_void_p()
    xy = np.ascontiguousarray(pts, dtype=np.float64)
    ptr = np.ascontiguousarray(np.arange(0, 3 * len(tri) + 1, 3), dtype=np.int64)
    vtx = np.ascontiguousarray(np.asarray(tri, dtype=np.int64).ravel())
    args = (len(pts), xy.ctypes.data_as(ctypes.c_void_p), len(tri), ptr.ctypes.data_as(ctypes.c_void_p),
            vtx.ctypes.data_as(ctypes.c_void_p), 2)
    for Lx, Ly in ((-1.0, 10.0), (10.0, float("inf")), (float("nan"), 0.0)):
        assert lib.build_fv_mesh_periodic(*args, Lx, Ly, ctypes.byref(out)) == bz.EINVAL
    p2, t2 = _periodic(2)          # 2 cells wide: two edges join the same pair of periodic vertices
    with pytest.raises(bz.BzError):
        bz.Mesh(p2, t2, order=2, periodic=(10.0, 10.0))
    m = bz.Mesh(pts, tri, order=2, periodic=(0.0, 0.0))      # no period: the plain mesh
    assert m.n_faces_boundary == 16


def test_isentropic_vortex_time_order(bz):
    """Sec. 4.1, Table conv_1e-2: the Boltzmann model at eps = 1e-2 on one
    periodic triangulation with h = 1/3, t_f = 9e-3, steps 1.8e-3 .. 2.25e-4
    against a 32 times finer step: second order in time, with density errors
    of the size the paper prints (2.6e-6, 6.4e-7, 1.6e-7 at the three
    smaller steps)."""
    from paper_2103_14890_gb300 import convergence
    rows = convergence.time_study(1e-2)
    assert abs(rows[0]["h"] - 1 / 3) < 0.02
    for key in ("rho_L1", "rho_L2", "T_L1", "T_L2"):
        o = convergence.orders(rows, key, by="dt")
        assert min(o) > 1.85, (key, o)
    assert 5e-7 < rows[1]["rho_L1"] < 5e-6 and 3e-8 < rows[3]["rho_L1"] < 3e-7, rows


def test_isentropic_vortex_space_time_limit(bz):
    """Sec. 4.1, Table conv_0 (eps -> 0) on periodic Voronoi tessellations
    with h = 0.38, 0.20, 0.13: errors against the exact advected vortex fall
    at close to second order (measured in L1: 1.78 and 1.90 for the density,
    2.05 and 2.43 for the temperature; the paper prints 2.5, 2.1 and 2.6,
    2.4) and well below the first-order scheme's."""
    from paper_2103_14890_gb300 import convergence
    modes = bz.Modes(bz.Grid(2, 30, 10.0), 0.0)
    rows = convergence.space_study((678, 2603, 5739), modes=modes, mesh="voronoi")
    for key, lo in (("rho_L1", 1.6), ("rho_L2", 1.6), ("T_L1", 1.8), ("T_L2", 1.8)):
        o = convergence.orders(rows, key)
        assert min(o) > lo, (key, o, rows)
    assert rows[0]["rho_L1"] < 0.1 and abs(rows[0]["h"] - 0.384) < 0.01
    first = convergence.space_study((5739,), modes=modes, order=1, mesh="voronoi")[0]
    assert first["rho_L1"] > 4 * rows[-1]["rho_L1"] and first["T_L1"] > 4 * rows[-1]["T_L1"]


@pytest.mark.parametrize("order", [1, 2])
def test_periodic_voronoi_matches_oracle(bz, fvo, order):
    """Polygons of 4 to 8 vertices (a periodic Voronoi tessellation, the
    meshes of Table conv_0): FP64 and FP32 against the oracle, and the
    coupled step."""
    import torch
    N, Lv = 16, 8.0
    pts, cells = workloads.periodic_voronoi(60, seed=12)
    om = fvo.Mesh(pts, cells, periodic=(10.0, 10.0))
    m = bz.Mesh(pts, cells, order=order, periodic=(10.0, 10.0))
    assert m.n_faces_boundary == 0 and m.max_faces == max(len(c) for c in cells) > 6
    f, _, _ = workloads.vortex_states(om.bary, N, Lv, t=1.7)
    for precision, u, eta in (("fp64", U64, ETA64), ("fp32", U32, ETA32)):
        fin = as_input(f, precision)
        dt = torch.float64 if precision == "fp64" else torch.float32
        out = torch.full(f.shape, float("nan"), dtype=dt, device="cuda")
        Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, precision), out, precision=precision)
        bz.check()
        _check(Lr.double().cpu().numpy(), fvo.transport_residual(om, fin, N, Lv, order=order), om, fin, N, Lv,
               order, fvo, u, eta)
    import oracle
    k = oracle.Kernel(2, N, Lv, 0.0)
    Lres = np.zeros((3,) + f.shape)
    for l in range(2):
        _, F, _, _ = k.imex_step(f, 2e-3, 5e-2, Lres=Lres, stages=True)
        Lres[l] = fvo.transport_residual(om, F[l], N, Lv, order=order)
    want = k.imex_step(f, 2e-3, 5e-2, Lres=Lres)
    got = bz.imex_step_fv(bz.Modes(bz.Grid(2, N, Lv), 0.0), m, to_dev(f, "fp64"), 2e-3, 5e-2, precision="fp64")
    bz.check()
    assert relerr(got.cpu().numpy(), want) < TOL64


def _magnitude3(om, f, N, L, fvo, walls=None):
    """M_ik of the module docstring for the degree-2 reconstruction: each
    coefficient bounded by the largest magnitude any CWENO polynomial of the
    cell can give it (|R| applied to |f_j| + |f_i|; the weighted combination
    is convex), the face values at the Gauss points by |f_i| + sum_l G_l
    |phi_l|."""
    v1, v2 = fvo.velocity_grid(N, L)
    af = np.abs(np.asarray(f, dtype=np.float64))
    n = len(om.cells)
    G = np.zeros((n, 5, af.shape[1]))
    basis = [fvo.quadratic_basis(om, i) for i in range(n)]
    for i in range(n):
        xb, h, mu = basis[i]
        sub = np.array([0.0, 0.0, mu[2], mu[3], mu[4]])
        st = om.central_stencil_shifted(i, count=11)
        A = np.array([fvo._quadratic_means(om.xy[om.cells[j]] + s, xb, h) - sub for j, s in st])
        R = np.abs(np.linalg.solve(A.T @ A, A.T))
        gc = R @ (af[[j for j, _ in st]] + af[i])
        polys = []
        for a, sa, b, sb in om.sectors_shifted(i):
            Rs = np.abs(np.linalg.inv(np.array([(om.bary[a] + sa - xb) / h, (om.bary[b] + sb - xb) / h])))
            p = np.zeros_like(gc)
            p[:2] = Rs @ np.stack([af[a] + af[i], af[b] + af[i]])
            polys.append(p)
        cand = [gc] + polys
        if polys:
            cand.append((gc + 0.25 * sum(polys) / len(polys)) / 0.75)
        G[i] = np.max(cand, axis=0)
    M = np.zeros_like(af)
    for i, c in enumerate(om.cells):
        for q, (j, ln, nx, ny, mx, my) in enumerate(om.faces[i]):
            avn = ln * ((np.abs(v1) + 0.25 * L) * abs(nx) + (np.abs(v2) + 0.25 * L) * abs(ny))
            xa, xe = om.xy[c[q]], om.xy[c[(q + 1) % len(c)]]
            wall = None if (walls is None or j >= 0) else walls.get(frozenset(om.face_vertices[i][q]))
            for t in fvo.GAUSS2:
                x = xa + t * (xe - xa)
                fl_ = af[i] + np.abs(fvo.quadratic_phi(x, *basis[i])) @ G[i]
                fr_ = fl_ if j < 0 else af[j] + np.abs(fvo.quadratic_phi(x - om.face_shift[i][q], *basis[j])) @ G[j]
                if wall is not None:
                    vn = v1 * nx + v2 * ny
                    mw = fvo.wall_maxwellian(v1, v2, *wall)
                    fr_ = fl_ + (fl_ * np.abs(vn))[vn > 0].sum() / (mw * np.abs(vn))[vn < 0].sum() * mw
                M[i] += 0.5 * avn * (fl_ + fr_)
        M[i] /= om.area[i]
    return M


def _check3(got, want, om, fin, N, L, fvo, u, eta, walls=None):
    """As _check (the wall constant included) with the degree-2 magnitudes."""
    err = np.abs(got - want)
    C = 64 if walls is None else 64 + 4 * np.log2(N * N) + 16
    bound = C * (u * _magnitude3(om, fin, N, L, fvo, walls) +
                 eta * _magnitude3(om, np.ones_like(fin), N, L, fvo, walls))
    assert np.isfinite(got).all()
    assert (err <= bound).all(), float((err / np.maximum(bound, 1e-300)).max())


def _order3_meshes():
    pts, tri = _tri(12)
    vp, vc = workloads.periodic_voronoi(60, seed=12)
    pp, pt = _periodic(8)
    return {"tri": (pts, tri, None), "mixed": _mixed() + (None,), "voronoi_periodic": (vp, vc, (10.0, 10.0)),
            "tri_periodic": (pp, pt, (10.0, 10.0))}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["tri", "mixed", "voronoi_periodic", "tri_periodic"])
def test_order3_matches_oracle(bz, fvo, kind, precision):
    """CWENO of degree 2 with two Gauss points per face (the third-order
    scheme) against the oracle on triangles, a mixed mesh and periodic
    triangle and Voronoi meshes, within the running-error bound."""
    import torch
    pts, cells, per = _order3_meshes()[kind]
    N, Lv = 8, 8.0
    om = fvo.Mesh(pts, cells, periodic=per)
    if per is None:
        f = workloads.mesh_states(om.bary, N, Lv, jump=True)
    else:
        f, _, _ = workloads.vortex_states(om.bary, N, Lv, t=0.7)
    fin = as_input(f, precision)
    m = bz.Mesh(pts, cells, order=3, periodic=per)
    assert m.order == 3
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = torch.full(f.shape, float("nan"), dtype=dt, device="cuda")
    Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, precision), out, precision=precision)
    bz.check()
    want = fvo.transport_residual(om, fin, N, Lv, order=3)
    u, eta = (U64, ETA64) if precision == "fp64" else (U32, ETA32)
    _check3(Lr.double().cpu().numpy(), want, om, fin, N, Lv, fvo, u, eta)


def test_order3_imex_step_and_limits(bz, fvo):
    """BPR(3,4,3) with the degree-2 transport (the paper's third-order
    scheme) against the oracle's composed stages."""
    import oracle
    N, Lv, dt, eps = 8, 6.0, 2e-3, 5e-2
    pts, cells = _tri(10)
    om = fvo.Mesh(pts, cells)
    f = workloads.mesh_states(om.bary, N, Lv, jump=True)
    k = oracle.Kernel(2, N, Lv, 0.0)
    s = bz.STAGES["bpr343"]
    Lres = np.zeros((s,) + f.shape)
    for l in range(s - 1):
        _, F, _, _ = k.imex_step(f, dt, eps, scheme="bpr343", Lres=Lres, stages=True)
        Lres[l] = fvo.transport_residual(om, F[l], N, Lv, order=3)
    want = k.imex_step(f, dt, eps, scheme="bpr343", Lres=Lres)
    m = bz.Mesh(pts, cells, order=3)
    got = bz.imex_step_fv(bz.Modes(bz.Grid(2, N, Lv), 0.0), m, to_dev(f, "fp64"), dt, eps, scheme="bpr343",
                          precision="fp64")
    bz.check()
    assert relerr(got.cpu().numpy(), want) < TOL64


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["tri", "mixed"])
def test_order3_walls_match_oracle(bz, fvo, kind, precision):
    """Walls with full accommodation on an order-3 mesh (the balance of
    eq. MU at each Gauss point): the residual against the oracle, mass
    conservation in the closed box, and the coupled BPR(3,4,3) step."""
    N, Lv = 8, 6.0
    pts, cells = _tri(12) if kind == "tri" else _mixed()
    om = fvo.Mesh(pts, cells)
    edges, params, walls = _walls(om)
    f = workloads.mesh_states(om.bary, N, Lv, jump=True)
    fin = as_input(f, precision)
    m = bz.Mesh(pts, cells, order=3)
    m.set_walls(edges, params)
    Lr = bz.transport_residual(m, bz.Grid(2, N, Lv), to_dev(f, precision), precision=precision)
    bz.check()
    want = fvo.transport_residual(om, fin, N, Lv, order=3, walls=walls)
    u, eta = (U64, ETA64) if precision == "fp64" else (U32, ETA32)
    _check3(Lr.double().cpu().numpy(), want, om, fin, N, Lv, fvo, u, eta, walls)
    if precision == "fp64":
        tot = (om.area[:, None] * Lr.cpu().numpy()).sum()
        assert abs(tot) < 1e-12 * (om.area[:, None] * np.abs(want)).sum()
        import oracle
        k = oracle.Kernel(2, N, Lv, 0.0)
        s = bz.STAGES["bpr343"]
        Lres = np.zeros((s,) + f.shape)
        for l in range(s - 1):
            _, F, _, _ = k.imex_step(f, 2e-3, 5e-2, scheme="bpr343", Lres=Lres, stages=True)
            Lres[l] = fvo.transport_residual(om, F[l], N, Lv, order=3, walls=walls)
        want_s = k.imex_step(f, 2e-3, 5e-2, scheme="bpr343", Lres=Lres)
        got = bz.imex_step_fv(bz.Modes(bz.Grid(2, N, Lv), 0.0), m, to_dev(f, "fp64"), 2e-3, 5e-2,
                              scheme="bpr343", precision="fp64")
        bz.check()
        assert relerr(got.cpu().numpy(), want_s) < TOL64


def test_isentropic_vortex_third_order(bz):
    """The third-order scheme (CWENO of degree 2, BPR(3,4,3)): Table conv_1e-2's
    O3 column, third order in time for the density (the paper prints 2.9, 2.9;
    errors 5.1e-8, 6.8e-9, 8.8e-10), and the space-time limit on Voronoi
    meshes, faster than the second-order scheme on the finer pair."""
    from paper_2103_14890_gb300 import convergence
    modes = bz.Modes(bz.Grid(2, 30, 10.0), 0.0)
    rows = convergence.time_study(1e-2, order=3, scheme="bpr343", modes=modes)
    o = convergence.orders(rows, "rho_L1", by="dt")
    assert min(o) > 2.8, (o, rows)
    assert 5e-9 < rows[1]["rho_L1"] < 1e-7 and 5e-11 < rows[3]["rho_L1"] < 2e-9, rows
    sp = convergence.space_study((2603, 5739), modes=modes, order=3, scheme="bpr343", mesh="voronoi")
    o3 = convergence.orders(sp, "rho_L1")[0]
    assert o3 > 2.3 and sp[-1]["rho_L1"] < 7e-3, (o3, sp)


def test_order3_scalar_paths(bz, fvo):
    """Degree 2 with one velocity per thread on a triangle mesh: N = 6 (4 does
    not divide N) and rows that start off a 16-byte boundary."""
    import torch
    pts, cells = _tri(10)
    om = fvo.Mesh(pts, cells)
    m = bz.Mesh(pts, cells, order=3)
    for N in (6, 8):
        Lv = 6.0
        f = workloads.mesh_states(om.bary, N, Lv, jump=True)
        want = fvo.transport_residual(om, f, N, Lv, order=3)
        g = bz.Grid(2, N, Lv)
        buf = torch.zeros(f.size + 1, dtype=torch.float64, device="cuda")
        fd = buf[1:].view(f.shape)
        fd.copy_(torch.from_numpy(f))
        out = torch.full((f.size + 1,), float("nan"), dtype=torch.float64, device="cuda")[1:].view(f.shape)
        for src, dst in ((to_dev(f, "fp64"), None), (fd, out)):
            Lr = bz.transport_residual(m, g, src, dst, precision="fp64")
            bz.check()
            _check3(Lr.cpu().numpy(), want, om, f, N, Lv, fvo, U64, ETA64)
