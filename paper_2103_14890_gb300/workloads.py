"""Seeded synthetic inputs for the collision operator and the IMEX step.

This module only synthesises input data (sums of Gaussians sampled on the
velocity grid, noise, a seeded triangulation).  It holds none of the
operator's arithmetic: no transforms, no kernel modes, no moments.  Both the
CUDA path and the CPU oracle consume what it returns.

The recipes follow the paper's workloads (2-D velocity grids of 16^2/32^2
points on boxes [-8,8]^2 and [-10,10]^2, Maxwell-molecule and hard-sphere
kernels, the states of the explosion problem of Sec. 4.2) and are the ones
the benchmark and the parity tests use.
"""
import math

import numpy as np

POLYTROPIC_GAMMA = 2.0   # gas polytropic index used for Mach numbers (Sec. 4)


def velocity_nodes(N, L):
    """Periodic grid v_j = -L + j * 2L/N, j = 0..N-1."""
    return -L + (2.0 * L / N) * np.arange(N)


def _gaussian(dim, N, L, rho, u, theta):
    """rho (2 pi theta)^(-d/2) exp(-|v-u|^2 / (2 theta)) on the grid; rho, theta
    of shape (n,), u of shape (n, d).  Returns (n, N^d) float64."""
    v = velocity_nodes(N, L)
    n = len(rho)
    r2 = np.zeros((n,) + (N,) * dim)
    for i in range(dim):
        shape = [1] * (dim + 1)
        shape[i + 1] = N
        vi = v.reshape(shape)
        r2 = r2 + (vi - u[:, i].reshape((n,) + (1,) * dim)) ** 2
    th = theta.reshape((n,) + (1,) * dim)
    out = rho.reshape((n,) + (1,) * dim) / (2.0 * math.pi * th) ** (dim / 2.0) * np.exp(-r2 / (2.0 * th))
    return out.reshape(n, N ** dim)


def bi_maxwellian(n_cells, dim, N, L, seed, noise=0.0):
    """Each cell: sum of two Gaussians with density U[0.5,2], mean velocity
    U[-1,1]^d and temperature U[0.5,1.5]; optionally times (1 + noise*xi),
    xi ~ U[-1,1] per grid point (multiplicative, so f stays >= 0)."""
    rng = np.random.default_rng(seed)
    f = np.zeros((n_cells, N ** dim))
    for _ in range(2):
        rho = rng.uniform(0.5, 2.0, n_cells)
        u = rng.uniform(-1.0, 1.0, (n_cells, dim))
        th = rng.uniform(0.5, 1.5, n_cells)
        f += _gaussian(dim, N, L, rho, u, th)
    if noise:
        f *= 1.0 + noise * rng.uniform(-1.0, 1.0, f.shape)
    return f


def shifted_maxwellians(n_cells, dim, N, L, seed, mach_max=3.0):
    """Each cell: two Gaussians, each drifting at Mach U[0, mach_max] (sound
    speed sqrt(gamma theta), gamma = 2) in a uniform random direction, with
    temperature U[0.5,1.5] and density U[0.5,2]."""
    rng = np.random.default_rng(seed)
    f = np.zeros((n_cells, N ** dim))
    for _ in range(2):
        rho = rng.uniform(0.5, 2.0, n_cells)
        th = rng.uniform(0.5, 1.5, n_cells)
        mach = rng.uniform(0.0, mach_max, n_cells)
        direc = rng.normal(size=(n_cells, dim))
        direc /= np.linalg.norm(direc, axis=1, keepdims=True)
        u = direc * (mach * np.sqrt(POLYTROPIC_GAMMA * th))[:, None]
        f += _gaussian(dim, N, L, rho, u, th)
    return f


def single_maxwellian(n_cells, dim, N, L, seed):
    """Near-equilibrium cells: one Gaussian per cell (same parameter ranges)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, n_cells)
    u = rng.uniform(-1.0, 1.0, (n_cells, dim))
    th = rng.uniform(0.5, 1.5, n_cells)
    return _gaussian(dim, N, L, rho, u, th)


def bkw_initial(N, L, t=0.0):
    """The 2-D BKW profile of Sec. 4.1 at time t (closed form, used as data)."""
    v = velocity_nodes(N, L)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    r2 = V1 ** 2 + V2 ** 2
    S = 1.0 - math.exp(-t / 8.0) / 2.0
    f = np.exp(-r2 / (2 * S)) / (2 * math.pi * S ** 2) * (2 * S - 1 + (1 - S) / (2 * S) * r2)
    return f.reshape(1, N * N)


def sod_triangulation(n_side=100, seed=1004, jitter=0.3):
    """Jittered n_side x n_side lattice in [0,1]^2 (interior nodes moved by up
    to jitter x spacing, boundary nodes clipped to the square), triangulated.
    Returns the vertices (n_vtx, 2) and the triangles (n_tri, 3) as vertex
    indices.  Uses scipy's Delaunay when available, else the structured
    diagonal split of every lattice square."""
    rng = np.random.default_rng(seed)
    hs = 1.0 / (n_side - 1)
    g = np.linspace(0.0, 1.0, n_side)
    X, Y = np.meshgrid(g, g, indexing="ij")
    X = X + rng.uniform(-jitter, jitter, X.shape) * hs
    Y = Y + rng.uniform(-jitter, jitter, Y.shape) * hs
    X = np.clip(X, 0.0, 1.0)
    Y = np.clip(Y, 0.0, 1.0)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    try:
        from scipy.spatial import Delaunay
        tri = Delaunay(pts).simplices
    except Exception:  # structured split of every lattice square into two triangles
        idx = np.arange(n_side * n_side).reshape(n_side, n_side)
        a = idx[:-1, :-1].ravel(); b = idx[1:, :-1].ravel()
        c = idx[:-1, 1:].ravel(); d = idx[1:, 1:].ravel()
        tri = np.concatenate([np.stack([a, b, d], 1), np.stack([a, d, c], 1)])
    return pts, np.ascontiguousarray(tri, dtype=np.int64)


def periodic_triangulation(n_side, Lx=10.0, Ly=10.0, seed=1006, jitter=0.25):
    """Triangulated jittered lattice of the periodic box [0,Lx] x [0,Ly]: the
    n_side x n_side nodes of the torus are jittered (by up to jitter x spacing)
    and repeated with the periods, so the left and right (bottom and top)
    boundaries are translates of each other; every lattice quadrilateral is
    split along a randomly chosen diagonal.  Returns the vertices
    ((n_side + 1)^2, 2) and the triangles (2 n_side^2, 3)."""
    rng = np.random.default_rng(seed)
    n = n_side
    hx, hy = Lx / n, Ly / n
    jx = rng.uniform(-jitter, jitter, (n, n)) * hx
    jy = rng.uniform(-jitter, jitter, (n, n)) * hy
    a = np.arange(n + 1)
    A, B = np.meshgrid(a, a, indexing="ij")
    X = A * hx + jx[A % n, B % n]
    Y = B * hy + jy[A % n, B % n]
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    idx = np.arange((n + 1) ** 2).reshape(n + 1, n + 1)
    flip = rng.uniform(size=(n, n)) < 0.5
    tri = []
    for i in range(n):
        for j in range(n):
            p0, p1, p2, p3 = idx[i, j], idx[i + 1, j], idx[i + 1, j + 1], idx[i, j + 1]
            if flip[i, j]:
                tri += [(p0, p1, p2), (p0, p2, p3)]
            else:
                tri += [(p0, p1, p3), (p1, p2, p3)]
    return pts, np.asarray(tri, dtype=np.int64)


def periodic_voronoi(n_cells, Lx=10.0, Ly=10.0, seed=1007, lloyd=6, max_vertices=8):
    """Voronoi tessellation of the periodic box [0,Lx] x [0,Ly] (the polygonal
    meshes of Sec. 4.1): n_cells seeded random generators, moved `lloyd`
    times to the centroids of their cells (Lloyd's iteration, which makes the
    cells close to hexagons; continued until no cell has more than
    max_vertices vertices), the diagram computed on the 3 x 3 tiling of the
    box and the cells of the middle copy kept.  A vertex that lies outside
    the box is the periodic image of one used by a cell on the other side;
    the mesh joins them through the periods.  Returns the vertices (m, 2) and
    the cells (lists of vertex indices, counter-clockwise)."""
    from scipy.spatial import Voronoi
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.0, 1.0, (n_cells, 2)) * [Lx, Ly]
    shifts = np.array([(a * Lx, b * Ly) for a in (-1, 0, 1) for b in (-1, 0, 1)])
    mid = 4                                                  # index of the (0, 0) shift

    def diagram(p):
        vor = Voronoi(np.concatenate([p + s for s in shifts]))
        cells = []
        for c in range(mid * n_cells, (mid + 1) * n_cells):
            reg = vor.regions[vor.point_region[c]]
            assert reg and -1 not in reg
            cells.append(reg)
        return vor.vertices, cells

    def centroid(P):
        x, y = P[:, 0], P[:, 1]
        xn, yn = np.roll(x, -1), np.roll(y, -1)
        cr = x * yn - xn * y
        a = 0.5 * cr.sum()
        return np.array([((x + xn) * cr).sum(), ((y + yn) * cr).sum()]) / (6.0 * a)

    it = 0
    while True:
        V, cells = diagram(p)
        if it >= lloyd and max(len(c) for c in cells) <= max_vertices:
            break
        if it >= lloyd + 60:
            raise ValueError("Voronoi cells with more than %d vertices remain; try another seed" % max_vertices)
        p = np.array([centroid(V[c]) for c in cells]) % [Lx, Ly]
        it += 1
    used = sorted({v for c in cells for v in c})
    remap = {v: i for i, v in enumerate(used)}
    out = []
    for c in cells:
        P = V[c]
        x, y = P[:, 0], P[:, 1]
        ccw = (x * np.roll(y, -1) - np.roll(x, -1) * y).sum() > 0
        out.append([remap[v] for v in (c if ccw else c[::-1])])
    return V[used], out


def vortex_states(bary, N, L, t=0.0, Lx=10.0, Ly=10.0, beta=5.0, gamma=2.0):
    """Maxwellians of the isentropic vortex of Sec. 4.1 (the Euler solution,
    advected by the mean flow (1, 1) over the periodic box) at the points
    bary (n, 2) at time t: delta T = -(gamma-1) beta^2/(8 gamma pi^2)
    e^{1-r^2}, rho = (1 + delta T)^{1/(gamma-1)}, u = (1, 1) + beta/(2 pi)
    e^{(1-r^2)/2} (-(y-5), x-5), T = 1 + delta T, r measured from the
    vortex centre (5, 5) + t (1, 1) taken periodically.  Returns
    (f (n, N^2), rho (n,), T (n,))."""
    x = (bary[:, 0] - t) % Lx
    y = (bary[:, 1] - t) % Ly
    dx, dy = x - 5.0, y - 5.0
    r2 = dx * dx + dy * dy
    dT = -(gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    du = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = np.stack([1.0 - du * dy, 1.0 + du * dx], axis=1)
    T = 1.0 + dT
    return _gaussian(2, N, L, rho, u, T), rho, T


def sod_mesh(n_side=100, seed=1004, jitter=0.3):
    """Triangle centroids (n_tri, 2) of sod_triangulation and the mesh size
    h = sqrt(mean area)."""
    pts, tri = sod_triangulation(n_side, seed, jitter)
    P = pts[tri]
    cent = P.mean(axis=1)
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                        - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    return cent, float(np.sqrt(area.mean()))


def mesh_states(bary, N, L, jump=False):
    """Maxwellians on the velocity grid for cells with barycentres bary
    (n, 2): smooth fields rho = 1 + 0.3 sin(2 pi x) cos(2 pi y),
    u = 0.3 (cos(2 pi y), sin(2 pi x)), theta = 1 + 0.2 cos(2 pi (x + y)); with
    jump=True the explosion-problem states (1, 0, 1) for x < 0.5 and
    (0.125, 0, 0.8) for x >= 0.5 instead."""
    x, y = bary[:, 0], bary[:, 1]
    if jump:
        left = x < 0.5
        rho = np.where(left, 1.0, 0.125)
        th = np.where(left, 1.0, 0.8)
        u = np.zeros((len(x), 2))
    else:
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
        u = 0.3 * np.stack([np.cos(2 * np.pi * y), np.sin(2 * np.pi * x)], axis=1)
        th = 1.0 + 0.2 * np.cos(2 * np.pi * (x + y))
    return _gaussian(2, N, L, rho, u, th)


def sod_cells(N, L, n_side=100, seed=1004):
    """Cell data of the density/temperature jump across x = 0.5 (the states of
    the explosion problem of Sec. 4.2): (rho, u, theta) = (1, 0, 1) left and
    (0.125, 0, 0.8) right, as Gaussians on the velocity grid."""
    cent, h = sod_mesh(n_side, seed)
    left = cent[:, 0] < 0.5
    n = len(cent)
    rho = np.where(left, 1.0, 0.125)
    th = np.where(left, 1.0, 0.8)
    u = np.zeros((n, 2))
    return _gaussian(2, N, L, rho, u, th), h


def grouped_instances(seed=1005, L=10.0):
    """Heterogeneous batch: 8 instances with cell counts log-uniform in
    [1e3, 5e4] and N drawn from {16, 24, 32, 48} (each at least once), plus
    two 3-D 16^3 instances of 1000 cells.  Returns a list of dicts with
    dim, N, L, n_cells, seed (inputs are drawn per instance with bi_maxwellian)."""
    rng = np.random.default_rng(seed)
    Ns = [16, 24, 32, 48] + list(rng.choice([16, 24, 32, 48], size=4))
    rng.shuffle(Ns)
    out = []
    for i, N in enumerate(Ns):
        cells = int(round(math.exp(rng.uniform(math.log(1e3), math.log(5e4)))))
        out.append(dict(dim=2, N=int(N), L=L, n_cells=cells, seed=seed * 100 + i))
    for i in range(2):
        out.append(dict(dim=3, N=16, L=L, n_cells=1000, seed=seed * 100 + 8 + i))
    return out
