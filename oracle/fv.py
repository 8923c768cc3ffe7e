"""Plain FP64 oracle of the finite-volume transport residual of Sec. 3.2.

TEST INFRASTRUCTURE ONLY: imported by the tests and by the benchmark's
CPU-baseline leg; the CUDA library never imports it.  It shares no code with
the library (geometry, stencils, reconstruction and fluxes are written here
from the paper's definitions; every loop runs over cells in index order and is
vectorised only over the discrete velocities).

What is computed, per polygonal cell P_i and discrete velocity v_k (2-D
space, 2-D velocity grid v = (-L + j1 dv, -L + j2 dv), k = j1 N + j2):

  L_{k,i} = (1/|P_i|) sum over the faces e of P_i of |e| F(f_L, f_R; v_k . n_e)

with F the Rusanov flux of the linear flux v f (eq. finite_vol5):
  F = (v.n)(f_L + f_R)/2 - |v.n| (f_R - f_L)/2,
f_L, f_R the reconstructed values on either side at the face midpoint (the
midpoint rule is exact for reconstructions of degree <= 1), and a
transmissive boundary (f_R = f_L on faces without a neighbour) unless the face
is a wall with full accommodation (transport_residual's `walls`).

Reconstruction (eq. CWENO:Popt, CWENO:P0, CWENO:Prec, eqn.weights) for the
degree M = 1: with the zero-mean Taylor basis about the barycentre x_b
(eq. Dubiner_phi_spatial), every polynomial that keeps the cell average is
p(x) = fbar_i + g . (x - x_b,i), and the cell average of p over P_j is
fbar_i + g . (x_b,j - x_b,i).  Hence
  - p_opt: g_opt = least-squares solution over the central stencil of
    n_e = 2 * M(M) = 6 cells (the cell and its 5 nearest cells), from its
    normal equations A^T A g = A^T d (A: barycentre offsets, d: differences
    of the averages);
  - p^L (L = 1..#sectors): the gradient that reproduces the averages of the
    sector's two other cells exactly;
  - p^0 = (p_opt - sum_L lambda_L p^L) / lambda_0;
  - f^w = sum_s omega_s p^s with omega_s proportional to
    lambda_s / (sigma_s + eps)^r, eps = 1e-14, r = 4 (printed values),
    sigma_s = h_i^2 |g_s|^2.
For M = 0, f^w = fbar (first order).

Degree M = 2 (order=3, the third-order scheme of Sec. 4.1's O3 columns): the
zero-mean Taylor basis about x_b scaled by h (eq. Dubiner_phi_spatial),
  phi = (xi, eta, xi^2 - <xi^2>_i, xi eta - <xi eta>_i, eta^2 - <eta^2>_i),
  xi = (x - x_b,i)/h_i, eta = (y - y_b,i)/h_i, <.>_i the mean over P_i,
p = fbar_i + sum_l c_l phi_l.  Cell means of quadratics are exact: the polygon
is split into the fan of triangles from its first vertex and each triangle's
three edge midpoints, with a third of its area each, integrate quadratics
exactly.
  - p_opt: least squares over the cell and its 11 nearest cells
    (n_e = 2 M(M) = 12), rows = the means of phi over P_j;
  - p^L: the degree-1 sector polynomials above (coefficients (h g, 0, 0, 0));
  - p^0 = (p_opt - sum_L lambda_L p^L) / lambda_0;
  - sigma_s = (1/|P_i|) int_{P_i} (h^2 |grad p|^2 + h^4 (p_xx^2 + p_xy^2 +
    p_yy^2)) dx, the same indicator (h^2 |g|^2) for the linear polynomials;
  - the face integrals use the 2-point Gauss-Legendre rule on every edge
    (exact for the cubic v.n p along a straight edge).

Readings of points the paper leaves open:
  - central stencil: the 5 cells nearest to P_i by barycentre distance
    among the cells that share a vertex with P_i or with one of its
    vertex neighbours (ties by cell index);
  - sectors: for every pair of consecutive faces of P_i that both have a
    neighbour, the stencil {P_i, neighbour across the first, neighbour across
    the second}; a sector whose two barycentre offsets are (numerically)
    collinear is dropped;
  - linear weights lambda_0 = 3/4 and lambda_L = (1/4) / #sectors (lambda_0 =
    1 with no sector);
  - h_i = the largest distance from the barycentre to a vertex of P_i;
  - sigma_s = h_i^2 |g_s|^2, the gradient part of the usual smoothness
    indicator for a linear polynomial.
"""
import numpy as np

LAMBDA0 = 0.75
EPS = 1e-14
R_EXP = 4


class Mesh:
    """Geometry of a polygonal mesh: vertices xy (n_vtx, 2), cells as a list of
    vertex-index lists (any orientation; stored counter-clockwise).

    periodic=(Lx, Ly) makes the mesh periodic in x and/or y (0: not periodic in
    that direction): vertices whose coordinates agree modulo the periods are
    one point of the torus.  Neighbour relations then carry a shift s, the
    translation that takes the neighbour's coordinates into the cell's frame,
    and every offset to a neighbour's barycentre or face midpoint uses
    bary_j + s."""

    def __init__(self, xy, cells, periodic=None):
        self.xy = np.asarray(xy, dtype=np.float64)
        self.cells = []
        n = len(cells)
        self.area = np.zeros(n)
        self.bary = np.zeros((n, 2))
        self.h = np.zeros(n)
        for i, c in enumerate(cells):
            c = [int(v) for v in c]
            a, b = self._shoelace(c)
            if a < 0:
                c = c[::-1]
                a, b = self._shoelace(c)
            self.cells.append(c)
            self.area[i] = a
            self.bary[i] = b
            self.h[i] = np.sqrt(((self.xy[c] - b) ** 2).sum(axis=1)).max()
        # periodic classes of the vertices (the vertex itself without periodicity)
        self.vclass = np.arange(len(self.xy))
        self.period = (0.0, 0.0)
        if periodic is not None and (periodic[0] > 0 or periodic[1] > 0):
            Lx, Ly = float(periodic[0]), float(periodic[1])
            self.period = (Lx, Ly)
            tol = 1e-9 * max(Lx, Ly)
            reps = {}
            for v, (x, y) in enumerate(self.xy):
                kx = round((x % Lx) / tol) % round(Lx / tol) if Lx > 0 else round(x / tol)
                ky = round((y % Ly) / tol) % round(Ly / tol) if Ly > 0 else round(y / tol)
                self.vclass[v] = reps.setdefault((kx, ky), v)
        # faces: edge a -> b of a counter-clockwise polygon has the outward
        # normal (y_b - y_a, -(x_b - x_a)) / |e|; the neighbour owns the edge
        # b -> a (periodic classes), the shift is the difference of the copies
        # of a
        owner = {}
        for i, c in enumerate(self.cells):
            for q in range(len(c)):
                a, b = c[q], c[(q + 1) % len(c)]
                key = (self.vclass[a], self.vclass[b])
                if key in owner:         # the pairing of this edge would be ambiguous
                    raise ValueError("an edge is used twice in the same direction (overlapping cells, "
                                     "inconsistent orientation, or a period only two cells wide)")
                owner[key] = (i, a)
        self.faces = []          # per cell: list of (neighbour or -1, length, nx, ny, midx, midy)
        self.face_vertices = []  # per cell: the vertex pair (a, b) of every face
        self.face_shift = []     # per cell: the neighbour's shift across every face
        for i, c in enumerate(self.cells):
            fl, sh = [], []
            self.face_vertices.append([(c[q], c[(q + 1) % len(c)]) for q in range(len(c))])
            for q in range(len(c)):
                a, b = c[q], c[(q + 1) % len(c)]
                d = self.xy[b] - self.xy[a]
                ln = float(np.hypot(d[0], d[1]))
                mid = 0.5 * (self.xy[a] + self.xy[b])
                j, shift = -1, np.zeros(2)
                o = owner.get((self.vclass[b], self.vclass[a]))
                if o is not None:
                    j = o[0]
                    # the neighbour's copy of b (its edge runs b -> a): the
                    # vertex of the same class on the neighbour's edge
                    cj = self.cells[j]
                    wb = next(w for w in cj if self.vclass[w] == self.vclass[b])
                    shift = self._lattice(self.xy[b] - self.xy[wb])
                fl.append((j, ln, d[1] / ln, -d[0] / ln, mid[0], mid[1]))
                sh.append(shift)
            self.faces.append(fl)
            self.face_shift.append(sh)
        # vertex class -> (cell, vertex)
        vc = {}
        for i, c in enumerate(self.cells):
            for v in c:
                vc.setdefault(self.vclass[v], []).append((i, v))
        self.vertex_cells = vc

    def _lattice(self, s):
        """A shift rounded to the nearest multiple of the periods (zero along a
        direction without periodicity)."""
        out = np.zeros(2)
        for d in range(2):
            if self.period[d] > 0:
                out[d] = round(s[d] / self.period[d]) * self.period[d]
        return out

    def _shoelace(self, c):
        """Signed area and barycentre of the polygon c, with coordinates taken
        relative to its first vertex (the shoelace sums then do not cancel)."""
        P = self.xy[c] - self.xy[c[0]]
        x, y = P[:, 0], P[:, 1]
        xn, yn = np.roll(x, -1), np.roll(y, -1)
        cross = x * yn - xn * y
        a = 0.5 * cross.sum()
        b = self.xy[c[0]] + np.array([((x + xn) * cross).sum(), ((y + yn) * cross).sum()]) / (6 * a)
        return a, b

    def vertex_neighbours(self, i):
        """{(j, sx, sy)}: cells sharing a (periodic) vertex with cell i, with the
        shift of j's copy into i's frame; (i, 0, 0) excluded."""
        out = set()
        for v in self.cells[i]:
            for (j, w) in self.vertex_cells[self.vclass[v]]:
                s = self._lattice(self.xy[v] - self.xy[w])
                out.add((j, float(s[0]), float(s[1])))
        out.discard((i, 0.0, 0.0))
        return out

    def central_stencil_shifted(self, i, count=5):
        """The 5 nearest (cell, shift) images by barycentre distance among the
        vertex neighbours and their vertex neighbours (ties by index, shift)."""
        cand = set()
        first = self.vertex_neighbours(i)
        cand.update(first)
        for (j, sx, sy) in first:
            for (k, tx, ty) in self.vertex_neighbours(j):
                cand.add((k, sx + tx, sy + ty))
        cand.discard((i, 0.0, 0.0))
        d = [(float(np.hypot(self.bary[j, 0] + sx - self.bary[i, 0], self.bary[j, 1] + sy - self.bary[i, 1])),
              j, sx, sy) for (j, sx, sy) in cand]
        d.sort()
        return [(j, np.array([sx, sy])) for _, j, sx, sy in d[:count]]

    def central_stencil(self, i, count=5):
        return [j for j, _ in self.central_stencil_shifted(i, count)]

    def sectors_shifted(self, i):
        """[(a, s_a, b, s_b)]: consecutive face neighbours with their shifts."""
        fl = self.faces[i]
        out = []
        for q in range(len(fl)):
            q2 = (q + 1) % len(fl)
            a, b = fl[q][0], fl[q2][0]
            if a < 0 or b < 0:
                continue
            sa, sb = self.face_shift[i][q], self.face_shift[i][q2]
            A = np.array([self.bary[a] + sa - self.bary[i], self.bary[b] + sb - self.bary[i]])
            if abs(np.linalg.det(A)) <= 1e-12 * float(np.abs(A).max()) ** 2:
                continue
            out.append((a, sa, b, sb))
        return out

    def sectors(self, i):
        return [(a, b) for a, _, b, _ in self.sectors_shifted(i)]


def velocity_grid(N, L):
    v = -L + (2.0 * L / N) * np.arange(N)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    return V1.ravel(), V2.ravel()


def reconstruct_gradients(mesh, f, order, weights="nonlinear"):
    """CWENO gradient g (n_cells, 2, nv) of f^w in every cell; zero for order 1;
    weights="linear" returns the optimal (least-squares) gradient."""
    f = np.asarray(f, dtype=np.float64)
    n, nv = f.shape
    g = np.zeros((n, 2, nv))
    if order == 1:
        return g
    for i in range(n):
        st = mesh.central_stencil_shifted(i)
        A = np.array([mesh.bary[j] + s - mesh.bary[i] for j, s in st])     # (5, 2)
        d = np.array([f[j] - f[i] for j, _ in st])                          # (5, nv)
        g_opt = np.linalg.solve(A.T @ A, A.T @ d)       # normal equations of the least-squares fit
        secs = mesh.sectors_shifted(i)
        if weights == "linear" or not secs:
            g[i] = g_opt
            continue
        lam_l = (1.0 - LAMBDA0) / len(secs)
        gs = []
        for a, sa, b, sb in secs:
            A2 = np.array([mesh.bary[a] + sa - mesh.bary[i], mesh.bary[b] + sb - mesh.bary[i]])
            gs.append(np.linalg.solve(A2, np.array([f[a] - f[i], f[b] - f[i]])))
        g0 = (g_opt - lam_l * sum(gs)) / LAMBDA0
        polys = [g0] + gs
        lams = [LAMBDA0] + [lam_l] * len(gs)
        h2 = mesh.h[i] ** 2
        wt = [lm / (h2 * (gg ** 2).sum(axis=0) + EPS) ** R_EXP for lm, gg in zip(lams, polys)]
        tot = sum(wt)
        g[i] = sum((w / tot) * gg for w, gg in zip(wt, polys))
    return g


GAUSS2 = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # 2-point Gauss-Legendre on [0, 1]


def _quadratic_means(P, xb, h):
    """Means over the polygon with vertices P (k, 2), taken in order, of
    (xi, eta, xi^2, xi eta, eta^2), xi = (x - xb_x)/h, eta = (y - xb_y)/h."""
    Q = (np.asarray(P, dtype=np.float64) - xb) / h
    tot, area = np.zeros(5), 0.0
    for t in range(1, len(Q) - 1):
        a, b, c = Q[0], Q[t], Q[t + 1]
        at = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]))
        for m in (0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)):
            tot += (at / 3.0) * np.array([m[0], m[1], m[0] * m[0], m[0] * m[1], m[1] * m[1]])
        area += at
    return tot / area


def quadratic_basis(mesh, i):
    """(x_b, h, mu): the expansion point, the scale and the means over P_i of
    (xi, eta, xi^2, xi eta, eta^2) (the first two vanish: x_b is the centroid)."""
    xb, h = mesh.bary[i], mesh.h[i]
    return xb, h, _quadratic_means(mesh.xy[mesh.cells[i]], xb, h)


def quadratic_phi(x, xb, h, mu):
    """The zero-mean basis (xi, eta, xi^2 - mu_20, xi eta - mu_11, eta^2 - mu_02) at x."""
    xi, eta = (x[0] - xb[0]) / h, (x[1] - xb[1]) / h
    return np.array([xi, eta, xi * xi - mu[2], xi * eta - mu[3], eta * eta - mu[4]])


def quadratic_indicator(c, mu):
    """sigma of the module docstring for coefficients c (5, nv): the cell mean
    of (d/dxi p)^2 + (d/deta p)^2 plus the squares of the second derivatives."""
    c1, c2, c3, c4, c5 = c
    return (c1 * c1 + c2 * c2
            + 4 * c3 * c3 * mu[2] + 4 * c3 * c4 * mu[3] + c4 * c4 * mu[4]
            + c4 * c4 * mu[2] + 4 * c4 * c5 * mu[3] + 4 * c5 * c5 * mu[4]
            + 4 * c3 * c3 + c4 * c4 + 4 * c5 * c5)


def reconstruct_quadratic(mesh, f, weights="nonlinear"):
    """CWENO coefficients C (n_cells, 5, nv) of degree 2 in the basis of
    quadratic_phi; weights="linear" returns p_opt (for the exactness pins)."""
    f = np.asarray(f, dtype=np.float64)
    n, nv = f.shape
    C = np.zeros((n, 5, nv))
    for i in range(n):
        xb, h, mu = quadratic_basis(mesh, i)
        sub = np.array([0.0, 0.0, mu[2], mu[3], mu[4]])
        st = mesh.central_stencil_shifted(i, count=11)
        A = np.array([_quadratic_means(mesh.xy[mesh.cells[j]] + s, xb, h) - sub for j, s in st])
        d = np.array([f[j] - f[i] for j, _ in st])
        c_opt = np.linalg.solve(A.T @ A, A.T @ d)
        secs = mesh.sectors_shifted(i)
        if weights == "linear" or not secs:
            C[i] = c_opt
            continue
        lam_l = (1.0 - LAMBDA0) / len(secs)
        polys = []
        for a, sa, b, sb in secs:
            A2 = np.array([(mesh.bary[a] + sa - xb) / h, (mesh.bary[b] + sb - xb) / h])
            cs = np.zeros((5, nv))
            cs[:2] = np.linalg.solve(A2, np.array([f[a] - f[i], f[b] - f[i]]))
            polys.append(cs)
        c0 = (c_opt - lam_l * sum(polys)) / LAMBDA0
        allp = [c0] + polys
        lams = [LAMBDA0] + [lam_l] * len(polys)
        wt = [lm / (quadratic_indicator(cc, mu) + EPS) ** R_EXP for lm, cc in zip(lams, allp)]
        tot = sum(wt)
        C[i] = sum((w / tot) * cc for w, cc in zip(wt, allp))
    return C


def _residual_quadratic(mesh, f, N, L, weights, walls=None):
    """L_{k,i} with the degree-2 reconstruction and 2 Gauss points per face; at
    a wall face the mass balance of eq. MU holds at each Gauss point (the
    point value of the outgoing flux against the wall Maxwellian's incoming
    one)."""
    v1, v2 = velocity_grid(N, L)
    C = reconstruct_quadratic(mesh, f, weights)
    basis = [quadratic_basis(mesh, i) for i in range(len(f))]
    out = np.zeros_like(f)
    for i, c in enumerate(mesh.cells):
        acc = np.zeros(f.shape[1])
        for q, (j, ln, nx, ny, mx, my) in enumerate(mesh.faces[i]):
            vn = v1 * nx + v2 * ny
            xa, xe = mesh.xy[c[q]], mesh.xy[c[(q + 1) % len(c)]]
            wall = None if walls is None else walls.get(frozenset(mesh.face_vertices[i][q]))
            for t in GAUSS2:
                x = xa + t * (xe - xa)
                fl = f[i] + quadratic_phi(x, *basis[i]) @ C[i]
                if j < 0 and wall is not None:
                    mw = wall_maxwellian(v1, v2, *wall)
                    out_ = vn > 0
                    mu = (fl * vn)[out_].sum() / (mw * -vn)[~out_].sum()
                    fr = np.where(out_, fl, mu * mw)
                elif j < 0:
                    fr = fl
                else:
                    fr = f[j] + quadratic_phi(x - mesh.face_shift[i][q], *basis[j]) @ C[j]
                acc += 0.5 * ln * (0.5 * vn * (fl + fr) - 0.5 * np.abs(vn) * (fr - fl))
        out[i] = acc / mesh.area[i]
    return out


def wall_maxwellian(v1, v2, theta, u1, u2):
    """Unit-mass 2-D Maxwellian of the wall (eq. MAXB)."""
    return np.exp(-((v1 - u1) ** 2 + (v2 - u2) ** 2) / (2 * theta)) / (2 * np.pi * theta)


def transport_residual(mesh, f, N, L, order=2, walls=None, weights="nonlinear"):
    """L_{k,i} of the module docstring for f of shape (n_cells, N*N); order 1,
    2 (degree 0, 1) or 3 (degree 2); weights="linear" keeps p_opt (for pins).

    walls: optional {frozenset({a, b}): (theta_w, u_w1, u_w2)} for boundary
    edges with vertices a, b that are walls with full accommodation
    (eq. BOU with alpha = 1, eq. MAXB, eq. MU): velocities leaving the domain
    through the face carry the reconstructed inner value f_L, velocities
    entering it carry mu M_w(v), with mu such that the discrete mass fluxes
    balance, mu sum_{v.n < 0} M_w |v.n| = sum_{v.n > 0} f_L v.n (n the outer
    normal; the velocity-cell volume cancels)."""
    f = np.asarray(f, dtype=np.float64)
    if order == 3:
        return _residual_quadratic(mesh, f, N, L, weights, walls)
    v1, v2 = velocity_grid(N, L)
    g = reconstruct_gradients(mesh, f, order, weights)
    out = np.zeros_like(f)
    for i in range(len(f)):
        acc = np.zeros(f.shape[1])
        for q, (j, ln, nx, ny, mx, my) in enumerate(mesh.faces[i]):
            vn = v1 * nx + v2 * ny
            fl = f[i] + g[i, 0] * (mx - mesh.bary[i, 0]) + g[i, 1] * (my - mesh.bary[i, 1])
            wall = None if walls is None else walls.get(frozenset(mesh.face_vertices[i][q]))
            if j < 0 and wall is not None:
                mw = wall_maxwellian(v1, v2, *wall)
                out_ = vn > 0
                mu = (fl * vn)[out_].sum() / (mw * -vn)[~out_].sum()
                fr = np.where(out_, fl, mu * mw)
            elif j < 0:
                fr = fl
            else:
                sx, sy = mesh.face_shift[i][q]
                fr = f[j] + g[j, 0] * (mx - sx - mesh.bary[j, 0]) + g[j, 1] * (my - sy - mesh.bary[j, 1])
            acc += ln * (0.5 * vn * (fl + fr) - 0.5 * np.abs(vn) * (fr - fl))
        out[i] = acc / mesh.area[i]
    return out
