// fv_mesh.cpp -- host set-up of the finite-volume transport step (Sec. 3.2):
// polygon geometry, face pairing, CWENO stencils and their reconstruction
// matrices, uploaded once per mesh.
//
// Geometry.  Every cell is stored counter-clockwise (shoelace sign); its area
// and barycentre x_b come from the polygon formulas, h_i is the largest
// distance from x_b to a vertex (the characteristic length that scales the
// smoothness indicators).  Edge a -> b of a counter-clockwise polygon has the
// outward normal (y_b - y_a, -(x_b - x_a)) / |e|; the cell owning edge b -> a
// is the neighbour; an edge without one is a (transmissive) boundary face.
//
// CWENO of degree 1 (eq. CWENO:Popt, CWENO:P0, CWENO:Prec).  With the
// zero-mean Taylor basis about x_b (eq. Dubiner_phi_spatial) a polynomial
// that keeps the cell average is fbar_i + g . (x - x_b,i), and its average
// over P_j is fbar_i + g . (x_b,j - x_b,i).  So
//   - the optimal polynomial's gradient is the least-squares solution over
//     the central stencil: g_opt = (A^T A)^-1 A^T d, A's rows the barycentre
//     offsets of the 2 M(M) - 1 = 5 nearest cells (among the cells that share
//     a vertex with P_i or with one of its vertex neighbours; ties by index),
//     d the differences of their averages to fbar_i;
//   - a sector polynomial (cell, neighbour across face q, neighbour across
//     face q + 1) reproduces both averages: g_L = A_L^-1 d_L, skipped when
//     the two offsets are numerically collinear.
// The device keeps R_c = (A^T A)^-1 A^T and A_L^-1 per cell; the nonlinear
// weights are formed per velocity by the gradient kernel.
#include <math.h>

#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <unordered_map>
#include <utility>
#include <vector>

#include "bz_internal.h"

namespace bz {

namespace {

struct HostMesh {
    int64_t n = 0;
    std::vector<int> nface, nb, nbq, ncen, cen, nsec, sec, order;
    std::vector<double> inv_area, h2, fn, off_i, off_j, Rc, Rs;
    // order 3
    std::vector<int> ncen3, cen3;
    std::vector<double> mu, Rc3, phi_i, phi_j;
};

constexpr int64_t kReal3PerCell = 3 + kFvCoef3 * kFvCentral3 + 2 * kFvMaxFaces * 2 * kFvCoef3;

template <typename T>
FvTables3<T> carve3(void *base, int64_t n) {
    T *p = static_cast<T *>(base);
    FvTables3<T> t;
    t.mu = p; p += n * 3;
    t.Rc = p; p += n * kFvCoef3 * kFvCentral3;
    t.phi_i = p; p += n * kFvMaxFaces * 2 * kFvCoef3;
    t.phi_j = p;
    return t;
}

// Means over a polygon (vertices px, py in order, translated by (sx, sy)) of
// xi, eta, xi^2, xi eta, eta^2 with xi = (x - x0)/hh, eta = (y - y0)/hh: the
// fan of triangles from the first vertex, each integrated exactly for
// quadratics by its three edge midpoints (a third of the area each).
void quad_means(const std::vector<int64_t> &c, const double *xy, double sx, double sy, double x0, double y0,
                double hh, double out[5]) {
    double acc[5] = {0, 0, 0, 0, 0}, area = 0.0;
    auto X = [&](int64_t v) { return (xy[2 * v] + sx - x0) / hh; };
    auto Y = [&](int64_t v) { return (xy[2 * v + 1] + sy - y0) / hh; };
    const double ax = X(c[0]), ay = Y(c[0]);
    for (size_t t = 1; t + 1 < c.size(); ++t) {
        const double bx = X(c[t]), by = Y(c[t]), cx = X(c[t + 1]), cy = Y(c[t + 1]);
        const double at = 0.5 * ((bx - ax) * (cy - ay) - (cx - ax) * (by - ay));
        const double mx[3] = {0.5 * (ax + bx), 0.5 * (bx + cx), 0.5 * (cx + ax)};
        const double my[3] = {0.5 * (ay + by), 0.5 * (by + cy), 0.5 * (cy + ay)};
        for (int q = 0; q < 3; ++q) {
            const double w = at / 3.0;
            acc[0] += w * mx[q];
            acc[1] += w * my[q];
            acc[2] += w * mx[q] * mx[q];
            acc[3] += w * mx[q] * my[q];
            acc[4] += w * my[q] * my[q];
        }
        area += at;
    }
    for (int l = 0; l < 5; ++l) out[l] = acc[l] / area;
}

// Solve the symmetric positive definite 5 x 5 system M X = B (B: 5 x nc,
// row-major, overwritten with X) by Gaussian elimination with partial
// pivoting.  Returns false when a pivot falls below tol times the largest
// diagonal entry (the stencil does not determine a quadratic).
bool solve5(double M[5][5], double *B, int nc, double tol) {
    double dmax = 0.0;
    for (int r = 0; r < 5; ++r) dmax = std::max(dmax, fabs(M[r][r]));
    for (int col = 0; col < 5; ++col) {
        int piv = col;
        for (int r = col + 1; r < 5; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (!(fabs(M[piv][col]) > tol * dmax)) return false;
        if (piv != col) {
            for (int q = 0; q < 5; ++q) std::swap(M[piv][q], M[col][q]);
            for (int q = 0; q < nc; ++q) std::swap(B[piv * nc + q], B[col * nc + q]);
        }
        for (int r = 0; r < 5; ++r) {
            if (r == col) continue;
            const double fct = M[r][col] / M[col][col];
            if (fct == 0.0) continue;
            for (int q = col; q < 5; ++q) M[r][q] -= fct * M[col][q];
            for (int q = 0; q < nc; ++q) B[r * nc + q] -= fct * B[col * nc + q];
        }
    }
    for (int r = 0; r < 5; ++r)
        for (int q = 0; q < nc; ++q) B[r * nc + q] /= M[r][r];
    return true;
}

template <typename T>
FvTables<T> carve(void *base, int64_t n) {
    T *p = static_cast<T *>(base);
    FvTables<T> t;
    t.inv_area = p; p += n;
    t.h2 = p; p += n;
    t.fn = p; p += n * kFvMaxFaces * 2;
    t.off_i = p; p += n * kFvMaxFaces * 2;
    t.off_j = p; p += n * kFvMaxFaces * 2;
    t.Rc = p; p += n * 2 * kFvCentral;
    t.Rs = p;
    return t;
}
constexpr int64_t kRealPerCell = 1 + 1 + 3 * kFvMaxFaces * 2 + 2 * kFvCentral + kFvMaxFaces * 4;

void fill_real(const HostMesh &h, std::vector<double> &out) {
    const int64_t n = h.n;
    out.assign((size_t)(n * kRealPerCell), 0.0);
    double *p = out.data();
    auto put = [&p](const std::vector<double> &v) {
        memcpy(p, v.data(), sizeof(double) * v.size());
        p += v.size();
    };
    put(h.inv_area);
    put(h.h2);
    put(h.fn);
    put(h.off_i);
    put(h.off_j);
    put(h.Rc);
    put(h.Rs);
}

template <typename X> cudaError_t upload(X **d, const std::vector<X> &v) {
    cudaError_t e = dev_malloc(d, sizeof(X) * v.size());
    if (e == cudaSuccess) e = cudaMemcpy(*d, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

void fv_mesh_destroy(bz_mesh *m) {
    if (!m) return;
    dev_free(m->d_nface);
    dev_free(m->d_nb);
    dev_free(m->d_tripos);
    dev_free(m->d_ncen);
    dev_free(m->d_cen);
    dev_free(m->d_nsec);
    dev_free(m->d_sec);
    dev_free(m->d_order);
    dev_free(m->d_wall);
    dev_free(m->d_wall64);
    dev_free(m->d_wall32);
    free(m->h_ptr);
    free(m->h_vtx);
    free(m->h_nb);
    dev_free(m->d_real64);
    dev_free(m->d_real32);
    dev_free(m->d_ncen3);
    dev_free(m->d_cen3);
    dev_free(m->d_real3_64);
    dev_free(m->d_real3_32);
    free(m);
}

int fv_mesh_create(int n_vertices, const double *xy, int64_t n_cells, const int64_t *cell_ptr,
                   const int64_t *cell_vertices, int order, double Lx, double Ly, bz_mesh **out) {
    if (!out) return fail(BZ_EINVAL, "build_fv_mesh: out is NULL");
    *out = nullptr;
    if (n_vertices < 3 || !xy) return fail(BZ_EINVAL, "build_fv_mesh: need >= 3 vertices and their coordinates");
    if (n_cells < 1 || n_cells > (int64_t)1 << 30 || !cell_ptr || !cell_vertices)
        return fail(BZ_EINVAL, "build_fv_mesh: bad cell list");
    if (order < 1 || order > 3) return fail(BZ_EINVAL, "build_fv_mesh: order must be 1, 2 or 3");
    if (cell_ptr[0] != 0) return fail(BZ_EINVAL, "build_fv_mesh: cell_ptr[0] must be 0");
    if (!(Lx >= 0) || !(Ly >= 0) || !std::isfinite(Lx) || !std::isfinite(Ly))
        return fail(BZ_EINVAL, "build_fv_mesh: periods must be finite and >= 0");
    const int64_t n = n_cells;
    HostMesh h;
    h.n = n;
    std::vector<std::vector<int64_t>> cells((size_t)n);
    std::vector<double> area(n), bx(n), by(n);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t a = cell_ptr[i], b = cell_ptr[i + 1];
        if (b - a < 3 || b - a > kFvMaxFaces)
            return fail(BZ_EINVAL, "build_fv_mesh: cells need 3 to 8 vertices");
        std::vector<int64_t> c(cell_vertices + a, cell_vertices + b);
        for (int64_t v : c)
            if (v < 0 || v >= n_vertices) return fail(BZ_EINVAL, "build_fv_mesh: vertex index out of range");
        // shoelace area and polygon barycentre, coordinates relative to the
        // first vertex (absolute coordinates would cancel in the cross
        // products of a small cell); store counter-clockwise
        auto geom = [&](const std::vector<int64_t> &cc, double &A, double &cx, double &cy) {
            A = cx = cy = 0.0;
            const size_t k = cc.size();
            const double ox = xy[2 * cc[0]], oy = xy[2 * cc[0] + 1];
            for (size_t q = 0; q < k; ++q) {
                const double x0 = xy[2 * cc[q]] - ox, y0 = xy[2 * cc[q] + 1] - oy;
                const double x1 = xy[2 * cc[(q + 1) % k]] - ox, y1 = xy[2 * cc[(q + 1) % k] + 1] - oy;
                const double cr = x0 * y1 - x1 * y0;
                A += cr;
                cx += (x0 + x1) * cr;
                cy += (y0 + y1) * cr;
            }
            A *= 0.5;
            cx = ox + cx / (6.0 * A);
            cy = oy + cy / (6.0 * A);
        };
        double A, cx, cy;
        geom(c, A, cx, cy);
        if (A < 0) {
            std::reverse(c.begin(), c.end());
            geom(c, A, cx, cy);
        }
        if (!(A > 0)) return fail(BZ_EINVAL, "build_fv_mesh: degenerate cell (zero area)");
        area[i] = A;
        bx[i] = cx;
        by[i] = cy;
        double hm = 0.0;
        for (int64_t v : c) hm = std::max(hm, hypot(xy[2 * v] - cx, xy[2 * v + 1] - cy));
        h.inv_area.push_back(1.0 / A);
        h.h2.push_back(hm * hm);
        cells[i] = std::move(c);
    }
    // periodic classes: vertices whose coordinates agree modulo the periods
    // are one point (a vertex is its own class without periodicity); a shift
    // is kept as integer multiples (kx, ky) of the periods
    std::vector<int64_t> vclass(n_vertices);
    for (int v = 0; v < n_vertices; ++v) vclass[v] = v;
    const double pmax = std::max(Lx, Ly), qtol = 1e-9 * pmax;
    if (pmax > 0) {
        std::map<std::pair<int64_t, int64_t>, int64_t> rep;
        auto wrap = [qtol](double x, double P) -> int64_t {
            if (P <= 0) return llround(x / qtol);
            const int64_t per = llround(P / qtol);
            int64_t k = llround(x / qtol) % per;
            return k < 0 ? k + per : k;
        };
        for (int v = 0; v < n_vertices; ++v) {
            vclass[v] = rep.emplace(std::make_pair(wrap(xy[2 * v], Lx), wrap(xy[2 * v + 1], Ly)), v).first->second;
        }
    }
    auto lattice = [&](double dx, double dy, int &kx, int &ky) {
        kx = Lx > 0 ? (int)llround(dx / Lx) : 0;
        ky = Ly > 0 ? (int)llround(dy / Ly) : 0;
    };
    // directed edge (classes) -> owning cell and its copy of the edge's first vertex
    std::unordered_map<uint64_t, std::pair<int64_t, int64_t>> owner;
    owner.reserve((size_t)(n * 4));
    auto key = [](int64_t a, int64_t b) { return ((uint64_t)a << 32) | (uint64_t)b; };
    for (int64_t i = 0; i < n; ++i) {
        const auto &c = cells[i];
        for (size_t q = 0; q < c.size(); ++q) {
            const int64_t a = c[q], b = c[(q + 1) % c.size()];
            if (!owner.emplace(key(vclass[a], vclass[b]), std::make_pair(i, a)).second)
                return fail(BZ_EINVAL, "build_fv_mesh: an edge is used twice in the same direction (overlapping or "
                                       "inconsistently oriented cells)");
        }
    }
    h.nface.assign(n, 0);
    h.nb.assign(n * kFvMaxFaces, -1);
    h.nbq.assign(n * kFvMaxFaces, -1);
    h.fn.assign(n * kFvMaxFaces * 2, 0.0);
    h.off_i.assign(n * kFvMaxFaces * 2, 0.0);
    h.off_j.assign(n * kFvMaxFaces * 2, 0.0);
    std::vector<double> fsx(n * kFvMaxFaces, 0.0), fsy(n * kFvMaxFaces, 0.0);   // neighbour shifts
    int64_t interior = 0, boundary = 0;
    int maxf = 0;
    for (int64_t i = 0; i < n; ++i) {
        const auto &c = cells[i];
        const int k = (int)c.size();
        h.nface[i] = k;
        maxf = std::max(maxf, k);
        for (int q = 0; q < k; ++q) {
            const int64_t a = c[q], b = c[(q + 1) % k];
            const double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
            const double mx = 0.5 * (xy[2 * a] + xy[2 * b]), my = 0.5 * (xy[2 * a + 1] + xy[2 * b + 1]);
            const size_t s = (size_t)i * kFvMaxFaces + q;
            h.fn[2 * s] = dy;                 // |e| n_e = (dy, -dx)
            h.fn[2 * s + 1] = -dx;
            h.off_i[2 * s] = mx - bx[i];
            h.off_i[2 * s + 1] = my - by[i];
            auto it = owner.find(key(vclass[b], vclass[a]));
            if (it != owner.end()) {
                const int64_t j = it->second.first, wb = it->second.second;   // j's copy of b
                int kx, ky;
                lattice(xy[2 * b] - xy[2 * wb], xy[2 * b + 1] - xy[2 * wb + 1], kx, ky);
                fsx[s] = kx * Lx;
                fsy[s] = ky * Ly;
                h.nb[s] = (int)j;
                for (size_t t = 0; t < cells[j].size(); ++t)     // j's face starting at its copy of b
                    if (cells[j][t] == wb) h.nbq[s] = (int)t;
                h.off_j[2 * s] = mx - fsx[s] - bx[j];
                h.off_j[2 * s + 1] = my - fsy[s] - by[j];
                ++interior;
            } else {
                ++boundary;
            }
        }
    }
    h.ncen.assign(n, 0);
    h.cen.assign(n * kFvCentral, 0);
    h.Rc.assign(n * 2 * kFvCentral, 0.0);
    h.nsec.assign(n, 0);
    h.sec.assign(n * kFvMaxFaces * 2, 0);
    h.Rs.assign(n * kFvMaxFaces * 4, 0.0);
    if (order == 3) {
        h.ncen3.assign(n, 0);
        h.cen3.assign(n * kFvCentral3, 0);
        h.mu.assign(n * 3, 0.0);
        h.Rc3.assign(n * kFvCoef3 * kFvCentral3, 0.0);
        h.phi_i.assign(n * kFvMaxFaces * 2 * kFvCoef3, 0.0);
        h.phi_j.assign(n * kFvMaxFaces * 2 * kFvCoef3, 0.0);
        for (int64_t i = 0; i < n; ++i) {
            double q[5];
            quad_means(cells[i], xy, 0.0, 0.0, bx[i], by[i], sqrt(h.h2[i]), q);
            h.mu[3 * i] = q[2];
            h.mu[3 * i + 1] = q[3];
            h.mu[3 * i + 2] = q[4];
        }
    }
    if (order >= 2) {
        const int ncen_max = order == 3 ? kFvCentral3 : kFvCentral;
        // vertex class -> (cell, vertex)
        std::vector<int64_t> vptr(n_vertices + 1, 0);
        std::vector<std::pair<int64_t, int64_t>> vcell;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t v : cells[i]) ++vptr[vclass[v] + 1];
        for (int v = 0; v < n_vertices; ++v) vptr[v + 1] += vptr[v];
        vcell.assign(vptr[n_vertices], {0, 0});
        std::vector<int64_t> fillp(vptr.begin(), vptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t v : cells[i]) vcell[fillp[vclass[v]]++] = {i, v};
        struct Img {
            int64_t j;
            int kx, ky;
            bool operator<(const Img &o) const {
                return j != o.j ? j < o.j : kx != o.kx ? kx < o.kx : ky < o.ky;
            }
            bool operator==(const Img &o) const { return j == o.j && kx == o.kx && ky == o.ky; }
        };
        // cells sharing a (periodic) vertex with cell i, with the shift of
        // their copy into i's frame, offset by (ox, oy)
        auto vertex_neighbours = [&](int64_t i, int ox, int oy, std::vector<Img> &out) {
            for (int64_t v : cells[i])
                for (int64_t p = vptr[vclass[v]]; p < vptr[vclass[v] + 1]; ++p) {
                    const int64_t j = vcell[p].first, w = vcell[p].second;
                    int kx, ky;
                    lattice(xy[2 * v] - xy[2 * w], xy[2 * v + 1] - xy[2 * w + 1], kx, ky);
                    out.push_back({j, kx + ox, ky + oy});
                }
        };
        std::vector<Img> ring, cand;
        struct Cand {
            double d;
            Img m;
            bool operator<(const Cand &o) const {
                return d != o.d ? d < o.d : o.m.j != m.j ? m.j < o.m.j : m.kx != o.m.kx ? m.kx < o.m.kx : m.ky < o.m.ky;
            }
        };
        std::vector<Cand> dist;
        for (int64_t i = 0; i < n; ++i) {
            ring.clear();
            vertex_neighbours(i, 0, 0, ring);
            cand = ring;
            for (const Img &r : ring) vertex_neighbours(r.j, r.kx, r.ky, cand);
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            dist.clear();
            for (const Img &c : cand) {
                if (c.j == i && c.kx == 0 && c.ky == 0) continue;
                dist.push_back({hypot(bx[c.j] + c.kx * Lx - bx[i], by[c.j] + c.ky * Ly - by[i]), c});
            }
            std::sort(dist.begin(), dist.end());
            const double hi = sqrt(h.h2[i]);
            if (order == 3) {
                // least squares for the 5 coefficients of the zero-mean scaled
                // Taylor basis over the cell's 11 nearest cells (row q: the
                // basis' means over cell q, translated into this cell's frame)
                const int nc = (int)std::min<size_t>(kFvCentral3, dist.size());
                double A[kFvCentral3][5];
                for (int q = 0; q < nc; ++q) {
                    const Img &c = dist[q].m;
                    h.cen3[i * kFvCentral3 + q] = (int)c.j;
                    quad_means(cells[c.j], xy, c.kx * Lx, c.ky * Ly, bx[i], by[i], hi, A[q]);
                    A[q][2] -= h.mu[3 * i];
                    A[q][3] -= h.mu[3 * i + 1];
                    A[q][4] -= h.mu[3 * i + 2];
                }
                h.ncen3[i] = nc;
                double M[5][5], B[5 * kFvCentral3];
                for (int r = 0; r < 5; ++r) {
                    for (int col = 0; col < 5; ++col) {
                        double sum = 0.0;
                        for (int q = 0; q < nc; ++q) sum += A[q][r] * A[q][col];
                        M[r][col] = sum;
                    }
                    for (int q = 0; q < nc; ++q) B[r * nc + q] = A[q][r];
                }
                if (nc < 5 || !solve5(M, B, nc, 1e-12))
                    return fail(BZ_EINVAL, "build_fv_mesh: order 3 needs a cell neighbourhood that determines a "
                                           "quadratic (mesh too small or degenerate)");
                for (int r = 0; r < 5; ++r)
                    for (int q = 0; q < nc; ++q) h.Rc3[((size_t)i * kFvCoef3 + r) * kFvCentral3 + q] = B[r * nc + q];
            }
            const int nc = (int)std::min<size_t>(kFvCentral, dist.size());
            double ata[3] = {0, 0, 0};
            double axs[kFvCentral], ays[kFvCentral];
            for (int q = 0; q < nc; ++q) {
                const Img &c = dist[q].m;
                h.cen[i * kFvCentral + q] = (int)c.j;
                axs[q] = bx[c.j] + c.kx * Lx - bx[i];
                ays[q] = by[c.j] + c.ky * Ly - by[i];
                ata[0] += axs[q] * axs[q];
                ata[1] += axs[q] * ays[q];
                ata[2] += ays[q] * ays[q];
            }
            h.ncen[i] = nc;
            const double det = ata[0] * ata[2] - ata[1] * ata[1];
            if (nc >= 2 && det > 1e-300) {
                const double i00 = ata[2] / det, i01 = -ata[1] / det, i11 = ata[0] / det;
                for (int q = 0; q < nc; ++q) {
                    h.Rc[(i * 2 + 0) * kFvCentral + q] = i00 * axs[q] + i01 * ays[q];
                    h.Rc[(i * 2 + 1) * kFvCentral + q] = i01 * axs[q] + i11 * ays[q];
                }
            }
            // sectors: consecutive faces with neighbours on both
            const int k = h.nface[i];
            int ns = 0;
            for (int q = 0; q < k; ++q) {
                const size_t sa = (size_t)i * kFvMaxFaces + q, sb = (size_t)i * kFvMaxFaces + (q + 1) % k;
                const int a = h.nb[sa], b = h.nb[sb];
                if (a < 0 || b < 0) continue;
                const double a0 = bx[a] + fsx[sa] - bx[i], a1 = by[a] + fsy[sa] - by[i];
                const double b0 = bx[b] + fsx[sb] - bx[i], b1 = by[b] + fsy[sb] - by[i];
                const double mxa = std::max(std::max(fabs(a0), fabs(a1)), std::max(fabs(b0), fabs(b1)));
                const double dt = a0 * b1 - a1 * b0;
                if (fabs(dt) <= 1e-12 * mxa * mxa) continue;
                // A = [[a0, a1], [b0, b1]] (rows: offsets), g = A^-1 (d_a, d_b);
                // degree 2 takes the coefficients of xi = (x - x_b)/h: h g
                const double sc = order == 3 ? hi : 1.0;
                double *R = &h.Rs[((size_t)i * kFvMaxFaces + ns) * 4];
                R[0] = sc * b1 / dt;
                R[1] = -sc * a1 / dt;
                R[2] = -sc * b0 / dt;
                R[3] = sc * a0 / dt;
                h.sec[((size_t)i * kFvMaxFaces + ns) * 2] = a;
                h.sec[((size_t)i * kFvMaxFaces + ns) * 2 + 1] = b;
                ++ns;
            }
            h.nsec[i] = ns;
            // A triangle with three sectors whose face neighbours all lie in
            // its central stencil (nearly every interior cell of a triangle
            // mesh): the stencil is reordered to start with the face
            // neighbours in face order and the cell is flagged, so that the
            // FP32 reconstruction loads every neighbour row once for the
            // central and the sector gradients (sector s joins faces s and
            // s + 1 mod 3).  The same for the degree-2 stencil.
            auto face_first = [&](int *cn, double *R, int nrow, int width, int ncs, int &flagged) {
                if (k != 3 || ns != 3) return;
                int perm[kFvCentral3];
                bool used[kFvCentral3] = {};
                for (int q = 0; q < 3; ++q) {
                    const int j = h.nb[(size_t)i * kFvMaxFaces + q];
                    int hit = -1;
                    for (int t = 0; t < ncs && hit < 0; ++t)
                        if (!used[t] && cn[t] == j) hit = t;
                    if (hit < 0) return;
                    used[hit] = true;
                    perm[q] = hit;
                }
                for (int t = 0, p = 3; t < ncs; ++t)
                    if (!used[t]) perm[p++] = t;
                int c0[kFvCentral3];
                std::vector<double> r0((size_t)nrow * ncs);
                for (int t = 0; t < ncs; ++t) {
                    c0[t] = cn[t];
                    for (int r = 0; r < nrow; ++r) r0[(size_t)r * ncs + t] = R[(size_t)r * width + t];
                }
                for (int t = 0; t < ncs; ++t) {
                    cn[t] = c0[perm[t]];
                    for (int r = 0; r < nrow; ++r) R[(size_t)r * width + t] = r0[(size_t)r * ncs + perm[t]];
                }
                flagged |= kFvRegularTri;
            };
            if (nc == kFvCentral) {
                int fl = 0;
                face_first(&h.cen[i * kFvCentral], &h.Rc[i * 2 * kFvCentral], 2, kFvCentral, nc, fl);
                h.ncen[i] = nc | fl;
            }
            if (order == 3 && h.ncen3[i] == kFvCentral3) {
                int fl = 0;
                face_first(&h.cen3[i * kFvCentral3], &h.Rc3[(size_t)i * kFvCoef3 * kFvCentral3], kFvCoef3,
                           kFvCentral3, kFvCentral3, fl);
                h.ncen3[i] = kFvCentral3 | fl;
            }
        }
    }
    if (order == 3) {
        // the basis of the cell and of its neighbour at the face's two
        // Gauss-Legendre points x_a + t (x_b - x_a), t = 1/2 -+ 1/(2 sqrt 3)
        const double tg[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
        auto basis = [&](int64_t c, double x, double y, double *out) {
            const double hc = sqrt(h.h2[c]);
            const double xi = (x - bx[c]) / hc, eta = (y - by[c]) / hc;
            out[0] = xi;
            out[1] = eta;
            out[2] = xi * xi - h.mu[3 * c];
            out[3] = xi * eta - h.mu[3 * c + 1];
            out[4] = eta * eta - h.mu[3 * c + 2];
        };
        for (int64_t i = 0; i < n; ++i) {
            const auto &c = cells[i];
            const int k = (int)c.size();
            for (int q = 0; q < k; ++q) {
                const int64_t a = c[q], b = c[(q + 1) % k];
                const size_t sidx = (size_t)i * kFvMaxFaces + q;
                for (int g = 0; g < 2; ++g) {
                    const double x = xy[2 * a] + tg[g] * (xy[2 * b] - xy[2 * a]);
                    const double y = xy[2 * a + 1] + tg[g] * (xy[2 * b + 1] - xy[2 * a + 1]);
                    basis(i, x, y, &h.phi_i[(sidx * 2 + g) * kFvCoef3]);
                    const int j = h.nb[sidx];
                    if (j >= 0) basis(j, x - fsx[sidx], y - fsy[sidx], &h.phi_j[(sidx * 2 + g) * kFvCoef3]);
                }
            }
        }
    }
    // processing order: the kernels take cells along a Morton (Z-order) curve
    // of the barycentres, so CTAs resident at the same time read neighbouring
    // rows of f and of the gradients and share them in L2 (the results do not
    // depend on the order)
    {
        double x0 = bx[0], x1 = bx[0], y0 = by[0], y1 = by[0];
        for (int64_t i = 1; i < n; ++i) {
            x0 = std::min(x0, bx[i]);
            x1 = std::max(x1, bx[i]);
            y0 = std::min(y0, by[i]);
            y1 = std::max(y1, by[i]);
        }
        const double sx = x1 > x0 ? 65535.0 / (x1 - x0) : 0.0, sy = y1 > y0 ? 65535.0 / (y1 - y0) : 0.0;
        auto spread = [](uint32_t v) {
            uint64_t x = v & 0xffffu;
            x = (x | (x << 8)) & 0x00ff00ffu;
            x = (x | (x << 4)) & 0x0f0f0f0fu;
            x = (x | (x << 2)) & 0x33333333u;
            x = (x | (x << 1)) & 0x55555555u;
            return x;
        };
        std::vector<std::pair<uint64_t, int>> key((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            const uint32_t qx = (uint32_t)((bx[i] - x0) * sx), qy = (uint32_t)((by[i] - y0) * sy);
            key[i] = {spread(qx) | (spread(qy) << 1), (int)i};
        }
        std::sort(key.begin(), key.end());
        h.order.resize(n);
        for (int64_t i = 0; i < n; ++i) h.order[i] = key[i].second;
    }
    bz_mesh *m = (bz_mesh *)calloc(1, sizeof(bz_mesh));
    if (!m) return fail(BZ_ENOMEM, "build_fv_mesh: host allocation");
    cudaGetDevice(&m->device);
    m->order = order;
    m->n_cells = n;
    m->n_faces_interior = interior / 2;
    m->n_faces_boundary = boundary;
    m->max_faces = maxf;
    std::vector<double> real;
    fill_real(h, real);
    std::vector<float> real32(real.size());
    for (size_t q = 0; q < real.size(); ++q) real32[q] = (float)real[q];
    cudaError_t e = upload(&m->d_nface, h.nface);
    if (e == cudaSuccess) e = upload(&m->d_nb, h.nb);
    if (e == cudaSuccess) e = upload(&m->d_ncen, h.ncen);
    if (e == cudaSuccess) e = upload(&m->d_cen, h.cen);
    if (e == cudaSuccess) e = upload(&m->d_nsec, h.nsec);
    if (e == cudaSuccess) e = upload(&m->d_sec, h.sec);
    if (e == cudaSuccess) e = upload(&m->d_order, h.order);
    if (e == cudaSuccess && maxf <= 3) {
        std::vector<int4> tp((size_t)n * 3);
        for (int64_t p = 0; p < n; ++p) {
            const int i = h.order[p];
            const int *nb = &h.nb[(size_t)i * kFvMaxFaces], *nq = &h.nbq[(size_t)i * kFvMaxFaces];
            const int *c = &h.cen[(size_t)i * kFvCentral];
            int qbits = 0;
            for (int q = 0; q < 3; ++q)
                if (nb[q] >= 0) qbits |= (nq[q] & 3) << (2 * q);
            tp[3 * p] = make_int4(i, h.ncen[i], h.nsec[i], qbits);
            tp[3 * p + 1] = make_int4(c[0], c[1], c[2], c[3]);
            tp[3 * p + 2] = make_int4(c[4], nb[0], nb[1], nb[2]);
        }
        e = upload(&m->d_tripos, tp);
    }
    double *r64 = nullptr;
    float *r32 = nullptr;
    if (e == cudaSuccess) e = upload(&r64, real);
    m->d_real64 = r64;
    if (e == cudaSuccess) e = upload(&r32, real32);
    m->d_real32 = r32;
    if (e != cudaSuccess) {
        fv_mesh_destroy(m);
        return cuda_fail(e, "build_fv_mesh: device tables");
    }
    m->t64 = carve<double>(m->d_real64, n);
    m->t32 = carve<float>(m->d_real32, n);
    if (order == 3) {
        std::vector<double> r3((size_t)(n * kReal3PerCell));
        double *p3 = r3.data();
        for (const std::vector<double> *v : {&h.mu, &h.Rc3, &h.phi_i, &h.phi_j}) {
            memcpy(p3, v->data(), sizeof(double) * v->size());
            p3 += v->size();
        }
        std::vector<float> r3f(r3.size());
        for (size_t q = 0; q < r3.size(); ++q) r3f[q] = (float)r3[q];
        double *d3 = nullptr;
        float *d3f = nullptr;
        e = upload(&m->d_ncen3, h.ncen3);
        if (e == cudaSuccess) e = upload(&m->d_cen3, h.cen3);
        if (e == cudaSuccess) e = upload(&d3, r3);
        m->d_real3_64 = d3;
        if (e == cudaSuccess) e = upload(&d3f, r3f);
        m->d_real3_32 = d3f;
        if (e != cudaSuccess) {
            fv_mesh_destroy(m);
            return cuda_fail(e, "build_fv_mesh: degree-2 tables");
        }
        m->u64 = carve3<double>(m->d_real3_64, n);
        m->u32 = carve3<float>(m->d_real3_32, n);
    }
    // host copies for fv_mesh_set_walls
    m->h_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    m->h_vtx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cell_ptr[n]);
    m->h_nb = (int *)malloc(sizeof(int) * h.nb.size());
    if (!m->h_ptr || !m->h_vtx || !m->h_nb) {
        fv_mesh_destroy(m);
        return fail(BZ_ENOMEM, "build_fv_mesh: host copies");
    }
    m->h_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        m->h_ptr[i + 1] = m->h_ptr[i] + (int64_t)cells[i].size();
        memcpy(m->h_vtx + m->h_ptr[i], cells[i].data(), sizeof(int64_t) * cells[i].size());
    }
    memcpy(m->h_nb, h.nb.data(), sizeof(int) * h.nb.size());
    *out = m;
    return BZ_OK;
}

// Walls with full accommodation on the boundary edges given by their vertex
// pairs (either order); n_edges = 0 removes every wall.
int fv_mesh_set_walls(bz_mesh *m, int64_t n_edges, const int64_t *edges, const double *params) {
    if (!m) return fail(BZ_EINVAL, "fv_mesh_set_walls: mesh is NULL");
    if (n_edges < 0 || (n_edges > 0 && (!edges || !params)))
        return fail(BZ_EINVAL, "fv_mesh_set_walls: bad edge list");
    dev_free(m->d_wall);
    dev_free(m->d_wall64);
    dev_free(m->d_wall32);
    m->d_wall = nullptr;
    m->d_wall64 = nullptr;
    m->d_wall32 = nullptr;
    m->n_walls = 0;
    if (n_edges == 0) return BZ_OK;
    const int64_t n = m->n_cells;
    std::unordered_map<uint64_t, int64_t> bface;           // unordered vertex pair -> cell * K + face
    auto key = [](int64_t a, int64_t b) {
        if (a > b) std::swap(a, b);
        return ((uint64_t)a << 32) | (uint64_t)b;
    };
    for (int64_t i = 0; i < n; ++i) {
        const int64_t a0 = m->h_ptr[i], k = m->h_ptr[i + 1] - a0;
        for (int64_t q = 0; q < k; ++q)
            if (m->h_nb[i * kFvMaxFaces + q] < 0)
                bface[key(m->h_vtx[a0 + q], m->h_vtx[a0 + (q + 1) % k])] = i * kFvMaxFaces + q;
    }
    std::vector<int> wall((size_t)n * kFvMaxFaces, -1);
    std::vector<double> p64((size_t)n_edges * 3);
    for (int64_t e = 0; e < n_edges; ++e) {
        auto it = bface.find(key(edges[2 * e], edges[2 * e + 1]));
        if (it == bface.end()) return fail(BZ_EINVAL, "fv_mesh_set_walls: an edge is not a boundary edge of the mesh");
        if (!(params[3 * e] > 0)) return fail(BZ_EINVAL, "fv_mesh_set_walls: wall temperature must be > 0");
        wall[(size_t)it->second] = (int)e;
        for (int c = 0; c < 3; ++c) p64[3 * e + c] = params[3 * e + c];
    }
    std::vector<float> p32(p64.size());
    for (size_t q = 0; q < p64.size(); ++q) p32[q] = (float)p64[q];
    cudaError_t err = upload(&m->d_wall, wall);
    if (err == cudaSuccess) err = upload(&m->d_wall64, p64);
    if (err == cudaSuccess) err = upload(&m->d_wall32, p32);
    if (err != cudaSuccess) {
        dev_free(m->d_wall);
        dev_free(m->d_wall64);
        dev_free(m->d_wall32);
        m->d_wall = nullptr;
        m->d_wall64 = nullptr;
        m->d_wall32 = nullptr;
        return cuda_fail(err, "fv_mesh_set_walls: device tables");
    }
    m->n_walls = n_edges;
    return BZ_OK;
}

}  // namespace bz
