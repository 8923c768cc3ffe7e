// host_setup.cpp -- host-side, FP64 set-up of the velocity grid and the kernel
// modes (Sec. 3.1 and Sec. 3.3 of Boscheri & Dimarco, arXiv 2103.14890).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "bz_internal.h"

namespace bz {

// Gauss-Legendre rule on [-1, 1].  Nodes by Newton iteration started from
// Tricomi's asymptotic estimate; P_n and P_n' from the three-term recurrence.
static void legendre_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = M_PI;
    for (int i = 1; i <= (n + 1) / 2; ++i) {
        double th = pi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
        double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
        double pn = 0.0, dpn = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm1 = 1.0, p = z;                 // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
                pm1 = p;
                p = pk;
            }
            pn = p;
            dpn = n * (pm1 - z * p) / (1.0 - z * z);
            double step = pn / dpn;
            z -= step;
            if (fabs(step) < 4e-16) break;
        }
        double pm1 = 1.0, p = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
            pm1 = p;
            p = pk;
        }
        dpn = n * (pm1 - z * p) / (1.0 - z * z);
        double wi = 2.0 / ((1.0 - z * z) * dpn * dpn);
        x[i - 1] = -z;
        x[n - i] = z;
        w[i - 1] = wi;
        w[n - i] = wi;
    }
}

// Radius of the ball the relative velocity is truncated to, in the box
// [-pi,pi]^d: 2 lambda pi with lambda = 2 / (3 + sqrt 2) (Sec. 3.3, eq. KM).
static double q_cutoff() { return 4.0 * M_PI / (3.0 + sqrt(2.0)); }

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

static int auto_nodes(const GridView &g) {
    // fastest phase of the radial integrand: cutoff * (|l+m| + |l-m|)/2 with
    // |l+m| <= h sqrt d and |l-m| <= 2 h sqrt d
    double phase = q_cutoff() * 1.5 * g.h * sqrt((double)g.dim);
    int n = (int)ceil(0.75 * phase) + 40;
    return n < 64 ? 64 : n;
}

// Eq. KM for an angle-independent kernel |q| sigma = b0 |q|^gamma reduces to a
// radial integral: the average of exp(-i x.w) over the unit sphere is J0(|x|)
// (2-D, times 2 pi) or sin|x|/|x| (3-D, times 4 pi), once for omega and once
// for the direction of q, giving
//   2-D: (2 pi)^2 b0 int_0^c r^(gamma+1) J0(r a/2) J0(r b/2) dr
//   3-D: (4 pi)^2 b0 int_0^c r^(gamma+2) sinc(r a/2) sinc(r b/2) dr
// with a = |l+m|, b = |l-m|, c = q_cutoff().  Tabulated over the squared norms.
static void kernel_table(const GridView &g, double gamma, double b0, int nq, int arows,
                         int bcols, std::vector<double> &F) {
    std::vector<double> x, w;
    legendre_rule(nq, x, w);
    const double c = q_cutoff();
    const double pref = (g.dim == 2 ? 4.0 * M_PI * M_PI : 16.0 * M_PI * M_PI) * b0;
    std::vector<double> wr(nq);                       // weight * r^power * pref
    std::vector<double> rad((size_t)bcols * nq);      // J0 or sinc at each node
    for (int q = 0; q < nq; ++q) {
        double r = 0.5 * c * (1.0 + x[q]);
        double pw = (g.dim == 2) ? gamma + 1.0 : gamma + 2.0;
        wr[q] = pref * 0.5 * c * w[q] * pow(r, pw);
        for (int n2 = 0; n2 < bcols; ++n2) {
            double arg = 0.5 * r * sqrt((double)n2);
            rad[(size_t)n2 * nq + q] = (g.dim == 2) ? j0(arg) : sinc(arg);
        }
    }
    F.assign((size_t)arows * bcols, 0.0);
    for (int a2 = 0; a2 < arows; ++a2) {
        const double *ra = &rad[(size_t)a2 * nq];
        for (int b2 = 0; b2 < bcols; ++b2) {
            const double *rb = &rad[(size_t)b2 * nq];
            double s = 0.0;
            // product of the two radial factors first: symmetric in (a2, b2)
            for (int q = 0; q < nq; ++q) s += wr[q] * (ra[q] * rb[q]);
            F[(size_t)a2 * bcols + b2] = s;
        }
    }
}

int grid_create(int dim, int N, double L, bz_grid **out) {
    if (!out) return fail(BZ_EINVAL, "init_velocity_grid: out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(BZ_EINVAL, "init_velocity_grid: dim must be 2 or 3");
    int nmax = (dim == 2) ? 64 : 16;
    if (N < 4 || N > nmax || (N % 2))
        return fail(BZ_EINVAL, "init_velocity_grid: N must be even, 4 <= N <= " + std::to_string(nmax));
    if (!(L > 0.0) || !isfinite(L)) return fail(BZ_EINVAL, "init_velocity_grid: L must be > 0");
    bz_grid *g = (bz_grid *)calloc(1, sizeof(bz_grid));
    if (!g) return fail(BZ_ENOMEM, "init_velocity_grid: host allocation");
    GridView &v = g->v;
    v.dim = dim;
    v.N = N;
    v.h = N / 2 - 1;
    v.M = 2 * v.h + 1;
    v.nv = 1;
    v.nm = 1;
    for (int i = 0; i < dim; ++i) { v.nv *= N; v.nm *= v.M; }
    v.nhalf = (int64_t)(v.h + 1) * (v.nm / v.M);
    v.L = L;
    v.dv = 2.0 * L / N;
    v.s = L / M_PI;
    cudaGetDevice(&g->device);

    // 1-D factors (-1)^k exp(-2 pi i (k j mod N) / N)
    std::vector<double2> E64((size_t)v.M * N);
    std::vector<float2> E32((size_t)v.M * N);
    for (int k = -v.h; k <= v.h; ++k) {
        for (int j = 0; j < N; ++j) {
            long r = ((long)k * j) % N;
            if (r < 0) r += N;
            double ang = 2.0 * M_PI * (double)r / N;
            double sg = (k & 1) ? -1.0 : 1.0;
            double2 e = make_double2(sg * cos(ang), -sg * sin(ang));
            E64[(size_t)(k + v.h) * N + j] = e;
            E32[(size_t)(k + v.h) * N + j] = make_float2((float)e.x, (float)e.y);
        }
    }
    cudaError_t e = dev_malloc(&g->d_E64, sizeof(double2) * E64.size());
    if (e == cudaSuccess) e = dev_malloc(&g->d_E32, sizeof(float2) * E32.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_E64, E64.data(), sizeof(double2) * E64.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_E32, E32.data(), sizeof(float2) * E32.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(g->d_E64);
        dev_free(g->d_E32);
        free(g);
        return cuda_fail(e, "init_velocity_grid: device tables");
    }

    // Gram matrix of the collision invariants phi = (1, v_1..v_d, |v|^2) on the
    // grid and its inverse (used by the conservation projection).
    int nc = dim + 2;
    double Gm[25] = {0}, inv[25] = {0};
    for (int64_t idx = 0; idx < v.nv; ++idx) {
        double phi[5];
        int64_t t = idx;
        double v2 = 0.0;
        for (int i = dim - 1; i >= 0; --i) {
            double vi = -L + (double)(t % N) * v.dv;
            t /= N;
            phi[1 + i] = vi;
            v2 += vi * vi;
        }
        phi[0] = 1.0;
        phi[dim + 1] = v2;
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b) Gm[a * nc + b] += phi[a] * phi[b];
    }
    // Gauss-Jordan with partial pivoting
    double aug[5][10];
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < 2 * nc; ++b) aug[a][b] = (b < nc) ? Gm[a * nc + b] : (b - nc == a ? 1.0 : 0.0);
    for (int c = 0; c < nc; ++c) {
        int p = c;
        for (int r = c + 1; r < nc; ++r)
            if (fabs(aug[r][c]) > fabs(aug[p][c])) p = r;
        if (p != c)
            for (int b = 0; b < 2 * nc; ++b) { double t = aug[c][b]; aug[c][b] = aug[p][b]; aug[p][b] = t; }
        double d = aug[c][c];
        for (int b = 0; b < 2 * nc; ++b) aug[c][b] /= d;
        for (int r = 0; r < nc; ++r) {
            if (r == c) continue;
            double f = aug[r][c];
            for (int b = 0; b < 2 * nc; ++b) aug[r][b] -= f * aug[c][b];
        }
    }
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) inv[a * nc + b] = aug[a][nc + b];
    memcpy(g->cinv, inv, sizeof inv);
    *out = g;
    return BZ_OK;
}

void grid_destroy(bz_grid *g) {
    if (!g) return;
    dev_free(g->d_E64);
    dev_free(g->d_E32);
    free(g);
}

int modes_build_fp32_tables(bz_modes *m);   // k_modesum32.cu host part
void modes_destroy(bz_modes *m);
int64_t symmetric_pair_count(const GridView &g);

int modes_create(const bz_grid *g, double gamma, double b0, int nq, bz_modes **out) {
    if (!out) return fail(BZ_EINVAL, "build_kernel_modes: out is NULL");
    *out = nullptr;
    if (!g) return fail(BZ_EINVAL, "build_kernel_modes: grid is NULL");
    if (!(gamma >= 0.0 && gamma <= 2.0)) return fail(BZ_EINVAL, "build_kernel_modes: gamma in [0,2]");
    if (nq < 0 || nq > 4096) return fail(BZ_EINVAL, "build_kernel_modes: quad_nodes in [0,4096]");
    const GridView &v = g->v;
    bz_modes *m = (bz_modes *)calloc(1, sizeof(bz_modes));
    if (!m) return fail(BZ_ENOMEM, "build_kernel_modes: host allocation");
    m->g = g;
    m->penalty = 1.0;
    m->gamma = gamma;
    m->b0 = (b0 > 0.0) ? b0 : (v.dim == 2 ? 1.0 / (2.0 * M_PI) : 1.0 / (4.0 * M_PI));
    m->nq = nq > 0 ? nq : auto_nodes(v);
    m->arows = v.dim * v.h * v.h + 1;
    m->bcols = v.dim * (2 * v.h) * (2 * v.h) + 1;
    m->scale = pow(v.s, v.dim + gamma);
    std::vector<double> F;
    kernel_table(v, gamma, m->b0, m->nq, m->arows, m->bcols, F);
    size_t nF = F.size();
    m->h_F = (double *)malloc(sizeof(double) * nF);
    if (!m->h_F) { free(m); return fail(BZ_ENOMEM, "build_kernel_modes: host table"); }
    memcpy(m->h_F, F.data(), sizeof(double) * nF);
    std::vector<float> F32(nF);
    for (size_t i = 0; i < nF; ++i) F32[i] = (float)F[i];
    cudaError_t e = dev_malloc(&m->d_F64, sizeof(double) * nF);
    if (e == cudaSuccess) e = dev_malloc(&m->d_F32, sizeof(float) * nF);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_F64, F.data(), sizeof(double) * nF, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_F32, F32.data(), sizeof(float) * nF, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(m->d_F64);
        dev_free(m->d_F32);
        free(m->h_F);
        free(m);
        return cuda_fail(e, "build_kernel_modes: device tables");
    }
    m->pairs_sym = symmetric_pair_count(v);
    int rc = modes_build_fp32_tables(m);
    if (rc == BZ_OK && dft32_tile_supported(v)) {
        rc = dft32_setup();
        m->tile_dft = rc == BZ_OK;
    }
    if (rc != BZ_OK) {
        modes_destroy(m);        // also the variant tables built before the failure
        return rc;
    }
    *out = m;
    return BZ_OK;
}

// Fast spectral form (Sec. 3.3, eq. defQBCarleman / eq. Btilde / eq. FKM /
// eq. ode), 2-D Maxwell molecules |q| sigma = b0.  The Carleman weight is the
// constant 2 b0; with x = rho e_theta, y = rho' e_theta^perp (theta in
// [0, pi), |rho|, |rho'| <= R, R = 2 lambda pi the truncation radius),
//   B_F(l,m) = 2 b0 int_0^pi phi(l.e_theta) phi(m.e_theta^perp) dtheta,
//   phi(xi) = int_{-R}^{R} e^{i rho xi} drho = 2 sin(R xi) / xi,
// and the rectangle rule on theta_p = p pi / A gives the direction factors
// alpha_p(k) = (2 pi b0 / A) phi(k.e_p), alpha'_p(k) = phi(k.e_p^perp).
// The loss weight is Lambda(m) = B_F(m,m) = sum_p alpha_p(m) alpha'_p(m).
// For even A, e_{p+A/2} = e_p^perp and e_{p+A/2}^perp = -e_p, so (with phi
// even) alpha_{p+A/2} = w alpha'_p and alpha'_{p+A/2} = alpha_p / w,
// w = 2 pi b0 / A: the two directions give the same gain product
// IDFT(alpha f-hat) IDFT(alpha' f-hat), and the kernel evaluates A/2 of them
// with weight 2 (the l <-> m symmetry of the gain sum).
int fast_modes_create(const bz_grid *g, double b0, int ndirs, bz_modes **out) {
    if (!out) return fail(BZ_EINVAL, "build_fast_modes: out is NULL");
    *out = nullptr;
    if (!g) return fail(BZ_EINVAL, "build_fast_modes: grid is NULL");
    if (ndirs < 1 || ndirs > 1024) return fail(BZ_EINVAL, "build_fast_modes: n_dirs in [1, 1024]");
    const GridView &v = g->v;
    if (!fast_supported(v))
        return fail(BZ_ENOTSUP, "build_fast_modes: the fast form is built for 2-D grids with N in {8, 16, 24, 32, 48}");
    bz_modes *m = (bz_modes *)calloc(1, sizeof(bz_modes));
    if (!m) return fail(BZ_ENOMEM, "build_fast_modes: host allocation");
    m->g = g;
    m->penalty = 1.0;
    m->gamma = 0.0;
    m->b0 = (b0 > 0.0) ? b0 : 1.0 / (2.0 * M_PI);
    m->scale = pow(v.s, 2.0);
    m->method = 1;
    m->ndirs = ndirs;
    m->nconv = (ndirs % 2 == 0) ? ndirs / 2 : ndirs;
    const int nconv = m->nconv;
    const double cw = (ndirs % 2 == 0) ? 2.0 : 1.0;
    m->variant = -1;
    m->variant64 = -1;
    m->pairs_sym = symmetric_pair_count(v);
    const int M = v.M, h = v.h;
    const size_t nmm = (size_t)M * M;
    const double R = 2.0 * (2.0 / (3.0 + sqrt(2.0))) * M_PI;
    auto phi = [R](double xi) { return xi == 0.0 ? 2.0 * R : 2.0 * sin(R * xi) / xi; };
    const double wa = 2.0 * M_PI * m->b0 / ndirs;
    std::vector<double> cf(2 * (nconv + 1) * nmm, 0.0), lam(nmm, 0.0);
    for (int p = 0; p < ndirs; ++p) {
        const double th = M_PI * p / ndirs, ct = cos(th), st = sin(th);
        for (int k1 = -h; k1 <= h; ++k1)
            for (int k2 = -h; k2 <= h; ++k2) {
                const size_t i = (size_t)(k1 + h) * M + (k2 + h);
                const double a = wa * phi(k1 * ct + k2 * st);      // k . e_p
                const double b = phi(-k1 * st + k2 * ct);          // k . e_p^perp
                if (p < nconv) {
                    cf[2 * ((size_t)p * nmm + i)] = cw * a;
                    cf[2 * ((size_t)p * nmm + i) + 1] = b;
                }
                lam[i] += a * b;
            }
    }
    for (size_t i = 0; i < nmm; ++i) {
        cf[2 * ((size_t)nconv * nmm + i)] = 1.0;
        cf[2 * ((size_t)nconv * nmm + i) + 1] = lam[i];
    }
    std::vector<float> cf32(cf.size());
    for (size_t i = 0; i < cf.size(); ++i) cf32[i] = (float)cf[i];
    m->h_fast = (double *)malloc(sizeof(double) * cf.size());
    cudaError_t e = m->h_fast ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
        memcpy(m->h_fast, cf.data(), sizeof(double) * cf.size());
        e = dev_malloc(&m->d_fast64, sizeof(double) * cf.size());
    }
    if (e == cudaSuccess) e = dev_malloc(&m->d_fast32, sizeof(float) * cf.size());
    if (e == cudaSuccess) e = cudaMemcpy(m->d_fast64, cf.data(), sizeof(double) * cf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_fast32, cf32.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        modes_destroy(m);
        return cuda_fail(e, "build_fast_modes: direction factors");
    }
    int rc = fast_setup();
    if (rc == BZ_OK && dft32_tile_supported(v)) {
        rc = dft32_setup();
        m->tile_dft = rc == BZ_OK;
    }
    if (rc != BZ_OK) {
        modes_destroy(m);
        return rc;
    }
    *out = m;
    return BZ_OK;
}

void modes_destroy(bz_modes *m) {
    if (!m) return;
    dev_free(m->d_fast64);
    dev_free(m->d_fast32);
    free(m->h_fast);
    dev_free(m->d_F64);
    dev_free(m->d_F32);
    dev_free(m->w64);
    dev_free(m->wx2);
    dev_free(m->task64);
    for (int v = 0; v < kModesumVariants; ++v) {
        dev_free(m->var_W[v]);
        dev_free(m->var_task[v]);
        for (int k = 0; k < kSplitTables; ++k) dev_free(m->var_task_split[v][k]);
    }
    free(m->h_F);
    free(m);
}

// beta-hat(l,m) = F(|l+m|^2, |l-m|^2) - F(0, |2m|^2) (the loss weight B-hat(m,m)
// has |l-m| = 0 and is read at the symmetric position).
double beta_host(const bz_modes *m, const int *l, const int *mm) {
    const GridView &v = m->g->v;
    int a2 = 0, b2 = 0, c2 = 0;
    for (int i = 0; i < v.dim; ++i) {
        a2 += (l[i] + mm[i]) * (l[i] + mm[i]);
        b2 += (l[i] - mm[i]) * (l[i] - mm[i]);
        c2 += 4 * mm[i] * mm[i];
    }
    return m->h_F[(size_t)a2 * m->bcols + b2] - m->h_F[c2];
}

// beta-hat_F(l,m) = B_F(l,m) - Lambda(m) of the fast form, from the direction
// factors (flat mode indices of K_h, 2-D).
double fast_beta_host(const bz_modes *m, int64_t li, int64_t mi) {
    const size_t nmm = (size_t)m->g->v.nm;
    const double *c = m->h_fast;
    double acc = 0.0;
    for (int p = 0; p < m->nconv; ++p) {
        if (m->nconv == m->ndirs) {
            acc += c[2 * (p * nmm + li)] * c[2 * (p * nmm + mi) + 1];
        } else {   // directions p and p + A/2 from the stored factors (alpha doubled)
            acc += 0.5 * (c[2 * (p * nmm + li)] * c[2 * (p * nmm + mi) + 1] +
                          c[2 * (p * nmm + li) + 1] * c[2 * (p * nmm + mi)]);
        }
    }
    return acc - c[2 * ((size_t)m->nconv * nmm + mi) + 1];
}

// Unordered pairs {l, m} with l + m = k summed per cell by the symmetric
// kernel, over the half spectrum k_1 >= 0 (the rest follows from Hermitian
// symmetry): for each k, pairs split by l_1 < m_1 (counted once) and the
// diagonal l_1 = m_1 (all of them).
int64_t symmetric_pair_count(const GridView &g) {
    int h = g.h;
    auto count1 = [h](int k) {           // number of l in [-h,h] with k-l in [-h,h]
        int lo = k - h > -h ? k - h : -h, hi = k + h < h ? k + h : h;
        return hi >= lo ? hi - lo + 1 : 0;
    };
    int64_t rest = 0;                       // sum over the remaining d-1 coordinates
    int64_t per = 0;
    for (int k = -h; k <= h; ++k) per += count1(k);
    rest = 1;
    for (int i = 1; i < g.dim; ++i) rest *= per;
    int64_t total = 0;
    for (int k1 = 0; k1 <= h; ++k1) {
        int lo = k1 - h;                        // l1 in [k1-h, floor(k1/2)]
        int hi = k1 / 2;
        total += (int64_t)(hi - lo + 1) * rest;
    }
    return total;
}

}  // namespace bz
