/*
 * bzoracle.c -- plain FP64 CPU oracle (see bzoracle.h for the conventions).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load it; the CUDA library never does.  It is
 * written for readability, not speed: every sum is the definition written
 * out, evaluated in FP64 in the order stated.  The only concession to run
 * time is (i) a table of the 1-D exponentials e^{-i k u_j} used by the DFTs
 * and (ii) a cache of the radial kernel integral indexed by the squared
 * integer norms it depends on.  OpenMP runs independent cells in parallel.
 *
 * Pins (tests/test_oracle_*.py): Lommel closed forms and brute-force
 * quadrature of eq. KM for the kernel modes, exact trigonometric
 * polynomials for the DFTs, brute-force quadrature of the truncated
 * collision integral for the whole operator, the BKW closed form of
 * Sec. 4.1, invariants (mass, equivariance, Q(M) ~ 0) and closed-form
 * amplification factors for the IMEX tableaux.
 */
#include "bzoracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- grid --- */

/* Sec. 3.1 (eq. disc_space): Cartesian grid v_j = j*dv + a with a = -L and the
 * periodic box [-L,L]^d of Sec. 3.3; s = L/pi rescales the box to [-pi,pi]. */
int orc_grid_init(orc_grid *g, int dim, int N, double L) {
    if (!g || (dim != 2 && dim != 3) || N < 4 || (N % 2) || !(L > 0)) return -1;
    g->dim = dim;
    g->N = N;
    g->h = N / 2 - 1;
    g->M = 2 * g->h + 1;
    g->nv = 1;
    g->nm = 1;
    for (int i = 0; i < dim; ++i) { g->nv *= N; g->nm *= g->M; }
    g->L = L;
    g->dv = 2.0 * L / N;
    g->s = L / M_PI;
    return 0;
}

double orc_velocity(const orc_grid *g, int j) { return -g->L + j * g->dv; }

/* split a flat velocity index into its d components (j_1 slowest) */
static void vel_index(const orc_grid *g, int64_t idx, int *j) {
    for (int i = g->dim - 1; i >= 0; --i) { j[i] = (int)(idx % g->N); idx /= g->N; }
}

/* split a flat mode index into its d components k_i in [-h, h] */
static void mode_index(const orc_grid *g, int64_t idx, int *k) {
    for (int i = g->dim - 1; i >= 0; --i) { k[i] = (int)(idx % g->M) - g->h; idx /= g->M; }
}

/* flat mode index of k, or -1 when some |k_i| > h */
static int64_t mode_flat(const orc_grid *g, const int *k) {
    int64_t idx = 0;
    for (int i = 0; i < g->dim; ++i) {
        if (k[i] < -g->h || k[i] > g->h) return -1;
        idx = idx * g->M + (k[i] + g->h);
    }
    return idx;
}

/* ------------------------------------------------------ kernel modes --- */

/* Gauss-Legendre rule on [-1,1]: Newton's method on P_n with the three-term
 * recurrence (textbook construction). */
void orc_gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double p0 = 1.0, p1 = z, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            /* P_n(z) and P_{n-1}(z) by the Bonnet recurrence */
            p0 = 1.0;
            p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);   /* P_n'(z) */
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) <= 1e-15 * fabs(z) + 1e-300) break;
        }
        /* derivative at the converged node */
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Cut-off radius of the relative velocity in the computational box:
 * |q| <= 2R with R = lambda*pi, lambda = 2/(3+sqrt 2) (Sec. 3.3, eq. KM). */
static double cutoff_radius(void) { return 2.0 * (2.0 / (3.0 + sqrt(2.0))) * M_PI; }

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* Eq. KM with sigma independent of the angle and |q| sigma = b0 |q|^gamma.
 * Writing l.q+ + m.q- = ((l+m).q + |q| (l-m).omega)/2, the omega integral over
 * S^{d-1} and the angular part of the q integral are both plane-wave averages:
 *   d=2: int_{S^1} e^{-i x.w} dw = 2 pi J0(|x|),
 *   d=3: int_{S^2} e^{-i x.w} dw = 4 pi sin|x|/|x|,
 * so with a = |l+m|, b = |l-m| and rho = |q|:
 *   d=2: B-hat = b0 (2pi)^2 int_0^{2R} rho^{gamma+1} J0(rho a/2) J0(rho b/2) drho
 *   d=3: B-hat = b0 (4pi)^2 int_0^{2R} rho^{gamma+2} sinc(rho a/2) sinc(rho b/2) drho
 * evaluated here with an nq-point Gauss-Legendre rule on [0, 2R]. */
double orc_radial_Bhat(int dim, double gamma, double b0, int nq, double a, double b) {
    double *x = (double *)malloc(sizeof(double) * nq);
    double *w = (double *)malloc(sizeof(double) * nq);
    orc_gauss_legendre(nq, x, w);
    double Rc = cutoff_radius();
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) {
        double rho = 0.5 * Rc * (x[q] + 1.0);
        double wr = 0.5 * Rc * w[q];
        if (dim == 2)
            acc += wr * pow(rho, gamma + 1.0) * j0(0.5 * rho * a) * j0(0.5 * rho * b);
        else
            acc += wr * pow(rho, gamma + 2.0) * sinc(0.5 * rho * a) * sinc(0.5 * rho * b);
    }
    free(x);
    free(w);
    double c = (dim == 2) ? 2.0 * M_PI : 4.0 * M_PI;
    return b0 * c * c * acc;
}

/* Default node count: enough Gauss-Legendre nodes for the fastest oscillation
 * of the integrand (phase up to 2R (a+b)/2 with a <= h sqrt d, b <= 2h sqrt d). */
static int default_nodes(const orc_grid *g) {
    double phase = cutoff_radius() * 1.5 * g->h * sqrt((double)g->dim);
    int n = (int)ceil(0.75 * phase) + 40;
    return n < 64 ? 64 : n;
}

/* Cache of B-hat over the squared integer norms (|l+m|^2, |l-m|^2).  Each entry
 * is the same Gauss-Legendre sum as orc_radial_Bhat, with the per-node
 * radial factors tabulated once per squared norm.  Rows cover |l+m|^2 <= d h^2
 * (every k = l+m in K_h); columns cover |l-m|^2 <= d (2h)^2.  The loss term
 * B-hat(m,m) has |l-m| = 0 and is read at the transposed position, which holds
 * the same number because F(a,b) is formed symmetrically. */
int orc_kernel_init(orc_kernel *k, const orc_grid *g, double gamma, double b0, int nq) {
    memset(k, 0, sizeof *k);
    k->penalty = 1.0;
    k->g = *g;
    k->gamma = gamma;
    k->b0 = (b0 > 0) ? b0 : (g->dim == 2 ? 1.0 / (2.0 * M_PI) : 1.0 / (4.0 * M_PI));
    k->nq = (nq > 0) ? nq : default_nodes(g);
    k->arows = g->dim * g->h * g->h + 1;
    k->amax2 = g->dim * (2 * g->h) * (2 * g->h);
    int n2 = k->amax2 + 1;
    int nqq = k->nq;
    double *x = (double *)malloc(sizeof(double) * nqq);
    double *w = (double *)malloc(sizeof(double) * nqq);
    double *rad = (double *)malloc(sizeof(double) * (size_t)n2 * nqq);  /* J0 or sinc per node */
    double *wq = (double *)malloc(sizeof(double) * nqq);               /* weight * rho^power */
    k->F = (double *)malloc(sizeof(double) * (size_t)k->arows * n2);
    if (!x || !w || !rad || !wq || !k->F) {
        free(x); free(w); free(rad); free(wq); free(k->F); k->F = NULL;
        return -1;
    }
    orc_gauss_legendre(nqq, x, w);
    double Rc = cutoff_radius();
    double c = (g->dim == 2) ? 2.0 * M_PI : 4.0 * M_PI;
    for (int q = 0; q < nqq; ++q) {
        double rho = 0.5 * Rc * (x[q] + 1.0);
        double p = (g->dim == 2) ? gamma + 1.0 : gamma + 2.0;
        wq[q] = 0.5 * Rc * w[q] * pow(rho, p);
        for (int a2 = 0; a2 < n2; ++a2) {
            double arg = 0.5 * rho * sqrt((double)a2);
            rad[(size_t)a2 * nqq + q] = (g->dim == 2) ? j0(arg) : sinc(arg);
        }
    }
    #pragma omp parallel for schedule(dynamic, 4)
    for (int a2 = 0; a2 < k->arows; ++a2) {
        for (int b2 = 0; b2 < n2; ++b2) {
            double acc = 0.0;
            for (int q = 0; q < nqq; ++q)
                /* the radial product is formed first so that F(a,b) == F(b,a) bitwise */
                acc += wq[q] * (rad[(size_t)a2 * nqq + q] * rad[(size_t)b2 * nqq + q]);
            k->F[(size_t)a2 * n2 + b2] = k->b0 * c * c * acc;
        }
    }
    free(x); free(w); free(rad); free(wq);
    return 0;
}

void orc_kernel_free(orc_kernel *k) {
    free(k->F);
    free(k->alpha);
    free(k->alphap);
    k->F = k->alpha = k->alphap = NULL;
}

/* ------------------------------------------ fast spectral (Carleman) --- */

/* Sec. 3.3, eq. defQBCarleman / eq. Btilde / eq. FKM, for Maxwell molecules
 * in 2-D.  With |q| sigma = b0 the Carleman weight is the constant
 * B-tilde = 2 b0.  Writing x = rho e_theta and y = rho' e_theta^perp
 * (theta in [0, pi), rho and rho' over the whole line) resolves delta(x.y):
 * dx dy delta(x.y) becomes drho drho' dtheta.  The truncation x, y in
 * B_0(R), R = 2 lambda pi (the same radius as |q| <= 2 lambda pi of eq. KM),
 * bounds rho and rho' by R, so
 *   B_F(l,m) = 2 b0 int_0^pi phi(l.e_theta) phi(m.e_theta^perp) dtheta,
 *   phi(xi)  = int_{-R}^{R} e^{i rho xi} drho = 2 sin(R xi) / xi.
 * The theta integral is taken by the ndirs-point rectangle rule on
 * theta_p = p pi / ndirs (the integrand has period pi), which is the
 * decomposition B_F(l,m) ~ sum_p alpha_p(l) alpha'_p(m) that turns eq. ode
 * into ndirs convolutions, with
 *   alpha_p(k) = (2 b0 pi / ndirs) phi(k.e_p),  alpha'_p(k) = phi(k.e_p^perp). */
static double carleman_phi(double xi) {
    double R = cutoff_radius();
    return 2.0 * R * sinc(R * xi);
}

int orc_fast_kernel_init(orc_kernel *k, const orc_grid *g, double b0, int ndirs) {
    if (!k || !g || g->dim != 2 || ndirs < 1) return -1;
    memset(k, 0, sizeof *k);
    k->penalty = 1.0;
    k->g = *g;
    k->gamma = 0.0;
    k->b0 = (b0 > 0) ? b0 : 1.0 / (2.0 * M_PI);
    k->ndirs = ndirs;
    k->alpha = (double *)malloc(sizeof(double) * (size_t)ndirs * g->nm);
    k->alphap = (double *)malloc(sizeof(double) * (size_t)ndirs * g->nm);
    if (!k->alpha || !k->alphap) {
        orc_kernel_free(k);
        return -1;
    }
    double w = 2.0 * k->b0 * M_PI / ndirs;
    int kk[3];
    for (int p = 0; p < ndirs; ++p) {
        double th = M_PI * p / ndirs;
        double e1 = cos(th), e2 = sin(th);          /* e_p */
        for (int64_t ki = 0; ki < g->nm; ++ki) {
            mode_index(g, ki, kk);
            double x = kk[0] * e1 + kk[1] * e2;       /* k . e_p */
            double y = -kk[0] * e2 + kk[1] * e1;      /* k . e_p^perp, e_p^perp = (-sin, cos) */
            k->alpha[(size_t)p * g->nm + ki] = w * carleman_phi(x);
            k->alphap[(size_t)p * g->nm + ki] = carleman_phi(y);
        }
    }
    return 0;
}

/* B_F(l,m) = sum_p alpha_p(l) alpha'_p(m), summed in order of p. */
static double fast_Bhat(const orc_kernel *k, const int *l, const int *m) {
    int64_t li = mode_flat(&k->g, l), mi = mode_flat(&k->g, m);
    double acc = 0.0;
    for (int p = 0; p < k->ndirs; ++p)
        acc += k->alpha[(size_t)p * k->g.nm + li] * k->alphap[(size_t)p * k->g.nm + mi];
    return acc;
}

/* B-hat(l,m) of eq. KM through a = |l+m|, b = |l-m| (or B_F(l,m) of the fast
 * method when the kernel was built by orc_fast_kernel_init). */
double orc_Bhat(const orc_kernel *k, const int *l, const int *m) {
    if (k->ndirs > 0) return fast_Bhat(k, l, m);
    int a2 = 0, b2 = 0;
    for (int i = 0; i < k->g.dim; ++i) {
        a2 += (l[i] + m[i]) * (l[i] + m[i]);
        b2 += (l[i] - m[i]) * (l[i] - m[i]);
    }
    if (a2 >= k->arows) { int t = a2; a2 = b2; b2 = t; }
    if (a2 >= k->arows || b2 > k->amax2)   /* outside the cache: evaluate directly */
        return orc_radial_Bhat(k->g.dim, k->gamma, k->b0, k->nq, sqrt((double)a2), sqrt((double)b2));
    return k->F[(size_t)a2 * (k->amax2 + 1) + b2];
}

/* beta-hat(l,m) = B-hat(l,m) - B-hat(m,m)  (Sec. 3.3, after eq. CF1). */
double orc_beta(const orc_kernel *k, const int *l, const int *m) {
    return orc_Bhat(k, l, m) - orc_Bhat(k, m, m);
}

void orc_beta_table(const orc_kernel *k, double *beta) {
    const orc_grid *g = &k->g;
    int l[3], m[3];
    for (int64_t li = 0; li < g->nm; ++li) {
        mode_index(g, li, l);
        for (int64_t mi = 0; mi < g->nm; ++mi) {
            mode_index(g, mi, m);
            beta[li * g->nm + mi] = orc_beta(k, l, m);
        }
    }
}

/* beta-hat for a list of (l, m) pairs given by flat mode indices: the
 * weights of the terms of eq. CF1 (all pairs the truncated sum visits have
 * l + m in K_h, which the radial cache covers). */
void orc_beta_pairs(const orc_kernel *k, int64_t n, const int64_t *li, const int64_t *mi, double *out) {
    const orc_grid *g = &k->g;
    for (int64_t p = 0; p < n; ++p) {
        int l[3], m[3];
        mode_index(g, li[p], l);
        mode_index(g, mi[p], m);
        out[p] = orc_beta(k, l, m);
    }
}

/* ---------------------------------------------------------- transforms --- */

/* 1-D exponentials E[k+h][j] = e^{-i k u_j} with u_j = -pi + 2 pi j / N,
 * written as (-1)^k e^{-2 pi i (k j mod N)/N} to keep the angle small. */
static void twiddles(const orc_grid *g, double *Ere, double *Eim) {
    for (int k = -g->h; k <= g->h; ++k) {
        for (int j = 0; j < g->N; ++j) {
            long r = ((long)k * j) % g->N;
            if (r < 0) r += g->N;
            double ang = 2.0 * M_PI * (double)r / g->N;
            double sgn = (k % 2 == 0) ? 1.0 : -1.0;
            Ere[(k + g->h) * g->N + j] = sgn * cos(ang);
            Eim[(k + g->h) * g->N + j] = -sgn * sin(ang);
        }
    }
}

/* Eq. FC sampled on the grid: f-hat_k = N^{-d} sum_j f_j e^{-i k . u_j},
 * for every k in K_h.  The d-dimensional exponential is the product of the
 * 1-D ones. */
void orc_dft_forward(const orc_grid *g, const double *f, double *fhat) {
    int n = g->N, M = g->M;
    double *Ere = (double *)malloc(sizeof(double) * M * n);
    double *Eim = (double *)malloc(sizeof(double) * M * n);
    twiddles(g, Ere, Eim);
    double norm = 1.0;
    for (int i = 0; i < g->dim; ++i) norm /= n;
    int k[3], j[3];
    for (int64_t ki = 0; ki < g->nm; ++ki) {
        mode_index(g, ki, k);
        double sre = 0.0, sim = 0.0;
        for (int64_t ji = 0; ji < g->nv; ++ji) {
            vel_index(g, ji, j);
            double pre = 1.0, pim = 0.0;
            for (int i = 0; i < g->dim; ++i) {
                double ere = Ere[(k[i] + g->h) * n + j[i]];
                double eim = Eim[(k[i] + g->h) * n + j[i]];
                double t = pre * ere - pim * eim;
                pim = pre * eim + pim * ere;
                pre = t;
            }
            sre += f[ji] * pre;
            sim += f[ji] * pim;
        }
        fhat[2 * ki] = norm * sre;
        fhat[2 * ki + 1] = norm * sim;
    }
    free(Ere);
    free(Eim);
}

/* Eq. CF1 restricted to K_h: Q-hat_k = sum over l in K_h with m = k - l in K_h
 * of beta-hat(l,m) f-hat_l f-hat_m, accumulated in lexicographic order of l. */
void orc_mode_sum(const orc_kernel *kern, const double *fhat, double *Qhat) {
    const orc_grid *g = &kern->g;
    int k[3], l[3], m[3];
    for (int64_t ki = 0; ki < g->nm; ++ki) {
        mode_index(g, ki, k);
        double are = 0.0, aim = 0.0;
        for (int64_t li = 0; li < g->nm; ++li) {
            mode_index(g, li, l);
            for (int i = 0; i < g->dim; ++i) m[i] = k[i] - l[i];
            int64_t mi = mode_flat(g, m);
            if (mi < 0) continue;
            double b = orc_beta(kern, l, m);
            double lr = fhat[2 * li], lim = fhat[2 * li + 1];
            double mr = fhat[2 * mi], mim = fhat[2 * mi + 1];
            are += b * (lr * mr - lim * mim);
            aim += b * (lr * mim + lim * mr);
        }
        Qhat[2 * ki] = are;
        Qhat[2 * ki + 1] = aim;
    }
}

/* Eq. FU evaluated on the grid and taken back to physical units:
 * Q_j = scale * Re sum_{k in K_h} Q-hat_k e^{i k . u_j}. */
void orc_dft_inverse(const orc_grid *g, const double *Qhat, double scale, double *Q) {
    int n = g->N, M = g->M;
    double *Ere = (double *)malloc(sizeof(double) * M * n);
    double *Eim = (double *)malloc(sizeof(double) * M * n);
    twiddles(g, Ere, Eim);
    int k[3], j[3];
    for (int64_t ji = 0; ji < g->nv; ++ji) {
        vel_index(g, ji, j);
        double sre = 0.0;
        for (int64_t ki = 0; ki < g->nm; ++ki) {
            mode_index(g, ki, k);
            double pre = 1.0, pim = 0.0;   /* e^{+i k.u_j} = conj of the forward factor */
            for (int i = 0; i < g->dim; ++i) {
                double ere = Ere[(k[i] + g->h) * n + j[i]];
                double eim = -Eim[(k[i] + g->h) * n + j[i]];
                double t = pre * ere - pim * eim;
                pim = pre * eim + pim * ere;
                pre = t;
            }
            sre += Qhat[2 * ki] * pre - Qhat[2 * ki + 1] * pim;
        }
        Q[ji] = scale * sre;
    }
    free(Ere);
    free(Eim);
}

/* Collision invariants phi = (1, v_1..v_d, |v|^2) at grid point ji. */
static void invariants(const orc_grid *g, int64_t ji, double *phi) {
    int j[3];
    vel_index(g, ji, j);
    double v2 = 0.0;
    phi[0] = 1.0;
    for (int i = 0; i < g->dim; ++i) {
        double v = orc_velocity(g, j[i]);
        phi[1 + i] = v;
        v2 += v * v;
    }
    phi[1 + g->dim] = v2;
}

/* Solve the n x n system A x = b by Gaussian elimination with partial
 * pivoting (A and b are overwritten). */
static void solve_small(int n, double *A, double *b) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (p != c) {
            for (int q = 0; q < n; ++q) { double t = A[c * n + q]; A[c * n + q] = A[p * n + q]; A[p * n + q] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int q = c; q < n; ++q) A[r * n + q] -= f * A[c * n + q];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int q = r + 1; q < n; ++q) s -= A[r * n + q] * b[q];
        b[r] = s / A[r * n + r];
    }
}

/* Conservation fix (Sec. 3.1 notes that truncation breaks conservation and
 * cites fixes): the smallest L2 change of Q that makes the discrete moments of
 * (1, v, |v|^2) vanish, Q <- Q - C^T (C C^T)^{-1} C Q with C the (d+2) x N^d
 * matrix of collision invariants on the grid. */
void orc_conserve(const orc_grid *g, double *Q) {
    int nc = g->dim + 2;
    double A[25], b[5], phi[5];
    memset(A, 0, sizeof A);
    memset(b, 0, sizeof b);
    for (int64_t ji = 0; ji < g->nv; ++ji) {
        invariants(g, ji, phi);
        for (int r = 0; r < nc; ++r) {
            b[r] += phi[r] * Q[ji];
            for (int c = 0; c < nc; ++c) A[r * nc + c] += phi[r] * phi[c];
        }
    }
    solve_small(nc, A, b);
    for (int64_t ji = 0; ji < g->nv; ++ji) {
        invariants(g, ji, phi);
        double corr = 0.0;
        for (int r = 0; r < nc; ++r) corr += phi[r] * b[r];
        Q[ji] -= corr;
    }
}

/* One collision evaluation: Sec. 3.3 steps (DFT, eq. CF1, inverse DFT) and the
 * physical scale.  With v = s u the collision integral picks up dv_* = s^d du_*
 * and |q|^gamma = s^gamma |q_u|^gamma, so Q(f)(v) = s^{d+gamma} Q_u(f)(u). */
static void collide_one(const orc_kernel *k, const double *f, double *Q, int conserve,
                        double *fhat, double *Qhat) {
    const orc_grid *g = &k->g;
    orc_dft_forward(g, f, fhat);
    orc_mode_sum(k, fhat, Qhat);
    double scale = pow(g->s, g->dim + k->gamma);
    orc_dft_inverse(g, Qhat, scale, Q);
    if (conserve) orc_conserve(g, Q);
}

int orc_collide(const orc_kernel *k, const double *f, double *Q, int64_t ncells, int conserve) {
    const orc_grid *g = &k->g;
    int err = 0;
    #pragma omp parallel
    {
        double *fhat = (double *)malloc(sizeof(double) * 2 * g->nm);
        double *Qhat = (double *)malloc(sizeof(double) * 2 * g->nm);
        if (!fhat || !Qhat) {
            #pragma omp atomic write
            err = -1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t c = 0; c < ncells; ++c)
                collide_one(k, f + c * g->nv, Q + c * g->nv, conserve, fhat, Qhat);
        }
        free(fhat);
        free(Qhat);
    }
    return err;
}

/* --------------------------------------------- moments and Maxwellian --- */

/* Eq. Mo on the grid: rho = dv^d sum f, rho u = dv^d sum v f,
 * E = (1/2) dv^d sum |v|^2 f. */
void orc_moments(const orc_grid *g, const double *f, double *U) {
    int d = g->dim;
    double w = 1.0;
    for (int i = 0; i < d; ++i) w *= g->dv;
    double phi[5], acc[5] = {0, 0, 0, 0, 0};
    for (int64_t ji = 0; ji < g->nv; ++ji) {
        invariants(g, ji, phi);
        for (int r = 0; r < d + 2; ++r) acc[r] += phi[r] * f[ji];
    }
    for (int r = 0; r < d + 1; ++r) U[r] = w * acc[r];
    U[d + 1] = 0.5 * w * acc[d + 1];
}

/* Eq. M sampled at the grid points (the "e.g." choice of Sec. 3.1), with
 * u = (rho u)/rho and theta from E = (d/2) rho theta + (1/2) rho |u|^2. */
void orc_maxwellian(const orc_grid *g, const double *U, double *Mout) {
    int d = g->dim;
    double rho = U[0], u[3] = {0, 0, 0}, u2 = 0.0;
    for (int i = 0; i < d; ++i) { u[i] = U[1 + i] / rho; u2 += u[i] * u[i]; }
    double theta = (2.0 * U[d + 1] / rho - u2) / d;
    double pref = rho / pow(2.0 * M_PI * theta, 0.5 * d);
    int j[3];
    for (int64_t ji = 0; ji < g->nv; ++ji) {
        vel_index(g, ji, j);
        double r2 = 0.0;
        for (int i = 0; i < d; ++i) { double dvi = orc_velocity(g, j[i]) - u[i]; r2 += dvi * dvi; }
        Mout[ji] = pref * exp(-r2 / (2.0 * theta));
    }
}

/* ------------------------------------------------------------- IMEX --- */

#define MAXS 5

/* Butcher tableaux of Sec. 3.4.  Explicit At (strictly lower) and implicit
 * A (lower, diagonal included); all three schemes are stiffly accurate (last
 * row = weights), so f^{n+1} is the last stage value. */
static int tableau(int scheme, int *s, double At[MAXS][MAXS], double A[MAXS][MAXS]) {
    memset(At, 0, sizeof(double) * MAXS * MAXS);
    memset(A, 0, sizeof(double) * MAXS * MAXS);
    if (scheme == 0) {               /* ARS(2,2,2) */
        double gm = 1.0 - 1.0 / sqrt(2.0);
        double dl = 1.0 - 1.0 / (2.0 * gm);
        *s = 3;
        At[1][0] = gm;
        At[2][0] = dl; At[2][1] = 1.0 - dl;
        A[1][1] = gm;
        A[2][1] = 1.0 - gm; A[2][2] = gm;
        return 0;
    }
    if (scheme == 1) {               /* BPR(3,4,3) */
        *s = 5;
        At[1][0] = 1.0;
        At[2][0] = 4.0 / 9.0; At[2][1] = 2.0 / 9.0;
        At[3][0] = 0.25; At[3][2] = 0.75;
        At[4][0] = 0.25; At[4][2] = 0.75;
        A[1][0] = 0.5; A[1][1] = 0.5;
        A[2][0] = 5.0 / 18.0; A[2][1] = -1.0 / 9.0; A[2][2] = 0.5;
        A[3][0] = 0.5; A[3][3] = 0.5;
        A[4][0] = 0.25; A[4][2] = 0.75; A[4][3] = -0.5; A[4][4] = 0.5;
        return 0;
    }
    if (scheme == 2) {               /* first-order IMEX Euler: forward Euler for
                                        the explicit part, backward Euler for the
                                        implicit penalty (Sec. 3.4 names it but
                                        prints no tableau) */
        *s = 2;
        At[1][0] = 1.0;
        A[1][1] = 1.0;
        return 0;
    }
    return -1;
}

/* Penalised IMEX step of Sec. 3.4 (eq. Bref2 and the scheme after it) for one
 * cell, with the cell-centred BGK operator nu (M - F) implicit and
 * G = Q - nu (M - F) explicit.  The paper leaves the penalty rate nu open:
 * nu = rho for the BGK model (its collision frequency) and nu = c rho for the
 * Boltzmann model, c = k->penalty (1 unless set).  Stage l:
 *   R_l = f^n + dt sum_{m<l} [ At_lm (G_m/eps - L_m) + A_lm P_m/eps ]
 *   U_l = moments(R_l), nu_l = rho_l (times c for Boltzmann), M_l = M[U_l]
 *   F_l = (R_l + dt A_ll (nu_l/eps) M_l) / (1 + dt A_ll nu_l/eps)
 *   P_l = nu_l (M_l - F_l),   G_l = Q(F_l) - P_l  (Boltzmann) or 0 (BGK).
 * G enters with a plus sign, consistent with eq. Bref2.  The stage moments are
 * the discrete moments of R_l (equal to the paper's flux-only update whenever
 * the collision term conserves them). */
static void imex_one(const orc_kernel *k, int s, double At[MAXS][MAXS], double A[MAXS][MAXS],
                     int model, double dt, double eps, const double *fn,
                     const double *Lres, int64_t lstride, double *out,
                     double *F, double *G, double *P, double *R, double *Mx, double *Qv,
                     double *fhat, double *Qhat, int conserve,
                     double *Fst, double *Gst, double *Pst, int64_t sstride) {
    const orc_grid *g = &k->g;
    int64_t nv = g->nv;
    int d = g->dim;
    for (int l = 0; l < s; ++l) {
        for (int64_t j = 0; j < nv; ++j) {
            double r = fn[j];
            for (int m = 0; m < l; ++m) {
                double lm = Lres ? Lres[m * lstride + j] : 0.0;
                r += dt * (At[l][m] * (G[m * nv + j] / eps - lm) + A[l][m] * P[m * nv + j] / eps);
            }
            R[j] = r;
        }
        double U[5];
        orc_moments(g, R, U);
        orc_maxwellian(g, U, Mx);
        double nu = (model == 0) ? k->penalty * U[0] : U[0];
        double c = dt * A[l][l] * nu / eps;
        (void)d;
        for (int64_t j = 0; j < nv; ++j) {
            F[l * nv + j] = (R[j] + c * Mx[j]) / (1.0 + c);
            P[l * nv + j] = nu * (Mx[j] - F[l * nv + j]);
        }
        int need_G = 0;
        for (int q = l + 1; q < s; ++q) if (At[q][l] != 0.0) need_G = 1;
        if (model == 0 && need_G) {
            collide_one(k, F + l * nv, Qv, conserve, fhat, Qhat);
            for (int64_t j = 0; j < nv; ++j) G[l * nv + j] = Qv[j] - P[l * nv + j];
        } else {
            for (int64_t j = 0; j < nv; ++j) G[l * nv + j] = 0.0;
        }
        if (Fst) memcpy(Fst + l * sstride, F + l * nv, sizeof(double) * nv);
        if (Gst) memcpy(Gst + l * sstride, G + l * nv, sizeof(double) * nv);
        if (Pst) memcpy(Pst + l * sstride, P + l * nv, sizeof(double) * nv);
    }
    memcpy(out, F + (s - 1) * nv, sizeof(double) * nv);
}

static int imex_impl(const orc_kernel *k, int scheme, int model, double dt, double eps,
                     const double *f_n, const double *Lres, double *f_out, int64_t ncells,
                     int conserve, double *Fst, double *Gst, double *Pst) {
    int s;
    double At[MAXS][MAXS], A[MAXS][MAXS];
    if (tableau(scheme, &s, At, A)) return -1;
    if (model != 0 && model != 1) return -1;
    const orc_grid *g = &k->g;
    int64_t nv = g->nv;
    int err = 0;
    #pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * (size_t)nv * (3 * MAXS + 3));
        double *fh = (double *)malloc(sizeof(double) * 4 * g->nm);
        if (!buf || !fh) {
            #pragma omp atomic write
            err = -1;
        } else {
            double *F = buf, *G = F + MAXS * nv, *P = G + MAXS * nv;
            double *R = P + MAXS * nv, *Mx = R + nv, *Qv = Mx + nv;
            #pragma omp for schedule(dynamic, 1)
            for (int64_t c = 0; c < ncells; ++c) {
                imex_one(k, s, At, A, model, dt, eps, f_n + c * nv,
                         Lres ? Lres + c * nv : NULL, ncells * nv, f_out + c * nv,
                         F, G, P, R, Mx, Qv, fh, fh + 2 * g->nm, conserve,
                         Fst ? Fst + c * nv : NULL, Gst ? Gst + c * nv : NULL,
                         Pst ? Pst + c * nv : NULL, ncells * nv);
            }
        }
        free(buf);
        free(fh);
    }
    return err;
}

int orc_imex_step(const orc_kernel *k, int scheme, int model, double dt, double eps,
                  const double *f_n, const double *Lres, double *f_out,
                  int64_t ncells, int conserve) {
    return imex_impl(k, scheme, model, dt, eps, f_n, Lres, f_out, ncells, conserve,
                     NULL, NULL, NULL);
}

/* Same step, also returning every stage's F, G and P ([stages][ncells][nv]). */
int orc_imex_step_stages(const orc_kernel *k, int scheme, int model, double dt, double eps,
                         const double *f_n, const double *Lres, double *f_out,
                         int64_t ncells, int conserve, double *Fst, double *Gst, double *Pst) {
    return imex_impl(k, scheme, model, dt, eps, f_n, Lres, f_out, ncells, conserve,
                     Fst, Gst, Pst);
}
