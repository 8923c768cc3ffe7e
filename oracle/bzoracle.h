/*
 * bzoracle.h -- plain FP64 CPU oracle for the spectral Boltzmann collision
 * operator and the local penalised IMEX step of Boscheri & Dimarco
 * (arXiv 2103.14890).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper.  Only the tests, the smoke check of the package entry
 * point and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Conventions (fixed here, restated from the paper in plain terms):
 *   - d in {2,3} velocity dimensions, N (even) points per dimension on the
 *     periodic box [-L,L]^d, dv = 2L/N, v_j = -L + j*dv, j = 0..N-1
 *     (Sec. 3.1, eq. disc_space with a = -L; periodic extension of Sec. 3.3).
 *   - scale s = L/pi maps v to the computational box u = v/s in [-pi,pi)^d
 *     (Sec. 3.3: "take T = pi").
 *   - modes k in K_h = {-h..h}^d with h = N/2 - 1 (the Nyquist mode is
 *     dropped, so Q-hat_0 = 0 exactly and Q is real).
 *   - distribution arrays are [cells][N^d], velocity index row-major
 *     (j_1 slowest).  Mode arrays are [M^d] complex, M = 2h+1, row-major in
 *     (k_1+h, ..., k_d+h), stored as interleaved (re, im) doubles.
 *
 * Parity status of each function is given at its definition in bzoracle.c.
 */
#ifndef BZORACLE_H
#define BZORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;          /* d */
    int N;            /* grid points per dimension */
    int h;            /* largest retained mode, N/2 - 1 */
    int M;            /* modes per dimension, 2h + 1 */
    int64_t nv;       /* N^d */
    int64_t nm;       /* M^d */
    double L;         /* half width of the velocity box */
    double dv;        /* grid spacing 2L/N */
    double s;         /* L / pi */
} orc_grid;

/* Kernel-mode description: B(|q|) = b0 |q|^gamma, radial quadrature with nq
 * Gauss-Legendre nodes, plus a cache of the radial function indexed by the
 * squared integer norms |l+m|^2 and |l-m|^2. */
typedef struct {
    orc_grid g;
    double gamma, b0;
    int nq;
    int arows;        /* cached |l+m|^2 values: 0 .. d h^2 */
    int amax2;        /* largest cached |l-m|^2: d (2h)^2 */
    double *F;        /* arows x (amax2+1) entries, F[a2*(amax2+1)+b2] */
    /* Fast spectral method (Carleman form), 2-D only: ndirs > 0 replaces the
     * radial table by the direction factors below (orc_fast_kernel_init). */
    int ndirs;        /* A, number of collision directions; 0 for eq. KM */
    double *alpha;    /* [ndirs][nm]: alpha_p(k)  */
    double *alphap;   /* [ndirs][nm]: alpha'_p(k) */
    double penalty;   /* c of the Boltzmann model's penalty rate nu = c rho (1 after init) */
} orc_kernel;

int    orc_grid_init(orc_grid *g, int dim, int N, double L);
double orc_velocity(const orc_grid *g, int j);

/* Gauss-Legendre nodes/weights on [-1,1]. */
void   orc_gauss_legendre(int n, double *x, double *w);

/* One radial integral: the kernel mode B-hat(l,m) depends on l and m only
 * through a = |l+m| and b = |l-m|.  Returns B-hat for those norms. */
double orc_radial_Bhat(int dim, double gamma, double b0, int nq, double a, double b);

int    orc_kernel_init(orc_kernel *k, const orc_grid *g, double gamma, double b0, int nq);
void   orc_kernel_free(orc_kernel *k);
/* Fast spectral method of Sec. 3.3 (eq. defQBCarleman, eq. Btilde, eq. FKM,
 * eq. ode) for Maxwell molecules in 2-D (|q| sigma = b0, b0 <= 0: 1/(2 pi)):
 * the kernel modes become B_F(l,m) = sum_p alpha_p(l) alpha'_p(m) over ndirs
 * collision directions.  Every other function below then evaluates the fast
 * operator (orc_Bhat returns B_F, orc_collide and the IMEX step use it).
 * Returns -1 for dim != 2 or ndirs < 1. */
int    orc_fast_kernel_init(orc_kernel *k, const orc_grid *g, double b0, int ndirs);

/* B-hat(l,m) and beta-hat(l,m) = B-hat(l,m) - B-hat(m,m), l,m given as
 * integer d-vectors. */
double orc_Bhat(const orc_kernel *k, const int *l, const int *m);
double orc_beta(const orc_kernel *k, const int *l, const int *m);
/* Full table beta[lidx * nm + midx] (nm^2 doubles) for small grids. */
void   orc_beta_table(const orc_kernel *k, double *beta);
/* beta-hat(l, m) for n pairs of flat mode indices li[p], mi[p] */
void   orc_beta_pairs(const orc_kernel *k, int64_t n, const int64_t *li, const int64_t *mi, double *out);

/* Steps of one collision evaluation (one cell). */
void   orc_dft_forward(const orc_grid *g, const double *f, double *fhat);
void   orc_mode_sum(const orc_kernel *k, const double *fhat, double *Qhat);
void   orc_dft_inverse(const orc_grid *g, const double *Qhat, double scale, double *Q);
void   orc_conserve(const orc_grid *g, double *Q);

/* Whole operator for a batch of cells: Q = s^(d+gamma) Re IDFT(modesum(DFT f)),
 * optionally projected onto the conserving subspace.  OpenMP over cells. */
int    orc_collide(const orc_kernel *k, const double *f, double *Q, int64_t ncells, int conserve);

/* Moments U = (rho, rho u_1..u_d, E) (d+2 values) and the Maxwellian. */
void   orc_moments(const orc_grid *g, const double *f, double *U);
void   orc_maxwellian(const orc_grid *g, const double *U, double *Mout);

/* Penalised IMEX Runge-Kutta local step for a batch of cells.
 *   scheme: 0 = ARS(2,2,2), 1 = BPR(3,4,3), 2 = first-order IMEX Euler
 *   model : 0 = Boltzmann (explicit G = Q - BGK, implicit BGK penalty),
 *           1 = BGK only (G = 0)
 *   Lres  : optional transport residuals [stages][ncells][nv] or NULL.
 * f_out = f^{n+1}. */
int    orc_imex_step(const orc_kernel *k, int scheme, int model, double dt, double eps,
                     const double *f_n, const double *Lres, double *f_out,
                     int64_t ncells, int conserve);

/* Same step, also returning every stage's F, G = Q(F) - P and P = nu (M - F)
 * as [stages][ncells][nv] (any of the three may be NULL). */
int    orc_imex_step_stages(const orc_kernel *k, int scheme, int model, double dt, double eps,
                            const double *f_n, const double *Lres, double *f_out,
                            int64_t ncells, int conserve, double *Fst, double *Gst, double *Pst);

int    orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
