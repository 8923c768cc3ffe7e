/*
 * bzcoll.h -- C ABI of the GB300 spectral Boltzmann collision library.
 *
 * The library evaluates the Fourier-spectral Boltzmann collision operator of
 * Boscheri & Dimarco, "High order finite volume schemes with IMEX time
 * stepping for the Boltzmann model on unstructured meshes" (arXiv 2103.14890),
 * Sec. 3.3, independently in every mesh cell, and the cell-local part of the
 * penalised IMEX Runge-Kutta stage of Sec. 3.4.  Every step runs in
 * hand-written CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by all calls
 * -------------------------------
 *  - Velocity grid (Sec. 3.1, eq. disc_space, with the periodic box of
 *    Sec. 3.3): d in {2,3} dimensions, N (even) points per dimension on
 *    [-L,L]^d, dv = 2L/N, v_j = -L + j dv.  The computational box is
 *    u = v/s in [-pi,pi)^d with s = L/pi.
 *  - Retained Fourier modes: K_h = {-h..h}^d, h = N/2 - 1 (the Nyquist mode
 *    is dropped, so the operator conserves mass exactly and Q is real).
 *  - Distribution arrays (f, Q, stage buffers) are caller-owned DEVICE
 *    pointers, laid out [n_cells][N^d], contiguous, velocity index row-major
 *    (j_1 slowest).  Element type: double for BZ_FP64, float for the mixed
 *    forms.  The physical Q is returned (the 1/eps Knudsen factor is not
 *    applied).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Calls are asynchronous on that stream.  Errors found on
 *    the host are returned at once; errors found by a kernel (non-finite input
 *    under BZ_CHECK_INPUT, a wait that ran out) are latched in a device error
 *    word and returned by bz_check().
 *  - Ownership: handles (bz_grid, bz_modes) and all device tables behind them
 *    are owned by the library and released by the destroy functions.  Scratch
 *    needed by a call is taken from a library-owned stream-ordered memory pool
 *    on the caller's stream and returned on that stream before the call
 *    returns; after the first call of a given size no new device memory is
 *    requested.
 *  - Return codes: 0 on success, a negative BZ_E* code on failure; the
 *    thread-local message is available from bz_last_error().  No C++
 *    exception crosses this boundary.
 */
#ifndef BZCOLL_H
#define BZCOLL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ codes --- */
#define BZ_OK          0
#define BZ_EINVAL     -1   /* bad argument (size, pointer, enum, handle) */
#define BZ_ENOMEM     -2   /* device or host allocation failed */
#define BZ_ECUDA      -3   /* a CUDA runtime call failed */
#define BZ_ENOTSUP    -4   /* configuration not supported in this precision */
#define BZ_ETIMEOUT   -5   /* a kernel wait gave up (device error word) */
#define BZ_ENONFINITE -6   /* non-finite input seen under BZ_CHECK_INPUT */

/* Precision forms of the operator.
 *   BZ_FP64   : every step in FP64 (the plain form).
 *   BZ_FP32   : DFTs and the mode sum in FP32 with compensated accumulation
 *               of the mode sum; moments, Maxwellian and the conservation
 *               fix in FP64.
 *   BZ_FP32X2 : FP32 arrays in and out (as BZ_FP32); the forward DFT in FP64,
 *               the mode sum of eq. CF1 in double-float arithmetic on the FP32
 *               pipe (spectra and weights as FP32 high and low parts, every
 *               product split exactly by FMA, every running sum by TwoSum:
 *               the compensated dot product of Ogita, Rump and Oishi), Q-hat
 *               rounded to FP32, the inverse DFT and the IMEX stage arithmetic
 *               as BZ_FP32.  Its error against the FP64 operator is the FP32
 *               rounding of the result and of the inverse DFT, independent of
 *               the gain/loss cancellation that bounds BZ_FP32.  Served for
 *               the direct sum (build_kernel_modes) on 2-D grids with N <= 48
 *               and 3-D grids with N <= 16; other handles return BZ_ENOTSUP.
 *               Not accepted by collide_batch_noalloc or transport_residual. */
#define BZ_FP64    0
#define BZ_FP32    1
#define BZ_FP32X2  2

/* flags */
#define BZ_CONSERVE     1  /* project Q so its discrete moments of 1, v, |v|^2 vanish */
#define BZ_CHECK_INPUT  2  /* flag non-finite f in the device error word */

/* IMEX schemes (Sec. 3.4) and collision models */
#define BZ_ARS222   0      /* ARS(2,2,2), 3 stages, 2nd order */
#define BZ_BPR343   1      /* BPR(3,4,3), 5 stages, 3rd order */
#define BZ_IMEX_EULER 2    /* first-order IMEX Euler, 2 stages (forward Euler
                              explicit part, backward Euler penalty) */
#define BZ_BOLTZMANN 0     /* explicit G = Q - BGK, implicit BGK penalty */
#define BZ_BGK       1     /* BGK relaxation only (G = 0) */

typedef struct bz_grid bz_grid;    /* opaque, library-owned */
typedef struct bz_modes bz_modes;  /* opaque, library-owned */
typedef struct bz_mesh bz_mesh;    /* opaque, library-owned (transport step) */

/* init_velocity_grid -- Sec. 3.1 (eq. disc_space) and Sec. 3.3 (periodic box,
 * eq. FU / eq. FC).  Builds the velocity grid, the 1-D DFT factors
 * (-1)^k e^{-2 pi i k j/N} for k in K_h in FP64 and FP32 and uploads them to
 * the current CUDA device.
 *   dim          : 2 or 3
 *   n_per_dim    : N, even, 4 <= N <= 64 (2-D) or 4 <= N <= 16 (3-D)
 *   half_width_L : L > 0
 *   out          : receives the handle (NULL on failure)
 * Errors: BZ_EINVAL (bad sizes, out == NULL), BZ_ENOMEM, BZ_ECUDA. */
int init_velocity_grid(int dim, int n_per_dim, double half_width_L, bz_grid **out);

/* build_kernel_modes -- Sec. 3.3, eq. KM and eq. CF1.  Computes on the host, in
 * FP64, the kernel modes B-hat(l,m) for |q| sigma = b0 |q|^gamma by
 * Gauss-Legendre quadrature of the Bessel (2-D) / sinc (3-D) reduced radial
 * integral over |q| <= 2 lambda pi, lambda = 2/(3+sqrt 2), and the weights
 * beta-hat(l,m) = B-hat(l,m) - B-hat(m,m) of the mode sum; uploads FP64 and
 * FP32 copies (plus the symmetrised weight tiles of the FP32 kernels).
 * For 2-D grids with N <= 48 the register-blocked FP32 mode-sum kernel has
 * several variants (see bz_modes_info); the first build for a (dim, N, SM count)
 * times those that fit the grid on the current device (a few ms, zero spectra)
 * and keeps the fastest.  The choice is cached in the process and, if the
 * environment variable BZ_TUNE_CACHE names a writable file, appended there as
 * lines "dim N sms variant" and read back by later processes.
 * BZ_MODESUM_VARIANT=1, 2, 3, 4 or 5 fixes the variant without timing (ignored
 * if that variant does not fit the grid).  With a 32-cell variant chosen by
 * timing, collide calls run the whole waves of CTAs on it and the last partial
 * wave on the 16-cell variant (a second launch); a fixed variant runs every
 * tile.  The call synchronises the current device.
 *   g          : grid handle (not consumed; must outlive the modes handle)
 *   gamma      : 0 = Maxwell molecules, 1 = hard spheres (VHS); 0 <= gamma <= 2
 *   b0         : kernel constant; <= 0 selects 1/(2 pi) in 2-D, 1/(4 pi) in 3-D
 *   quad_nodes : Gauss-Legendre nodes; 0 = automatic (resolves the fastest
 *                oscillation of the integrand for this grid)
 *   out        : receives the handle
 * Errors: BZ_EINVAL, BZ_ENOMEM, BZ_ECUDA. */
int build_kernel_modes(const bz_grid *g, double gamma, double b0, int quad_nodes,
                       bz_modes **out);

/* build_fast_modes -- the fast spectral form of Sec. 3.3 (Carleman
 * representation, eq. defQBCarleman with the weight of eq. Btilde; kernel
 * modes of eq. FKM; mode sum of eq. ode) for 2-D Maxwell molecules,
 * |q| sigma = b0.  With x = rho e_theta, y = rho' e_theta^perp the kernel
 * modes are B_F(l,m) = 2 b0 int_0^pi phi(l.e_theta) phi(m.e_theta^perp) dtheta,
 * phi(xi) = 2 sin(R xi)/xi, R = 2 lambda pi; the rectangle rule on
 * theta_p = p pi / n_dirs splits them into n_dirs products
 * alpha_p(l) alpha'_p(m), and the mode sum becomes n_dirs + 1 convolutions
 * (the last one the loss term B_F(m,m)), evaluated by FFTs on a zero-padded
 * P x P grid (P >= 3h + 1; bz_fast_info).  The direction factors are built on
 * the host in FP64 and uploaded in FP64 and FP32.  The returned handle is a
 * bz_modes accepted by every call that takes one (collide_batch,
 * collide_batch_host, collide_batch_noalloc, group_collide, imex_stage_local,
 * imex_step, bz_modes_beta); those calls then evaluate the fast operator with
 * the same forward / inverse transforms and epilogues.  It does not change
 * the meaning of the precision argument: BZ_FP64 or BZ_FP32 arithmetic.
 *   g      : grid handle, dim = 2 and N in {8, 16, 24, 32, 48}
 *   b0     : kernel constant; <= 0 selects 1/(2 pi)
 *   n_dirs : number of collision directions A, 1 <= A <= 1024
 *   out    : receives the handle (release with bz_modes_destroy)
 * Errors: BZ_EINVAL (NULL pointer, n_dirs out of range), BZ_ENOTSUP (grid not
 * served: 3-D or another N), BZ_ENOMEM, BZ_ECUDA. */
int build_fast_modes(const bz_grid *g, double b0, int n_dirs, bz_modes **out);

/* collide_batch -- one evaluation of Q(f,f) in each of n_cells independent
 * cells (Sec. 3.3: forward DFT, the weighted sum of eq. CF1 over l + m = k in
 * K_h, inverse DFT, times s^(d+gamma) to return to physical units; with
 * BZ_CONSERVE, the smallest L2 correction that zeroes the discrete moments of
 * 1, v, |v|^2).
 *   m         : modes handle
 *   precision : BZ_FP64 (f, Q are double) or BZ_FP32 (float)
 *   flags     : BZ_CONSERVE | BZ_CHECK_INPUT
 *   f, Q      : device arrays [n_cells][N^d]; may not overlap
 *   n_cells   : >= 0 (0 is a no-op)
 * Errors: BZ_EINVAL, BZ_ENOTSUP, BZ_ENOMEM, BZ_ECUDA; device-side
 * BZ_ENONFINITE via bz_check(). */
int collide_batch(const bz_modes *m, int precision, int flags, const void *f, void *Q,
                  int64_t n_cells, void *stream);

/* collide_batch_host -- collide_batch on HOST buffers (the operator of Sec.
 * 3.3 for callers whose distributions live in host memory).
 *   f_host, Q_host : host arrays [n_cells][N^d], float64 for BZ_FP64, float32
 *                    for BZ_FP32; caller-owned, must not overlap
 *   other arguments: as collide_batch
 * The batch moves in chunks of one full wave of the handle's mode-sum kernel
 * (SM count x the cells one SM holds: 7296 cells for the 32x32 grid's
 * three 16-cell CTAs per SM on a 152-SM GPU, 32 x SM count for the fast form;
 * a long batch starts and ends with chunks of 1/8, 1/4 and 1/2 of that, so
 * that the copies that fill and drain the pipeline are short) through two
 * device slots taken from the library's pool in one allocation.  The copies
 * run on two library-owned copy streams; each chunk's forward transform,
 * mode sum and inverse transform run on library-owned streams (the transforms
 * at the greatest stream priority, the mode sums of even and odd chunks on
 * two streams of the least), so that one chunk's mode sum overlaps the
 * previous one's end; all are ordered by events and forked from and joined
 * back to `stream`.  Asynchronous like the other
 * calls: Q_host is complete once `stream` has completed (bz_check(stream) or
 * cudaStreamSynchronize).  The copies overlap only if the host buffers are
 * page-locked (cudaHostAlloc / cudaHostRegister); pageable buffers give the
 * same results without overlap.  Not available inside a stream capture.
 * Errors: as collide_batch; BZ_EINVAL inside a capture. */
int collide_batch_host(const bz_modes *m, int precision, int flags, const void *f_host, void *Q_host,
                       int64_t n_cells, void *stream);

/* imex_stage_local -- stage l (1-based) of the penalised IMEX Runge-Kutta step
 * of Sec. 3.4 (eq. Bref2: Q = G_P + Q_BGK with G_P explicit and the BGK
 * operator nu (M - f) implicit; nu = rho for BZ_BGK, nu = c rho for
 * BZ_BOLTZMANN with c set by bz_modes_set_penalty, 1 by default), cell by cell:
 *   R_l = f^n + dt sum_{m<l} [ At_lm (G_m/eps - L_m) + A_lm P_m/eps ]
 *   U_l = moments(R_l), nu_l = (c) rho_l, M_l = Maxwellian(U_l)   (FP64)
 *   F_l = (R_l + dt A_ll (nu_l/eps) M_l) / (1 + dt A_ll nu_l/eps)
 *   P_l = nu_l (M_l - F_l),  G_l = Q(F_l) - P_l  (G_l = 0 for BZ_BGK or when no
 *   later stage uses it).
 *   scheme      : BZ_ARS222, BZ_BPR343 (tableaux of Sec. 3.4) or BZ_IMEX_EULER
 *                 (the first-order scheme Sec. 3.4 names without a tableau:
 *                 At = [[0,0],[1,0]], A = [[0,0],[0,1]])
 *   stage       : 1 .. stages(scheme)
 *   model       : BZ_BOLTZMANN or BZ_BGK
 *   dt, eps     : time step and Knudsen number (> 0)
 *   f_n         : device [n_cells][N^d]
 *   F, G, P     : device [stages][n_cells][N^d]; slots m < l are read, slot l
 *                 is written (F_l, G_l, P_l)
 *   L_res       : device [stages][n_cells][N^d] transport residuals or NULL (= 0)
 * Element type follows `precision` as for collide_batch.
 * Errors: as collide_batch. */
int imex_stage_local(const bz_modes *m, int scheme, int stage, int model, double dt,
                     double eps, const void *f_n, void *F, void *G, void *P,
                     const void *L_res, int64_t n_cells, int precision, int flags,
                     void *stream);

/* bz_modes_set_penalty -- the penalty rate of the Boltzmann model in the IMEX
 * stages, nu = c rho (Sec. 3.4, eq. Bref2 leaves nu open; the default c = 1).
 * Near the fluid limit the explicit part G_P / eps acts on the distance to
 * equilibrium, and with ARS(2,2,2) that distance is multiplied per step by
 * g(K) = ((1 - d) K^2 + (d - 1 + gamma) K) / gamma, K = 1 + lambda / nu over
 * the spectrum lambda of the linearised Q (gamma = 1 - 1/sqrt 2, d = 1 -
 * 1/(2 gamma)); |g| > 1 for complex K near 0.41, which the spectral Q of
 * Maxwell molecules reaches with c = 1 (eigenvalues down to about -1.03 rho
 * with imaginary parts up to 0.24 rho).  c = 3 keeps K in [0.65, 1] and the
 * step stable.  The BGK model keeps nu = rho (its collision frequency).
 * Changing c drops the CUDA graphs captured by imex_step for these modes.
 * Errors: BZ_EINVAL (NULL modes, c not finite or <= 0). */
int bz_modes_set_penalty(bz_modes *m, double c);

/* imex_step -- all stages of one IMEX step (the schemes are stiffly accurate,
 * so f^{n+1} is the last stage value): f_out = step(f_n).  Stage buffers are
 * library scratch.  L_res as above (NULL = homogeneous step).
 * On a non-default stream that is not being captured, the first call with a
 * given argument set (pointers, n_cells, dt, eps, scheme, model, precision,
 * flags) captures the whole step into a CUDA graph with its own scratch
 * (cudaMalloc, once); later calls with the same arguments replay it with one
 * cudaGraphLaunch.  Up to 8 such graphs are cached (least recently used
 * dropped); destroying the modes handle drops its graphs.  On the legacy
 * stream, or inside a caller's capture, the kernels are launched directly.
 * Errors: as collide_batch. */
int imex_step(const bz_modes *m, int scheme, int model, double dt, double eps,
              const void *f_n, void *f_out, const void *L_res, int64_t n_cells,
              int precision, int flags, void *stream);

/* group_collide -- one collision evaluation for several independent instances
 * (each its own grid N / dimension / kernel and cell batch) in one call.  The
 * FP32 mode sums of all instances served by the register-blocked kernel
 * (2-D N <= 48, 3-D N <= 16) share one launch per kernel variant (up to 16
 * instances per launch, longest first by per-cell work); other instances
 * (and the FP64 and FP32X2 forms) use one launch each.  The instances of one
 * variant, with their forward and inverse DFTs, form a lane; the lanes run on
 * up to four library-owned streams forked from `stream` (longest lane first)
 * and joined back to it, so that one lane's partial waves overlap the others'
 * work.  The call is asynchronous on `stream` like collide_batch: the results
 * are complete once `stream` has completed.  Results equal collide_batch on
 * each instance.
 *   items     : n_items descriptors; item.modes must belong to the current
 *               device; item.f / item.Q are device arrays [n_cells][N^d]
 *   precision : BZ_FP32, BZ_FP32X2 or BZ_FP64 (all items alike)
 *   flags     : BZ_CONSERVE | BZ_CHECK_INPUT, applied to every item
 * Errors: as collide_batch. */
typedef struct bz_group_item {
    const bz_modes *modes;
    const void *f;
    void *Q;
    int64_t n_cells;
} bz_group_item;
int group_collide(const bz_group_item *items, int n_items, int precision, int flags, void *stream);

/* ------------------------------------------------ transport step --- */

/* build_fv_mesh -- the finite-volume mesh of Sec. 3.2: polygonal cells in 2-D
 * physical space, their geometry, face pairing and CWENO stencils.  Cells may
 * be given in either orientation and are stored counter-clockwise; an edge
 * owned by one cell only is a boundary face (transmissive: the outer state
 * equals the inner one).  order 1: piecewise-constant reconstruction (the
 * first-order scheme of eq. finite_vol5); order 2: CWENO of degree 1
 * (eq. CWENO:Popt / CWENO:P0 / CWENO:Prec / eqn.weights): the optimal
 * polynomial by constrained least squares over the cell and its 5 nearest
 * cells (by barycentre, among the cells sharing a vertex with the cell or
 * with one of its vertex neighbours), one sector polynomial per pair of
 * consecutive faces with neighbours on both, linear weights 3/4 (central) and
 * 1/4 shared by the sectors, smoothness h^2 |grad p|^2 (h: largest
 * barycentre-to-vertex distance), eps = 1e-14, r = 4.  order 3: CWENO of
 * degree 2 (the third-order scheme): the optimal quadratic by least squares
 * over the cell and its 11 nearest cells in the zero-mean Taylor basis about
 * the barycentre scaled by h (eq. Dubiner_phi_spatial; cell means of the
 * basis exact for quadratics), the same degree-1 sectors and weights with
 * the indicator extended by the squared scaled second derivatives, and the
 * fluxes at the two Gauss-Legendre points of every face.  The tables are
 * built in FP64 on the host and uploaded to the current device in FP64 and
 * FP32.
 *   n_vertices, xy     : vertices, xy[2 v] = x, xy[2 v + 1] = y (host)
 *   n_cells            : cells, 1 .. 2^30
 *   cell_ptr           : n_cells + 1 offsets into cell_vertices, cell_ptr[0] = 0
 *   cell_vertices      : vertex indices of every cell (3 to 8 per cell)
 *   order              : 1, 2 or 3
 *   out                : receives the handle (release with bz_mesh_destroy)
 * Errors: BZ_EINVAL (bad sizes or indices, degenerate or overlapping cells; for
 * order 3 a neighbourhood that does not determine a quadratic), BZ_ENOMEM,
 * BZ_ECUDA. */
int build_fv_mesh(int n_vertices, const double *xy, int64_t n_cells, const int64_t *cell_ptr,
                  const int64_t *cell_vertices, int order, bz_mesh **out);

/* build_fv_mesh_periodic -- build_fv_mesh on a mesh that is periodic with
 * period Lx in x and/or Ly in y (0: not periodic in that direction), as for
 * the isentropic vortex of Sec. 4.  Vertices whose coordinates agree modulo
 * the periods (within 1e-9 max(Lx, Ly)) are one point; a boundary edge whose
 * periodic image is an edge of another cell pairs with it, and the
 * neighbour's barycentre enters the face offsets, the least-squares stencil
 * and the sectors translated by the multiple of the periods that brings it
 * next to the cell.  Stencil candidates are (cell, translation) pairs, so a
 * cell can appear in a stencil more than once on a mesh that is a few cells
 * wide.  The remaining boundary edges stay transmissive.
 *   Lx, Ly : periods, >= 0 (both 0: the same as build_fv_mesh)
 * Other arguments and errors as build_fv_mesh; BZ_EINVAL also for negative
 * or non-finite periods. */
int build_fv_mesh_periodic(int n_vertices, const double *xy, int64_t n_cells, const int64_t *cell_ptr,
                           const int64_t *cell_vertices, int order, double Lx, double Ly, bz_mesh **out);

/* fv_mesh_set_walls -- make boundary edges walls with full accommodation
 * (Sec. 2, eq. BOU with alpha = 1, eq. MAXB, eq. MU): at a wall face the
 * velocities leaving the domain carry the reconstructed inner value f_L, the
 * velocities entering it carry mu M_w(v), M_w the unit-mass Maxwellian of the
 * wall's temperature and velocity, mu such that the discrete mass fluxes
 * through the face balance, mu sum_{v.n<0} M_w |v.n| = sum_{v.n>0} f_L v.n
 * (n the outer normal).  Boundary edges that are not walls stay transmissive.
 * The call replaces the mesh's walls; n_edges = 0 removes them; on an error
 * the mesh is left without walls.
 *   edge_vertices : 2 n_edges vertex indices (host), each pair a boundary edge
 *                   of the mesh in either order
 *   wall_params   : 3 n_edges values (host): theta_w > 0, u_w1, u_w2
 * A mesh with walls needs N divisible by 4 and N^2 <= 1024 in
 * transport_residual and imex_step_fv (BZ_ENOTSUP otherwise): one CTA forms
 * each cell's mu over all its velocities.
 * On an order-3 mesh the balance holds at each of the face's two Gauss points.
 * Errors: BZ_EINVAL (NULL mesh, not a boundary edge, theta_w <= 0), BZ_ECUDA. */
int fv_mesh_set_walls(bz_mesh *mesh, int64_t n_edges, const int64_t *edge_vertices, const double *wall_params);

/* transport_residual -- <L(f^w)>_x of eq. ho for every cell and discrete
 * velocity: L[i][k] = (1/|P_i|) sum over the faces e of P_i of
 * |e| F(f_L, f_R; v_k . n_e), with F the Rusanov flux of v f,
 * F = (v.n)(f_L + f_R)/2 - |v.n| (f_R - f_L)/2, f_L, f_R the reconstructed
 * values at the face midpoint.  The velocity grid is g's (2-D only; v_k as in
 * the collision operator).
 *   f, L      : device arrays [n_cells][N^2] (n_cells of the mesh), double for
 *               BZ_FP64, float for BZ_FP32; must not overlap
 * Boundary faces are transmissive (the outer state equals the inner one)
 * unless fv_mesh_set_walls made them walls.
 * Scratch (order 2: 2 n_cells N^2 values, 3 n_cells N^2 in FP32 on triangle
 * meshes without walls; order 3: 5 n_cells N^2) comes from the
 * stream-ordered pool.
 * Errors: BZ_EINVAL, BZ_ENOTSUP (3-D grid; walls with N not divisible by 4 or
 * N^2 > 1024), BZ_ECUDA. */
int transport_residual(const bz_mesh *mesh, const bz_grid *g, int precision, const void *f, void *L,
                       void *stream);

/* imex_step_fv -- one penalised IMEX step of the full scheme of Sec. 3.4
 * (eq. GIMEX_n / eq. GIMEX_n2) on the mesh: the stages of imex_step with the
 * transport residual of every stage value computed by transport_residual and
 * entering the explicit part of the later stages.  The correction Delta Q of
 * the paper vanishes for this reconstruction, which keeps the cell averages.
 * f_n, f_out: device arrays [n_cells][N^2]; other arguments as imex_step.
 * Errors: BZ_EINVAL, BZ_ENOTSUP (3-D grid), BZ_ENOMEM, BZ_ECUDA. */
int imex_step_fv(const bz_modes *m, const bz_mesh *mesh, int scheme, int model, double dt, double eps,
                 const void *f_n, void *f_out, int precision, int flags, void *stream);

/* bz_mesh_info -- out[0] = cells, out[1] = interior faces, out[2] = boundary
 * faces, out[3] = most faces of a cell, out[4] = order. */
int bz_mesh_info(const bz_mesh *mesh, int64_t out[5]);

/* bz_mesh_destroy -- release a mesh handle (NULL is ignored). */
void bz_mesh_destroy(bz_mesh *mesh);

/* bz_check -- synchronise `stream`, read and clear the device error word.
 * Returns BZ_OK, BZ_ENONFINITE, BZ_ETIMEOUT or BZ_ECUDA. */
int bz_check(void *stream);

/* bz_last_error -- message of the last failing call on this thread ("" if none). */
const char *bz_last_error(void);

/* bz_modes_info -- sizes of a modes handle: out[0] = dim, out[1] = N,
 * out[2] = h, out[3] = N^d, out[4] = half-spectrum modes (h+1) (2h+1)^(d-1),
 * out[5] = Gauss-Legendre nodes used, out[6] = unordered mode pairs summed
 * per cell by the symmetric FP32 kernel (algorithmic work unit), out[7] =
 * register-blocked FP32 mode-sum variant in use: 1 = 8 outputs per thread,
 * 16 warps, 32-cell tiles; 2 = 4 outputs per thread, 32 warps, 32-cell tiles;
 * 3 = 4 outputs per thread, 16 warps, 16-cell tiles; 4 = 4 outputs per
 * thread, 16 warps, 8-cell tiles (3-D 16^3); 5 = two cells per thread in
 * FP32x2 register pairs, 4 outputs per thread, 16 warps, 32-cell tiles;
 * 0 = FP32 mode sums run on the generic kernel (2-D grids with N > 48). */
int bz_modes_info(const bz_modes *m, int64_t out[8]);

/* bz_fast_info -- out[0] = method of a modes handle (0: eq. KM / eq. CF1
 * direct sum, 1: fast form of build_fast_modes), out[1] = collision
 * directions A, out[2] = padded FFT length P, out[3] = cells per CTA of the
 * fast kernel (out[1..3] are 0 for method 0). */
int bz_fast_info(const bz_modes *m, int64_t out[4]);

/* bz_modes_beta -- copy beta-hat(l,m) for l, m in K_h (row-major flat mode
 * indices, (2h+1)^d each) into host memory `out` ((2h+1)^(2d) doubles); entries
 * with l + m outside K_h are 0. For testing the FP64 quadrature (for a fast
 * handle: sum_p alpha_p(l) alpha'_p(m) - B_F(m,m) from the FP64 factors). */
int bz_modes_beta(const bz_modes *m, double *out);

/* bz_profile -- per-kernel timing for measurement (tracing).  enable = 1
 * clears the record and brackets every kernel the library launches from then
 * on with a pair of CUDA events recorded on the launching stream; enable = 0
 * stops recording.  Not for use during CUDA graph capture.
 * Errors: BZ_ECUDA if events cannot be created. */
int bz_profile(int enable);

/* bz_profile_read -- synchronise on the recorded events and report, per kernel
 * name, the number of launches and their total device time in milliseconds.
 * names: max_kernels slots of 64 bytes (NUL-terminated names); total_ms and
 * launches: max_kernels entries.  Returns the number of kernels written (>= 0)
 * or a negative BZ_E* code.  The record is cleared. */
int bz_profile_read(char *names, int names_bytes, double *total_ms, int64_t *launches,
                    int max_kernels);

/* bz_inject_alloc_failure -- host-side fault injection for tests of the error
 * paths (no GPU fault is involved).  after >= 0 arms a countdown: the
 * library's next `after` device allocations succeed and the one after them
 * fails as if the device were out of memory (the allocation is not attempted),
 * after which injection is off again; after < 0 turns it off.  Counted
 * allocations: the per-call scratch of every entry point (stream-ordered
 * pool), imex_step's graph scratch, the device tables of init_velocity_grid,
 * build_kernel_modes, build_fast_modes, build_fv_mesh(_periodic) and
 * fv_mesh_set_walls, the autotuner's timing batch and the device error word
 * of BZ_CHECK_INPUT / bz_check.  The entry point that meets the failure
 * returns BZ_ENOMEM, releases what it had taken (bz_alloc_stats returns to
 * its earlier values once the stream has completed), writes no handle, and
 * leaves every existing handle usable.  The countdown is process-wide: arm it
 * only while no other thread calls the library.  Returns BZ_OK. */
int bz_inject_alloc_failure(int64_t after);

/* bz_alloc_stats -- live_blocks (process-wide): device blocks the library
 * holds outside its pools (tables of live handles, cached graph scratch,
 * device error words, FFT tables excluded: those are __constant__ data);
 * pool_used_bytes: bytes currently allocated from the library's
 * stream-ordered pools on all devices (zero between calls once their streams
 * have completed).  Either pointer may be NULL.  Errors: BZ_ECUDA. */
int bz_alloc_stats(int64_t *live_blocks, uint64_t *pool_used_bytes);

/* collide_batch_noalloc -- the same operator as collide_batch, for callers
 * that cannot allocate device memory: applications whose device memory is
 * owned by another allocator (a framework's caching allocator, or a host
 * program that reserved the whole device up front), where an allocation by
 * this library would fail or eat into that budget, and real-time loops that
 * must not meet an allocation's latency or an allocation failure part-way
 * through a run.  The paper has no counterpart; this is a deployment
 * convenience of the library.
 *
 * The call requests no device memory and launches exactly the kernels of
 * collide_batch (same results, bit for bit): the Fourier scratch of the cells
 * lives in one file-scope __device__ array of 32 MiB, which every GPU that
 * loads the library holds until the process exits.  That bounds the batch:
 * with S = 32 MiB, at most floor(S / (2 * 32 * H * c)) * 32 cells per call,
 * H = half-spectrum modes (bz_modes_info out[4]), c = 8 bytes (BZ_FP32) or 16
 * (BZ_FP64) -- 4224 cells of a 32x32 grid in FP32, 2112 in FP64, 1856 of a
 * 48x48 grid in FP32.  Larger n_cells are rejected with BZ_EINVAL and a
 * message giving the limit.
 *   precision : BZ_FP32 or BZ_FP64
 *   flags     : 0 or BZ_CONSERVE (BZ_CHECK_INPUT is not accepted: its error
 *               word would be allocated on first use)
 *   f, Q, n_cells, stream : as for collide_batch; the device that owns the
 *               modes handle must be current.
 * Every call shares the one array and the array keeps the last call's
 * contents; nothing in it needs to start at zero (each value a call uses was
 * written earlier by the same call).  Calls that overlap on the GPU (on
 * different streams, or from several host threads without ordering) race on
 * the array and produce wrong results: order them.  Set-up: the first call on
 * each device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture begins, and do not call
 * cudaDeviceReset on a device after its first call (the kept address would be
 * stale).
 * Errors: BZ_EINVAL (arguments, size limit, wrong current device), BZ_ECUDA. */
int collide_batch_noalloc(const bz_modes *m, int precision, int flags, const void *f, void *Q,
                          int64_t n_cells, void *stream);

void bz_grid_destroy(bz_grid *g);
void bz_modes_destroy(bz_modes *m);

#ifdef __cplusplus
}
#endif
#endif
