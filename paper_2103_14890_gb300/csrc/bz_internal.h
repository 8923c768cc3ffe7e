// bz_internal.h -- internal declarations shared by the host set-up code, the
// C ABI and the CUDA kernels of the spectral collision library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/bzcoll.h"

namespace bz {

constexpr int kMaxDim = 3;
constexpr int kTile = 32;          // cells per tile in the Fourier scratch layout

// Set the thread-local message and return `code`.
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// Device memory the library holds beyond one call (grid, kernel and mesh
// tables, the autotuner's batch, cached graph scratch, the error word).  Every
// such block goes through dev_malloc / dev_free, which count the live blocks;
// alloc_fault_due() consumes one step of the host-side failure countdown that
// bz_inject_alloc_failure arms (true: fail this allocation without calling
// CUDA).  The per-call pool scratch draws on the same countdown.
cudaError_t dev_malloc(void **p, size_t bytes);
template <typename X> cudaError_t dev_malloc(X **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
void dev_free(void *p);
bool alloc_fault_due();

// Device error word (one per device context), latched by kernels.
enum DeviceError : int { kDevOk = 0, kDevNonFinite = 1, kDevTimeout = 2 };

// Kernel-facing view of a grid.
struct GridView {
    int dim, N, h, M;
    int64_t nv;        // N^d
    int64_t nm;        // M^d (full mode set)
    int64_t nhalf;     // (h+1) M^(d-1): modes with k_1 >= 0
    double L, dv, s;
};

}  // namespace bz

struct bz_grid {
    bz::GridView v;
    int device;
    // 1-D DFT factors E[k+h][j] = (-1)^k exp(-2 pi i (k j mod N)/N), k in K_h.
    double2 *d_E64;
    float2 *d_E32;
    // conservation: inverse Gram matrix of the invariants (1, v, |v|^2) on the grid
    double cinv[25];
};

constexpr int kModesumVariants = 10;   // register-blocked FP32 mode-sum kernel variants
constexpr int kSplitTables = 3;       // task tables for a tile split over 2, 4, 8 CTAs

struct bz_modes {
    const bz_grid *g;
    double gamma, b0;
    int nq;
    // radial table F(a2, b2) = B-hat for |l+m|^2 = a2 <= d h^2, |l-m|^2 = b2 <= d (2h)^2
    int arows, bcols;
    double *h_F;        // host copy (FP64)
    double *d_F64;
    float *d_F32;
    // symmetric weight streams and task tables of the FP32 2-D kernel, one per
    // variant (k_modesum32.cu); d_W32 / d_task / w32_rowmax alias the variant
    // in use (null if the generic kernel serves this grid)
    float *var_W[kModesumVariants];
    int *var_task[kModesumVariants];
    int *var_task_split[kModesumVariants][kSplitTables];   // 32-cell variants: tile split over 2, 4, 8 CTAs
    int var_rowmax[kModesumVariants];
    int variant;          // index of the selected variant
    int variant_fixed;    // 1: chosen by BZ_MODESUM_VARIANT (no last-wave split)
    void *w64;            // FP64 weight stream and task table, null if unused
    int *task64;
    int rowmax64;
    int variant64;        // layout of the FP64 tables (entry of the variant list), -1 if none
    float *wx2;           // FP32X2 weight stream: the FP64 stream's layout and task table, each
                          // step's weights as FP32 (hi, lo) parts; null if unused
    int modesum_variant;  // variant id reported to callers (index + 1; 0: generic kernel)
    float *d_W32;
    int w32_rowmax;       // largest staged weight row (floats)
    int *d_task;
    int64_t pairs_sym;   // unordered pairs per cell (algorithmic unit)
    int tile_dft;        // 1: the tile FFT kernels of k_dft32.cu serve this grid
    double scale;        // s^(d + gamma)
    double penalty;      // c of the Boltzmann model's penalty rate nu = c rho (IMEX stages)
    // fast spectral (Carleman) form, k_fast.cu: method 1 replaces the mode sum
    // of eq. CF1 by nconv + 1 FFT convolutions with the direction factors
    // [(nconv + 1)][M][M] complex: (c_p alpha_p + i alpha'_p)(k), then
    // (1 + i Lambda)(k).  For even ndirs, direction p + ndirs/2 is direction p
    // with alpha and alpha' exchanged (same gain product), so nconv = ndirs/2
    // and c_p = 2; for odd ndirs nconv = ndirs and c_p = 1.
    int method;          // 0: eq. KM / eq. CF1 direct sum; 1: fast form
    int ndirs;
    int nconv;
    double *h_fast;      // host FP64 copy (interleaved re, im)
    double2 *d_fast64;
    float2 *d_fast32;
};

namespace bz {
// Finite-volume mesh of the transport step (fv_mesh.cpp, k_transport.cu):
// polygonal cells with at most kFvMaxFaces faces, per-cell tables in
// [cell][slot] layout, FP64 and FP32 copies of the real-valued ones.
constexpr int kFvMaxFaces = 8;
constexpr int kFvCentral = 5;       // central stencil: the cell and its 5 nearest cells (2 x 3 cells)
constexpr int kFvCentral3 = 11;     // degree 2: the cell and its 11 nearest cells (2 x 6 cells)
constexpr int kFvCoef3 = 5;         // degree 2: coefficients of xi, eta, xi^2, xi eta, eta^2
constexpr int kFvRegularTri = 0x100;  // flag in ncen: a triangle whose stencil starts with its 3 face neighbours

template <typename T> struct FvTables {
    const T *inv_area;      // [cell]
    const T *h2;            // [cell] h_i^2
    const T *fn;            // [cell][face][2]  |e| n_e
    const T *off_i;         // [cell][face][2]  x_face - x_b,i
    const T *off_j;         // [cell][face][2]  x_face - x_b,j (neighbour side)
    const T *Rc;            // [cell][2][kFvCentral] least-squares gradient rows
    const T *Rs;            // [cell][face][4]  sector inverses (row-major 2 x 2); degree 2: in the
                            //                   scaled coordinates (x - x_b) / h
};
// Degree-2 reconstruction (order 3): zero-mean scaled Taylor basis
// phi = (xi, eta, xi^2 - mu20, xi eta - mu11, eta^2 - mu02), xi = (x - x_b)/h.
template <typename T> struct FvTables3 {
    const T *mu;            // [cell][3]  cell means of xi^2, xi eta, eta^2
    const T *Rc;            // [cell][5][kFvCentral3] least-squares coefficient rows
    const T *phi_i;         // [cell][face][2 Gauss points][5] basis of the cell at the face's Gauss points
    const T *phi_j;         // [cell][face][2][5] the neighbour's basis at the same points
};
}  // namespace bz

struct bz_mesh {
    int device;
    int order;              // 1: piecewise constant, 2: CWENO of degree 1, 3: CWENO of degree 2
    int64_t n_cells, n_faces_interior, n_faces_boundary;
    int max_faces;
    int *d_nface;           // [cell] faces
    int *d_nb;              // [cell][face] neighbour, -1 boundary
    // triangle meshes (max_faces <= 3): per position p of the processing order
    // three int4 {i, ncen[i], nsec[i], qbits}, {cen[i][0..3]}, {cen[i][4], nb[i][0..2]}
    // with i = order[p] and qbits holding, in 2 bits per face, the index of
    // the same face in the neighbour; one level of loads gives a block all its
    // indices
    int4 *d_tripos;
    int *d_ncen;            // [cell] central stencil size (<= kFvCentral), | kFvRegularTri for a triangle
                            // whose stencil starts with its face neighbours, sector s on faces s, s+1
    int *d_cen;             // [cell][kFvCentral]
    int *d_nsec;            // [cell] sectors
    int *d_sec;             // [cell][face][2] sector cells
    int *d_order;           // [cell] processing order: cells sorted along a Morton curve of their barycentres
    // walls with full accommodation (fv_mesh_set_walls): per face the wall
    // index (-1: none), per wall (theta_w, u_w1, u_w2) in FP64 and FP32
    int *d_wall;
    double *d_wall64;
    float *d_wall32;
    int64_t n_walls;
    // host copies for the wall look-up: counter-clockwise vertex lists (CSR)
    // and the neighbour of every face
    int64_t *h_ptr, *h_vtx;
    int *h_nb;
    void *d_real64;         // one block holding the FvTables<double> arrays
    void *d_real32;         // one block holding the FvTables<float> arrays
    bz::FvTables<double> t64;
    bz::FvTables<float> t32;
    // order 3 only
    int *d_ncen3;           // [cell] central stencil size (<= kFvCentral3)
    int *d_cen3;            // [cell][kFvCentral3]
    void *d_real3_64, *d_real3_32;
    bz::FvTables3<double> u64;
    bz::FvTables3<float> u32;
};

namespace bz {

// ---- kernels (k_dft.cu) ---------------------------------------------------
// Forward DFT of f [n][N^d] into the tiled half spectrum fhat
// [ceil(n/32)][nhalf][32] complex.  hi/lo split output when lo != nullptr.
cudaError_t launch_dft_forward_f64(const GridView &g, const double2 *E, const double *f,
                                   double2 *fhat, int64_t n, cudaStream_t st);
cudaError_t launch_dft_forward_f32(const GridView &g, const float2 *E, const float *f,
                                   float2 *fhat, int64_t n, cudaStream_t st);
// FP64 transform of FP32 input (the FP32X2 form's forward DFT).
cudaError_t launch_dft_forward_f64_f32in(const GridView &g, const double2 *E, const float *f,
                                         double2 *fhat, int64_t n, cudaStream_t st);

// Inverse Gram matrix of the collision invariants, passed by value to kernels.
struct Cinv {
    double v[25];
};

// Epilogue options of the inverse DFT.
struct InvEpilogue {
    int conserve;             // apply the conservation projection
    int check;                // unused here (input check is done on f)
    const void *P;            // if non-null: write G = Q - P instead of Q
};
cudaError_t launch_dft_inverse_f64(const GridView &g, const double2 *E, const double2 *Qhat,
                                   double *Q, int64_t n, double scale, const double *cinv,
                                   const InvEpilogue &ep, cudaStream_t st);
cudaError_t launch_dft_inverse_f32(const GridView &g, const float2 *E, const float2 *Qhat,
                                   float *Q, int64_t n, double scale, const double *cinv,
                                   const InvEpilogue &ep, cudaStream_t st);

// ---- tile FFT kernels (k_dft32.cu), FP32 and FP64, 2-D, N in {16, 24, 32, 48} ----
bool dft32_tile_supported(const GridView &g);
int dft32_setup();   // twiddles on the current device
cudaError_t launch_dft32_forward_tile(const GridView &g, const float *f, float2 *fhat, int64_t n, cudaStream_t st);
cudaError_t launch_dft32_inverse_tile(const GridView &g, const float2 *Qhat, float *Q, int64_t n, double scale,
                                      const double *cinv, const InvEpilogue &ep, cudaStream_t st);
cudaError_t launch_dft64_forward_tile(const GridView &g, const double *f, double2 *fhat, int64_t n,
                                      cudaStream_t st);
cudaError_t launch_dft64_forward_tile_f32in(const GridView &g, const float *f, double2 *fhat, int64_t n,
                                            cudaStream_t st);
cudaError_t launch_dft64_inverse_tile(const GridView &g, const double2 *Qhat, double *Q, int64_t n, double scale,
                                      const double *cinv, const InvEpilogue &ep, cudaStream_t st);

// ---- register-blocked FP32 2-D mode sum (k_modesum32.cu) --------------------
constexpr int kMaxGroup = 16;      // instances per grouped launch
struct Mode32Item {
    const void *fhat;     // float2 or double2 spectra, tiled layout
    void *Qhat;
    const void *W;        // weight stream of the kernel's scalar type
    const int *tasks;     // task table for WARPS x split warps
    int h, M, nhalf, wrow_max;
    int64_t n;
    int split;            // CTAs per tile (1, or 2, 4, 8 for a last partial wave)
};
struct Mode32Group {
    int nitems;
    int64_t tile_start[kMaxGroup + 1];   // prefix sums of 32-cell tiles
    Mode32Item item[kMaxGroup];
};
bool modesum32_available(const bz_modes *m);
cudaError_t launch_modesum32(const bz_modes *m, const float2 *fhat, float2 *Qhat, int64_t n, cudaStream_t st);
int64_t modesum32_split(const bz_modes *m, int64_t n, int *tail_v, int *tail_split);
// Cells one SM holds at a time in the handle's FP32 mode-sum kernel (CTAs per
// SM x cells per CTA; 32 where the register-blocked kernels do not serve it).
int modesum32_wave_cells_per_sm(const bz_modes *m);
// Whether the handle's FP32 mode sum splits the tiles of a partial wave over
// several CTAs (32-cell variants chosen by timing).
bool modesum32_tail_splits(const bz_modes *m);
// Whether batches of at most half a wave run on a one-CTA-per-SM sibling of
// the handle's variant (bit-identical results).
bool modesum32_small_batches_fast(const bz_modes *m);
bool modesum64_available(const bz_modes *m);
cudaError_t launch_modesum64(const bz_modes *m, const double2 *fhat, double2 *Qhat, int64_t n, cudaStream_t st);
cudaError_t launch_modesum32_part(const bz_modes *m, int v, const float2 *fhat, float2 *Qhat, int64_t n,
                                  cudaStream_t st);
// FP32X2 (double-float) mode sum on the FP64 tables: FP64 spectra in, Q-hat
// rounded to FP32 out (k_modesum32.cu).
bool modesum_x2_available(const bz_modes *m);
cudaError_t launch_modesum_x2(const bz_modes *m, const double2 *fhat, float2 *Qhat, int64_t n, cudaStream_t st);
cudaError_t launch_modesum32_group(const bz_modes *const *ms, const float2 *const *fhat, float2 *const *Qhat,
                                   const int64_t *n, int count, cudaStream_t st);

// ---- fast spectral form (k_fast.cu), 2-D, N in {8, 16, 24, 32, 48} --------
bool fast_supported(const GridView &g);
int fast_pad_length(int N);        // P of the zero-padded convolution grid
int fast_cells_per_cta(int N);
int fast_setup();                  // twiddles of k_fast.cu on the current device
cudaError_t launch_fast_f32(const bz_modes *m, const float2 *fhat, float2 *Qhat, int64_t n, cudaStream_t st);
cudaError_t launch_fast_f64(const bz_modes *m, const double2 *fhat, double2 *Qhat, int64_t n, cudaStream_t st);

// ---- kernels (k_modesum.cu) -----------------------------------------------
cudaError_t launch_modesum_generic_f64(const GridView &g, const double *F, int bcols,
                                       const double2 *fhat, double2 *Qhat, int64_t n,
                                       cudaStream_t st);
cudaError_t launch_modesum_generic_f32(const GridView &g, const float *F, int bcols,
                                       const float2 *fhat, float2 *Qhat, int64_t n,
                                       cudaStream_t st);

// ---- kernels (k_imex.cu) --------------------------------------------------
struct StageCoef {
    int stage;                 // 0-based l
    int nprev;                 // l
    double at[5], a[5];        // At[l][m], A[l][m] for m < l
    double all;                // A[l][l]
    double dt, eps;
    double nuf;                // penalty rate nu = nuf * rho
    int store_F;               // 0: F_l equals f^n exactly (stage 0 of a step) and is not written
};
cudaError_t launch_imex_stage_f64(const GridView &g, const StageCoef &c, const double *fn,
                                  double *F, const double *G, double *P, const double *Lres,
                                  int64_t stride, int64_t n, cudaStream_t st);
cudaError_t launch_imex_stage_f32(const GridView &g, const StageCoef &c, const float *fn,
                                  float *F, const float *G, float *P, const float *Lres,
                                  int64_t stride, int64_t n, cudaStream_t st);
cudaError_t launch_check_input_f64(const double *f, int64_t count, int *err, cudaStream_t st);
cudaError_t launch_check_input_f32(const float *f, int64_t count, int *err, cudaStream_t st);
cudaError_t launch_fill_zero(void *p, int64_t bytes, cudaStream_t st);

// ---- transport residual (k_transport.cu) ----------------------------------
// G [cell][2][nv] CWENO gradients (order 2 only), then
// L [cell][nv] = (1/|P_i|) sum_e |e| F_Rusanov(f_L, f_R; v . n_e).
cudaError_t launch_fv_gradient_f64(const bz_mesh *mesh, const GridView &g, const double *f, double *G,
                                   cudaStream_t st);
cudaError_t launch_fv_gradient_f32(const bz_mesh *mesh, const GridView &g, const float *f, float *G,
                                   cudaStream_t st);
cudaError_t launch_fv_flux_f64(const bz_mesh *mesh, const GridView &g, const double *f, const double *G, double *L,
                               cudaStream_t st);
// walls need one CTA to hold all velocities of a cell
bool fv_walls_supported(const bz_mesh *mesh, const GridView &g);
// FP32 triangle meshes without walls (N divisible by 4, 16-byte aligned rows):
// the reconstruction writes each cell's values at its three face midpoints,
// FV [cell][3][nv], and the flux pass reads those of the cell and of its
// neighbours (indices from the position records d_tripos).
bool fv_face_mode(const bz_mesh *mesh, const GridView &g, const void *f, const void *L, const void *FV);
cudaError_t launch_fv_faces_f32(const bz_mesh *mesh, const GridView &g, const float *f, float *FV, cudaStream_t st);
cudaError_t launch_fv_flux_faces_f32(const bz_mesh *mesh, const GridView &g, const float *FV, float *L,
                                     cudaStream_t st);
// order 3: coefficients C [cell][5][nv] of the degree-2 CWENO polynomial, then
// the fluxes at two Gauss points per face
cudaError_t launch_fv_coef3_f64(const bz_mesh *mesh, const GridView &g, const double *f, double *C,
                                cudaStream_t st);
cudaError_t launch_fv_coef3_f32(const bz_mesh *mesh, const GridView &g, const float *f, float *C, cudaStream_t st);
cudaError_t launch_fv_flux3_f64(const bz_mesh *mesh, const GridView &g, const double *f, const double *C,
                                double *L, cudaStream_t st);
cudaError_t launch_fv_flux3_f32(const bz_mesh *mesh, const GridView &g, const float *f, const float *C, float *L,
                                cudaStream_t st);
cudaError_t launch_fv_flux_f32(const bz_mesh *mesh, const GridView &g, const float *f, const float *G, float *L,
                               cudaStream_t st);

// Device error word of the current device (allocated on first use; api.cu).
int *device_error_word();

// One collision evaluation (forward DFT, mode sum, inverse DFT; the launches of
// collide_batch) with the Fourier scratch at `scratch`, which must hold
// collide_scratch_size() bytes; requests no device memory (api.cu).
size_t collide_scratch_size(const bz_modes *m, int precision, int64_t n);
int collide_on_scratch(const bz_modes *m, int precision, int flags, const void *f, void *Q, int64_t n,
                       void *scratch, cudaStream_t st);

}  // namespace bz
