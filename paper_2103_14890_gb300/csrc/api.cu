// api.cu -- the extern "C" entry points declared in include/bzcoll.h: argument
// checks, scratch from a library-owned stream-ordered pool, and the kernel
// sequences of each call.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "bz_internal.h"

namespace bz {

static thread_local std::string t_err;

int fail(int code, const std::string &msg) {
    t_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    t_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? BZ_ENOMEM : BZ_ECUDA;
}

// Host-side allocation failure injection: -1 = off, k >= 0 = the next k
// allocations succeed and the one after fails (then off again).
static std::atomic<int64_t> g_fail_after{-1};
static std::atomic<int64_t> g_live_blocks{0};

bool alloc_fault_due() {
    int64_t v = g_fail_after.load(std::memory_order_relaxed);
    while (v >= 0)
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}

cudaError_t dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    if (alloc_fault_due()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) *p = nullptr;
    else if (*p) g_live_blocks.fetch_add(1);
    return e;
}

void dev_free(void *p) {
    if (p && cudaFree(p) == cudaSuccess) g_live_blocks.fetch_sub(1);
}

int grid_create(int dim, int N, double L, bz_grid **out);
void grid_destroy(bz_grid *g);
int modes_create(const bz_grid *g, double gamma, double b0, int nq, bz_modes **out);
int fast_modes_create(const bz_grid *g, double b0, int ndirs, bz_modes **out);
int fv_mesh_create(int n_vertices, const double *xy, int64_t n_cells, const int64_t *cell_ptr,
                   const int64_t *cell_vertices, int order, double Lx, double Ly, bz_mesh **out);
void fv_mesh_destroy(bz_mesh *m);
int fv_mesh_set_walls(bz_mesh *m, int64_t n_edges, const int64_t *edges, const double *params);
void modes_destroy(bz_modes *m);
double beta_host(const bz_modes *m, const int *l, const int *mm);
double fast_beta_host(const bz_modes *m, int64_t li, int64_t mi);

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int *g_err_word[kMaxDevices];
cudaMemPool_t g_pool[kMaxDevices];
bool g_pool_ok[kMaxDevices];

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

cudaMemPool_t pool_for(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pool_ok[dev]) {
        cudaMemPoolProps p;
        memset(&p, 0, sizeof p);
        p.allocType = cudaMemAllocationTypePinned;
        p.location.type = cudaMemLocationTypeDevice;
        p.location.id = dev;
        if (cudaMemPoolCreate(&g_pool[dev], &p) != cudaSuccess) return nullptr;
        uint64_t thr = UINT64_MAX;   // keep freed blocks for reuse: no re-allocation after warm-up
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
        g_pool_ok[dev] = true;
    }
    return g_pool[dev];
}

// Stream-ordered scratch block, returned to the pool on the same stream.
struct Scratch {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t alloc(size_t bytes, cudaStream_t s) {
        st = s;
        if (bytes == 0) return cudaSuccess;
        if (alloc_fault_due()) return cudaErrorMemoryAllocation;
        cudaMemPool_t pool = pool_for(current_device());
        if (!pool) return cudaErrorMemoryAllocation;
        return cudaMallocFromPoolAsync(&p, bytes, pool, s);
    }
    ~Scratch() {
        if (p) cudaFreeAsync(p, st);
    }
};

// Switch to the handle's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// ---- optional per-kernel timing (bz_profile) ----
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;

thread_local bool t_capturing = false;     // inside the library's own stream capture

struct ProfScope {
    ProfRec r{nullptr, nullptr, nullptr};
    cudaStream_t st;
    ProfScope(const char *name, cudaStream_t s) : st(s) {
        if (!g_prof_on || t_capturing) return;
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
        r.name = name;
        cudaEventRecord(r.a, st);
    }
    ~ProfScope() {
        if (!r.name) return;
        cudaEventRecord(r.b, st);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.push_back(r);
    }
};

#define BZ_LAUNCH(name, st, expr, what)                     \
    do {                                                    \
        ProfScope _ps(name, st);                            \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_fail(_e, what);  \
    } while (0)

#define BZ_TRY(expr, what)                        \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// Butcher tableaux of Sec. 3.4 (explicit At, implicit A), all stiffly accurate.
struct Tableau {
    int s;
    double At[5][5], A[5][5];
};

bool tableau(int scheme, Tableau &t) {
    memset(&t, 0, sizeof t);
    if (scheme == BZ_ARS222) {
        const double gm = 1.0 - 1.0 / sqrt(2.0), dl = 1.0 - 1.0 / (2.0 * gm);
        t.s = 3;
        t.At[1][0] = gm;
        t.At[2][0] = dl;
        t.At[2][1] = 1.0 - dl;
        t.A[1][1] = gm;
        t.A[2][1] = 1.0 - gm;
        t.A[2][2] = gm;
        return true;
    }
    if (scheme == BZ_BPR343) {
        t.s = 5;
        t.At[1][0] = 1.0;
        t.At[2][0] = 4.0 / 9.0;
        t.At[2][1] = 2.0 / 9.0;
        t.At[3][0] = 0.25;
        t.At[3][2] = 0.75;
        t.At[4][0] = 0.25;
        t.At[4][2] = 0.75;
        t.A[1][0] = 0.5;
        t.A[1][1] = 0.5;
        t.A[2][0] = 5.0 / 18.0;
        t.A[2][1] = -1.0 / 9.0;
        t.A[2][2] = 0.5;
        t.A[3][0] = 0.5;
        t.A[3][3] = 0.5;
        t.A[4][0] = 0.25;
        t.A[4][2] = 0.75;
        t.A[4][3] = -0.5;
        t.A[4][4] = 0.5;
        return true;
    }
    if (scheme == BZ_IMEX_EULER) {
        t.s = 2;
        t.At[1][0] = 1.0;
        t.A[1][1] = 1.0;
        return true;
    }
    return false;
}

int check_modes(const bz_modes *m, int precision, const char *who) {
    if (!m || !m->g) return fail(BZ_EINVAL, std::string(who) + ": modes handle is NULL");
    if (precision != BZ_FP64 && precision != BZ_FP32 && precision != BZ_FP32X2)
        return fail(BZ_EINVAL, std::string(who) + ": unknown precision");
    if (precision == BZ_FP32X2 && (m->method != 0 || !modesum_x2_available(m)))
        return fail(BZ_ENOTSUP, std::string(who) + ": the FP32X2 form serves the direct sum on 2-D grids with "
                                                    "N <= 48 and 3-D grids with N <= 16");
    return BZ_OK;
}


// The three phases of one collision evaluation over n cells, with the Fourier
// scratch fh (forward spectra) and qh (mode sums) in the tiled layout.
int phase_forward(const bz_modes *m, int precision, const void *f, void *fh, int64_t n, cudaStream_t st) {
    const bz_grid *g = m->g;
    const GridView &v = g->v;
    if (precision == BZ_FP32X2 && m->tile_dft) {
        BZ_LAUNCH("dft_forward_x2", st,
                  launch_dft64_forward_tile_f32in(v, static_cast<const float *>(f), static_cast<double2 *>(fh), n, st),
                  "collide: forward DFT");
    } else if (precision == BZ_FP32X2) {
        BZ_LAUNCH("dft_forward_x2_generic", st,
                  launch_dft_forward_f64_f32in(v, g->d_E64, static_cast<const float *>(f), static_cast<double2 *>(fh),
                                               n, st),
                  "collide: forward DFT");
    } else if (precision == BZ_FP64 && m->tile_dft) {
        BZ_LAUNCH("dft_forward_f64", st,
                  launch_dft64_forward_tile(v, static_cast<const double *>(f), static_cast<double2 *>(fh), n, st),
                  "collide: forward DFT");
    } else if (precision == BZ_FP64) {
        BZ_LAUNCH("dft_forward_f64_generic", st,
                  launch_dft_forward_f64(v, g->d_E64, static_cast<const double *>(f), static_cast<double2 *>(fh), n, st),
                  "collide: forward DFT");
    } else if (m->tile_dft) {
        BZ_LAUNCH("dft_forward_f32", st,
                  launch_dft32_forward_tile(v, static_cast<const float *>(f), static_cast<float2 *>(fh), n, st),
                  "collide: forward DFT");
    } else {
        BZ_LAUNCH("dft_forward_f32_generic", st,
                  launch_dft_forward_f32(v, g->d_E32, static_cast<const float *>(f), static_cast<float2 *>(fh), n, st),
                  "collide: forward DFT");
    }
    return BZ_OK;
}

int phase_modesum(const bz_modes *m, int precision, const void *fh, void *qh, int64_t n, cudaStream_t st) {
    const GridView &v = m->g->v;
    if (precision == BZ_FP32X2) {
        BZ_LAUNCH("modesum_x2", st,
                  launch_modesum_x2(m, static_cast<const double2 *>(fh), static_cast<float2 *>(qh), n, st),
                  "collide: mode sum");
    } else if (m->method == 1 && precision == BZ_FP64) {
        BZ_LAUNCH("fast_f64", st,
                  launch_fast_f64(m, static_cast<const double2 *>(fh), static_cast<double2 *>(qh), n, st),
                  "collide: fast spectral convolutions");
    } else if (m->method == 1) {
        BZ_LAUNCH("fast_f32", st,
                  launch_fast_f32(m, static_cast<const float2 *>(fh), static_cast<float2 *>(qh), n, st),
                  "collide: fast spectral convolutions");
    } else if (precision == BZ_FP64 && modesum64_available(m)) {
        BZ_LAUNCH("modesum_f64", st,
                  launch_modesum64(m, static_cast<const double2 *>(fh), static_cast<double2 *>(qh), n, st),
                  "collide: mode sum");
    } else if (precision == BZ_FP64) {
        BZ_LAUNCH("modesum_f64_generic", st,
                  launch_modesum_generic_f64(v, m->d_F64, m->bcols, static_cast<const double2 *>(fh),
                                             static_cast<double2 *>(qh), n, st),
                  "collide: mode sum");
    } else if (modesum32_available(m)) {
        // whole waves on the selected variant, the last partial wave split
        // (one launch), or on the 16-cell variant (a second launch)
        BZ_LAUNCH("modesum_f32", st,
                  launch_modesum32(m, static_cast<const float2 *>(fh), static_cast<float2 *>(qh), n, st),
                  "collide: mode sum");
    } else {
        BZ_LAUNCH("modesum_f32_generic", st,
                  launch_modesum_generic_f32(v, m->d_F32, m->bcols, static_cast<const float2 *>(fh),
                                             static_cast<float2 *>(qh), n, st),
                  "collide: mode sum");
    }
    return BZ_OK;
}

int phase_inverse(const bz_modes *m, int precision, int flags, const void *qh, void *Q, const void *P, int64_t n,
                  cudaStream_t st) {
    const bz_grid *g = m->g;
    const GridView &v = g->v;
    InvEpilogue ep;
    ep.conserve = (flags & BZ_CONSERVE) ? 1 : 0;
    ep.check = 0;
    ep.P = P;
    if (precision == BZ_FP64 && m->tile_dft) {
        BZ_LAUNCH("dft_inverse_f64", st,
                  launch_dft64_inverse_tile(v, static_cast<const double2 *>(qh), static_cast<double *>(Q), n, m->scale,
                                            g->cinv, ep, st),
                  "collide: inverse DFT");
    } else if (precision == BZ_FP64) {
        BZ_LAUNCH("dft_inverse_f64_generic", st,
                  launch_dft_inverse_f64(v, g->d_E64, static_cast<const double2 *>(qh), static_cast<double *>(Q), n,
                                         m->scale, g->cinv, ep, st),
                  "collide: inverse DFT");
    } else if (m->tile_dft) {
        BZ_LAUNCH("dft_inverse_f32", st,
                  launch_dft32_inverse_tile(v, static_cast<const float2 *>(qh), static_cast<float *>(Q), n, m->scale,
                                            g->cinv, ep, st),
                  "collide: inverse DFT");
    } else {
        BZ_LAUNCH("dft_inverse_f32_generic", st,
                  launch_dft_inverse_f32(v, g->d_E32, static_cast<const float2 *>(qh), static_cast<float *>(Q), n,
                                         m->scale, g->cinv, ep, st),
                  "collide: inverse DFT");
    }
    return BZ_OK;
}

// Fourier scratch of one collision evaluation over n cells: the forward
// spectra (FP64 for the FP64 and FP32X2 forms, FP32 otherwise) followed by the
// mode sums (FP64 for the FP64 form, FP32 otherwise), both in the tiled layout.
size_t spectrum_bytes(const bz_modes *m, int precision, int64_t n) {
    const int64_t ntile = (n + kTile - 1) / kTile;
    const size_t celem = (size_t)ntile * m->g->v.nhalf * kTile;
    return celem * (precision == BZ_FP32 ? sizeof(float2) : sizeof(double2));
}

size_t collide_scratch_bytes(const bz_modes *m, int precision, int64_t n) {
    const int64_t ntile = (n + kTile - 1) / kTile;
    const size_t celem = (size_t)ntile * m->g->v.nhalf * kTile;
    return spectrum_bytes(m, precision, n) + celem * (precision == BZ_FP64 ? sizeof(double2) : sizeof(float2));
}

// Q (or G = Q - P when P != nullptr) of n cells: forward DFT, mode sum, inverse DFT.
// Scratch: `ext` if given (collide_scratch_bytes), else the stream-ordered pool.
int collide_chain(const bz_modes *m, int precision, int flags, const void *f, void *Q, const void *P,
                  int64_t n, cudaStream_t st, void *ext = nullptr) {
    const size_t bytes = collide_scratch_bytes(m, precision, n);
    Scratch s;
    if (!ext) BZ_TRY(s.alloc(bytes, st), "collide: scratch");
    char *fh = static_cast<char *>(ext ? ext : s.p), *qh = fh + spectrum_bytes(m, precision, n);
    int rc = phase_forward(m, precision, f, fh, n, st);
    if (!rc) rc = phase_modesum(m, precision, fh, qh, n, st);
    if (!rc) rc = phase_inverse(m, precision, flags, qh, Q, P, n, st);
    return rc;
}

// Transport residual L [cell][nv] of f over the mesh: CWENO gradients into
// scratch (`ext` if given: transport_scratch_bytes), then the fluxes.
size_t transport_scratch_bytes(const bz_mesh *mesh, const bz_grid *g, int precision) {
    if (mesh->order == 1) return 0;
    // values per (cell, velocity): 5 coefficients, 3 face values (FP32 triangles without walls) or 2 gradients
    const bool faces = precision == BZ_FP32 && mesh->max_faces <= 3 && mesh->n_walls == 0;
    const size_t per = mesh->order == 3 ? (size_t)kFvCoef3 : faces ? 3 : 2;
    return per * mesh->n_cells * g->v.nv * (precision == BZ_FP64 ? sizeof(double) : sizeof(float));
}

int transport_chain(const bz_mesh *mesh, const bz_grid *g, int precision, const void *f, void *L, cudaStream_t st,
                    void *ext = nullptr) {
    const GridView &v = g->v;
    if (!fv_walls_supported(mesh, v))
        return fail(BZ_ENOTSUP, "transport: walls need N divisible by 4 and at most 32^2 velocities");
    Scratch s;
    if (mesh->order == 3) {
        if (!ext) BZ_TRY(s.alloc(transport_scratch_bytes(mesh, g, precision), st), "transport: scratch");
        void *C = ext ? ext : s.p;
        if (precision == BZ_FP64) {
            BZ_LAUNCH("fv_coef3_f64", st,
                      launch_fv_coef3_f64(mesh, v, static_cast<const double *>(f), static_cast<double *>(C), st),
                      "transport: reconstruction");
            BZ_LAUNCH("fv_flux3_f64", st,
                      launch_fv_flux3_f64(mesh, v, static_cast<const double *>(f), static_cast<const double *>(C),
                                          static_cast<double *>(L), st),
                      "transport: fluxes");
        } else {
            BZ_LAUNCH("fv_coef3_f32", st,
                      launch_fv_coef3_f32(mesh, v, static_cast<const float *>(f), static_cast<float *>(C), st),
                      "transport: reconstruction");
            BZ_LAUNCH("fv_flux3_f32", st,
                      launch_fv_flux3_f32(mesh, v, static_cast<const float *>(f), static_cast<const float *>(C),
                                          static_cast<float *>(L), st),
                      "transport: fluxes");
        }
        return BZ_OK;
    }
    void *G = nullptr;
    if (mesh->order == 2) {
        if (!ext) BZ_TRY(s.alloc(transport_scratch_bytes(mesh, g, precision), st), "transport: scratch");
        G = ext ? ext : s.p;
        if (precision == BZ_FP32 && fv_face_mode(mesh, v, f, L, G)) {
            BZ_LAUNCH("fv_gradient_f32", st,
                      launch_fv_faces_f32(mesh, v, static_cast<const float *>(f), static_cast<float *>(G), st),
                      "transport: reconstruction");
            BZ_LAUNCH("fv_flux_f32", st,
                      launch_fv_flux_faces_f32(mesh, v, static_cast<const float *>(G), static_cast<float *>(L), st),
                      "transport: fluxes");
            return BZ_OK;
        }
        if (precision == BZ_FP64)
            BZ_LAUNCH("fv_gradient_f64", st,
                      launch_fv_gradient_f64(mesh, v, static_cast<const double *>(f), static_cast<double *>(G), st),
                      "transport: reconstruction");
        else
            BZ_LAUNCH("fv_gradient_f32", st,
                      launch_fv_gradient_f32(mesh, v, static_cast<const float *>(f), static_cast<float *>(G), st),
                      "transport: reconstruction");
    }
    if (precision == BZ_FP64)
        BZ_LAUNCH("fv_flux_f64", st,
                  launch_fv_flux_f64(mesh, v, static_cast<const double *>(f), static_cast<const double *>(G),
                                     static_cast<double *>(L), st),
                  "transport: fluxes");
    else
        BZ_LAUNCH("fv_flux_f32", st,
                  launch_fv_flux_f32(mesh, v, static_cast<const float *>(f), static_cast<const float *>(G),
                                     static_cast<float *>(L), st),
                  "transport: fluxes");
    return BZ_OK;
}

int check_input(int precision, const void *f, int64_t count, cudaStream_t st) {
    int *err = device_error_word();
    if (!err) return fail(BZ_ENOMEM, "device error word allocation failed");
    cudaError_t e = (precision == BZ_FP64) ? launch_check_input_f64(static_cast<const double *>(f), count, err, st)
                                           : launch_check_input_f32(static_cast<const float *>(f), count, err, st);
    if (e != cudaSuccess) return cuda_fail(e, "input check");
    return BZ_OK;
}

// One IMEX stage: F_l, P_l by the stage kernel, then G_l = Q(F_l) - P_l.
// in_step: called by step_sequence (library scratch): stage 0's F (= f^n
// exactly when A_00 = 0) is not written and the collision reads f^n, and the
// last stage's G, which no stage reads, is not zeroed.
int run_stage(const bz_modes *m, const Tableau &t, int l, int model, double dt, double eps, const void *f_n,
              void *F_l, void *G, void *P, const void *L_res, int64_t n, int precision, int flags,
              cudaStream_t st, void *ext = nullptr, bool in_step = false) {
    const GridView &v = m->g->v;
    StageCoef c;
    memset(&c, 0, sizeof c);
    c.stage = l;
    c.nprev = l;
    for (int q = 0; q < l; ++q) {
        c.at[q] = t.At[l][q];
        c.a[q] = t.A[l][q];
    }
    c.all = t.A[l][l];
    c.dt = dt;
    c.eps = eps;
    c.nuf = (model == BZ_BOLTZMANN) ? m->penalty : 1.0;
    const bool f0 = in_step && l == 0 && c.all == 0.0;     // F_0 = f^n
    c.store_F = f0 ? 0 : 1;
    const int64_t stride = n * v.nv;
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    cudaError_t e;
    {
    ProfScope ps(precision == BZ_FP64 ? "imex_stage_f64" : "imex_stage_f32", st);
    if (precision == BZ_FP64)
        e = launch_imex_stage_f64(v, c, static_cast<const double *>(f_n), static_cast<double *>(F_l),
                                  static_cast<const double *>(G), static_cast<double *>(P),
                                  static_cast<const double *>(L_res), stride, n, st);
    else
        e = launch_imex_stage_f32(v, c, static_cast<const float *>(f_n), static_cast<float *>(F_l),
                                  static_cast<const float *>(G), static_cast<float *>(P),
                                  static_cast<const float *>(L_res), stride, n, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "imex stage");
    bool needG = false;
    for (int q = l + 1; q < t.s; ++q)
        if (t.At[q][l] != 0.0) needG = true;
    char *Gl = static_cast<char *>(G) + (size_t)l * stride * es;
    const char *Pl = static_cast<const char *>(P) + (size_t)l * stride * es;
    if (model == BZ_BOLTZMANN && needG)
        return collide_chain(m, precision, flags, f0 ? f_n : F_l, Gl, Pl, n, st, ext);
    if (in_step && l == t.s - 1) return BZ_OK;
    e = launch_fill_zero(Gl, (int64_t)(stride * es), st);
    if (e != cudaSuccess) return cuda_fail(e, "imex stage: zero G");
    return BZ_OK;
}

// ---- CUDA-graph cache of imex_step ----
// One captured graph per distinct argument set (pointers, sizes, dt, eps,
// scheme, model, precision, flags); each entry owns its scratch, allocated
// once outside the capture.  Replays cost one cudaGraphLaunch.
struct StepKey {
    const bz_modes *m;
    int scheme, model, precision, flags, device;
    double dt, eps;
    const void *fn, *fout, *L;
    int64_t n;
    bool operator==(const StepKey &o) const {
        return m == o.m && scheme == o.scheme && model == o.model && precision == o.precision && flags == o.flags &&
               device == o.device && dt == o.dt && eps == o.eps && fn == o.fn && fout == o.fout && L == o.L &&
               n == o.n;
    }
};
struct StepGraph {
    StepKey key;
    cudaGraphExec_t exec;
    void *scratch;
    uint64_t stamp;
};
constexpr size_t kMaxGraphs = 8;
std::mutex g_graph_mu;
std::vector<StepGraph> g_graphs;
uint64_t g_graph_clock = 0;

void drop_graph(StepGraph &e) {
    cudaGraphExecDestroy(e.exec);
    dev_free(e.scratch);
}

void purge_graphs(const bz_modes *m) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (size_t i = 0; i < g_graphs.size();) {
        if (g_graphs[i].key.m == m) {
            drop_graph(g_graphs[i]);
            g_graphs.erase(g_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

// The stage sequence of one step with all scratch at `scratch`.
int step_sequence(const bz_modes *m, const Tableau &t, int model, double dt, double eps, const void *f_n,
                  void *f_out, const void *L_res, int64_t n, int precision, int flags, cudaStream_t st,
                  void *scratch) {
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    const int64_t stride = n * m->g->v.nv;
    char *G = static_cast<char *>(scratch);
    char *P = G + (size_t)t.s * stride * es;
    char *Fbuf = P + (size_t)t.s * stride * es;
    char *coll = Fbuf + (size_t)stride * es;
    for (int l = 0; l < t.s; ++l) {
        void *F_l = (l == t.s - 1) ? f_out : static_cast<void *>(Fbuf);
        int rc = run_stage(m, t, l, model, dt, eps, f_n, F_l, G, P, L_res, n, precision, flags, st, coll, true);
        if (rc) return rc;
    }
    return BZ_OK;
}

// The stage sequence coupled to the transport step: after stage l the
// residual L_l = <L(F_l^w)>_x of the stage value enters the explicit part of
// every later stage (eq. GIMEX_n; the correction Delta Q vanishes for a
// reconstruction that keeps the cell averages).  Scratch: step scratch, then
// [stages][cell][nv] residuals, then the reconstruction's gradients.
int step_sequence_fv(const bz_modes *m, const bz_mesh *mesh, const Tableau &t, int model, double dt, double eps,
                     const void *f_n, void *f_out, int64_t n, int precision, int flags, cudaStream_t st,
                     void *scratch, size_t step_bytes) {
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    const int64_t stride = n * m->g->v.nv;
    char *G = static_cast<char *>(scratch);
    char *P = G + (size_t)t.s * stride * es;
    char *Fbuf = P + (size_t)t.s * stride * es;
    char *coll = Fbuf + (size_t)stride * es;
    char *Lbuf = static_cast<char *>(scratch) + step_bytes;
    char *tsc = Lbuf + (size_t)t.s * stride * es;
    for (int l = 0; l < t.s; ++l) {
        void *F_l = (l == t.s - 1) ? f_out : static_cast<void *>(Fbuf);
        int rc = run_stage(m, t, l, model, dt, eps, f_n, F_l, G, P, Lbuf, n, precision, flags, st, coll);
        if (rc) return rc;
        if (l < t.s - 1) {
            rc = transport_chain(mesh, m->g, precision, F_l, Lbuf + (size_t)l * stride * es, st, tsc);
            if (rc) return rc;
        }
    }
    return BZ_OK;
}

size_t step_scratch_bytes(const bz_modes *m, const Tableau &t, int64_t n, int precision) {
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    const size_t stage = (size_t)(2 * t.s + 1) * n * m->g->v.nv * es;
    return stage + collide_scratch_bytes(m, precision, n);
}

int check_imex_args(const bz_modes *m, int scheme, int model, double dt, double eps, int precision,
                    int64_t n, const char *who, Tableau &t) {
    int rc = check_modes(m, precision, who);
    if (rc) return rc;
    if (!tableau(scheme, t)) return fail(BZ_EINVAL, std::string(who) + ": unknown scheme");
    if (model != BZ_BOLTZMANN && model != BZ_BGK) return fail(BZ_EINVAL, std::string(who) + ": unknown model");
    if (!(dt > 0.0) || !(eps > 0.0)) return fail(BZ_EINVAL, std::string(who) + ": dt and eps must be > 0");
    if (n < 0) return fail(BZ_EINVAL, std::string(who) + ": n_cells < 0");
    return BZ_OK;
}

// ---- host-buffer entry point --------------------------------------------
// Copy streams per device (non-blocking, created on first use).
cudaStream_t g_copy_streams[kMaxDevices][2];
bool g_copy_ok[kMaxDevices];

int copy_streams(int dev, cudaStream_t out[2]) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_copy_ok[dev]) {
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = cudaStreamCreateWithFlags(&g_copy_streams[dev][i], cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "collide_batch_host: copy stream");
        }
        g_copy_ok[dev] = true;
    }
    out[0] = g_copy_streams[dev][0];
    out[1] = g_copy_streams[dev][1];
    return BZ_OK;
}

// Streams of group_collide's lanes per device (non-blocking, created on first use).
constexpr int kGroupStreams = 4;
cudaStream_t g_group_streams[kMaxDevices][kGroupStreams];
bool g_group_ok[kMaxDevices];

int group_streams(int dev, cudaStream_t out[kGroupStreams]) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_group_ok[dev]) {
        for (int i = 0; i < kGroupStreams; ++i) {
            cudaError_t e = cudaStreamCreateWithFlags(&g_group_streams[dev][i], cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "group_collide: stream");
        }
        g_group_ok[dev] = true;
    }
    for (int i = 0; i < kGroupStreams; ++i) out[i] = g_group_streams[dev][i];
    return BZ_OK;
}

// Compute streams of collide_batch_host per device (non-blocking, created on
// first use): forward and inverse transforms at the greatest priority, the
// mode sums of even and odd chunks at the least, so that a chunk's inverse
// transform takes the SMs the moment its mode sum ends, ahead of the CTAs of
// the next chunk's mode sum, which fill the SMs the previous one frees.
constexpr int kHostStreams = 4;    // forward, inverse, mode sum (even chunks), mode sum (odd chunks)
cudaStream_t g_host_streams[kMaxDevices][kHostStreams];
bool g_host_ok[kMaxDevices];

int host_streams(int dev, cudaStream_t out[kHostStreams]) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_host_ok[dev]) {
        int lo = 0, hi = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e != cudaSuccess) return cuda_fail(e, "collide_batch_host: stream priorities");
        for (int i = 0; i < kHostStreams; ++i) {
            e = cudaStreamCreateWithPriority(&g_host_streams[dev][i], cudaStreamNonBlocking, i < 2 ? hi : lo);
            if (e != cudaSuccess) return cuda_fail(e, "collide_batch_host: compute stream");
        }
        g_host_ok[dev] = true;
    }
    for (int i = 0; i < kHostStreams; ++i) out[i] = g_host_streams[dev][i];
    return BZ_OK;
}

// Cells per pipeline stage of collide_batch_host: one full wave of the
// handle's mode-sum kernel (every SM holding as many CTAs as fit), so that no
// chunk leaves SMs idle at its end.
int64_t host_chunk_cells(const bz_modes *m) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->g->device) != cudaSuccess || sms <= 0)
        sms = 128;
    // two waves where a short launch would run on the one-CTA sibling: the
    // overlapping chunks keep the faster several-CTA kernel busy
    return (int64_t)sms * modesum32_wave_cells_per_sm(m);
}

}  // namespace

// collide_chain on caller-provided Fourier scratch of collide_scratch_bytes()
// bytes (the allocation-free entry point, noalloc.cu): the same kernels and
// launches as collide_batch, no allocation.
size_t collide_scratch_size(const bz_modes *m, int precision, int64_t n) {
    return collide_scratch_bytes(m, precision, n);
}

int collide_on_scratch(const bz_modes *m, int precision, int flags, const void *f, void *Q, int64_t n,
                       void *scratch, cudaStream_t st) {
    if (!scratch) return fail(BZ_EINVAL, "collide: scratch is NULL");
    return collide_chain(m, precision, flags, f, Q, nullptr, n, st, scratch);
}

int *device_error_word() {
    int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_err_word[dev]) {
        int *p = nullptr;
        if (dev_malloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
            dev_free(p);
            return nullptr;
        }
        g_err_word[dev] = p;
    }
    return g_err_word[dev];
}

}  // namespace bz

using namespace bz;

extern "C" {

int init_velocity_grid(int dim, int n_per_dim, double half_width_L, bz_grid **out) {
    return grid_create(dim, n_per_dim, half_width_L, out);
}

int build_kernel_modes(const bz_grid *g, double gamma, double b0, int quad_nodes, bz_modes **out) {
    if (g) {
        DeviceGuard dg(g->device);
        return modes_create(g, gamma, b0, quad_nodes, out);
    }
    return modes_create(g, gamma, b0, quad_nodes, out);
}

int build_fast_modes(const bz_grid *g, double b0, int n_dirs, bz_modes **out) {
    return fast_modes_create(g, b0, n_dirs, out);
}

int collide_batch(const bz_modes *m, int precision, int flags, const void *f, void *Q, int64_t n_cells,
                  void *stream) {
    int rc = check_modes(m, precision, "collide_batch");
    if (rc) return rc;
    if (n_cells < 0) return fail(BZ_EINVAL, "collide_batch: n_cells < 0");
    if (n_cells == 0) return BZ_OK;
    if (!f || !Q) return fail(BZ_EINVAL, "collide_batch: f or Q is NULL");
    if (flags & ~(BZ_CONSERVE | BZ_CHECK_INPUT)) return fail(BZ_EINVAL, "collide_batch: unknown flag");
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    const size_t bytes = (size_t)n_cells * m->g->v.nv * es;
    const char *fb = static_cast<const char *>(f);
    const char *qb = static_cast<const char *>(Q);
    if (fb < qb + bytes && qb < fb + bytes) return fail(BZ_EINVAL, "collide_batch: f and Q overlap");
    DeviceGuard dg(m->g->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (flags & BZ_CHECK_INPUT) {
        rc = check_input(precision, f, n_cells * m->g->v.nv, st);
        if (rc) return rc;
    }
    return collide_chain(m, precision, flags, f, Q, nullptr, n_cells, st);
}

int collide_batch_host(const bz_modes *m, int precision, int flags, const void *f_host, void *Q_host,
                       int64_t n_cells, void *stream) {
    int rc = check_modes(m, precision, "collide_batch_host");
    if (rc) return rc;
    if (n_cells < 0) return fail(BZ_EINVAL, "collide_batch_host: n_cells < 0");
    if (n_cells == 0) return BZ_OK;
    if (!f_host || !Q_host) return fail(BZ_EINVAL, "collide_batch_host: f or Q is NULL");
    if (flags & ~(BZ_CONSERVE | BZ_CHECK_INPUT)) return fail(BZ_EINVAL, "collide_batch_host: unknown flag");
    DeviceGuard dg(m->g->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(BZ_EINVAL, "collide_batch_host: not available inside a stream capture");
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    const size_t cell_bytes = (size_t)m->g->v.nv * es;
    const int64_t chunk = std::min(n_cells, host_chunk_cells(m));
    // chunk boundaries: one mode-sum wave each, except that where a short
    // chunk runs in proportion to its size (the 32-cell kernels split a partial
    // wave's tiles over several CTAs; kernels with several CTAs per SM run a
    // short chunk on their one-CTA sibling; the fast form's wave holds four
    // CTAs per SM) a long batch starts and ends with chunks of 1/8, 1/4 and 1/2
    // of a wave, so that the copy that fills the pipeline and the one that
    // drains it are short
    std::vector<int64_t> bnd{0};
    {
        const bool ramped = m->method != 0 || (precision == BZ_FP32 && (modesum32_tail_splits(m) ||
                                                                           modesum32_small_batches_fast(m)));
        auto part = [&](int d) { return std::max<int64_t>(32, (chunk / d + 31) / 32 * 32); };
        const int64_t ramp = part(8) + part(4) + part(2);
        if (ramped && n_cells > 2 * ramp + chunk) {
            int64_t at = 0;
            for (int d : {8, 4, 2}) bnd.push_back(at += part(d));
            const int64_t mid_end = n_cells - ramp;
            while (mid_end - at > chunk) bnd.push_back(at += chunk);
            bnd.push_back(at = mid_end);
            for (int d : {2, 4}) bnd.push_back(at += part(d));
        } else {
            int64_t at = 0;
            while (n_cells - at > chunk) bnd.push_back(at += chunk);
        }
        if (bnd.back() != n_cells) bnd.push_back(n_cells);
    }
    const int64_t nchunks = (int64_t)bnd.size() - 1;
    cudaStream_t cp[2], hs[kHostStreams];
    if ((rc = copy_streams(m->g->device, cp))) return rc;
    if ((rc = host_streams(m->g->device, hs))) return rc;
    cudaStream_t s_in = cp[0], s_out = cp[1], s_fwd = hs[0], s_inv = hs[1], s_ms[2] = {hs[2], hs[3]};
    // two device slots, each an (f, Q) chunk pair and the chunk's Fourier
    // scratch, from the pool on the caller's stream
    const size_t sbytes = (collide_scratch_bytes(m, precision, chunk) + 255) / 256 * 256;
    const size_t fbytes = (chunk * cell_bytes + 255) / 256 * 256;
    Scratch buf;
    BZ_TRY(buf.alloc(2 * (2 * fbytes + sbytes), st), "collide_batch_host: chunk buffers");
    char *fd[2], *qd[2], *fh[2], *qh[2];
    for (int i = 0; i < 2; ++i) {
        char *b = static_cast<char *>(buf.p) + (size_t)i * (2 * fbytes + sbytes);
        fd[i] = b;
        qd[i] = b + fbytes;
        fh[i] = b + 2 * fbytes;
        qh[i] = fh[i] + spectrum_bytes(m, precision, chunk);
    }
    // events per slot: in (f copied), fw (forward transform done: f slot
    // free), ms (mode sum done: spectrum free), done (inverse done: Q ready,
    // Q-hat free), out (Q copied back: Q slot free); ready (buffers allocated)
    // and one end event per compute stream
    constexpr int kEv = 1 + 5 * 2 + kHostStreams;
    cudaEvent_t ev[kEv] = {};
    for (int i = 0; i < kEv; ++i) {
        cudaError_t e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int q = 0; q < i; ++q) cudaEventDestroy(ev[q]);
            return cuda_fail(e, "collide_batch_host: events");
        }
    }
    cudaEvent_t ready = ev[0], *in = ev + 1, *fw = ev + 3, *ms = ev + 5, *done = ev + 7, *out = ev + 9,
                *fin = ev + 11;
    auto run = [&]() -> int {
        BZ_TRY(cudaEventRecord(ready, st), "collide_batch_host: record");
        for (cudaStream_t x : {s_in, s_out, s_fwd, s_inv, s_ms[0], s_ms[1]})
            BZ_TRY(cudaStreamWaitEvent(x, ready, 0), "collide_batch_host: wait");
        for (int64_t c = 0; c < nchunks; ++c) {
            const int i = (int)(c & 1);
            const int64_t off = bnd[c], nc = bnd[c + 1] - bnd[c];
            const size_t bytes = (size_t)nc * cell_bytes;
            int r2;
            // host -> device once the slot's f has been transformed (chunk c - 2)
            if (c >= 2) BZ_TRY(cudaStreamWaitEvent(s_in, fw[i], 0), "collide_batch_host: wait");
            BZ_TRY(cudaMemcpyAsync(fd[i], static_cast<const char *>(f_host) + (size_t)off * cell_bytes, bytes,
                                   cudaMemcpyHostToDevice, s_in),
                   "collide_batch_host: host to device copy");
            BZ_TRY(cudaEventRecord(in[i], s_in), "collide_batch_host: record");
            // forward transform once the slot's spectrum is free (mode sum of c - 2)
            BZ_TRY(cudaStreamWaitEvent(s_fwd, in[i], 0), "collide_batch_host: wait");
            if (c >= 2) BZ_TRY(cudaStreamWaitEvent(s_fwd, ms[i], 0), "collide_batch_host: wait");
            if (flags & BZ_CHECK_INPUT) {
                if ((r2 = check_input(precision, fd[i], nc * m->g->v.nv, s_fwd))) return r2;
            }
            if ((r2 = phase_forward(m, precision, fd[i], fh[i], nc, s_fwd))) return r2;
            BZ_TRY(cudaEventRecord(fw[i], s_fwd), "collide_batch_host: record");
            // mode sum once Q-hat of c - 2 has been inverse-transformed
            BZ_TRY(cudaStreamWaitEvent(s_ms[i], fw[i], 0), "collide_batch_host: wait");
            if (c >= 2) BZ_TRY(cudaStreamWaitEvent(s_ms[i], done[i], 0), "collide_batch_host: wait");
            if ((r2 = phase_modesum(m, precision, fh[i], qh[i], nc, s_ms[i]))) return r2;
            BZ_TRY(cudaEventRecord(ms[i], s_ms[i]), "collide_batch_host: record");
            // inverse transform once Q of c - 2 has been copied back
            BZ_TRY(cudaStreamWaitEvent(s_inv, ms[i], 0), "collide_batch_host: wait");
            if (c >= 2) BZ_TRY(cudaStreamWaitEvent(s_inv, out[i], 0), "collide_batch_host: wait");
            if ((r2 = phase_inverse(m, precision, flags, qh[i], qd[i], nullptr, nc, s_inv))) return r2;
            BZ_TRY(cudaEventRecord(done[i], s_inv), "collide_batch_host: record");
            BZ_TRY(cudaStreamWaitEvent(s_out, done[i], 0), "collide_batch_host: wait");
            BZ_TRY(cudaMemcpyAsync(static_cast<char *>(Q_host) + (size_t)off * cell_bytes, qd[i], bytes,
                                   cudaMemcpyDeviceToHost, s_out),
                   "collide_batch_host: device to host copy");
            BZ_TRY(cudaEventRecord(out[i], s_out), "collide_batch_host: record");
        }
        return BZ_OK;
    };
    rc = run();
    // the caller's stream continues after every stream of the pipeline (also
    // after an error part-way), so that the slots return to the pool only when
    // nothing uses them
    {
        cudaStream_t all[kHostStreams + 2] = {s_fwd, s_inv, s_ms[0], s_ms[1], s_in, s_out};
        for (int k = 0; k < kHostStreams + 2; ++k) {
            cudaEvent_t e = k < kHostStreams ? fin[k] : (k == kHostStreams ? in[0] : out[0]);
            cudaError_t x = cudaEventRecord(e, all[k]);
            if (x == cudaSuccess) x = cudaStreamWaitEvent(st, e, 0);
            if (x != cudaSuccess && !rc) rc = cuda_fail(x, "collide_batch_host: join");
        }
    }
    for (int i = 0; i < kEv; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

int imex_stage_local(const bz_modes *m, int scheme, int stage, int model, double dt, double eps,
                     const void *f_n, void *F, void *G, void *P, const void *L_res, int64_t n_cells,
                     int precision, int flags, void *stream) {
    Tableau t;
    int rc = check_imex_args(m, scheme, model, dt, eps, precision, n_cells, "imex_stage_local", t);
    if (rc) return rc;
    if (stage < 1 || stage > t.s) return fail(BZ_EINVAL, "imex_stage_local: stage out of range");
    if (n_cells == 0) return BZ_OK;
    if (!f_n || !F || !G || !P) return fail(BZ_EINVAL, "imex_stage_local: NULL buffer");
    if (flags & ~(BZ_CONSERVE | BZ_CHECK_INPUT)) return fail(BZ_EINVAL, "imex_stage_local: unknown flag");
    DeviceGuard dg(m->g->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int l = stage - 1;
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    const int64_t stride = n_cells * m->g->v.nv;
    if ((flags & BZ_CHECK_INPUT) && l == 0) {
        rc = check_input(precision, f_n, stride, st);
        if (rc) return rc;
    }
    void *F_l = static_cast<char *>(F) + (size_t)l * stride * es;
    return run_stage(m, t, l, model, dt, eps, f_n, F_l, G, P, L_res, n_cells, precision, flags, st);
}

int imex_step(const bz_modes *m, int scheme, int model, double dt, double eps, const void *f_n, void *f_out,
              const void *L_res, int64_t n_cells, int precision, int flags, void *stream) {
    Tableau t;
    int rc = check_imex_args(m, scheme, model, dt, eps, precision, n_cells, "imex_step", t);
    if (rc) return rc;
    if (n_cells == 0) return BZ_OK;
    if (!f_n || !f_out) return fail(BZ_EINVAL, "imex_step: NULL buffer");
    if (f_n == f_out) return fail(BZ_EINVAL, "imex_step: f_n and f_out must differ");
    if (flags & ~(BZ_CONSERVE | BZ_CHECK_INPUT)) return fail(BZ_EINVAL, "imex_step: unknown flag");
    DeviceGuard dg(m->g->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t stride = n_cells * m->g->v.nv;
    if (flags & BZ_CHECK_INPUT) {
        rc = check_input(precision, f_n, stride, st);
        if (rc) return rc;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (st) cudaStreamIsCapturing(st, &cap);
    if (!st || cap != cudaStreamCaptureStatusNone) {
        // legacy stream or a caller's capture: plain launches, pool scratch
        Scratch s;
        BZ_TRY(s.alloc(step_scratch_bytes(m, t, n_cells, precision), st), "imex_step: scratch");
        return step_sequence(m, t, model, dt, eps, f_n, f_out, L_res, n_cells, precision, flags, st, s.p);
    }
    StepKey key{m, scheme, model, precision, flags, m->g->device, dt, eps, f_n, f_out, L_res, n_cells};
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto &e : g_graphs) {
        if (e.key == key) {
            e.stamp = ++g_graph_clock;
            BZ_TRY(cudaGraphLaunch(e.exec, st), "imex_step: graph launch");
            return BZ_OK;
        }
    }
    StepGraph ne;
    ne.key = key;
    ne.stamp = ++g_graph_clock;
    ne.scratch = nullptr;
    ne.exec = nullptr;
    cudaError_t e = dev_malloc(&ne.scratch, step_scratch_bytes(m, t, n_cells, precision));
    if (e != cudaSuccess) return cuda_fail(e, "imex_step: graph scratch");
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        dev_free(ne.scratch);
        return cuda_fail(e, "imex_step: begin capture");
    }
    t_capturing = true;
    rc = step_sequence(m, t, model, dt, eps, f_n, f_out, L_res, n_cells, precision, flags, st, ne.scratch);
    t_capturing = false;
    e = cudaStreamEndCapture(st, &graph);
    if (rc == BZ_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ne.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != BZ_OK || e != cudaSuccess) {
        dev_free(ne.scratch);
        return rc != BZ_OK ? rc : cuda_fail(e, "imex_step: capture");
    }
    if (g_graphs.size() >= kMaxGraphs) {
        size_t old = 0;
        for (size_t i = 1; i < g_graphs.size(); ++i)
            if (g_graphs[i].stamp < g_graphs[old].stamp) old = i;
        drop_graph(g_graphs[old]);
        g_graphs.erase(g_graphs.begin() + old);
    }
    g_graphs.push_back(ne);
    BZ_TRY(cudaGraphLaunch(ne.exec, st), "imex_step: graph launch");
    return BZ_OK;
}

int imex_step_fv(const bz_modes *m, const bz_mesh *mesh, int scheme, int model, double dt, double eps,
                 const void *f_n, void *f_out, int precision, int flags, void *stream) {
    Tableau t;
    if (!mesh) return fail(BZ_EINVAL, "imex_step_fv: mesh is NULL");
    int rc = check_imex_args(m, scheme, model, dt, eps, precision, mesh->n_cells, "imex_step_fv", t);
    if (rc) return rc;
    if (m->g->v.dim != 2) return fail(BZ_ENOTSUP, "imex_step_fv: the transport step needs a 2-D velocity grid");
    if (mesh->device != m->g->device) return fail(BZ_EINVAL, "imex_step_fv: mesh and modes on different devices");
    if (!f_n || !f_out) return fail(BZ_EINVAL, "imex_step_fv: NULL buffer");
    if (f_n == f_out) return fail(BZ_EINVAL, "imex_step_fv: f_n and f_out must differ");
    if (flags & ~(BZ_CONSERVE | BZ_CHECK_INPUT)) return fail(BZ_EINVAL, "imex_step_fv: unknown flag");
    DeviceGuard dg(m->g->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = mesh->n_cells;
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    if (flags & BZ_CHECK_INPUT) {
        rc = check_input(precision, f_n, n * m->g->v.nv, st);
        if (rc) return rc;
    }
    const size_t step_bytes = (step_scratch_bytes(m, t, n, precision) + 255) / 256 * 256;
    const size_t bytes = step_bytes + (size_t)t.s * n * m->g->v.nv * es + transport_scratch_bytes(mesh, m->g, precision);
    Scratch s;
    BZ_TRY(s.alloc(bytes, st), "imex_step_fv: scratch");
    return step_sequence_fv(m, mesh, t, model, dt, eps, f_n, f_out, n, precision, flags, st, s.p, step_bytes);
}

int build_fv_mesh(int n_vertices, const double *xy, int64_t n_cells, const int64_t *cell_ptr,
                  const int64_t *cell_vertices, int order, bz_mesh **out) {
    return fv_mesh_create(n_vertices, xy, n_cells, cell_ptr, cell_vertices, order, 0.0, 0.0, out);
}

int build_fv_mesh_periodic(int n_vertices, const double *xy, int64_t n_cells, const int64_t *cell_ptr,
                           const int64_t *cell_vertices, int order, double Lx, double Ly, bz_mesh **out) {
    return fv_mesh_create(n_vertices, xy, n_cells, cell_ptr, cell_vertices, order, Lx, Ly, out);
}

int transport_residual(const bz_mesh *mesh, const bz_grid *g, int precision, const void *f, void *L, void *stream) {
    if (!mesh || !g) return fail(BZ_EINVAL, "transport_residual: NULL mesh or grid");
    if (precision != BZ_FP64 && precision != BZ_FP32) return fail(BZ_EINVAL, "transport_residual: unknown precision");
    if (g->v.dim != 2) return fail(BZ_ENOTSUP, "transport_residual: the transport step needs a 2-D velocity grid");
    if (mesh->device != g->device) return fail(BZ_EINVAL, "transport_residual: mesh and grid on different devices");
    if (!f || !L) return fail(BZ_EINVAL, "transport_residual: f or L is NULL");
    const size_t bytes = (size_t)mesh->n_cells * g->v.nv * (precision == BZ_FP64 ? sizeof(double) : sizeof(float));
    const char *fb = static_cast<const char *>(f);
    const char *lb = static_cast<const char *>(L);
    if (fb < lb + bytes && lb < fb + bytes) return fail(BZ_EINVAL, "transport_residual: f and L overlap");
    DeviceGuard dg(g->device);
    return transport_chain(mesh, g, precision, f, L, static_cast<cudaStream_t>(stream));
}

int fv_mesh_set_walls(bz_mesh *mesh, int64_t n_edges, const int64_t *edge_vertices, const double *wall_params) {
    if (!mesh) return fail(BZ_EINVAL, "fv_mesh_set_walls: mesh is NULL");
    DeviceGuard dg(mesh->device);
    return bz::fv_mesh_set_walls(mesh, n_edges, edge_vertices, wall_params);
}

int bz_mesh_info(const bz_mesh *mesh, int64_t out[5]) {
    if (!mesh || !out) return fail(BZ_EINVAL, "bz_mesh_info: NULL argument");
    out[0] = mesh->n_cells;
    out[1] = mesh->n_faces_interior;
    out[2] = mesh->n_faces_boundary;
    out[3] = mesh->max_faces;
    out[4] = mesh->order;
    return BZ_OK;
}

void bz_mesh_destroy(bz_mesh *mesh) { fv_mesh_destroy(mesh); }

int group_collide(const bz_group_item *items, int n_items, int precision, int flags, void *stream) {
    if (!items || n_items < 0 || n_items > 1024) return fail(BZ_EINVAL, "group_collide: bad item list");
    if (precision != BZ_FP64 && precision != BZ_FP32 && precision != BZ_FP32X2)
        return fail(BZ_EINVAL, "group_collide: precision");
    if (flags & ~(BZ_CONSERVE | BZ_CHECK_INPUT)) return fail(BZ_EINVAL, "group_collide: unknown flag");
    if (n_items == 0) return BZ_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    for (int i = 0; i < n_items; ++i) {
        const bz_group_item &it = items[i];
        if (!it.modes || !it.modes->g) return fail(BZ_EINVAL, "group_collide: item without modes");
        if (it.n_cells < 0) return fail(BZ_EINVAL, "group_collide: n_cells < 0");
        if (it.n_cells > 0 && (!it.f || !it.Q)) return fail(BZ_EINVAL, "group_collide: NULL buffer");
        if (it.modes->g->device != dev) return fail(BZ_EINVAL, "group_collide: items must live on the current device");
        int rc0 = check_modes(it.modes, precision, "group_collide");
        if (rc0) return rc0;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // longest first: per-cell work (pairs of the symmetric sum) decides the order
    std::vector<int> order;
    for (int i = 0; i < n_items; ++i)
        if (items[i].n_cells > 0) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return items[a].modes->pairs_sym > items[b].modes->pairs_sym;
    });
    std::vector<size_t> off(order.size() + 1, 0);
    for (size_t q = 0; q < order.size(); ++q) {
        size_t b = collide_scratch_bytes(items[order[q]].modes, precision, items[order[q]].n_cells);
        off[q + 1] = off[q] + (b + 255) / 256 * 256;
    }
    Scratch s;
    BZ_TRY(s.alloc(off.back(), st), "group_collide: scratch");
    char *base = static_cast<char *>(s.p);
    auto fh_of = [&](size_t q) { return base + off[q]; };
    auto qh_of = [&](size_t q) {
        return base + off[q] + spectrum_bytes(items[order[q]].modes, precision, items[order[q]].n_cells);
    };
    int rc;
    if (flags & BZ_CHECK_INPUT) {
        for (size_t q = 0; q < order.size(); ++q) {
            const bz_group_item &it = items[order[q]];
            rc = check_input(precision, it.f, it.n_cells * it.modes->g->v.nv, st);
            if (rc) return rc;
        }
    }
    // Lanes: the FP32 instances on one register-blocked variant form one lane
    // (one grouped mode-sum launch for up to kMaxGroup of them); every other
    // instance is a lane of its own.  Each lane runs its forward transforms,
    // mode sum and inverse transforms in order on one of the library's group
    // streams, forked from the caller's stream and joined back to it, so that
    // the last partial wave of one lane's launches overlaps the others' work.
    struct Lane {
        std::vector<size_t> qs;
        double work = 0.0;
        bool grouped = false;
    };
    std::vector<Lane> lanes;
    std::vector<int> lane_of_var(kModesumVariants, -1);
    for (size_t q = 0; q < order.size(); ++q) {
        const bz_group_item &it = items[order[q]];
        const double w = (double)it.modes->pairs_sym * (double)it.n_cells;
        if (precision == BZ_FP32 && modesum32_available(it.modes)) {
            int &l = lane_of_var[it.modes->variant];
            if (l < 0) {
                l = (int)lanes.size();
                lanes.emplace_back();
                lanes.back().grouped = true;
            }
            lanes[l].qs.push_back(q);
            lanes[l].work += w;
        } else {
            lanes.emplace_back();
            lanes.back().qs.push_back(q);
            lanes.back().work = w;
        }
    }
    auto run_lane = [&](const Lane &ln, cudaStream_t ls) -> int {
        int r;
        for (size_t q : ln.qs) {
            const bz_group_item &it = items[order[q]];
            if ((r = phase_forward(it.modes, precision, it.f, fh_of(q), it.n_cells, ls))) return r;
        }
        if (ln.grouped) {
            for (size_t a = 0; a < ln.qs.size(); a += kMaxGroup) {
                std::vector<const bz_modes *> gm;
                std::vector<const float2 *> gf;
                std::vector<float2 *> gq;
                std::vector<int64_t> gn;
                for (size_t b = a; b < ln.qs.size() && b < a + kMaxGroup; ++b) {
                    const bz_group_item &it = items[order[ln.qs[b]]];
                    gm.push_back(it.modes);
                    gf.push_back(reinterpret_cast<const float2 *>(fh_of(ln.qs[b])));
                    gq.push_back(reinterpret_cast<float2 *>(qh_of(ln.qs[b])));
                    gn.push_back(it.n_cells);
                }
                BZ_LAUNCH("modesum_f32_group", ls,
                          launch_modesum32_group(gm.data(), gf.data(), gq.data(), gn.data(), (int)gm.size(), ls),
                          "group_collide: grouped mode sum");
            }
        } else {
            const bz_group_item &it = items[order[ln.qs[0]]];
            if ((r = phase_modesum(it.modes, precision, fh_of(ln.qs[0]), qh_of(ln.qs[0]), it.n_cells, ls))) return r;
        }
        for (size_t q : ln.qs) {
            const bz_group_item &it = items[order[q]];
            if ((r = phase_inverse(it.modes, precision, flags, qh_of(q), it.Q, nullptr, it.n_cells, ls))) return r;
        }
        return BZ_OK;
    };
    if (lanes.size() == 1) return run_lane(lanes[0], st);
    // longest lane first onto the least loaded stream
    cudaStream_t gs[kGroupStreams];
    if ((rc = group_streams(dev, gs))) return rc;
    std::vector<int> lorder(lanes.size());
    for (size_t i = 0; i < lanes.size(); ++i) lorder[i] = (int)i;
    std::stable_sort(lorder.begin(), lorder.end(), [&](int a, int b) { return lanes[a].work > lanes[b].work; });
    const int K = (int)std::min<size_t>(kGroupStreams, lanes.size());
    std::vector<double> load(K, 0.0);
    std::vector<int> lane_stream(lanes.size(), 0);
    for (int l : lorder) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[k] += lanes[l].work;
        lane_stream[l] = k;
    }
    cudaEvent_t ev[kGroupStreams + 1] = {};
    for (int k = 0; k <= K; ++k) {
        cudaError_t e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int q = 0; q < k; ++q) cudaEventDestroy(ev[q]);
            return cuda_fail(e, "group_collide: events");
        }
    }
    // fork: every stream starts after the caller's stream (scratch allocated,
    // inputs written); join: the caller's stream continues after all of them,
    // also after an error part-way (the scratch returns to the pool on it)
    rc = BZ_OK;
    cudaError_t e = cudaEventRecord(ev[K], st);
    for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(gs[k], ev[K], 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "group_collide: fork");
    for (int l : lorder) {
        if (rc) break;
        rc = run_lane(lanes[l], gs[lane_stream[l]]);
    }
    for (int k = 0; k < K; ++k) {
        e = cudaEventRecord(ev[k], gs[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[k], 0);
        if (e != cudaSuccess && !rc) rc = cuda_fail(e, "group_collide: join");
    }
    for (int k = 0; k <= K; ++k) cudaEventDestroy(ev[k]);
    return rc;
}

int bz_check(void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "bz_check: stream synchronize");
    int *w = device_error_word();
    if (!w) return fail(BZ_ENOMEM, "bz_check: device error word");
    int code = 0;
    e = cudaMemcpy(&code, w, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "bz_check: read error word");
    if (code) {
        e = cudaMemset(w, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "bz_check: clear error word");
    }
    if (code == kDevNonFinite) return fail(BZ_ENONFINITE, "non-finite input value seen by a kernel");
    if (code == kDevTimeout) return fail(BZ_ETIMEOUT, "a kernel wait gave up");
    if (code) return fail(BZ_ECUDA, "unknown device error code " + std::to_string(code));
    return BZ_OK;
}

const char *bz_last_error(void) { return t_err.c_str(); }

int bz_modes_info(const bz_modes *m, int64_t out[8]) {
    if (!m || !out) return fail(BZ_EINVAL, "bz_modes_info: NULL argument");
    const GridView &v = m->g->v;
    out[0] = v.dim;
    out[1] = v.N;
    out[2] = v.h;
    out[3] = v.nv;
    out[4] = v.nhalf;
    out[5] = m->nq;
    out[6] = m->pairs_sym;
    out[7] = modesum32_available(m) ? m->modesum_variant : 0;
    return BZ_OK;
}

int bz_fast_info(const bz_modes *m, int64_t out[4]) {
    if (!m || !out) return fail(BZ_EINVAL, "bz_fast_info: NULL argument");
    out[0] = m->method;
    out[1] = m->method == 1 ? m->ndirs : 0;
    out[2] = m->method == 1 ? fast_pad_length(m->g->v.N) : 0;
    out[3] = m->method == 1 ? fast_cells_per_cta(m->g->v.N) : 0;
    return BZ_OK;
}

int bz_modes_set_penalty(bz_modes *m, double c) {
    if (!m) return fail(BZ_EINVAL, "bz_modes_set_penalty: NULL modes");
    if (!(c > 0.0) || !std::isfinite(c)) return fail(BZ_EINVAL, "bz_modes_set_penalty: c must be finite and > 0");
    if (c != m->penalty) {
        purge_graphs(m);          // captured steps hold the old rate
        m->penalty = c;
    }
    return BZ_OK;
}

int bz_modes_beta(const bz_modes *m, double *out) {
    if (!m || !out) return fail(BZ_EINVAL, "bz_modes_beta: NULL argument");
    const GridView &v = m->g->v;
    int l[3], mm[3], kk[3];
    for (int64_t li = 0; li < v.nm; ++li) {
        int64_t t = li;
        for (int i = v.dim - 1; i >= 0; --i) { l[i] = (int)(t % v.M) - v.h; t /= v.M; }
        for (int64_t mi = 0; mi < v.nm; ++mi) {
            int64_t u = mi;
            bool ok = true;
            for (int i = v.dim - 1; i >= 0; --i) {
                mm[i] = (int)(u % v.M) - v.h;
                u /= v.M;
            }
            for (int i = 0; i < v.dim; ++i) {
                kk[i] = l[i] + mm[i];
                if (kk[i] < -v.h || kk[i] > v.h) ok = false;
            }
            out[li * v.nm + mi] = !ok ? 0.0 : m->method == 1 ? fast_beta_host(m, li, mi) : beta_host(m, l, mm);
        }
    }
    return BZ_OK;
}

int bz_profile(int enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof.clear();
    g_prof_on = enable != 0;
    return BZ_OK;
}

int bz_profile_read(char *names, int names_bytes, double *total_ms, int64_t *launches, int max_kernels) {
    if (!names || !total_ms || !launches || max_kernels <= 0 || names_bytes < 64 * max_kernels)
        return fail(BZ_EINVAL, "bz_profile_read: bad buffers");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<std::string> nm;
    std::vector<double> ms;
    std::vector<int64_t> cnt;
    int rc = BZ_OK;
    for (auto &r : g_prof) {
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_fail(e, "bz_profile_read");
        size_t i = 0;
        while (i < nm.size() && nm[i] != r.name) ++i;
        if (i == nm.size()) {
            nm.push_back(r.name);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[i] += t;
        cnt[i] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof.clear();
    if (rc) return rc;
    int n = (int)nm.size() < max_kernels ? (int)nm.size() : max_kernels;
    memset(names, 0, (size_t)names_bytes);
    for (int i = 0; i < n; ++i) {
        strncpy(names + 64 * i, nm[i].c_str(), 63);
        total_ms[i] = ms[i];
        launches[i] = cnt[i];
    }
    return n;
}

int bz_inject_alloc_failure(int64_t after) {
    g_fail_after.store(after < 0 ? -1 : after);
    return BZ_OK;
}

int bz_alloc_stats(int64_t *live_blocks, uint64_t *pool_used_bytes) {
    if (live_blocks) *live_blocks = g_live_blocks.load();
    if (!pool_used_bytes) return BZ_OK;
    uint64_t total = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int d = 0; d < kMaxDevices; ++d) {
        if (!g_pool_ok[d]) continue;
        uint64_t used = 0;
        cudaError_t e = cudaMemPoolGetAttribute(g_pool[d], cudaMemPoolAttrUsedMemCurrent, &used);
        if (e != cudaSuccess) return cuda_fail(e, "bz_alloc_stats: pool attribute");
        total += used;
    }
    *pool_used_bytes = total;
    return BZ_OK;
}

void bz_grid_destroy(bz_grid *g) { grid_destroy(g); }
void bz_modes_destroy(bz_modes *m) {
    if (!m) return;
    purge_graphs(m);
    modes_destroy(m);
}

}  // extern "C"
