// noalloc.cu -- collide_batch_noalloc: the collision operator without any
// device allocation, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or use a memory pool: code that runs
// while a CUDA graph is being captured into a graph that may not contain
// allocation nodes, host code with a fixed memory budget that has handed every
// byte to its own allocator, or real-time loops that must not risk an
// allocation failure or its latency mid-run.  This entry point runs the same
// kernels as collide_batch, but its Fourier scratch (the forward spectra and the
// mode sums of the cells) lives in one statically sized device array defined in
// this file, so the call itself requests no memory.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoallocScratchBytes) until the process exits.  Host code
// cannot use its name as a device address; the address is looked up once per
// device with cudaGetSymbolAddress on that device's first call.
#include <mutex>
#include <string>

#include "bz_internal.h"

namespace bz {

// 32 MiB: 4224 cells of a 32x32 grid in FP32 (2112 in FP64).
constexpr size_t kNoallocScratchBytes = 32u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDev = 64;
std::mutex g_na_mu;
void *g_na_ptr[kMaxDev];

// Device address of the static scratch on the current device (set-up on the
// first call per device).
int noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "collide_batch_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDev) return fail(BZ_EINVAL, "collide_batch_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "collide_batch_noalloc: cudaGetSymbolAddress");
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return BZ_OK;
}
}  // namespace

cudaError_t launch_modesum32(const bz_modes *m, const float2 *fhat, float2 *Qhat, int64_t n,
                                cudaStream_t st);
bool modesum32_available(const bz_modes *m);

namespace {
// The kernel sequence of collide_batch (forward DFT, mode sum, inverse DFT)
// with the Fourier scratch at `scratch`.
int run_with_scratch(const bz_modes *m, int precision, int flags, const void *f, void *Q, int64_t n,
                     void *scratch, cudaStream_t st) {
    const bz_grid *g = m->g;
    const GridView &v = g->v;
    const int64_t ntile = (n + kTile - 1) / kTile;
    const size_t celem = (size_t)ntile * v.nhalf * kTile;
    InvEpilogue ep;
    ep.conserve = (flags & BZ_CONSERVE) ? 1 : 0;
    ep.check = 0;
    ep.P = nullptr;
    cudaError_t e;
    if (precision == BZ_FP64) {
        double2 *fh = static_cast<double2 *>(scratch), *qh = fh + celem;
        e = m->tile_dft ? launch_dft64_forward_tile(v, static_cast<const double *>(f), fh, n, st)
                        : launch_dft_forward_f64(v, g->d_E64, static_cast<const double *>(f), fh, n, st);
        if (e == cudaSuccess)
            e = m->method == 1          ? launch_fast_f64(m, fh, qh, n, st)
                : modesum64_available(m) ? launch_modesum64(m, fh, qh, n, st)
                                         : launch_modesum_generic_f64(v, m->d_F64, m->bcols, fh, qh, n, st);
        if (e == cudaSuccess)
            e = m->tile_dft ? launch_dft64_inverse_tile(v, qh, static_cast<double *>(Q), n, m->scale, g->cinv, ep, st)
                            : launch_dft_inverse_f64(v, g->d_E64, qh, static_cast<double *>(Q), n, m->scale, g->cinv,
                                                     ep, st);
    } else {
        float2 *fh = static_cast<float2 *>(scratch), *qh = fh + celem;
        const float *fin = static_cast<const float *>(f);
        float *qout = static_cast<float *>(Q);
        e = m->tile_dft ? launch_dft32_forward_tile(v, fin, fh, n, st)
                    : launch_dft_forward_f32(v, g->d_E32, fin, fh, n, st);
        if (e == cudaSuccess)
            e = m->method == 1          ? launch_fast_f32(m, fh, qh, n, st)
                : modesum32_available(m) ? launch_modesum32(m, fh, qh, n, st)
                                         : launch_modesum_generic_f32(v, m->d_F32, m->bcols, fh, qh, n, st);
        if (e == cudaSuccess)
            e = m->tile_dft ? launch_dft32_inverse_tile(v, qh, qout, n, m->scale, g->cinv, ep, st)
                        : launch_dft_inverse_f32(v, g->d_E32, qh, qout, n, m->scale, g->cinv, ep, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "collide_batch_noalloc: kernel launch");
    return BZ_OK;
}
}  // namespace

}  // namespace bz

using namespace bz;

extern "C" int collide_batch_noalloc(const bz_modes *m, int precision, int flags, const void *f, void *Q,
                                     int64_t n_cells, void *stream) {
    if (!m || !m->g) return fail(BZ_EINVAL, "collide_batch_noalloc: modes handle is NULL");
    if (precision != BZ_FP64 && precision != BZ_FP32)
        return fail(BZ_EINVAL, "collide_batch_noalloc: precision must be BZ_FP64 or BZ_FP32");
    if (flags & ~BZ_CONSERVE)
        return fail(BZ_EINVAL, "collide_batch_noalloc: only BZ_CONSERVE is accepted");
    if (n_cells < 0) return fail(BZ_EINVAL, "collide_batch_noalloc: n_cells < 0");
    if (n_cells == 0) return BZ_OK;
    if (!f || !Q) return fail(BZ_EINVAL, "collide_batch_noalloc: f or Q is NULL");
    const GridView &v = m->g->v;
    const size_t cplx = (precision == BZ_FP64) ? 16 : 8;
    const int64_t ntile = (n_cells + kTile - 1) / kTile;
    const size_t need = 2 * (size_t)ntile * v.nhalf * kTile * cplx;
    if (need > kNoallocScratchBytes) {
        const int64_t max_cells = (int64_t)(kNoallocScratchBytes / (2 * (size_t)v.nhalf * kTile * cplx)) * kTile;
        return fail(BZ_EINVAL, "collide_batch_noalloc: n_cells = " + std::to_string(n_cells) +
                                   " exceeds the static scratch (" + std::to_string(max_cells) +
                                   " cells at most for this grid and precision)");
    }
    const size_t es = (precision == BZ_FP64) ? sizeof(double) : sizeof(float);
    const size_t bytes = (size_t)n_cells * v.nv * es;
    const char *fb = static_cast<const char *>(f);
    const char *qb = static_cast<const char *>(Q);
    if (fb < qb + bytes && qb < fb + bytes) return fail(BZ_EINVAL, "collide_batch_noalloc: f and Q overlap");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->g->device)
        return fail(BZ_EINVAL, "collide_batch_noalloc: the modes handle belongs to another device; make it current");
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    return run_with_scratch(m, precision, flags, f, Q, n_cells, scratch, static_cast<cudaStream_t>(stream));
}
