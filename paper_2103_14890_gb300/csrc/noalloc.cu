// noalloc.cu -- collide_batch_noalloc: the collision operator without any
// device allocation, for callers that cannot allocate device memory.
//
// Some callers of this library must not allocate device memory while they
// run: an application whose device memory is owned by another allocator (a
// framework's caching allocator or a host program that reserved the whole
// device up front) so that a cudaMalloc or a pool allocation by the library
// would fail or fragment that budget, and real-time loops that cannot take an
// allocation's latency or an allocation failure part-way through a run.  This
// entry point launches exactly the kernels of collide_batch (the same
// dispatch, api.cu), but the Fourier scratch (the forward spectra and the mode
// sums of the cells) lives in one statically sized device array defined in
// this file, so the call itself requests no memory.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoallocScratchBytes) until the process exits.  In host
// code its name is only a host-side stand-in for the device variable, not a
// device address: passed to a kernel it would fault, or, where the GPU can
// reach host memory, silently use the wrong memory.  The device address is
// therefore looked up with cudaGetSymbolAddress, once per device, on that
// device's first call, with the device current.
#include <mutex>
#include <string>

#include "bz_internal.h"

namespace bz {

// 32 MiB: 4224 cells of a 32x32 grid in FP32 (2112 in FP64), 1856 of a 48x48
// grid in FP32.
constexpr size_t kNoallocScratchBytes = 32u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDev = 64;
std::mutex g_na_mu;
void *g_na_ptr[kMaxDev];

// Device address of the static scratch on the current device; the first call
// per device looks it up (set-up), later calls read the cached address.
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
    if (collide_scratch_size(m, precision, n_cells) > kNoallocScratchBytes) {
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
    return collide_on_scratch(m, precision, flags, f, Q, n_cells, scratch, static_cast<cudaStream_t>(stream));
}
