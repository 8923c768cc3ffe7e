// k_modesum32.cu -- register-blocked FP32 mode sum for 2-D grids (filled in
// by the symmetric sliding-window kernel; until then the generic kernel runs).
#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

int modes_build_fp32_tables(bz_modes *m) {
    m->d_W32 = nullptr;
    m->w32_floats = 0;
    m->d_task = nullptr;
    m->ntask = 0;
    return BZ_OK;
}

bool modesum32_2d_available(const bz_modes *m) { return m->d_W32 != nullptr; }

cudaError_t launch_modesum32_2d(const bz_modes *, const float2 *, float2 *, int64_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace bz
