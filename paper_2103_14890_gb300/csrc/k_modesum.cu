// k_modesum.cu -- generic direct mode sum of eq. CF1 (Sec. 3.3) on the half
// spectrum, any dimension, FP64 or FP32:
//   Q-hat_k = sum over l in K_h with m = k - l in K_h of beta-hat(l,m) f-hat_l f-hat_m,
// for k with k_1 >= 0 (Q is real, so Q-hat_{-k} = conj(Q-hat_k)).  The weights
// come from the radial table: beta-hat(l,m) = F(|k|^2, |2l-k|^2) - F(0, |2m|^2).
// One warp per (32-cell tile, k); lane = cell, so every load of a Fourier
// coefficient is a coalesced 32-cell row of the tiled layout and every weight
// load is warp-uniform.  This is the reference-precision kernel (FP64 pipe
// bound); the FP32 2-D path has its own register-blocked kernel.
#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int kWarps = 8;

template <typename V>
__device__ __forceinline__ V load_coef(const V *tile, int M, int h, int dim, const int *l) {
    // modes with l_1 < 0 are the conjugates of the stored -l
    bool neg = l[0] < 0;
    int64_t idx = 0;
    for (int i = 0; i < dim; ++i) idx = idx * M + ((neg ? -l[i] : l[i]) + h);
    // drop the offset of the k_1 < 0 rows: stored rows start at k_1 = 0
    idx -= (int64_t)h * (dim == 2 ? M : M * M);
    V v = tile[idx * 32];
    if (neg) v.y = -v.y;
    return v;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kWarps * 32) modesum_generic_kernel(GridView g, const T *__restrict__ F, int bcols,
                                                                      const typename C2<T>::type *__restrict__ fhat,
                                                                      typename C2<T>::type *__restrict__ Qhat,
                                                                      int64_t n) {
    using V = typename C2<T>::type;
    const int lane = threadIdx.x & 31;
    const int64_t kk = (int64_t)blockIdx.y * kWarps + (threadIdx.x >> 5);
    if (kk >= g.nhalf) return;
    const int64_t tile = blockIdx.x;
    const int h = g.h, M = g.M;
    int k[3];
    {
        int64_t t = kk;
        for (int i = DIM - 1; i >= 1; --i) { k[i] = (int)(t % M) - h; t /= M; }
        k[0] = (int)t;                                   // k_1 in [0, h]
    }
    const V *tp = fhat + tile * g.nhalf * 32 + lane;
    int a2 = 0;
    for (int i = 0; i < DIM; ++i) a2 += k[i] * k[i];
    const T *Fa = F + (int64_t)a2 * bcols;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int i = 0; i < DIM; ++i) {
        lo[i] = max(-h, k[i] - h);
        hi[i] = min(h, k[i] + h);
    }
    V acc = cmk<V>(0, 0);
    int l[3] = {0, 0, 0}, m[3] = {0, 0, 0};
    auto term = [&]() {
        int b2 = 0, c2 = 0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            m[i] = k[i] - l[i];
            int dlm = l[i] - m[i];
            b2 += dlm * dlm;
            c2 += 4 * m[i] * m[i];
        }
        T beta = Fa[b2] - F[c2];
        V fl = load_coef(tp, M, h, DIM, l);
        V fm = load_coef(tp, M, h, DIM, m);
        V p;                                   // fl * fm
        p.x = fma(fl.x, fm.x, -fl.y * fm.y);
        p.y = fma(fl.x, fm.y, fl.y * fm.x);
        acc.x = fma(beta, p.x, acc.x);
        acc.y = fma(beta, p.y, acc.y);
    };
    for (l[0] = lo[0]; l[0] <= hi[0]; ++l[0]) {
        for (l[1] = lo[1]; l[1] <= hi[1]; ++l[1]) {
            if constexpr (DIM == 2) {
                term();
            } else {
                for (l[2] = lo[2]; l[2] <= hi[2]; ++l[2]) term();
            }
        }
    }
    if (tile * 32 + lane < n) Qhat[tile * g.nhalf * 32 + kk * 32 + lane] = acc;
}

template <typename T>
cudaError_t launch(const GridView &g, const T *F, int bcols, const typename C2<T>::type *fhat,
                   typename C2<T>::type *Qhat, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((g.nhalf + kWarps - 1) / kWarps));
    if (g.dim == 2)
        modesum_generic_kernel<T, 2><<<grid, kWarps * 32, 0, st>>>(g, F, bcols, fhat, Qhat, n);
    else
        modesum_generic_kernel<T, 3><<<grid, kWarps * 32, 0, st>>>(g, F, bcols, fhat, Qhat, n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_modesum_generic_f64(const GridView &g, const double *F, int bcols, const double2 *fhat,
                                       double2 *Qhat, int64_t n, cudaStream_t st) {
    return launch<double>(g, F, bcols, fhat, Qhat, n, st);
}
cudaError_t launch_modesum_generic_f32(const GridView &g, const float *F, int bcols, const float2 *fhat,
                                       float2 *Qhat, int64_t n, cudaStream_t st) {
    return launch<float>(g, F, bcols, fhat, Qhat, n, st);
}

}  // namespace bz
