// k_dft.cu -- separable forward / inverse DFT of each cell's distribution on
// the truncated mode set K_h (Sec. 3.3, eq. FU and eq. FC), generic in the
// dimension and the precision.  One CTA per cell, shared-memory staging.
//
// Forward:  f-hat_k = N^-d sum_j f_j prod_i E[k_i][j_i],   only k_1 >= 0
//           (the other half is the complex conjugate: f is real).
// Inverse:  Q_j = scale * Re sum_{k in K_h} Q-hat_k prod_i conj(E[k_i][j_i])
//               = scale * sum_{k_1 >= 0} c_{k_1} Re(...),  c_0 = 1, c_{k_1>0} = 2.
// E[k][j] = (-1)^k exp(-2 pi i k j / N) = exp(-i k u_j), u_j = -pi + 2 pi j/N.
#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int kThreads = 256;

// Shared memory needed by one forward / inverse CTA, in bytes.
template <typename T> size_t fwd_smem(const GridView &g) {
    using V = typename C2<T>::type;
    int N = g.N, M = g.M, H = g.h + 1;
    if (g.dim == 2) return sizeof(T) * N * N + sizeof(V) * (size_t)H * N;
    // 3-D: f (N^3) and two complex stage buffers (H N N and H M N)
    return sizeof(T) * (size_t)N * N * N + sizeof(V) * ((size_t)H * N * N + (size_t)H * M * N);
}

template <typename T> size_t inv_smem(const GridView &g) {
    using V = typename C2<T>::type;
    int N = g.N, M = g.M, H = g.h + 1;
    size_t q = sizeof(T) * (size_t)g.nv + 64 * sizeof(double) * 5;
    if (g.dim == 2) return q + sizeof(V) * ((size_t)H * M + (size_t)H * N);
    return q + sizeof(V) * ((size_t)H * M * M + (size_t)H * M * N + (size_t)H * N * N);
}

template <typename T, typename TI = T>
__global__ void __launch_bounds__(kThreads) dft_forward_kernel(GridView g, const typename C2<T>::type *__restrict__ E,
                                                               const TI *__restrict__ f,
                                                               typename C2<T>::type *__restrict__ fhat) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t cell = blockIdx.x;
    const int N = g.N, M = g.M, h = g.h, H = h + 1;
    const T invN = (T)1 / (T)N;
    T *fs = reinterpret_cast<T *>(smem_raw);
    const TI *fc = f + cell * g.nv;
    for (int64_t i = threadIdx.x; i < g.nv; i += blockDim.x) fs[i] = (T)fc[i];
    __syncthreads();
    if (g.dim == 2) {
        V *A = reinterpret_cast<V *>(fs + N * N);          // A[k1][j2], k1 = 0..h
        for (int idx = threadIdx.x; idx < H * N; idx += blockDim.x) {
            int k1 = idx / N, j2 = idx % N;
            const V *e = E + (size_t)(k1 + h) * N;
            V acc = cmk<V>(0, 0);
            for (int j1 = 0; j1 < N; ++j1) {
                T x = fs[j1 * N + j2];
                acc.x = fma(e[j1].x, x, acc.x);
                acc.y = fma(e[j1].y, x, acc.y);
            }
            A[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < H * M; idx += blockDim.x) {
            int k1 = idx / M, k2 = idx % M;                  // k2 index = k2 + h
            const V *e = E + (size_t)k2 * N;
            V acc = cmk<V>(0, 0);
            for (int j2 = 0; j2 < N; ++j2) cmac(acc, A[k1 * N + j2], e[j2]);
            acc.x *= invN * invN;
            acc.y *= invN * invN;
            fhat[tiled_index(cell, idx, g.nhalf)] = acc;
        }
    } else {
        V *A1 = reinterpret_cast<V *>(fs + N * N * N);     // A1[k1][j2][j3]
        V *A2 = A1 + (size_t)H * N * N;                     // A2[k1][k2][j3]
        for (int idx = threadIdx.x; idx < H * N * N; idx += blockDim.x) {
            int k1 = idx / (N * N), r = idx % (N * N);
            const V *e = E + (size_t)(k1 + h) * N;
            V acc = cmk<V>(0, 0);
            for (int j1 = 0; j1 < N; ++j1) {
                T x = fs[j1 * N * N + r];
                acc.x = fma(e[j1].x, x, acc.x);
                acc.y = fma(e[j1].y, x, acc.y);
            }
            A1[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < H * M * N; idx += blockDim.x) {
            int k1 = idx / (M * N), r = idx % (M * N), k2 = r / N, j3 = r % N;
            const V *e = E + (size_t)k2 * N;
            V acc = cmk<V>(0, 0);
            for (int j2 = 0; j2 < N; ++j2) cmac(acc, A1[(k1 * N + j2) * N + j3], e[j2]);
            A2[idx] = acc;
        }
        __syncthreads();
        const T s3 = invN * invN * invN;
        for (int idx = threadIdx.x; idx < H * M * M; idx += blockDim.x) {
            int k1 = idx / (M * M), r = idx % (M * M), k2 = r / M, k3 = r % M;
            const V *e = E + (size_t)k3 * N;
            V acc = cmk<V>(0, 0);
            for (int j3 = 0; j3 < N; ++j3) cmac(acc, A2[(k1 * M + k2) * N + j3], e[j3]);
            acc.x *= s3;
            acc.y *= s3;
            fhat[tiled_index(cell, idx, g.nhalf)] = acc;
        }
    }
}

// conj(e) * q  accumulated: acc += q * conj(e)
template <typename V> __device__ __forceinline__ void cmac_conj(V &acc, V q, V e) {
    acc.x = fma(q.x, e.x, acc.x);
    acc.x = fma(q.y, e.y, acc.x);
    acc.y = fma(q.y, e.x, acc.y);
    acc.y = fma(-q.x, e.y, acc.y);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) dft_inverse_kernel(GridView g, const typename C2<T>::type *__restrict__ E,
                                                               const typename C2<T>::type *__restrict__ Qhat,
                                                               T *__restrict__ Q, double scale,
                                                               Cinv cinv, int conserve,
                                                               const T *__restrict__ P) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t cell = blockIdx.x;
    const int N = g.N, M = g.M, h = g.h, H = h + 1;
    double *red = reinterpret_cast<double *>(smem_raw);             // 64 * 5 doubles
    T *qs = reinterpret_cast<T *>(red + 64 * 5);                    // Q on the grid
    V *qh = reinterpret_cast<V *>(qs + g.nv);                       // half spectrum
    for (int64_t i = threadIdx.x; i < g.nhalf; i += blockDim.x) qh[i] = Qhat[tiled_index(cell, i, g.nhalf)];
    __syncthreads();
    if (g.dim == 2) {
        V *B = qh + H * M;                                          // B[k1][j2]
        for (int idx = threadIdx.x; idx < H * N; idx += blockDim.x) {
            int k1 = idx / N, j2 = idx % N;
            V acc = cmk<V>(0, 0);
            for (int k2 = 0; k2 < M; ++k2) cmac_conj(acc, qh[k1 * M + k2], E[(size_t)k2 * N + j2]);
            B[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
            int j1 = idx / N, j2 = idx % N;
            T acc = 0;
            for (int k1 = 0; k1 < H; ++k1) {
                V b = B[k1 * N + j2], e = E[(size_t)(k1 + h) * N + j1];
                // Re(b * conj(e)) = b.x e.x + b.y e.y, weight 2 for k1 > 0
                T re = fma(b.x, e.x, b.y * e.y);
                acc = fma(k1 == 0 ? (T)1 : (T)2, re, acc);
            }
            qs[idx] = acc * (T)scale;
        }
    } else {
        V *B3 = qh + (size_t)H * M * M;                             // [k1][k2][j3]
        V *B2 = B3 + (size_t)H * M * N;                             // [k1][j2][j3]
        for (int idx = threadIdx.x; idx < H * M * N; idx += blockDim.x) {
            int k12 = idx / N, j3 = idx % N;
            V acc = cmk<V>(0, 0);
            for (int k3 = 0; k3 < M; ++k3) cmac_conj(acc, qh[k12 * M + k3], E[(size_t)k3 * N + j3]);
            B3[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < H * N * N; idx += blockDim.x) {
            int k1 = idx / (N * N), r = idx % (N * N), j2 = r / N, j3 = r % N;
            V acc = cmk<V>(0, 0);
            for (int k2 = 0; k2 < M; ++k2) cmac_conj(acc, B3[(k1 * M + k2) * N + j3], E[(size_t)k2 * N + j2]);
            B2[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < N * N * N; idx += blockDim.x) {
            int j1 = idx / (N * N), r = idx % (N * N);
            T acc = 0;
            for (int k1 = 0; k1 < H; ++k1) {
                V b = B2[k1 * N * N + r], e = E[(size_t)(k1 + h) * N + j1];
                T re = fma(b.x, e.x, b.y * e.y);
                acc = fma(k1 == 0 ? (T)1 : (T)2, re, acc);
            }
            qs[idx] = acc * (T)scale;
        }
    }
    __syncthreads();
    T *out = Q + cell * g.nv;
    const T *pc = P ? P + cell * g.nv : nullptr;
    if (conserve) {
        // Smallest L2 change making sum_j phi(v_j) Q_j = 0 for phi = (1, v, |v|^2):
        // Q <- Q - phi^T (C C^T)^{-1} (C Q), all in FP64.
        const int nc = g.dim + 2;
        double b[5] = {0, 0, 0, 0, 0};
        for (int64_t i = threadIdx.x; i < g.nv; i += blockDim.x) {
            double q = (double)qs[i], v2 = 0.0;
            b[0] += q;
            for (int d = 0; d < g.dim; ++d) {
                double vd = grid_velocity(i, d, g.dim, N, g.L, g.dv);
                b[1 + d] += vd * q;
                v2 += vd * vd;
            }
            b[g.dim + 1] += v2 * q;
        }
        block_sum<5>(b, red);
        double x[5];
        for (int a = 0; a < nc; ++a) {
            double s = 0.0;
            for (int c = 0; c < nc; ++c) s += cinv.v[a * nc + c] * b[c];
            x[a] = s;
        }
        for (int64_t i = threadIdx.x; i < g.nv; i += blockDim.x) {
            double v2 = 0.0, corr = x[0];
            for (int d = 0; d < g.dim; ++d) {
                double vd = grid_velocity(i, d, g.dim, N, g.L, g.dv);
                corr += x[1 + d] * vd;
                v2 += vd * vd;
            }
            corr += x[g.dim + 1] * v2;
            double q = (double)qs[i] - corr;
            out[i] = pc ? (T)(q - (double)pc[i]) : (T)q;
        }
    } else {
        for (int64_t i = threadIdx.x; i < g.nv; i += blockDim.x) out[i] = pc ? qs[i] - pc[i] : qs[i];
    }
}

template <typename T, typename TI = T>
cudaError_t forward(const GridView &g, const typename C2<T>::type *E, const TI *f,
                    typename C2<T>::type *fhat, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    size_t sm = fwd_smem<T>(g);
    cudaError_t e =
        cudaFuncSetAttribute(dft_forward_kernel<T, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dft_forward_kernel<T, TI><<<(unsigned)n, kThreads, sm, st>>>(g, E, f, fhat);
    return cudaGetLastError();
}

template <typename T>
cudaError_t inverse(const GridView &g, const typename C2<T>::type *E, const typename C2<T>::type *Qhat,
                    T *Q, int64_t n, double scale, const double *cinv, const InvEpilogue &ep,
                    cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    size_t sm = inv_smem<T>(g);
    cudaError_t e = cudaFuncSetAttribute(dft_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    Cinv ci;
    for (int i = 0; i < 25; ++i) ci.v[i] = cinv[i];
    dft_inverse_kernel<T><<<(unsigned)n, kThreads, sm, st>>>(g, E, Qhat, Q, scale, ci, ep.conserve,
                                                             static_cast<const T *>(ep.P));
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dft_forward_f64(const GridView &g, const double2 *E, const double *f, double2 *fhat,
                                   int64_t n, cudaStream_t st) {
    return forward<double>(g, E, f, fhat, n, st);
}
cudaError_t launch_dft_forward_f32(const GridView &g, const float2 *E, const float *f, float2 *fhat,
                                   int64_t n, cudaStream_t st) {
    return forward<float>(g, E, f, fhat, n, st);
}
cudaError_t launch_dft_forward_f64_f32in(const GridView &g, const double2 *E, const float *f, double2 *fhat,
                                         int64_t n, cudaStream_t st) {
    return forward<double, float>(g, E, f, fhat, n, st);
}
cudaError_t launch_dft_inverse_f64(const GridView &g, const double2 *E, const double2 *Qhat, double *Q,
                                   int64_t n, double scale, const double *cinv, const InvEpilogue &ep,
                                   cudaStream_t st) {
    return inverse<double>(g, E, Qhat, Q, n, scale, cinv, ep, st);
}
cudaError_t launch_dft_inverse_f32(const GridView &g, const float2 *E, const float2 *Qhat, float *Q,
                                   int64_t n, double scale, const double *cinv, const InvEpilogue &ep,
                                   cudaStream_t st) {
    return inverse<float>(g, E, Qhat, Q, n, scale, cinv, ep, st);
}

}  // namespace bz
