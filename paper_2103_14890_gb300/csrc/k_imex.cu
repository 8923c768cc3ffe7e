// k_imex.cu -- cell-local stage of the penalised IMEX Runge-Kutta scheme
// (Sec. 3.4, eq. Bref2 and the scheme after it) and small utility kernels.
//
// Stage l of one cell (one CTA per cell):
//   R_l = f^n + dt sum_{m<l} [ At_lm (G_m/eps - L_m) + A_lm P_m/eps ]
//   U_l = (rho, rho u, E) = discrete moments of R_l                (FP64)
//   M_l = rho (2 pi theta)^(-d/2) exp(-|v - u|^2 / (2 theta))     (parameters FP64)
//   F_l = (R_l + c M_l) / (1 + c),   c = dt A_ll rho / eps
//   P_l = rho (M_l - F_l)
// G_l = Q(F_l) - P_l is formed by the inverse-DFT epilogue of the collision
// chain that follows this kernel.
#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double dexp(double x) { return exp(x); }

template <typename T>
__global__ void __launch_bounds__(kThreads) imex_stage_kernel(GridView g, StageCoef c, const T *__restrict__ fn,
                                                              T *__restrict__ F, const T *__restrict__ G,
                                                              T *__restrict__ P, const T *__restrict__ Lres,
                                                              int64_t stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *red = reinterpret_cast<double *>(smem_raw);         // 32 * 5
    T *R = reinterpret_cast<T *>(red + 32 * 5);                  // nv
    const int64_t cell = blockIdx.x;
    const int64_t base = cell * g.nv;
    const T dt = (T)c.dt, ieps = (T)(1.0 / c.eps);
    double mom[5] = {0, 0, 0, 0, 0};
    for (int64_t i = threadIdx.x; i < g.nv; i += blockDim.x) {
        T r = fn[base + i];
        for (int m = 0; m < c.nprev; ++m) {
            const int64_t o = (int64_t)m * stride + base + i;
            T gm = G[o] * ieps;
            if (Lres) gm -= Lres[o];
            r = fma(dt * (T)c.at[m], gm, r);
            r = fma(dt * (T)c.a[m] * ieps, P[o], r);
        }
        R[i] = r;
        double rd = (double)r, v2 = 0.0;
        mom[0] += rd;
        for (int d = 0; d < g.dim; ++d) {
            double vd = grid_velocity(i, d, g.dim, g.N, g.L, g.dv);
            mom[1 + d] += vd * rd;
            v2 += vd * vd;
        }
        mom[g.dim + 1] += 0.5 * v2 * rd;
    }
    block_sum<5>(mom, red);
    double w = 1.0;
    for (int d = 0; d < g.dim; ++d) w *= g.dv;
    const double rho = w * mom[0];
    double u[3] = {0, 0, 0}, u2 = 0.0;
    for (int d = 0; d < g.dim; ++d) {
        u[d] = w * mom[1 + d] / rho;
        u2 += u[d] * u[d];
    }
    const double E = w * mom[g.dim + 1];
    const double theta = (2.0 * E / rho - u2) / g.dim;
    const double pref = rho * pow(2.0 * M_PI * theta, -0.5 * g.dim);
    const double inv2t = 0.5 / theta;
    const double cc = c.dt * c.all * rho / c.eps;
    const T cT = (T)cc, denom = (T)(1.0 / (1.0 + cc)), rhoT = (T)rho;
    T *Fo = F + base;
    T *Po = P + (int64_t)c.stage * stride + base;
    for (int64_t i = threadIdx.x; i < g.nv; i += blockDim.x) {
        double r2 = 0.0;
        for (int d = 0; d < g.dim; ++d) {
            double dv = grid_velocity(i, d, g.dim, g.N, g.L, g.dv) - u[d];
            r2 += dv * dv;
        }
        T Mx;
        if constexpr (sizeof(T) == 8)
            Mx = (T)(pref * dexp(-r2 * inv2t));
        else
            Mx = (T)pref * expf((float)(-r2 * inv2t));   // exponent in FP64, exp in the state precision
        T Fi = (R[i] + cT * Mx) * denom;
        Fo[i] = Fi;
        Po[i] = rhoT * (Mx - Fi);
    }
}

// Fast 2-D path (N <= 32): one warp per cell, lane = column j2, loop over
// rows j1.  Moments: per-lane sums along j1 in the state precision (FP32: with
// a TwoSum error term), combined across the warp in FP64.  The Maxwellian of
// a 2-D grid factorises, M(v1, v2) = pref e1(v1) e2(v2), so each lane evaluates
// two exponentials in FP64 (its row and its column factor) instead of one per
// grid point.
template <typename T>
__device__ __forceinline__ void acc2(T &s, T &e, T x) {
    if constexpr (sizeof(T) == 4) {
        T t = s + x, bb = t - s;
        e += (s - (t - bb)) + (x - bb);
        s = t;
    } else {
        s += x;
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(256) imex_stage2d_kernel(GridView g, StageCoef c, const T *__restrict__ fn,
                                                           T *__restrict__ F, const T *__restrict__ G,
                                                           T *__restrict__ P, const T *__restrict__ Lres,
                                                           int64_t stride, int64_t n) {
    const int lane = threadIdx.x & 31;
    const int64_t cell = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (cell >= n) return;
    constexpr int NV = N * N;
    const bool on = lane < N;
    const int64_t base = cell * NV + (on ? lane : 0);
    const T dt = (T)c.dt, ieps = (T)(1.0 / c.eps);
    T R[N];
#pragma unroll
    for (int j = 0; j < N; ++j) R[j] = on ? fn[base + j * N] : (T)0;
    for (int m = 0; m < c.nprev; ++m) {
        const T ca = dt * (T)c.at[m] * ieps, cb = dt * (T)c.a[m] * ieps, cl = dt * (T)c.at[m];
        const int64_t o = (int64_t)m * stride + base;
        if (on) {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                T r = fma(ca, G[o + j * N], R[j]);
                r = fma(cb, P[o + j * N], r);
                if (Lres) r = fma(-cl, Lres[o + j * N], r);
                R[j] = r;
            }
        }
    }
    // moments: sums along the column (j1), then across lanes in FP64
    T s0 = 0, e0 = 0, s1 = 0, e1 = 0, s3 = 0, e3 = 0;
    const T L = (T)g.L, dv = (T)g.dv;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const T v1 = fma((T)j, dv, -L);
        acc2(s0, e0, R[j]);
        acc2(s1, e1, v1 * R[j]);
        acc2(s3, e3, v1 * v1 * R[j]);
    }
    const double vv = on ? -g.L + lane * g.dv : 0.0;
    double S0 = (double)s0 + (double)e0, S1 = (double)s1 + (double)e1, S3 = (double)s3 + (double)e3;
    double mom[4] = {S0, S1, vv * S0, S3 + vv * vv * S0};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mom[k] += __shfl_xor_sync(0xffffffffu, mom[k], o);
    const double w = g.dv * g.dv;
    const double rho = w * mom[0];
    const double u1 = w * mom[1] / rho, u2 = w * mom[2] / rho;
    const double E = 0.5 * w * mom[3];
    const double theta = (2.0 * E / rho - (u1 * u1 + u2 * u2)) / 2.0;
    const double pref = rho / (2.0 * M_PI * theta);
    const double inv2t = 0.5 / theta;
    // separable Maxwellian: this lane's column factor and row factor j1 = lane;
    // exponents in FP64, the exponential in the state precision
    const double d2 = vv - u2, d1 = (-g.L + lane * g.dv) - u1;
    const T fcol = (T)pref * exp((T)(-d2 * d2 * inv2t));
    const T frow_l = exp((T)(-d1 * d1 * inv2t));
    const double cc = c.dt * c.all * rho / c.eps;
    const T cT = (T)cc, denom = (T)(1.0 / (1.0 + cc)), rhoT = (T)rho;
    T *Fo = F + base;
    T *Po = P + (int64_t)c.stage * stride + base;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const T frow = __shfl_sync(0xffffffffu, frow_l, j);
        const T Mx = fcol * frow;
        const T Fi = (R[j] + cT * Mx) * denom;
        if (on) {
            Fo[j * N] = Fi;
            Po[j * N] = rhoT * (Mx - Fi);
        }
    }
}

template <typename T>
__global__ void check_input_kernel(const T *__restrict__ f, int64_t count, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t step = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < count; i += step) bad |= !isfinite(f[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_device_error(err, kDevNonFinite);
}

template <typename T>
cudaError_t stage(const GridView &g, const StageCoef &c, const T *fn, T *F, const T *G, T *P,
                  const T *Lres, int64_t stride, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (g.dim == 2 && (g.N == 16 || g.N == 24 || g.N == 32)) {
        const unsigned blocks = (unsigned)((n + 7) / 8);
        if (g.N == 16) imex_stage2d_kernel<T, 16><<<blocks, 256, 0, st>>>(g, c, fn, F, G, P, Lres, stride, n);
        if (g.N == 24) imex_stage2d_kernel<T, 24><<<blocks, 256, 0, st>>>(g, c, fn, F, G, P, Lres, stride, n);
        if (g.N == 32) imex_stage2d_kernel<T, 32><<<blocks, 256, 0, st>>>(g, c, fn, F, G, P, Lres, stride, n);
        return cudaGetLastError();
    }
    size_t sm = sizeof(double) * 32 * 5 + sizeof(T) * (size_t)g.nv;
    cudaError_t e = cudaFuncSetAttribute(imex_stage_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    imex_stage_kernel<T><<<(unsigned)n, kThreads, sm, st>>>(g, c, fn, F, G, P, Lres, stride);
    return cudaGetLastError();
}

template <typename T> cudaError_t check(const T *f, int64_t count, int *err, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    check_input_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(f, count, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_imex_stage_f64(const GridView &g, const StageCoef &c, const double *fn, double *F,
                                  const double *G, double *P, const double *Lres, int64_t stride,
                                  int64_t n, cudaStream_t st) {
    return stage<double>(g, c, fn, F, G, P, Lres, stride, n, st);
}
cudaError_t launch_imex_stage_f32(const GridView &g, const StageCoef &c, const float *fn, float *F,
                                  const float *G, float *P, const float *Lres, int64_t stride,
                                  int64_t n, cudaStream_t st) {
    return stage<float>(g, c, fn, F, G, P, Lres, stride, n, st);
}
cudaError_t launch_check_input_f64(const double *f, int64_t count, int *err, cudaStream_t st) {
    return check<double>(f, count, err, st);
}
cudaError_t launch_check_input_f32(const float *f, int64_t count, int *err, cudaStream_t st) {
    return check<float>(f, count, err, st);
}
cudaError_t launch_fill_zero(void *p, int64_t bytes, cudaStream_t st) {
    if (bytes <= 0) return cudaSuccess;
    return cudaMemsetAsync(p, 0, (size_t)bytes, st);
}

}  // namespace bz
