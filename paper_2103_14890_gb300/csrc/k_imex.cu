// k_imex.cu -- cell-local stage of the penalised IMEX Runge-Kutta scheme
// (Sec. 3.4, eq. Bref2 and the scheme after it) and small utility kernels.
//
// Stage l of one cell (one CTA per cell):
//   R_l = f^n + dt sum_{m<l} [ At_lm (G_m/eps - L_m) + A_lm P_m/eps ]
//   U_l = (rho, rho u, E) = discrete moments of R_l                (FP64)
//   M_l = rho (2 pi theta)^(-d/2) exp(-|v - u|^2 / (2 theta))     (parameters FP64)
//   F_l = (R_l + c M_l) / (1 + c),   c = dt A_ll nu / eps
//   P_l = nu (M_l - F_l),   nu = nuf rho (nuf = 1 for BGK, the modes' penalty
//   factor for the Boltzmann model)
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
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            if (m >= c.nprev) break;
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
    const double nu = c.nuf * rho;
    const double cc = c.dt * c.all * nu / c.eps;
    const T cT = (T)cc, denom = (T)(1.0 / (1.0 + cc)), nuT = (T)nu;
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
        if (c.store_F) Fo[i] = Fi;
        Po[i] = nuT * (Mx - Fi);
    }
}

// Fast 2-D path (N <= 32): one warp per cell, lane = column j2, loop over
// rows j1, 8 cells per CTA.  FP64 work is what limits this kernel on a GPU
// whose FP64 rate is 1/74 of FP32, so it is arranged to keep the FP64 pipe's
// lanes busy with distinct work:
//   * per lane, sums along j1 in the state precision (FP32: with a TwoSum
//     error term), turned into FP64 once (S0, S1, S3 and the v2 products);
//   * the 32 lane partials of each cell are summed in FP64 by four threads per
//     (cell, moment) from shared memory, not by a shuffle tree on every lane;
//   * the Maxwellian parameters (rho, u, theta, ...) of the CTA's 8 cells are
//     computed by 8 lanes of one warp, one cell per lane;
//   * the Maxwellian of a 2-D grid factorises, M(v1, v2) = pref e1(v1) e2(v2):
//     each lane forms its row and column offsets v - u in FP64 and the rest of
//     the exponent and the exponential in the state precision.
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

constexpr int kStageCells = 8;    // cells (warps) per CTA of the 2-D stage kernel (two CTAs per SM)

template <typename T, int N>
__global__ void __launch_bounds__(kStageCells * 32) imex_stage2d_kernel(GridView g, StageCoef c,
                                                                       const T *__restrict__ fn, T *__restrict__ F,
                                                                       const T *__restrict__ G, T *__restrict__ P,
                                                                       const T *__restrict__ Lres, int64_t stride,
                                                                       int64_t n) {
    __shared__ double part[kStageCells][4][33];   // per-lane moment partials (pitch 33: no bank conflicts)
    __shared__ double par[kStageCells][8];        // nu, u1, u2, inv2t, pref, c, 1/(1+c)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t cell = (int64_t)blockIdx.x * kStageCells + wib;
    const bool live = cell < n;
    constexpr int NV = N * N;
    const bool on = lane < N && live;
    const int64_t base = (live ? cell : 0) * NV + (lane < N ? lane : 0);
    const T dt = (T)c.dt, ieps = (T)(1.0 / c.eps);
    T R[N];
#pragma unroll
    for (int j = 0; j < N; ++j) R[j] = on ? fn[base + j * N] : (T)0;
#pragma unroll
    for (int m = 0; m < 5; ++m) {              // compile-time index into the coefficient arrays
        if (m >= c.nprev) break;
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
    // this lane's partial moments (column j2 = lane)
    {
        T s0 = 0, e0 = 0, s1 = 0, e1 = 0, s3 = 0, e3 = 0;
        const T L = (T)g.L, dv = (T)g.dv;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T v1 = fma((T)j, dv, -L);
            acc2(s0, e0, R[j]);
            acc2(s1, e1, v1 * R[j]);
            acc2(s3, e3, v1 * v1 * R[j]);
        }
        const double vv = -g.L + lane * g.dv;
        const double S0 = (double)s0 + (double)e0, S1 = (double)s1 + (double)e1, S3 = (double)s3 + (double)e3;
        part[wib][0][lane] = S0;
        part[wib][1][lane] = S1;
        part[wib][2][lane] = vv * S0;
        part[wib][3][lane] = S3 + vv * vv * S0;
    }
    __syncthreads();
    // sums over the 32 lanes of each cell: four threads per (cell, moment) sum
    // eight partials each, then combine by shuffles (a fixed order)
    if (threadIdx.x < kStageCells * 16) {
        const int cc = threadIdx.x >> 4, q = (threadIdx.x >> 2) & 3, pp = threadIdx.x & 3;
        double tot = 0.0;
#pragma unroll
        for (int l = 0; l < 8; ++l) tot += part[cc][q][pp * 8 + l];
        tot += __shfl_xor_sync(0xffffffffu, tot, 1);
        tot += __shfl_xor_sync(0xffffffffu, tot, 2);
        if (pp == 0) part[cc][q][32] = tot;
    }
    __syncthreads();
    // Maxwellian parameters, one cell per lane of warp 0
    if (threadIdx.x < kStageCells) {
        const int cc = threadIdx.x;
        const double w = g.dv * g.dv;
        const double rho = w * part[cc][0][32];
        const double u1 = w * part[cc][1][32] / rho, u2 = w * part[cc][2][32] / rho;
        const double E = 0.5 * w * part[cc][3][32];
        const double theta = (2.0 * E / rho - (u1 * u1 + u2 * u2)) / 2.0;
        const double cst = c.dt * c.all * c.nuf * rho / c.eps;
        par[cc][0] = c.nuf * rho;          // penalty rate nu
        par[cc][1] = u1;
        par[cc][2] = u2;
        par[cc][3] = 0.5 / theta;
        par[cc][4] = rho / (2.0 * M_PI * theta);
        par[cc][5] = cst;
        par[cc][6] = 1.0 / (1.0 + cst);
    }
    __syncthreads();
    if (!live) return;
    // separable Maxwellian: this lane's column factor and row factor j1 = lane;
    // offsets v - u in FP64, the rest of the exponent and the exp in T
    const double vl = -g.L + lane * g.dv;
    const T d2 = (T)(vl - par[wib][2]), d1 = (T)(vl - par[wib][1]);
    const T i2t = (T)par[wib][3];
    const T fcol = (T)par[wib][4] * exp(-d2 * d2 * i2t);
    const T frow_l = exp(-d1 * d1 * i2t);
    const T cT = (T)par[wib][5], denom = (T)par[wib][6], nuT = (T)par[wib][0];
    T *Fo = F + base;
    T *Po = P + (int64_t)c.stage * stride + base;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const T frow = __shfl_sync(0xffffffffu, frow_l, j);
        const T Mx = fcol * frow;
        const T Fi = (R[j] + cT * Mx) * denom;
        if (on) {
            if (c.store_F) Fo[j * N] = Fi;
            Po[j * N] = nuT * (Mx - Fi);
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
        const unsigned blocks = (unsigned)((n + kStageCells - 1) / kStageCells);
        const unsigned thr = kStageCells * 32;
        if (g.N == 16) imex_stage2d_kernel<T, 16><<<blocks, thr, 0, st>>>(g, c, fn, F, G, P, Lres, stride, n);
        if (g.N == 24) imex_stage2d_kernel<T, 24><<<blocks, thr, 0, st>>>(g, c, fn, F, G, P, Lres, stride, n);
        if (g.N == 32) imex_stage2d_kernel<T, 32><<<blocks, thr, 0, st>>>(g, c, fn, F, G, P, Lres, stride, n);
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
