// k_dft32.cu -- tile-based FP32 forward / inverse DFT of the collision operator
// (Sec. 3.3, eq. FC and eq. FU sampled on the grid) for 2-D grids with N in
// {16, 24, 32, 48}, computed by FFTs held in registers.
//
// The 2-D transform is separable; each axis is an FFT of length N (or of
// length N/2 for the real axis, by packing even and odd samples into one
// complex sequence).  A CTA handles C cells of the tiled Fourier layout
// [tile][mode][cell]; the intermediate A (forward) / B (inverse) lives in
// shared memory as [k1][j2][cell] with the cell stride padded to C + 1.
// Thread mapping: the grid-space stage (f or Q columns) uses one thread per
// (cell, column j2), so rows of f / Q are coalesced across the columns; the
// spectral stage uses one thread per (cell, row k1), so a mode's C cells are
// one coalesced segment of the tiled layout.
#include <math.h>

#include "bz_device.cuh"
#include "bz_internal.h"
#include "fft_reg.cuh"

namespace bz {

namespace {

// Inverse-DFT epilogue of one cell held as one column j2 = lane per thread:
// optional conservation projection, optional G = Q - P, coalesced store.
template <typename T, int N>
__device__ __forceinline__ void inv32_epilogue(T (&q)[N], int64_t cell, int lane, const Cinv &cinv,
                                               int conserve, const T *__restrict__ P, T *__restrict__ Q,
                                               T L, T dv, int64_t n) {
    using S = T;
    constexpr int NV = N * N;
    if (conserve) {
        // velocities in the working precision (L and dv arrive as T): in FP64
        // the compiler hoisted their 32 conversions out of this branch into
        // the common path, where FP64 at 1/64 of the FP32 rate bound the kernel
        const S v2 = -L + (S)lane * dv;
        // moments of Q over the cell: FP32 partials along j1 with a TwoSum
        // error term, combined in FP64 across the lanes; then the projection
        // Q -= phi . (C C^T)^{-1} (C Q) with phi = (1, v1, v2, |v|^2)
        double mom[4];
        {
            S s0 = (S)0., e0 = (S)0., s1 = (S)0., e1 = (S)0., s3 = (S)0., e3 = (S)0.;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const S v1 = -L + (S)j * dv;
                const S t0 = lane < N ? q[j] : (S)0.;
                S s, bb;
                s = s0 + t0; bb = s - s0; e0 += (s0 - (s - bb)) + (t0 - bb); s0 = s;
                const S t1 = v1 * t0;
                s = s1 + t1; bb = s - s1; e1 += (s1 - (s - bb)) + (t1 - bb); s1 = s;
                const S t3 = v1 * v1 * t0;
                s = s3 + t3; bb = s - s3; e3 += (s3 - (s - bb)) + (t3 - bb); s3 = s;
            }
            const double S0 = (double)s0 + e0, S1 = (double)s1 + e1, S3 = (double)s3 + e3;
            const double vv = lane < N ? (double)(-L + lane * dv) : 0.0;
            mom[0] = S0;
            mom[1] = S1;
            mom[2] = vv * S0;
            mom[3] = S3 + vv * vv * S0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mom[k] += __shfl_xor_sync(0xffffffffu, mom[k], o);
        double x[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c) s += cinv.v[a * 4 + c] * mom[c];
            x[a] = s;
        }
        const S x0 = (S)x[0], x1 = (S)x[1], x2 = (S)x[2], x3 = (S)x[3];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const S v1 = -L + (S)j * dv;
            q[j] -= x0 + x1 * v1 + x2 * v2 + x3 * (v1 * v1 + v2 * v2);
        }
    }
    if (cell < n && lane < N) {
        S *out = Q + cell * NV + lane;
        const S *pc = P ? P + cell * NV + lane : nullptr;
#pragma unroll
        for (int j = 0; j < N; ++j) out[j * N] = pc ? q[j] - pc[j * N] : q[j];
    }
}

// ---------------------------------------------------------------------------
// Radix-2 FFT form (N = 16, 32).
//
// With omega = e^{2 pi i / N} and u_j = -pi + 2 pi j / N, e^{-i k u_j} =
// (-1)^k omega^{-k j}, so
//   f-hat[k1][k2] = N^-2 (-1)^(k1+k2) sum_j1 sum_j2 f[j1][j2] omega^-(k1 j1 + k2 j2)
//   Q[j1][j2]     = s^(d+gamma) Re sum_{k1 >= 0} c_k1 (-1)^k1 omega^(k1 j1)
//                   sum_k2 (-1)^k2 Q-hat[k1][k2] omega^(k2 j2).
// Forward: per column j2, a real length-N transform over j1 (packed into a
// complex length-N/2 FFT plus the even/odd untangling), k1 = 0..N/2-1 kept;
// per row k1, a complex length-N FFT over j2, k2 = -h..h kept.  Inverse:
// per row k1, a complex length-N inverse FFT over k2 (the Nyquist slot k2 =
// N/2 is zero); per column j2, a Hermitian-to-real inverse over k1 through a
// complex length-N/2 inverse FFT.  All loops are unrolled with compile-time
// indices, so the data stay in registers and the twiddles are constant-bank
// operands.

// One CTA handles C cells (C = 32: a whole 32-cell tile of the Fourier layout,
// or C = 16: half of one, so that two CTAs fit an SM and one's memory traffic
// overlaps the other's arithmetic) with 16 C threads.
template <typename T, int N, int C, typename TI = T>
__global__ void __launch_bounds__(C * 16)
fft_fwd32_kernel(const TI *__restrict__ f, typename C2<T>::type *__restrict__ fhat, int64_t n) {
    using V2 = typename C2<T>::type;
    using S = T;
    constexpr int H = N / 2, M = N - 1, NV = N * N, LH = ilog2(H), LN = ilog2(N);
    constexpr int NW = C / 2, P = C + 1;                // warps; cell pitch of the shared rows
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2 *As = reinterpret_cast<V2 *>(smem_raw);        // [H][N][P]
    const int64_t tile = blockIdx.x / (32 / C);
    const int sub = (int)(blockIdx.x % (32 / C)) * C;   // first cell of this CTA within the tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- stage 1: lane = column j2 of cells warp, warp + NW, ...; real FFT over j1 ----
    if (lane < N) {
#pragma unroll 1
        for (int c = warp; c < C; c += NW) {
            const int64_t g = tile * 32 + sub + c;
            const bool ok = g < n;
            const TI *fc = f + g * NV + lane;
            V2 z[H];
#pragma unroll
            for (int p = 0; p < H; ++p) {
                const S x0 = ok ? (S)__ldg(fc + (2 * p) * N) : (S)0.;
                const S x1 = ok ? (S)__ldg(fc + (2 * p + 1) * N) : (S)0.;
                z[bitrev(p, LH)] = cmk<V2>(x0, x1);   // packed even / odd samples
            }
            fft_dit<H, -1>(z);
            // untangle: X[k] = E[k] + omega^-k O[k], E = (Z_k + conj Z_-k)/2,
            // O = (Z_k - conj Z_-k)/(2i); scale (-1)^k / N
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const V2 zk = z[k], zc = z[(H - k) % H];
                const S ex = (S)0.5 * (zk.x + zc.x), ey = (S)0.5 * (zk.y - zc.y);
                const S ox = (S)0.5 * (zk.y + zc.y), oy = -(S)0.5 * (zk.x - zc.x);
                const V2 w = tw32<V2>(k * (32 / N));
                const S xr = ex + (w.x * ox - w.y * oy);
                const S xi = ey + (w.x * oy + w.y * ox);
                const S sc = (k & 1) ? -(S)1. / N : (S)1. / N;
                As[(k * N + lane) * P + c] = cmk<V2>(xr * sc, xi * sc);
            }
        }
    }
    __syncthreads();
    // ---- stage 2: thread = (cell, row k1); complex FFT over j2 ----
    const int cell = threadIdx.x % C;
    const int64_t gc = tile * 32 + sub + cell;
#pragma unroll 1
    for (int k1 = threadIdx.x / C; k1 < H; k1 += 16) {
        V2 a[N];
#pragma unroll
        for (int j = 0; j < N; ++j) a[bitrev(j, LN)] = As[(k1 * N + j) * P + cell];
        fft_dit<N, -1>(a);
        if (gc < n) {
            V2 *out = fhat + tile * (int64_t)(H * M) * 32 + (int64_t)k1 * M * 32 + sub + cell;
#pragma unroll
            for (int kk = 0; kk < M; ++kk) {
                const int k2 = kk - (H - 1);
                const S sc = (k2 & 1) ? -(S)1. / N : (S)1. / N;
                const V2 v = a[k2 & (N - 1)];
                out[kk * 32] = cmk<V2>(v.x * sc, v.y * sc);
            }
        }
    }
}

template <typename T, int N, int C>
__global__ void __launch_bounds__(C * 16)
fft_inv32_kernel(const typename C2<T>::type *__restrict__ Qhat, T *__restrict__ Q, T scale, Cinv cinv,
                 int conserve, const T *__restrict__ P_, T L, T dv, int64_t n) {
    using V2 = typename C2<T>::type;
    using S = T;
    constexpr int H = N / 2, M = N - 1, LH = ilog2(H), LN = ilog2(N);
    constexpr int NW = C / 2, P = C + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2 *Bs = reinterpret_cast<V2 *>(smem_raw);        // [H][N][P]
    const int64_t tile = blockIdx.x / (32 / C);
    const int sub = (int)(blockIdx.x % (32 / C)) * C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- stage 1: thread = (cell, row k1); inverse complex FFT over k2 ----
    {
        const int cell = threadIdx.x % C;
        const V2 *qt = Qhat + tile * (int64_t)(H * M) * 32 + sub + cell;
#pragma unroll 1
        for (int k1 = threadIdx.x / C; k1 < H; k1 += 16) {
            V2 a[N];
            a[bitrev(H, LN)] = cmk<V2>((S)0., (S)0.);   // Nyquist slot k2 = N/2
#pragma unroll
            for (int kk = 0; kk < M; ++kk) {
                const int k2 = kk - (H - 1);
                const V2 v = qt[(k1 * M + kk) * 32];
                a[bitrev(k2 & (N - 1), LN)] = (k2 & 1) ? cmk<V2>(-v.x, -v.y) : v;
            }
            fft_dit<N, +1>(a);
            const S sc = (k1 & 1) ? -scale : scale; // s^(d+gamma) (-1)^k1
#pragma unroll
            for (int j = 0; j < N; ++j) Bs[(k1 * N + j) * P + cell] = cmk<V2>(a[j].x * sc, a[j].y * sc);
        }
    }
    __syncthreads();
    // ---- stage 2: lane = column j2 of cells warp, warp + NW, ...; Hermitian-to-real over k1 ----
#pragma unroll 1
    for (int c = warp; c < C; c += NW) {
        S q[N];
        if (lane < N) {
            V2 x[H + 1];
#pragma unroll
            for (int k = 0; k < H; ++k) x[k] = Bs[(k * N + lane) * P + c];
            x[0].y = (S)0.;                                // real part of the k1 = 0 row
            x[H] = cmk<V2>((S)0., (S)0.);
            // Z[k] = E[k] + i O[k], E = X_k + conj X_{H-k}, O = (X_k - conj X_{H-k}) omega^k
            V2 z[H];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const V2 xk = x[k], xc = cmk<V2>(x[H - k].x, -x[H - k].y);
                S ex, ey, ox, oy;
                if (k == 0) {
                    ex = xk.x; ey = xk.y; ox = xk.x; oy = xk.y;
                } else {
                    ex = xk.x + xc.x;
                    ey = xk.y + xc.y;
                    const S dx = xk.x - xc.x, dy = xk.y - xc.y;
                    const V2 w = tw32<V2>(k * (32 / N));           // omega^k = conj(w)
                    ox = dx * w.x + dy * w.y;
                    oy = dy * w.x - dx * w.y;
                }
                z[bitrev(k, LH)] = cmk<V2>(ex - oy, ey + ox);
            }
            fft_dit<H, +1>(z);
#pragma unroll
            for (int p = 0; p < H; ++p) {
                q[2 * p] = z[p].x;
                q[2 * p + 1] = z[p].y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) q[j] = (S)0.;
        }
        inv32_epilogue<T, N>(q, tile * 32 + sub + c, lane, cinv, conserve, P_, Q, L, dv, n);
    }
}


// ---------------------------------------------------------------------------
// Mixed-radix form for N = 24 and 48 (N/2 and N are 3 * 2^p).  Same sums as
// above; a length-3Q transform is split by Cooley-Tukey into Q-point
// transforms of the three residue classes n = Q n1 + n2 (3-point DFTs over
// n1, twiddles omega_L^(n2 k1), then Q-point FFTs over n2; output index
// k1 + 3 k2).  A 48-column cell does not fit one warp, so the column stages
// use TPC = 32 or 64 threads per cell (one or two whole warps).

template <int N> constexpr int threads_per_cell() { return N <= 32 ? 32 : 64; }

template <typename T, int N, int C, typename TI = T>
__global__ void __launch_bounds__(C * threads_per_cell<N>())
fftg_fwd_kernel(const TI *__restrict__ f, typename C2<T>::type *__restrict__ fhat, int64_t n) {
    using V2 = typename C2<T>::type;
    using S = T;
    constexpr int H = N / 2, M = N - 1, NV = N * N, P = C + 1, NT = C * threads_per_cell<N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2 *As = reinterpret_cast<V2 *>(smem_raw);        // [H][N][P]
    const int64_t tile = blockIdx.x / (32 / C);
    const int sub = (int)(blockIdx.x % (32 / C)) * C;
    // ---- stage 1: thread = (cell, column j2); real transform over j1 ----
#pragma unroll 1
    for (int t = threadIdx.x; t < C * N; t += NT) {
        const int c = t / N, j2 = t % N;
        const int64_t g = tile * 32 + sub + c;
        const bool ok = g < n;
        const TI *fc = f + g * NV + j2;
        V2 z[H];
#pragma unroll
        for (int p = 0; p < H; ++p)
            z[p] = cmk<V2>(ok ? (S)__ldg(fc + (2 * p) * N) : (S)0., ok ? (S)__ldg(fc + (2 * p + 1) * N) : (S)0.);
        fft_nat<H, -1>(z);
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const V2 zk = z[k], zc = z[(H - k) % H];
            const S ex = (S)0.5 * (zk.x + zc.x), ey = (S)0.5 * (zk.y - zc.y);
            const S ox = (S)0.5 * (zk.y + zc.y), oy = -(S)0.5 * (zk.x - zc.x);
            const V2 w = tw<N, V2>(k);
            const S xr = ex + (w.x * ox - w.y * oy);
            const S xi = ey + (w.x * oy + w.y * ox);
            const S sc = (k & 1) ? -(S)1. / N : (S)1. / N;
            As[(k * N + j2) * P + c] = cmk<V2>(xr * sc, xi * sc);
        }
    }
    __syncthreads();
    // ---- stage 2: thread = (cell, row k1); complex transform over j2 ----
#pragma unroll 1
    for (int t = threadIdx.x; t < C * H; t += NT) {
        const int c = t % C, k1 = t / C;
        const int64_t g = tile * 32 + sub + c;
        V2 a[N];
#pragma unroll
        for (int j = 0; j < N; ++j) a[j] = As[(k1 * N + j) * P + c];
        fft_nat<N, -1>(a);
        if (g < n) {
            V2 *out = fhat + tile * (int64_t)(H * M) * 32 + (int64_t)k1 * M * 32 + sub + c;
#pragma unroll
            for (int kk = 0; kk < M; ++kk) {
                const int k2 = kk - (H - 1);
                const S sc = (k2 & 1) ? -(S)1. / N : (S)1. / N;
                const V2 v = a[(k2 + N) % N];
                out[kk * 32] = cmk<V2>(v.x * sc, v.y * sc);
            }
        }
    }
}

// Epilogue for one column j2 of one cell, TPC threads per cell (whole warps):
// conservation projection (moments reduced over the cell's warps in a fixed
// order), G = Q - P, store.  red: shared scratch of (T/32) * 4 doubles.
template <typename T, int N, int TPC>
__device__ __forceinline__ void invg_epilogue(T (&q)[N], int64_t cell, int j2, const Cinv &cinv,
                                              int conserve, const T *__restrict__ P,
                                              T *__restrict__ Q, T L, T dv, int64_t n,
                                              double *red) {
    using S = T;
    constexpr int NV = N * N;
    const bool col = j2 < N;
    if (conserve) {
        const S v2 = -L + (S)j2 * dv;          // working precision (FP64 is 1/64 of the FP32 rate)
        double mom[4];
        {
            S s0 = (S)0., e0 = (S)0., s1 = (S)0., e1 = (S)0., s3 = (S)0., e3 = (S)0.;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const S v1 = -L + (S)j * dv;
                const S t0 = col ? q[j] : (S)0.;
                S s, bb;
                s = s0 + t0; bb = s - s0; e0 += (s0 - (s - bb)) + (t0 - bb); s0 = s;
                const S t1 = v1 * t0;
                s = s1 + t1; bb = s - s1; e1 += (s1 - (s - bb)) + (t1 - bb); s1 = s;
                const S t3 = v1 * v1 * t0;
                s = s3 + t3; bb = s - s3; e3 += (s3 - (s - bb)) + (t3 - bb); s3 = s;
            }
            const double S0 = (double)s0 + e0, S1 = (double)s1 + e1, S3 = (double)s3 + e3;
            const double vv = col ? (double)(-L + j2 * dv) : 0.0;
            mom[0] = S0;
            mom[1] = S1;
            mom[2] = vv * S0;
            mom[3] = S3 + vv * vv * S0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mom[k] += __shfl_xor_sync(0xffffffffu, mom[k], o);
        if constexpr (TPC > 32) {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 4; ++k) red[warp * 4 + k] = mom[k];
            __syncthreads();
            const int w0 = warp - warp % (TPC / 32);   // first warp of this cell
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double s = 0.0;
#pragma unroll
                for (int w = 0; w < TPC / 32; ++w) s += red[(w0 + w) * 4 + k];
                mom[k] = s;
            }
            __syncthreads();
        }
        double x[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c) s += cinv.v[a * 4 + c] * mom[c];
            x[a] = s;
        }
        const S x0 = (S)x[0], x1 = (S)x[1], x2 = (S)x[2], x3 = (S)x[3];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const S v1 = -L + (S)j * dv;
            q[j] -= x0 + x1 * v1 + x2 * v2 + x3 * (v1 * v1 + v2 * v2);
        }
    }
    if (cell < n && col) {
        S *out = Q + cell * NV + j2;
        const S *pc = P ? P + cell * NV + j2 : nullptr;
#pragma unroll
        for (int j = 0; j < N; ++j) out[j * N] = pc ? q[j] - pc[j * N] : q[j];
    }
}

template <typename T, int N, int C>
__global__ void __launch_bounds__(C * threads_per_cell<N>())
fftg_inv_kernel(const typename C2<T>::type *__restrict__ Qhat, T *__restrict__ Q, T scale, Cinv cinv,
                int conserve, const T *__restrict__ P_, T L, T dv, int64_t n) {
    using V2 = typename C2<T>::type;
    using S = T;
    constexpr int H = N / 2, M = N - 1, P = C + 1, TPC = threads_per_cell<N>(), NT = C * TPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2 *Bs = reinterpret_cast<V2 *>(smem_raw);        // [H][N][P], then NT/32 * 4 doubles
    double *red = reinterpret_cast<double *>(Bs + (size_t)H * N * P);
    const int64_t tile = blockIdx.x / (32 / C);
    const int sub = (int)(blockIdx.x % (32 / C)) * C;
    // ---- stage 1: thread = (cell, row k1); inverse complex transform over k2 ----
#pragma unroll 1
    for (int t = threadIdx.x; t < C * H; t += NT) {
        const int c = t % C, k1 = t / C;
        const V2 *qt = Qhat + tile * (int64_t)(H * M) * 32 + sub + c;
        V2 a[N];
        a[H] = cmk<V2>((S)0., (S)0.);                   // Nyquist slot k2 = N/2
#pragma unroll
        for (int kk = 0; kk < M; ++kk) {
            const int k2 = kk - (H - 1);
            const V2 v = qt[(k1 * M + kk) * 32];
            a[(k2 + N) % N] = (k2 & 1) ? cmk<V2>(-v.x, -v.y) : v;
        }
        fft_nat<N, +1>(a);
        const S sc = (k1 & 1) ? -scale : scale;     // s^(d+gamma) (-1)^k1
#pragma unroll
        for (int j = 0; j < N; ++j) Bs[(k1 * N + j) * P + c] = cmk<V2>(a[j].x * sc, a[j].y * sc);
    }
    __syncthreads();
    // ---- stage 2: thread = (cell, column j2), TPC threads per cell ----
    const int c = threadIdx.x / TPC, j2 = threadIdx.x % TPC;
    S q[N];
    if (j2 < N) {
        V2 x[H + 1];
#pragma unroll
        for (int k = 0; k < H; ++k) x[k] = Bs[(k * N + j2) * P + c];
        x[0].y = (S)0.;                                    // real part of the k1 = 0 row
        x[H] = cmk<V2>((S)0., (S)0.);
        V2 z[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const V2 xk = x[k], xc = cmk<V2>(x[H - k].x, -x[H - k].y);
            S ex, ey, ox, oy;
            if (k == 0) {
                ex = xk.x; ey = xk.y; ox = xk.x; oy = xk.y;
            } else {
                ex = xk.x + xc.x;
                ey = xk.y + xc.y;
                const S dx = xk.x - xc.x, dy = xk.y - xc.y;
                const V2 w = tw<N, V2>(k);                   // omega^k = conj(w)
                ox = dx * w.x + dy * w.y;
                oy = dy * w.x - dx * w.y;
            }
            z[k] = cmk<V2>(ex - oy, ey + ox);
        }
        fft_nat<H, +1>(z);
#pragma unroll
        for (int p = 0; p < H; ++p) {
            q[2 * p] = z[p].x;
            q[2 * p + 1] = z[p].y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j) q[j] = (S)0.;
    }
    invg_epilogue<T, N, TPC>(q, tile * 32 + sub + c, j2, cinv, conserve, P_, Q, L, dv, n, red);
}

template <typename T, int N, int C> size_t fftg_smem() {
    return 2 * sizeof(T) * (size_t)(N / 2) * N * (C + 1) + sizeof(double) * 4 * (C * threads_per_cell<N>() / 32);
}
template <typename T, int N, int C> size_t fft_smem() { return 2 * sizeof(T) * (size_t)(N / 2) * N * (C + 1); }

// Cells per CTA: FP32 16 (8 for 48^2, whose columns take two warps per cell);
// FP64 half of that (twice the bytes per value).
template <typename T, int N> constexpr int fft_cells() {
    return (N == 48 ? 8 : 16) / (sizeof(T) == 8 ? 2 : 1);
}
// The inverse keeps 128 registers per thread; 8-cell CTAs let four share an SM.
template <typename T, int N> constexpr int ifft_cells() { return (N == 16 || N == 32) ? 8 : fft_cells<T, N>(); }

template <typename T, int N, typename TI = T>
cudaError_t fwd_tile(const TI *f, typename C2<T>::type *fhat, int64_t n, cudaStream_t st) {
    constexpr int C = fft_cells<T, N>();
    const unsigned grid = (unsigned)(((n + 31) / 32) * (32 / C));
    cudaError_t e;
    if constexpr (N == 16 || N == 32) {
        const size_t sm = fft_smem<T, N, C>();
        e = cudaFuncSetAttribute(fft_fwd32_kernel<T, N, C, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        fft_fwd32_kernel<T, N, C, TI><<<grid, C * 16, sm, st>>>(f, fhat, n);
    } else {
        const size_t sm = fftg_smem<T, N, C>();
        e = cudaFuncSetAttribute(fftg_fwd_kernel<T, N, C, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        fftg_fwd_kernel<T, N, C, TI><<<grid, C * threads_per_cell<N>(), sm, st>>>(f, fhat, n);
    }
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t inv_tile(const GridView &g, const typename C2<T>::type *Qhat, T *Q, int64_t n, double scale,
                     const Cinv &ci, const InvEpilogue &ep, cudaStream_t st) {
    constexpr int C = ifft_cells<T, N>();
    const unsigned grid = (unsigned)(((n + 31) / 32) * (32 / C));
    const T *P = static_cast<const T *>(ep.P);
    cudaError_t e;
    if constexpr (N == 16 || N == 32) {
        const size_t sm = fft_smem<T, N, C>();
        e = cudaFuncSetAttribute(fft_inv32_kernel<T, N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        fft_inv32_kernel<T, N, C><<<grid, C * 16, sm, st>>>(Qhat, Q, (T)scale, ci, ep.conserve, P, (T)g.L, (T)g.dv,
                                                             n);
    } else {
        const size_t sm = fftg_smem<T, N, C>();
        e = cudaFuncSetAttribute(fftg_inv_kernel<T, N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        fftg_inv_kernel<T, N, C><<<grid, C * threads_per_cell<N>(), sm, st>>>(Qhat, Q, (T)scale, ci, ep.conserve,
                                                                             P, (T)g.L, (T)g.dv, n);
    }
    return cudaGetLastError();
}

template <typename T, typename TI = T>
cudaError_t fwd_any(const GridView &g, const TI *f, typename C2<T>::type *fhat, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    switch (g.N) {
        case 16: return fwd_tile<T, 16, TI>(f, fhat, n, st);
        case 24: return fwd_tile<T, 24, TI>(f, fhat, n, st);
        case 32: return fwd_tile<T, 32, TI>(f, fhat, n, st);
        case 48: return fwd_tile<T, 48, TI>(f, fhat, n, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t inv_any(const GridView &g, const typename C2<T>::type *Qhat, T *Q, int64_t n, double scale,
                    const double *cinv, const InvEpilogue &ep, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    Cinv ci;
    for (int i = 0; i < 25; ++i) ci.v[i] = cinv[i];
    switch (g.N) {
        case 16: return inv_tile<T, 16>(g, Qhat, Q, n, scale, ci, ep, st);
        case 24: return inv_tile<T, 24>(g, Qhat, Q, n, scale, ci, ep, st);
        case 32: return inv_tile<T, 32>(g, Qhat, Q, n, scale, ci, ep, st);
        case 48: return inv_tile<T, 48>(g, Qhat, Q, n, scale, ci, ep, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool dft32_tile_supported(const GridView &g) {
    return g.dim == 2 && (g.N == 16 || g.N == 24 || g.N == 32 || g.N == 48);
}

// Twiddles of the FFT kernels on the current device (constant memory is per
// device, so this runs for every modes handle, on its device).
int dft32_setup() {
    cudaError_t e = upload_fft_twiddles();
    if (e != cudaSuccess) return cuda_fail(e, "build_kernel_modes: FFT twiddles");
    return BZ_OK;
}

cudaError_t launch_dft32_forward_tile(const GridView &g, const float *f, float2 *fhat, int64_t n, cudaStream_t st) {
    return fwd_any<float>(g, f, fhat, n, st);
}
cudaError_t launch_dft64_forward_tile(const GridView &g, const double *f, double2 *fhat, int64_t n,
                                      cudaStream_t st) {
    return fwd_any<double>(g, f, fhat, n, st);
}
cudaError_t launch_dft64_forward_tile_f32in(const GridView &g, const float *f, double2 *fhat, int64_t n,
                                            cudaStream_t st) {
    return fwd_any<double, float>(g, f, fhat, n, st);
}
cudaError_t launch_dft32_inverse_tile(const GridView &g, const float2 *Qhat, float *Q, int64_t n, double scale,
                                      const double *cinv, const InvEpilogue &ep, cudaStream_t st) {
    return inv_any<float>(g, Qhat, Q, n, scale, cinv, ep, st);
}
cudaError_t launch_dft64_inverse_tile(const GridView &g, const double2 *Qhat, double *Q, int64_t n, double scale,
                                      const double *cinv, const InvEpilogue &ep, cudaStream_t st) {
    return inv_any<double>(g, Qhat, Q, n, scale, cinv, ep, st);
}

}  // namespace bz
