// k_dft32.cu -- tile-based FP32 forward / inverse DFT for 2-D grids with
// N in {16, 24, 32} (Sec. 3.3, eq. FC and eq. FU sampled on the grid).
//
// N = 16 and 32 use register-resident radix-2 FFTs (fft_fwd32_kernel,
// fft_inv32_kernel, below); N = 24 uses the dense matrix form
// (dft_fwd32_kernel, dft_inv32_kernel).  Both compute the same sums; the FFT
// needs about a fifth of the instructions.
//
// One CTA handles one tile of 32 cells (the unit of the tiled Fourier layout
// [tile][mode][cell]).  The 2-D transform is separable:
//   forward  A[k1][j2]  = sum_j1 E1[j1][k1] f[j1][j2]           (k1 = 0..h)
//            fhat[k1][k2] = sum_j2 A[k1][j2] E2[j2][k2]          (k2 = -h..h)
//   inverse  B[k1][j2]  = sum_k2 Qhat[k1][k2] conj(E2[j2][k2])
//            Q[j1][j2]  = sum_k1 c_k1 Re(B[k1][j2] conj(E1[j1][k1]))
// with E(k, j) = (-1)^k exp(-2 pi i k j/N) / N (forward; the 1/N of each axis
// folded in) and c_0 = s^(d+gamma), c_{k1>0} = 2 s^(d+gamma) for the inverse
// (Hermitian half spectrum, physical scale folded in).
//
// Thread mapping: the grid-space stages use warp = cell pair, lane = j2 (rows
// of f / Q are coalesced 128-byte lines); the spectral stages use lane = cell
// (rows of the tiled layout are coalesced 256-byte lines) and warp = (pair of
// k1 rows, block of 16 k2 or j2).  Twiddles are read as warp-uniform float4
// (two complex values).  The intermediate A / B lives in shared memory as
// [k1][j2][cell] with the cell stride padded to 33 to spread banks.
#include <math.h>

#include <utility>
#include <vector>

#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int kThreads = 512;
constexpr int kPitch = 33;          // cells per (k1, j2) row of A / B in shared memory

// Twiddle tables (built on the host per grid, in global memory):
//   T1[j][k1]  : (-1)^k1 e^{-2 pi i k1 j/N}/N for k1 = 0..H-1       (forward stage 1)
//   T2[j][kk]  : E(kk - h, j)/N for kk = 0..M-1, rows padded to 32   (forward stage 2 / inverse stage 1)
//   T3[k1][j]  : c_k1 E(k1, j) (no 1/N), j = 0..N-1                   (inverse stage 2)

template <int N>
__global__ void __launch_bounds__(kThreads, 1)
dft_fwd32_kernel(const float *__restrict__ f, float2 *__restrict__ fhat, const float2 *__restrict__ T1,
                 const float2 *__restrict__ T2, int64_t n) {
    constexpr int H = N / 2, M = N - 1, NV = N * N;
    extern __shared__ __align__(16) float2 As[];        // [H][N][kPitch], then T1s, T2s
    float2 *T1s = As + H * N * kPitch;                  // [N][H]
    float2 *T2s = T1s + N * H;                          // [N][32]
    for (int i = threadIdx.x; i < N * H; i += blockDim.x) T1s[i] = T1[i];
    for (int i = threadIdx.x; i < N * 32; i += blockDim.x) T2s[i] = T2[i];
    const int64_t tile = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    // ---- stage 1: grid-space rows -> A ----
    {
        const int c0 = warp, c1 = warp + 16;
        const int64_t g0 = tile * 32 + c0, g1 = tile * 32 + c1;
        const bool ok0 = g0 < n && lane < N, ok1 = g1 < n && lane < N;
        const float *f0 = f + g0 * NV + lane, *f1 = f + g1 * NV + lane;
        float2 a0[H], a1[H];
#pragma unroll
        for (int k = 0; k < H; ++k) a0[k] = a1[k] = make_float2(0.f, 0.f);
        constexpr int JB = 8;                           // rows of f in flight per thread and cell
        for (int jb = 0; jb < N; jb += JB) {
            float xs0[JB], xs1[JB];
#pragma unroll
            for (int q = 0; q < JB; ++q) {
                xs0[q] = ok0 ? __ldg(f0 + (jb + q) * N) : 0.f;
                xs1[q] = ok1 ? __ldg(f1 + (jb + q) * N) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < JB; ++q) {
            const int j1 = jb + q;
            const float x0 = xs0[q], x1 = xs1[q];
            const float4 *t = reinterpret_cast<const float4 *>(T1s + j1 * H);
#pragma unroll
            for (int k = 0; k < H; k += 2) {
                const float4 e = t[k / 2];
                a0[k].x = fmaf(e.x, x0, a0[k].x);
                a0[k].y = fmaf(e.y, x0, a0[k].y);
                a0[k + 1].x = fmaf(e.z, x0, a0[k + 1].x);
                a0[k + 1].y = fmaf(e.w, x0, a0[k + 1].y);
                a1[k].x = fmaf(e.x, x1, a1[k].x);
                a1[k].y = fmaf(e.y, x1, a1[k].y);
                a1[k + 1].x = fmaf(e.z, x1, a1[k + 1].x);
                a1[k + 1].y = fmaf(e.w, x1, a1[k + 1].y);
            }
            }
        }
        if (lane < N) {
#pragma unroll
            for (int k = 0; k < H; ++k) {
                As[(k * N + lane) * kPitch + c0] = a0[k];
                As[(k * N + lane) * kPitch + c1] = a1[k];
            }
        }
    }
    __syncthreads();
    // ---- stage 2: lane = cell, tasks = (k1 pair, block of 16 k2) ----
    constexpr int NP = (H + 1) / 2, NB = (M + 15) / 16;
    const int64_t gc = tile * 32 + lane;
    for (int task = warp; task < NP * NB; task += 16) {
        const int p = task % NP, blk = task / NP;
        const int k1a = 2 * p, k1b = 2 * p + 1;
        const bool hasb = k1b < H;
        float2 q0[16], q1[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) q0[i] = q1[i] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int j2 = 0; j2 < N; ++j2) {
            const float2 a = As[(k1a * N + j2) * kPitch + lane];
            const float2 b = hasb ? As[(k1b * N + j2) * kPitch + lane] : make_float2(0.f, 0.f);
            const float4 *t = reinterpret_cast<const float4 *>(T2s + j2 * 32 + blk * 16);
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const float4 e = t[i / 2];
                cmac(q0[i], a, make_float2(e.x, e.y));
                cmac(q0[i + 1], a, make_float2(e.z, e.w));
                cmac(q1[i], b, make_float2(e.x, e.y));
                cmac(q1[i + 1], b, make_float2(e.z, e.w));
            }
        }
        if (gc < n) {
            float2 *out = fhat + tile * (int64_t)(H * M) * 32 + lane;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int kk = blk * 16 + i;
                if (kk < M) {
                    out[(k1a * M + kk) * 32] = q0[i];
                    if (hasb) out[(k1b * M + kk) * 32] = q1[i];
                }
            }
        }
    }
}

// acc += q * conj(e)
__device__ __forceinline__ void cmac_conj32(float2 &acc, float2 q, float ex, float ey) {
    acc.x = fmaf(q.x, ex, acc.x);
    acc.x = fmaf(q.y, ey, acc.x);
    acc.y = fmaf(q.y, ex, acc.y);
    acc.y = fmaf(-q.x, ey, acc.y);
}

// Inverse-DFT epilogue of one cell held as one column j2 = lane per thread:
// optional conservation projection, optional G = Q - P, coalesced store.
template <int N>
__device__ __forceinline__ void inv32_epilogue(float (&q)[N], int64_t cell, int lane, const Cinv &cinv,
                                               int conserve, const float *__restrict__ P, float *__restrict__ Q,
                                               double L, double dv, int64_t n) {
    constexpr int NV = N * N;
    const float v2 = (float)(-L + lane * dv);          // velocity of column j2
    if (conserve) {
        // moments of Q over the cell: FP32 partials along j1 with a TwoSum
        // error term, combined in FP64 across the lanes; then the projection
        // Q -= phi . (C C^T)^{-1} (C Q) with phi = (1, v1, v2, |v|^2)
        double mom[4];
        {
            float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f, s3 = 0.f, e3 = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const float v1 = (float)(-L + j * dv);
                const float t0 = lane < N ? q[j] : 0.f;
                float s, bb;
                s = s0 + t0; bb = s - s0; e0 += (s0 - (s - bb)) + (t0 - bb); s0 = s;
                const float t1 = v1 * t0;
                s = s1 + t1; bb = s - s1; e1 += (s1 - (s - bb)) + (t1 - bb); s1 = s;
                const float t3 = v1 * v1 * t0;
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
        const float x0 = (float)x[0], x1 = (float)x[1], x2 = (float)x[2], x3 = (float)x[3];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const float v1 = (float)(-L + j * dv);
            q[j] -= x0 + x1 * v1 + x2 * v2 + x3 * (v1 * v1 + v2 * v2);
        }
    }
    if (cell < n && lane < N) {
        float *out = Q + cell * NV + lane;
        const float *pc = P ? P + cell * NV + lane : nullptr;
#pragma unroll
        for (int j = 0; j < N; ++j) out[j * N] = pc ? q[j] - pc[j * N] : q[j];
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 1)
dft_inv32_kernel(const float2 *__restrict__ Qhat, float *__restrict__ Q, const float2 *__restrict__ T2i,
                 const float2 *__restrict__ T3, Cinv cinv, int conserve, const float *__restrict__ P,
                 double L, double dv, int64_t n) {
    constexpr int H = N / 2, M = N - 1;
    extern __shared__ __align__(16) float2 Bs[];        // [H][N][kPitch], then T2s, T3s
    float2 *T2s = Bs + H * N * kPitch;                  // [M][32]
    float2 *T3s = T2s + M * 32;                         // [H][N]
    for (int i = threadIdx.x; i < M * 32; i += blockDim.x) T2s[i] = T2i[i];
    for (int i = threadIdx.x; i < H * N; i += blockDim.x) T3s[i] = T3[i];
    __syncthreads();
    const int64_t tile = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- stage 1: lane = cell, tasks = (k1 pair, block of 16 j2) ----
    constexpr int NP = (H + 1) / 2, NB = (N + 15) / 16;
    const float2 *qt = Qhat + tile * (int64_t)(H * M) * 32 + lane;
    for (int task = warp; task < NP * NB; task += 16) {
        const int p = task % NP, blk = task / NP;
        const int k1a = 2 * p, k1b = 2 * p + 1;
        const bool hasb = k1b < H;
        float2 b0[16], b1[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) b0[i] = b1[i] = make_float2(0.f, 0.f);
        constexpr int KB = 8;                           // spectral rows in flight per thread
        for (int kb = 0; kb < M; kb += KB) {
            float2 qas[KB], qbs[KB];
#pragma unroll
            for (int q = 0; q < KB; ++q) {
                const bool in = kb + q < M;
                qas[q] = in ? qt[(k1a * M + kb + q) * 32] : make_float2(0.f, 0.f);
                qbs[q] = (in && hasb) ? qt[(k1b * M + kb + q) * 32] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < KB; ++q) {
            const int kk = kb + q;
            if (kk >= M) break;
            const float2 qa = qas[q], qb = qbs[q];
            const float4 *t = reinterpret_cast<const float4 *>(T2s + kk * 32 + blk * 16);
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const float4 e = t[i / 2];
                cmac_conj32(b0[i], qa, e.x, e.y);
                cmac_conj32(b0[i + 1], qa, e.z, e.w);
                cmac_conj32(b1[i], qb, e.x, e.y);
                cmac_conj32(b1[i + 1], qb, e.z, e.w);
            }
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j2 = blk * 16 + i;
            if (j2 < N) {
                Bs[(k1a * N + j2) * kPitch + lane] = b0[i];
                if (hasb) Bs[(k1b * N + j2) * kPitch + lane] = b1[i];
            }
        }
    }
    __syncthreads();
    // ---- stage 2: warp = cell pair, lane = j2 ----
    const int c0 = warp, c1 = warp + 16;
    float q0[N], q1[N];
#pragma unroll
    for (int j = 0; j < N; ++j) q0[j] = q1[j] = 0.f;
    if (lane < N) {
#pragma unroll 2
        for (int k1 = 0; k1 < H; ++k1) {
            const float2 ba = Bs[(k1 * N + lane) * kPitch + c0];
            const float2 bb = Bs[(k1 * N + lane) * kPitch + c1];
            const float4 *t = reinterpret_cast<const float4 *>(T3s + k1 * N);
#pragma unroll
            for (int j = 0; j < N; j += 2) {
                const float4 e = t[j / 2];             // Re(b conj(e)) = b.x e.x + b.y e.y
                q0[j] = fmaf(ba.x, e.x, fmaf(ba.y, e.y, q0[j]));
                q0[j + 1] = fmaf(ba.x, e.z, fmaf(ba.y, e.w, q0[j + 1]));
                q1[j] = fmaf(bb.x, e.x, fmaf(bb.y, e.y, q1[j]));
                q1[j + 1] = fmaf(bb.x, e.z, fmaf(bb.y, e.w, q1[j + 1]));
            }
        }
    }
    inv32_epilogue<N>(q0, tile * 32 + c0, lane, cinv, conserve, P, Q, L, dv, n);
    inv32_epilogue<N>(q1, tile * 32 + c1, lane, cinv, conserve, P, Q, L, dv, n);
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

__constant__ float2 c_w32[32];          // e^{-2 pi i k / 32}, k = 0..31

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// In-place radix-2 decimation-in-time FFT of length L <= 32 whose input sits
// in bit-reversed order; output in natural order.  SIGN = -1: sum x_n
// e^{-2 pi i k n / L}; SIGN = +1: sum x_n e^{+2 pi i k n / L} (unnormalised).
template <int L, int SIGN>
__device__ __forceinline__ void fft_dit(float2 (&a)[L]) {
#pragma unroll
    for (int m = 1; m < L; m <<= 1) {
#pragma unroll
        for (int g = 0; g < L; g += 2 * m) {
#pragma unroll
            for (int j = 0; j < m; ++j) {
                const float2 b = a[g + j + m];
                float2 t;
                if (j == 0) {
                    t = b;
                } else if (2 * j == m) {                       // twiddle -i (forward) or +i (inverse)
                    t = SIGN < 0 ? make_float2(b.y, -b.x) : make_float2(-b.y, b.x);
                } else {
                    const float2 w = c_w32[j * (32 / (2 * m))];
                    const float wy = SIGN < 0 ? w.y : -w.y;    // conj for the inverse
                    t = make_float2(b.x * w.x - b.y * wy, b.x * wy + b.y * w.x);
                }
                const float2 u = a[g + j];
                a[g + j] = make_float2(u.x + t.x, u.y + t.y);
                a[g + j + m] = make_float2(u.x - t.x, u.y - t.y);
            }
        }
    }
}

// One CTA handles C cells (C = 32: a whole 32-cell tile of the Fourier layout,
// or C = 16: half of one, so that two CTAs fit an SM and one's memory traffic
// overlaps the other's arithmetic) with 16 C threads.
template <int N, int C>
__global__ void __launch_bounds__(C * 16)
fft_fwd32_kernel(const float *__restrict__ f, float2 *__restrict__ fhat, int64_t n) {
    constexpr int H = N / 2, M = N - 1, NV = N * N, LH = ilog2(H), LN = ilog2(N);
    constexpr int NW = C / 2, P = C + 1;                // warps; cell pitch of the shared rows
    extern __shared__ __align__(16) float2 As[];        // [H][N][P]
    const int64_t tile = blockIdx.x / (32 / C);
    const int sub = (int)(blockIdx.x % (32 / C)) * C;   // first cell of this CTA within the tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- stage 1: lane = column j2 of cells warp, warp + NW, ...; real FFT over j1 ----
    if (lane < N) {
#pragma unroll 1
        for (int c = warp; c < C; c += NW) {
            const int64_t g = tile * 32 + sub + c;
            const bool ok = g < n;
            const float *fc = f + g * NV + lane;
            float2 z[H];
#pragma unroll
            for (int p = 0; p < H; ++p) {
                const float x0 = ok ? __ldg(fc + (2 * p) * N) : 0.f;
                const float x1 = ok ? __ldg(fc + (2 * p + 1) * N) : 0.f;
                z[bitrev(p, LH)] = make_float2(x0, x1);   // packed even / odd samples
            }
            fft_dit<H, -1>(z);
            // untangle: X[k] = E[k] + omega^-k O[k], E = (Z_k + conj Z_-k)/2,
            // O = (Z_k - conj Z_-k)/(2i); scale (-1)^k / N
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const float2 zk = z[k], zc = z[(H - k) % H];
                const float ex = 0.5f * (zk.x + zc.x), ey = 0.5f * (zk.y - zc.y);
                const float ox = 0.5f * (zk.y + zc.y), oy = -0.5f * (zk.x - zc.x);
                const float2 w = c_w32[k * (32 / N)];
                const float xr = ex + (w.x * ox - w.y * oy);
                const float xi = ey + (w.x * oy + w.y * ox);
                const float sc = (k & 1) ? -1.f / N : 1.f / N;
                As[(k * N + lane) * P + c] = make_float2(xr * sc, xi * sc);
            }
        }
    }
    __syncthreads();
    // ---- stage 2: thread = (cell, row k1); complex FFT over j2 ----
    const int cell = threadIdx.x % C;
    const int64_t gc = tile * 32 + sub + cell;
#pragma unroll 1
    for (int k1 = threadIdx.x / C; k1 < H; k1 += 16) {
        float2 a[N];
#pragma unroll
        for (int j = 0; j < N; ++j) a[bitrev(j, LN)] = As[(k1 * N + j) * P + cell];
        fft_dit<N, -1>(a);
        if (gc < n) {
            float2 *out = fhat + tile * (int64_t)(H * M) * 32 + (int64_t)k1 * M * 32 + sub + cell;
#pragma unroll
            for (int kk = 0; kk < M; ++kk) {
                const int k2 = kk - (H - 1);
                const float sc = (k2 & 1) ? -1.f / N : 1.f / N;
                const float2 v = a[k2 & (N - 1)];
                out[kk * 32] = make_float2(v.x * sc, v.y * sc);
            }
        }
    }
}

template <int N, int C>
__global__ void __launch_bounds__(C * 16)
fft_inv32_kernel(const float2 *__restrict__ Qhat, float *__restrict__ Q, float scale, Cinv cinv, int conserve,
                 const float *__restrict__ P_, double L, double dv, int64_t n) {
    constexpr int H = N / 2, M = N - 1, LH = ilog2(H), LN = ilog2(N);
    constexpr int NW = C / 2, P = C + 1;
    extern __shared__ __align__(16) float2 Bs[];        // [H][N][P]
    const int64_t tile = blockIdx.x / (32 / C);
    const int sub = (int)(blockIdx.x % (32 / C)) * C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- stage 1: thread = (cell, row k1); inverse complex FFT over k2 ----
    {
        const int cell = threadIdx.x % C;
        const float2 *qt = Qhat + tile * (int64_t)(H * M) * 32 + sub + cell;
#pragma unroll 1
        for (int k1 = threadIdx.x / C; k1 < H; k1 += 16) {
            float2 a[N];
            a[bitrev(H, LN)] = make_float2(0.f, 0.f);   // Nyquist slot k2 = N/2
#pragma unroll
            for (int kk = 0; kk < M; ++kk) {
                const int k2 = kk - (H - 1);
                const float2 v = qt[(k1 * M + kk) * 32];
                a[bitrev(k2 & (N - 1), LN)] = (k2 & 1) ? make_float2(-v.x, -v.y) : v;
            }
            fft_dit<N, +1>(a);
            const float sc = (k1 & 1) ? -scale : scale; // s^(d+gamma) (-1)^k1
#pragma unroll
            for (int j = 0; j < N; ++j) Bs[(k1 * N + j) * P + cell] = make_float2(a[j].x * sc, a[j].y * sc);
        }
    }
    __syncthreads();
    // ---- stage 2: lane = column j2 of cells warp, warp + NW, ...; Hermitian-to-real over k1 ----
#pragma unroll 1
    for (int c = warp; c < C; c += NW) {
        float q[N];
        if (lane < N) {
            float2 x[H + 1];
#pragma unroll
            for (int k = 0; k < H; ++k) x[k] = Bs[(k * N + lane) * P + c];
            x[0].y = 0.f;                                // real part of the k1 = 0 row
            x[H] = make_float2(0.f, 0.f);
            // Z[k] = E[k] + i O[k], E = X_k + conj X_{H-k}, O = (X_k - conj X_{H-k}) omega^k
            float2 z[H];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const float2 xk = x[k], xc = make_float2(x[H - k].x, -x[H - k].y);
                float ex, ey, ox, oy;
                if (k == 0) {
                    ex = xk.x; ey = xk.y; ox = xk.x; oy = xk.y;
                } else {
                    ex = xk.x + xc.x;
                    ey = xk.y + xc.y;
                    const float dx = xk.x - xc.x, dy = xk.y - xc.y;
                    const float2 w = c_w32[k * (32 / N)];           // omega^k = conj(w)
                    ox = dx * w.x + dy * w.y;
                    oy = dy * w.x - dx * w.y;
                }
                z[bitrev(k, LH)] = make_float2(ex - oy, ey + ox);
            }
            fft_dit<H, +1>(z);
#pragma unroll
            for (int p = 0; p < H; ++p) {
                q[2 * p] = z[p].x;
                q[2 * p + 1] = z[p].y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) q[j] = 0.f;
        }
        inv32_epilogue<N>(q, tile * 32 + sub + c, lane, cinv, conserve, P_, Q, L, dv, n);
    }
}

template <int N, int C> size_t fft_smem() { return sizeof(float2) * (size_t)(N / 2) * N * (C + 1); }
constexpr int kFftCells = 16;   // cells per CTA of the FFT kernels

template <int N> size_t fwd_smem() { return sizeof(float2) * ((N / 2) * N * kPitch + N * (N / 2) + N * 32); }
template <int N> size_t inv_smem() { return sizeof(float2) * ((N / 2) * N * kPitch + (N - 1) * 32 + (N / 2) * N); }

}  // namespace

bool dft32_tile_supported(const GridView &g) { return g.dim == 2 && (g.N == 16 || g.N == 24 || g.N == 32); }

// Host-built twiddle tables for the tile kernels (see the table comments above).
int dft32_tables(const GridView &g, double scale, float2 **out_T1, float2 **out_T2, float2 **out_T2i,
                 float2 **out_T3) {
    const int N = g.N, H = g.h + 1, h = g.h, M = g.M;
    std::vector<float2> T1((size_t)N * H), T2((size_t)N * 32), T2i((size_t)M * 32), T3((size_t)H * N);
    auto E = [&](int k, int j) {              // (-1)^k exp(-2 pi i (k j mod N)/N)
        long r = ((long)k * j) % N;
        if (r < 0) r += N;
        double ang = 2.0 * M_PI * (double)r / N, sg = (k & 1) ? -1.0 : 1.0;
        return std::make_pair(sg * cos(ang), -sg * sin(ang));
    };
    for (int j = 0; j < N; ++j)
        for (int k = 0; k < H; ++k) {
            auto e = E(k, j);
            T1[(size_t)j * H + k] = make_float2((float)(e.first / N), (float)(e.second / N));
        }
    for (int j = 0; j < N; ++j)
        for (int kk = 0; kk < 32; ++kk) {
            float2 v = make_float2(0.f, 0.f);
            if (kk < M) {
                auto e = E(kk - h, j);
                v = make_float2((float)(e.first / N), (float)(e.second / N));
            }
            T2[(size_t)j * 32 + kk] = v;
        }
    for (int kk = 0; kk < M; ++kk)
        for (int j = 0; j < 32; ++j) {
            float2 v = make_float2(0.f, 0.f);
            if (j < N) {
                auto e = E(kk - h, j);
                v = make_float2((float)e.first, (float)e.second);
            }
            T2i[(size_t)kk * 32 + j] = v;
        }
    for (int k = 0; k < H; ++k)
        for (int j = 0; j < N; ++j) {
            auto e = E(k, j);
            double c = (k == 0 ? 1.0 : 2.0) * scale;
            T3[(size_t)k * N + j] = make_float2((float)(c * e.first), (float)(c * e.second));
        }
    // twiddles of the FFT kernels, on the current device (constant memory is per device)
    float2 w32[32];
    for (int k = 0; k < 32; ++k) w32[k] = make_float2((float)cos(2.0 * M_PI * k / 32), (float)-sin(2.0 * M_PI * k / 32));
    cudaError_t ew = cudaMemcpyToSymbol(c_w32, w32, sizeof w32);
    if (ew != cudaSuccess) return cuda_fail(ew, "build_kernel_modes: FFT twiddles");
    float2 *d[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<float2> *src[4] = {&T1, &T2, &T2i, &T3};
    for (int i = 0; i < 4; ++i) {
        cudaError_t e = cudaMalloc(&d[i], sizeof(float2) * src[i]->size());
        if (e == cudaSuccess)
            e = cudaMemcpy(d[i], src[i]->data(), sizeof(float2) * src[i]->size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            for (int q = 0; q <= i; ++q) cudaFree(d[q]);
            return cuda_fail(e, "build_kernel_modes: DFT tables");
        }
    }
    *out_T1 = d[0];
    *out_T2 = d[1];
    *out_T2i = d[2];
    *out_T3 = d[3];
    return BZ_OK;
}

cudaError_t launch_dft32_forward_tile(const GridView &g, const float2 *T1, const float2 *T2, const float *f,
                                      float2 *fhat, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const unsigned ntile = (unsigned)((n + 31) / 32);
    cudaError_t e = cudaSuccess;
#define BZ_FWD(NN)                                                                                       \
    case NN: {                                                                                           \
        size_t sm = fwd_smem<NN>();                                                                      \
        e = cudaFuncSetAttribute(dft_fwd32_kernel<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e != cudaSuccess) return e;                                                                  \
        dft_fwd32_kernel<NN><<<ntile, kThreads, sm, st>>>(f, fhat, T1, T2, n);                           \
        break;                                                                                           \
    }
#define BZ_FFT_FWD(NN)                                                                                   \
    case NN: {                                                                                           \
        size_t sm = fft_smem<NN, kFftCells>();                                                           \
        e = cudaFuncSetAttribute(fft_fwd32_kernel<NN, kFftCells>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e != cudaSuccess) return e;                                                                  \
        fft_fwd32_kernel<NN, kFftCells><<<ntile * (32 / kFftCells), kFftCells * 16, sm, st>>>(f, fhat, n); \
        break;                                                                                           \
    }
    switch (g.N) {
        BZ_FFT_FWD(16)
        BZ_FWD(24)
        BZ_FFT_FWD(32)
        default: return cudaErrorInvalidValue;
    }
#undef BZ_FWD
#undef BZ_FFT_FWD
    return cudaGetLastError();
}

cudaError_t launch_dft32_inverse_tile(const GridView &g, const float2 *T2i, const float2 *T3, const float2 *Qhat,
                                      float *Q, int64_t n, double scale, const double *cinv, const InvEpilogue &ep,
                                      cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const unsigned ntile = (unsigned)((n + 31) / 32);
    Cinv ci;
    for (int i = 0; i < 25; ++i) ci.v[i] = cinv[i];
    cudaError_t e = cudaSuccess;
#define BZ_INV(NN)                                                                                       \
    case NN: {                                                                                           \
        size_t sm = inv_smem<NN>();                                                                      \
        e = cudaFuncSetAttribute(dft_inv32_kernel<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e != cudaSuccess) return e;                                                                  \
        dft_inv32_kernel<NN><<<ntile, kThreads, sm, st>>>(Qhat, Q, T2i, T3, ci, ep.conserve,             \
                                                          static_cast<const float *>(ep.P), g.L, g.dv, n); \
        break;                                                                                           \
    }
#define BZ_FFT_INV(NN)                                                                                   \
    case NN: {                                                                                           \
        size_t sm = fft_smem<NN, kFftCells>();                                                           \
        e = cudaFuncSetAttribute(fft_inv32_kernel<NN, kFftCells>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e != cudaSuccess) return e;                                                                  \
        fft_inv32_kernel<NN, kFftCells><<<ntile * (32 / kFftCells), kFftCells * 16, sm, st>>>(           \
            Qhat, Q, (float)scale, ci, ep.conserve, static_cast<const float *>(ep.P), g.L, g.dv, n);     \
        break;                                                                                           \
    }
    switch (g.N) {
        BZ_FFT_INV(16)
        BZ_INV(24)
        BZ_FFT_INV(32)
        default: return cudaErrorInvalidValue;
    }
#undef BZ_INV
#undef BZ_FFT_INV
    return cudaGetLastError();
}

}  // namespace bz
