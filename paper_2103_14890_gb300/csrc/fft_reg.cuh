// fft_reg.cuh -- register-resident FFTs of small lengths (2^p <= 32,
// 3 * 2^p <= 48 and 72), unrolled with compile-time indices so that the data stay in
// registers and the twiddles are constant-bank operands.  Each translation
// unit that includes this header gets its own copy of the twiddle tables in
// constant memory and must fill it with upload_fft_twiddles() on every device
// it launches on.
#pragma once

#include <math.h>

#include "bz_device.cuh"

namespace bz {
namespace {

__constant__ float2 c_w32[32];          // e^{-2 pi i k / 32}, k = 0..31
__constant__ double2 c_w32d[32];

template <typename V> __device__ __forceinline__ V tw32(int k);
template <> __device__ __forceinline__ float2 tw32<float2>(int k) { return c_w32[k]; }
template <> __device__ __forceinline__ double2 tw32<double2>(int k) { return c_w32d[k]; }

// Complex sums and differences: one FP32x2 instruction for float2 (two IEEE
// FP32 additions, the results of the scalar form), two scalar ones otherwise.
template <typename V> __device__ __forceinline__ V c_add(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V c_sub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <> __device__ __forceinline__ float2 c_add<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 c_sub<float2>(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// In-place radix-2 decimation-in-time FFT of length L <= 32 whose input sits
// in bit-reversed order; output in natural order.  SIGN = -1: sum x_n
// e^{-2 pi i k n / L}; SIGN = +1: sum x_n e^{+2 pi i k n / L} (unnormalised).
template <int L, int SIGN, typename V>
__device__ __forceinline__ void fft_dit(V (&a)[L]) {
    using S = decltype(V::x);
    using V2 = V;
#pragma unroll
    for (int m = 1; m < L; m <<= 1) {
#pragma unroll
        for (int g = 0; g < L; g += 2 * m) {
#pragma unroll
            for (int j = 0; j < m; ++j) {
                const V2 b = a[g + j + m];
                V2 t;
                if (j == 0) {
                    t = b;
                } else if (2 * j == m) {                       // twiddle -i (forward) or +i (inverse)
                    t = SIGN < 0 ? cmk<V2>(b.y, -b.x) : cmk<V2>(-b.y, b.x);
                } else {
                    const V w = tw32<V>(j * (32 / (2 * m)));
                    const S wy = SIGN < 0 ? w.y : -w.y;    // conj for the inverse
                    t = cmk<V2>(b.x * w.x - b.y * wy, b.x * wy + b.y * w.x);
                }
                const V2 u = a[g + j];
                a[g + j] = c_add(u, t);
                a[g + j + m] = c_sub(u, t);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Mixed-radix form for lengths 3 * 2^p (<= 48) and 72: a length-3Q transform
// is split by Cooley-Tukey into Q-point transforms of the three residue
// classes n = Q n1 + n2 (3-point DFTs over n1, twiddles omega_L^(n2 k1), then
// Q-point FFTs over n2; output index k1 + 3 k2).

__constant__ float2 c_w48[48];          // e^{-2 pi i k / 48}, k = 0..47
__constant__ double2 c_w48d[48];
__constant__ float2 c_w72[72];          // e^{-2 pi i k / 72}, k = 0..71
__constant__ double2 c_w72d[72];

template <typename V> __device__ __forceinline__ V tw48(int k);
template <> __device__ __forceinline__ float2 tw48<float2>(int k) { return c_w48[k]; }
template <> __device__ __forceinline__ double2 tw48<double2>(int k) { return c_w48d[k]; }
template <typename V> __device__ __forceinline__ V tw72(int k);
template <> __device__ __forceinline__ float2 tw72<float2>(int k) { return c_w72[k]; }
template <> __device__ __forceinline__ double2 tw72<double2>(int k) { return c_w72d[k]; }

// e^{-2 pi i k / L} for any L dividing 32, 48 or 72
template <int L, typename V> __device__ __forceinline__ V twl(int k) {
    static_assert(32 % L == 0 || 48 % L == 0 || 72 % L == 0, "length divides 32, 48 or 72");
    if constexpr (32 % L == 0) return tw32<V>(k * (32 / L));
    else if constexpr (48 % L == 0) return tw48<V>(k * (48 / L));
    else return tw72<V>(k * (72 / L));
}

// Transform of length L (2^p <= 32, 3 * 2^p <= 48, or 72) from natural to
// natural order; SIGN as in fft_dit.
template <int L, int SIGN, typename V>
__device__ __forceinline__ void fft_nat(V (&a)[L]) {
    using S = decltype(V::x);
    using V2 = V;
    if constexpr ((L & (L - 1)) == 0) {
        V2 b[L];
#pragma unroll
        for (int i = 0; i < L; ++i) b[bitrev(i, ilog2(L))] = a[i];
        fft_dit<L, SIGN>(b);
#pragma unroll
        for (int i = 0; i < L; ++i) a[i] = b[i];
    } else {
        static_assert(L % 3 == 0 && (L <= 48 || L == 72), "length 3 * 2^p <= 48 or 72");
        constexpr int Q = L / 3;
        constexpr S kS3 = (S)0.866025403784438647;    // sqrt(3) / 2
        V2 y0[Q], y1[Q], y2[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            const V2 p = a[n2], q = a[Q + n2], r = a[2 * Q + n2];
            const V2 sq = c_add(q, r), dq = c_sub(q, r);
            y0[n2] = c_add(p, sq);
            const V2 mq = cmk<V2>(p.x - (S)0.5 * sq.x, p.y - (S)0.5 * sq.y);
            // -i (sqrt3/2) d for the forward transform, +i (sqrt3/2) d for the inverse
            const V2 iq = SIGN < 0 ? cmk<V2>(kS3 * dq.y, -kS3 * dq.x) : cmk<V2>(-kS3 * dq.y, kS3 * dq.x);
            V2 u1 = c_add(mq, iq), u2 = c_sub(mq, iq);
            if (n2 > 0) {
                const V w1 = twl<L, V>(n2), w2 = twl<L, V>(2 * n2);
                const S w1y = SIGN < 0 ? w1.y : -w1.y, w2y = SIGN < 0 ? w2.y : -w2.y;
                u1 = cmk<V2>(u1.x * w1.x - u1.y * w1y, u1.x * w1y + u1.y * w1.x);
                u2 = cmk<V2>(u2.x * w2.x - u2.y * w2y, u2.x * w2y + u2.y * w2.x);
            }
            y1[n2] = u1;
            y2[n2] = u2;
        }
        fft_nat<Q, SIGN>(y0);
        fft_nat<Q, SIGN>(y1);
        fft_nat<Q, SIGN>(y2);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
            a[3 * k2] = y0[k2];
            a[3 * k2 + 1] = y1[k2];
            a[3 * k2 + 2] = y2[k2];
        }
    }
}

// fft_nat of length L = 3Q for input whose middle third a[Q .. 2Q-1] is zero
// (a spectrum of modes |k| < L/3 zero-padded to L: the indices k and L - |k|
// occupy the first and last thirds only).  The first stage's 3-point DFTs
// then take two inputs: the sums with the zero third are left out.
template <int L, int SIGN, typename V>
__device__ __forceinline__ void fft_nat_mid0(V (&a)[L]) {
    using S = decltype(V::x);
    using V2 = V;
    static_assert(L % 3 == 0 && (L <= 48 || L == 72), "length 3 * 2^p <= 48 or 72");
    constexpr int Q = L / 3;
    constexpr S kS3 = (S)0.866025403784438647;    // sqrt(3) / 2
    V2 y0[Q], y1[Q], y2[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
        const V2 p = a[n2], r = a[2 * Q + n2];
        y0[n2] = c_add(p, r);
        const V2 mq = cmk<V2>(p.x - (S)0.5 * r.x, p.y - (S)0.5 * r.y);
        // the 3-point DFT's +/- i (sqrt3/2)(q - r) with q = 0
        const V2 iq = SIGN < 0 ? cmk<V2>(-kS3 * r.y, kS3 * r.x) : cmk<V2>(kS3 * r.y, -kS3 * r.x);
        V2 u1 = c_add(mq, iq), u2 = c_sub(mq, iq);
        if (n2 > 0) {
            const V w1 = twl<L, V>(n2), w2 = twl<L, V>(2 * n2);
            const S w1y = SIGN < 0 ? w1.y : -w1.y, w2y = SIGN < 0 ? w2.y : -w2.y;
            u1 = cmk<V2>(u1.x * w1.x - u1.y * w1y, u1.x * w1y + u1.y * w1.x);
            u2 = cmk<V2>(u2.x * w2.x - u2.y * w2y, u2.x * w2y + u2.y * w2.x);
        }
        y1[n2] = u1;
        y2[n2] = u2;
    }
    fft_nat<Q, SIGN>(y0);
    fft_nat<Q, SIGN>(y1);
    fft_nat<Q, SIGN>(y2);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
        a[3 * k2] = y0[k2];
        a[3 * k2 + 1] = y1[k2];
        a[3 * k2 + 2] = y2[k2];
    }
}

// e^{-2 pi i k / N} for N in {16, 24, 32, 48}
template <int N, typename V> __device__ __forceinline__ V tw(int k) {
    if constexpr (N == 16 || N == 32) return tw32<V>(k * (32 / N));
    else return tw48<V>(k * (48 / N));
}

// Fill this translation unit's twiddle tables on the current device.
inline cudaError_t upload_fft_twiddles() {
    float2 w32[32], w48[48], w72[72];
    double2 d32[32], d48[48], d72[72];
    for (int k = 0; k < 32; ++k) {
        d32[k] = make_double2(cos(2.0 * M_PI * k / 32), -sin(2.0 * M_PI * k / 32));
        w32[k] = make_float2((float)d32[k].x, (float)d32[k].y);
    }
    for (int k = 0; k < 48; ++k) {
        d48[k] = make_double2(cos(2.0 * M_PI * k / 48), -sin(2.0 * M_PI * k / 48));
        w48[k] = make_float2((float)d48[k].x, (float)d48[k].y);
    }
    for (int k = 0; k < 72; ++k) {
        d72[k] = make_double2(cos(2.0 * M_PI * k / 72), -sin(2.0 * M_PI * k / 72));
        w72[k] = make_float2((float)d72[k].x, (float)d72[k].y);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_w32, w32, sizeof w32);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w48, w48, sizeof w48);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w32d, d32, sizeof d32);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w48d, d48, sizeof d48);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w72, w72, sizeof w72);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w72d, d72, sizeof d72);
    return e;
}

}  // namespace
}  // namespace bz
