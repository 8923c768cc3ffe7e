// k_transport.cu -- transport residual of the finite-volume scheme (Sec. 3.2,
// eq. finite_vol5 / eq. ho): CWENO reconstruction of degree 1 and Rusanov
// fluxes, for every cell and every discrete velocity of a 2-D grid.
//
// Layout: f, L are [cell][nv] (the collision operator's layout), so one
// cell's velocities are contiguous.  A block takes 1024 velocities of one cell
// (4 per thread on triangle meshes): every table entry of the cell is a
// warp-uniform load shared by 4 velocities and every f access is a 16-byte
// vector of one coalesced row segment (neighbour rows come from L2: a 32^2
// grid of 20k cells holds 81 MB in FP32).  Cells are taken along a Morton
// curve of their barycentres (the mesh's order table).  On FP32 triangle
// meshes without walls both passes of degree 1 are persistent: a block walks
// the order in steps of the grid, staging the next cell's rows in shared
// memory while it computes the current one.
//
// Pass 1 (order 2): gradient of the CWENO polynomial per (cell, velocity),
// stored as G [cell][2][nv] (FP32 triangle meshes without walls: the values at
// the three face midpoints, FV [cell][3][nv]).  The central (least-squares)
// gradient g_opt and
// the sector gradients g_L are linear in the averages (tables R_c, R_s of
// fv_mesh.cpp); the central polynomial's gradient is g_0 = (g_opt - sum_L
// lambda_L g_L) / lambda_0 (eq. CWENO:P0, lambda_0 = 3/4, lambda_L = 1/4 /
// #sectors); smoothness sigma_s = h^2 |g_s|^2; weights omega_s proportional
// to lambda_s / (sigma_s + eps)^4 with eps = 1e-14 (eqn.weights), formed
// as lambda_s ((sigma_min + eps) / (sigma_s + eps))^4 so that no power
// underflows in FP32.
//
// The flux passes take the cells in the reverse of the reconstruction's
// order, so that they start on the rows the reconstruction wrote last, which
// are still in L2.
//
// Pass 2: per face, f_L = fbar_i + g_i . (x_f - x_b,i), f_R the same from the
// neighbour (f_L on a boundary face: transmissive), Rusanov flux of v f:
// |e| F = (v.|e|n)(f_L + f_R)/2 - |v.|e|n| (f_R - f_L)/2, summed and scaled
// by 1/|P_i|.  The face midpoint rule is exact for degree-1 reconstructions.
#include <algorithm>
#include <atomic>

#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int kFvThreads = 256;

// VEC consecutive velocities per thread: the cell's table entries are loaded
// once for all of them and f moves in 16-byte vectors (the row length N^2 is
// a multiple of 4, and the host checks 16-byte alignment, else VEC = 1).
template <typename T, int VEC> struct Vec {
    T v[VEC];
};
template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ldv(const T *__restrict__ p) {
    Vec<T, VEC> r;
    if constexpr (VEC == 4 && sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else if constexpr (VEC == 4 && sizeof(T) == 8) {
        const double2 q0 = reinterpret_cast<const double2 *>(p)[0], q1 = reinterpret_cast<const double2 *>(p)[1];
        r.v[0] = q0.x; r.v[1] = q0.y; r.v[2] = q1.x; r.v[3] = q1.y;
    } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) r.v[u] = p[u];
    }
    return r;
}
template <typename T, int VEC>
__device__ __forceinline__ void stv(T *__restrict__ p, const Vec<T, VEC> &r) {
    if constexpr (VEC == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else if constexpr (VEC == 4 && sizeof(T) == 8) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(r.v[0], r.v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(r.v[2], r.v[3]);
    } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) p[u] = r.v[u];
    }
}

// FP32x2 arithmetic on pairs of velocities: one FADD2 / FMUL2 / FFMA2 rounds
// each lane as its scalar instruction does.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 lo2(const float4 &a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(const float4 &a) { return make_float2(a.z, a.w); }
// approximate reciprocal (1 ulp; the argument is a normal number here)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }

// CWENO gradient of one pair of velocities of a flagged triangle (kFvRegularTri):
// d[q] = fbar_{cen q} - fbar_i, the face neighbours in d[0..2]; sector s
// joins faces s and s + 1 mod 3.  The steps are those of the generic kernel
// below (central gradient, sector gradients, g_0, smoothness, weights as
// lambda_s ((sigma_min + eps) / (sigma_s + eps))^4, normalised sum).
__device__ __forceinline__ void cweno_pair_tri(const float2 (&d)[kFvCentral], const float (&rx)[kFvCentral],
                                               const float (&ry)[kFvCentral], const float4 (&R)[3], float h2,
                                               float2 &gx_out, float2 &gy_out) {
    constexpr float kLam0 = 0.75f, kInvLam0 = (float)(4.0 / 3.0), kEps = 1e-14f;
    const float lamL = 0.25f / 3.0f;
    float2 gx = mul2(dup2(rx[0]), d[0]), gy = mul2(dup2(ry[0]), d[0]);
#pragma unroll
    for (int q = 1; q < kFvCentral; ++q) {
        gx = fma2(dup2(rx[q]), d[q], gx);
        gy = fma2(dup2(ry[q]), d[q], gy);
    }
    float2 sx[3], sy[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const float2 da = d[s], db = d[(s + 1) % 3];
        sx[s] = fma2(dup2(R[s].x), da, mul2(dup2(R[s].y), db));
        sy[s] = fma2(dup2(R[s].z), da, mul2(dup2(R[s].w), db));
    }
    const float2 sumx = add2(add2(sx[0], sx[1]), sx[2]), sumy = add2(add2(sy[0], sy[1]), sy[2]);
    const float2 g0x = mul2(fma2(dup2(-lamL), sumx, gx), dup2(kInvLam0));
    const float2 g0y = mul2(fma2(dup2(-lamL), sumy, gy), dup2(kInvLam0));
    const float2 H = dup2(h2), E = dup2(kEps);
    const float2 sig0 = mul2(H, fma2(g0x, g0x, mul2(g0y, g0y)));
    float2 sig[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) sig[s] = mul2(H, fma2(sx[s], sx[s], mul2(sy[s], sy[s])));
    const float2 smin = make_float2(fminf(fminf(sig0.x, sig[0].x), fminf(sig[1].x, sig[2].x)),
                                    fminf(fminf(sig0.y, sig[0].y), fminf(sig[1].y, sig[2].y)));
    const float2 num = add2(smin, E);
    float2 r = mul2(num, rcp2(add2(sig0, E)));
    r = mul2(r, r);
    float2 w = mul2(dup2(kLam0), mul2(r, r));
    float2 wsum = w, ax = mul2(w, g0x), ay = mul2(w, g0y);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        r = mul2(num, rcp2(add2(sig[s], E)));
        r = mul2(r, r);
        w = mul2(dup2(lamL), mul2(r, r));
        wsum = add2(wsum, w);
        ax = fma2(w, sx[s], ax);
        ay = fma2(w, sy[s], ay);
    }
    const float2 iw = rcp2(wsum);
    gx_out = mul2(ax, iw);
    gy_out = mul2(ay, iw);
}

// Gradient of the 4 velocities k..k+3 of a flagged triangle in FP32x2: six
// rows of f (the cell and its stencil, the face neighbours first), each
// loaded once.  FACE: the output is the reconstruction's value at the three
// face midpoints, f_i + g . (x_f - x_b,i), rows [cell][face][nv], in place of
// the gradient rows [cell][2][nv].
template <bool FACE>
__device__ __forceinline__ void tri_x2_rows(float *__restrict__ G, const FvTables<float> &tb,
                                            const float4 (&fr)[kFvCentral], int64_t i, int k, int nv,
                                            const float4 fi) {
    float rx[kFvCentral], ry[kFvCentral];
#pragma unroll
    for (int q = 0; q < kFvCentral; ++q) {
        rx[q] = __ldg(tb.Rc + (i * 2) * kFvCentral + q);
        ry[q] = __ldg(tb.Rc + (i * 2 + 1) * kFvCentral + q);
    }
    float4 R[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) R[s] = __ldg(reinterpret_cast<const float4 *>(tb.Rs + (i * kFvMaxFaces + s) * 4));
    const float h2 = __ldg(tb.h2 + i);
    float2 gx[2], gy[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float2 nf = neg2(p == 0 ? lo2(fi) : hi2(fi));
        float2 d[kFvCentral];
#pragma unroll
        for (int q = 0; q < kFvCentral; ++q) d[q] = add2(p == 0 ? lo2(fr[q]) : hi2(fr[q]), nf);
        cweno_pair_tri(d, rx, ry, R, h2, gx[p], gy[p]);
    }
    if constexpr (FACE) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float2 ox = dup2(__ldg(tb.off_i + 2 * (i * kFvMaxFaces + q)));
            const float2 oy = dup2(__ldg(tb.off_i + 2 * (i * kFvMaxFaces + q) + 1));
            const float2 a = fma2(gy[0], oy, fma2(gx[0], ox, lo2(fi)));
            const float2 b = fma2(gy[1], oy, fma2(gx[1], ox, hi2(fi)));
            *reinterpret_cast<float4 *>(G + (i * 3 + q) * nv + k) = make_float4(a.x, a.y, b.x, b.y);
        }
    } else {
        *reinterpret_cast<float4 *>(G + (i * 2) * nv + k) = make_float4(gx[0].x, gx[0].y, gx[1].x, gx[1].y);
        *reinterpret_cast<float4 *>(G + (i * 2 + 1) * nv + k) = make_float4(gy[0].x, gy[0].y, gy[1].x, gy[1].y);
    }
}

template <bool FACE>
__device__ __forceinline__ void gradient_tri_x2(const float *__restrict__ f, float *__restrict__ G,
                                                const FvTables<float> &tb, const int (&jc)[kFvCentral], int64_t i,
                                                int k, int nv, const float4 fi) {
    float4 fr[kFvCentral];
#pragma unroll
    for (int q = 0; q < kFvCentral; ++q) fr[q] = *reinterpret_cast<const float4 *>(f + (int64_t)jc[q] * nv + k);
    tri_x2_rows<FACE>(G, tb, fr, i, k, nv, fi);
}

// Reconstruction of cell i for the VEC velocities k.. of a thread (any
// polygon; MAXS bounds its sectors): gradients, or with FACE the values at
// the three face midpoints of a triangle.
template <typename T, int VEC, int MAXS, bool FACE>
__device__ __forceinline__ void gradient_generic(const T *__restrict__ f, T *__restrict__ G, const FvTables<T> &tb,
                                                 const int *__restrict__ cen, const int *__restrict__ nsec,
                                                 const int *__restrict__ sec, int64_t i, int ncf, int k, int nv,
                                                 const Vec<T, VEC> &fi) {
    const int nc = ncf & (kFvRegularTri - 1), ns = __ldg(nsec + i);
    // central least-squares gradient
    T gx[VEC], gy[VEC];
    {
        Vec<T, VEC> fj[kFvCentral];
        T rx[kFvCentral], ry[kFvCentral];
#pragma unroll
        for (int q = 0; q < kFvCentral; ++q) {
            rx[q] = ry[q] = (T)0;
            fj[q] = fi;
            if (q < nc) {
                const int j = __ldg(cen + i * kFvCentral + q);
                rx[q] = __ldg(tb.Rc + (i * 2) * kFvCentral + q);
                ry[q] = __ldg(tb.Rc + (i * 2 + 1) * kFvCentral + q);
                fj[q] = ldv<T, VEC>(f + (int64_t)j * nv + k);
            }
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
            gx[u] = gy[u] = (T)0;
#pragma unroll
            for (int q = 0; q < kFvCentral; ++q) {
                const T d = fj[q].v[u] - fi.v[u];
                gx[u] += rx[q] * d;
                gy[u] += ry[q] * d;
            }
        }
    }
    if (ns > 0) {
        constexpr T kLam0 = (T)0.75, kInvLam0 = (T)(4.0 / 3.0), kEps = (T)1e-14;
        const T lamL = (T)0.25 / (T)ns, h2 = __ldg(tb.h2 + i);
        T sx[MAXS][VEC], sy[MAXS][VEC];
        {
            Vec<T, VEC> fa[MAXS], fb[MAXS];
            T R[MAXS][4];
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                fa[s] = fi;
                fb[s] = fi;
                R[s][0] = R[s][1] = R[s][2] = R[s][3] = (T)0;
                if (s < ns) {
                    const int a = __ldg(sec + (i * kFvMaxFaces + s) * 2), b = __ldg(sec + (i * kFvMaxFaces + s) * 2 + 1);
                    const T *Rp = tb.Rs + (i * kFvMaxFaces + s) * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c) R[s][c] = __ldg(Rp + c);
                    fa[s] = ldv<T, VEC>(f + (int64_t)a * nv + k);
                    fb[s] = ldv<T, VEC>(f + (int64_t)b * nv + k);
                }
            }
#pragma unroll
            for (int s = 0; s < MAXS; ++s)
#pragma unroll
                for (int u = 0; u < VEC; ++u) {
                    const T da = fa[s].v[u] - fi.v[u], db = fb[s].v[u] - fi.v[u];
                    sx[s][u] = R[s][0] * da + R[s][1] * db;
                    sy[s][u] = R[s][2] * da + R[s][3] * db;
                }
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
            T sumx = (T)0, sumy = (T)0;
#pragma unroll
            for (int s = 0; s < MAXS; ++s)
                if (s < ns) {
                    sumx += sx[s][u];
                    sumy += sy[s][u];
                }
            const T g0x = (gx[u] - lamL * sumx) * kInvLam0, g0y = (gy[u] - lamL * sumy) * kInvLam0;
            const T sig0 = h2 * (g0x * g0x + g0y * g0y);
            T sig[MAXS];
            T smin = sig0;
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                sig[s] = h2 * (sx[s][u] * sx[s][u] + sy[s][u] * sy[s][u]);
                if (s < ns) smin = fmin(smin, sig[s]);
            }
            // weight ratios: FP32 takes the fast division (2 ulp; the weights
            // are smooth in sigma), FP64 the correctly rounded one
            const T num = smin + kEps;
            auto ratio = [](T a, T b) {
                if constexpr (sizeof(T) == 4) return __fdividef(a, b);
                else return a / b;
            };
            T r = ratio(num, sig0 + kEps);
            r = r * r;
            T w = kLam0 * (r * r);
            T wsum = w, ax = w * g0x, ay = w * g0y;
#pragma unroll
            for (int s = 0; s < MAXS; ++s)
                if (s < ns) {
                    r = ratio(num, sig[s] + kEps);
                    r = r * r;
                    w = lamL * (r * r);
                    wsum += w;
                    ax += w * sx[s][u];
                    ay += w * sy[s][u];
                }
            const T iw = (T)1 / wsum;
            gx[u] = ax * iw;
            gy[u] = ay * iw;
        }
    }
    if constexpr (FACE) {
        static_assert(MAXS == 3, "face values: triangle meshes");
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T ofx = __ldg(tb.off_i + 2 * (i * kFvMaxFaces + q)), ofy = __ldg(tb.off_i + 2 * (i * kFvMaxFaces + q) + 1);
            Vec<T, VEC> o;
#pragma unroll
            for (int u = 0; u < VEC; ++u) o.v[u] = fi.v[u] + gx[u] * ofx + gy[u] * ofy;
            stv<T, VEC>(G + (i * 3 + q) * nv + k, o);
        }
    } else {
        Vec<T, VEC> ox, oy;
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
            ox.v[u] = gx[u];
            oy.v[u] = gy[u];
        }
        stv<T, VEC>(G + (i * 2) * nv + k, ox);
        stv<T, VEC>(G + (i * 2 + 1) * nv + k, oy);
    }
}

// MAXS / MAXF: compile-time bound on the sectors / faces of a cell (3 for
// triangle meshes, kFvMaxFaces otherwise).  Every loop over them is unrolled
// with a predicate, so all neighbour rows of a cell are requested before the
// first one is used (the kernels are latency-bound otherwise).
template <typename T, int VEC, int MAXS>
__global__ void __launch_bounds__(kFvThreads, (sizeof(T) == 4 && VEC == 4) ? 4 : 1)
fv_gradient_kernel(const T *__restrict__ f, T *__restrict__ G, FvTables<T> tb, const int *__restrict__ ncen,
                   const int *__restrict__ cen, const int *__restrict__ nsec, const int *__restrict__ sec,
                   const int *__restrict__ order, int nv) {
    const int64_t i = __ldg(order + blockIdx.x);
    const int ncf = __ldg(ncen + i);
    const int k = (blockIdx.y * kFvThreads + threadIdx.x) * VEC;
    if (k >= nv) return;
    const Vec<T, VEC> fi = ldv<T, VEC>(f + i * nv + k);
    if constexpr (sizeof(T) == 4 && VEC == 4 && MAXS == 3) {
        if (ncf & kFvRegularTri) {      // uniform over the block: one cell per block
            int jc[kFvCentral];
#pragma unroll
            for (int q = 0; q < kFvCentral; ++q) jc[q] = __ldg(cen + i * kFvCentral + q);
            gradient_tri_x2<false>(f, G, tb, jc, i, k, nv, make_float4(fi.v[0], fi.v[1], fi.v[2], fi.v[3]));
            return;
        }
    }
    gradient_generic<T, VEC, MAXS, false>(f, G, tb, cen, nsec, sec, i, ncf, k, nv, fi);
}

template <typename T, bool kGrad, int VEC, int MAXF>
__global__ void __launch_bounds__(kFvThreads, (sizeof(T) == 4 && VEC == 4 && MAXF <= 3) ? 4 : 1)
fv_flux_kernel(const T *__restrict__ f, const T *__restrict__ G, T *__restrict__ L, FvTables<T> tb,
               const int *__restrict__ nface, const int *__restrict__ nb, const int *__restrict__ order, int nv,
               int N, T Lv, T dv) {
    const int64_t i = __ldg(order + (gridDim.x - 1 - blockIdx.x));
    const int k = (blockIdx.y * kFvThreads + threadIdx.x) * VEC;
    if (k >= nv) return;
    const int nf = __ldg(nface + i);
    const Vec<T, VEC> fi = ldv<T, VEC>(f + i * nv + k);
    Vec<T, VEC> gxi, gyi;
    if (kGrad) {
        gxi = ldv<T, VEC>(G + (i * 2) * nv + k);
        gyi = ldv<T, VEC>(G + (i * 2 + 1) * nv + k);
    }
    // every face's neighbour row first
    int jn[MAXF];
    Vec<T, VEC> fj[MAXF], gxj[MAXF], gyj[MAXF];
#pragma unroll
    for (int q = 0; q < MAXF; ++q) {
        jn[q] = q < nf ? __ldg(nb + i * kFvMaxFaces + q) : -1;
        fj[q] = fi;
        if (kGrad) {
            gxj[q] = gxi;
            gyj[q] = gyi;
        }
        if (jn[q] >= 0) {
            fj[q] = ldv<T, VEC>(f + (int64_t)jn[q] * nv + k);
            if (kGrad) {
                gxj[q] = ldv<T, VEC>(G + ((int64_t)jn[q] * 2) * nv + k);
                gyj[q] = ldv<T, VEC>(G + ((int64_t)jn[q] * 2 + 1) * nv + k);
            }
        }
    }
    // velocities in the working precision; the VEC velocities of a thread lie
    // in one row of the grid (the host takes VEC = 4 only when 4 divides N)
    const int j1 = k / N, j2 = k - j1 * N;
    const T v1 = -Lv + (T)j1 * dv;
    T v2[VEC], acc[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
        v2[u] = -Lv + (T)(j2 + u) * dv;
        acc[u] = (T)0;
    }
#pragma unroll
    for (int q = 0; q < MAXF; ++q) {
        if (q >= nf) continue;
        const int64_t s = i * kFvMaxFaces + q;
        const T nx = __ldg(tb.fn + 2 * s), ny = __ldg(tb.fn + 2 * s + 1);
        T oix = (T)0, oiy = (T)0, ojx = (T)0, ojy = (T)0;
        if (kGrad) {
            oix = __ldg(tb.off_i + 2 * s);
            oiy = __ldg(tb.off_i + 2 * s + 1);
            ojx = __ldg(tb.off_j + 2 * s);
            ojy = __ldg(tb.off_j + 2 * s + 1);
        }
        if constexpr (sizeof(T) == 4 && VEC == 4) {
            // the same face flux on pairs of velocities in FP32x2
            const float2 v1nx = dup2(v1 * nx), hf = dup2(0.5f);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int u = 2 * p;
                const float2 vn = fma2(make_float2(v2[u], v2[u + 1]), dup2(ny), v1nx);
                float2 fl = make_float2(fi.v[u], fi.v[u + 1]);
                if (kGrad)
                    fl = fma2(make_float2(gyi.v[u], gyi.v[u + 1]), dup2(oiy),
                              fma2(make_float2(gxi.v[u], gxi.v[u + 1]), dup2(oix), fl));
                float2 fr = fl;
                if (jn[q] >= 0) {
                    fr = make_float2(fj[q].v[u], fj[q].v[u + 1]);
                    if (kGrad)
                        fr = fma2(make_float2(gyj[q].v[u], gyj[q].v[u + 1]), dup2(ojy),
                                  fma2(make_float2(gxj[q].v[u], gxj[q].v[u + 1]), dup2(ojx), fr));
                }
                const float2 h = mul2(hf, vn), nah = make_float2(-fabsf(h.x), -fabsf(h.y));
                float2 a = make_float2(acc[u], acc[u + 1]);
                a = fma2(h, add2(fl, fr), a);
                a = fma2(nah, add2(fr, neg2(fl)), a);
                acc[u] = a.x;
                acc[u + 1] = a.y;
            }
        } else {
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
                const T vn = v1 * nx + v2[u] * ny;
                T fl = fi.v[u];
                if (kGrad) fl += gxi.v[u] * oix + gyi.v[u] * oiy;
                T fr = fl;
                if (jn[q] >= 0) {
                    fr = fj[q].v[u];
                    if (kGrad) fr += gxj[q].v[u] * ojx + gyj[q].v[u] * ojy;
                }
                acc[u] += (T)0.5 * vn * (fl + fr) - (T)0.5 * fabs(vn) * (fr - fl);
            }
        }
    }
    const T ia = __ldg(tb.inv_area + i);
    Vec<T, VEC> o;
#pragma unroll
    for (int u = 0; u < VEC; ++u) o.v[u] = acc[u] * ia;
    stv<T, VEC>(L + i * nv + k, o);
}

// ---- persistent forms of the two face-value passes --------------------------
// A block takes one of every (SMs x blocks per SM) positions of the
// processing order, walking them in steps of the grid; while it computes one cell, the rows of
// the next one travel into shared memory by cp.async (16 bytes per thread and
// row, each thread copying exactly the slots it reads back, so no block
// barrier is needed and threads past nv leave at once), and the index
// records of the cell after that are already being loaded.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

constexpr int kFaceRows = 6;         // rows staged per cell: f_i and 5 stencil rows / 3 own and 3 neighbour face rows
// blocks per SM: 3 for the reconstruction (85 registers, no spills; 4 spill
// its record prefetch), 4 for the flux pass (64 registers)
constexpr int kFacesCtasPerSm = 3, kFluxCtasPerSm = 4;
constexpr size_t kFaceStageBytes = 2 * kFaceRows * kFvThreads * sizeof(float4);   // 48 KB

// Index record of position p needed by the reconstruction: cell, flags, stencil.
struct RecG {
    int i, ncf, c[kFvCentral];
};
__device__ __forceinline__ RecG rec_g(const int4 *__restrict__ tripos, int64_t p) {
    const int4 a = __ldg(tripos + 3 * p), b = __ldg(tripos + 3 * p + 1), c = __ldg(tripos + 3 * p + 2);
    return RecG{a.x, a.y, {b.x, b.y, b.z, b.w, c.x}};
}

template <int CPS>
__global__ void __launch_bounds__(kFvThreads, CPS)
fv_faces_persist_kernel(const float *__restrict__ f, float *__restrict__ FV, FvTables<float> tb,
                        const int *__restrict__ cen, const int *__restrict__ nsec, const int *__restrict__ sec,
                        const int4 *__restrict__ tripos, int64_t n, int nv) {
    extern __shared__ float4 stage[];            // [2][kFaceRows][kFvThreads]
    const int t = threadIdx.x;
    const int k = (blockIdx.y * kFvThreads + t) * 4;
    if (k >= nv || (int64_t)blockIdx.x >= n) return;
    const int64_t G = gridDim.x;
    auto issue = [&](const RecG &r, int buf) {
        float4 *sl = stage + buf * kFaceRows * kFvThreads + t;
        cp_async16(sl, f + (int64_t)r.i * nv + k);
#pragma unroll
        for (int q = 0; q < kFvCentral; ++q) cp_async16(sl + (q + 1) * kFvThreads, f + (int64_t)r.c[q] * nv + k);
    };
    int64_t p = blockIdx.x;
    RecG cur = rec_g(tripos, p);
    issue(cur, 0);
    cp_async_commit();
    RecG nxt = cur;
    if (p + G < n) nxt = rec_g(tripos, p + G);
    for (int it = 0;; ++it) {
        const bool more = p + G < n;
        if (more) issue(nxt, (it + 1) & 1);
        cp_async_commit();
        RecG nn = nxt;
        if (p + 2 * G < n) nn = rec_g(tripos, p + 2 * G);
        cp_async_wait_prev();
        const float4 *sl = stage + (it & 1) * kFaceRows * kFvThreads + t;
        const float4 fi = sl[0];
        if (cur.ncf & kFvRegularTri) {
            float4 fr[kFvCentral];
#pragma unroll
            for (int q = 0; q < kFvCentral; ++q) fr[q] = sl[(q + 1) * kFvThreads];
            tri_x2_rows<true>(FV, tb, fr, cur.i, k, nv, fi);
        } else {
            Vec<float, 4> fv;
            fv.v[0] = fi.x; fv.v[1] = fi.y; fv.v[2] = fi.z; fv.v[3] = fi.w;
            gradient_generic<float, 4, 3, true>(f, FV, tb, cen, nsec, sec, cur.i, cur.ncf, k, nv, fv);
        }
        if (!more) break;
        p += G;
        cur = nxt;
        nxt = nn;
    }
}

// Index record of position p needed by the flux pass: cell, neighbours, their face indices.
struct RecF {
    int i, qbits, nb[3];
};
__device__ __forceinline__ RecF rec_f(const int4 *__restrict__ tripos, int64_t p) {
    const int4 a = __ldg(tripos + 3 * p), c = __ldg(tripos + 3 * p + 2);
    return RecF{a.x, a.w, {c.y, c.z, c.w}};
}

__global__ void __launch_bounds__(kFvThreads, kFluxCtasPerSm)
fv_flux_faces_persist_kernel(const float *__restrict__ FV, float *__restrict__ L, FvTables<float> tb,
                             const int4 *__restrict__ tripos, int64_t n, int nv, int N, float Lv, float dv) {
    extern __shared__ float4 stage[];            // [2][kFaceRows][kFvThreads]
    const int t = threadIdx.x;
    const int k = (blockIdx.y * kFvThreads + t) * 4;
    if (k >= nv || (int64_t)blockIdx.x >= n) return;
    const int64_t G = gridDim.x;
    // positions from the end of the order (the rows the reconstruction wrote last are still in L2)
    auto pos = [&](int64_t p) { return n - 1 - p; };
    auto issue = [&](const RecF &r, int buf) {
        float4 *sl = stage + buf * kFaceRows * kFvThreads + t;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            cp_async16(sl + q * kFvThreads, FV + ((int64_t)r.i * 3 + q) * nv + k);
            if (r.nb[q] >= 0)
                cp_async16(sl + (3 + q) * kFvThreads, FV + ((int64_t)r.nb[q] * 3 + ((r.qbits >> (2 * q)) & 3)) * nv + k);
        }
    };
    const int j1 = k / N, j2 = k - j1 * N;
    const float v1 = -Lv + (float)j1 * dv;
    float2 v2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) v2[h] = make_float2(-Lv + (float)(j2 + 2 * h) * dv, -Lv + (float)(j2 + 2 * h + 1) * dv);
    const float2 hf = dup2(0.5f);
    int64_t p = blockIdx.x;
    RecF cur = rec_f(tripos, pos(p));
    issue(cur, 0);
    cp_async_commit();
    RecF nxt = cur;
    if (p + G < n) nxt = rec_f(tripos, pos(p + G));
    for (int it = 0;; ++it) {
        const bool more = p + G < n;
        if (more) issue(nxt, (it + 1) & 1);
        cp_async_commit();
        RecF nn = nxt;
        if (p + 2 * G < n) nn = rec_f(tripos, pos(p + 2 * G));
        cp_async_wait_prev();
        const float4 *sl = stage + (it & 1) * kFaceRows * kFvThreads + t;
        const int64_t i = cur.i;
        float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 fl = sl[q * kFvThreads];
            const float4 fr = cur.nb[q] >= 0 ? sl[(3 + q) * kFvThreads] : fl;
            const int64_t s = i * kFvMaxFaces + q;
            const float nx = __ldg(tb.fn + 2 * s), ny = __ldg(tb.fn + 2 * s + 1);
            const float2 v1nx = dup2(v1 * nx);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 a = h == 0 ? lo2(fl) : hi2(fl), b = h == 0 ? lo2(fr) : hi2(fr);
                const float2 vn = fma2(v2[h], dup2(ny), v1nx);
                const float2 hv = mul2(hf, vn), nah = make_float2(-fabsf(hv.x), -fabsf(hv.y));
                acc[h] = fma2(hv, add2(a, b), acc[h]);
                acc[h] = fma2(nah, add2(b, neg2(a)), acc[h]);
            }
        }
        const float2 ia = dup2(__ldg(tb.inv_area + i));
        const float2 o0 = mul2(acc[0], ia), o1 = mul2(acc[1], ia);
        *reinterpret_cast<float4 *>(L + i * nv + k) = make_float4(o0.x, o0.y, o1.x, o1.y);
        if (!more) break;
        p += G;
        cur = nxt;
        nxt = nn;
    }
}

// Flux pass of a mesh with walls (full accommodation, eq. BOU with alpha = 1,
// eq. MAXB, eq. MU): one CTA holds all nv <= 1024 velocities of its cell, 4
// per thread, so the wall density mu of a face -- the ratio of the outgoing
// mass flux sum_{v.n > 0} f_L v.n to the incoming flux of the unit wall
// Maxwellian sum_{v.n < 0} M_w |v.n| -- is a block reduction (FP64, fixed
// order).  Velocities entering the domain through the wall carry mu M_w(v),
// the others the reconstructed inner value; other faces as in fv_flux_kernel.
template <typename T, bool VLOAD>
__device__ __forceinline__ Vec<T, 4> ld4(const T *__restrict__ p) {
    if constexpr (VLOAD) {
        return ldv<T, 4>(p);
    } else {
        Vec<T, 4> r;
#pragma unroll
        for (int u = 0; u < 4; ++u) r.v[u] = p[u];
        return r;
    }
}

template <typename T, bool kGrad, int MAXF, bool VLOAD>
__global__ void __launch_bounds__(kFvThreads)
fv_flux_wall_kernel(const T *__restrict__ f, const T *__restrict__ G, T *__restrict__ L, FvTables<T> tb,
                    const int *__restrict__ nface, const int *__restrict__ nb, const int *__restrict__ order,
                    const int *__restrict__ wall, const T *__restrict__ wallp, int nv, int N, T Lv, T dv) {
    __shared__ double red[2 * (kFvThreads / 32)];
    const int64_t i = __ldg(order + (gridDim.x - 1 - blockIdx.x));
    const int kt = threadIdx.x * 4;
    const bool act = kt < nv;
    const int k = act ? kt : 0;                  // idle threads read row 0 and store nothing
    const int nf = __ldg(nface + i);
    const Vec<T, 4> fi = ld4<T, VLOAD>(f + i * nv + k);
    Vec<T, 4> gxi, gyi;
    if (kGrad) {
        gxi = ld4<T, VLOAD>(G + (i * 2) * nv + k);
        gyi = ld4<T, VLOAD>(G + (i * 2 + 1) * nv + k);
    }
    int jn[MAXF];
    Vec<T, 4> fj[MAXF], gxj[MAXF], gyj[MAXF];
#pragma unroll
    for (int q = 0; q < MAXF; ++q) {
        jn[q] = q < nf ? __ldg(nb + i * kFvMaxFaces + q) : -1;
        fj[q] = fi;
        if (kGrad) {
            gxj[q] = gxi;
            gyj[q] = gyi;
        }
        if (jn[q] >= 0) {
            fj[q] = ld4<T, VLOAD>(f + (int64_t)jn[q] * nv + k);
            if (kGrad) {
                gxj[q] = ld4<T, VLOAD>(G + ((int64_t)jn[q] * 2) * nv + k);
                gyj[q] = ld4<T, VLOAD>(G + ((int64_t)jn[q] * 2 + 1) * nv + k);
            }
        }
    }
    const int j1 = k / N, j2 = k - j1 * N;
    const T v1 = -Lv + (T)j1 * dv;
    T v2[4], acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        v2[u] = -Lv + (T)(j2 + u) * dv;
        acc[u] = (T)0;
    }
#pragma unroll
    for (int q = 0; q < MAXF; ++q) {
        if (q >= nf) continue;                   // uniform over the CTA (one cell)
        const int64_t s = i * kFvMaxFaces + q;
        const T nx = __ldg(tb.fn + 2 * s), ny = __ldg(tb.fn + 2 * s + 1);
        T oix = (T)0, oiy = (T)0, ojx = (T)0, ojy = (T)0;
        if (kGrad) {
            oix = __ldg(tb.off_i + 2 * s);
            oiy = __ldg(tb.off_i + 2 * s + 1);
            ojx = __ldg(tb.off_j + 2 * s);
            ojy = __ldg(tb.off_j + 2 * s + 1);
        }
        T vn[4], fl[4], fr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            vn[u] = v1 * nx + v2[u] * ny;
            fl[u] = fi.v[u];
            if (kGrad) fl[u] += gxi.v[u] * oix + gyi.v[u] * oiy;
            fr[u] = fl[u];
            if (jn[q] >= 0) {
                fr[u] = fj[q].v[u];
                if (kGrad) fr[u] += gxj[q].v[u] * ojx + gyj[q].v[u] * ojy;
            }
        }
        const int w = jn[q] < 0 ? __ldg(wall + s) : -1;      // uniform over the CTA
        if (w >= 0) {
            const T th = __ldg(wallp + 3 * w), uw1 = __ldg(wallp + 3 * w + 1), uw2 = __ldg(wallp + 3 * w + 2);
            const T inv2th = (T)0.5 / th, norm = (T)(0.15915494309189535) / th;   // 1 / (2 pi theta)
            T mw[4];
            double num = 0.0, den = 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T d1 = v1 - uw1, d2 = v2[u] - uw2;
                mw[u] = norm * exp(-(d1 * d1 + d2 * d2) * inv2th);
                if (act && vn[u] > (T)0) num += (double)(fl[u] * vn[u]);
                if (act && vn[u] < (T)0) den += (double)(mw[u] * -vn[u]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                num += __shfl_xor_sync(0xffffffffu, num, o);
                den += __shfl_xor_sync(0xffffffffu, den, o);
            }
            __syncthreads();                     // red is reused face after face
            if ((threadIdx.x & 31) == 0) {
                red[2 * (threadIdx.x >> 5)] = num;
                red[2 * (threadIdx.x >> 5) + 1] = den;
            }
            __syncthreads();
            num = den = 0.0;
#pragma unroll
            for (int q2 = 0; q2 < kFvThreads / 32; ++q2) {
                num += red[2 * q2];
                den += red[2 * q2 + 1];
            }
            const T mu = (T)(num / den);
#pragma unroll
            for (int u = 0; u < 4; ++u) fr[u] = vn[u] > (T)0 ? fl[u] : mu * mw[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += (T)0.5 * vn[u] * (fl[u] + fr[u]) - (T)0.5 * fabs(vn[u]) * (fr[u] - fl[u]);
    }
    if (act) {
        const T ia = __ldg(tb.inv_area + i);
#pragma unroll
        for (int u = 0; u < 4; ++u) L[i * nv + k + u] = acc[u] * ia;
    }
}


// ---- degree 2 (order 3) -----------------------------------------------------
// Coefficients of the CWENO polynomial of degree 2 per (cell, velocity) in the
// zero-mean scaled Taylor basis phi = (xi, eta, xi^2 - mu20, xi eta - mu11,
// eta^2 - mu02), xi = (x - x_b)/h: p_opt from the least-squares rows over the
// cell's 11 nearest cells, the degree-1 sector polynomials (coefficients of
// xi and eta only), p_0 = (p_opt - lambda_L sum_L p_L) / lambda_0, and the
// weights lambda_s / (sigma_s + eps)^4 in the same ratio form as degree 1,
// sigma_s the cell mean of |h grad p|^2 plus the squared scaled second
// derivatives (for the linear sectors: |h grad p|^2).  VEC velocities per
// thread (4 on triangle meshes with aligned rows: the table entries, uniform
// over the CTA, are then loaded once per 4 velocities); C is [cell][5][nv].
// Degree-2 coefficients of the 4 velocities k..k+3 of a flagged triangle in
// FP32x2 (its 11-cell stencil starts with the face neighbours; sector s joins
// faces s and s + 1 mod 3): the steps of the generic kernel below, each
// neighbour row loaded once.
__device__ __forceinline__ void coef3_tri_x2(const float *__restrict__ f, float *__restrict__ C,
                                             const FvTables<float> &tb, const FvTables3<float> &t3,
                                             const int *__restrict__ cen, int64_t i, int k, int nv, const float4 fi) {
    constexpr float kInvLam0 = (float)(4.0 / 3.0), kLam0 = 0.75f, kEps = 1e-14f;
    const float lamL = 0.25f / 3.0f;
    const float2 nf[2] = {neg2(lo2(fi)), neg2(hi2(fi))};
    const float *Rc = t3.Rc + i * kFvCoef3 * kFvCentral3;
    float2 c[kFvCoef3][2], dface[3][2];
#pragma unroll
    for (int q = 0; q < kFvCentral3; ++q) {
        const int j = __ldg(cen + i * kFvCentral3 + q);
        const float4 r = *reinterpret_cast<const float4 *>(f + (int64_t)j * nv + k);
        const float2 d0 = add2(lo2(r), nf[0]), d1 = add2(hi2(r), nf[1]);
        if (q < 3) {
            dface[q][0] = d0;
            dface[q][1] = d1;
        }
#pragma unroll
        for (int l = 0; l < kFvCoef3; ++l) {
            const float2 R = dup2(__ldg(Rc + l * kFvCentral3 + q));
            c[l][0] = q == 0 ? mul2(R, d0) : fma2(R, d0, c[l][0]);
            c[l][1] = q == 0 ? mul2(R, d1) : fma2(R, d1, c[l][1]);
        }
    }
    float2 sx[3][2], sy[3][2];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const float4 R = __ldg(reinterpret_cast<const float4 *>(tb.Rs + (i * kFvMaxFaces + s) * 4));
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float2 da = dface[s][p], db = dface[(s + 1) % 3][p];
            sx[s][p] = fma2(dup2(R.x), da, mul2(dup2(R.y), db));
            sy[s][p] = fma2(dup2(R.z), da, mul2(dup2(R.w), db));
        }
    }
    const float m20 = __ldg(t3.mu + 3 * i), m11 = __ldg(t3.mu + 3 * i + 1), m02 = __ldg(t3.mu + 3 * i + 2);
    // smoothness of the central polynomial: sum of its squared derivatives
    // over the scaled cell, a quadratic form in p0 with these coefficients
    const float2 A22 = dup2(4.f * m20 + 4.f), A33 = dup2(m02 + m20 + 1.f), A44 = dup2(4.f * m02 + 4.f);
    const float2 A23 = dup2(4.f * m11), E = dup2(kEps);
    float2 out[kFvCoef3][2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float2 sumx = add2(add2(sx[0][p], sx[1][p]), sx[2][p]), sumy = add2(add2(sy[0][p], sy[1][p]), sy[2][p]);
        float2 p0[kFvCoef3];
        p0[0] = mul2(fma2(dup2(-lamL), sumx, c[0][p]), dup2(kInvLam0));
        p0[1] = mul2(fma2(dup2(-lamL), sumy, c[1][p]), dup2(kInvLam0));
#pragma unroll
        for (int l = 2; l < kFvCoef3; ++l) p0[l] = mul2(c[l][p], dup2(kInvLam0));
        float2 sig0 = fma2(p0[0], p0[0], mul2(p0[1], p0[1]));
        sig0 = fma2(mul2(A22, p0[2]), p0[2], sig0);
        sig0 = fma2(mul2(A33, p0[3]), p0[3], sig0);
        sig0 = fma2(mul2(A44, p0[4]), p0[4], sig0);
        sig0 = fma2(mul2(A23, p0[2]), p0[3], sig0);
        sig0 = fma2(mul2(A23, p0[3]), p0[4], sig0);
        float2 sig[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) sig[s] = fma2(sx[s][p], sx[s][p], mul2(sy[s][p], sy[s][p]));
        const float2 smin = make_float2(fminf(fminf(sig0.x, sig[0].x), fminf(sig[1].x, sig[2].x)),
                                        fminf(fminf(sig0.y, sig[0].y), fminf(sig[1].y, sig[2].y)));
        const float2 num = add2(smin, E);
        float2 r = mul2(num, rcp2(add2(sig0, E)));
        r = mul2(r, r);
        float2 w = mul2(dup2(kLam0), mul2(r, r));
        float2 wsum = w, acc[kFvCoef3];
#pragma unroll
        for (int l = 0; l < kFvCoef3; ++l) acc[l] = mul2(w, p0[l]);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            r = mul2(num, rcp2(add2(sig[s], E)));
            r = mul2(r, r);
            w = mul2(dup2(lamL), mul2(r, r));
            wsum = add2(wsum, w);
            acc[0] = fma2(w, sx[s][p], acc[0]);
            acc[1] = fma2(w, sy[s][p], acc[1]);
        }
        const float2 iw = rcp2(wsum);
#pragma unroll
        for (int l = 0; l < kFvCoef3; ++l) out[l][p] = mul2(acc[l], iw);
    }
#pragma unroll
    for (int l = 0; l < kFvCoef3; ++l)
        *reinterpret_cast<float4 *>(C + (i * kFvCoef3 + l) * nv + k) =
            make_float4(out[l][0].x, out[l][0].y, out[l][1].x, out[l][1].y);
}

template <typename T, int VEC, int MAXS>
__device__ __forceinline__ void coef3_body(const T *__restrict__ f, T *__restrict__ C, const FvTables<T> &tb,
                                           const FvTables3<T> &t3, const int *__restrict__ ncen,
                                           const int *__restrict__ cen, const int *__restrict__ nsec,
                                           const int *__restrict__ sec, const int *__restrict__ order, int nv) {
    const int64_t i = __ldg(order + blockIdx.x);
    const int k = (blockIdx.y * kFvThreads + threadIdx.x) * VEC;
    if (k >= nv) return;
    const Vec<T, VEC> fi = ldv<T, VEC>(f + i * nv + k);
    const int ncf = __ldg(ncen + i);
    if constexpr (sizeof(T) == 4 && VEC == 4 && MAXS == 3) {
        if (ncf & kFvRegularTri) {      // uniform over the block: one cell per block
            coef3_tri_x2(f, C, tb, t3, cen, i, k, nv, make_float4(fi.v[0], fi.v[1], fi.v[2], fi.v[3]));
            return;
        }
    }
    T c[kFvCoef3][VEC];
#pragma unroll
    for (int l = 0; l < kFvCoef3; ++l)
#pragma unroll
        for (int u = 0; u < VEC; ++u) c[l][u] = (T)0;
    const int nc = ncf & (kFvRegularTri - 1);
    const T *Rc = t3.Rc + i * kFvCoef3 * kFvCentral3;
#pragma unroll
    for (int q = 0; q < kFvCentral3; ++q) {
        if (q < nc) {
            const int j = __ldg(cen + i * kFvCentral3 + q);
            const Vec<T, VEC> fj = ldv<T, VEC>(f + (int64_t)j * nv + k);
#pragma unroll
            for (int l = 0; l < kFvCoef3; ++l) {
                const T r = __ldg(Rc + l * kFvCentral3 + q);
#pragma unroll
                for (int u = 0; u < VEC; ++u) c[l][u] += r * (fj.v[u] - fi.v[u]);
            }
        }
    }
    const int ns = __ldg(nsec + i);
    if (ns > 0) {
        constexpr T kInvLam0 = (T)(4.0 / 3.0), kLam0 = (T)0.75, kEps = (T)1e-14;
        const T lamL = (T)0.25 / (T)ns;
        T sx[MAXS][VEC], sy[MAXS][VEC];
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
#pragma unroll
            for (int u = 0; u < VEC; ++u) sx[s][u] = sy[s][u] = (T)0;
            if (s < ns) {
                const int a = __ldg(sec + (i * kFvMaxFaces + s) * 2), b = __ldg(sec + (i * kFvMaxFaces + s) * 2 + 1);
                const T *R = tb.Rs + (i * kFvMaxFaces + s) * 4;
                const T r0 = __ldg(R), r1 = __ldg(R + 1), r2 = __ldg(R + 2), r3 = __ldg(R + 3);
                const Vec<T, VEC> fa = ldv<T, VEC>(f + (int64_t)a * nv + k), fb = ldv<T, VEC>(f + (int64_t)b * nv + k);
#pragma unroll
                for (int u = 0; u < VEC; ++u) {
                    const T da = fa.v[u] - fi.v[u], db = fb.v[u] - fi.v[u];
                    sx[s][u] = r0 * da + r1 * db;
                    sy[s][u] = r2 * da + r3 * db;
                }
            }
        }
        const T m20 = __ldg(t3.mu + 3 * i), m11 = __ldg(t3.mu + 3 * i + 1), m02 = __ldg(t3.mu + 3 * i + 2);
        auto ratio = [](T a, T b) {
            if constexpr (sizeof(T) == 4) return __fdividef(a, b);
            else return a / b;
        };
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
            T sumx = (T)0, sumy = (T)0;
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                sumx += sx[s][u];
                sumy += sy[s][u];
            }
            T p0[kFvCoef3];
            p0[0] = (c[0][u] - lamL * sumx) * kInvLam0;
            p0[1] = (c[1][u] - lamL * sumy) * kInvLam0;
#pragma unroll
            for (int l = 2; l < kFvCoef3; ++l) p0[l] = c[l][u] * kInvLam0;
            const T sig0 = p0[0] * p0[0] + p0[1] * p0[1] + (T)4 * p0[2] * p0[2] * m20 + (T)4 * p0[2] * p0[3] * m11 +
                           p0[3] * p0[3] * m02 + p0[3] * p0[3] * m20 + (T)4 * p0[3] * p0[4] * m11 +
                           (T)4 * p0[4] * p0[4] * m02 + (T)4 * p0[2] * p0[2] + p0[3] * p0[3] + (T)4 * p0[4] * p0[4];
            T sig[MAXS], smin = sig0;
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                sig[s] = sx[s][u] * sx[s][u] + sy[s][u] * sy[s][u];
                if (s < ns) smin = fmin(smin, sig[s]);
            }
            const T num = smin + kEps;
            T r = ratio(num, sig0 + kEps);
            r = r * r;
            T w = kLam0 * (r * r);
            T wsum = w, acc[kFvCoef3];
#pragma unroll
            for (int l = 0; l < kFvCoef3; ++l) acc[l] = w * p0[l];
#pragma unroll
            for (int s = 0; s < MAXS; ++s)
                if (s < ns) {
                    r = ratio(num, sig[s] + kEps);
                    r = r * r;
                    w = lamL * (r * r);
                    wsum += w;
                    acc[0] += w * sx[s][u];
                    acc[1] += w * sy[s][u];
                }
            const T iw = (T)1 / wsum;
#pragma unroll
            for (int l = 0; l < kFvCoef3; ++l) c[l][u] = acc[l] * iw;
        }
    }
#pragma unroll
    for (int l = 0; l < kFvCoef3; ++l) {
        Vec<T, VEC> o;
#pragma unroll
        for (int u = 0; u < VEC; ++u) o.v[u] = c[l][u];
        stv<T, VEC>(C + (i * kFvCoef3 + l) * nv + k, o);
    }
}

template <typename T, int VEC, int MAXS>
__global__ void __launch_bounds__(kFvThreads)
fv_coef3_kernel(const T *__restrict__ f, T *__restrict__ C, FvTables<T> tb, FvTables3<T> t3,
                const int *__restrict__ ncen, const int *__restrict__ cen, const int *__restrict__ nsec,
                const int *__restrict__ sec, const int *__restrict__ order, int nv) {
    coef3_body<T, VEC, MAXS>(f, C, tb, t3, ncen, cen, nsec, sec, order, nv);
}

// FP32 triangles, 4 velocities per thread: four blocks per SM (64 registers;
// measured 0.194 -> 0.180 ms on 19802 cells x 32^2 against three).  A bound
// on the template above would also change the register allocation of its
// other instantiations.
__global__ void __launch_bounds__(kFvThreads, 4)
fv_coef3_tri_kernel(const float *__restrict__ f, float *__restrict__ C, FvTables<float> tb, FvTables3<float> t3,
                    const int *__restrict__ ncen, const int *__restrict__ cen, const int *__restrict__ nsec,
                    const int *__restrict__ sec, const int *__restrict__ order, int nv) {
    coef3_body<float, 4, 3>(f, C, tb, t3, ncen, cen, nsec, sec, order, nv);
}

// Flux pass of degree 2: the reconstruction on both sides at the face's two
// Gauss-Legendre points (weights 1/2), the Rusanov flux at each; transmissive
// boundary faces take f_R = f_L.  VEC velocities of one grid row per thread
// (the host takes VEC = 4 only when 4 divides N).
template <typename T, int VEC, int MAXF>
__global__ void __launch_bounds__(kFvThreads, (sizeof(T) == 4 && VEC == 4 && MAXF <= 3) ? 3 : 1)
fv_flux3_kernel(const T *__restrict__ f, const T *__restrict__ C, T *__restrict__ L, FvTables<T> tb,
                FvTables3<T> t3, const int *__restrict__ nface, const int *__restrict__ nb,
                const int *__restrict__ order, int nv, int N, T Lv, T dv) {
    const int64_t i = __ldg(order + (gridDim.x - 1 - blockIdx.x));
    const int k = (blockIdx.y * kFvThreads + threadIdx.x) * VEC;
    if (k >= nv) return;
    const int nf = __ldg(nface + i);
    const Vec<T, VEC> fi = ldv<T, VEC>(f + i * nv + k);
    Vec<T, VEC> ci[kFvCoef3];
#pragma unroll
    for (int l = 0; l < kFvCoef3; ++l) ci[l] = ldv<T, VEC>(C + (i * kFvCoef3 + l) * nv + k);
    const int j1 = k / N, j2 = k - j1 * N;
    const T v1 = -Lv + (T)j1 * dv;
    T v2[VEC], acc[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
        v2[u] = -Lv + (T)(j2 + u) * dv;
        acc[u] = (T)0;
    }
#pragma unroll
    for (int q = 0; q < MAXF; ++q) {
        if (q >= nf) continue;
        const int64_t s = i * kFvMaxFaces + q;
        const T nx = __ldg(tb.fn + 2 * s), ny = __ldg(tb.fn + 2 * s + 1);
        const int jn = __ldg(nb + s);
        Vec<T, VEC> fj = fi, cj[kFvCoef3];
#pragma unroll
        for (int l = 0; l < kFvCoef3; ++l) cj[l] = ci[l];
        if (jn >= 0) {
            fj = ldv<T, VEC>(f + (int64_t)jn * nv + k);
#pragma unroll
            for (int l = 0; l < kFvCoef3; ++l) cj[l] = ldv<T, VEC>(C + ((int64_t)jn * kFvCoef3 + l) * nv + k);
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            T pi[kFvCoef3], pj[kFvCoef3];
#pragma unroll
            for (int l = 0; l < kFvCoef3; ++l) {
                pi[l] = __ldg(t3.phi_i + (s * 2 + g) * kFvCoef3 + l);
                pj[l] = jn >= 0 ? __ldg(t3.phi_j + (s * 2 + g) * kFvCoef3 + l) : (T)0;
            }
            if constexpr (sizeof(T) == 4 && VEC == 4) {
                // the same Gauss-point flux on pairs of velocities in FP32x2
                const float2 v1nx = dup2(v1 * nx), qf = dup2(0.25f);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int u = 2 * h;
                    float2 fl = make_float2(fi.v[u], fi.v[u + 1]);
#pragma unroll
                    for (int l = 0; l < kFvCoef3; ++l) fl = fma2(make_float2(ci[l].v[u], ci[l].v[u + 1]), dup2(pi[l]), fl);
                    float2 fr = fl;
                    if (jn >= 0) {
                        fr = make_float2(fj.v[u], fj.v[u + 1]);
#pragma unroll
                        for (int l = 0; l < kFvCoef3; ++l)
                            fr = fma2(make_float2(cj[l].v[u], cj[l].v[u + 1]), dup2(pj[l]), fr);
                    }
                    const float2 vn = fma2(make_float2(v2[u], v2[u + 1]), dup2(ny), v1nx);
                    const float2 hv = mul2(qf, vn), nah = make_float2(-fabsf(hv.x), -fabsf(hv.y));
                    float2 a = make_float2(acc[u], acc[u + 1]);
                    a = fma2(hv, add2(fl, fr), a);
                    a = fma2(nah, add2(fr, neg2(fl)), a);
                    acc[u] = a.x;
                    acc[u + 1] = a.y;
                }
            } else {
#pragma unroll
                for (int u = 0; u < VEC; ++u) {
                    T fl = fi.v[u];
#pragma unroll
                    for (int l = 0; l < kFvCoef3; ++l) fl += ci[l].v[u] * pi[l];
                    T fr = fl;
                    if (jn >= 0) {
                        fr = fj.v[u];
#pragma unroll
                        for (int l = 0; l < kFvCoef3; ++l) fr += cj[l].v[u] * pj[l];
                    }
                    const T vn = v1 * nx + v2[u] * ny;
                    acc[u] += (T)0.25 * (vn * (fl + fr) - fabs(vn) * (fr - fl));
                }
            }
        }
    }
    const T ia = __ldg(tb.inv_area + i);
    Vec<T, VEC> o;
#pragma unroll
    for (int u = 0; u < VEC; ++u) o.v[u] = acc[u] * ia;
    stv<T, VEC>(L + i * nv + k, o);
}


// Flux pass of degree 2 on a mesh with walls: as fv_flux_wall_kernel (one CTA
// per cell, 4 velocities per thread, nv <= 1024), with the reconstruction at
// the two Gauss points of every face; at a wall face the mass balance of
// eq. MU holds at each Gauss point, so one block reduction forms the two
// outgoing fluxes and the wall Maxwellian's incoming flux together.
template <typename T, int MAXF, bool VLOAD>
__global__ void __launch_bounds__(kFvThreads)
fv_flux3_wall_kernel(const T *__restrict__ f, const T *__restrict__ C, T *__restrict__ L, FvTables<T> tb,
                     FvTables3<T> t3, const int *__restrict__ nface, const int *__restrict__ nb,
                     const int *__restrict__ order, const int *__restrict__ wall, const T *__restrict__ wallp, int nv,
                     int N, T Lv, T dv) {
    __shared__ double red[3 * (kFvThreads / 32)];
    const int64_t i = __ldg(order + (gridDim.x - 1 - blockIdx.x));
    const int kt = threadIdx.x * 4;
    const bool act = kt < nv;
    const int k = act ? kt : 0;                  // idle threads read row 0 and store nothing
    const int nf = __ldg(nface + i);
    const Vec<T, 4> fi = ld4<T, VLOAD>(f + i * nv + k);
    Vec<T, 4> ci[kFvCoef3];
#pragma unroll
    for (int l = 0; l < kFvCoef3; ++l) ci[l] = ld4<T, VLOAD>(C + (i * kFvCoef3 + l) * nv + k);
    const int j1 = k / N, j2 = k - j1 * N;
    const T v1 = -Lv + (T)j1 * dv;
    T v2[4], acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        v2[u] = -Lv + (T)(j2 + u) * dv;
        acc[u] = (T)0;
    }
#pragma unroll
    for (int q = 0; q < MAXF; ++q) {
        if (q >= nf) continue;                   // uniform over the CTA (one cell)
        const int64_t s = i * kFvMaxFaces + q;
        const T nx = __ldg(tb.fn + 2 * s), ny = __ldg(tb.fn + 2 * s + 1);
        const int jn = __ldg(nb + s);
        Vec<T, 4> fj = fi, cj[kFvCoef3];
#pragma unroll
        for (int l = 0; l < kFvCoef3; ++l) cj[l] = ci[l];
        if (jn >= 0) {
            fj = ld4<T, VLOAD>(f + (int64_t)jn * nv + k);
#pragma unroll
            for (int l = 0; l < kFvCoef3; ++l) cj[l] = ld4<T, VLOAD>(C + ((int64_t)jn * kFvCoef3 + l) * nv + k);
        }
        T vn[4], fl[2][4], fr[2][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) vn[u] = v1 * nx + v2[u] * ny;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            T pi[kFvCoef3], pj[kFvCoef3];
#pragma unroll
            for (int l = 0; l < kFvCoef3; ++l) {
                pi[l] = __ldg(t3.phi_i + (s * 2 + g) * kFvCoef3 + l);
                pj[l] = jn >= 0 ? __ldg(t3.phi_j + (s * 2 + g) * kFvCoef3 + l) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                T a = fi.v[u];
#pragma unroll
                for (int l = 0; l < kFvCoef3; ++l) a += ci[l].v[u] * pi[l];
                fl[g][u] = a;
                T b = a;
                if (jn >= 0) {
                    b = fj.v[u];
#pragma unroll
                    for (int l = 0; l < kFvCoef3; ++l) b += cj[l].v[u] * pj[l];
                }
                fr[g][u] = b;
            }
        }
        const int w = jn < 0 ? __ldg(wall + s) : -1;         // uniform over the CTA
        if (w >= 0) {
            const T th = __ldg(wallp + 3 * w), uw1 = __ldg(wallp + 3 * w + 1), uw2 = __ldg(wallp + 3 * w + 2);
            const T inv2th = (T)0.5 / th, norm = (T)(0.15915494309189535) / th;   // 1 / (2 pi theta)
            T mw[4];
            double num0 = 0.0, num1 = 0.0, den = 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T d1 = v1 - uw1, d2 = v2[u] - uw2;
                mw[u] = norm * exp(-(d1 * d1 + d2 * d2) * inv2th);
                if (act && vn[u] > (T)0) {
                    num0 += (double)(fl[0][u] * vn[u]);
                    num1 += (double)(fl[1][u] * vn[u]);
                }
                if (act && vn[u] < (T)0) den += (double)(mw[u] * -vn[u]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                num0 += __shfl_xor_sync(0xffffffffu, num0, o);
                num1 += __shfl_xor_sync(0xffffffffu, num1, o);
                den += __shfl_xor_sync(0xffffffffu, den, o);
            }
            __syncthreads();                     // red is reused face after face
            if ((threadIdx.x & 31) == 0) {
                red[3 * (threadIdx.x >> 5)] = num0;
                red[3 * (threadIdx.x >> 5) + 1] = num1;
                red[3 * (threadIdx.x >> 5) + 2] = den;
            }
            __syncthreads();
            num0 = num1 = den = 0.0;
#pragma unroll
            for (int q2 = 0; q2 < kFvThreads / 32; ++q2) {
                num0 += red[3 * q2];
                num1 += red[3 * q2 + 1];
                den += red[3 * q2 + 2];
            }
            const T mu0 = (T)(num0 / den), mu1 = (T)(num1 / den);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                fr[0][u] = vn[u] > (T)0 ? fl[0][u] : mu0 * mw[u];
                fr[1][u] = vn[u] > (T)0 ? fl[1][u] : mu1 * mw[u];
            }
        }
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                acc[u] += (T)0.25 * (vn[u] * (fl[g][u] + fr[g][u]) - fabs(vn[u]) * (fr[g][u] - fl[g][u]));
    }
    if (act) {
        const T ia = __ldg(tb.inv_area + i);
#pragma unroll
        for (int u = 0; u < 4; ++u) L[i * nv + k + u] = acc[u] * ia;
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

template <typename T> const FvTables<T> &pick(const bz_mesh *m);
template <> const FvTables<double> &pick<double>(const bz_mesh *m) { return m->t64; }
template <> const FvTables<float> &pick<float>(const bz_mesh *m) { return m->t32; }
template <typename T> const FvTables3<T> &pick3(const bz_mesh *m);
template <> const FvTables3<double> &pick3<double>(const bz_mesh *m) { return m->u64; }
template <> const FvTables3<float> &pick3<float>(const bz_mesh *m) { return m->u32; }

template <typename T>
cudaError_t coef3(const bz_mesh *m, const GridView &g, const T *f, T *C, cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    const int nv = (int)g.nv;
    const bool v4 = m->max_faces <= 3 && nv % 4 == 0 && aligned16(f) && aligned16(C);
    const int vec = v4 ? 4 : 1;
    const dim3 grid((unsigned)m->n_cells, (unsigned)((nv / vec + kFvThreads - 1) / kFvThreads));
    if constexpr (sizeof(T) == 4) {
        if (v4) {
            fv_coef3_tri_kernel<<<grid, kFvThreads, 0, st>>>(f, C, pick<T>(m), pick3<T>(m), m->d_ncen3, m->d_cen3,
                                                             m->d_nsec, m->d_sec, m->d_order, nv);
            return cudaGetLastError();
        }
    }
    if (v4)
        fv_coef3_kernel<T, 4, 3><<<grid, kFvThreads, 0, st>>>(f, C, pick<T>(m), pick3<T>(m), m->d_ncen3, m->d_cen3,
                                                               m->d_nsec, m->d_sec, m->d_order, nv);
    else if (m->max_faces <= 3)
        fv_coef3_kernel<T, 1, 3><<<grid, kFvThreads, 0, st>>>(f, C, pick<T>(m), pick3<T>(m), m->d_ncen3, m->d_cen3,
                                                               m->d_nsec, m->d_sec, m->d_order, nv);
    else
        fv_coef3_kernel<T, 1, kFvMaxFaces><<<grid, kFvThreads, 0, st>>>(f, C, pick<T>(m), pick3<T>(m), m->d_ncen3,
                                                                         m->d_cen3, m->d_nsec, m->d_sec, m->d_order,
                                                                         nv);
    return cudaGetLastError();
}

template <typename T>
cudaError_t flux3(const bz_mesh *m, const GridView &g, const T *f, const T *C, T *L, cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    const int nv = (int)g.nv;
    if (m->n_walls > 0) {
        if (!fv_walls_supported(m, g)) return cudaErrorInvalidValue;
        const T *wp = static_cast<const T *>(sizeof(T) == 8 ? static_cast<const void *>(m->d_wall64)
                                                            : static_cast<const void *>(m->d_wall32));
        const bool al = aligned16(f) && aligned16(C) && aligned16(L);
        const unsigned grid = (unsigned)m->n_cells;
        if (m->max_faces <= 3 && al)
            fv_flux3_wall_kernel<T, 3, true><<<grid, kFvThreads, 0, st>>>(f, C, L, pick<T>(m), pick3<T>(m), m->d_nface,
                                                                          m->d_nb, m->d_order, m->d_wall, wp, nv, g.N,
                                                                          (T)g.L, (T)g.dv);
        else if (m->max_faces <= 3)
            fv_flux3_wall_kernel<T, 3, false><<<grid, kFvThreads, 0, st>>>(f, C, L, pick<T>(m), pick3<T>(m),
                                                                           m->d_nface, m->d_nb, m->d_order, m->d_wall,
                                                                           wp, nv, g.N, (T)g.L, (T)g.dv);
        else if (al)
            fv_flux3_wall_kernel<T, kFvMaxFaces, true><<<grid, kFvThreads, 0, st>>>(
                f, C, L, pick<T>(m), pick3<T>(m), m->d_nface, m->d_nb, m->d_order, m->d_wall, wp, nv, g.N, (T)g.L,
                (T)g.dv);
        else
            fv_flux3_wall_kernel<T, kFvMaxFaces, false><<<grid, kFvThreads, 0, st>>>(
                f, C, L, pick<T>(m), pick3<T>(m), m->d_nface, m->d_nb, m->d_order, m->d_wall, wp, nv, g.N, (T)g.L,
                (T)g.dv);
        return cudaGetLastError();
    }
    const bool al = g.N % 4 == 0 && aligned16(f) && aligned16(C) && aligned16(L);
    // polygons in FP32 also take 4 velocities per thread here (measured: 0.082 -> 0.064 ms on a
    // 2603-cell Voronoi mesh; the reconstruction passes lose occupancy to registers and keep 1)
    const bool v4 = m->max_faces <= 3 && al, p4 = m->max_faces > 3 && al && sizeof(T) == 4;
    const int vec = (v4 || p4) ? 4 : 1;
    const dim3 grid((unsigned)m->n_cells, (unsigned)((nv / vec + kFvThreads - 1) / kFvThreads));
    if (v4)
        fv_flux3_kernel<T, 4, 3><<<grid, kFvThreads, 0, st>>>(f, C, L, pick<T>(m), pick3<T>(m), m->d_nface, m->d_nb,
                                                               m->d_order, nv, g.N, (T)g.L, (T)g.dv);
    else if (m->max_faces <= 3)
        fv_flux3_kernel<T, 1, 3><<<grid, kFvThreads, 0, st>>>(f, C, L, pick<T>(m), pick3<T>(m), m->d_nface, m->d_nb,
                                                               m->d_order, nv, g.N, (T)g.L, (T)g.dv);
    else if (p4) {
        if constexpr (sizeof(T) == 4)
            fv_flux3_kernel<T, 4, kFvMaxFaces><<<grid, kFvThreads, 0, st>>>(f, C, L, pick<T>(m), pick3<T>(m),
                                                                             m->d_nface, m->d_nb, m->d_order, nv,
                                                                             g.N, (T)g.L, (T)g.dv);
    } else
        fv_flux3_kernel<T, 1, kFvMaxFaces><<<grid, kFvThreads, 0, st>>>(f, C, L, pick<T>(m), pick3<T>(m),
                                                                         m->d_nface, m->d_nb, m->d_order, nv, g.N,
                                                                         (T)g.L, (T)g.dv);
    return cudaGetLastError();
}

template <typename T, int VEC, int MAXS>
void gradient_launch(const bz_mesh *m, int nv, const T *f, T *G, cudaStream_t st) {
    const dim3 grid((unsigned)m->n_cells, (unsigned)((nv / VEC + kFvThreads - 1) / kFvThreads));
    fv_gradient_kernel<T, VEC, MAXS><<<grid, kFvThreads, 0, st>>>(f, G, pick<T>(m), m->d_ncen, m->d_cen, m->d_nsec,
                                                                  m->d_sec, m->d_order, nv);
}

template <typename T, bool kGrad, int VEC, int MAXF>
void flux_launch(const bz_mesh *m, const GridView &g, const T *f, const T *G, T *L, cudaStream_t st) {
    const int nv = (int)g.nv;
    const dim3 grid((unsigned)m->n_cells, (unsigned)((nv / VEC + kFvThreads - 1) / kFvThreads));
    fv_flux_kernel<T, kGrad, VEC, MAXF><<<grid, kFvThreads, 0, st>>>(f, G, L, pick<T>(m), m->d_nface, m->d_nb,
                                                                     m->d_order, nv, g.N, (T)g.L, (T)g.dv);
}

// Triangle meshes with 16-byte aligned rows take 4 velocities per thread and
// unrolled 3-face loops; other meshes one velocity per thread and 8-face loops.
template <typename T>
cudaError_t gradient(const bz_mesh *m, const GridView &g, const T *f, T *G, cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    const int nv = (int)g.nv;
    if (m->max_faces <= 3 && nv % 4 == 0 && aligned16(f) && aligned16(G))
        gradient_launch<T, 4, 3>(m, nv, f, G, st);
    else if (m->max_faces <= 3)
        gradient_launch<T, 1, 3>(m, nv, f, G, st);
    else
        gradient_launch<T, 1, kFvMaxFaces>(m, nv, f, G, st);
    return cudaGetLastError();
}

template <typename T, bool kGrad, int MAXF, bool VLOAD>
void flux_wall_launch(const bz_mesh *m, const GridView &g, const T *f, const T *G, T *L, cudaStream_t st) {
    const T *wp = static_cast<const T *>(sizeof(T) == 8 ? static_cast<const void *>(m->d_wall64)
                                                        : static_cast<const void *>(m->d_wall32));
    fv_flux_wall_kernel<T, kGrad, MAXF, VLOAD><<<(unsigned)m->n_cells, kFvThreads, 0, st>>>(
        f, G, L, pick<T>(m), m->d_nface, m->d_nb, m->d_order, m->d_wall, wp, (int)g.nv, g.N, (T)g.L, (T)g.dv);
}

template <typename T>
cudaError_t flux_walls(const bz_mesh *m, const GridView &g, const T *f, const T *G, T *L, cudaStream_t st) {
    const bool al = aligned16(f) && aligned16(L) && (!G || aligned16(G));
    const bool tri = m->max_faces <= 3;
    if (G) {
        if (tri && al) flux_wall_launch<T, true, 3, true>(m, g, f, G, L, st);
        else if (tri) flux_wall_launch<T, true, 3, false>(m, g, f, G, L, st);
        else if (al) flux_wall_launch<T, true, kFvMaxFaces, true>(m, g, f, G, L, st);
        else flux_wall_launch<T, true, kFvMaxFaces, false>(m, g, f, G, L, st);
    } else {
        if (tri && al) flux_wall_launch<T, false, 3, true>(m, g, f, G, L, st);
        else if (tri) flux_wall_launch<T, false, 3, false>(m, g, f, G, L, st);
        else if (al) flux_wall_launch<T, false, kFvMaxFaces, true>(m, g, f, G, L, st);
        else flux_wall_launch<T, false, kFvMaxFaces, false>(m, g, f, G, L, st);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t flux(const bz_mesh *m, const GridView &g, const T *f, const T *G, T *L, cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    if (m->n_walls > 0) {
        if (!fv_walls_supported(m, g)) return cudaErrorInvalidValue;
        return flux_walls<T>(m, g, f, G, L, st);
    }
    const bool tri = m->max_faces <= 3;
    const bool v4 = tri && g.N % 4 == 0 && aligned16(f) && aligned16(L) && (!G || aligned16(G));
    if (G) {
        if (v4) flux_launch<T, true, 4, 3>(m, g, f, G, L, st);
        else if (tri) flux_launch<T, true, 1, 3>(m, g, f, G, L, st);
        else flux_launch<T, true, 1, kFvMaxFaces>(m, g, f, G, L, st);
    } else {
        if (v4) flux_launch<T, false, 4, 3>(m, g, f, G, L, st);
        else if (tri) flux_launch<T, false, 1, 3>(m, g, f, G, L, st);
        else flux_launch<T, false, 1, kFvMaxFaces>(m, g, f, G, L, st);
    }
    return cudaGetLastError();
}

}  // namespace

bool fv_face_mode(const bz_mesh *m, const GridView &g, const void *f, const void *L, const void *FV) {
    return m->order == 2 && m->max_faces <= 3 && m->d_tripos && m->n_walls == 0 && g.N % 4 == 0 && aligned16(f) &&
           aligned16(L) &&
           aligned16(FV);
}

static int fv_sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

// persistent grid: cps blocks per SM over the velocity blocks
static dim3 faces_grid(const bz_mesh *m, int nv, int cps) {
    const int gy = (nv / 4 + kFvThreads - 1) / kFvThreads;
    const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(m->n_cells, (int64_t)fv_sm_count() * cps / gy));
    return dim3((unsigned)gx, (unsigned)gy);
}

cudaError_t launch_fv_faces_f32(const bz_mesh *m, const GridView &g, const float *f, float *FV, cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    const int nv = (int)g.nv;
    fv_faces_persist_kernel<kFacesCtasPerSm><<<faces_grid(m, nv, kFacesCtasPerSm), kFvThreads, kFaceStageBytes, st>>>(
        f, FV, m->t32, m->d_cen, m->d_nsec, m->d_sec, m->d_tripos, m->n_cells, nv);
    return cudaGetLastError();
}

cudaError_t launch_fv_flux_faces_f32(const bz_mesh *m, const GridView &g, const float *FV, float *L,
                                     cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    const int nv = (int)g.nv;
    fv_flux_faces_persist_kernel<<<faces_grid(m, nv, kFluxCtasPerSm), kFvThreads, kFaceStageBytes, st>>>(
        FV, L, m->t32, m->d_tripos, m->n_cells, nv, g.N, (float)g.L, (float)g.dv);
    return cudaGetLastError();
}

bool fv_walls_supported(const bz_mesh *m, const GridView &g) {
    return m->n_walls == 0 || (g.N % 4 == 0 && g.nv <= 4 * kFvThreads);
}

cudaError_t launch_fv_gradient_f64(const bz_mesh *m, const GridView &g, const double *f, double *G, cudaStream_t st) {
    return gradient<double>(m, g, f, G, st);
}
cudaError_t launch_fv_gradient_f32(const bz_mesh *m, const GridView &g, const float *f, float *G, cudaStream_t st) {
    return gradient<float>(m, g, f, G, st);
}
cudaError_t launch_fv_flux_f64(const bz_mesh *m, const GridView &g, const double *f, const double *G, double *L,
                               cudaStream_t st) {
    return flux<double>(m, g, f, G, L, st);
}
cudaError_t launch_fv_flux_f32(const bz_mesh *m, const GridView &g, const float *f, const float *G, float *L,
                               cudaStream_t st) {
    return flux<float>(m, g, f, G, L, st);
}

cudaError_t launch_fv_coef3_f64(const bz_mesh *m, const GridView &g, const double *f, double *C, cudaStream_t st) {
    return coef3<double>(m, g, f, C, st);
}
cudaError_t launch_fv_coef3_f32(const bz_mesh *m, const GridView &g, const float *f, float *C, cudaStream_t st) {
    return coef3<float>(m, g, f, C, st);
}
cudaError_t launch_fv_flux3_f64(const bz_mesh *m, const GridView &g, const double *f, const double *C, double *L,
                                cudaStream_t st) {
    return flux3<double>(m, g, f, C, L, st);
}
cudaError_t launch_fv_flux3_f32(const bz_mesh *m, const GridView &g, const float *f, const float *C, float *L,
                                cudaStream_t st) {
    return flux3<float>(m, g, f, C, L, st);
}

}  // namespace bz
