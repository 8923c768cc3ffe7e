// k_transport.cu -- transport residual of the finite-volume scheme (Sec. 3.2,
// eq. finite_vol5 / eq. ho): CWENO reconstruction of degree 1 and Rusanov
// fluxes, for every cell and every discrete velocity of a 2-D grid.
//
// Layout: f, L are [cell][nv] (the collision operator's layout), so one
// cell's velocities are contiguous.  A block takes 256 velocities of one
// cell: every table entry of the cell is a warp-uniform load and every f
// access is one coalesced row segment (neighbour rows come from L2: a 32^2
// grid of 20k cells holds 81 MB in FP32).
//
// Pass 1 (order 2): gradient of the CWENO polynomial per (cell, velocity),
// stored as G [cell][2][nv].  The central (least-squares) gradient g_opt and
// the sector gradients g_L are linear in the averages (tables R_c, R_s of
// fv_mesh.cpp); the central polynomial's gradient is g_0 = (g_opt - sum_L
// lambda_L g_L) / lambda_0 (eq. CWENO:P0, lambda_0 = 3/4, lambda_L = 1/4 /
// #sectors); smoothness sigma_s = h^2 |g_s|^2; weights omega_s proportional
// to lambda_s / (sigma_s + eps)^4 with eps = 1e-14 (eqn.weights), formed
// as lambda_s ((sigma_min + eps) / (sigma_s + eps))^4 so that no power
// underflows in FP32.
//
// Pass 2: per face, f_L = fbar_i + g_i . (x_f - x_b,i), f_R the same from the
// neighbour (f_L on a boundary face: transmissive), Rusanov flux of v f:
// |e| F = (v.|e|n)(f_L + f_R)/2 - |v.|e|n| (f_R - f_L)/2, summed and scaled
// by 1/|P_i|.  The face midpoint rule is exact for degree-1 reconstructions.
#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int kFvThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kFvThreads)
fv_gradient_kernel(const T *__restrict__ f, T *__restrict__ G, FvTables<T> tb, const int *__restrict__ ncen,
                   const int *__restrict__ cen, const int *__restrict__ nsec, const int *__restrict__ sec, int nv) {
    const int64_t i = blockIdx.x;
    const int k = blockIdx.y * kFvThreads + threadIdx.x;
    if (k >= nv) return;
    const T fi = f[i * nv + k];
    const int nc = __ldg(ncen + i);
    T gx = (T)0, gy = (T)0;
    for (int q = 0; q < nc; ++q) {
        const int j = __ldg(cen + i * kFvCentral + q);
        const T d = f[(int64_t)j * nv + k] - fi;
        gx += __ldg(tb.Rc + (i * 2) * kFvCentral + q) * d;
        gy += __ldg(tb.Rc + (i * 2 + 1) * kFvCentral + q) * d;
    }
    const int ns = __ldg(nsec + i);
    if (ns > 0) {
        constexpr T kLam0 = (T)0.75, kEps = (T)1e-14;
        const T lamL = (T)0.25 / (T)ns, h2 = __ldg(tb.h2 + i);
        T sx[kFvMaxFaces], sy[kFvMaxFaces];
        T sumx = (T)0, sumy = (T)0;
        for (int s = 0; s < ns; ++s) {
            const int a = __ldg(sec + (i * kFvMaxFaces + s) * 2), b = __ldg(sec + (i * kFvMaxFaces + s) * 2 + 1);
            const T da = f[(int64_t)a * nv + k] - fi, db = f[(int64_t)b * nv + k] - fi;
            const T *R = tb.Rs + (i * kFvMaxFaces + s) * 4;
            sx[s] = __ldg(R) * da + __ldg(R + 1) * db;
            sy[s] = __ldg(R + 2) * da + __ldg(R + 3) * db;
            sumx += sx[s];
            sumy += sy[s];
        }
        const T g0x = (gx - lamL * sumx) / kLam0, g0y = (gy - lamL * sumy) / kLam0;
        const T sig0 = h2 * (g0x * g0x + g0y * g0y);
        T smin = sig0;
        for (int s = 0; s < ns; ++s) smin = fmin(smin, h2 * (sx[s] * sx[s] + sy[s] * sy[s]));
        auto weight = [&](T lam, T sig) {
            T r = (smin + kEps) / (sig + kEps);
            r = r * r;
            return lam * (r * r);
        };
        T w = weight(kLam0, sig0);
        T wsum = w, ax = w * g0x, ay = w * g0y;
        for (int s = 0; s < ns; ++s) {
            w = weight(lamL, h2 * (sx[s] * sx[s] + sy[s] * sy[s]));
            wsum += w;
            ax += w * sx[s];
            ay += w * sy[s];
        }
        gx = ax / wsum;
        gy = ay / wsum;
    }
    G[(i * 2) * nv + k] = gx;
    G[(i * 2 + 1) * nv + k] = gy;
}

template <typename T, bool kGrad>
__global__ void __launch_bounds__(kFvThreads)
fv_flux_kernel(const T *__restrict__ f, const T *__restrict__ G, T *__restrict__ L, FvTables<T> tb,
               const int *__restrict__ nface, const int *__restrict__ nb, int nv, int N, double Lv, double dv) {
    const int64_t i = blockIdx.x;
    const int k = blockIdx.y * kFvThreads + threadIdx.x;
    if (k >= nv) return;
    const T v1 = (T)(-Lv + (k / N) * dv), v2 = (T)(-Lv + (k % N) * dv);
    const T fi = f[i * nv + k];
    T gxi = (T)0, gyi = (T)0;
    if (kGrad) {
        gxi = G[(i * 2) * nv + k];
        gyi = G[(i * 2 + 1) * nv + k];
    }
    const int nf = __ldg(nface + i);
    T acc = (T)0;
    for (int q = 0; q < nf; ++q) {
        const int64_t s = i * kFvMaxFaces + q;
        const int j = __ldg(nb + s);
        const T vn = v1 * __ldg(tb.fn + 2 * s) + v2 * __ldg(tb.fn + 2 * s + 1);
        T fl = fi, fr;
        if (kGrad) fl += gxi * __ldg(tb.off_i + 2 * s) + gyi * __ldg(tb.off_i + 2 * s + 1);
        if (j >= 0) {
            fr = f[(int64_t)j * nv + k];
            if (kGrad)
                fr += G[((int64_t)j * 2) * nv + k] * __ldg(tb.off_j + 2 * s) +
                      G[((int64_t)j * 2 + 1) * nv + k] * __ldg(tb.off_j + 2 * s + 1);
        } else {
            fr = fl;
        }
        acc += (T)0.5 * vn * (fl + fr) - (T)0.5 * fabs(vn) * (fr - fl);
    }
    L[i * nv + k] = acc * __ldg(tb.inv_area + i);
}

template <typename T> const FvTables<T> &pick(const bz_mesh *m);
template <> const FvTables<double> &pick<double>(const bz_mesh *m) { return m->t64; }
template <> const FvTables<float> &pick<float>(const bz_mesh *m) { return m->t32; }

template <typename T>
cudaError_t gradient(const bz_mesh *m, const GridView &g, const T *f, T *G, cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    const dim3 grid((unsigned)m->n_cells, (unsigned)((g.nv + kFvThreads - 1) / kFvThreads));
    fv_gradient_kernel<T><<<grid, kFvThreads, 0, st>>>(f, G, pick<T>(m), m->d_ncen, m->d_cen, m->d_nsec, m->d_sec,
                                                       (int)g.nv);
    return cudaGetLastError();
}

template <typename T>
cudaError_t flux(const bz_mesh *m, const GridView &g, const T *f, const T *G, T *L, cudaStream_t st) {
    if (m->n_cells <= 0) return cudaSuccess;
    const dim3 grid((unsigned)m->n_cells, (unsigned)((g.nv + kFvThreads - 1) / kFvThreads));
    if (G)
        fv_flux_kernel<T, true><<<grid, kFvThreads, 0, st>>>(f, G, L, pick<T>(m), m->d_nface, m->d_nb, (int)g.nv,
                                                             g.N, g.L, g.dv);
    else
        fv_flux_kernel<T, false><<<grid, kFvThreads, 0, st>>>(f, nullptr, L, pick<T>(m), m->d_nface, m->d_nb,
                                                              (int)g.nv, g.N, g.L, g.dv);
    return cudaGetLastError();
}

}  // namespace

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

}  // namespace bz
