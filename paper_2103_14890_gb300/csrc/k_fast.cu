// k_fast.cu -- the fast spectral form of the collision operator (Sec. 3.3,
// Carleman representation: eq. defQBCarleman, eq. Btilde, eq. FKM, eq. ode)
// for 2-D Maxwell molecules, evaluated as FFT convolutions.
//
// With the direction decomposition B_F(l,m) ~ sum_p alpha_p(l) alpha'_p(m)
// over A collision directions, the mode sum of eq. ode is
//   Q-hat_k = sum_p sum_{l+m=k} (alpha_p f-hat)_l (alpha'_p f-hat)_m
//           - sum_{l+m=k} f-hat_l (Lambda f-hat)_m,     Lambda(m) = B_F(m,m),
// A + 1 products of band-limited functions (A/2 + 1 for even A: direction
// p + A/2 is direction p with alpha and alpha' exchanged, which leaves the
// gain product unchanged, so the host folds it into direction p's weight).  Each product is formed on a
// zero-padded P x P grid with P >= 3h + 1, where the circular convolution of
// two spectra supported in K_h equals the linear one at every k in K_h.
// alpha_p, alpha'_p and Lambda are real and even and f-hat is Hermitian, so
// a = IDFT(alpha_p f-hat) and b = IDFT(alpha'_p f-hat) are real: one complex
// inverse transform of (alpha_p + i alpha'_p) f-hat yields a + i b and the
// product is Re * Im.  The sum g of the A + 1 products goes back through one
// real forward transform; Q-hat keeps k in K_h with k_1 >= 0 (tiled layout).
//
// A CTA takes C cells with C * P threads (96 for P <= 48; 144 FP32 / 72 FP64
// threads for the P = 72 of 48^2 grids).  Per direction: pass A, one
// thread per (cell, k1 in [-h, h]) transforms along k2 into Y (shared);
// pass B, one thread per (cell, j2) transforms Y along k1 and accumulates the
// product into g (shared; each thread owns its column of g for the whole
// call).  Then pass C (thread per (cell, j2)) transforms g along j1 for
// k1 = 0..h, and pass D (three threads per (cell, k1), one per residue class
// of the output index) along j2, scales by P^-2 and stores Q-hat.  Every shared-memory array keeps the cell index fastest, so
// consecutive threads touch consecutive words.
//
// Two other organisations were measured on a GB300 and were slower at A = 8
// (65536 cells, 32^2): two warp groups running pass A of direction p and
// pass B of direction p - 1 at the same time on a double-buffered Y (fewer
// CTAs per SM, idle warps at the pipeline's fill and drain: +23 %), and one
// shared FFT body for all passes with cp.async loads of the half spectrum
// (the paired-cell pass C it needs runs on half the threads: +3 %).
#include <limits.h>

#include "bz_device.cuh"
#include "bz_internal.h"
#include "fft_reg.cuh"

namespace bz {

namespace {

// Smallest register-FFT length >= n (lengths 2^p <= 32, 3 * 2^p <= 48, 72).
constexpr int fast_pad(int n) {
    return n <= 2 ? 2 : n <= 3 ? 3 : n <= 4 ? 4 : n <= 6 ? 6 : n <= 8 ? 8 : n <= 12 ? 12
         : n <= 16 ? 16 : n <= 24 ? 24 : n <= 32 ? 32 : n <= 48 ? 48 : n <= 72 ? 72 : 0;
}

// Cells per CTA: C * P = 96 threads for P <= 48; for P = 72 (48^2 grids) two
// FP32 cells (144 threads) or one FP64 cell, whose scratch fills 111 KB.
constexpr int fast_cells(int P, int bytes) { return P <= 48 ? 96 / P : (bytes == 4 ? 2 : 1); }

template <typename T, int N> struct FastShape {
    static constexpr int H = N / 2 - 1, M = 2 * H + 1;
    static constexpr int P = fast_pad(3 * H + 1);
    static constexpr int C = fast_cells(P, (int)sizeof(T));
    static constexpr int NT = C * P;                           // threads per CTA
    static_assert(P > 0 && C * M <= NT, "grid not served by the fast kernel");
    static constexpr int TS = P * C + C;                       // padded k1 stride of pass C/D
    static constexpr int nYa = M * P * C, nYb = (H + 1) * TS;
    static constexpr int nY = nYa > nYb ? nYa : nYb;           // complex
    static constexpr int nF = (H + 1) * M * C;                 // complex
    static constexpr int nG = P * P * C;                       // real
    static constexpr int nCF = (H + 1) * M;                    // complex: one direction's rows k1 >= 0
};

template <typename T, int N> constexpr size_t fast_smem() {
    using Sh = FastShape<T, N>;
    return 2 * sizeof(T) * (size_t)(Sh::nY + Sh::nF + Sh::nCF) + sizeof(T) * (size_t)Sh::nG;
}

// Asynchronous copy of one 8- or 16-byte value into shared memory.
template <int BYTES> __device__ __forceinline__ void cp_async_val(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

template <typename T, int N>
__global__ void __launch_bounds__(FastShape<T, N>::NT)
fast_collide_kernel(const typename C2<T>::type *__restrict__ fh, typename C2<T>::type *__restrict__ qh,
                    const typename C2<T>::type *__restrict__ coef, int nconv, int64_t nhalf, int64_t n) {
    using V2 = typename C2<T>::type;
    using S = T;
    using Sh = FastShape<T, N>;
    constexpr int H = Sh::H, M = Sh::M, P = Sh::P, C = Sh::C, TS = Sh::TS;
    static_assert(3 * H < P && P % 3 == 0, "the padded modes fill the middle third of every transform");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2 *Y = reinterpret_cast<V2 *>(smem_raw);     // pass A/B: [P][M][C]; pass C/D: [H+1][TS]
    V2 *F = Y + Sh::nY;                           // half spectrum [H+1][M][C]
    S *G = reinterpret_cast<S *>(F + Sh::nF);     // products [P][P][C]
    V2 *CF = reinterpret_cast<V2 *>(G + Sh::nG);  // direction factors of one direction, rows k1 = 0..H
    const int tid = threadIdx.x;
    const int64_t cell0 = (int64_t)blockIdx.x * C;
    // the factors are even in k, so rows k1 >= 0 serve every row; each
    // direction's are copied in while the previous direction's pass B runs
    auto stage_cf = [&](int p) {
        const V2 *src = coef + ((size_t)p * M + H) * M;
        for (int i = tid; i < Sh::nCF; i += Sh::NT) cp_async_val<(int)sizeof(V2)>(CF + i, src + i);
    };
    stage_cf(0);
    for (int i = tid; i < Sh::nF; i += Sh::NT) {
        const int c = i % C, mode = i / C;
        const int64_t cell = cell0 + c;
        F[i] = cell < n ? fh[tiled_index(cell, mode, nhalf)] : cmk<V2>((S)0., (S)0.);
    }
    cp_async_commit_wait_all();
    __syncthreads();

    const int c = tid % C, col = tid / C;
    for (int p = 0; p <= nconv; ++p) {            // p == nconv: the loss term
        // pass A: (cell c, row k1): along k2, sum_k2 w(k) f-hat(k) e^{+2 pi i j2 k2 / P}
        if (tid < C * M) {
            const int k1 = col - H, a1 = k1 > 0 ? k1 : -k1;
            const V2 *frow = F + (a1 * M + H) * C + c;    // row |k1| at column 0
            const V2 *crow = CF + a1 * M + H;
            V2 a[P];
#pragma unroll
            for (int j = 0; j < P; ++j) a[j] = cmk<V2>((S)0., (S)0.);
            if (k1 > 0) {
#pragma unroll
                for (int k2 = -H; k2 <= H; ++k2) {
                    const V2 fv = frow[k2 * C], w = crow[k2];
                    a[(k2 + P) % P] = cmk<V2>(w.x * fv.x - w.y * fv.y, w.x * fv.y + w.y * fv.x);
                }
            } else {
                // f-hat(k) = conj f-hat(-k) and w(k) = w(-k): row -k1 read backwards
#pragma unroll
                for (int k2 = -H; k2 <= H; ++k2) {
                    const V2 t = frow[-k2 * C], w = crow[-k2];
                    const V2 fv = cmk<V2>(t.x, -t.y);
                    a[(k2 + P) % P] = cmk<V2>(w.x * fv.x - w.y * fv.y, w.x * fv.y + w.y * fv.x);
                }
            }
            fft_nat_mid0<P, +1>(a);            // k2 in [-H, H]: the middle third is padding
#pragma unroll
            for (int j2 = 0; j2 < P; ++j2) Y[(j2 * M + k1 + H) * C + c] = a[j2];
        }
        __syncthreads();
        if (p < nconv) stage_cf(p + 1);           // pass A is done with this direction's factors
        // pass B: (cell c, column j2): along k1, then g += Re * Im (gain) or -= (loss)
        {
            const int j2 = col;
            V2 b[P];
#pragma unroll
            for (int j = 0; j < P; ++j) b[j] = cmk<V2>((S)0., (S)0.);
#pragma unroll
            for (int k1 = -H; k1 <= H; ++k1) b[(k1 + P) % P] = Y[(j2 * M + k1 + H) * C + c];
            fft_nat_mid0<P, +1>(b);            // k1 in [-H, H]: the middle third is padding
            S *g = G + j2 * C + c;
            if (p == 0) {
#pragma unroll
                for (int j1 = 0; j1 < P; ++j1) g[j1 * P * C] = b[j1].x * b[j1].y;
            } else if (p < nconv) {
#pragma unroll
                for (int j1 = 0; j1 < P; ++j1) g[j1 * P * C] = fma(b[j1].x, b[j1].y, g[j1 * P * C]);
            } else {
#pragma unroll
                for (int j1 = 0; j1 < P; ++j1) g[j1 * P * C] = fma(-b[j1].x, b[j1].y, g[j1 * P * C]);
            }
        }
        cp_async_commit_wait_all();
        __syncthreads();
    }

    // pass C: (cell c, column j2): real transform of g along j1, k1 = 0..h,
    // through a complex length-P/2 FFT of (g[2q] + i g[2q+1]) and the
    // even/odd untangling X(k) = E(k) + e^{-2 pi i k / P} O(k)
    {
        constexpr int P2 = P / 2;
        const int j2 = col;
        const S *g = G + j2 * C + c;
        V2 z[P2];
#pragma unroll
        for (int q = 0; q < P2; ++q) z[q] = cmk<V2>(g[(2 * q) * P * C], g[(2 * q + 1) * P * C]);
        fft_nat<P2, -1>(z);
#pragma unroll
        for (int k1 = 0; k1 <= H; ++k1) {
            const V2 zk = z[k1 % P2], zc = z[(P2 - k1) % P2];
            const S ex = (S)0.5 * (zk.x + zc.x), ey = (S)0.5 * (zk.y - zc.y);
            const S ox = (S)0.5 * (zk.y + zc.y), oy = -(S)0.5 * (zk.x - zc.x);
            const V2 w = twl<P, V2>(k1);
            Y[k1 * TS + j2 * C + c] = cmk<V2>(ex + (w.x * ox - w.y * oy), ey + (w.x * oy + w.y * ox));
        }
    }
    __syncthreads();
    // pass D: (cell, row k1 >= 0, residue r): the length-P transform along j2,
    // keep k2 in [-h, h], scale P^-2.  P = 3Q, split over three threads by the
    // residue r of the output index (3 k' + r): thread r forms the r-th output
    // of the 3-point DFTs over (n, n + Q, n + 2Q) times the twiddle of its
    // class and finishes with one Q-point transform (the first stage of the
    // mixed-radix fft_nat, spread over three threads instead of one).
    {
        static_assert(P % 3 == 0, "pass D splits P = 3Q");
        constexpr int Q = P / 3, ROWS = C * (H + 1);
        static_assert(3 * ROWS <= Sh::NT, "three threads per output row");
        if (tid < 3 * ROWS) {
            const int r = tid / ROWS, rest = tid % ROWS;
            const int cd = rest % C, k1 = rest / C;
            const V2 *yr = Y + k1 * TS + cd;
            constexpr S kS3 = (S)0.866025403784438647;   // sqrt(3) / 2
            V2 y[Q];
#pragma unroll
            for (int n2 = 0; n2 < Q; ++n2) {
                const V2 a0 = yr[n2 * C], a1 = yr[(Q + n2) * C], a2 = yr[(2 * Q + n2) * C];
                const S sx = a1.x + a2.x, sy = a1.y + a2.y;
                if (r == 0) {
                    y[n2] = cmk<V2>(a0.x + sx, a0.y + sy);
                } else {
                    // e^{-2 pi i r / 3}: the forward transform's 3-point DFT
                    const S mx = a0.x - (S)0.5 * sx, my = a0.y - (S)0.5 * sy;
                    const S dx = a1.x - a2.x, dy = a1.y - a2.y;
                    const S ix = kS3 * dy, iy = -kS3 * dx;
                    V2 u = r == 1 ? cmk<V2>(mx + ix, my + iy) : cmk<V2>(mx - ix, my - iy);
                    if (n2 > 0) {
                        const V2 w = twl<P, V2>(r * n2);
                        u = cmk<V2>(u.x * w.x - u.y * w.y, u.x * w.y + u.y * w.x);
                    }
                    y[n2] = u;
                }
            }
            fft_nat<Q, -1>(y);
            const int64_t cell = cell0 + cd;
            if (cell < n) {
                const S sc = (S)(1.0 / ((double)P * (double)P));
#pragma unroll
                for (int kq = 0; kq < Q; ++kq) {
                    const int idx = 3 * kq + r;
                    const int k2 = idx <= H ? idx : idx - P;
                    if (k2 >= -H && k2 <= H) {
                        const V2 v = y[kq];
                        qh[tiled_index(cell, (int64_t)k1 * M + k2 + H, nhalf)] = cmk<V2>(v.x * sc, v.y * sc);
                    }
                }
            }
        }
    }
}

template <typename T, int N>
cudaError_t launch_fast_n(const GridView &g, const typename C2<T>::type *fh, typename C2<T>::type *qh,
                          const typename C2<T>::type *coef, int nconv, int64_t n, cudaStream_t st) {
    constexpr size_t sm = fast_smem<T, N>();
    constexpr int C = FastShape<T, N>::C;
    const int64_t blocks = (n + C - 1) / C;
    if (blocks > INT_MAX) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fast_collide_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    fast_collide_kernel<T, N><<<(unsigned)blocks, FastShape<T, N>::NT, sm, st>>>(fh, qh, coef, nconv, g.nhalf, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fast_any(const bz_modes *m, const typename C2<T>::type *fh, typename C2<T>::type *qh, int64_t n,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const GridView &g = m->g->v;
    const void *cv = sizeof(T) == 8 ? static_cast<const void *>(m->d_fast64) : static_cast<const void *>(m->d_fast32);
    const auto *coef = static_cast<const typename C2<T>::type *>(cv);
    switch (g.N) {
        case 8: return launch_fast_n<T, 8>(g, fh, qh, coef, m->nconv, n, st);
        case 16: return launch_fast_n<T, 16>(g, fh, qh, coef, m->nconv, n, st);
        case 24: return launch_fast_n<T, 24>(g, fh, qh, coef, m->nconv, n, st);
        case 32: return launch_fast_n<T, 32>(g, fh, qh, coef, m->nconv, n, st);
        case 48: return launch_fast_n<T, 48>(g, fh, qh, coef, m->nconv, n, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool fast_supported(const GridView &g) {
    return g.dim == 2 && (g.N == 8 || g.N == 16 || g.N == 24 || g.N == 32 || g.N == 48);
}

int fast_pad_length(int N) { return fast_pad(3 * (N / 2 - 1) + 1); }
int fast_cells_per_cta(int N) { return fast_cells(fast_pad_length(N), 4); }

int fast_setup() {
    cudaError_t e = upload_fft_twiddles();
    if (e != cudaSuccess) return cuda_fail(e, "build_fast_modes: FFT twiddles");
    return BZ_OK;
}

cudaError_t launch_fast_f32(const bz_modes *m, const float2 *fh, float2 *qh, int64_t n, cudaStream_t st) {
    return launch_fast_any<float>(m, fh, qh, n, st);
}
cudaError_t launch_fast_f64(const bz_modes *m, const double2 *fh, double2 *qh, int64_t n, cudaStream_t st) {
    return launch_fast_any<double>(m, fh, qh, n, st);
}

}  // namespace bz
