// k_modesum32.cu -- register-blocked FP32 mode sum of eq. CF1 (Sec. 3.3) for
// 2-D velocity grids with N <= 48 and 3-D grids with N <= 16.
//
// Work reduction (exact algebra, no approximation):
//   * Q is real, so only k_1 >= 0 is computed (Q-hat_{-k} = conj(Q-hat_k)).
//   * The product f-hat_l f-hat_m is symmetric in (l, m): pairs with l_1 < m_1
//     are summed once with the weight beta-hat(l,m) + beta-hat(m,l); pairs with
//     l_1 = m_1 keep beta-hat(l,m).  So for outputs with first index k_1 only
//     l_1 in [k_1 - h, floor(k_1/2)] is visited and m_1 = k_1 - l_1 >= 0 always
//     lies in the stored half spectrum; f-hat_l with l_1 < 0 is conj(f-hat_{-l}).
//   * A "row" is the line of modes along the last axis with all other indices
//     fixed: (k_1) in 2-D, (k_1, k_2) in 3-D.  Each task's weight stream names
//     the pairs of rows (row of l, row of m) it visits, so the kernel body is
//     the same in both dimensions.
//
// Layout and blocking:
//   * one CTA = one tile of C cells (C = 32, or 16 for grids whose spectrum
//     does not fit 32 cells in shared memory); the tile's half spectrum
//     (complex FP32, [mode][cell]) sits in shared memory with lane % C = cell,
//     so every weight load is uniform over the lanes that share it and every
//     Fourier load is a conflict-free row of C cells.
//   * a task = (k_1, block of RT consecutive k_2).  With C = 32 a thread owns
//     all RT = R outputs of its cell; with C = 16 the two half-warps split the
//     block, each thread owning R = RT/2 of them.  Walking l_2 upwards slides
//     the window of f-hat_m values (m_2 = k_2 - l_2) down by one, so each step
//     loads one new f-hat_m, one f-hat_l and R weights for 6 R FP32 operations.
//   * each task's weights form a contiguous stream of row pairs, each a
//     16-byte header (which rows of l and m) followed by [l (padded to a
//     multiple of RT)][r]; one row pair is staged into a per-warp
//     shared-memory double buffer with cp.async while the previous one is used.
//   * the rows of the spectrum are stored back to back, with kPad zero columns
//     before the first and after the last row only.  A column index that falls
//     outside [-h, h] therefore reads a neighbouring row's (finite) value or a
//     zero, and always meets a zero weight: the weight stream is zero wherever
//     l_2, m_2 or k_2 leaves K_h.  The host checks that every column touched
//     stays within kPad of [-h, h].
//   * accumulation: plain FP32 along an l_1 row (<= 48 terms), then a TwoSum
//     fold of the row sum into a (hi, lo) pair per output every 4 rows.
//   * several kernel variants (R, warps, C) are compiled; the fastest one for a
//     grid is chosen once by timing (autotune below).
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "bz_device.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

// Kernel variants: outputs per thread R along k_2, warps per CTA, cells per
// CTA, cells per thread (pack: 1, or 2 for the packed two-cell kernel, whose
// lanes hold cells c and c + 16 of a 32-cell tile in FP32x2 register pairs),
// wdup: each weight stored twice (w, w) as an FP32x2 operand, pq: the FP32x2
// form with one cell per lane (modesum_pq_kernel), orient: 2 when the two
// halves of a warp hold the same cells and run each task plain and mirrored
// (paired orientations).  Variant ids reported by bz_modes_info are index + 1.
struct Variant {
    int R, warps, cells, pack, wdup, pq, orient;
};
constexpr int kNumVariants = kModesumVariants;   // FP32 variants (timed by the autotuner)
// entries 0..9: the FP32 variants; entries 10, 11: layouts of the FP64 and FP32X2
// forms only (2 outputs per thread, 8 warps, 8- and 4-cell tiles) for grids
// whose 16-byte-per-value spectrum needs them (48^2, 16^3)
constexpr Variant kVariants[kNumVariants + 2] = {
    {8, 16, 32, 1, 0, 0, 1}, {4, 32, 32, 1, 0, 0, 1}, {4, 16, 16, 1, 0, 0, 1}, {4, 16, 8, 1, 0, 0, 1},
    {4, 16, 32, 2, 1, 0, 1}, {8, 12, 32, 1, 0, 1, 1}, {8, 16, 32, 1, 0, 1, 1}, {8, 16, 16, 1, 0, 1, 2},
    {8, 8, 16, 1, 0, 1, 2},  {8, 4, 16, 1, 0, 1, 2},  {2, 8, 8, 1, 0, 0, 1},   {2, 8, 4, 1, 0, 0, 1}};

// lane groups splitting a task's outputs, and outputs per task (RT)
constexpr int variant_groups(int v) { return 32 / kVariants[v].cells * kVariants[v].pack / kVariants[v].orient; }
constexpr int variant_rt(int v) { return kVariants[v].R * variant_groups(v); }
// Whether an FP32 variant's tables compute k_2 < 0 on the reflected spectrum
// (every output block of k_2 >= 0 fits within the row: R T <= h + 1); all
// variants that do sum each output in one order, as do all that do not.
constexpr bool variant_reflects(int v, int h) { return kVariants[v].pack == 1 && variant_rt(v) <= h + 1; }
constexpr int kTaskInts = 12;   // ints per task record

constexpr int kPad = 8;         // zero guard columns before the first and after the last row
constexpr int kRowHeadBytes = 16;   // row-pair header in front of each weight row

struct TaskRec {
    int orow, k20, nrows, l2lo, nblk, woff, rfirst;   // rfirst: first r (of RT) this task stores
    int rowf, flags, crow, pad2, pad3;                // rowf: elements per row pair (header + weights);
                                                      // flags: kTask*; crow: row of the conjugate outputs
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPENDING> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPENDING) : "memory");
}

// Knuth's TwoSum: s + e == a + b exactly.
template <typename T> __device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = a + b;
    T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Stage `nbytes` bytes (multiple of 16) of a weight row into shared memory.
__device__ __forceinline__ void stage_row(void *dst, const void *src, int nbytes, int lane) {
    char *d = static_cast<char *>(dst);
    const char *g = static_cast<const char *>(src);
    for (int i = lane * 16; i < nbytes; i += 512) cp_async16(d + i, g + i);
    cp_async_commit();
}

// R consecutive weights (16-byte aligned) into registers.
__device__ __forceinline__ void load_w4(float *wv, const float *p) {
    const float4 w4 = *reinterpret_cast<const float4 *>(p);
    wv[0] = w4.x;
    wv[1] = w4.y;
    wv[2] = w4.z;
    wv[3] = w4.w;
}
__device__ __forceinline__ void load_w4(double *wv, const double *p) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    wv[0] = a.x;
    wv[1] = a.y;
    wv[2] = b.x;
    wv[3] = b.y;
}

// One block of RR l_2 steps.  The window of f-hat_m values lives in a 2RR-slot
// register array used under two alternating namings (PH = 0, 1): logical slot
// j is physical slot (j + PH RR) mod 2RR, so moving the window by RR between
// blocks costs no register moves; logical slot j of a block holds the column
// mp + j CS, and output r at step s reads logical slot r - s + RR - 1.
// f-hat_l is read at lp, lp + D, lp + 2 D, ... with D = DIR CS: for DIR = -1
// (l_1 < 0) the row is that of -l_1 read backwards and f-hat_l = conj of the
// value read, which only flips the signs of two FMA operands.  DIR = 0 takes
// the direction at run time (D = dcs, sgn = +/-1 multiplies the value's
// imaginary part): the products are those of DIR = +1 on the conjugated value,
// which are exactly those of DIR = -1 on the value read (negation is exact), so
// the results equal the specialised bodies' bit for bit with half the code.
// The weights of step s are wb[s * WS + r].
//
// RAMP: the first block of a task whose steps start one before the lowest l_2
// of its first output (l2lo = k2_0 - h - 1, outputs k2_0 + r >= 0): pair
// (s, r) lies in K_h exactly when s > r, so only those pairs are evaluated
// (the others have zero weights and would add exact zeros), and the window
// slots it needs are only the RR - 1 it loads itself.
template <typename T, int RR, int CS, int WS, int PH, int DIR, bool RAMP>
__device__ __forceinline__ void block_body(typename C2<T>::type (&win)[2 * RR],
                                           const typename C2<T>::type *__restrict__ mp,
                                           const typename C2<T>::type *__restrict__ lp, int dcs, T sgn,
                                           const T *__restrict__ wb, typename C2<T>::type (&acc)[RR]) {
    using V2 = typename C2<T>::type;
#pragma unroll
    for (int j = 0; j < (RAMP ? RR - 1 : RR); ++j) win[(j + PH * RR) & (2 * RR - 1)] = mp[j * CS];
#pragma unroll
    for (int s = RAMP ? 1 : 0; s < RR; ++s) {
        V2 fl = (DIR == 0) ? lp[s * dcs] : lp[s * DIR * CS];
        if (DIR == 0) fl.y *= sgn;
        T wv[RR];
        if constexpr (RR % 4 == 0) {
#pragma unroll
            for (int q = 0; q < RR; q += 4)
                if (!RAMP || q < s) load_w4(wv + q, wb + s * WS + q);
        } else {
            static_assert(RR == 2 && sizeof(T) == 8 && !RAMP, "two-output blocks are used by the FP64 form only");
            const double2 w2 = *reinterpret_cast<const double2 *>(wb + s * WS);
            wv[0] = w2.x;
            wv[1] = w2.y;
        }
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            if (RAMP && r >= s) continue;
            const V2 b = win[(r - s + RR - 1 + PH * RR) & (2 * RR - 1)];
            const T tx = wv[r] * fl.x, ty = wv[r] * fl.y;       // weight * value read
            if (DIR >= 0) {                                     // acc += w f-hat_l b
                acc[r].x = fma(tx, b.x, acc[r].x);
                acc[r].x = fma(-ty, b.y, acc[r].x);
                acc[r].y = fma(tx, b.y, acc[r].y);
                acc[r].y = fma(ty, b.x, acc[r].y);
            } else {                                            // acc += w conj(value) b
                acc[r].x = fma(tx, b.x, acc[r].x);
                acc[r].x = fma(ty, b.y, acc[r].x);
                acc[r].y = fma(tx, b.y, acc[r].y);
                acc[r].y = fma(-ty, b.x, acc[r].y);
            }
        }
    }
}

// One row pair of a task for this thread's RR outputs:
// acc[r] += sum_l2 w(l2, r) f-hat_l(l2) f-hat_m(k2_0 + r - l2) over nblk
// blocks of RR steps from l2lo.  rowl / rowm point at column 0 of the rows of
// l (or -l) and m (this thread's cell); wrow at this thread's first weight of
// the row.  The blocks run as pairs (PH 0, PH 1) and a last PH 0; with ramp
// (RAMPS only) the first block is the ramp body.
template <typename T, int RR, int CS, int WS, int DIR, bool RAMPS>
__device__ __forceinline__ void row_pass(const typename C2<T>::type *__restrict__ rowl,
                                         const typename C2<T>::type *__restrict__ rowm, const T *__restrict__ wrow,
                                         int nblk, int l2lo, int mbase0, int dir, bool ramp,
                                         typename C2<T>::type (&acc)[RR]) {
    using V2 = typename C2<T>::type;
    V2 win[2 * RR];
    const int dcs = (DIR == 0 ? dir : DIR) * CS;
    const T sgn = (T)dir;
    const V2 *mp = rowm + mbase0 * CS;
    const V2 *lp = rowl + l2lo * dcs;
    int blk = 0;
    bool ramped = false;
    if constexpr (RAMPS) {
        if (ramp) {
            // the ramp block under the PH 1 naming leaves the window exactly
            // as the preload below does for a first block under PH 0
            block_body<T, RR, CS, WS, 1, DIR, true>(win, mp, lp, dcs, sgn, wrow, acc);
            mp -= RR * CS;
            lp += RR * dcs;
            blk = 1;
            ramped = true;
        }
    }
    if (!ramped) {
#pragma unroll
        for (int j = RR; j < 2 * RR - 1; ++j) win[j] = mp[j * CS];
    }
    for (; blk + 1 < nblk; blk += 2) {
        block_body<T, RR, CS, WS, 0, DIR, false>(win, mp, lp, dcs, sgn, wrow + blk * RR * WS, acc);
        block_body<T, RR, CS, WS, 1, DIR, false>(win, mp - RR * CS, lp + RR * dcs, dcs, sgn,
                                                 wrow + (blk + 1) * RR * WS, acc);
        mp -= 2 * RR * CS;
        lp += 2 * RR * dcs;
    }
    if (blk < nblk) block_body<T, RR, CS, WS, 0, DIR, false>(win, mp, lp, dcs, sgn, wrow + blk * RR * WS, acc);
}

// Copy this CTA's cells of the tile's half spectrum into shared memory
// ([kPad + nhalf + kPad][CELLS], zero guards), or with every row's columns
// reversed (rev: mode (row, c) <- (row, -c), the spectrum of f reflected in
// the last velocity axis).
template <typename V2, int CELLS>
__device__ __forceinline__ void stage_spectrum(uint4 *smem16, const V2 *fhat, int64_t tile, int sub, int nhalf,
                                               int M, bool rev) {
    constexpr int VEC = 16 / (int)sizeof(V2);                    // cells per 16-byte vector
    constexpr int Q4 = CELLS / VEC, ROW = 32 / VEC;              // vectors per mode: this CTA, whole tile
    const uint4 *src = reinterpret_cast<const uint4 *>(fhat + tile * (int64_t)nhalf * 32) + sub * Q4;
    const int body = nhalf * Q4, guard = kPad * Q4;
    for (int i = threadIdx.x; i < body + 2 * guard; i += blockDim.x) {
        const int b = i - guard;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (b >= 0 && b < body) {
            int mode = b / Q4;
            if (rev) {
                const int row = mode / M;
                mode = row * M + (M - 1) - (mode - row * M);
            }
            v = src[mode * ROW + (b % Q4)];
        }
        smem16[i] = v;
    }
}

// Task flags (TaskRec.flags)
constexpr int kTaskRamp = 1;     // first block is the ramp (l2lo = k2_0 - h - 1)
constexpr int kTaskRefl = 2;     // reflected block: on the reflected spectrum (restaged, or read mirrored); output k_2 at column -k_2
constexpr int kTaskConj = 4;     // k_1 = 0 row: also stores conj(Q-hat) at (row crow, column -k_2), k_2 > 0

// The task table: 2 W + 1 offsets (W = warps x split), then the records.
// Warp w's phase-0 tasks are [off[w], off[w + 1]) and its phase-1 tasks
// [off[W + w], off[W + w + 1]); phase 1 (tasks flagged kTaskRefl) runs after
// the CTA has restaged its spectrum reversed.  Tables without reflected
// tasks have an empty phase 1.
template <typename T, int RR, int WARPS, int CELLS, bool RTDIR = false>
__global__ void __launch_bounds__(WARPS * 32, 1) modesum32_kernel(const Mode32Group gd) {
    using V2 = typename C2<T>::type;
    constexpr int G = 32 / CELLS;     // lane groups splitting a task's outputs
    constexpr int RT = RR * G;        // outputs per task
    constexpr int HEAD = kRowHeadBytes / (int)sizeof(T);
    constexpr bool RAMPS = (G == 1);  // ramped tasks need every lane on the same outputs
    extern __shared__ __align__(16) uint4 smem16[];
    // this CTA's instance and tile (instances are ordered longest-first)
    int it = 0;
    while (it + 1 < gd.nitems && (int64_t)blockIdx.x >= gd.tile_start[it + 1]) ++it;
    const Mode32Item &ip = gd.item[it];
    const V2 *__restrict__ fhat = static_cast<const V2 *>(ip.fhat);
    V2 *__restrict__ Qhat = static_cast<V2 *>(ip.Qhat);
    const T *__restrict__ W = static_cast<const T *>(ip.W);
    const int *__restrict__ tasks = ip.tasks;
    const int h = ip.h, M = ip.M, nhalf = ip.nhalf, wrow_max = ip.wrow_max;
    const int64_t n = ip.n;
    // a tile may be split over ip.split CTAs, each taking one part of the
    // task table (the last partial wave of a launch)
    const int64_t cta0 = (int64_t)blockIdx.x - gd.tile_start[it];
    const int part = (int)(cta0 % ip.split);
    const int64_t cta = cta0 / ip.split;
    const int64_t tile = cta / G;                                    // 32-cell tile of the scratch layout
    const int sub = (int)(cta % G);                                  // which CELLS-cell part of it
    V2 *Fs = reinterpret_cast<V2 *>(smem16);                         // [kPad + nhalf + kPad][CELLS]
    T *wsm = reinterpret_cast<T *>(Fs + (size_t)(nhalf + 2 * kPad) * CELLS);   // [warps][2][wrow_max]
    stage_spectrum<V2, CELLS>(smem16, fhat, tile, sub, nhalf, M, false);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cell = lane % CELLS, grp = lane / CELLS;
    T *wbuf0 = wsm + (size_t)warp * 2 * wrow_max;
    T *wbuf1 = wbuf0 + wrow_max;
    const int NW = WARPS * ip.split;                                 // task lists of the table
    int t = tasks[part * WARPS + warp], tend = tasks[part * WARPS + warp + 1];
    bool phase1 = false;
    const TaskRec *trec = reinterpret_cast<const TaskRec *>(tasks + 2 * NW + 1);
    const V2 *F0 = Fs + (size_t)(kPad + h) * CELLS + cell;          // (row 0, column 0) of this cell
    const bool valid = tile * 32 + sub * CELLS + cell < n;          // this lane's cell exists
    V2 *const qt = Qhat + tile * (int64_t)nhalf * 32 + sub * CELLS + cell;   // its (row 0, column -h)

    for (;;) {
        if (t >= tend) {
            // phase 1 (the same for the whole CTA: one table) after a restage;
            // the item's fields are read again from the parameters here rather
            // than kept in registers through the task loop
            if (phase1) break;
            const Mode32Item &iq = gd.item[it];
            const int *tq = iq.tasks;
            const int nw = WARPS * iq.split;
            if (tq[2 * nw] == tq[nw]) break;
            __syncthreads();                                         // every warp is done with the spectrum
            const int64_t c1 = (int64_t)blockIdx.x - gd.tile_start[it];
            const int64_t ct = c1 / iq.split;
            stage_spectrum<V2, CELLS>(smem16, static_cast<const V2 *>(iq.fhat), ct / G, (int)(ct % G), iq.nhalf,
                                      iq.M, true);
            __syncthreads();
            const int w1 = (int)(c1 % iq.split) * WARPS + (int)(threadIdx.x >> 5);
            t = tq[nw + w1];
            tend = tq[nw + w1 + 1];
            phase1 = true;
            continue;
        }
        const TaskRec tk = trec[t++];
        const int rowf = tk.rowf;                         // elements per row pair
        const bool ramp = RAMPS && (tk.flags & kTaskRamp) != 0;
        const T *wsrc = W + tk.woff;
        V2 hi[RR], lo[RR], acc[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) hi[r] = lo[r] = acc[r] = cmk<V2>(0, 0);
        const int k20 = tk.k20 + grp * RR;                // this thread's first output column
        const int mbase0 = k20 - tk.l2lo - (RR - 1);
        stage_row(wbuf0, wsrc, rowf * (int)sizeof(T), lane);
        for (int i = 0; i < tk.nrows; ++i) {
            const T *wcur = (i & 1) ? wbuf1 : wbuf0;
            if (i + 1 < tk.nrows) {
                stage_row((i & 1) ? wbuf0 : wbuf1, wsrc + (size_t)(i + 1) * rowf, rowf * (int)sizeof(T), lane);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            // row header: element offsets of the rows of l and m, and the
            // direction of l (-1: f-hat_l = conj(f-hat_{-l}), row of -l read backwards)
            const int4 hd = *reinterpret_cast<const int4 *>(wcur);
            const int dir = hd.z > 0 ? 1 : -1;
            if constexpr (RTDIR)
                row_pass<T, RR, CELLS, RT, 0, RAMPS>(F0 + hd.x, F0 + hd.y, wcur + HEAD + grp * RR, tk.nblk * G,
                                                     tk.l2lo, mbase0, dir, ramp, acc);
            else if (dir > 0)
                row_pass<T, RR, CELLS, RT, 1, RAMPS>(F0 + hd.x, F0 + hd.y, wcur + HEAD + grp * RR, tk.nblk * G,
                                                     tk.l2lo, mbase0, dir, ramp, acc);
            else
                row_pass<T, RR, CELLS, RT, -1, RAMPS>(F0 + hd.x, F0 + hd.y, wcur + HEAD + grp * RR, tk.nblk * G,
                                                      tk.l2lo, mbase0, dir, ramp, acc);
            __syncwarp();
            // fold the row sums (<= 4 rows) into (hi, lo)
            if ((i & 3) == 3 || i + 1 == tk.nrows) {
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    T s, e;
                    two_sum(hi[r].x, acc[r].x, s, e);
                    hi[r].x = s;
                    lo[r].x += e;
                    two_sum(hi[r].y, acc[r].y, s, e);
                    hi[r].y = s;
                    lo[r].y += e;
                    acc[r] = cmk<V2>(0, 0);
                }
            }
        }
        if (valid) {
            // the record's output fields are read again here (volatile: not
            // kept in registers through the row loop)
            const volatile TaskRec *tv = trec + (t - 1);
            const int orow = tv->orow, rfirst = tv->rfirst, flags = tv->flags, crow = tv->crow;
            const int k2o = tv->k20 + grp * RR;
            V2 *out = qt + (int64_t)orow * M * 32;
            const bool refl = (flags & kTaskRefl) != 0, cj = (flags & kTaskConj) != 0;
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int k2 = k2o + r;
                if (grp * RR + r >= rfirst && k2 <= h) {
                    const V2 q = cmk<V2>(hi[r].x + lo[r].x, hi[r].y + lo[r].y);
                    out[(refl ? h - k2 : k2 + h) * 32] = q;
                    if (cj && k2 > 0) qt[((int64_t)crow * M + h - k2) * 32] = cmk<V2>(q.x, -q.y);
                }
            }
        }
    }
}

// ---- packed two-cell form ------------------------------------------------------
// The same sums with two cells per thread: lane p of a lane group holds cells
// p and p + 16 of the 32-cell tile, every spectrum entry in shared memory is
// one float4 (re_p, re_{p+16}, im_p, im_{p+16}), and every product and
// accumulation is one FP32x2 instruction (__fmul2_rn / __ffma2_rn: two
// independent IEEE FP32 operations, the same results as two scalar ones).
// Each weight is stored twice, (w, w), so it is an FP32x2 operand as loaded.
// Every lane performs exactly the operations of the scalar kernels, in the
// same order (tx = w a_re, ty = w a_im, re += tx b_re then += (-ty) b_im, im
// += tx b_im then += ty b_re, with the signs of a conjugated f-hat_l for
// l_1 < 0), so its results equal theirs bit for bit and the variants can
// share one batch (whole waves on one, the last wave on another).  The two
// lane groups of a warp split a task's 2 R outputs as in the 16-cell variant.
struct P2Acc {
    float2 re, im;
};

template <int RR, int PH, int DIR>
__device__ __forceinline__ void block_pass_p2(float4 (&win)[2 * RR], const float4 *__restrict__ mp,
                                              const float4 *__restrict__ lp, const float *__restrict__ wb,
                                              P2Acc (&acc)[RR]) {
    constexpr int CS = 16, RT = 2 * RR;
#pragma unroll
    for (int j = 0; j < RR; ++j) win[(j + PH * RR) & (2 * RR - 1)] = mp[j * CS];
#pragma unroll
    for (int s = 0; s < RR; ++s) {
        const float4 av = lp[s * DIR * CS];
        const float2 ar = make_float2(av.x, av.y);
        const float2 ai = make_float2(av.z, av.w), an = make_float2(-av.z, -av.w);
        float2 w2[RR];
#pragma unroll
        for (int q = 0; q < RR; q += 2) {
            const float4 w4 = *reinterpret_cast<const float4 *>(wb + s * 2 * RT + 2 * q);
            w2[q] = make_float2(w4.x, w4.y);
            w2[q + 1] = make_float2(w4.z, w4.w);
        }
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const float4 bv = win[(r - s + RR - 1 + PH * RR) & (2 * RR - 1)];
            const float2 br = make_float2(bv.x, bv.y), bi = make_float2(bv.z, bv.w);
            const float2 tx = __fmul2_rn(w2[r], ar);
            const float2 ty = __fmul2_rn(w2[r], ai), tn = __fmul2_rn(w2[r], an);   // w a_im, -(w a_im)
            acc[r].re = __ffma2_rn(tx, br, acc[r].re);
            acc[r].re = __ffma2_rn(DIR > 0 ? tn : ty, bi, acc[r].re);
            acc[r].im = __ffma2_rn(tx, bi, acc[r].im);
            acc[r].im = __ffma2_rn(DIR > 0 ? ty : tn, br, acc[r].im);
        }
    }
}

template <int RR, int DIR>
__device__ __forceinline__ void row_pass_p2(const float4 *__restrict__ rowl, const float4 *__restrict__ rowm,
                                            const float *__restrict__ wrow, int nblk, int l2lo, int mbase0,
                                            P2Acc (&acc)[RR]) {
    constexpr int CS = 16, RT = 2 * RR;
    float4 win[2 * RR];
    const float4 *mp = rowm + mbase0 * CS;
    const float4 *lp = rowl + DIR * l2lo * CS;
#pragma unroll
    for (int j = RR; j < 2 * RR - 1; ++j) win[j] = mp[j * CS];
    int blk = 0;
    for (; blk + 1 < nblk; blk += 2) {
        block_pass_p2<RR, 0, DIR>(win, mp, lp, wrow + blk * RR * 2 * RT, acc);
        block_pass_p2<RR, 1, DIR>(win, mp - RR * CS, lp + RR * DIR * CS, wrow + (blk + 1) * RR * 2 * RT, acc);
        mp -= 2 * RR * CS;
        lp += 2 * RR * DIR * CS;
    }
    if (blk < nblk) block_pass_p2<RR, 0, DIR>(win, mp, lp, wrow + blk * RR * 2 * RT, acc);
}

// TwoSum on both lanes of an FP32x2 pair (each lane exact as the scalar form).
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, make_float2(-a.x, -a.y));
    const float2 t = __fadd2_rn(s, make_float2(-bb.x, -bb.y));
    e = __fadd2_rn(__fadd2_rn(a, make_float2(-t.x, -t.y)), __fadd2_rn(b, make_float2(-bb.x, -bb.y)));
}

template <int RR, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) modesum_p2_kernel(const Mode32Group gd) {
    constexpr int G = 2, CS = 16;
    constexpr int HEADF = kRowHeadBytes / (int)sizeof(float);
    extern __shared__ __align__(16) uint4 smem16[];
    int it = 0;
    while (it + 1 < gd.nitems && (int64_t)blockIdx.x >= gd.tile_start[it + 1]) ++it;
    const Mode32Item &ip = gd.item[it];
    const float2 *__restrict__ fhat = static_cast<const float2 *>(ip.fhat);
    float2 *__restrict__ Qhat = static_cast<float2 *>(ip.Qhat);
    const float *__restrict__ W = static_cast<const float *>(ip.W);
    const int *__restrict__ tasks = ip.tasks;
    const int h = ip.h, M = ip.M, nhalf = ip.nhalf, wrow_max = ip.wrow_max;
    const int64_t n = ip.n;
    const int64_t cta0 = (int64_t)blockIdx.x - gd.tile_start[it];
    const int part = (int)(cta0 % ip.split);
    const int64_t tile = cta0 / ip.split;
    float4 *Fs = reinterpret_cast<float4 *>(smem16);                        // [kPad + nhalf + kPad][16]
    float *wsm = reinterpret_cast<float *>(Fs + (size_t)(nhalf + 2 * kPad) * CS);   // [warps][2][wrow_max]
    {
        // the tile's half spectrum as cell pairs (c, c + 16); zero guard rows
        const float2 *src = fhat + tile * (int64_t)nhalf * 32;
        const int rows = nhalf + 2 * kPad;
        for (int i = threadIdx.x; i < rows * CS; i += blockDim.x) {
            const int row = i / CS - kPad, pr = i % CS;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row >= 0 && row < nhalf) {
                const float2 x = src[(int64_t)row * 32 + pr], y = src[(int64_t)row * 32 + pr + 16];
                v = make_float4(x.x, y.x, x.y, y.y);
            }
            Fs[i] = v;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pr = lane % CS, grp = lane / CS;
    float *wbuf0 = wsm + (size_t)warp * 2 * wrow_max;
    float *wbuf1 = wbuf0 + wrow_max;
    const int vw = part * WARPS + warp;
    const int tbeg = tasks[vw], tend = tasks[vw + 1];
    const TaskRec *trec = reinterpret_cast<const TaskRec *>(tasks + 2 * WARPS * ip.split + 1);
    const float4 *F0 = Fs + (size_t)(kPad + h) * CS + pr;

    for (int t = tbeg; t < tend; ++t) {
        const TaskRec tk = trec[t];
        const int rowf = tk.rowf;
        const float *wsrc = W + tk.woff;
        float2 hre[RR], lre[RR], him[RR], lim[RR];
        P2Acc acc[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            hre[r] = lre[r] = him[r] = lim[r] = make_float2(0.f, 0.f);
            acc[r].re = acc[r].im = make_float2(0.f, 0.f);
        }
        const int k20 = tk.k20 + grp * RR;
        const int mbase0 = k20 - tk.l2lo - (RR - 1);
        stage_row(wbuf0, wsrc, rowf * (int)sizeof(float), lane);
        for (int i = 0; i < tk.nrows; ++i) {
            const float *wcur = (i & 1) ? wbuf1 : wbuf0;
            if (i + 1 < tk.nrows) {
                stage_row((i & 1) ? wbuf0 : wbuf1, wsrc + (size_t)(i + 1) * rowf, rowf * (int)sizeof(float), lane);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            const int4 hd = *reinterpret_cast<const int4 *>(wcur);
            if (hd.z > 0)
                row_pass_p2<RR, 1>(F0 + hd.x, F0 + hd.y, wcur + HEADF + 2 * grp * RR, tk.nblk * G, tk.l2lo, mbase0,
                                   acc);
            else
                row_pass_p2<RR, -1>(F0 + hd.x, F0 + hd.y, wcur + HEADF + 2 * grp * RR, tk.nblk * G, tk.l2lo, mbase0,
                                    acc);
            __syncwarp();
            if ((i & 3) == 3 || i + 1 == tk.nrows) {
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    float2 sm, e;
                    two_sum2(hre[r], acc[r].re, sm, e);
                    hre[r] = sm;
                    lre[r] = __fadd2_rn(lre[r], e);
                    two_sum2(him[r], acc[r].im, sm, e);
                    him[r] = sm;
                    lim[r] = __fadd2_rn(lim[r], e);
                    acc[r].re = acc[r].im = make_float2(0.f, 0.f);
                }
            }
        }
        const int64_t c0 = tile * 32 + pr, c1 = c0 + 16;
        float2 *out = Qhat + tile * (int64_t)nhalf * 32 + (int64_t)tk.orow * M * 32 + pr;
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const int k2 = k20 + r;
            if (grp * RR + r >= tk.rfirst && k2 <= h) {
                const float2 re = __fadd2_rn(hre[r], lre[r]), im = __fadd2_rn(him[r], lim[r]);
                if (c0 < n) out[(k2 + h) * 32] = make_float2(re.x, im.x);
                if (c1 < n) out[(k2 + h) * 32 + 16] = make_float2(re.y, im.y);
            }
        }
    }
}

// ---- FP32x2 form with one cell per lane ----------------------------------------
// The sums of modesum32_kernel (tiles of 32 cells, one cell per lane, RR
// outputs per thread, reflected and ramped task tables) with the complex
// product w f-hat_l b (b = f-hat_m from the window) split as
//   U = w b                 (one FP32x2 multiply: (w b_x, w b_y)),
//   P += U f_x, Q += U f_y  (two FP32x2 FMAs; f = f-hat_l, f_y negated for a
//                            conjugated value),
// so that Re = P_x - Q_y and Im = P_y + Q_x.  Three FP32x2 instructions per
// pair in place of six scalar ones, the same six FP32 operations: the kernel
// is bounded by the FMA pipe rather than by instruction issue.  The weights
// are read as in the scalar kernels (16 bytes = four outputs' weights; a
// broadcast 16-byte shared-memory load takes two wavefronts, so a stream of
// (w, w) pairs would make shared memory the bound).  P and Q are folded into the (hi, lo) pair of each output every
// four rows as (P_x - Q_y, P_y + Q_x); the sums differ in rounding from the
// scalar kernels', so the last partial wave of a batch stays on this kernel.
template <int RR, int WS, int PH, bool RAMP, int DIR>
__device__ __forceinline__ void block_pq(float2 (&win)[2 * RR], const float2 *__restrict__ mp, int mcs,
                                         const float2 *__restrict__ lp, int dcs,
                                         const float *__restrict__ wb, float2 (&P)[RR], float2 (&Q)[RR]) {
#pragma unroll
    for (int j = 0; j < (RAMP ? RR - 1 : RR); ++j) win[(j + PH * RR) & (2 * RR - 1)] = mp[j * mcs];
#pragma unroll
    for (int s = RAMP ? 1 : 0; s < RR; ++s) {
        const float2 fl = lp[s * dcs];
        const float fy = DIR > 0 ? fl.y : -fl.y;       // f-hat_l conjugated for DIR < 0
        const float2 fxx = make_float2(fl.x, fl.x), fyy = make_float2(fy, fy);
        // all products U first, then the P and then the Q updates: no FMA
        // waits on the multiply issued just before it
        float wv[RR];
#pragma unroll
        for (int q = 0; q < RR; q += 4)
            if (!RAMP || q < s) load_w4(wv + q, wb + s * WS + q);   // outputs q .. q + 3 before the ramp
        float2 u[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r)
            if (!RAMP || r < s) u[r] = __fmul2_rn(make_float2(wv[r], wv[r]), win[(r - s + RR - 1 + PH * RR) & (2 * RR - 1)]);
#pragma unroll
        for (int r = 0; r < RR; ++r)
            if (!RAMP || r < s) P[r] = __ffma2_rn(u[r], fxx, P[r]);
#pragma unroll
        for (int r = 0; r < RR; ++r)
            if (!RAMP || r < s) Q[r] = __ffma2_rn(u[r], fyy, Q[r]);
    }
}

// One row pair (as row_pass): the ramp block under the PH 1 naming, or the
// preload, then pairs of blocks (PH 0, PH 1) and a last PH 0.  mirror: the
// task of a reflected output block, read from the unreflected spectrum: every
// column index is negated, so f-hat_l and the window run the other way.
template <int RR, int WS, int CS, int DIR>
__device__ __forceinline__ void row_pass_pq(const float2 *__restrict__ rowl, const float2 *__restrict__ rowm,
                                            const float *__restrict__ wrow, int nblk, int l2lo, int mbase0,
                                            bool ramp, bool mirror, float2 (&P)[RR], float2 (&Q)[RR]) {
    float2 win[2 * RR];
    const int dcs = (mirror ? -DIR : DIR) * CS;          // between consecutive l_2
    const int mcs = mirror ? -CS : CS;                   // between consecutive window columns
    const float2 *mp = rowm + mbase0 * mcs;
    const float2 *lp = rowl + l2lo * dcs;
    int blk = 0;
    if (ramp) {
        block_pq<RR, WS, 1, true, DIR>(win, mp, mcs, lp, dcs, wrow, P, Q);
        mp -= RR * mcs;
        lp += RR * dcs;
        blk = 1;
    } else {
#pragma unroll
        for (int j = RR; j < 2 * RR - 1; ++j) win[j] = mp[j * mcs];
    }
    for (; blk + 1 < nblk; blk += 2) {
        block_pq<RR, WS, 0, false, DIR>(win, mp, mcs, lp, dcs, wrow + blk * RR * WS, P, Q);
        block_pq<RR, WS, 1, false, DIR>(win, mp - RR * mcs, mcs, lp + RR * dcs, dcs, wrow + (blk + 1) * RR * WS, P,
                                        Q);
        mp -= 2 * RR * mcs;
        lp += 2 * RR * dcs;
    }
    if (blk < nblk) block_pq<RR, WS, 0, false, DIR>(win, mp, mcs, lp, dcs, wrow + blk * RR * WS, P, Q);
}

// CELLS = 32: one cell per lane; reflected blocks are separate tasks (read
// mirrored).  CELLS = 16 (paired orientations, for grids whose 32-cell
// spectrum does not fit shared memory): lanes c and c + 16 hold cell c, the
// upper half running every task mirrored, i.e. the task's reflected twin with
// the same weights and control flow, so all lanes take the same outputs and
// the ramp applies; the table holds no reflected tasks and k_2 = 0 is the
// lower half's.
template <int RR, int WARPS, int CELLS>
__global__ void __launch_bounds__(WARPS * 32, WARPS <= 4 ? 3 : WARPS <= 8 ? 2 : 1) modesum_pq_kernel(const Mode32Group gd) {
    constexpr bool PAIRED = (CELLS == 16);
    constexpr int G = 32 / CELLS;                // CTAs per 32-cell tile
    constexpr int WS = RR;                       // floats per l_2 step
    constexpr int HEAD = kRowHeadBytes / (int)sizeof(float);
    extern __shared__ __align__(16) uint4 smem16[];
    int it = 0;
    while (it + 1 < gd.nitems && (int64_t)blockIdx.x >= gd.tile_start[it + 1]) ++it;
    const Mode32Item &ip = gd.item[it];
    const float2 *__restrict__ fhat = static_cast<const float2 *>(ip.fhat);
    float2 *__restrict__ Qhat = static_cast<float2 *>(ip.Qhat);
    const float *__restrict__ W = static_cast<const float *>(ip.W);
    const int *__restrict__ tasks = ip.tasks;
    const int h = ip.h, M = ip.M, nhalf = ip.nhalf, wrow_max = ip.wrow_max;
    const int64_t cta0 = (int64_t)blockIdx.x - gd.tile_start[it];
    const int part = (int)(cta0 % ip.split);
    const int64_t cta = cta0 / ip.split;
    const int64_t tile = cta / G;
    const int sub = (int)(cta % G);
    float2 *Fs = reinterpret_cast<float2 *>(smem16);                 // [kPad + nhalf + kPad][CELLS]
    float *wsm = reinterpret_cast<float *>(Fs + (size_t)(nhalf + 2 * kPad) * CELLS);
    stage_spectrum<float2, CELLS>(smem16, fhat, tile, sub, nhalf, M, false);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cell = lane % CELLS;
    const bool upper = PAIRED && lane >= CELLS;                      // runs every task mirrored
    float *wbuf0 = wsm + (size_t)warp * 2 * wrow_max;
    float *wbuf1 = wbuf0 + wrow_max;
    const int NW = WARPS * ip.split;                 // one phase: every task reads this spectrum
    int t = tasks[part * WARPS + warp], tend = tasks[part * WARPS + warp + 1];
    const TaskRec *trec = reinterpret_cast<const TaskRec *>(tasks + 2 * NW + 1);
    const float2 *F0 = Fs + (size_t)(kPad + h) * CELLS + cell;
    const bool valid = tile * 32 + sub * CELLS + cell < ip.n;
    float2 *const qt = Qhat + tile * (int64_t)nhalf * 32 + sub * CELLS + cell;

    for (; t < tend;) {
        const TaskRec tk = trec[t++];
        const int rowf = tk.rowf;
        const bool ramp = (tk.flags & kTaskRamp) != 0, mirror = ((tk.flags & kTaskRefl) != 0) != upper;
        const float *wsrc = W + tk.woff;
        float2 hi[RR], lo[RR], P[RR], Q[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) hi[r] = lo[r] = P[r] = Q[r] = make_float2(0.f, 0.f);
        const int mbase0 = tk.k20 - tk.l2lo - (RR - 1);
        stage_row(wbuf0, wsrc, rowf * (int)sizeof(float), lane);
        for (int i = 0; i < tk.nrows; ++i) {
            const float *wcur = (i & 1) ? wbuf1 : wbuf0;
            if (i + 1 < tk.nrows) {
                stage_row((i & 1) ? wbuf0 : wbuf1, wsrc + (size_t)(i + 1) * rowf, rowf * (int)sizeof(float), lane);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            const int4 hd = *reinterpret_cast<const int4 *>(wcur);
            if (hd.z > 0)
                row_pass_pq<RR, WS, CELLS, 1>(F0 + hd.x, F0 + hd.y, wcur + HEAD, tk.nblk, tk.l2lo, mbase0, ramp,
                                              mirror, P, Q);
            else
                row_pass_pq<RR, WS, CELLS, -1>(F0 + hd.x, F0 + hd.y, wcur + HEAD, tk.nblk, tk.l2lo, mbase0, ramp,
                                               mirror, P, Q);
            __syncwarp();
            if ((i & 3) == 3 || i + 1 == tk.nrows) {
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    // (re, im) TwoSum as FP32x2 operations: the scalar ones, pairwise
                    const float2 a = make_float2(P[r].x - Q[r].y, P[r].y + Q[r].x);
                    float2 sm, e;
                    two_sum2(hi[r], a, sm, e);
                    hi[r] = sm;
                    lo[r] = __fadd2_rn(lo[r], e);
                    P[r] = Q[r] = make_float2(0.f, 0.f);
                }
            }
        }
        if (valid) {
            const volatile TaskRec *tv = trec + (t - 1);
            const int orow = tv->orow, rfirst = tv->rfirst, flags = tv->flags, crow = tv->crow, k20 = tv->k20;
            float2 *out = qt + (int64_t)orow * M * 32;
            const bool refl = ((flags & kTaskRefl) != 0) != upper, cj = (flags & kTaskConj) != 0;
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int k2 = k20 + r;
                if (r >= rfirst && k2 <= h && !(upper && k2 == 0)) {
                    const float2 q = make_float2(hi[r].x + lo[r].x, hi[r].y + lo[r].y);
                    out[(refl ? h - k2 : k2 + h) * 32] = q;
                    if (cj && k2 > 0) qt[((int64_t)crow * M + h - k2) * 32] = make_float2(q.x, -q.y);
                }
            }
        }
    }
}

// ---- FP32X2 form: double-float arithmetic on the FP32 pipe ------------------
// Every value is an unevaluated sum hi + lo of two FP32 numbers (|lo| <= u |hi|).
// For each term w f-hat_l f-hat_m of eq. CF1 the product X = w f-hat_l is
// formed exactly in its high part (TwoProd: fmaf(a, b, -fl(a b)) is the exact
// rounding error of a b) with the low parts of w and f-hat_l added to its
// error; each of the four real products X b of the complex product is split
// exactly the same way, its high part enters the running sum by TwoSum (exact
// error), and every error and the cross terms with the low part of b
// accumulate in a second FP32 sum.  This is the compensated dot product
// ("Dot2") of Ogita, Rump and Oishi (2005), accurate as if computed in twice
// the working precision; the operations are pinned with the _rn intrinsics
// so the compiler cannot fuse them into FMAs that would break the exact splits.
// The real and imaginary parts run as the two lanes of FP32x2 instructions:
// every lane performs exactly the scalar operations in the scalar order
// (the products (-y) x of the imaginary part are formed as y (-x), the same
// value), so the result is that of the scalar form bit for bit.
struct X2Acc {
    float2 s;         // running sums of the high parts (real, imaginary)
    float2 c;         // accumulated errors and low-order terms
};

__device__ __forceinline__ float2 x2_neg(float2 a) { return make_float2(-a.x, -a.y); }

// acc += w a b with w = wh + wl (real), a = ah + al (conjugated for DIR < 0),
// b = bh + bl; bs, ls are bh and bl with their lanes exchanged.
template <int DIR>
__device__ __forceinline__ void x2_term(X2Acc &acc, float wh, float wl, float2 ah, float2 al, float2 bh,
                                        float2 bl, float2 bs, float2 ls) {
    // X = w a: high parts exact products, errors plus the low-part terms
    const float2 W = make_float2(wh, wh);
    const float2 X = __fmul2_rn(W, ah);
    float2 E = __ffma2_rn(W, ah, x2_neg(X));
    E = __ffma2_rn(make_float2(wl, wl), ah, E);
    E = __ffma2_rn(W, al, E);
    // with xi the imaginary part of X after the optional conjugation, yn = -xi:
    // X b = xx (bx, by) + (yn by, -yn bx)
    const float yn = DIR > 0 ? -X.y : X.y, en = DIR > 0 ? -E.y : E.y;
    const float2 XX = make_float2(X.x, X.x), YN = make_float2(yn, -yn);
    float2 sm, d;
    const float2 P = __fmul2_rn(XX, bh);
    const float2 qp = __ffma2_rn(XX, bh, x2_neg(P));
    two_sum2(acc.s, P, sm, d);
    acc.s = sm;
    float2 c = __fadd2_rn(qp, d);
    const float2 Q = __fmul2_rn(YN, bs);
    const float2 qq = __ffma2_rn(YN, bs, x2_neg(Q));
    two_sum2(acc.s, Q, sm, d);
    acc.s = sm;
    c = __fadd2_rn(c, __fadd2_rn(qq, d));
    acc.c = __fadd2_rn(acc.c, c);
    acc.c = __ffma2_rn(make_float2(E.x, E.x), bh, acc.c);
    acc.c = __ffma2_rn(make_float2(en, -en), bs, acc.c);
    acc.c = __ffma2_rn(XX, bl, acc.c);
    acc.c = __ffma2_rn(YN, ls, acc.c);
}

// RR consecutive FP32 weights (RR = 4: 16-byte aligned, RR = 2: 8-byte aligned).
template <int RR> __device__ __forceinline__ void load_wx(float *wv, const float *p) {
    if constexpr (RR == 4) {
        const float4 w4 = *reinterpret_cast<const float4 *>(p);
        wv[0] = w4.x;
        wv[1] = w4.y;
        wv[2] = w4.z;
        wv[3] = w4.w;
    } else {
        static_assert(RR == 2, "FP32X2 blocks hold 2 or 4 outputs per thread");
        const float2 w2 = *reinterpret_cast<const float2 *>(p);
        wv[0] = w2.x;
        wv[1] = w2.y;
    }
}

// One block of RR l_2 steps of the FP32X2 form: the window scheme of
// block_pass, with the high and low parts of each spectrum value LO elements
// apart in shared memory and the weights of step s at wb + s * 2 RT (high
// parts) and wb + s * 2 RT + RT (low parts).  The read direction of f-hat_l is
// chosen at run time (dcs = +/-CS, sgn = +/-1 on the imaginary parts):
// x2_term<+1> on the conjugated value performs exactly the
// operations of x2_term<-1> on the value read, each negated (rounding is
// symmetric), so the results are those of direction-specialised bodies with
// half the code (four specialised bodies overflow the instruction cache).
template <int RR, int CS, int RT, int PH>
__device__ __forceinline__ void block_pass_x2_rt(float2 (&wh)[2 * RR], float2 (&wl)[2 * RR],
                                                 const float2 *__restrict__ mp, const float2 *__restrict__ lp, int dcs,
                                                 float sgn, int LO, const float *__restrict__ wb, X2Acc (&acc)[RR]) {
#pragma unroll
    for (int j = 0; j < RR; ++j) {
        wh[(j + PH * RR) & (2 * RR - 1)] = mp[j * CS];
        wl[(j + PH * RR) & (2 * RR - 1)] = mp[j * CS + LO];
    }
#pragma unroll
    for (int s = 0; s < RR; ++s) {
        float2 ah = lp[s * dcs], al = lp[s * dcs + LO];
        ah.y *= sgn;
        al.y *= sgn;
        float whi[RR], wlo[RR];
        load_wx<RR>(whi, wb + s * 2 * RT);
        load_wx<RR>(wlo, wb + s * 2 * RT + RT);
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const int q = (r - s + RR - 1 + PH * RR) & (2 * RR - 1);
            x2_term<1>(acc[r], whi[r], wlo[r], ah, al, wh[q], wl[q], make_float2(wh[q].y, wh[q].x),
                       make_float2(wl[q].y, wl[q].x));
        }
    }
}

template <int RR, int CS, int RT>
__device__ __forceinline__ void row_pass_x2(const float2 *__restrict__ rowl, const float2 *__restrict__ rowm, int LO,
                                            const float *__restrict__ wrow, int nblk, int l2lo, int mbase0, int dir,
                                            X2Acc (&acc)[RR]) {
    float2 wh[2 * RR], wl[2 * RR];
    const int dcs = dir * CS;
    const float sgn = (float)dir;
    const float2 *mp = rowm + mbase0 * CS;
    const float2 *lp = rowl + l2lo * dcs;
#pragma unroll
    for (int j = RR; j < 2 * RR - 1; ++j) {
        wh[j] = mp[j * CS];
        wl[j] = mp[j * CS + LO];
    }
    int blk = 0;
    for (; blk + 1 < nblk; blk += 2) {
        block_pass_x2_rt<RR, CS, RT, 0>(wh, wl, mp, lp, dcs, sgn, LO, wrow + blk * RR * 2 * RT, acc);
        block_pass_x2_rt<RR, CS, RT, 1>(wh, wl, mp - RR * CS, lp + RR * dcs, dcs, sgn, LO,
                                        wrow + (blk + 1) * RR * 2 * RT, acc);
        mp -= 2 * RR * CS;
        lp += 2 * RR * dcs;
    }
    if (blk < nblk) block_pass_x2_rt<RR, CS, RT, 0>(wh, wl, mp, lp, dcs, sgn, LO, wrow + blk * RR * 2 * RT, acc);
}

// The FP32X2 mode sum: the task structure and shared-memory layout of
// modesum32_kernel on the FP64 tables (same tasks, same row pairs; a weight's
// 8 bytes hold its FP32 high and low parts).  Input: FP64 spectra in the tiled
// layout, split into FP32 high and low parts while they are staged; output:
// Q-hat rounded to FP32 (hi + lo), tiled layout.
template <int RR, int WARPS, int CELLS>
__global__ void __launch_bounds__(WARPS * 32, 1)
modesum_x2_kernel(const double2 *__restrict__ fhat, float2 *__restrict__ Qhat, const float *__restrict__ W,
                  const int *__restrict__ tasks, int h, int M, int nhalf, int wrow_max, int64_t n) {
    constexpr int G = 32 / CELLS;
    constexpr int RT = RR * G;
    constexpr int HEADF = kRowHeadBytes / (int)sizeof(float);
    extern __shared__ __align__(16) uint4 smem16[];
    const int64_t tile = (int64_t)blockIdx.x / G;
    const int sub = (int)(blockIdx.x % G);
    const int rows = nhalf + 2 * kPad;
    float2 *Fh = reinterpret_cast<float2 *>(smem16);              // [rows][CELLS] high parts
    float2 *Fl = Fh + (size_t)rows * CELLS;                       // [rows][CELLS] low parts
    float *wsm = reinterpret_cast<float *>(Fl + (size_t)rows * CELLS);   // [warps][2][2 wrow_max]
    const int LO = rows * CELLS;
    {
        const double2 *src = fhat + tile * (int64_t)nhalf * 32 + sub * CELLS;
        for (int i = threadIdx.x; i < rows * CELLS; i += blockDim.x) {
            const int row = i / CELLS - kPad, c = i % CELLS;
            float2 hv = make_float2(0.f, 0.f), lv = make_float2(0.f, 0.f);
            if (row >= 0 && row < nhalf) {
                const double2 x = src[(int64_t)row * 32 + c];
                hv.x = __double2float_rn(x.x);
                hv.y = __double2float_rn(x.y);
                lv.x = __double2float_rn(x.x - (double)hv.x);
                lv.y = __double2float_rn(x.y - (double)hv.y);
            }
            Fh[i] = hv;
            Fl[i] = lv;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cell = lane % CELLS, grp = lane / CELLS;
    float *wbuf0 = wsm + (size_t)warp * 4 * wrow_max;             // wrow_max counts 8-byte slots
    float *wbuf1 = wbuf0 + 2 * wrow_max;
    const int tbeg = tasks[warp], tend = tasks[warp + 1];
    const TaskRec *trec = reinterpret_cast<const TaskRec *>(tasks + 2 * WARPS + 1);
    const float2 *F0 = Fh + (size_t)(kPad + h) * CELLS + cell;

    for (int t = tbeg; t < tend; ++t) {
        const TaskRec tk = trec[t];
        const int rowb = tk.rowf * 8;                      // bytes per row pair
        const float *wsrc = W + 2 * (size_t)tk.woff;
        X2Acc acc[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) acc[r] = X2Acc{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        const int k20 = tk.k20 + grp * RR;
        const int mbase0 = k20 - tk.l2lo - (RR - 1);
        stage_row(wbuf0, wsrc, rowb, lane);
        for (int i = 0; i < tk.nrows; ++i) {
            const float *wcur = (i & 1) ? wbuf1 : wbuf0;
            if (i + 1 < tk.nrows) {
                stage_row((i & 1) ? wbuf0 : wbuf1, wsrc + (size_t)(i + 1) * 2 * tk.rowf, rowb, lane);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            const int4 hd = *reinterpret_cast<const int4 *>(wcur);
            row_pass_x2<RR, CELLS, RT>(F0 + hd.x, F0 + hd.y, LO, wcur + HEADF + grp * RR, tk.nblk * G, tk.l2lo,
                                       mbase0, hd.z > 0 ? 1 : -1, acc);
            __syncwarp();
        }
        const int64_t c = tile * 32 + sub * CELLS + cell;
        if (c < n) {
            float2 *out = Qhat + tile * (int64_t)nhalf * 32 + (int64_t)tk.orow * M * 32 + sub * CELLS + cell;
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int k2 = k20 + r;
                if (grp * RR + r >= tk.rfirst && k2 <= h)
                    out[(k2 + h) * 32] = __fadd2_rn(acc[r].s, acc[r].c);
            }
        }
    }
}

template <typename T> size_t smem_bytes(const GridView &g, int wrow_max, int v) {
    return 2 * sizeof(T) * (size_t)(g.nhalf + 2 * kPad) * kVariants[v].cells +
           sizeof(T) * (size_t)kVariants[v].warps * 2 * wrow_max;
}

}  // namespace

// Host part: weight streams and the task table, built once per modes handle.
double beta_host(const bz_modes *m, const int *l, const int *mm);

// Weight stream (with row-pair headers) and task table of one variant, with
// weights of type T; false if the grid is not covered by this variant (another
// variant or the generic kernel serves it).  With T = double and outX2 set, a
// second stream of the same byte layout for the FP32X2 form: the RT doubles of
// each l_2 step become RT FP32 high parts followed by RT FP32 low parts
// (hi = fl32(w), lo = fl32(w - hi)), headers copied as they are.
template <typename T>
static bool build_variant(bz_modes *m, int v, int &rc, void **outW, int **outT, int *outRowmax,
                          float **outX2 = nullptr, int **outSplit = nullptr) {
    constexpr int HEAD = kRowHeadBytes / (int)sizeof(T);
    const int R = variant_rt(v);                                // outputs per task (RT)
    const int kWarps = kVariants[v].warps;
    const int pack = kVariants[v].pack;                         // cells per lane
    rc = BZ_OK;
    const GridView &gv = m->g->v;
    const int d = gv.dim, h = gv.h, M = gv.M;
    if (!((d == 2 && gv.N <= 48) || (d == 3 && gv.N <= 16))) return false;
    // shared memory of the spectrum alone must leave room for the weight buffers
    if (2 * sizeof(T) * (size_t)(gv.nhalf + 2 * kPad) * kVariants[v].cells > 200 * 1024) return false;
    const int nb = (M + R - 1) / R;
    const int lo_col = -h - kPad, hi_col = h + kPad;         // addressable columns
    std::vector<TaskRec> tasks;
    std::vector<T> W;
    std::vector<float> X2;                                  // FP32X2 stream (T = double only)
    const bool want_x2 = outX2 != nullptr && sizeof(T) == 8;
    std::vector<double> stepw(R);
    std::vector<double> cost;
    std::vector<int> phase;                                 // 1: runs on the reflected spectrum
    // reflect: the FP32 variants with one cell per lane whose output blocks
    // fit the row compute k_2 < 0 as k_2 > 0 of the spectrum reflected in the
    // last axis (beta-hat is invariant under that reflection); ramped: with
    // one lane group and R dividing h + 1, every task starts with the ramp
    // block and no step is padding
    const int G = variant_groups(v);
    const bool reflect = sizeof(T) == 4 && variant_reflects(v, h);
    const bool ramped = reflect && G == 1 && (h + 1) % R == 0;
    const bool twins = reflect && kVariants[v].orient == 1;   // paired orientations need no reflected tasks
    // paired orientations compute k_2 < 0 in the mirrored half of every task:
    // only with blocks of k_2 >= 0 (else both halves would write one output)
    if (kVariants[v].orient == 2 && !reflect) return false;
    const int nmid = (d == 3) ? M : 1;                      // values of the middle index (3-D)
    struct Pair { int l[2], m[2]; };                         // leading indices of l and m
    for (int k1 = 0; k1 <= h; ++k1) {
        for (int i2 = 0; i2 < nmid; ++i2) {
            const int k2 = (d == 3) ? i2 - h : 0;
            const int orow = (d == 3) ? k1 * M + i2 : k1;
            std::vector<Pair> pairs;                         // row pairs visited for this output row
            for (int l1 = k1 - h; l1 <= k1 / 2; ++l1) {
                const int m1 = k1 - l1;
                if (d == 2) {
                    pairs.push_back({{l1, 0}, {m1, 0}});
                } else {
                    for (int l2 = std::max(-h, k2 - h); l2 <= std::min(h, k2 + h); ++l2)
                        pairs.push_back({{l1, l2}, {m1, k2 - l2}});
                }
            }
            // blocks of R consecutive last-axis outputs.  reflect: the blocks
            // start at 0, R, 2R, ... and cover k_2 >= 0; each is run a second
            // time on the reflected spectrum for k_2 <= 0 (same weights), except
            // in the k_1 = 0 row, whose k_2 < 0 outputs are the conjugates of its
            // k_2 > 0 ones.  Otherwise they tile [-h, h], the last one ending at
            // h (it may overlap the previous block, whose outputs it then does
            // not store) and a block wider than the row starting at -h.
            std::vector<int> starts;
            if (reflect) {
                for (int k = 0; k <= h; k += R) starts.push_back(k);
            } else {
                for (int b = 0; b < nb; ++b) starts.push_back(std::max(-h, std::min(-h + R * b, h - R + 1)));
            }
            int prev_end = -h - 1;
            for (const int k20 : starts) {
                const int k2last = k20 + R - 1;
                int l2lo = 0, nblk = 0, npad = 0;
                if (ramped) {
                    // one step before the lowest l_2 of output k20, through h:
                    // 2h + 2 - k20 steps, a multiple of R when R divides h + 1
                    l2lo = k20 - h - 1;
                    npad = 2 * h + 2 - k20;
                    nblk = npad / R;
                } else {
                    const int lo = std::max(-h, k20 - h), hi = std::min(h, k2last + h);
                    const int len = hi - lo + 1;
                    nblk = (len + R - 1) / R;
                    npad = nblk * R;
                    // place the padded range [l2lo, l2lo + npad - 1] so that every
                    // f-hat_l column and every window column k - l lies within kPad
                    // of [-h, h]
                    bool placed = false;
                    for (int cand = lo - (npad - len); cand <= lo && !placed; ++cand) {
                        const int last = cand + npad - 1;
                        if (cand < lo_col || last > hi_col) continue;
                        if (k20 - last < lo_col || k2last - cand > hi_col) continue;
                        l2lo = cand;
                        placed = true;
                    }
                    if (!placed) return false;
                }
                TaskRec t;
                t.orow = orow;
                t.k20 = k20;
                t.nrows = (int)pairs.size();
                t.l2lo = l2lo;
                t.nblk = nblk;
                t.woff = (int)W.size();
                t.rfirst = reflect ? 0 : std::max(0, prev_end + 1 - k20);
                t.rowf = HEAD + npad * R * (kVariants[v].wdup ? 2 : 1);
                t.flags = (ramped ? kTaskRamp : 0) | (twins && k1 == 0 ? kTaskConj : 0);
                t.crow = (d == 3) ? (M - 1 - i2) : 0;        // k_1 = 0: row of -k (middle index -k_2)
                t.pad2 = t.pad3 = 0;
                prev_end = k2last;
                for (const Pair &p : pairs) {
                    // row of l (that of -l read backwards when l_1 < 0) and row of m
                    const bool neg = p.l[0] < 0;
                    const int a1 = neg ? -p.l[0] : p.l[0], a2 = neg ? -p.l[1] : p.l[1];
                    const int lrow = (d == 3) ? a1 * M + (a2 + h) : a1;
                    const int mrow = (d == 3) ? p.m[0] * M + (p.m[1] + h) : p.m[0];
                    const int cs = kVariants[v].cells / pack;   // shared-memory entries per mode
                    const int head[4] = {lrow * M * cs, mrow * M * cs, neg ? -1 : 1, 0};
                    static_assert(sizeof head == kRowHeadBytes, "16-byte row header");
                    T hw[HEAD];
                    std::memcpy(hw, head, sizeof head);
                    for (int q = 0; q < HEAD; ++q) W.push_back(hw[q]);
                    if (want_x2) {
                        float hf[4];
                        std::memcpy(hf, head, sizeof head);
                        for (int q = 0; q < 4; ++q) X2.push_back(hf[q]);
                    }
                    for (int j = 0; j < npad; ++j) {
                        const int lz = l2lo + j;
                        for (int r = 0; r < R; ++r) {
                            const int kz = k20 + r, mz = kz - lz;
                            double w = 0.0;
                            if (kz <= h && lz >= -h && lz <= h && mz >= -h && mz <= h) {
                                int l[3], mm[3];
                                l[0] = p.l[0];
                                mm[0] = p.m[0];
                                if (d == 3) {
                                    l[1] = p.l[1];
                                    mm[1] = p.m[1];
                                }
                                l[d - 1] = lz;
                                mm[d - 1] = mz;
                                w = beta_host(m, l, mm);
                                if (p.l[0] < p.m[0]) w += beta_host(m, mm, l);
                            }
                            W.push_back((T)w);
                            if (kVariants[v].wdup) W.push_back((T)w);
                            stepw[r] = w;
                        }
                        if (want_x2) {
                            for (int r = 0; r < R; ++r) X2.push_back((float)stepw[r]);
                            for (int r = 0; r < R; ++r) X2.push_back((float)(stepw[r] - (double)(float)stepw[r]));
                        }
                    }
                }
                // evaluated pairs (a ramp skips R (R + 1) / 2 of each row pair's)
                const double c = (double)t.nrows * ((double)npad * R - (ramped ? R * (R + 1) / 2 : 0) + 2.0 * npad);
                tasks.push_back(t);
                cost.push_back(c);
                phase.push_back(0);
                if (twins && k1 > 0) {
                    TaskRec tr = t;                      // the same weights on the reflected spectrum
                    tr.flags = (t.flags & kTaskRamp) | kTaskRefl;
                    tr.rfirst = (k20 == 0) ? 1 : 0;      // k_2 = 0 is the unreflected task's
                    tasks.push_back(tr);
                    cost.push_back(c);
                    phase.push_back(kVariants[v].pq ? 0 : 1);   // the FP32x2 kernel reads it mirrored
                }
            }
        }
    }
    // longest-processing-time-first assignment of tasks to nw warps: the
    // offsets of each warp's list, then the task records
    auto make_table = [&](int nw) {
        std::vector<std::vector<int>> per(2 * nw);
        for (int ph = 0; ph < 2; ++ph) {
            std::vector<int> order;
            for (size_t i = 0; i < tasks.size(); ++i)
                if (phase[i] == ph) order.push_back((int)i);
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
            std::vector<double> load(nw, 0.0);
            for (int i : order) {
                int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                load[w] += cost[i];
                per[ph * nw + w].push_back(i);
            }
        }
        std::vector<int> t(2 * nw + 1 + tasks.size() * kTaskInts);
        int pos = 0;
        for (int q = 0; q < 2 * nw; ++q) {
            t[q] = pos;
            for (int i : per[q]) {
                std::memcpy(&t[2 * nw + 1 + (size_t)pos * kTaskInts], &tasks[i], sizeof(TaskRec));
                ++pos;
            }
        }
        t[2 * nw] = pos;
        return t;
    };
    const std::vector<int> tab = make_table(kWarps);
    int wrow_max = 0;
    for (auto &t : tasks) wrow_max = std::max(wrow_max, t.rowf);   // staging buffer: one row pair
    if (smem_bytes<T>(gv, wrow_max, v) > 227 * 1024) return false;   // does not fit
    T *dW = nullptr;
    int *dT = nullptr;
    float *dX = nullptr;
    cudaError_t e = dev_malloc(&dW, sizeof(T) * W.size());
    if (e == cudaSuccess) e = dev_malloc(&dT, sizeof(int) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(dW, W.data(), sizeof(T) * W.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dT, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && want_x2) {
        e = dev_malloc(&dX, sizeof(float) * X2.size());
        if (e == cudaSuccess) e = cudaMemcpy(dX, X2.data(), sizeof(float) * X2.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        dev_free(dW);
        dev_free(dT);
        dev_free(dX);
        rc = cuda_fail(e, "build_kernel_modes: weight stream");
        return false;
    }
    // tables for one tile split over S = 2, 4, 8 CTAs (S x kWarps warps; the
    // last partial wave of a launch of a 32-cell variant)
    if (outSplit) {
        for (int k = 0; k < kSplitTables && e == cudaSuccess; ++k) {
            const std::vector<int> ts = make_table(kWarps << (k + 1));
            e = dev_malloc(&outSplit[k], sizeof(int) * ts.size());
            if (e == cudaSuccess) e = cudaMemcpy(outSplit[k], ts.data(), sizeof(int) * ts.size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            for (int k = 0; k < kSplitTables; ++k) dev_free(outSplit[k]), outSplit[k] = nullptr;
            dev_free(dW);
            dev_free(dT);
            dev_free(dX);
            rc = cuda_fail(e, "build_kernel_modes: split task tables");
            return false;
        }
    }
    *outW = dW;
    *outT = dT;
    *outRowmax = wrow_max;
    if (want_x2) *outX2 = dX;
    return true;
}

bool modesum32_available(const bz_modes *m) { return m->d_W32 != nullptr; }

template <typename T, int RR, int WARPS, int CELLS, bool RTDIR = false>
static cudaError_t launch_instance(const Mode32Group &gd, size_t sm, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(modesum32_kernel<T, RR, WARPS, CELLS, RTDIR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    modesum32_kernel<T, RR, WARPS, CELLS, RTDIR><<<(unsigned)gd.tile_start[gd.nitems], WARPS * 32, sm, st>>>(gd);
    return cudaGetLastError();
}

template <int RR, int WARPS, int CELLS>
static cudaError_t launch_pq(const Mode32Group &gd, size_t sm, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(modesum_pq_kernel<RR, WARPS, CELLS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    modesum_pq_kernel<RR, WARPS, CELLS><<<(unsigned)gd.tile_start[gd.nitems], WARPS * 32, sm, st>>>(gd);
    return cudaGetLastError();
}

static cudaError_t launch_group(const Mode32Group &gd, int v, size_t sm, cudaStream_t st) {
    switch (v) {
        case 0: return launch_instance<float, 8, 16, 32, true>(gd, sm, st);
        case 1: return launch_instance<float, 4, 32, 32>(gd, sm, st);
        case 2: return launch_instance<float, 4, 16, 16>(gd, sm, st);
        case 3: return launch_instance<float, 4, 16, 8>(gd, sm, st);
        case 4: {
            cudaError_t e = cudaFuncSetAttribute(modesum_p2_kernel<4, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
            if (e != cudaSuccess) return e;
            modesum_p2_kernel<4, 16><<<(unsigned)gd.tile_start[gd.nitems], 16 * 32, sm, st>>>(gd);
            return cudaGetLastError();
        }
        case 5: return launch_pq<8, 12, 32>(gd, sm, st);
        case 6: return launch_pq<8, 16, 32>(gd, sm, st);
        case 7: return launch_pq<8, 16, 16>(gd, sm, st);
        case 8: return launch_pq<8, 8, 16>(gd, sm, st);
        case 9: return launch_pq<8, 4, 16>(gd, sm, st);
        default: return cudaErrorInvalidValue;
    }
}

static void fill_item(Mode32Item &it, const bz_modes *m, const void *W, const int *tasks, int rowmax,
                      const void *fhat, void *Qhat, int64_t n, int split = 1) {
    it.split = split;
    const GridView &gv = m->g->v;
    it.fhat = fhat;
    it.Qhat = Qhat;
    it.W = W;
    it.tasks = tasks;
    it.h = gv.h;
    it.M = gv.M;
    it.nhalf = (int)gv.nhalf;
    it.wrow_max = rowmax;
    it.n = n;
}

// CTAs of an instance of n cells: one per CELLS cells of each 32-cell tile.
static int64_t ctas_for(int v, int64_t n) {
    const int G = 32 / kVariants[v].cells;      // CTAs per 32-cell tile
    return ((n + 31) / 32) * G;
}

static cudaError_t launch_variant(const bz_modes *m, int v, const float2 *fhat, float2 *Qhat, int64_t n,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    Mode32Group gd;
    memset(&gd, 0, sizeof gd);
    gd.nitems = 1;
    fill_item(gd.item[0], m, m->var_W[v], m->var_task[v], m->var_rowmax[v], fhat, Qhat, n);
    gd.tile_start[0] = 0;
    gd.tile_start[1] = ctas_for(v, n);
    return launch_group(gd, v, smem_bytes<float>(m->g->v, m->var_rowmax[v], v), st);
}

// FP64 form: the same kernel on double spectra and weights, on 16-cell tiles
// (variant entry 2) or, where the double spectrum of 16 cells does not fit
// shared memory, on 8- or 4-cell tiles (entries 10, 11: 48^2, 16^3); no
// last-wave split.  The FP32X2 form runs on the same layout.
constexpr int kFp64Variants[3] = {2, 10, 11};

bool modesum64_available(const bz_modes *m) { return m->w64 != nullptr; }

cudaError_t launch_modesum64(const bz_modes *m, const double2 *fhat, double2 *Qhat, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (!m->w64) return cudaErrorInvalidValue;
    Mode32Group gd;
    memset(&gd, 0, sizeof gd);
    gd.nitems = 1;
    fill_item(gd.item[0], m, m->w64, m->task64, m->rowmax64, fhat, Qhat, n);
    gd.tile_start[0] = 0;
    gd.tile_start[1] = ctas_for(m->variant64, n);
    const size_t sm = smem_bytes<double>(m->g->v, m->rowmax64, m->variant64);
    if (m->variant64 == kFp64Variants[0]) return launch_instance<double, 4, 16, 16>(gd, sm, st);
    if (m->variant64 == kFp64Variants[1]) return launch_instance<double, 2, 8, 8>(gd, sm, st);
    if (m->variant64 == kFp64Variants[2]) return launch_instance<double, 2, 8, 4>(gd, sm, st);
    return cudaErrorInvalidValue;
}

// FP32X2 form on the FP64 layout (the entries of kFp64Variants).
bool modesum_x2_available(const bz_modes *m) { return m->wx2 != nullptr && m->variant64 >= 0; }

template <int RR, int WARPS, int CELLS>
static cudaError_t launch_x2_instance(const bz_modes *m, const double2 *fhat, float2 *Qhat, int64_t n, size_t sm,
                                      cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(modesum_x2_kernel<RR, WARPS, CELLS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const GridView &gv = m->g->v;
    modesum_x2_kernel<RR, WARPS, CELLS><<<(unsigned)ctas_for(m->variant64, n), WARPS * 32, sm, st>>>(
        fhat, Qhat, m->wx2, m->task64, gv.h, gv.M, (int)gv.nhalf, m->rowmax64, n);
    return cudaGetLastError();
}

cudaError_t launch_modesum_x2(const bz_modes *m, const double2 *fhat, float2 *Qhat, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (!modesum_x2_available(m)) return cudaErrorInvalidValue;
    // the FP64 layout's shared memory: spectra of 16 bytes per value (hi, lo
    // parts of FP32 instead of one double) and weight rows of 8-byte slots
    const size_t sm = smem_bytes<double>(m->g->v, m->rowmax64, m->variant64);
    if (m->variant64 == kFp64Variants[0]) return launch_x2_instance<4, 16, 16>(m, fhat, Qhat, n, sm, st);
    if (m->variant64 == kFp64Variants[1]) return launch_x2_instance<2, 8, 8>(m, fhat, Qhat, n, sm, st);
    if (m->variant64 == kFp64Variants[2]) return launch_x2_instance<2, 8, 4>(m, fhat, Qhat, n, sm, st);
    return cudaErrorInvalidValue;
}

static int sm_count();

// A launch over n cells ends with a partial wave of tiles; the SMs that run
// one tile fewer idle meanwhile.  With a 32-cell variant chosen by timing,
// the whole waves run one tile per CTA and the T remaining tiles are split
// over S = 2, 4 or 8 CTAs each (each CTA takes one part of the tile's tasks),
// S the largest with T S <= SM count; when no such S exists (T > SMs / 2)
// and the 16-cell variant fits the grid, the remaining tiles run on it (twice
// the CTAs, each half as long).  Every output is computed by one task in
// either case, with the same arithmetic (the one-cell-per-lane variants sum
// each output over the same terms in the same order), so the results do not
// depend on the split.  Returns the cells of the main part; *tail_v is the tail's variant
// (-1: no tail) and *tail_split its split.
int64_t modesum32_split(const bz_modes *m, int64_t n, int *tail_v, int *tail_split) {
    *tail_v = -1;
    *tail_split = 1;
    if (m->variant_fixed || kVariants[m->variant].cells != 32) return n;
    const int64_t sms = sm_count();
    const int64_t ntiles = (n + 31) / 32, full = (ntiles / sms) * sms;
    const int64_t T = ntiles - full;
    if (T == 0) return n;
    for (int k = kSplitTables - 1; k >= 0; --k) {
        const int S = 2 << k;
        if (T * S <= sms && m->var_task_split[m->variant][k]) {
            *tail_v = m->variant;
            *tail_split = S;
            return full * 32;
        }
    }
    // the 16-cell variant, if it sums every output in the order of this one
    if (!m->var_W[2] || kVariants[m->variant].pq ||
        variant_reflects(2, m->g->v.h) != variant_reflects(m->variant, m->g->v.h))
        return n;
    *tail_v = 2;
    return full * 32;
}

// CTAs per SM of a variant's kernel (its launch bounds: the FP32x2 kernels
// with 8 or 4 warps are built for 2 or 3 resident CTAs).
static int variant_ctas_per_sm(int v) {
    if (!kVariants[v].pq) return 1;
    return kVariants[v].warps <= 4 ? 3 : kVariants[v].warps <= 8 ? 2 : 1;
}

bool modesum32_tail_splits(const bz_modes *m) {
    return m->method == 0 && modesum32_available(m) && !m->variant_fixed && kVariants[m->variant].cells == 32 &&
           m->var_task_split[m->variant][0] != nullptr;
}

// A variant that holds several CTAs per SM fills only part of each SM in a
// launch of less than half a wave (and a lone wave loses about a sixth: all
// CTAs stage their spectra at once and the SMs empty unevenly).  Its sibling
// with one 16-warp CTA per SM runs the same tasks in the same order
// (bit-identical results), so launches of at most half a wave take it.
static int small_batch_variant(const bz_modes *m, int64_t n) {
    const int v = m->variant;
    if (m->variant_fixed || variant_ctas_per_sm(v) == 1) return v;
    if (n > (int64_t)sm_count() * variant_ctas_per_sm(v) * kVariants[v].cells / 2) return v;
    for (int s = 0; s < kNumVariants; ++s) {
        const Variant &a = kVariants[s], &b = kVariants[v];
        if (s != v && m->var_W[s] && variant_ctas_per_sm(s) == 1 && a.R == b.R && a.cells == b.cells &&
            a.pack == b.pack && a.wdup == b.wdup && a.pq == b.pq && a.orient == b.orient)
            return s;
    }
    return v;
}

bool modesum32_small_batches_fast(const bz_modes *m) {
    return m->method == 0 && modesum32_available(m) && small_batch_variant(m, 1) != m->variant;
}

int modesum32_wave_cells_per_sm(const bz_modes *m) {
    if (m->method != 0 || !modesum32_available(m)) return 32;
    return variant_ctas_per_sm(m->variant) * kVariants[m->variant].cells;
}

// One launch for the whole batch: the main part (one tile per CTA) and the
// last partial wave (split tiles, or the 16-cell variant) as two items.
cudaError_t launch_modesum32(const bz_modes *m, const float2 *fhat, float2 *Qhat, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int sv = small_batch_variant(m, n);
    if (sv != m->variant) return launch_variant(m, sv, fhat, Qhat, n, st);
    int tv = -1, ts = 1;
    const int64_t nm = modesum32_split(m, n, &tv, &ts);
    const int v = m->variant;
    if (tv >= 0 && tv != v) {
        // tail on another variant: two launches (different kernels)
        cudaError_t e = nm > 0 ? launch_variant(m, v, fhat, Qhat, nm, st) : cudaSuccess;
        const size_t off = (size_t)(nm / 32) * m->g->v.nhalf * 32;
        if (e == cudaSuccess) e = launch_variant(m, tv, fhat + off, Qhat + off, n - nm, st);
        return e;
    }
    Mode32Group gd;
    memset(&gd, 0, sizeof gd);
    gd.tile_start[0] = 0;
    int k = 0;
    if (nm > 0) {
        fill_item(gd.item[k], m, m->var_W[v], m->var_task[v], m->var_rowmax[v], fhat, Qhat, nm);
        gd.tile_start[k + 1] = gd.tile_start[k] + ctas_for(v, nm);
        ++k;
    }
    if (tv >= 0 && n > nm) {
        const size_t off = (size_t)(nm / 32) * m->g->v.nhalf * 32;
        int lg = 0;
        while ((2 << lg) != ts) ++lg;
        fill_item(gd.item[k], m, m->var_W[v], m->var_task_split[v][lg], m->var_rowmax[v], fhat + off, Qhat + off,
                  n - nm, ts);
        gd.tile_start[k + 1] = gd.tile_start[k] + ctas_for(v, n - nm) * ts;
        ++k;
    }
    gd.nitems = k;
    return launch_group(gd, v, smem_bytes<float>(m->g->v, m->var_rowmax[v], v), st);
}

cudaError_t launch_modesum32_part(const bz_modes *m, int v, const float2 *fhat, float2 *Qhat, int64_t n,
                                  cudaStream_t st) {
    return launch_variant(m, v, fhat, Qhat, n, st);
}

// Heterogeneous instances in one launch; all items must use the same kernel
// variant and be ordered as they should be scheduled (longest first);
// count <= kMaxGroup.
cudaError_t launch_modesum32_group(const bz_modes *const *ms, const float2 *const *fhat, float2 *const *Qhat,
                                   const int64_t *n, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (count > kMaxGroup) return cudaErrorInvalidValue;
    const int v = ms[0]->variant;
    Mode32Group gd;
    memset(&gd, 0, sizeof gd);
    gd.nitems = count;
    size_t sm = 0;
    int64_t ctas = 0;
    for (int i = 0; i < count; ++i) {
        if (ms[i]->variant != v) return cudaErrorInvalidValue;
        fill_item(gd.item[i], ms[i], ms[i]->var_W[v], ms[i]->var_task[v], ms[i]->var_rowmax[v], fhat[i], Qhat[i],
                  n[i]);
        gd.tile_start[i] = ctas;
        ctas += ctas_for(v, n[i]);
        sm = std::max(sm, smem_bytes<float>(ms[i]->g->v, ms[i]->var_rowmax[v], v));
    }
    gd.tile_start[count] = ctas;
    if (ctas == 0) return cudaSuccess;
    if (sm > 227 * 1024) return cudaErrorInvalidValue;
    return launch_group(gd, v, sm, st);
}

// ---- autotuner ------------------------------------------------------------
// Times every buildable variant once per (dimension, N, SM count) on a
// synthetic batch (zero spectra: the kernel's cost does not depend on the
// values) of twelve 32-cell tiles per SM and keeps the fastest.  Results are
// cached for the process and, when BZ_TUNE_CACHE names a file, in that file as
// lines "dim N sms variant" (variant = index + 1).
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tune;

// SM count of the current device (cached per device; 0 entries are unset).
static int sm_count() {
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

static void tune_file_load() {
    const char *path = getenv("BZ_TUNE_CACHE");
    if (!path) return;
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    int d, N, sms, id;
    while (fscanf(fp, "%d %d %d %d", &d, &N, &sms, &id) == 4) g_tune[std::make_tuple(d, N, sms)] = id - 1;
    fclose(fp);
}

static void tune_file_store(int d, int N, int sms, int v) {
    const char *path = getenv("BZ_TUNE_CACHE");
    if (!path) return;
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%d %d %d %d\n", d, N, sms, v + 1);
    fclose(fp);
}

static int autotune(bz_modes *m, int &rc) {
    rc = BZ_OK;
    const GridView &gv = m->g->v;
    int avail[kNumVariants], na = 0;
    for (int v = 0; v < kNumVariants; ++v)
        if (m->var_W[v]) avail[na++] = v;
    if (na == 1) return avail[0];
    const int sms = sm_count();
    const auto key = std::make_tuple(gv.dim, gv.N, sms);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune.empty()) tune_file_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end())
        for (int q = 0; q < na; ++q)
            if (avail[q] == it->second) return avail[q];
    // twelve 32-cell tiles per SM (several waves of every variant, so that
    // neither the tail nor a single wave decides); two rounds over the
    // variants, best of three launches each
    const int64_t n = (int64_t)12 * sms * 32;
    const size_t bytes = 2 * sizeof(float2) * (size_t)((n + 31) / 32) * gv.nhalf * 32;
    void *buf = nullptr;
    cudaError_t e = dev_malloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaMemset(buf, 0, bytes);
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best[kNumVariants];
    for (int q = 0; q < kNumVariants; ++q) best[q] = 1e30f;
    const float2 *fh = static_cast<const float2 *>(buf);
    float2 *qh = static_cast<float2 *>(buf) + bytes / (2 * sizeof(float2));
    for (int round = 0; round < 2 && e == cudaSuccess; ++round) {
        for (int q = 0; q < na && e == cudaSuccess; ++q) {
            const int v = avail[q];
            e = launch_variant(m, v, fh, qh, n, nullptr);              // warm-up
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(a, nullptr);
                if (e == cudaSuccess) e = launch_variant(m, v, fh, qh, n, nullptr);
                if (e == cudaSuccess) e = cudaEventRecord(b, nullptr);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (e == cudaSuccess) best[v] = std::min(best[v], ms);
            }
        }
    }
    int pick = avail[0];
    for (int q = 1; q < na; ++q)
        if (best[avail[q]] < best[pick]) pick = avail[q];
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    dev_free(buf);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "build_kernel_modes: autotune");
        return avail[0];
    }
    g_tune[key] = pick;
    tune_file_store(gv.dim, gv.N, sms, pick);
    return pick;
}

int modes_build_fp32_tables(bz_modes *m) {
    m->d_W32 = nullptr;
    m->d_task = nullptr;
    m->variant = 0;
    m->variant_fixed = 0;
    m->modesum_variant = 0;
    int rc = BZ_OK;
    bool any = false;
    for (int v = 0; v < kNumVariants; ++v) {
        m->var_W[v] = nullptr;
        m->var_task[v] = nullptr;
        m->var_rowmax[v] = 0;
        void *w = nullptr;
        for (int k = 0; k < kSplitTables; ++k) m->var_task_split[v][k] = nullptr;
        int **split = kVariants[v].cells == 32 ? m->var_task_split[v] : nullptr;
        if (build_variant<float>(m, v, rc, &w, &m->var_task[v], &m->var_rowmax[v], nullptr, split)) {
            m->var_W[v] = static_cast<float *>(w);
            any = true;
        }
        if (rc) return rc;
    }
    // FP64 tables (16-cell tiles) where the double spectrum fits shared memory
    m->w64 = nullptr;
    m->task64 = nullptr;
    m->rowmax64 = 0;
    m->variant64 = -1;
    m->wx2 = nullptr;
    for (int q = 0; q < 3 && m->variant64 < 0; ++q) {
        if (build_variant<double>(m, kFp64Variants[q], rc, &m->w64, &m->task64, &m->rowmax64, &m->wx2))
            m->variant64 = kFp64Variants[q];
        if (rc) return rc;
    }
    if (!any) return BZ_OK;
    const char *force = getenv("BZ_MODESUM_VARIANT");   // fixed choice (1-based id), no timing
    int v = -1;
    if (force) {
        const int id = atoi(force) - 1;
        if (id >= 0 && id < kNumVariants && m->var_W[id]) v = id;
    }
    m->variant_fixed = v >= 0;      // a fixed variant also serves the last partial wave
    if (v < 0) v = autotune(m, rc);
    if (rc) return rc;
    m->variant = v;
    m->d_W32 = m->var_W[v];
    m->d_task = m->var_task[v];
    m->w32_rowmax = m->var_rowmax[v];
    m->modesum_variant = v + 1;
    return BZ_OK;
}

}  // namespace bz
