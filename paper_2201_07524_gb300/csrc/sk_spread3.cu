// 3-D spreading and interpolation by column tasks (adjoint NFFT / NFFT steps
// of Eq. (fastsum) for d = 3).
//
// Points are sorted by bin (4 x 4 x 8 cells) and, inside a bin, by cell with
// the z axis fastest, so each xy-column of a bin (8 cells along z) is a
// contiguous range of points.  Every point of a column touches the same W x W
// rows of grid cells (W = 2m taps per dimension) over the z-cells of its own
// window, so a warp keeps the column's whole window -- W^2 rows by (8 + W - 1)
// z-cells -- in registers, two rows per lane for W = 8:
//
//   * one lane per point evaluates that point's 3W window weights into its
//     row of a per-warp table in shared memory; a column's points come in
//     non-decreasing z-offset (the sort key), so the points of equal offset
//     are consecutive rows and every segment of equal offset has
//     compile-time register indices;
//   * for each point, every lane scales its rows by the x (and y) weights and
//     adds (or, when interpolating, gathers) the W z-taps with plain FMAs;
//   * spreading flushes a finished column into the bin's shared-memory
//     sub-grid with shared-memory atomics (one per register, not one per tap),
//     and the block adds the sub-grid to the global grid once;
//   * interpolation runs a persistent grid whose warps take columns from a
//     global queue, loads each column's window from the grid once, reduces
//     each point's 32 lane partials through shared memory, and runs the FP64
//     epilogue with one lane per point.
#include <algorithm>
#include <type_traits>
#include <utility>

#include "sk_internal.cuh"
#include "sk_device.cuh"

namespace sk {

template <int W, typename T = float> struct Col3 {
    static constexpr int BX = 4, BY = 4, BZ = 8;
    static constexpr int NCOL = BX * BY;
    static constexpr int SX = BX + W - 1, SY = BY + W - 1, SZ = BZ + W - 1;
    static constexpr int E = SZ;                       // z-cells of a column window
    static constexpr int ROWS = W * W;
    static constexpr int Q = (ROWS + 31) / 32;         // rows per lane
    // Table row of a point: wz | wx | wy, each padded to whole 16-byte vectors.
    static constexpr int VEC = 16 / int(sizeof(T));    // entries per 16-byte vector
    static constexpr int WP = (W + VEC - 1) / VEC * VEC;
    static constexpr int WZ = 0, WX = WP, WY = 2 * WP;
    // an odd number of 16-byte vectors per row keeps the vector stores of 8
    // consecutive lanes on distinct banks
    static constexpr int NV = (3 * WP) / VEC;
    static constexpr int STRIDE = (NV % 2 == 1 ? NV : NV + 1) * VEC;
    // FP32 spreading adds, after wz | wx | wy, the z-weights shifted by one
    // slot (0, wz[0], ..., wz[W-1], 0), for points at an odd z-offset (packed
    // taps, below); its rows are STRIDE_S apart
    static constexpr int WZS = 3 * WP;
    static constexpr int NS = (W + 2 + VEC - 1) / VEC * VEC;
    static constexpr int NVS = (3 * WP + NS) / VEC;
    static constexpr int STRIDE_S = (NVS % 2 == 1 ? NVS : NVS + 1) * VEC;
    static constexpr int EP = (BZ + W) / 2;           // z-cell pairs of a column window (E rounded up)
    static constexpr int SUB = SX * SY * SZ;
    // 16-byte-aligned z-chunks covering a column window: the window starts
    // LEAD entries into the first chunk
    static constexpr int ZA = (W / 2 - 1 + VEC - 1) / VEC * VEC;   // window start = z0 - (m-1) = z0 - ZA + LEAD
    static constexpr int LEAD = ZA - (W / 2 - 1);
    static constexpr int NCHUNK = (LEAD + E + VEC - 1) / VEC;
};

constexpr int kWarps = 8;         // warps per interpolation block
constexpr int kSpreadWarps = 8;   // warps per spreading block (one block per bin task)
// Row stride of the per-warp table of lane partials (a multiple of 4 floats, so
// a point's row is read with 16-byte loads; 36 keeps those loads conflict-free).
constexpr int kRedStride = 36;


// N values to 16-byte aligned shared memory with vector stores.
template <typename T, int N>
__device__ __forceinline__ void store_vec(T* dst, const T (&v)[N]) {
    if (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < N; k += 4)
            *reinterpret_cast<float4*>(dst + k) = make_float4(float(v[k]), k + 1 < N ? float(v[k + 1]) : 0.f,
                                                              k + 2 < N ? float(v[k + 2]) : 0.f,
                                                              k + 3 < N ? float(v[k + 3]) : 0.f);
    } else {
#pragma unroll
        for (int k = 0; k < N; k += 2)
            *reinterpret_cast<double2*>(dst + k) = make_double2(double(v[k]), k + 1 < N ? double(v[k + 1]) : 0.0);
    }
}

// Coordinates (and weight) of the point a lane will evaluate next, loaded one
// batch ahead so the global-load latency overlaps the current batch.
template <typename T>
struct Prefetch {
    T u0, u1, u2;
    double w;
    __device__ __forceinline__ void load(const T* c0, const T* c1, const T* c2, const double* wv, int p, bool ok) {
        if (ok) {
            u0 = c0[p];
            u1 = c1[p];
            u2 = c2[p];
            w = wv ? wv[p] : 1.0;
        }
    }
};

template <int W, typename T>
__device__ __forceinline__ void load_wz(const T* row, T (&wz)[W]) {
    if (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < W; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(row + k);
            wz[k] = v.x;
            if (k + 1 < W) wz[k + 1] = v.y;
            if (k + 2 < W) wz[k + 2] = v.z;
            if (k + 3 < W) wz[k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < W; k += 2) {
            const double2 v = *reinterpret_cast<const double2*>(row + k);
            wz[k] = v.x;
            if (k + 1 < W) wz[k + 1] = v.y;
        }
    }
}

template <int W, int Q, int E, int DZ0, typename T>
__device__ __forceinline__ void add_taps(T (&acc)[Q][E], const T (&a)[Q], const T (&wz)[W]) {
#pragma unroll
    for (int k = 0; k < W; ++k) {
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q][DZ0 + k] = fma(a[q], wz[k], acc[q][DZ0 + k]);
    }
}

// The column window of a lane's rows from the grid, as 16-byte vectors: chunk
// c of row q covers z = zc + VEC c ... zc + VEC c + VEC - 1 (zc is 16-byte
// aligned); chunks outside [0, n) read as zero (n is a multiple of VEC).
template <int W, typename T, int Q, int E>
__device__ __forceinline__ void load_window(T (&win)[Q][E], const T* __restrict__ grid, int n, int gx0, int gy0,
                                            int zc, const int (&ri)[Q], const int (&rj)[Q], const bool (&rv)[Q]) {
    using G = Col3<W, T>;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const T* grow = grid + (int64_t(gx0 + ri[q]) * n + (gy0 + rj[q])) * n;
#pragma unroll
        for (int c = 0; c < G::NCHUNK; ++c) {
            const int z = zc + c * G::VEC;
            T v[G::VEC];
            if (rv[q] && z >= 0 && z < n) {
                if (sizeof(T) == 4) {
                    const float4 f = __ldg(reinterpret_cast<const float4*>(grow + z));
                    v[0] = f.x;
                    v[1 % G::VEC] = f.y;
                    v[2 % G::VEC] = f.z;
                    v[3 % G::VEC] = f.w;
                } else {
                    const double2 f = __ldg(reinterpret_cast<const double2*>(grow + z));
                    v[0] = f.x;
                    v[1 % G::VEC] = f.y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < G::VEC; ++k) v[k] = T(0);
            }
#pragma unroll
            for (int k = 0; k < G::VEC; ++k) {
                const int e = c * G::VEC + k - G::LEAD;
                if (e >= 0 && e < E) win[q][e] = v[k];
            }
        }
    }
}

// Lanes owning a row (i, j) of the W x W column window: row lane + 32 q.
template <int W, int Q>
__device__ __forceinline__ void lane_rows(int lane, int (&ri)[Q], int (&rj)[Q], bool (&rv)[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = lane + 32 * q;
        rv[q] = r < W * W;
        ri[q] = rv[q] ? r / W : 0;
        rj[q] = rv[q] ? r % W : 0;
    }
}

template <int W, int Q, typename T>
__device__ __forceinline__ void row_products(const T* row, const int (&ri)[Q], const int (&rj)[Q],
                                             const bool (&rv)[Q], T (&av)[Q]) {
    using G = Col3<W, T>;
    if (32 % W == 0 && (W * W) % 32 == 0) {
        // every row of a lane has the same j (row = lane + 32 q, 32 a multiple of W)
        const T wy = row[G::WY + rj[0]];
#pragma unroll
        for (int q = 0; q < Q; ++q) av[q] = row[G::WX + ri[0] + q * (32 / W)] * wy;
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) av[q] = rv[q] ? row[G::WX + ri[q]] * row[G::WY + rj[q]] : T(0);
    }
}

// ------------------------------------------------------------ sorted batches
// The plan sorts points by (bin, cell inside the bin) with the z axis
// fastest, from the same rounded coordinates the kernels floor, so the
// points of a column -- and of every batch of 32 consecutive ones -- come in
// non-decreasing z-offset: lane l's point is table row l, and the points of
// equal offset are consecutive rows (a segment, counted with one ballot).

// With 32 a multiple of W and W^2 a multiple of 32, all rows of a lane share
// j = lane % W, and its x-taps are i = lane / W + q (32 / W), q < Q.  The
// lane then leaves wy[j] out of its partial (the batch reduction applies
// it), and the table stores wx permuted so that a lane's Q values are
// adjacent: position (i % (32 / W)) Q + i / (32 / W) holds wx[i].
template <int W>
struct SharedJ {
    static constexpr bool value = (32 % W == 0) && ((W * W) % 32 == 0);
};

template <int W, int Q>
__host__ __device__ constexpr int wx_slot(int i) {
    return (i % (32 / W)) * Q + i / (32 / W);
}

// Table row of a point of a sorted batch: wz (times `scale`), wx (permuted
// when SharedJ), wy.
template <int W, typename T, bool SHIFTED = false>
__device__ __forceinline__ void fill_row_sorted(T* row, T u0, T u1, T u2, T scale, const WindowPoly& wp) {
    using G = Col3<W, T>;
    int f;
    T w[W];
    window_poly<W, T>(u0, wp, T(1), f, w);
    if constexpr (SharedJ<W>::value) {
        T wpm[W];
#pragma unroll
        for (int i = 0; i < W; ++i) wpm[wx_slot<W, G::Q>(i)] = w[i];
        store_vec<T, W>(row + G::WX, wpm);
    } else {
        store_vec<T, W>(row + G::WX, w);
    }
    window_poly<W, T>(u1, wp, T(1), f, w);
    store_vec<T, W>(row + G::WY, w);
    window_poly<W, T>(u2, wp, scale, f, w);
    store_vec<T, W>(row + G::WZ, w);
    if constexpr (SHIFTED) {
        T ws[G::NS];
#pragma unroll
        for (int k = 0; k < G::NS; ++k) ws[k] = (k >= 1 && k <= W) ? w[k >= 1 && k <= W ? k - 1 : 0] : T(0);
        store_vec<T, G::NS>(row + G::WZS, ws);
    }
}

// A lane's Q adjacent (permuted) x-weights.
template <int Q, typename T>
__device__ __forceinline__ void load_wx(const T* src, T (&x)[Q]) {
    if constexpr (Q == 2 && sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(src);
        x[0] = v.x;
        x[1] = v.y;
    } else if constexpr (Q == 2 && sizeof(T) == 8) {
        const double2 v = *reinterpret_cast<const double2*>(src);
        x[0] = v.x;
        x[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) x[q] = src[q];
    }
}

// The W z-taps of one row from the point's window offset DZ0.
template <int W, int E, int DZ0, typename T>
__device__ __forceinline__ T row_taps(const T (&w)[E], const T (&wz)[W]) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < W; ++k) s = fma(w[DZ0 + k], wz[k], s);
    return s;
}

// One point's lane partial: sum over the lane's rows of (x or x*y weight) times its z-taps.
template <int W, int Q, int E, int DZ0, typename T>
__device__ __forceinline__ T point_partial(const T (&win)[Q][E], const T* row, int i0, const int (&ri)[Q],
                                           const int (&rj)[Q], const bool (&rv)[Q]) {
    using G = Col3<W, T>;
    T wz[W];
    load_wz<W, T>(row + G::WZ, wz);
    T av[Q];
    if constexpr (SharedJ<W>::value) {
        load_wx<Q, T>(row + G::WX + i0 * Q, av);
    } else {
        row_products<W, Q, T>(row, ri, rj, rv, av);
    }
    T r = T(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) r = fma(av[q], row_taps<W, E, DZ0, T>(win[q], wz), r);
    return r;
}

// Rows [p, pe) of the sorted batch, all at z-offset DZ0, two at a time.
template <int W, int Q, int E, int DZ0, typename T>
__device__ __forceinline__ void interp_rows(const T (&win)[Q][E], const T* wt, T* rd, int lane, int p, int pe, int i0,
                                            const int (&ri)[Q], const int (&rj)[Q], const bool (&rv)[Q]) {
    using G = Col3<W, T>;
    for (; p + 1 < pe; p += 2) {
        const T d0 = point_partial<W, Q, E, DZ0, T>(win, wt + p * G::STRIDE, i0, ri, rj, rv);
        const T d1 = point_partial<W, Q, E, DZ0, T>(win, wt + (p + 1) * G::STRIDE, i0, ri, rj, rv);
        rd[p * kRedStride + lane] = d0;
        rd[(p + 1) * kRedStride + lane] = d1;
    }
    if (p < pe) rd[p * kRedStride + lane] = point_partial<W, Q, E, DZ0, T>(win, wt + p * G::STRIDE, i0, ri, rj, rv);
}

// Segment DZ0 of a sorted batch: its rows start at `first`, which advances
// past them.
template <int W, int Q, int E, int DZ0, typename T>
__device__ __forceinline__ void interp_segment_sorted(const T (&win)[Q][E], const T* wt, T* rd, int lane, int mydz,
                                                      int& first, int i0, const int (&ri)[Q], const int (&rj)[Q],
                                                      const bool (&rv)[Q]) {
    const int cnt = __popc(__ballot_sync(0xffffffffu, mydz == DZ0));
    interp_rows<W, Q, E, DZ0, T>(win, wt, rd, lane, first, first + cnt, i0, ri, rj, rv);
    first += cnt;
}

template <int W, int Q, int E, typename T, int... DZ>
__device__ __forceinline__ void interp_sorted(const T (&win)[Q][E], const T* wt, T* rd, int lane, int mydz, int i0,
                                              const int (&ri)[Q], const int (&rj)[Q], const bool (&rv)[Q],
                                              std::integer_sequence<int, DZ...>) {
    int first = 0;
    (interp_segment_sorted<W, Q, E, DZ, T>(win, wt, rd, lane, mydz, first, i0, ri, rj, rv), ...);
}

// Spreading of rows [p, pe) of a sorted batch, all at z-offset DZ0: the
// lane's rows get (x y weight) times the point's scaled z-taps.
template <int W, int Q, typename T>
__device__ __forceinline__ void row_weights_sorted(const T* row, int i0, int j0, const int (&ri)[Q], const int (&rj)[Q],
                                                   const bool (&rv)[Q], T (&av)[Q]) {
    using G = Col3<W, T>;
    if constexpr (SharedJ<W>::value) {
        load_wx<Q, T>(row + G::WX + i0 * Q, av);
        const T wy = row[G::WY + j0];
#pragma unroll
        for (int q = 0; q < Q; ++q) av[q] *= wy;
    } else {
        row_products<W, Q, T>(row, ri, rj, rv, av);
    }
}

template <int W, int Q, int E, int DZ0, typename T>
__device__ __forceinline__ void spread_rows(T (&acc)[Q][E], const T* wt, int p, int pe, int i0, int j0,
                                            const int (&ri)[Q], const int (&rj)[Q], const bool (&rv)[Q]) {
    using G = Col3<W, T>;
    for (; p + 1 < pe; p += 2) {
        const T* r0 = wt + p * G::STRIDE;
        const T* r1 = r0 + G::STRIDE;
        T av0[Q], av1[Q], wz0[W], wz1[W];
        row_weights_sorted<W, Q, T>(r0, i0, j0, ri, rj, rv, av0);
        load_wz<W, T>(r0 + G::WZ, wz0);
        row_weights_sorted<W, Q, T>(r1, i0, j0, ri, rj, rv, av1);
        load_wz<W, T>(r1 + G::WZ, wz1);
        add_taps<W, Q, E, DZ0, T>(acc, av0, wz0);
        add_taps<W, Q, E, DZ0, T>(acc, av1, wz1);
    }
    if (p < pe) {
        const T* r0 = wt + p * G::STRIDE;
        T av0[Q], wz0[W];
        row_weights_sorted<W, Q, T>(r0, i0, j0, ri, rj, rv, av0);
        load_wz<W, T>(r0 + G::WZ, wz0);
        add_taps<W, Q, E, DZ0, T>(acc, av0, wz0);
    }
}

template <int W, int Q, int E, int DZ0, typename T>
__device__ __forceinline__ void spread_segment_sorted(T (&acc)[Q][E], const T* wt, int mydz, int& first, int i0,
                                                      int j0, const int (&ri)[Q], const int (&rj)[Q],
                                                      const bool (&rv)[Q]) {
    const int cnt = __popc(__ballot_sync(0xffffffffu, mydz == DZ0));
    spread_rows<W, Q, E, DZ0, T>(acc, wt, first, first + cnt, i0, j0, ri, rj, rv);
    first += cnt;
}

template <int W, int Q, int E, typename T, int... DZ>
__device__ __forceinline__ void spread_sorted(T (&acc)[Q][E], const T* wt, int mydz, int i0, int j0,
                                              const int (&ri)[Q], const int (&rj)[Q], const bool (&rv)[Q],
                                              std::integer_sequence<int, DZ...>) {
    int first = 0;
    (spread_segment_sorted<W, Q, E, DZ, T>(acc, wt, mydz, first, i0, j0, ri, rj, rv), ...);
}

// Packed taps (FP32 spreading): the lane's accumulators are pairs of adjacent
// z-cells (2t, 2t+1), and one packed FMA (FFMA2) adds two z-taps of a row.  A
// point at an even z-offset DZ0 takes its W z-weights as W/2 pairs into pairs
// DZ0/2 ...; one at an odd offset takes the shifted copy (0, wz[0], ...,
// wz[W-1], 0) as W/2 + 1 pairs into pairs (DZ0-1)/2 ...: W/2 or W/2 + 1
// packed FMAs per row in place of W.
template <int W, int Q, int EP, int DZ0>
__device__ __forceinline__ void add_taps_packed(float2 (&acc)[Q][EP], const float (&a)[Q], const float* row) {
    using G = Col3<W, float>;
    constexpr bool ODD = DZ0 % 2 == 1;
    constexpr int NP = ODD ? W / 2 + 1 : W / 2;
    constexpr int P0 = ODD ? (DZ0 - 1) / 2 : DZ0 / 2;
    const float* src = row + (ODD ? G::WZS : G::WZ);
    float2 wz2[NP];
#pragma unroll
    for (int t = 0; t < NP; t += 2) {
        const float4 v = *reinterpret_cast<const float4*>(src + 2 * t);
        wz2[t] = make_float2(v.x, v.y);
        if (t + 1 < NP) wz2[t + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const float2 a2 = make_float2(a[q], a[q]);
#pragma unroll
        for (int t = 0; t < NP; ++t) acc[q][P0 + t] = __ffma2_rn(a2, wz2[t], acc[q][P0 + t]);
    }
}

template <int W, int Q, int EP, int DZ0>
__device__ __forceinline__ void spread_rows_packed(float2 (&acc)[Q][EP], const float* wt, int p, int pe, int i0,
                                                   int j0, const int (&ri)[Q], const int (&rj)[Q],
                                                   const bool (&rv)[Q]) {
    using G = Col3<W, float>;
    for (; p + 1 < pe; p += 2) {
        const float* r0 = wt + p * G::STRIDE_S;
        const float* r1 = r0 + G::STRIDE_S;
        float av0[Q], av1[Q];
        row_weights_sorted<W, Q, float>(r0, i0, j0, ri, rj, rv, av0);
        row_weights_sorted<W, Q, float>(r1, i0, j0, ri, rj, rv, av1);
        add_taps_packed<W, Q, EP, DZ0>(acc, av0, r0);
        add_taps_packed<W, Q, EP, DZ0>(acc, av1, r1);
    }
    if (p < pe) {
        const float* r0 = wt + p * G::STRIDE_S;
        float av0[Q];
        row_weights_sorted<W, Q, float>(r0, i0, j0, ri, rj, rv, av0);
        add_taps_packed<W, Q, EP, DZ0>(acc, av0, r0);
    }
}

template <int W, int Q, int EP, int DZ0>
__device__ __forceinline__ void spread_segment_packed(float2 (&acc)[Q][EP], const float* wt, int mydz, int& first,
                                                      int i0, int j0, const int (&ri)[Q], const int (&rj)[Q],
                                                      const bool (&rv)[Q]) {
    const int cnt = __popc(__ballot_sync(0xffffffffu, mydz == DZ0));
    spread_rows_packed<W, Q, EP, DZ0>(acc, wt, first, first + cnt, i0, j0, ri, rj, rv);
    first += cnt;
}

template <int W, int Q, int EP, int... DZ>
__device__ __forceinline__ void spread_packed(float2 (&acc)[Q][EP], const float* wt, int mydz, int i0, int j0,
                                              const int (&ri)[Q], const int (&rj)[Q], const bool (&rv)[Q],
                                              std::integer_sequence<int, DZ...>) {
    int first = 0;
    (spread_segment_packed<W, Q, EP, DZ>(acc, wt, mydz, first, i0, j0, ri, rj, rv), ...);
}

// Kernel sum of the point in table row `pos`: its 32 lane partials, times
// wy[j] per lane group when the lanes left it out.
template <int W, typename T>
__device__ __forceinline__ T batch_sum(const T* rd, const T* row, int pos) {
    using G = Col3<W, T>;
    const T* pr = rd + pos * kRedStride;
    if constexpr (SharedJ<W>::value) {
        T g[W];
#pragma unroll
        for (int j = 0; j < W; ++j) g[j] = T(0);
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int l = 0; l < 32; l += 4) {
                const float4 v = *reinterpret_cast<const float4*>(pr + l);
                g[(l + 0) % W] += v.x;
                g[(l + 1) % W] += v.y;
                g[(l + 2) % W] += v.z;
                g[(l + 3) % W] += v.w;
            }
        } else {
#pragma unroll
            for (int l = 0; l < 32; l += 2) {
                const double2 v = *reinterpret_cast<const double2*>(pr + l);
                g[(l + 0) % W] += v.x;
                g[(l + 1) % W] += v.y;
            }
        }
        T wy[W];
        load_wz<W, T>(row + G::WY, wy);
        T t = T(0);
#pragma unroll
        for (int j = 0; j < W; ++j) t = fma(wy[j], g[j], t);
        return t;
    } else {
        T t0 = T(0), t1 = T(0);
#pragma unroll
        for (int l = 0; l < 32; l += 2) {
            t0 += pr[l];
            t1 += pr[l + 1];
        }
        return t0 + t1;
    }
}

template <int W, typename T>
__global__ void __launch_bounds__(kSpreadWarps * 32, sizeof(T) == 4 ? (W <= 8 ? 3 : 2) : (W <= 6 ? 2 : 1))
    k_spread3_col(SpreadArgs a) {
    using G = Col3<W, T>;
    constexpr int Q = G::Q, E = G::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sub = reinterpret_cast<T*>(smem_raw);
    T* tab = sub + ((G::SUB + 3) / 4) * 4;
    __shared__ int col_next;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool PACK = sizeof(T) == 4;   // packed taps (FP32)
    constexpr int RS = PACK ? G::STRIDE_S : G::STRIDE;
    T* wt = tab + warp * 32 * RS;

    const int bin = a.tasks[3 * blockIdx.x], col0 = a.tasks[3 * blockIdx.x + 1], col1 = a.tasks[3 * blockIdx.x + 2];
    const int bz = bin % a.nb[2], by = (bin / a.nb[2]) % a.nb[1], bx = bin / (a.nb[2] * a.nb[1]);
    for (int c = threadIdx.x; c < G::SUB; c += blockDim.x) sub[c] = T(0);
    if (threadIdx.x == 0) col_next = col0 + kSpreadWarps;
    __syncthreads();

    const T* c0 = static_cast<const T*>(a.coord[0]);
    const T* c1 = static_cast<const T*>(a.coord[1]);
    const T* c2 = static_cast<const T*>(a.coord[2]);
    int ri[Q], rj[Q];
    bool rv[Q];
    lane_rows<W, Q>(lane, ri, rj, rv);
    const int z0 = bz * G::BZ;
    const int64_t kbase = int64_t(bin) * (G::NCOL * G::BZ);

    int col = col0 + warp;
    while (col < col1) {
        const int start = a.key_start[kbase + col * G::BZ];
        const int end = a.key_start[kbase + (col + 1) * G::BZ];
        if (start < end) {
            // accumulators: T[Q][E], or (packed) float2[Q][EP] over the same z-cells
            using Acc = typename std::conditional<PACK, float2[Q][G::EP], T[Q][E]>::type;
            Acc acc;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if constexpr (PACK) {
#pragma unroll
                    for (int t = 0; t < G::EP; ++t) acc[q][t] = make_float2(0.f, 0.f);
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[q][e] = T(0);
                }
            }
            Prefetch<T> pf;
            pf.load(c0, c1, c2, a.w, start + lane, lane < end - start);
            for (int base = start; base < end; base += 32) {
                const int cnt = min(32, end - base);
                const int mydz = lane < cnt ? int(floor(pf.u2)) - z0 : -1;
                const int pos = lane;   // a column's points are ordered by z-offset (the sort key)
                if (lane < cnt) fill_row_sorted<W, T, PACK>(wt + pos * RS, pf.u0, pf.u1, pf.u2, T(pf.w), a.wp);
                pf.load(c0, c1, c2, a.w, base + 32 + lane, base + 32 + lane < end);
                __syncwarp();
                if constexpr (PACK)
                    spread_packed<W, Q, G::EP>(acc, wt, mydz, lane / W, lane % W, ri, rj, rv,
                                               std::make_integer_sequence<int, G::BZ>{});
                else
                    spread_sorted<W, Q, E, T>(acc, wt, mydz, lane / W, lane % W, ri, rj, rv,
                                              std::make_integer_sequence<int, G::BZ>{});
                __syncwarp();
            }
            const int cx = col / G::BY, cy = col % G::BY;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (!rv[q]) continue;
                T* srow = sub + ((cx + ri[q]) * G::SY + (cy + rj[q])) * G::SZ;
                if constexpr (PACK) {
#pragma unroll
                    for (int t = 0; t < G::EP; ++t) {
                        if (acc[q][t].x != 0.f) atomicAdd(srow + 2 * t, acc[q][t].x);
                        if (2 * t + 1 < E && acc[q][t].y != 0.f) atomicAdd(srow + 2 * t + 1, acc[q][t].y);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (acc[q][e] != T(0)) atomicAdd(srow + e, acc[q][e]);
                }
            }
        }
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&col_next, 1);
        col = __shfl_sync(0xffffffffu, nxt, 0);
    }
    __syncthreads();

    T* grid = static_cast<T*>(a.grid);
    const int n = a.n_os;
    const int ox = bx * G::BX - (W / 2 - 1), oy = by * G::BY - (W / 2 - 1), oz = z0 - (W / 2 - 1);
    for (int c = threadIdx.x; c < G::SUB; c += blockDim.x) {
        const T v = sub[c];
        if (v == T(0)) continue;
        const int lz = c % G::SZ, ly = (c / G::SZ) % G::SY, lx = c / (G::SZ * G::SY);
        const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
        if (gx < 0 || gx >= n || gy < 0 || gy >= n || gz < 0 || gz >= n) continue;
        atomicAdd(&grid[(int64_t(gx) * n + gy) * n + gz], v);
    }
}


// A queue entry: its (bin, column) code and the column's points [start, end).
struct ColumnRef {
    int code = 0, start = 0, end = 0;
};

template <int W, typename T>
__device__ __forceinline__ ColumnRef column_ref(const InterpArgs& a, int c) {
    using G = Col3<W, T>;
    ColumnRef r;
    if (c >= a.ncols) return r;
    r.code = a.cols[c];
    const int64_t k0 = int64_t(r.code / G::NCOL) * (G::NCOL * G::BZ) + (r.code % G::NCOL) * G::BZ;
    r.start = a.key_start[k0];
    r.end = a.key_start[k0 + G::BZ];
    return r;
}

// Interpolation with a persistent grid: each warp takes columns from a global
// queue (most points first), so the load balances at column granularity
// whatever the number of bins.  The next entry is taken, and its first batch
// of coordinates requested, while the current column is processed.
template <int W, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (W <= 8 ? 3 : 2) : (W <= 6 ? 2 : 1))
    k_interp3_col(InterpArgs a, Epilogue e) {
    using G = Col3<W, T>;
    constexpr int Q = G::Q, E = G::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    T* red = tab + kWarps * 32 * G::STRIDE;
    __shared__ unsigned warps_done;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* wt = tab + warp * 32 * G::STRIDE;
    T* rd = red + warp * 32 * kRedStride;

    if (threadIdx.x == 0) warps_done = 0u;
    __syncthreads();
    const T* c0 = static_cast<const T*>(a.coord[0]);
    const T* c1 = static_cast<const T*>(a.coord[1]);
    const T* c2 = static_cast<const T*>(a.coord[2]);
    const T* grid = static_cast<const T*>(a.grid);
    const int n = a.n_os;
    int ri[Q], rj[Q];
    bool rv[Q];
    lane_rows<W, Q>(lane, ri, rj, rv);
    double sq = 0.0, bad = 0.0, dot = 0.0;

    int c = queue_take(a.queue, lane);
    ColumnRef cur = column_ref<W, T>(a, c);
    Prefetch<T> pf;
    EpiPrefetch ep;
    pf.load(c0, c1, c2, nullptr, cur.start + lane, lane < cur.end - cur.start);
    ep.load(e, cur.start + lane, lane < cur.end - cur.start);
    while (c < a.ncols) {
        const int cn = queue_take(a.queue, lane);
        const ColumnRef nxt = column_ref<W, T>(a, cn);
        // the column's cell offsets: bin (bx, by, bz), column (cx, cy) inside it
        const int bin = cur.code / G::NCOL, col = cur.code % G::NCOL;
        const int bz = bin % a.nb[2], by = (bin / a.nb[2]) % a.nb[1], bx = bin / (a.nb[2] * a.nb[1]);
        const int z0 = bz * G::BZ;
        T win[Q][E];
        load_window<W, T>(win, grid, n, bx * G::BX + col / G::BY - (W / 2 - 1), by * G::BY + col % G::BY - (W / 2 - 1),
                          z0 - G::ZA, ri, rj, rv);
        for (int base = cur.start; base < cur.end; base += 32) {
            const int cnt = min(32, cur.end - base);
            const int mydz = lane < cnt ? int(floor(pf.u2)) - z0 : -1;
            const int pos = lane;   // a column's points are ordered by z-offset (the sort key)
            if (lane < cnt) fill_row_sorted<W, T>(wt + pos * G::STRIDE, pf.u0, pf.u1, pf.u2, T(1), a.wp);
            const EpiPrefetch epc = ep;
            // the next batch: this column's, else the next column's first
            const bool more = base + 32 < cur.end;
            const int nb = more ? base + 32 : nxt.start;
            const int ne = more ? cur.end : nxt.end;
            pf.load(c0, c1, c2, nullptr, nb + lane, nb + lane < ne);
            ep.load(e, nb + lane, nb + lane < ne);
            __syncwarp();
            interp_sorted<W, Q, E, T>(win, wt, rd, lane, mydz, lane / W, ri, rj, rv,
                                      std::make_integer_sequence<int, G::BZ>{});
            __syncwarp();
            if (lane < cnt)
                epi_point_pre(e, base + lane, double(batch_sum<W, T>(rd, wt + pos * G::STRIDE, pos)), epc.q, epc.a, sq,
                              bad, dot);
            __syncwarp();
        }
        c = cn;
        cur = nxt;
    }
    queue_leave(a.queue, lane);
    epi_finish_warps(e, sq, bad, dot, &warps_done);
}

// ------------------------------------------------------------ 2-D strips
// The 2-D interpolation on the CUDA cores (FP64 plans, or SK_KERNELS_SIMT)
// follows the same plan with one axis fewer.  A bin is a strip of
// BX = 33 - W x-cells by BY y-cells; every point of it touches x-rows
// x0 - (m-1) ... x0 + BX + m - 2, exactly 32 rows, so lane l owns row
// x0 - (m-1) + l over the E = BY + W - 1 y-cells of the strip's window, in
// registers.  Inside a bin the points are sorted by y-cell first, so a batch
// of 32 comes in non-decreasing y-offset (segments with compile-time
// register indices, as in 3-D).  For one point, the W lanes whose rows lie in
// its x-window take wx[lane - dx] and gather its W y-taps.  Tasks are runs of
// at most kStripMaxPts points of one bin, taken by warps from a queue (most
// points first); each point's lane partials are reduced through shared
// memory and the FP64 epilogue runs with one lane per point.
template <int W, typename T>
struct Strip2 {
    static constexpr int BX = 33 - W, BY = kStripBy;
    static constexpr int E = BY + W - 1;
    static constexpr int VEC = 16 / int(sizeof(T));
    static constexpr int WP = (W + VEC - 1) / VEC * VEC;
    static constexpr int WX = 0, WY = WP;
    static constexpr int NV = (2 * WP) / VEC;
    static constexpr int STRIDE = (NV % 2 == 1 ? NV : NV + 1) * VEC;
};

// Table row of a 2-D point: wx (times `scale`) and wy; returns the point's
// x-cell and y-cell.
template <int W, typename T>
__device__ __forceinline__ void fill_row2(T* row, T u0, T u1, T scale, const WindowPoly& wp, int& fx, int& fy) {
    using G = Strip2<W, T>;
    T w[W];
    window_poly<W, T>(u0, wp, scale, fx, w);
    store_vec<T, W>(row + G::WX, w);
    window_poly<W, T>(u1, wp, T(1), fy, w);
    store_vec<T, W>(row + G::WY, w);
}

// The x-weight lane `lane` takes from a point whose x-window starts dx rows
// into the strip's window (0 outside it).
template <int W, typename T>
__device__ __forceinline__ T lane_wx(const T* row, int lane, int dx) {
    const int off = lane - dx;
    return (off >= 0 && off < W) ? row[Strip2<W, T>::WX + off] : T(0);
}

template <int W, int E, int DY0, typename T>
__device__ __forceinline__ void strip_interp_segment(const T (&win)[E], const T* wt, const int* dxs, T* rd, int lane,
                                                     int mydy, int& first) {
    using G = Strip2<W, T>;
    const int cnt = __popc(__ballot_sync(0xffffffffu, mydy == DY0));
    for (int p = first; p < first + cnt; ++p) {
        const T* row = wt + p * G::STRIDE;
        const T ax = lane_wx<W, T>(row, lane, dxs[p]);
        T wy[W];
        load_wz<W, T>(row + G::WY, wy);
        T sacc = T(0);
#pragma unroll
        for (int k = 0; k < W; ++k) sacc = fma(win[DY0 + k], wy[k], sacc);
        rd[p * kRedStride + lane] = ax * sacc;
    }
    first += cnt;
}

template <int W, int E, typename T, int... DY>
__device__ __forceinline__ void strip_interp(const T (&win)[E], const T* wt, const int* dxs, T* rd, int lane, int mydy,
                                             std::integer_sequence<int, DY...>) {
    int first = 0;
    (strip_interp_segment<W, E, DY, T>(win, wt, dxs, rd, lane, mydy, first), ...);
}

// ------------------------------------------------------------ 2-D columns
// 2-D spreading by columns of a strip bin, the 2-D counterpart of
// k_spread3_col: a column is one x-cell of the bin (its BY cells along y, each
// a contiguous range of sorted points), and every point of it touches the
// same W x-rows of the grid.  A half-warp covers the column's window, lane
// i < W owning x-row i over the E = BY + W - 1 y-cells in registers; the two
// half-warps take alternate points of each cell, so one FMA instruction does
// the W y-taps of two points on 2 W of the 32 lanes (a strip layout, one point
// on all 32 lanes of which W are in its x-window, was 9 % slower).  A
// point's y-cell inside the bin is its cell's, so every cell is a segment
// with compile-time register indices.  Columns go to the block's warps; a
// finished column is added (both halves summed) into the bin's shared-memory
// sub-grid with shared-memory atomics, and the block adds the sub-grid to the
// global grid once.
template <int W, typename T>
struct Col2 {
    static constexpr int BX = 33 - W, BY = kStripBy;
    static constexpr int SX = BX + W - 1, SY = BY + W - 1, E = SY;
    static constexpr int SUB = SX * SY;
    static constexpr int VEC = 16 / int(sizeof(T));
    static constexpr int WP = (W + VEC - 1) / VEC * VEC;
    static constexpr int WX = 0, WY = WP;
    static constexpr int NV = (2 * WP) / VEC;
    static constexpr int STRIDE = (NV % 2 == 1 ? NV : NV + 1) * VEC;
    // FP32: after wx | wy the y-weights shifted by one slot (0, wy[0], ...,
    // wy[W-1], 0) for points at an odd y-offset (packed taps); rows STRIDE_S apart
    static constexpr int WYS = 2 * WP;
    static constexpr int NS = (W + 2 + VEC - 1) / VEC * VEC;
    static constexpr int NVS = (2 * WP + NS) / VEC;
    static constexpr int STRIDE_S = (NVS % 2 == 1 ? NVS : NVS + 1) * VEC;
    static constexpr int EP = (E + 1) / 2;         // y-cell pairs of the window
};

// Packed taps (FP32): one table row into the lane's row as pairs of adjacent
// y-cells, W/2 packed FMAs at an even y-offset DY, W/2 + 1 (the shifted copy)
// at an odd one.
template <int W, int EP, int DY>
__device__ __forceinline__ void col2_row_packed(float2 (&acc)[EP], const float* row, float ax) {
    using G = Col2<W, float>;
    constexpr bool ODD = DY % 2 == 1;
    constexpr int NP = ODD ? W / 2 + 1 : W / 2;
    constexpr int P0 = ODD ? (DY - 1) / 2 : DY / 2;
    const float* src = row + (ODD ? G::WYS : G::WY);
    float2 w2[NP];
#pragma unroll
    for (int t = 0; t < NP; t += 2) {
        const float4 v = *reinterpret_cast<const float4*>(src + 2 * t);
        w2[t] = make_float2(v.x, v.y);
        if (t + 1 < NP) w2[t + 1] = make_float2(v.z, v.w);
    }
    const float2 a2 = make_float2(ax, ax);
#pragma unroll
    for (int t = 0; t < NP; ++t) acc[P0 + t] = __ffma2_rn(a2, w2[t], acc[P0 + t]);
}

template <int W, int EP, int DY>
__device__ __forceinline__ void col2_segment_packed(float2 (&acc)[EP], const float* wt, int row_i, int h, int mydy,
                                                    int& first) {
    using G = Col2<W, float>;
    const int cnt = __popc(__ballot_sync(0xffffffffu, mydy == DY));
    const bool lane_ok = row_i < W;
    for (int q = h; q - h < cnt; q += 2) {
        const bool ok = q < cnt;
        const float* row = wt + (first + (ok ? q : 0)) * G::STRIDE_S;
        col2_row_packed<W, EP, DY>(acc, row, (ok && lane_ok) ? row[G::WX + row_i] : 0.f);
    }
    first += cnt;
}

template <int W, int EP, int... DY>
__device__ __forceinline__ void col2_segments_packed(float2 (&acc)[EP], const float* wt, int row_i, int h, int mydy,
                                                     std::integer_sequence<int, DY...>) {
    int first = 0;
    (col2_segment_packed<W, EP, DY>(acc, wt, row_i, h, mydy, first), ...);
}

// One table row's taps into the lane's row: x-weight `ax` (zero for lanes
// outside the window or without a row) times the W y-weights, at offset DY.
template <int W, int E, int DY, typename T>
__device__ __forceinline__ void col2_row(T (&acc)[E], const T* row, T ax) {
    using G = Col2<W, T>;
    T wy[W];
    load_wz<W, T>(row + G::WY, wy);
#pragma unroll
    for (int k = 0; k < W; ++k) acc[DY + k] = fma(ax, wy[k], acc[DY + k]);
}

// The table rows [first, first + cnt) (all of y-cell offset DY): half-warp h
// takes rows first + h, first + h + 2, ...; the loop bounds are the same for
// the whole warp.
template <int W, int E, int DY, typename T>
__device__ __forceinline__ void col2_segment(T (&acc)[E], const T* wt, int row_i, int h, int mydy, int& first) {
    using G = Col2<W, T>;
    const int cnt = __popc(__ballot_sync(0xffffffffu, mydy == DY));
    const bool lane_ok = row_i < W;
    for (int q = h; q - h < cnt; q += 2) {
        const bool ok = q < cnt;
        const T* row = wt + (first + (ok ? q : 0)) * G::STRIDE;
        col2_row<W, E, DY, T>(acc, row, (ok && lane_ok) ? row[G::WX + row_i] : T(0));
    }
    first += cnt;
}

template <int W, int E, typename T, int... DY>
__device__ __forceinline__ void col2_segments(T (&acc)[E], const T* wt, int row_i, int h, int mydy,
                                              std::integer_sequence<int, DY...>) {
    int first = 0;
    (col2_segment<W, E, DY, T>(acc, wt, row_i, h, mydy, first), ...);
}

// Column c's cells (c < c1): lane ly < BY gets cell ly's first point and count.
template <int BX, int BY>
__device__ __forceinline__ void col2_cells(const int* __restrict__ ks, int64_t kbase, int c, int c1, int lane, int& cs,
                                           int& cn) {
    cs = 0;
    cn = 0;
    if (c < c1 && lane < BY) {
        const int64_t k = kbase + lane * BX + c;
        cs = ks[k];
        cn = ks[k + 1] - cs;
    }
}

template <int W, typename T>
__global__ void __launch_bounds__(kSpreadWarps * 32, sizeof(T) == 4 ? (W <= 12 ? 4 : 3) : 2)
    k_spread2_col(SpreadArgs a) {
    using G = Col2<W, T>;
    constexpr int E = G::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sub = reinterpret_cast<T*>(smem_raw);
    T* tab = sub + ((G::SUB + 3) / 4) * 4;
    __shared__ int col_next;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = lane >> 4, row_i = lane & 15;
    constexpr bool PACK = sizeof(T) == 4;   // packed taps (FP32)
    constexpr int RS = PACK ? G::STRIDE_S : G::STRIDE;
    T* wt = tab + warp * 32 * RS;

    const int bin = a.tasks[3 * blockIdx.x], col0 = a.tasks[3 * blockIdx.x + 1], col1 = a.tasks[3 * blockIdx.x + 2];
    const int bx = bin / a.nb[1], by = bin - (bin / a.nb[1]) * a.nb[1];
    for (int c = threadIdx.x; c < G::SUB; c += blockDim.x) sub[c] = T(0);
    if (threadIdx.x == 0) col_next = col0 + kSpreadWarps;
    __syncthreads();

    const T* c0 = static_cast<const T*>(a.coord[0]);
    const T* c1 = static_cast<const T*>(a.coord[1]);
    const int64_t kbase = int64_t(bin) * (G::BX * G::BY);
    int col = col0 + warp;
    while (col < col1) {
        int cs, cn;
        col2_cells<G::BX, G::BY>(a.key_start, kbase, col, col1, lane, cs, cn);
        // the column's points before each cell's end (an inclusive scan)
        int incl = cn;
#pragma unroll
        for (int o = 1; o < G::BY; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, G::BY - 1);
        if (total > 0) {
            using Acc = typename std::conditional<PACK, float2[G::EP], T[E]>::type;
            Acc acc;
            if constexpr (PACK) {
#pragma unroll
                for (int t = 0; t < G::EP; ++t) acc[t] = make_float2(0.f, 0.f);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = T(0);
            }
            for (int base = 0; base < total; base += 32) {
                // lane's point: ordinal base + lane of the column, in cell ly
                const int o = base + lane;
                int ly = 0;
#pragma unroll
                for (int c = 0; c < G::BY - 1; ++c) ly += (o >= __shfl_sync(0xffffffffu, incl, c)) ? 1 : 0;
                const int start = __shfl_sync(0xffffffffu, cs, ly);
                const int before = __shfl_sync(0xffffffffu, incl - cn, ly);
                const int mydy = o < total ? ly : -1;
                if (o < total) {
                    const int p = start + (o - before);
                    T w[W];
                    int f;
                    window_poly<W, T>(c0[p], a.wp, T(a.w[p]), f, w);
                    store_vec<T, W>(wt + lane * RS + G::WX, w);
                    window_poly<W, T>(c1[p], a.wp, T(1), f, w);
                    store_vec<T, W>(wt + lane * RS + G::WY, w);
                    if constexpr (PACK) {
                        T ws[G::NS];
#pragma unroll
                        for (int k = 0; k < G::NS; ++k) ws[k] = (k >= 1 && k <= W) ? w[k >= 1 && k <= W ? k - 1 : 0] : T(0);
                        store_vec<T, G::NS>(wt + lane * RS + G::WYS, ws);
                    }
                }
                __syncwarp();
                if constexpr (PACK)
                    col2_segments_packed<W, G::EP>(acc, wt, row_i, h, mydy, std::make_integer_sequence<int, G::BY>{});
                else
                    col2_segments<W, E, T>(acc, wt, row_i, h, mydy, std::make_integer_sequence<int, G::BY>{});
                __syncwarp();
            }
            // both halves' partial sums of row row_i into the sub-grid
            T* srow = sub + (col + row_i) * G::SY;
            if constexpr (PACK) {
#pragma unroll
                for (int t = 0; t < G::EP; ++t) {
                    const float vx = acc[t].x + __shfl_xor_sync(0xffffffffu, acc[t].x, 16);
                    const float vy = acc[t].y + __shfl_xor_sync(0xffffffffu, acc[t].y, 16);
                    if (h == 0 && row_i < W) {
                        if (vx != 0.f) atomicAdd(srow + 2 * t, vx);
                        if (2 * t + 1 < E && vy != 0.f) atomicAdd(srow + 2 * t + 1, vy);
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const T v = acc[e] + __shfl_xor_sync(0xffffffffu, acc[e], 16);
                    if (h == 0 && row_i < W && v != T(0)) atomicAdd(srow + e, v);
                }
            }
        }
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&col_next, 1);
        col = __shfl_sync(0xffffffffu, nxt, 0);
    }
    __syncthreads();

    T* grid = static_cast<T*>(a.grid);
    const int n = a.n_os;
    const int ox = bx * G::BX - (W / 2 - 1), oy = by * G::BY - (W / 2 - 1);
    for (int c = threadIdx.x; c < G::SUB; c += blockDim.x) {
        const T v = sub[c];
        if (v == T(0)) continue;
        const int ly = c % G::SY, lx = c / G::SY;
        const int gx = ox + lx, gy = oy + ly;
        if (gx < 0 || gx >= n || gy < 0 || gy >= n) continue;
        atomicAdd(&grid[int64_t(gx) * n + gy], v);
    }
}

template <int W, typename T>
__global__ void __launch_bounds__(256) k_interp2_strip(InterpArgs a, Epilogue e) {
    using G = Strip2<W, T>;
    constexpr int E = G::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    T* red = tab + kWarps * 32 * G::STRIDE;
    int* dxall = reinterpret_cast<int*>(red + kWarps * 32 * kRedStride);
    __shared__ unsigned warps_done;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* wt = tab + warp * 32 * G::STRIDE;
    T* rd = red + warp * 32 * kRedStride;
    int* dxs = dxall + warp * 32;
    if (threadIdx.x == 0) warps_done = 0u;
    __syncthreads();
    const T* c0 = static_cast<const T*>(a.coord[0]);
    const T* c1 = static_cast<const T*>(a.coord[1]);
    const T* grid = static_cast<const T*>(a.grid);
    const int n = a.n_os;
    double sq = 0.0, bad = 0.0, dot = 0.0;
    for (int t = queue_take(a.queue, lane); t < a.nstasks; t = queue_take(a.queue, lane)) {
        const int bin = a.stasks[3 * t], start = a.stasks[3 * t + 1], end = a.stasks[3 * t + 2];
        const int x0 = (bin / a.nb[1]) * G::BX, y0 = (bin % a.nb[1]) * G::BY;
        // the lane's row of the strip's window
        T win[E];
        {
            const int xr = x0 - (W / 2 - 1) + lane;
            const bool okx = xr >= 0 && xr < n;
            const T* g = grid + int64_t(okx ? xr : 0) * n;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int yr = y0 - (W / 2 - 1) + k;
                win[k] = (okx && yr >= 0 && yr < n) ? __ldg(g + yr) : T(0);
            }
        }
        for (int base = start; base < end; base += 32) {
            const int cnt = min(32, end - base);
            int mydy = -1;
            double q = 0.0, am = 0.0;
            if (lane < cnt) {
                const int p = base + lane;
                int fx, fy;
                fill_row2<W, T>(wt + lane * G::STRIDE, c0[p], c1[p], T(1), a.wp, fx, fy);
                dxs[lane] = fx - x0;
                mydy = fy - y0;
                if (e.mode != EPI_APPLY) {
                    q = e.scal[p];
                    am = e.marg[p];
                }
            }
            __syncwarp();
            strip_interp<W, E, T>(win, wt, dxs, rd, lane, mydy, std::make_integer_sequence<int, G::BY>{});
            __syncwarp();
            if (lane < cnt) {
                T tsum = T(0);
                const T* pr = rd + lane * kRedStride;
#pragma unroll 8
                for (int l = 0; l < 32; ++l) tsum += pr[l];
                epi_point_pre(e, base + lane, double(tsum), q, am, sq, bad, dot);
            }
            __syncwarp();
        }
    }
    queue_leave(a.queue, lane);
    epi_finish_warps(e, sq, bad, dot, &warps_done);
}

// ------------------------------------------------------------------ dispatch
template <int W, typename T>
size_t spread3_smem() {
    using G = Col3<W, T>;
    constexpr int RS = sizeof(T) == 4 ? G::STRIDE_S : G::STRIDE;
    return (size_t((G::SUB + 3) / 4 * 4) + size_t(kSpreadWarps) * 32 * RS) * sizeof(T);
}

template <int W, typename T>
size_t interp3_smem() {
    using G = Col3<W, T>;
    return (size_t(kWarps) * 32 * G::STRIDE + size_t(kWarps) * 32 * kRedStride) * sizeof(T);
}

// Allow a kernel `bytes` of dynamic shared memory (once per device).  Set even
// below 48 KB: the default limit counts the kernel's static shared memory too.
template <auto K>
static cudaError_t opt_in(size_t bytes) {
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured & (1ull << (dev & 63))) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (err == cudaSuccess) configured |= (1ull << (dev & 63));
    return err;
}

template <int W, typename T>
static cudaError_t spread3_one(const SpreadArgs& a, cudaStream_t s) {
    const size_t bytes = spread3_smem<W, T>();
    cudaError_t err = opt_in<k_spread3_col<W, T>>(bytes);
    if (err != cudaSuccess) return err;
    if (a.ntasks == 0) return cudaSuccess;
    k_spread3_col<W, T><<<a.ntasks, kSpreadWarps * 32, bytes, s>>>(a);
    return cudaGetLastError();
}

// Blocks of the persistent interpolation grid: as many as fit on the GPU at
// once, but no more than the queue can keep busy.
template <int W, typename T>
static int interp3_grid(int ncols) {
    static int resident[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int& r = resident[dev & 63];
    if (r == 0) {
        int per_sm = 0, sms = 0;
        if (opt_in<k_interp3_col<W, T>>(interp3_smem<W, T>()) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interp3_col<W, T>, 256, interp3_smem<W, T>()) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        r = std::max(1, per_sm) * sms;
    }
    return std::max(1, std::min(r, (ncols + kWarps - 1) / kWarps));
}

template <int W, typename T>
static cudaError_t interp3_one(const InterpArgs& a, const Epilogue& e, cudaStream_t s) {
    const size_t bytes = interp3_smem<W, T>();
    cudaError_t err = opt_in<k_interp3_col<W, T>>(bytes);
    if (err != cudaSuccess) return err;
    const int blocks = interp3_grid<W, T>(a.ncols);
    if (blocks == 0) {
        const cudaError_t last = cudaGetLastError();
        return last != cudaSuccess ? last : cudaErrorInvalidValue;
    }
    if (a.ncols == 0) return cudaSuccess;
    k_interp3_col<W, T><<<blocks, 256, bytes, s>>>(a, e);
    return cudaGetLastError();
}

bool column_kernels(int d, int W) { return d == 3 && W <= 10; }

template <typename T>
cudaError_t launch_spread3(int W, const SpreadArgs& a, cudaStream_t s) {
    switch (W) {
        case 4: return spread3_one<4, T>(a, s);
        case 6: return spread3_one<6, T>(a, s);
        case 8: return spread3_one<8, T>(a, s);
        case 10: return spread3_one<10, T>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_interp3(int W, const InterpArgs& a, const Epilogue& e, cudaStream_t s) {
    switch (W) {
        case 4: return interp3_one<4, T>(a, e, s);
        case 6: return interp3_one<6, T>(a, e, s);
        case 8: return interp3_one<8, T>(a, e, s);
        case 10: return interp3_one<10, T>(a, e, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
int interp3_blocks(int W, int ncols) {
    switch (W) {
        case 4: return interp3_grid<4, T>(ncols);
        case 6: return interp3_grid<6, T>(ncols);
        case 8: return interp3_grid<8, T>(ncols);
        case 10: return interp3_grid<10, T>(ncols);
        default: return 0;
    }
}

template int interp3_blocks<float>(int, int);
template int interp3_blocks<double>(int, int);
// ------------------------------------------------------------ 2-D strip dispatch
template <int W, typename T>
size_t interp2_smem() {
    using G = Strip2<W, T>;
    return (size_t(kWarps) * 32 * G::STRIDE + size_t(kWarps) * 32 * kRedStride) * sizeof(T) +
           size_t(kWarps) * 32 * sizeof(int);
}

// Blocks of a persistent strip launch: all resident blocks, but no more than
// one warp per task -- except that a few tasks still get a block (an SM) each,
// since the strip loops are bound by the SM's FP64 or FP32 pipes, not by the
// warps they keep busy.
template <auto K>
static int resident_blocks(size_t smem, int tasks) {
    static int resident[64] = {0}, sm_count[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int& r = resident[dev & 63];
    if (r == 0) {
        int per_sm = 0, sms = 0;
        if (opt_in<K>(smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K, 256, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        r = std::max(1, per_sm) * sms;
        sm_count[dev & 63] = sms;
    }
    const int want = std::max((tasks + kWarps - 1) / kWarps, std::min(tasks, sm_count[dev & 63]));
    return std::max(1, std::min(r, want));
}

template <int W, typename T>
size_t spread2col_smem() {
    using G = Col2<W, T>;
    constexpr int RS = sizeof(T) == 4 ? G::STRIDE_S : G::STRIDE;
    return (size_t((G::SUB + 3) / 4 * 4) + size_t(kSpreadWarps) * 32 * RS) * sizeof(T);
}

// 2-D spreading: one block per column task (bin, first column, end column).
template <int W, typename T>
static cudaError_t spread2_one(const SpreadArgs& a, cudaStream_t s) {
    const size_t bytes = spread2col_smem<W, T>();
    cudaError_t err = opt_in<k_spread2_col<W, T>>(bytes);
    if (err != cudaSuccess) return err;
    if (a.ntasks == 0) return cudaSuccess;
    k_spread2_col<W, T><<<a.ntasks, kSpreadWarps * 32, bytes, s>>>(a);
    return cudaGetLastError();
}

template <int W, typename T>
static cudaError_t interp2_one(const InterpArgs& a, const Epilogue& e, cudaStream_t s) {
    const size_t bytes = interp2_smem<W, T>();
    cudaError_t err = opt_in<k_interp2_strip<W, T>>(bytes);
    if (err != cudaSuccess) return err;
    const int blocks = resident_blocks<k_interp2_strip<W, T>>(bytes, a.nstasks);
    if (blocks == 0) {
        const cudaError_t last = cudaGetLastError();
        return last != cudaSuccess ? last : cudaErrorInvalidValue;
    }
    if (a.nstasks == 0) return cudaSuccess;
    k_interp2_strip<W, T><<<blocks, 256, bytes, s>>>(a, e);
    return cudaGetLastError();
}

#define SK_STRIP_W(FN, ...)                        \
    switch (W) {                                   \
        case 4: return FN<4, T>(__VA_ARGS__);      \
        case 6: return FN<6, T>(__VA_ARGS__);      \
        case 8: return FN<8, T>(__VA_ARGS__);      \
        case 10: return FN<10, T>(__VA_ARGS__);    \
        case 12: return FN<12, T>(__VA_ARGS__);    \
        case 14: return FN<14, T>(__VA_ARGS__);    \
        case 16: return FN<16, T>(__VA_ARGS__);    \
        default: return cudaErrorInvalidValue;     \
    }

template <typename T>
cudaError_t launch_spread2(int W, const SpreadArgs& a, cudaStream_t s) {
    SK_STRIP_W(spread2_one, a, s)
}

template <typename T>
cudaError_t launch_interp2(int W, const InterpArgs& a, const Epilogue& e, cudaStream_t s) {
    SK_STRIP_W(interp2_one, a, e, s)
}
#undef SK_STRIP_W

template <typename T>
int strip2_blocks(int W, int ntasks) {
    switch (W) {
        case 4: return resident_blocks<k_interp2_strip<4, T>>(interp2_smem<4, T>(), ntasks);
        case 6: return resident_blocks<k_interp2_strip<6, T>>(interp2_smem<6, T>(), ntasks);
        case 8: return resident_blocks<k_interp2_strip<8, T>>(interp2_smem<8, T>(), ntasks);
        case 10: return resident_blocks<k_interp2_strip<10, T>>(interp2_smem<10, T>(), ntasks);
        case 12: return resident_blocks<k_interp2_strip<12, T>>(interp2_smem<12, T>(), ntasks);
        case 14: return resident_blocks<k_interp2_strip<14, T>>(interp2_smem<14, T>(), ntasks);
        case 16: return resident_blocks<k_interp2_strip<16, T>>(interp2_smem<16, T>(), ntasks);
        default: return 0;
    }
}

template cudaError_t launch_spread2<float>(int, const SpreadArgs&, cudaStream_t);
template cudaError_t launch_spread2<double>(int, const SpreadArgs&, cudaStream_t);
template cudaError_t launch_interp2<float>(int, const InterpArgs&, const Epilogue&, cudaStream_t);
template cudaError_t launch_interp2<double>(int, const InterpArgs&, const Epilogue&, cudaStream_t);
template int strip2_blocks<float>(int, int);
template int strip2_blocks<double>(int, int);

template cudaError_t launch_spread3<float>(int, const SpreadArgs&, cudaStream_t);
template cudaError_t launch_spread3<double>(int, const SpreadArgs&, cudaStream_t);
template cudaError_t launch_interp3<float>(int, const InterpArgs&, const Epilogue&, cudaStream_t);
template cudaError_t launch_interp3<double>(int, const InterpArgs&, const Epilogue&, cudaStream_t);

}  // namespace sk
