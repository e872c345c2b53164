// Batched pencil FFTs on the oversampled grid (the O(N log N) part of
// Eq. (fastsum)) and the pointwise multiply by the kernel's Fourier
// coefficients, written for shared memory:
//
//   * Every block loads P pencils of length n (P * n = kFftBlockElems complex
//     values, or one pencil when n is larger) into shared memory, transforms
//     them there and writes back.  The transform is a Stockham (self-sorting)
//     FFT of radix 8 (a last stage of radix 4 or 2 when log2 n is not a
//     multiple of 3): each of the n/8 threads of a pencil reads 8 elements,
//     applies the stage's twiddles, does its 8-point (or 2 x 4-point, or
//     4 x 2-point) DFT in registers and writes the 8 results back, so a
//     128-point pencil takes three stages with natural order in and out.
//     Blocks are small (n/8 threads per pencil), so a launch has many of them
//     and their load, barrier and store latencies overlap on every SM.
//     Element e of a pencil sits at slot pidx(e), a XOR swizzle of its low
//     bits, which keeps the stride-n/R reads and stride-Ns writes of every
//     stage and the parallel walks of the load phases free of shared-memory
//     bank conflicts.
//   * The grid is real, so the first pass packs two real rows into one complex
//     FFT and splits the result into two half spectra (k = 0..h along the
//     contiguous axis); the last inverse pass does the reverse.
//   * Only the 2h+1 = N+1 frequencies -N/2..N/2 survive the multiply, so the
//     forward passes keep only those and the inverse passes start from them.
//   * The multiply by c_k b_k / psihat(k)^2 is fused into the pass along
//     axis 0: forward FFT, multiply, inverse FFT in one kernel.
//
//   * Band pruning: every point and all its window taps lie inside a box
//     [lo_t, hi_t] per axis (known at plan time), so outside it the spread grid
//     is zero and the interpolated grid is never read.  The first pass only
//     transforms rows inside the box (and zeroes them after reading, so the next
//     spreading starts from a zero grid without a memset), the axis-1 passes
//     only pencils whose axis-0 index is inside the box, and the last pass only
//     rows inside the box, into a second grid that interpolation reads.
//
// Convolution pipeline (n = n_os, h = N/2, grid g[x][y][z] with z contiguous):
//   3-D: r2c(z) -> fwd(y, keep 2h+1) -> [fwd(x) * M, inv(x)] -> inv(y) -> c2r(z)
//   2-D: r2c(y) -> [fwd(x) * M, inv(x)] -> c2r(y)
//   1-D: r2c(x) -> * M -> c2r(x)            (the grid carries a second, zero row)
#include <algorithm>
#include <utility>

#include "sk_internal.cuh"

namespace sk {

enum { FULL = 0, CENTERED = 1 };

constexpr int kFftBlockElems = 512;

__host__ __device__ constexpr int fft_pencils(int n) { return n >= kFftBlockElems ? 1 : kFftBlockElems / n; }

// Elements of a pencil per thread: 8 in FP32 (radix-8 stages); 4 in FP64
// (radix-4 stages), whose arithmetic is slow enough on this GPU that the
// shorter per-thread chains and twice the threads pay -- except for pencils
// longer than 2048, which keep 8 so that a block stays within 512 threads.
template <typename T>
__host__ __device__ constexpr int fft_ept(int n) { return (sizeof(T) == 8 && n <= 2048) ? 4 : 8; }

// Threads of an FFT block (16 to 512).
template <typename T>
__host__ __device__ constexpr int fft_threads(int n) { return fft_pencils(n) * n / fft_ept<T>(n); }

// Slot of element e of a pencil of complex values C in shared memory: e with
// its low bits XOR-ed with higher ones (bits 3-6 into 0-3 for 8-byte values,
// bits 2-4 into 0-2 for 16-byte ones), a permutation of every aligned block
// of 16 (8) elements.  Every access of the Stockham stages -- a thread's
// reads at a stride of n/R, the writes at stride Ns -- then puts the lanes
// of one shared-memory wavefront (16 lanes of 8 bytes, 8 of 16) on distinct
// banks, and so do the contiguous walks of the load and store phases.  A
// pencil spans fft_stride<C>(n) slots: n plus a few, so that the pencils a
// wavefront spans (n <= 64, and the load phases that walk across pencils)
// start on different banks.
template <typename C>
__host__ __device__ constexpr int pidx(int e) {
    return sizeof(C) == 8 ? (e ^ ((e >> 3) & 15)) : (e ^ ((e >> 2) & 7));
}
template <typename C>
__host__ __device__ constexpr int fft_stride(int n) {
    return sizeof(C) == 8 ? (n == 32 ? 36 : (n == 64 ? 72 : n + 4)) : n + 2;
}

// Row pairs of the real passes: pair q covers rows r0 = o * ostride + y and
// r0 + 1 with o = olo + q / npo and y = ylo + 2 (q % npo).
struct RowPairs {
    int64_t olo, ostride;
    int ylo, npo;
    int64_t npairs;
};

__device__ __forceinline__ int64_t pair_row(const RowPairs& rp, int q) {
    const int qo = q / rp.npo;   // 32-bit: the row pairs of a grid fit in an int
    return (rp.olo + qo) * rp.ostride + rp.ylo + 2 * (q - qo * rp.npo);
}

// pair_row of row pair q, recomputed only when q changes (the elements a
// thread visits come in non-decreasing pair order).
struct PairRowCache {
    int q = -1;
    int64_t row = 0;
    __device__ __forceinline__ int64_t get(const RowPairs& rp, int qn) {
        if (qn != q) {
            q = qn;
            row = pair_row(rp, qn);
        }
        return row;
    }
};

__device__ __forceinline__ int ilog2(int p) { return __ffs(p) - 1; }   // p a power of two

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}

template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}

// a * (-i) for the forward transform, a * i for the inverse.
template <typename C, bool INV>
__device__ __forceinline__ C mul_mi(C a) {
    C r;
    r.x = INV ? -a.y : a.y;
    r.y = INV ? a.x : -a.x;
    return r;
}

// Twiddle exp(-+2 pi i m / n), 0 <= m < n, from the table of the first n/2.
template <typename C, bool INV>
__device__ __forceinline__ C twiddle(const C* tw, int m, int n) {
    const int h = n >> 1;
    C w = tw[m < h ? m : m - h];
    if (m >= h) {
        w.x = -w.x;
        w.y = -w.y;
    }
    if (INV) w.y = -w.y;
    return w;
}

// In-register DFTs (y_r = sum_q x_q w^(q r), w = exp(-+2 pi i / R)).
template <typename C, bool INV>
__device__ __forceinline__ void dft2(C* x) {
    const C a = x[0];
    x[0] = cadd(a, x[1]);
    x[1] = csub(a, x[1]);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C* x) {
    const C a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
    const C a2 = cadd(x[1], x[3]), a3 = mul_mi<C, INV>(csub(x[1], x[3]));
    x[0] = cadd(a0, a2);
    x[2] = csub(a0, a2);
    x[1] = cadd(a1, a3);
    x[3] = csub(a1, a3);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft8(C* x) {
    using T = decltype(x[0].x);
    const T h = T(0.70710678118654752440);   // 1/sqrt(2)
    C e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
    dft4<C, INV>(e);
    dft4<C, INV>(o);
    // o[r] *= w8^r, w8 = (1 -+ i) / sqrt(2)
    {
        const C a = o[1];
        o[1].x = INV ? (a.x - a.y) * h : (a.x + a.y) * h;
        o[1].y = INV ? (a.x + a.y) * h : (a.y - a.x) * h;
    }
    o[2] = mul_mi<C, INV>(o[2]);
    {
        const C a = o[3];
        o[3].x = INV ? -(a.x + a.y) * h : (a.y - a.x) * h;
        o[3].y = INV ? (a.x - a.y) * h : -(a.x + a.y) * h;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        x[r] = cadd(e[r], o[r]);
        x[r + 4] = csub(e[r], o[r]);
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor in the stream is finishing;
// griddep_wait() blocks until the predecessor has completed and its writes
// are visible (a no-op for a kernel launched the ordinary way), and
// griddep_launch() lets this kernel's own dependent start launching.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The barrier of an FFT unit (the block of a pass kernel).
struct SyncBlock {
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};

// One Stockham stage of radix R on the thread's E elements (E/R butterflies):
// butterfly jj reads x_q = X[jj + q n/R], scales it by w_L^(q k) (L = Ns R,
// k = jj mod Ns), takes the R-point DFT and writes y_r to
// X[(jj - k) R + k + r Ns].  All reads precede a barrier, then the writes.
// The twiddles of one Stockham stage are tabulated per butterfly class: row
// k (0 <= k < Ns) of a radix-R stage holds w_L^(q k), q = 1 .. R-1, L = Ns R,
// w_L = exp(-2 pi i / L), padded to RW(R) entries, so a butterfly reads its
// R-1 twiddles with vector loads (the table is a few KB, resident in L1);
// the stages follow one another in the table, and the first stage (Ns = 1,
// all twiddles 1) has none.
__host__ __device__ constexpr int row_width(int R) { return R == 8 ? 8 : (R == 4 ? 4 : 2); }

template <typename C, int RW>
__device__ __forceinline__ void load_row(const C* __restrict__ row, C (&w)[RW]) {
    if constexpr (sizeof(C) == 8) {
#pragma unroll
        for (int q = 0; q < RW; q += 2) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(row + q));
            w[q].x = v.x;
            w[q].y = v.y;
            w[q + 1].x = v.z;
            w[q + 1].y = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < RW; ++q) w[q] = __ldg(row + q);
    }
}

// One Stockham stage of radix R on the thread's E elements (E/R butterflies):
// butterfly jj reads x_q = X[jj + q n/R], scales it by w_L^(q k) (L = Ns R,
// k = jj mod Ns), takes the R-point DFT and writes y_r to
// X[(jj - k) R + k + r Ns].  All reads precede a barrier, then the writes.
// `rows` is the stage's twiddle table (unused when Ns = 1).
template <typename C, bool INV, int R, int E, class S>
__device__ __forceinline__ void stockham_stage(C* pen, int n, int Ns, int t, const C* __restrict__ rows) {
    constexpr int B = E / R;
    constexpr int RW = row_width(R);
    const int stride = n / R, per = n / E;
    C x[E];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int jj = t + b * per;
#pragma unroll
        for (int r = 0; r < R; ++r) x[b * R + r] = pen[pidx<C>(jj + r * stride)];
    }
    // the butterflies' twiddle rows, requested before the barrier
    C w[B][RW];
    if (Ns > 1) {
#pragma unroll
        for (int b = 0; b < B; ++b) load_row<C, RW>(rows + ((t + b * per) & (Ns - 1)) * RW, w[b]);
    }
    S::sync();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int jj = t + b * per;
        const int k = jj & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C wq = w[b][q - 1];
                if (INV) wq.y = -wq.y;
                x[b * R + q] = cmul(x[b * R + q], wq);
            }
        }
        if (R == 8) dft8<C, INV>(x + b * R);
        else if (R == 4) dft4<C, INV>(x + b * R);
        else dft2<C, INV>(x + b * R);
        const int base = (jj - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) pen[pidx<C>(base + r * Ns)] = x[b * R + r];
    }
    S::sync();
}

// Transform the unit's P pencils in place (natural order in and out; pencil
// p at buf + p * ns, element e at pidx<C>(e)); the unit has exactly
// fft_threads<T>(n) threads, `tid` is the thread's index in it.  `rows` is
// the plan's table of stage twiddle rows.  Radix E = fft_ept stages while
// they fit, then one of radix 4 or 2.
template <typename C, bool INV, int E, class S>
__device__ __forceinline__ void stockham_all(C* buf, int ns, int n, int log2n, const C* __restrict__ rows, int tid) {
    constexpr int LE = E == 8 ? 3 : 2;
    const int per = n / E;
    const int p = tid / per, t = tid - p * per;
    C* pen = buf + p * ns;
    int Ns = 1, rem = log2n;
    for (; rem >= LE; rem -= LE, Ns <<= LE) {
        stockham_stage<C, INV, E, E, S>(pen, n, Ns, t, rows);
        if (Ns > 1) rows += Ns * row_width(E);
    }
    if (rem == 2) stockham_stage<C, INV, 4, E, S>(pen, n, Ns, t, rows);
    else if (rem == 1) stockham_stage<C, INV, 2, E, S>(pen, n, Ns, t, rows);
}

// The same stage sequence for a length known at compile time (N = 2^L2): the
// stage parameters, pencil strides and shared-memory offsets fold into
// constants and immediate offsets.
template <typename C, bool INV, int E, class S, int N, int NS, int REM>
__device__ __forceinline__ void stages_ct(C* pen, int t, const C* __restrict__ rows) {
    constexpr int LE = E == 8 ? 3 : 2;
    if constexpr (REM >= LE) {
        stockham_stage<C, INV, E, E, S>(pen, N, NS, t, rows);
        stages_ct<C, INV, E, S, N, NS * E, REM - LE>(pen, t, NS > 1 ? rows + NS * row_width(E) : rows);
    } else if constexpr (REM == 2) {
        stockham_stage<C, INV, 4, E, S>(pen, N, NS, t, rows);
    } else if constexpr (REM == 1) {
        stockham_stage<C, INV, 2, E, S>(pen, N, NS, t, rows);
    }
}

template <typename T, bool INV, class S, int L2>
__device__ void fft_stockham(typename Cplx<T>::type* buf, int ns, int n, int log2n, const typename Cplx<T>::type* rows,
                             int tid) {
    using C = typename Cplx<T>::type;
    S::sync();
    if constexpr (L2 > 0) {
        constexpr int N = 1 << L2, E = fft_ept<T>(N), PER = N / E;
        const int p = tid / PER, t = tid - p * PER;
        stages_ct<C, INV, E, S, N, 1, L2>(buf + p * fft_stride<C>(N), t, rows);
    } else if (fft_ept<T>(n) == 4) {
        stockham_all<C, INV, 4, S>(buf, ns, n, log2n, rows, tid);
    } else {
        stockham_all<C, INV, 8, S>(buf, ns, n, log2n, rows, tid);
    }
}

// Radix of the stage that finds REM of log2 n left to do (E elements per
// thread): E while it fits, then 4 or 2.
__host__ __device__ constexpr int fft_radix(int rem, int E) { return rem >= (E == 8 ? 3 : 2) ? E : (rem == 2 ? 4 : 2); }
__host__ __device__ constexpr int fft_lg(int R) { return R == 8 ? 3 : (R == 4 ? 2 : 1); }

// Stages of an N = 2^L2 point transform with E elements per thread, and the
// twiddles one thread applies over all of them: a stage with Ns > 1 gives
// each of the thread's E / R butterflies R - 1 values.
__host__ __device__ constexpr int fft_stages(int L2, int E) {
    int count = 0;
    for (int rem = L2; rem > 0; rem -= fft_lg(fft_radix(rem, E))) ++count;
    return count;
}

__host__ __device__ constexpr int fft_tw_count(int L2, int E) {
    int count = 0, Ns = 1;
    for (int rem = L2; rem > 0;) {
        const int R = fft_radix(rem, E);
        if (Ns > 1) count += (E / R) * (R - 1);
        Ns *= R;
        rem -= fft_lg(R);
    }
    return count;
}

// A thread's twiddles for every stage of an N = 2^L2 point transform, read
// from the stage table into registers once per unit (before its data loads,
// so their latency overlaps), so that no stage waits on a table load and the
// unit's transforms of one direction or the other all reuse them.
template <typename T, int L2>
struct FftTw {
    using C = typename Cplx<T>::type;
    static constexpr int E = L2 > 0 ? fft_ept<T>(1 << L2) : 8;
    static constexpr int COUNT = L2 > 0 ? fft_tw_count(L2, E) : 0;
    static constexpr int SIZE = COUNT > 0 ? COUNT : 1;
    C w[SIZE];

    template <int N, int NS, int REM, int OFF>
    __device__ __forceinline__ void load_ct(const C* __restrict__ rows, int t) {
        if constexpr (REM > 0) {
            constexpr int R = fft_radix(REM, E), B = E / R, RW = row_width(R), PER = N / E;
            if constexpr (NS > 1) {
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int k = (t + b * PER) & (NS - 1);
#pragma unroll
                    for (int q = 1; q < R; ++q) w[OFF + b * (R - 1) + q - 1] = __ldg(rows + k * RW + q - 1);
                }
                load_ct<N, NS * R, REM - fft_lg(R), OFF + B * (R - 1)>(rows + NS * RW, t);
            } else {
                load_ct<N, NS * R, REM - fft_lg(R), OFF>(rows, t);
            }
        }
    }

    // thread `tid` of a unit (its index within its pencil is tid mod N/E)
    __device__ __forceinline__ void load(const C* __restrict__ rows, int tid) {
        if constexpr (L2 > 0) {
            constexpr int N = 1 << L2;
            load_ct<N, 1, L2, 0>(rows, tid & (N / E - 1));
        }
    }
};

// A stage as stockham_stage, out of place (reads `in`, writes `out`, so only
// the barrier after the writes is needed) and with the thread's twiddles in
// registers, from position OFF of `tw`.
template <typename C, bool INV, int R, int E, class S, int OFF, int TWN>
__device__ __forceinline__ void stockham_stage2(const C* in, C* out, int n, int Ns, int t, const C (&tw)[TWN]) {
    constexpr int B = E / R;
    const int stride = n / R, per = n / E;
    C x[E];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int jj = t + b * per;
#pragma unroll
        for (int r = 0; r < R; ++r) x[b * R + r] = in[pidx<C>(jj + r * stride)];
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int jj = t + b * per;
        const int k = jj & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C wq = tw[OFF + b * (R - 1) + q - 1];
                if (INV) wq.y = -wq.y;
                x[b * R + q] = cmul(x[b * R + q], wq);
            }
        }
        if (R == 8) dft8<C, INV>(x + b * R);
        else if (R == 4) dft4<C, INV>(x + b * R);
        else dft2<C, INV>(x + b * R);
        const int base = (jj - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[pidx<C>(base + r * Ns)] = x[b * R + r];
    }
    S::sync();
}

template <typename C, bool INV, int E, class S, int N, int NS, int REM, int OFF, int TWN>
__device__ __forceinline__ void stages_ct2(C* in, C* out, int t, const C (&tw)[TWN]) {
    if constexpr (REM > 0) {
        constexpr int R = fft_radix(REM, E);
        constexpr int NEXT = (NS > 1) ? OFF + (E / R) * (R - 1) : OFF;
        stockham_stage2<C, INV, R, E, S, OFF, TWN>(in, out, N, NS, t, tw);
        stages_ct2<C, INV, E, S, N, NS * R, REM - fft_lg(R), NEXT, TWN>(out, in, t, tw);
    }
}

// The unit's transform with two pencil buffers, `a` (input) and `b` (same
// layout): the stages alternate between them, one barrier each, with the
// twiddles `tw` holds.  Returns the buffer holding the result.  Lengths not
// known at compile time (L2 = 0) are transformed in place in `a`, with the
// twiddles read from the table `rows`.
template <typename T, bool INV, class S, int L2>
__device__ typename Cplx<T>::type* fft_stockham2(typename Cplx<T>::type* a, typename Cplx<T>::type* b, int ns, int n,
                                                 int log2n, const typename Cplx<T>::type* rows, int tid,
                                                 const FftTw<T, L2>& tw) {
    using C = typename Cplx<T>::type;
    if constexpr (L2 > 0) {
        constexpr int N = 1 << L2, E = fft_ept<T>(N), PER = N / E, NSP = fft_stride<C>(N);
        S::sync();
        const int p = tid / PER, t = tid - p * PER;
        stages_ct2<C, INV, E, S, N, 1, L2, 0, FftTw<T, L2>::SIZE>(a + p * NSP, b + p * NSP, t, tw.w);
        return (fft_stages(L2, E) % 2) ? b : a;
    } else {
        fft_stockham<T, INV, S, L2>(a, ns, n, log2n, rows, tid);
        return a;
    }
}

// Entries (complex) of the stage twiddle table of an n-point transform, and
// the table itself (computed in FP64 and rounded; one launch per stage).
template <typename T>
int fft_twiddle_rows(int n) {
    const int E = fft_ept<T>(n), LE = E == 8 ? 3 : 2;
    int log2n = 0;
    while ((1 << log2n) < n) ++log2n;
    int total = 0, Ns = 1, rem = log2n;
    for (; rem >= LE; rem -= LE, Ns <<= LE)
        if (Ns > 1) total += Ns * row_width(E);
    if (rem > 0 && Ns > 1) total += Ns * row_width(rem == 2 ? 4 : 2);
    return total;
}

template <typename C>
__global__ void k_twiddle_rows(C* __restrict__ rows, int Ns, int R) {
    const int RW = row_width(R);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ns * RW) return;
    const int k = i / RW, q = i - k * RW + 1;
    C v;
    v.x = 0;
    v.y = 0;
    if (q < R) {
        double sn, cs;
        sincospi(-2.0 * double((q * k) % (Ns * R)) / double(Ns * R), &sn, &cs);
        v.x = decltype(v.x)(cs);
        v.y = decltype(v.y)(sn);
    }
    rows[i] = v;
}

template <typename T>
cudaError_t launch_twiddle_rows(void* rows, int n, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const int E = fft_ept<T>(n), LE = E == 8 ? 3 : 2;
    int log2n = 0;
    while ((1 << log2n) < n) ++log2n;
    C* at = static_cast<C*>(rows);
    int Ns = 1, rem = log2n;
    auto stage = [&](int R) {
        const int cnt = Ns * row_width(R);
        k_twiddle_rows<C><<<unsigned((cnt + 255) / 256), 256, 0, s>>>(at, Ns, R);
        at += cnt;
    };
    for (; rem >= LE; rem -= LE, Ns <<= LE)
        if (Ns > 1) stage(E);
    if (rem > 0 && Ns > 1) stage(rem == 2 ? 4 : 2);
    return cudaGetLastError();
}

template int fft_twiddle_rows<float>(int);
template int fft_twiddle_rows<double>(int);
template cudaError_t launch_twiddle_rows<float>(void*, int, cudaStream_t);
template cudaError_t launch_twiddle_rows<double>(void*, int, cudaStream_t);

// Shared memory of an FFT block: two buffers of P pencils of fft_stride<C>(n)
// slots each (the input and the other buffer of fft_stockham2).
template <typename T>
struct FftSmem {
    using C = typename Cplx<T>::type;
    C* buf;
    __device__ __forceinline__ FftSmem() {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        buf = reinterpret_cast<C*>(smem_raw);
    }
};

// Elements a thread loads per round; a round's loads are all issued before
// any of them is stored, so their latencies overlap.
constexpr int kFftLoadsPerRound = 8;

// The passes below are written for one FFT unit: `nthr` threads (a block of a
// pass kernel) that transform the P pencils starting at pencil (or row pair)
// q0, thread `tid` of the unit, staging in `buf` (two buffers of P pencils of
// fft_stride<C>(n) slots, the transform alternating between them), with its
// barrier S::sync().  Data written by the previous pass is
// read once, with ld.global.cg (cached in L2 only).  Index arithmetic is
// 32-bit and free of divisions in the per-element loops (the pencil a thread
// works on is fixed per unit, the pencil count P is a power of two): a 64-bit
// division per element had made every pass several microseconds slower.

// Two real rows of length n -> two half spectra of length h+1 (output rows
// are the same row indices in A1).  The input rows are zeroed after reading.
template <typename T, class S, int L2>
__device__ __forceinline__ void r2c_unit(T* __restrict__ g, typename Cplx<T>::type* __restrict__ out,
                                         const RowPairs& rp, int n, int log2n, int h,
                                         const typename Cplx<T>::type* tw, typename Cplx<T>::type* buf, int q0,
                                         int tid, int nthr) {
    if constexpr (L2 > 0) {   // a length known at compile time
        n = 1 << L2;
        log2n = L2;
    }
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n);
    const int ns = fft_stride<C>(n);
    S::sync();   // the unit's previous pencils have been read out of buf
    FftTw<T, L2> twr;
    twr.load(tw, tid);
    PairRowCache rc;
    for (int e0 = 0; e0 < P * n; e0 += kFftLoadsPerRound * nthr) {
        C z[kFftLoadsPerRound];
        int64_t at[kFftLoadsPerRound];
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            const int q = q0 + (e >> log2n);
            z[j].x = T(0);
            z[j].y = T(0);
            at[j] = -1;
            if (e < P * n && q < rp.npairs) {
                at[j] = rc.get(rp, q) * n + (e & (n - 1));
                z[j].x = __ldcg(g + at[j]);
                z[j].y = __ldcg(g + at[j] + n);
            }
        }
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            if (e >= P * n) continue;
            if (at[j] >= 0) {
                g[at[j]] = T(0);
                g[at[j] + n] = T(0);
            }
            buf[(e >> log2n) * ns + pidx<C>(e & (n - 1))] = z[j];
        }
    }
    const C* res = fft_stockham2<T, false, S, L2>(buf, buf + P * ns, ns, n, log2n, tw, tid, twr);
    const int H = h + 1;
    // element e = p H + k of the output, walked without a division per element
    int p = tid / H, k = tid - (tid / H) * H;
    const int kstep = nthr % H, pstep = nthr / H;
    for (int e = tid; e < P * H; e += nthr) {
        const int q = q0 + p;
        if (q < rp.npairs) {
            const int64_t r0 = rc.get(rp, q);
            const C zk = res[p * ns + pidx<C>(k)];
            const C zm = res[p * ns + pidx<C>((n - k) & (n - 1))];
            C A, Bv;
            A.x = (zk.x + zm.x) * T(0.5);
            A.y = (zk.y - zm.y) * T(0.5);
            Bv.x = (zk.y + zm.y) * T(0.5);
            Bv.y = (zm.x - zk.x) * T(0.5);
            out[r0 * H + k] = A;
            out[(r0 + 1) * H + k] = Bv;
        }
        k += kstep;
        p += pstep;
        if (k >= H) {
            k -= H;
            ++p;
        }
    }
}

// Two half spectra -> two real rows, by Hermitian completion.
template <typename T, class S, int L2>
__device__ __forceinline__ void c2r_unit(const typename Cplx<T>::type* __restrict__ in, T* __restrict__ g,
                                         const RowPairs& rp, int n, int log2n, int h,
                                         const typename Cplx<T>::type* tw, typename Cplx<T>::type* buf, int q0,
                                         int tid, int nthr) {
    if constexpr (L2 > 0) {   // a length known at compile time
        n = 1 << L2;
        log2n = L2;
    }
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n);
    const int ns = fft_stride<C>(n);
    S::sync();   // the unit's previous pencils have been read out of buf
    FftTw<T, L2> twr;
    twr.load(tw, tid);
    const int H = h + 1;
    PairRowCache rc;
    for (int e0 = 0; e0 < P * n; e0 += kFftLoadsPerRound * nthr) {
        C A[kFftLoadsPerRound], Bv[kFftLoadsPerRound];
        int sgn[kFftLoadsPerRound];   // +1: k in 0..h, -1: -k in 1..h, 0: outside (zero)
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            const int pos = e & (n - 1);
            const int q = q0 + (e >> log2n);
            const int k = pos <= (n >> 1) ? pos : pos - n;
            sgn[j] = 0;
            A[j].x = A[j].y = Bv[j].x = Bv[j].y = T(0);
            if (e < P * n && q < rp.npairs && k >= -h && k <= h) {
                const int64_t r0 = rc.get(rp, q);
                const int ka = k >= 0 ? k : -k;
                sgn[j] = k >= 0 ? 1 : -1;
                A[j] = __ldcg(in + r0 * H + ka);
                Bv[j] = __ldcg(in + (r0 + 1) * H + ka);
            }
        }
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            if (e >= P * n) continue;
            const int pos = e & (n - 1);
            C z;
            if (sgn[j] > 0) {
                if (pos == 0) {
                    A[j].y = T(0);
                    Bv[j].y = T(0);
                }
                z.x = A[j].x - Bv[j].y;
                z.y = A[j].y + Bv[j].x;
            } else if (sgn[j] < 0) {
                z.x = A[j].x + Bv[j].y;
                z.y = Bv[j].x - A[j].y;
            } else {
                z.x = T(0);
                z.y = T(0);
            }
            buf[(e >> log2n) * ns + pidx<C>(pos)] = z;
        }
    }
    const C* res = fft_stockham2<T, true, S, L2>(buf, buf + P * ns, ns, n, log2n, tw, tid, twr);
    for (int e = tid; e < P * n; e += nthr) {
        const int p = e >> log2n;
        const int l = e & (n - 1);
        const int q = q0 + p;
        if (q >= rp.npairs) continue;
        const int64_t r0 = rc.get(rp, q);
        const C v = res[p * ns + pidx<C>(l)];
        g[r0 * n + l] = v.x;
        g[(r0 + 1) * n + l] = v.y;
    }
}

// Pencils along the middle axis of an (O, L, I) array: element k of pencil
// (o, i) sits at (o*L + k)*I + i.  FULL keeps all n entries along the axis;
// CENTERED stores frequencies -h..h at positions 0..2h.  Only pencils with
// o in [olo, olo + ocnt) are transformed, and a FULL output is stored only for
// k in [klo, klo + kcnt).
template <typename T, int INM, int OUTM, bool INV, class S, int L2>
__device__ __forceinline__ void axis_unit(const typename Cplx<T>::type* __restrict__ in,
                                          typename Cplx<T>::type* __restrict__ out, int olo, int ocnt, int I, int klo,
                                          int kcnt, int n, int log2n, int h, const typename Cplx<T>::type* tw,
                                          typename Cplx<T>::type* buf, int q0, int tid, int nthr) {
    if constexpr (L2 > 0) {   // a length known at compile time
        n = 1 << L2;
        log2n = L2;
    }
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n), lp = ilog2(P);
    const int ns = fft_stride<C>(n);
    const int Q = ocnt * I;
    const int Lin = INM == FULL ? n : 2 * h + 1;
    const int Lout = OUTM == FULL ? n : 2 * h + 1;
    const int k0 = OUTM == FULL ? klo : 0;
    const int kn = OUTM == FULL ? kcnt : Lout;
    S::sync();   // the unit's previous pencils have been read out of buf
    FftTw<T, L2> twr;
    twr.load(tw, tid);
    // the unit's threads are a multiple of P, so a thread always works on
    // pencil pl = tid mod P of the unit: pencil (o, i), o = olo + q / I
    const int pl = tid & (P - 1);
    const int q = q0 + pl;
    const bool qok = q < Q;
    const int qo = qok ? q / I : 0;
    const int64_t o = olo + qo, i = q - qo * I;
    const C* src = in + o * Lin * I + i;
    C* dst = out + o * Lout * I + i;
    if (INM == CENTERED) {
        for (int e = tid; e < P * ns; e += nthr) {
            buf[e].x = T(0);
            buf[e].y = T(0);
        }
        S::sync();
    }
    for (int e0 = 0; e0 < P * Lin; e0 += kFftLoadsPerRound * nthr) {
        C v[kFftLoadsPerRound];
        bool ok[kFftLoadsPerRound];
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            const int k = e >> lp;
            ok[j] = e < P * Lin && qok;
            if (ok[j]) v[j] = __ldcg(src + int64_t(k) * I);
        }
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            if (!ok[j]) continue;
            const int e = e0 + j * nthr + tid;
            const int k = e >> lp;
            const int pos = INM == FULL ? k : ((k - h) & (n - 1));
            buf[pl * ns + pidx<C>(pos)] = v[j];
        }
    }
    const C* res = fft_stockham2<T, INV, S, L2>(buf, buf + P * ns, ns, n, log2n, tw, tid, twr);
    if (!qok) return;
    for (int e = tid; e < P * kn; e += nthr) {
        const int k = k0 + (e >> lp);
        const int pos = OUTM == FULL ? k : ((k - h) & (n - 1));
        dst[int64_t(k) * I] = res[pl * ns + pidx<C>(pos)];
    }
}

// Pencils along axis 0 of an (n, I) array: forward FFT, multiply the kept
// frequencies by M[(k+h)*I + q] and zero the rest, inverse FFT, in place.
// Only axis-0 positions in [xlo, xlo + xcnt) are loaded (the rest are zero)
// and stored (the rest are never read).
template <typename T, class S, int L2>
__device__ __forceinline__ void convolve_unit(typename Cplx<T>::type* __restrict__ data, int I, int xlo, int xcnt,
                                              int n, int log2n, int h, const T* __restrict__ mult,
                                              const typename Cplx<T>::type* tw, typename Cplx<T>::type* buf,
                                              int q0, int tid, int nthr) {
    if constexpr (L2 > 0) {   // a length known at compile time
        n = 1 << L2;
        log2n = L2;
    }
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n), lp = ilog2(P);
    const int ns = fft_stride<C>(n);
    S::sync();   // the unit's previous pencils have been read out of buf
    FftTw<T, L2> twr;
    twr.load(tw, tid);
    griddep_wait();   // the previous pass's output
    for (int e0 = 0; e0 < P * n; e0 += kFftLoadsPerRound * nthr) {
        C v[kFftLoadsPerRound];
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            const int k = e >> lp;
            const int q = q0 + (e & (P - 1));
            v[j].x = T(0);
            v[j].y = T(0);
            if (e < P * n && q < I && k >= xlo && k < xlo + xcnt) v[j] = __ldcg(data + int64_t(k) * I + q);
        }
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            if (e >= P * n) continue;
            const int k = e >> lp;
            buf[(e & (P - 1)) * ns + pidx<C>(k)] = v[j];
        }
    }
    // when one round covers the unit, the multiplier of each element this
    // thread scales is loaded before the forward transform, so its latency
    // hides behind it
    const bool one_round = P * n <= kFftLoadsPerRound * nthr;
    T mv[kFftLoadsPerRound];
#pragma unroll
    for (int j = 0; j < kFftLoadsPerRound; ++j) {
        const int e = j * nthr + tid;
        const int pos = e >> lp;
        const int q = q0 + (e & (P - 1));
        const int k = pos <= (n >> 1) ? pos : pos - n;
        mv[j] = (one_round && e < P * n && q < I && k >= -h && k <= h) ? mult[int64_t(k + h) * I + q] : T(0);
    }
    C* res = fft_stockham2<T, false, S, L2>(buf, buf + P * ns, ns, n, log2n, tw, tid, twr);
    if (one_round) {
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = j * nthr + tid;
            if (e >= P * n) continue;
            const int pos = e >> lp;
            C& v = res[(e & (P - 1)) * ns + pidx<C>(pos)];
            v.x *= mv[j];
            v.y *= mv[j];
        }
    } else {
        for (int e = tid; e < P * n; e += nthr) {
            const int pos = e >> lp;
            const int pl = e & (P - 1);
            const int q = q0 + pl;
            const int k = pos <= (n >> 1) ? pos : pos - n;
            C& v = res[pl * ns + pidx<C>(pos)];
            if (q < I && k >= -h && k <= h) {
                const T m = mult[int64_t(k + h) * I + q];
                v.x *= m;
                v.y *= m;
            } else {
                v.x = T(0);
                v.y = T(0);
            }
        }
    }
    const C* res2 = fft_stockham2<T, true, S, L2>(res, res == buf ? buf + P * ns : buf, ns, n, log2n, tw, tid, twr);
    for (int e = tid; e < P * xcnt; e += nthr) {
        const int k = xlo + (e >> lp);
        const int pl = e & (P - 1);
        const int q = q0 + pl;
        if (q < I) data[int64_t(k) * I + q] = res2[pl * ns + pidx<C>(k)];
    }
}

// ------------------------------------------------------------ pass kernels
// One launch per pass; a block is one unit of fft_threads<T>(n) threads.

template <typename T, int L2>
__global__ void __launch_bounds__(512) k_fft_r2c_rows(T* __restrict__ g, typename Cplx<T>::type* __restrict__ out,
                                                      RowPairs rp, int n, int log2n, int h,
                                                      const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm;
    r2c_unit<T, SyncBlock, L2>(g, out, rp, n, log2n, h, twg, sm.buf, int(blockIdx.x) * fft_pencils(n),
                           int(threadIdx.x), int(blockDim.x));
}

template <typename T, int L2>
__global__ void __launch_bounds__(512) k_fft_c2r_rows(const typename Cplx<T>::type* __restrict__ in, T* __restrict__ g,
                                                      RowPairs rp, int n, int log2n, int h,
                                                      const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm;
    c2r_unit<T, SyncBlock, L2>(in, g, rp, n, log2n, h, twg, sm.buf, int(blockIdx.x) * fft_pencils(n),
                           int(threadIdx.x), int(blockDim.x));
}

template <typename T, int INM, int OUTM, bool INV, int L2>
__global__ void __launch_bounds__(512) k_fft_axis(const typename Cplx<T>::type* __restrict__ in,
                                                  typename Cplx<T>::type* __restrict__ out, int64_t olo, int64_t ocnt,
                                                  int64_t I, int klo, int kcnt, int n, int log2n, int h,
                                                  const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm;
    axis_unit<T, INM, OUTM, INV, SyncBlock, L2>(in, out, int(olo), int(ocnt), int(I), klo, kcnt, n, log2n, h, twg, sm.buf,
                                            int(blockIdx.x) * fft_pencils(n), int(threadIdx.x), int(blockDim.x));
}

template <typename T, int L2>
__global__ void __launch_bounds__(512) k_fft_axis0_convolve(typename Cplx<T>::type* __restrict__ data, int64_t I,
                                                            int xlo, int xcnt, int n, int log2n, int h,
                                                            const T* __restrict__ mult,
                                                            const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm;
    griddep_launch();
    convolve_unit<T, SyncBlock, L2>(data, int(I), xlo, xcnt, n, log2n, h, mult, twg, sm.buf,
                                int(blockIdx.x) * fft_pencils(n), int(threadIdx.x), int(blockDim.x));
}

// ------------------------------------------------------------ cluster planes
// In 3-D the two grid-side passes on each side of the axis-0 pass -- r2c along
// z then the forward y-transform, and the inverse y-transform then c2r along
// z -- touch one x-plane at a time, so they are done per plane by a
// thread-block cluster of CL blocks that hand the plane over through
// distributed shared memory instead of through global memory and a second
// launch.  Block r of a plane's cluster owns the row pairs
// [r pp, (r+1) pp) of the band (z-pencils, two real rows per complex FFT) and
// the kz-columns [r kp, (r+1) kp) (y-pencils, FULL along y).  Front: each
// block transforms its row pairs, splits them into half spectra and stores
// every (y, kz) value into the y-pencil of the block owning kz; after the
// cluster barrier each block transforms its y-pencils and writes the kept
// frequencies -h..h (CENTERED) to the spectrum.  Back: the reverse, with the
// Hermitian packing of two rows into one complex z-pencil done at the
// exchange.  Positions no block writes (y outside the band; z-frequencies
// h+1 .. n-h-1) are zeroed by their owner before the first cluster barrier,
// which also makes sure every block of the cluster is running before any
// block stores into its shared memory.

__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// The two halves of the cluster barrier (every thread of every block of the
// cluster takes part): arrive releases this thread's earlier shared-memory
// writes, wait acquires those of every thread that arrived.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
// Arrive without ordering this thread's earlier memory accesses (for a
// barrier that only has to show that every block of the cluster is running).
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Shared-memory address of `p` (this block's shared memory) in block `rank`
// of the cluster, and a store of a complex FP32 value there.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, unsigned rank) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// The elements e = tid, tid + nthr, ... of a two-level index e = a B + b,
// walked without a division per step.
struct Walk2 {
    int a, b, da, db, B;
    __device__ __forceinline__ Walk2(int tid, int nthr, int B_) : B(B_) {
        a = tid / B;
        b = tid - a * B;
        da = nthr / B;
        db = nthr - da * B;
    }
    __device__ __forceinline__ void next() {
        a += da;
        b += db;
        if (b >= B) {
            b -= B;
            ++a;
        }
    }
};

// Block of the cluster owning index k of items dealt out `per` to a block
// (k < CL per), and k's position there.
__device__ __forceinline__ int owner_of(int k, int per, int& local) {
    int owner = 0;
    while (k >= per) {
        k -= per;
        ++owner;
    }
    local = k;
    return owner;
}

// A 3-D plan's band as the cluster kernels see it: planes x0 .. x0 + gridDim.x / CL
// - 1, row pairs (ylo + 2 j, ylo + 2 j + 1) for j < np, pp row pairs and kp
// kz-columns per block, h = N/2.
struct Plane3 {
    int x0, ylo, np, pp, kp, h;
};

// Threads per block are PU * (N/8): PU = max(pp, kp) pencils of each kind.
template <int L2, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(512)
    k_fft_front3(float* __restrict__ g, float2* __restrict__ A2, Plane3 pl, const float2* __restrict__ tw) {
    using C = float2;
    constexpr int N = 1 << L2, NS = fft_stride<C>(N), PER = N / 8;
    const int H = pl.h + 1, K = 2 * pl.h + 1;
    const int tid = int(threadIdx.x), nthr = int(blockDim.x), PU = nthr / PER;
    const int r = int(cluster_ctarank());
    const int64_t x = pl.x0 + int(blockIdx.x) / CL;
    griddep_launch();
    FftTw<float, L2> twr;   // both transforms of the block share them
    twr.load(tw, tid);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* rbuf = reinterpret_cast<float2*>(smem_raw);   // PU z-pencils (this block's row pairs)
    float2* ybuf = rbuf + 2 * PU * NS;                    // PU y-pencils (this block's kz-columns)
    const int yhi = pl.ylo + 2 * pl.np;
    for (int e = tid; e < PU * N; e += nthr) {
        const int p = e >> L2, y = e & (N - 1);
        if (y < pl.ylo || y >= yhi || p >= pl.kp || r * pl.kp + p >= H) ybuf[p * NS + pidx<C>(y)] = make_float2(0.f, 0.f);
    }
    // (the zeroed positions are ones no other block writes)
    cluster_arrive_relaxed();

    // this block's row pairs into z-pencils (4 consecutive z per item); the
    // grid rows are zeroed after reading, for the next spreading
    constexpr int G4 = N / 4, IPT = G4 / PER;   // items per thread: 2
    griddep_wait();   // the spreading's grid
    float4 va[IPT], vb[IPT];
    int64_t at[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int e = tid + i * nthr;
        const int p = e / G4, c = e - p * G4;
        const int j = r * pl.pp + p;
        at[i] = -1;
        va[i] = vb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < pl.pp && j < pl.np) {
            at[i] = (x * N + (pl.ylo + 2 * j)) * N + 4 * c;
            va[i] = __ldcg(reinterpret_cast<const float4*>(g + at[i]));
            vb[i] = __ldcg(reinterpret_cast<const float4*>(g + at[i] + N));
        }
    }
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int e = tid + i * nthr;
        const int p = e / G4, c = e - p * G4;
        if (at[i] >= 0) {
            *reinterpret_cast<float4*>(g + at[i]) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(g + at[i] + N) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float2* pen = rbuf + p * NS;
        pen[pidx<C>(4 * c)] = make_float2(va[i].x, vb[i].x);
        pen[pidx<C>(4 * c + 1)] = make_float2(va[i].y, vb[i].y);
        pen[pidx<C>(4 * c + 2)] = make_float2(va[i].z, vb[i].z);
        pen[pidx<C>(4 * c + 3)] = make_float2(va[i].w, vb[i].w);
    }
    const float2* zr = fft_stockham2<float, false, SyncBlock, L2>(rbuf, rbuf + PU * NS, NS, N, L2, tw, tid, twr);
    cluster_wait();

    // half spectra of the two rows of pair j at kz = k, into the owner of column k
    const int nv = max(0, min(pl.pp, pl.np - r * pl.pp));   // this block's valid pairs
    Walk2 wk(tid, nthr, H);
    for (int e = tid; e < nv * H; e += nthr, wk.next()) {
        const int p = wk.a, k = wk.b;
        const float2 zk = zr[p * NS + pidx<C>(k)];
        const float2 zm = zr[p * NS + pidx<C>((N - k) & (N - 1))];
        const float2 a = make_float2((zk.x + zm.x) * 0.5f, (zk.y - zm.y) * 0.5f);
        const float2 b = make_float2((zk.y + zm.y) * 0.5f, (zm.x - zk.x) * 0.5f);
        int col;
        const int owner = owner_of(k, pl.kp, col);
        const int y0 = pl.ylo + 2 * (r * pl.pp + p);
        const uint32_t dst = cluster_addr(ybuf + col * NS, unsigned(owner));
        st_cluster(dst + uint32_t(sizeof(float2) * pidx<C>(y0)), a);
        st_cluster(dst + uint32_t(sizeof(float2) * pidx<C>(y0 + 1)), b);
    }
    cluster_arrive();
    cluster_wait();

    const float2* zy = fft_stockham2<float, false, SyncBlock, L2>(ybuf, ybuf + PU * NS, NS, N, L2, tw, tid, twr);
    const int kv = max(0, min(pl.kp, H - r * pl.kp));   // this block's valid columns
    if (kv > 0) {
        Walk2 wo(tid, nthr, kv);
        for (int e = tid; e < kv * K; e += nthr, wo.next()) {
            const int ky = wo.a, p = wo.b;
            A2[(x * K + ky) * H + r * pl.kp + p] = zy[p * NS + pidx<C>((ky - pl.h) & (N - 1))];
        }
    }
}

template <int L2, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(512)
    k_fft_back3(const float2* __restrict__ A2, float* __restrict__ gout, Plane3 pl, const float2* __restrict__ tw) {
    using C = float2;
    constexpr int N = 1 << L2, NS = fft_stride<C>(N), PER = N / 8;
    const int H = pl.h + 1, K = 2 * pl.h + 1;
    const int tid = int(threadIdx.x), nthr = int(blockDim.x), PU = nthr / PER;
    const int r = int(cluster_ctarank());
    const int64_t x = pl.x0 + int(blockIdx.x) / CL;
    FftTw<float, L2> twr;   // both transforms of the block share them
    twr.load(tw, tid);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* rbuf = reinterpret_cast<float2*>(smem_raw);   // PU z-pencils (this block's row pairs)
    float2* ybuf = rbuf + 2 * PU * NS;                    // PU y-pencils (this block's kz-columns)
    for (int e = tid; e < PU * N; e += nthr) {
        const int p = e >> L2, z = e & (N - 1);
        if ((z > pl.h && z < N - pl.h) || p >= pl.pp || r * pl.pp + p >= pl.np) rbuf[p * NS + pidx<C>(z)] = make_float2(0.f, 0.f);
    }
    // (the zeroed positions are ones no other block writes)
    cluster_arrive_relaxed();

    // this block's kz-columns: frequencies -h..h along y, the rest zero
    const int kv = max(0, min(pl.kp, H - r * pl.kp));
    griddep_wait();   // the axis-0 pass's spectrum
    for (int e = tid; e < PU * N; e += nthr) {
        const int p = e >> L2, y = e & (N - 1);
        if ((y > pl.h && y < N - pl.h) || p >= kv) ybuf[p * NS + pidx<C>(y)] = make_float2(0.f, 0.f);
    }
    if (kv > 0) {
        Walk2 wi(tid, nthr, kv);
        for (int e0 = 0; e0 < kv * K; e0 += kFftLoadsPerRound * nthr) {
            float2 v[kFftLoadsPerRound];
            int slot[kFftLoadsPerRound];
#pragma unroll
            for (int i = 0; i < kFftLoadsPerRound; ++i) {
                const int e = e0 + i * nthr + tid;
                slot[i] = -1;
                if (e < kv * K) {
                    const int ky = wi.a, p = wi.b;
                    v[i] = __ldcg(A2 + (x * K + ky) * H + r * pl.kp + p);
                    slot[i] = p * NS + pidx<C>((ky - pl.h) & (N - 1));
                }
                wi.next();
            }
#pragma unroll
            for (int i = 0; i < kFftLoadsPerRound; ++i)
                if (slot[i] >= 0) ybuf[slot[i]] = v[i];
        }
    }
    const float2* zy = fft_stockham2<float, true, SyncBlock, L2>(ybuf, ybuf + PU * NS, NS, N, L2, tw, tid, twr);
    cluster_wait();

    // rows y0, y0 + 1 of column kz packed into the z-pencil of pair j (its owner's)
    Walk2 ws(tid, nthr, max(kv, 1));
    for (int e = tid; e < kv * pl.np; e += nthr, ws.next()) {
        const int j = ws.a, p = ws.b;
        const int kz = r * pl.kp + p, y0 = pl.ylo + 2 * j;
        float2 a = zy[p * NS + pidx<C>(y0)], b = zy[p * NS + pidx<C>(y0 + 1)];
        int slot;
        const int owner = owner_of(j, pl.pp, slot);
        float2* pen = rbuf + slot * NS;
        if (kz == 0) {
            a.y = 0.f;
            b.y = 0.f;
        }
        st_cluster(cluster_addr(pen + pidx<C>(kz), unsigned(owner)), make_float2(a.x - b.y, a.y + b.x));
        if (kz > 0) st_cluster(cluster_addr(pen + pidx<C>(N - kz), unsigned(owner)), make_float2(a.x + b.y, b.x - a.y));
    }
    cluster_arrive();
    cluster_wait();

    const float2* zr = fft_stockham2<float, true, SyncBlock, L2>(rbuf, rbuf + PU * NS, NS, N, L2, tw, tid, twr);
    constexpr int G4 = N / 4;
    const int nv = max(0, min(pl.pp, pl.np - r * pl.pp));
    for (int e = tid; e < nv * G4; e += nthr) {
        const int p = e / G4, c = e - p * G4;
        const float2* pen = zr + p * NS;
        const float2 s0 = pen[pidx<C>(4 * c)], s1 = pen[pidx<C>(4 * c + 1)], s2 = pen[pidx<C>(4 * c + 2)],
                     s3 = pen[pidx<C>(4 * c + 3)];
        float* row = gout + (x * N + (pl.ylo + 2 * (r * pl.pp + p))) * N + 4 * c;
        *reinterpret_cast<float4*>(row) = make_float4(s0.x, s1.x, s2.x, s3.x);
        *reinterpret_cast<float4*>(row + N) = make_float4(s0.y, s1.y, s2.y, s3.y);
    }
}

// 1-D: multiply the half spectrum of row 0 by M[k], k = 0..h.
template <typename T>
__global__ void k_mult_half(typename Cplx<T>::type* __restrict__ A1, int h, const T* __restrict__ mult) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= h) {
        A1[k].x *= mult[k];
        A1[k].y *= mult[k];
    }
}

// Half spectrum S (dims (2h+1)^(d-1) x (h+1)) -> full Hermitian FP64 array over
// {-h..h}^d, divided by the window transform prod_t psihat(k_t).
template <typename T>
__global__ void k_extract_adjoint(const typename Cplx<T>::type* __restrict__ S, int d, int h,
                                  const double* __restrict__ psihat, double* __restrict__ out) {
    const int K = 2 * h + 1;
    int64_t total = 1;
    for (int t = 0; t < d; ++t) total *= K;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int k[3] = {0, 0, 0};
    int64_t rem = idx;
    for (int t = d - 1; t >= 0; --t) { k[t] = int(rem % K) - h; rem /= K; }
    const bool flip = k[d - 1] < 0;
    int64_t s = 0;
    double den = 1.0;
    for (int t = 0; t < d; ++t) {
        const int kt = flip ? -k[t] : k[t];
        s = (t == d - 1) ? s * (h + 1) + kt : s * K + (kt + h);
        den *= psihat[k[t] + h];
    }
    const double re = double(S[s].x), im = double(S[s].y);
    out[2 * idx] = re / den;
    out[2 * idx + 1] = (flip ? -im : im) / den;
}

// Hermitian FP64 array over {-h..h}^d -> half spectrum S with the weights c_k
// and the window deconvolution folded in.
template <typename T>
__global__ void k_fill_forward(const double* __restrict__ fhat, int d, int h, const double* __restrict__ psihat,
                               typename Cplx<T>::type* __restrict__ S) {
    const int K = 2 * h + 1;
    int64_t total = h + 1;
    for (int t = 0; t < d - 1; ++t) total *= K;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int k[3] = {0, 0, 0};
    int64_t rem = idx;
    k[d - 1] = int(rem % (h + 1));
    rem /= (h + 1);
    for (int t = d - 2; t >= 0; --t) { k[t] = int(rem % K) - h; rem /= K; }
    int64_t f = 0;
    double c = 1.0;
    for (int t = 0; t < d; ++t) {
        f = f * K + (k[t] + h);
        c /= psihat[k[t] + h];
    }
    c *= re_weight(k, d, h);
    S[idx].x = T(fhat[2 * f] * c);
    S[idx].y = T(fhat[2 * f + 1] * c);
}

// ------------------------------------------------------------------ launchers

template <typename T>
static size_t fft_smem_bytes(int n) {
    using C = typename Cplx<T>::type;
    return 2 * size_t(fft_pencils(n)) * size_t(fft_stride<C>(n)) * sizeof(C);
}

// Largest dynamic shared memory any FFT launch of this precision can use:
// two buffers of one pencil of the largest length, 4096.
template <typename T>
static size_t fft_smem_max() {
    using C = typename Cplx<T>::type;
    return 2 * size_t(fft_stride<C>(4096)) * sizeof(C);
}

// Opt a kernel into its largest shared-memory size once per device (the cache
// is per kernel: K is the kernel itself, not its type).
template <typename T, auto K>
static cudaError_t ensure_smem() {
    const size_t bytes = fft_smem_max<T>();
    if (bytes <= 48 * 1024) return cudaSuccess;
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured & (1ull << (dev & 63))) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) configured |= (1ull << (dev & 63));
    return e;
}

// A launch, with programmatic stream serialization when `pdl` (the kernel may
// start while its predecessor in the stream finishes; it waits in
// griddep_wait() before reading what the predecessor wrote).
template <typename... Exp, typename... Act>
static cudaError_t launch_pdl(bool pdl, void (*kern)(Exp...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t s, Act&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Act>(args)...);
}

#define SK_TRY(x)                                   \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

// Row pairs of the real passes for the plan's grid: all rows of the 1-D grid
// (the data row and its zero partner); in 2-D the rows x of the band, paired
// (x, x+1); in 3-D the rows (x, y) of the band, paired along y.
static RowPairs row_pairs(const FftPlan& f) {
    RowPairs rp{};
    if (f.d == 1) {
        rp.olo = 0; rp.ostride = 0; rp.ylo = 0; rp.npo = 1; rp.npairs = 1;
        return rp;
    }
    const int a = f.d == 2 ? 0 : 1;                 // the axis whose rows are paired
    const int ylo = f.lo[a] & ~1;
    const int yhi = f.hi[a] | 1;                    // inclusive, odd
    rp.ylo = ylo;
    rp.npo = (yhi - ylo + 1) / 2;
    if (f.d == 2) {
        rp.olo = 0; rp.ostride = 0; rp.npairs = rp.npo;
    } else {
        rp.olo = f.lo[0]; rp.ostride = f.n; rp.npairs = int64_t(f.hi[0] - f.lo[0] + 1) * rp.npo;
    }
    return rp;
}

// The pass kernels come in versions for the transform lengths the workloads
// use (2^6, 2^7, 2^8 and, in FP32, 2^10: the length a compile-time constant)
// and a version for any length (L2 = 0).
#define SK_FFT_LENGTHS(T, LOG2N, CALL)                        \
    switch (LOG2N) {                                          \
        case 6: { constexpr int L2 = 6; CALL; } break;         \
        case 7: { constexpr int L2 = 7; CALL; } break;         \
        case 8: { constexpr int L2 = 8; CALL; } break;         \
        case 10:                                              \
            if constexpr (sizeof(T) == 4) {                   \
                constexpr int L2 = 10;                        \
                CALL;                                         \
                break;                                        \
            }                                                 \
            [[fallthrough]];                                  \
        default: { constexpr int L2 = 0; CALL; } break;        \
    }

template <typename T, int L2>
static cudaError_t run_r2c_l(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_r2c_rows<T, L2>>()));
    const RowPairs rp = row_pairs(f);
    const int P = fft_pencils(f.n);
    k_fft_r2c_rows<T, L2><<<unsigned((rp.npairs + P - 1) / P), fft_threads<T>(f.n), fft_smem_bytes<T>(f.n), s>>>(
        static_cast<T*>(f.grid), static_cast<C*>(f.A1), rp, f.n, f.log2n, f.h, static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t run_r2c(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    SK_FFT_LENGTHS(T, f.log2n, return (run_r2c_l<T, L2>(f, launches, s)))
    return cudaErrorInvalidValue;
}

template <typename T, int L2>
static cudaError_t run_c2r_l(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_c2r_rows<T, L2>>()));
    const RowPairs rp = row_pairs(f);
    const int P = fft_pencils(f.n);
    k_fft_c2r_rows<T, L2><<<unsigned((rp.npairs + P - 1) / P), fft_threads<T>(f.n), fft_smem_bytes<T>(f.n), s>>>(
        static_cast<const C*>(f.A1), static_cast<T*>(f.grid_out), rp, f.n, f.log2n, f.h,
        static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t run_c2r(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    SK_FFT_LENGTHS(T, f.log2n, return (run_c2r_l<T, L2>(f, launches, s)))
    return cudaErrorInvalidValue;
}

template <typename T, int INM, int OUTM, bool INV, int L2>
static cudaError_t run_axis_l(const FftPlan& f, const void* in, void* out, int64_t olo, int64_t ocnt, int64_t I,
                              int klo, int kcnt, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_axis<T, INM, OUTM, INV, L2>>()));
    const int P = fft_pencils(f.n);
    const int64_t Q = ocnt * I;
    k_fft_axis<T, INM, OUTM, INV, L2><<<unsigned((Q + P - 1) / P), fft_threads<T>(f.n), fft_smem_bytes<T>(f.n), s>>>(
        static_cast<const C*>(in), static_cast<C*>(out), olo, ocnt, I, klo, kcnt, f.n, f.log2n, f.h,
        static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T, int INM, int OUTM, bool INV>
static cudaError_t run_axis(const FftPlan& f, const void* in, void* out, int64_t olo, int64_t ocnt, int64_t I,
                            int klo, int kcnt, int64_t* launches, cudaStream_t s) {
    SK_FFT_LENGTHS(T, f.log2n,
                   return (run_axis_l<T, INM, OUTM, INV, L2>(f, in, out, olo, ocnt, I, klo, kcnt, launches, s)))
    return cudaErrorInvalidValue;
}

// Axis-0 positions the spectra hold outside zero: the band, widened to the
// row pairs in 2-D (where axis 0 is the paired axis).
static void axis0_range(const FftPlan& f, int& lo, int& cnt) {
    lo = f.lo[0];
    int hi = f.hi[0];
    if (f.d == 2) {
        lo &= ~1;
        hi |= 1;
    }
    cnt = hi - lo + 1;
}

template <typename T, int L2>
static cudaError_t run_axis0_convolve_l(const FftPlan& f, void* data, int64_t I, int64_t* launches, cudaStream_t s,
                                        bool pdl = false) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_axis0_convolve<T, L2>>()));
    const int P = fft_pencils(f.n);
    int xlo, xcnt;
    axis0_range(f, xlo, xcnt);
    SK_TRY(launch_pdl(pdl, k_fft_axis0_convolve<T, L2>, unsigned((I + P - 1) / P), unsigned(fft_threads<T>(f.n)),
                      fft_smem_bytes<T>(f.n), s, static_cast<C*>(data), I, xlo, xcnt, f.n, f.log2n, f.h,
                      static_cast<const T*>(f.mult), static_cast<const C*>(f.tw)));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t run_axis0_convolve(const FftPlan& f, void* data, int64_t I, int64_t* launches, cudaStream_t s) {
    SK_FFT_LENGTHS(T, f.log2n, return (run_axis0_convolve_l<T, L2>(f, data, I, launches, s)))
    return cudaErrorInvalidValue;
}

// Smallest cluster the plane kernels use (a plane's work split over at least
// this many blocks, so that the ~60-120 planes of a band fill the GPU).
constexpr int kPlaneClusterMin = 2;

// Cluster size, band description and block size of the plane kernels for a
// plan; false where they do not apply (FP32 3-D plans with n_os = 64, 128 or
// 256, and at most 512 threads per block with clusters of up to 8).
static bool plane_shape(const FftPlan& f, int& CL, Plane3& pl, int& threads) {
    if (f.d != 3 || f.log2n < 6 || f.log2n > 8) return false;
    const int H = f.h + 1, per = f.n / 8;
    pl.x0 = f.lo[0];
    pl.ylo = f.lo[1] & ~1;
    pl.np = ((f.hi[1] | 1) - pl.ylo + 1) / 2;
    pl.h = f.h;
    for (CL = kPlaneClusterMin; CL <= 8; CL *= 2) {
        pl.pp = (pl.np + CL - 1) / CL;
        pl.kp = (H + CL - 1) / CL;
        threads = std::max(pl.pp, pl.kp) * per;
        if (threads <= 512) return true;
    }
    return false;
}

bool fft_planes_supported(const FftPlan& f, bool fp32) {
    int CL, threads;
    Plane3 pl;
    return fp32 && plane_shape(f, CL, pl, threads);
}

// Opt a plane kernel into the shared memory of its largest block once per
// device: 512 threads, i.e. 4096 / n pencils of each kind, two buffers each.
template <auto Kern, int L2>
static cudaError_t ensure_plane_smem() {
    constexpr size_t bytes = size_t(4) * (512 / ((1 << L2) / 8)) * fft_stride<float2>(1 << L2) * sizeof(float2);
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured & (1ull << (dev & 63))) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) configured |= (1ull << (dev & 63));
    return e;
}

template <int L2, int CL>
static cudaError_t run_planes_cl(const FftPlan& f, const Plane3& pl, int threads, int64_t* launches, cudaStream_t s) {
    SK_TRY((ensure_plane_smem<k_fft_front3<L2, CL>, L2>()));
    SK_TRY((ensure_plane_smem<k_fft_back3<L2, CL>, L2>()));
    const int64_t H = f.h + 1, K = 2 * f.h + 1;
    const unsigned blocks = unsigned((f.hi[0] - f.lo[0] + 1) * CL);
    const size_t smem = size_t(4) * (threads / ((1 << L2) / 8)) * fft_stride<float2>(1 << L2) * sizeof(float2);
    const float2* tw = static_cast<const float2*>(f.tw);
    SK_TRY(launch_pdl(f.pdl, k_fft_front3<L2, CL>, blocks, unsigned(threads), smem, s, static_cast<float*>(f.grid),
                      static_cast<float2*>(f.A2), pl, tw));
    if (launches) ++*launches;
    SK_TRY((run_axis0_convolve_l<float, L2>(f, f.A2, K * H, launches, s, f.pdl)));
    SK_TRY(launch_pdl(f.pdl, k_fft_back3<L2, CL>, blocks, unsigned(threads), smem, s,
                      static_cast<const float2*>(f.A2), static_cast<float*>(f.grid_out), pl, tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <int L2>
static cudaError_t run_planes_l(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    int CL, threads;
    Plane3 pl;
    if (!plane_shape(f, CL, pl, threads)) return cudaErrorInvalidValue;
    if (CL == 2) return run_planes_cl<L2, 2>(f, pl, threads, launches, s);
    if (CL == 4) return run_planes_cl<L2, 4>(f, pl, threads, launches, s);
    return run_planes_cl<L2, 8>(f, pl, threads, launches, s);
}

// 3-D FP32 product with the plane kernels: front (r2c z, forward y), the
// axis-0 pass with the multiply, back (inverse y, c2r z): three launches.
static cudaError_t run_planes(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    switch (f.log2n) {
        case 6: return run_planes_l<6>(f, launches, s);
        case 7: return run_planes_l<7>(f, launches, s);
        case 8: return run_planes_l<8>(f, launches, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_fft_convolve(const FftPlan& f, cudaStream_t s, int64_t* launches) {
    using C = typename Cplx<T>::type;
    const int64_t n = f.n, H = f.h + 1, K = 2 * f.h + 1;
    if constexpr (sizeof(T) == 4) {
        if (f.planes) return run_planes(f, launches, s);
    }
    if (f.d == 1) {
        SK_TRY(run_r2c<T>(f, launches, s));
        k_mult_half<T><<<unsigned((H + 255) / 256), 256, 0, s>>>(static_cast<C*>(f.A1), f.h,
                                                                 static_cast<const T*>(f.mult));
        if (launches) ++*launches;
        SK_TRY(cudaGetLastError());
        return run_c2r<T>(f, launches, s);
    }
    if (f.d == 2) {
        SK_TRY(run_r2c<T>(f, launches, s));
        SK_TRY(run_axis0_convolve<T>(f, f.A1, H, launches, s));
        return run_c2r<T>(f, launches, s);
    }
    const int64_t xlo = f.lo[0], xcnt = f.hi[0] - f.lo[0] + 1;
    const int ylo = f.lo[1] & ~1, ycnt = (f.hi[1] | 1) - ylo + 1;   // the row pairs of the real passes
    SK_TRY(run_r2c<T>(f, launches, s));
    SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A1, f.A2, xlo, xcnt, H, 0, 0, launches, s)));
    SK_TRY(run_axis0_convolve<T>(f, f.A2, K * H, launches, s));
    SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A2, f.A1, xlo, xcnt, H, ylo, ycnt, launches, s)));
    (void)n;
    return run_c2r<T>(f, launches, s);
}

template <typename T>
cudaError_t launch_fft_adjoint(const FftPlan& f, double* fhat, cudaStream_t s, int64_t* launches) {
    using C = typename Cplx<T>::type;
    const int64_t H = f.h + 1, K = 2 * f.h + 1;
    const void* S = nullptr;
    if (f.d == 1) {
        SK_TRY(run_r2c<T>(f, launches, s));
        S = f.A1;
    } else if (f.d == 2) {
        SK_TRY(run_r2c<T>(f, launches, s));
        SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A1, f.A3, 0, 1, H, 0, 0, launches, s)));
        S = f.A3;
    } else {
        SK_TRY(run_r2c<T>(f, launches, s));
        SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A1, f.A2, f.lo[0], f.hi[0] - f.lo[0] + 1, H, 0, 0,
                                                   launches, s)));
        SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A2, f.A3, 0, 1, K * H, 0, 0, launches, s)));
        S = f.A3;
    }
    int64_t total = 1;
    for (int t = 0; t < f.d; ++t) total *= K;
    k_extract_adjoint<T><<<unsigned((total + 255) / 256), 256, 0, s>>>(static_cast<const C*>(S), f.d, f.h,
                                                                      f.psihat, fhat);
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_forward(const FftPlan& f, const double* fhat, cudaStream_t s, int64_t* launches) {
    using C = typename Cplx<T>::type;
    const int64_t n = f.n, H = f.h + 1, K = 2 * f.h + 1;
    void* S = f.d == 1 ? f.A1 : f.A3;
    int64_t total = H;
    for (int t = 0; t < f.d - 1; ++t) total *= K;
    if (f.d == 1) SK_TRY(cudaMemsetAsync(f.A1, 0, size_t(2 * H) * sizeof(C), s));
    k_fill_forward<T><<<unsigned((total + 255) / 256), 256, 0, s>>>(fhat, f.d, f.h, f.psihat, static_cast<C*>(S));
    if (launches) ++*launches;
    SK_TRY(cudaGetLastError());
    int xlo, xcnt;
    axis0_range(f, xlo, xcnt);
    (void)n;
    if (f.d == 1) return run_c2r<T>(f, launches, s);
    if (f.d == 2) {
        SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A3, f.A1, 0, 1, H, xlo, xcnt, launches, s)));
        return run_c2r<T>(f, launches, s);
    }
    const int ylo = f.lo[1] & ~1, ycnt = (f.hi[1] | 1) - ylo + 1;
    SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A3, f.A2, 0, 1, K * H, xlo, xcnt, launches, s)));
    SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A2, f.A1, xlo, xcnt, H, ylo, ycnt, launches, s)));
    return run_c2r<T>(f, launches, s);
}

template cudaError_t launch_fft_convolve<float>(const FftPlan&, cudaStream_t, int64_t*);
template cudaError_t launch_fft_convolve<double>(const FftPlan&, cudaStream_t, int64_t*);
template cudaError_t launch_fft_adjoint<float>(const FftPlan&, double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_adjoint<double>(const FftPlan&, double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_forward<float>(const FftPlan&, const double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_forward<double>(const FftPlan&, const double*, cudaStream_t, int64_t*);

}  // namespace sk
