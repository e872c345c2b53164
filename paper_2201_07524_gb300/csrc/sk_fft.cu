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
//     Element e of a pencil sits at e + e/8 (one pad per 8 elements), which
//     keeps the stride-R stores of the first stages and the parallel walks of
//     the load phases off each other's shared-memory banks.
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
#include "sk_internal.cuh"

namespace sk {

enum { FULL = 0, CENTERED = 1 };

constexpr int kFftBlockElems = 256;

__host__ __device__ __forceinline__ int fft_pencils(int n) { return n >= kFftBlockElems ? 1 : kFftBlockElems / n; }

// Elements of a pencil per thread: 8 in FP32 (radix-8 stages); 4 in FP64
// (radix-4 stages), whose arithmetic is slow enough on this GPU that the
// shorter per-thread chains and twice the threads pay -- except for pencils
// longer than 2048, which keep 8 so that a block stays within 512 threads.
template <typename T>
__host__ __device__ __forceinline__ int fft_ept(int n) { return (sizeof(T) == 8 && n <= 2048) ? 4 : 8; }

// Threads of an FFT block (16 to 512).
template <typename T>
__host__ __device__ __forceinline__ int fft_threads(int n) { return fft_pencils(n) * n / fft_ept<T>(n); }

// Padded position of element e of a pencil; a pencil spans fft_stride(n) slots.
__host__ __device__ __forceinline__ int pidx(int e) { return e + (e >> 3); }
__host__ __device__ __forceinline__ int fft_stride(int n) { return n + n / 8; }

// Row pairs of the real passes: pair q covers rows r0 = o * ostride + y and
// r0 + 1 with o = olo + q / npo and y = ylo + 2 (q % npo).
struct RowPairs {
    int64_t olo, ostride;
    int ylo, npo;
    int64_t npairs;
};

__device__ __forceinline__ int64_t pair_row(const RowPairs& rp, int64_t q) {
    const int64_t o = rp.olo + q / rp.npo;
    return o * rp.ostride + rp.ylo + 2 * (q % rp.npo);
}

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

// Barriers of an FFT unit: a whole block (the pass kernels), or one warp (a
// unit of 32 threads inside the persistent kernel).
struct SyncBlock {
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};
struct SyncWarp {
    __device__ __forceinline__ static void sync() { __syncwarp(); }
};

// One Stockham stage of radix R on the thread's E elements (E/R butterflies):
// butterfly jj reads x_q = X[jj + q n/R], scales it by w_L^(q k) (L = Ns R,
// k = jj mod Ns), takes the R-point DFT and writes y_r to
// X[(jj - k) R + k + r Ns].  All reads precede a barrier, then the writes.
template <typename C, bool INV, int R, int E, class S>
__device__ __forceinline__ void stockham_stage(C* pen, int n, int Ns, int t, const C* tw) {
    constexpr int B = E / R;
    const int stride = n / R, per = n / E;
    C x[E];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int jj = t + b * per;
#pragma unroll
        for (int r = 0; r < R; ++r) x[b * R + r] = pen[pidx(jj + r * stride)];
    }
    S::sync();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int jj = t + b * per;
        const int k = jj & (Ns - 1);
        const int step = k * (n / (Ns * R));
#pragma unroll
        for (int q = 1; q < R; ++q) x[b * R + q] = cmul(x[b * R + q], twiddle<C, INV>(tw, q * step, n));
        if (R == 8) dft8<C, INV>(x + b * R);
        else if (R == 4) dft4<C, INV>(x + b * R);
        else dft2<C, INV>(x + b * R);
        const int base = (jj - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) pen[pidx(base + r * Ns)] = x[b * R + r];
    }
    S::sync();
}

// Transform the unit's P pencils in place (natural order in and out; pencil
// p at buf + p * ns, element e at pidx(e)); the unit has exactly
// fft_threads<T>(n) threads, `tid` is the thread's index in it.  `tw` is the
// block's shared copy of the n/2 twiddles.  Radix E = fft_ept stages while
// they fit, then one of radix 4 or 2.
template <typename C, bool INV, int E, class S>
__device__ __forceinline__ void stockham_all(C* buf, int ns, int n, int log2n, const C* tw, int tid) {
    constexpr int LE = E == 8 ? 3 : 2;
    const int per = n / E;
    const int p = tid / per, t = tid - p * per;
    C* pen = buf + p * ns;
    int Ns = 1, rem = log2n;
    for (; rem >= LE; rem -= LE, Ns <<= LE) stockham_stage<C, INV, E, E, S>(pen, n, Ns, t, tw);
    if (rem == 2) stockham_stage<C, INV, 4, E, S>(pen, n, Ns, t, tw);
    else if (rem == 1) stockham_stage<C, INV, 2, E, S>(pen, n, Ns, t, tw);
}

template <typename T, bool INV, class S>
__device__ void fft_stockham(typename Cplx<T>::type* buf, int ns, int n, int log2n, const typename Cplx<T>::type* tw,
                             int tid) {
    using C = typename Cplx<T>::type;
    S::sync();
    if (fft_ept<T>(n) == 4)
        stockham_all<C, INV, 4, S>(buf, ns, n, log2n, tw, tid);
    else
        stockham_all<C, INV, 8, S>(buf, ns, n, log2n, tw, tid);
}

// Shared memory of an FFT block: the n/2 twiddles, then P pencils of n + 1.
template <typename T>
struct FftSmem {
    using C = typename Cplx<T>::type;
    C* tw;
    C* buf;
    __device__ __forceinline__ explicit FftSmem(int n) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        tw = reinterpret_cast<C*>(smem_raw);
        buf = tw + n / 2;
    }
};

template <typename C>
__device__ __forceinline__ void load_twiddles(C* dst, const C* __restrict__ src, int n) {
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) dst[k] = src[k];
}

// Elements a thread loads per round; a round's loads are all issued before
// any of them is stored, so their latencies overlap.
constexpr int kFftLoadsPerRound = 8;

// The passes below are written for one FFT unit: `nthr` threads (a block of a
// pass kernel, or a warp of the persistent kernel) that transform the P
// pencils starting at pencil (or row pair) q0, thread `tid` of the unit,
// staging in `buf` (P pencils of fft_stride(n) slots).  Data written by an
// earlier pass is loaded with ld.global.cg (L2, not L1), so a persistent
// kernel that runs several passes never reads a stale line from L1.

// Two real rows of length n -> two half spectra of length h+1 (output rows
// are the same row indices in A1).  The input rows are zeroed after reading.
template <typename T, class S>
__device__ __forceinline__ void r2c_unit(T* __restrict__ g, typename Cplx<T>::type* __restrict__ out,
                                         const RowPairs& rp, int n, int log2n, int h,
                                         const typename Cplx<T>::type* tw, typename Cplx<T>::type* buf, int64_t q0,
                                         int tid, int nthr) {
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n);
    const int ns = fft_stride(n);
    S::sync();   // the unit's previous pencils have been read out of buf
    for (int e0 = 0; e0 < P * n; e0 += kFftLoadsPerRound * nthr) {
        C z[kFftLoadsPerRound];
        int64_t at[kFftLoadsPerRound];
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            const int64_t q = q0 + (e >> log2n);
            z[j].x = T(0);
            z[j].y = T(0);
            at[j] = -1;
            if (e < P * n && q < rp.npairs) {
                at[j] = pair_row(rp, q) * n + (e & (n - 1));
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
            buf[(e >> log2n) * ns + pidx(e & (n - 1))] = z[j];
        }
    }
    fft_stockham<T, false, S>(buf, ns, n, log2n, tw, tid);
    const int H = h + 1;
    for (int e = tid; e < P * H; e += nthr) {
        const int p = e / H;
        const int k = e - p * H;
        const int64_t q = q0 + p;
        if (q >= rp.npairs) continue;
        const int64_t r0 = pair_row(rp, q);
        const C zk = buf[p * ns + pidx(k)];
        const C zm = buf[p * ns + pidx((n - k) & (n - 1))];
        C A, Bv;
        A.x = (zk.x + zm.x) * T(0.5);
        A.y = (zk.y - zm.y) * T(0.5);
        Bv.x = (zk.y + zm.y) * T(0.5);
        Bv.y = (zm.x - zk.x) * T(0.5);
        out[r0 * H + k] = A;
        out[(r0 + 1) * H + k] = Bv;
    }
}

// Two half spectra -> two real rows, by Hermitian completion.
template <typename T, class S>
__device__ __forceinline__ void c2r_unit(const typename Cplx<T>::type* __restrict__ in, T* __restrict__ g,
                                         const RowPairs& rp, int n, int log2n, int h,
                                         const typename Cplx<T>::type* tw, typename Cplx<T>::type* buf, int64_t q0,
                                         int tid, int nthr) {
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n);
    const int ns = fft_stride(n);
    S::sync();   // the unit's previous pencils have been read out of buf
    const int H = h + 1;
    for (int e0 = 0; e0 < P * n; e0 += kFftLoadsPerRound * nthr) {
        C A[kFftLoadsPerRound], Bv[kFftLoadsPerRound];
        int sgn[kFftLoadsPerRound];   // +1: k in 0..h, -1: -k in 1..h, 0: outside (zero)
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            const int pos = e & (n - 1);
            const int64_t q = q0 + (e >> log2n);
            const int k = pos <= (n >> 1) ? pos : pos - n;
            sgn[j] = 0;
            A[j].x = A[j].y = Bv[j].x = Bv[j].y = T(0);
            if (e < P * n && q < rp.npairs && k >= -h && k <= h) {
                const int64_t r0 = pair_row(rp, q);
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
            buf[(e >> log2n) * ns + pidx(pos)] = z;
        }
    }
    fft_stockham<T, true, S>(buf, ns, n, log2n, tw, tid);
    for (int e = tid; e < P * n; e += nthr) {
        const int p = e >> log2n;
        const int l = e & (n - 1);
        const int64_t q = q0 + p;
        if (q >= rp.npairs) continue;
        const int64_t r0 = pair_row(rp, q);
        const C v = buf[p * ns + pidx(l)];
        g[r0 * n + l] = v.x;
        g[(r0 + 1) * n + l] = v.y;
    }
}

// Pencils along the middle axis of an (O, L, I) array: element k of pencil
// (o, i) sits at (o*L + k)*I + i.  FULL keeps all n entries along the axis;
// CENTERED stores frequencies -h..h at positions 0..2h.  Only pencils with
// o in [olo, olo + ocnt) are transformed, and a FULL output is stored only for
// k in [klo, klo + kcnt).
template <typename T, int INM, int OUTM, bool INV, class S>
__device__ __forceinline__ void axis_unit(const typename Cplx<T>::type* __restrict__ in,
                                          typename Cplx<T>::type* __restrict__ out, int64_t olo, int64_t ocnt,
                                          int64_t I, int klo, int kcnt, int n, int log2n, int h,
                                          const typename Cplx<T>::type* tw, typename Cplx<T>::type* buf, int64_t q0,
                                          int tid, int nthr) {
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n);
    const int ns = fft_stride(n);
    S::sync();   // the unit's previous pencils have been read out of buf
    const int64_t Q = ocnt * I;
    const int Lin = INM == FULL ? n : 2 * h + 1;
    const int Lout = OUTM == FULL ? n : 2 * h + 1;
    const int k0 = OUTM == FULL ? klo : 0;
    const int kn = OUTM == FULL ? kcnt : Lout;
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
            const int k = e / P;
            const int64_t q = q0 + (e - k * P);
            ok[j] = e < P * Lin && q < Q;
            if (ok[j]) v[j] = __ldcg(in + ((olo + q / I) * Lin + k) * I + q % I);
        }
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            if (!ok[j]) continue;
            const int e = e0 + j * nthr + tid;
            const int k = e / P;
            const int pos = INM == FULL ? k : ((k - h) & (n - 1));
            buf[(e - k * P) * ns + pidx(pos)] = v[j];
        }
    }
    fft_stockham<T, INV, S>(buf, ns, n, log2n, tw, tid);
    for (int e = tid; e < P * kn; e += nthr) {
        const int kk = e / P;
        const int pl = e - kk * P;
        const int64_t q = q0 + pl;
        if (q >= Q) continue;
        const int k = k0 + kk;
        const int64_t o = olo + q / I, i = q % I;
        const int pos = OUTM == FULL ? k : ((k - h) & (n - 1));
        out[(o * Lout + k) * I + i] = buf[pl * ns + pidx(pos)];
    }
}

// Pencils along axis 0 of an (n, I) array: forward FFT, multiply the kept
// frequencies by M[(k+h)*I + q] and zero the rest, inverse FFT, in place.
// Only axis-0 positions in [xlo, xlo + xcnt) are loaded (the rest are zero)
// and stored (the rest are never read).
template <typename T, class S>
__device__ __forceinline__ void convolve_unit(typename Cplx<T>::type* __restrict__ data, int64_t I, int xlo, int xcnt,
                                              int n, int log2n, int h, const T* __restrict__ mult,
                                              const typename Cplx<T>::type* tw, typename Cplx<T>::type* buf,
                                              int64_t q0, int tid, int nthr) {
    using C = typename Cplx<T>::type;
    const int P = fft_pencils(n);
    const int ns = fft_stride(n);
    S::sync();   // the unit's previous pencils have been read out of buf
    for (int e0 = 0; e0 < P * n; e0 += kFftLoadsPerRound * nthr) {
        C v[kFftLoadsPerRound];
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            const int k = e / P;
            const int64_t q = q0 + (e - k * P);
            v[j].x = T(0);
            v[j].y = T(0);
            if (e < P * n && q < I && k >= xlo && k < xlo + xcnt) v[j] = __ldcg(data + int64_t(k) * I + q);
        }
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = e0 + j * nthr + tid;
            if (e >= P * n) continue;
            const int k = e / P;
            buf[(e - k * P) * ns + pidx(k)] = v[j];
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
        const int pos = e / P;
        const int64_t q = q0 + (e - pos * P);
        const int k = pos <= (n >> 1) ? pos : pos - n;
        mv[j] = (one_round && e < P * n && q < I && k >= -h && k <= h) ? mult[int64_t(k + h) * I + q] : T(0);
    }
    fft_stockham<T, false, S>(buf, ns, n, log2n, tw, tid);
    if (one_round) {
#pragma unroll
        for (int j = 0; j < kFftLoadsPerRound; ++j) {
            const int e = j * nthr + tid;
            if (e >= P * n) continue;
            const int pos = e / P;
            C& v = buf[(e - pos * P) * ns + pidx(pos)];
            v.x *= mv[j];
            v.y *= mv[j];
        }
    } else {
        for (int e = tid; e < P * n; e += nthr) {
            const int pos = e / P;
            const int pl = e - pos * P;
            const int64_t q = q0 + pl;
            const int k = pos <= (n >> 1) ? pos : pos - n;
            C& v = buf[pl * ns + pidx(pos)];
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
    fft_stockham<T, true, S>(buf, ns, n, log2n, tw, tid);
    for (int e = tid; e < P * xcnt; e += nthr) {
        const int k = xlo + e / P;
        const int pl = e % P;
        const int64_t q = q0 + pl;
        if (q < I) data[int64_t(k) * I + q] = buf[pl * ns + pidx(k)];
    }
}

// ------------------------------------------------------------ pass kernels
// One launch per pass; a block is one unit of fft_threads<T>(n) threads.

template <typename T>
__global__ void __launch_bounds__(512) k_fft_r2c_rows(T* __restrict__ g, typename Cplx<T>::type* __restrict__ out,
                                                      RowPairs rp, int n, int log2n, int h,
                                                      const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm(n);
    load_twiddles(sm.tw, twg, n);
    r2c_unit<T, SyncBlock>(g, out, rp, n, log2n, h, sm.tw, sm.buf, int64_t(blockIdx.x) * fft_pencils(n),
                           int(threadIdx.x), int(blockDim.x));
}

template <typename T>
__global__ void __launch_bounds__(512) k_fft_c2r_rows(const typename Cplx<T>::type* __restrict__ in, T* __restrict__ g,
                                                      RowPairs rp, int n, int log2n, int h,
                                                      const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm(n);
    load_twiddles(sm.tw, twg, n);
    c2r_unit<T, SyncBlock>(in, g, rp, n, log2n, h, sm.tw, sm.buf, int64_t(blockIdx.x) * fft_pencils(n),
                           int(threadIdx.x), int(blockDim.x));
}

template <typename T, int INM, int OUTM, bool INV>
__global__ void __launch_bounds__(512) k_fft_axis(const typename Cplx<T>::type* __restrict__ in,
                                                  typename Cplx<T>::type* __restrict__ out, int64_t olo, int64_t ocnt,
                                                  int64_t I, int klo, int kcnt, int n, int log2n, int h,
                                                  const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm(n);
    load_twiddles(sm.tw, twg, n);
    axis_unit<T, INM, OUTM, INV, SyncBlock>(in, out, olo, ocnt, I, klo, kcnt, n, log2n, h, sm.tw, sm.buf,
                                            int64_t(blockIdx.x) * fft_pencils(n), int(threadIdx.x), int(blockDim.x));
}

template <typename T>
__global__ void __launch_bounds__(512) k_fft_axis0_convolve(typename Cplx<T>::type* __restrict__ data, int64_t I,
                                                            int xlo, int xcnt, int n, int log2n, int h,
                                                            const T* __restrict__ mult,
                                                            const typename Cplx<T>::type* __restrict__ twg) {
    const FftSmem<T> sm(n);
    load_twiddles(sm.tw, twg, n);
    convolve_unit<T, SyncBlock>(data, I, xlo, xcnt, n, log2n, h, mult, sm.tw, sm.buf,
                                int64_t(blockIdx.x) * fft_pencils(n), int(threadIdx.x), int(blockDim.x));
}

// ------------------------------------------------------------ persistent 3-D convolution
// All five passes of a 3-D product in one cooperative launch: one block of
// kCoopWarps = 16 warps per SM (so a thread may hold up to 128 registers),
// every warp an FFT unit (FP32 pencils of up to 256
// points: 32 threads), the twiddles loaded once per block.  Between passes
// the grid meets at a barrier; each pass's units are spread over all warps
// of the grid.  Every barrier wait is bounded.
constexpr int kCoopWarps = 16;

__device__ __forceinline__ unsigned long long fft_global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier number k (1, 2, ...): every block arrives once, then its first
// thread waits until all blocks have arrived k times.  The wait gives up
// after about a second (the global timer) or 2^24 polls: the block then sets
// bit 2 of the status word and the barrier returns false, so the kernel skips
// its remaining passes (the other blocks' waits run out the same way).
__device__ __forceinline__ bool coop_barrier(const FftPlan& f, unsigned k) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(f.bar, 1u);
        const unsigned target = k * gridDim.x + (f.inject ? 1u : 0u);
        bool good = false;
        unsigned long long t0 = 0ull;
        for (int it = 0; it < (1 << 24); ++it) {
            if (ld_acquire_gpu(f.bar) >= target) {
                good = true;
                break;
            }
            if ((it & 63) == 0) {
                const unsigned long long now = fft_global_ns();
                if (it == 0) t0 = now;
                else if (now - t0 > 1000000000ull) break;
            }
        }
        if (!good && f.status) atomicOr(f.status, 4);
        __threadfence();
        ok = good ? 1 : 0;
    }
    __syncthreads();
    return ok != 0;
}

// The last block to finish resets the barrier counters for the next launch
// (by then every block has left every wait).
__device__ __forceinline__ void coop_exit(const FftPlan& f) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(f.bar + 1, 1u) == gridDim.x - 1u) {
            atomicExch(f.bar, 0u);
            atomicExch(f.bar + 1, 0u);
            __threadfence();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kCoopWarps * 32, 1) k_fft3_convolve_coop(FftPlan f, RowPairs rp) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    const int n = f.n, log2n = f.log2n, h = f.h;
    const int P = fft_pencils(n), ns = fft_stride(n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C* buf = tw + n / 2 + warp * P * ns;
    load_twiddles(tw, static_cast<const C*>(f.tw), n);
    __syncthreads();
    // units go round-robin over the blocks first, so a pass with fewer units
    // than warps still spreads them over every SM
    const int64_t gw = int64_t(warp) * gridDim.x + blockIdx.x, nw = int64_t(gridDim.x) * kCoopWarps;
    const int64_t H = f.h + 1, K = 2 * f.h + 1;
    const int64_t xlo = f.lo[0], xcnt = f.hi[0] - f.lo[0] + 1;
    const int ylo = f.lo[1] & ~1, ycnt = (f.hi[1] | 1) - ylo + 1;
    C* A1 = static_cast<C*>(f.A1);
    C* A2 = static_cast<C*>(f.A2);
    // pass 1: real rows (z) -> half spectra, the spread grid zeroed behind
    for (int64_t u = gw; u * P < rp.npairs; u += nw)
        r2c_unit<T, SyncWarp>(static_cast<T*>(f.grid), A1, rp, n, log2n, h, tw, buf, u * P, lane, 32);
    // pass 2: y, keep -h..h
    if (coop_barrier(f, 1)) {
        for (int64_t u = gw; u * P < xcnt * H; u += nw)
            axis_unit<T, FULL, CENTERED, false, SyncWarp>(A1, A2, xlo, xcnt, H, 0, 0, n, log2n, h, tw, buf, u * P,
                                                         lane, 32);
        // pass 3: x, forward, multiply, inverse
        if (coop_barrier(f, 2)) {
            for (int64_t u = gw; u * P < K * H; u += nw)
                convolve_unit<T, SyncWarp>(A2, K * H, int(xlo), int(xcnt), n, log2n, h,
                                           static_cast<const T*>(f.mult), tw, buf, u * P, lane, 32);
            // pass 4: inverse y, the band's row pairs only
            if (coop_barrier(f, 3)) {
                for (int64_t u = gw; u * P < xcnt * H; u += nw)
                    axis_unit<T, CENTERED, FULL, true, SyncWarp>(A2, A1, xlo, xcnt, H, ylo, ycnt, n, log2n, h, tw,
                                                                buf, u * P, lane, 32);
                // pass 5: half spectra -> real rows of the interpolation grid
                if (coop_barrier(f, 4)) {
                    for (int64_t u = gw; u * P < rp.npairs; u += nw)
                        c2r_unit<T, SyncWarp>(A1, static_cast<T*>(f.grid_out), rp, n, log2n, h, tw, buf, u * P,
                                              lane, 32);
                }
            }
        }
    }
    coop_exit(f);
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
    return (size_t(n / 2) + size_t(fft_pencils(n)) * size_t(fft_stride(n))) * sizeof(typename Cplx<T>::type);
}

// Largest dynamic shared memory any FFT launch of this precision can use:
// one pencil of the largest length, 4096, and its twiddles.
template <typename T>
static size_t fft_smem_max() {
    return size_t(2048 + fft_stride(4096)) * sizeof(typename Cplx<T>::type);
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

template <typename T>
static cudaError_t run_r2c(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_r2c_rows<T>>()));
    const RowPairs rp = row_pairs(f);
    const int P = fft_pencils(f.n);
    k_fft_r2c_rows<T><<<unsigned((rp.npairs + P - 1) / P), fft_threads<T>(f.n), fft_smem_bytes<T>(f.n), s>>>(
        static_cast<T*>(f.grid), static_cast<C*>(f.A1), rp, f.n, f.log2n, f.h, static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t run_c2r(const FftPlan& f, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_c2r_rows<T>>()));
    const RowPairs rp = row_pairs(f);
    const int P = fft_pencils(f.n);
    k_fft_c2r_rows<T><<<unsigned((rp.npairs + P - 1) / P), fft_threads<T>(f.n), fft_smem_bytes<T>(f.n), s>>>(
        static_cast<const C*>(f.A1), static_cast<T*>(f.grid_out), rp, f.n, f.log2n, f.h,
        static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T, int INM, int OUTM, bool INV>
static cudaError_t run_axis(const FftPlan& f, const void* in, void* out, int64_t olo, int64_t ocnt, int64_t I,
                            int klo, int kcnt, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_axis<T, INM, OUTM, INV>>()));
    const int P = fft_pencils(f.n);
    const int64_t Q = ocnt * I;
    k_fft_axis<T, INM, OUTM, INV><<<unsigned((Q + P - 1) / P), fft_threads<T>(f.n), fft_smem_bytes<T>(f.n), s>>>(
        static_cast<const C*>(in), static_cast<C*>(out), olo, ocnt, I, klo, kcnt, f.n, f.log2n, f.h,
        static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
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

template <typename T>
static cudaError_t run_axis0_convolve(const FftPlan& f, void* data, int64_t I, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    SK_TRY((ensure_smem<T, k_fft_axis0_convolve<T>>()));
    const int P = fft_pencils(f.n);
    int xlo, xcnt;
    axis0_range(f, xlo, xcnt);
    k_fft_axis0_convolve<T><<<unsigned((I + P - 1) / P), fft_threads<T>(f.n), fft_smem_bytes<T>(f.n), s>>>(
        static_cast<C*>(data), I, xlo, xcnt, f.n, f.log2n, f.h, static_cast<const T*>(f.mult),
        static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

// Shared memory of the persistent kernel: the twiddles, then one unit's
// pencils per warp.
template <typename T>
static size_t coop_smem_bytes(int n) {
    return (size_t(n / 2) + size_t(kCoopWarps) * fft_pencils(n) * fft_stride(n)) * sizeof(typename Cplx<T>::type);
}

template <typename T>
int fft_coop_blocks(const FftPlan& f) {
    if constexpr (sizeof(T) != 4) {
        return 0;   // FP64 pencils take 64 threads per unit: the pass kernels
    }
    if (f.d != 3 || fft_threads<T>(f.n) != 32 || !f.bar) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    const size_t smem = coop_smem_bytes<T>(f.n);
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaFuncSetAttribute(k_fft3_convolve_coop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fft3_convolve_coop<T>, kCoopWarps * 32, smem)) {
        cudaGetLastError();
        return 0;
    }
    return per_sm >= 1 ? sms : 0;
}

template <typename T>
cudaError_t launch_fft_convolve(const FftPlan& f, cudaStream_t s, int64_t* launches) {
    using C = typename Cplx<T>::type;
    const int64_t n = f.n, H = f.h + 1, K = 2 * f.h + 1;
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
    if constexpr (sizeof(T) == 4) {
      if (f.coop_blocks > 0) {
        const RowPairs rp = row_pairs(f);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(unsigned(f.coop_blocks));
        cfg.blockDim = dim3(kCoopWarps * 32);
        cfg.dynamicSmemBytes = coop_smem_bytes<T>(f.n);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (launches) ++*launches;
        return cudaLaunchKernelEx(&cfg, k_fft3_convolve_coop<T>, f, rp);
      }
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

template int fft_coop_blocks<float>(const FftPlan&);
template int fft_coop_blocks<double>(const FftPlan&);
template cudaError_t launch_fft_convolve<float>(const FftPlan&, cudaStream_t, int64_t*);
template cudaError_t launch_fft_convolve<double>(const FftPlan&, cudaStream_t, int64_t*);
template cudaError_t launch_fft_adjoint<float>(const FftPlan&, double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_adjoint<double>(const FftPlan&, double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_forward<float>(const FftPlan&, const double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_forward<double>(const FftPlan&, const double*, cudaStream_t, int64_t*);

}  // namespace sk
