// Spreading (adjoint NFFT, first step of the inner sum of Eq. (fastsum)) and
// interpolation (NFFT, last step of the outer sum) with the Kaiser-Bessel
// window, plus the fused FP64 scaling update of Eq. (S1).
//
// Spreading: points are bin-sorted by grid cell at plan time.  One thread
// block takes one subproblem (at most kSpreadMaxPts points of one bin),
// accumulates their (2m)^d window taps into a shared-memory copy of the bin's
// padded sub-grid with shared-memory atomics, and then adds the sub-grid into
// the global grid.  Every point lies in the central half of the torus, so no
// tap ever wraps around.
//
// Interpolation: one thread per target point (sorted order, so neighbouring
// threads read neighbouring grid cells), FP32/FP64 accumulation of the
// tensor-product window taps, then the FP64 epilogue.
#include "sk_internal.cuh"

namespace sk {

// Bin shapes in cells (last axis fastest).  In 3-D a bin is 4 x 4 x 8 so that
// its 16 xy-columns of 8 cells feed the column kernels (sk_spread3.cu); in 2-D
// a bin is a strip of 33 - W by 8 cells for the strip kernels (same file); the
// per-point kernels here serve 1-D plans and 3-D plans with W > 10.
template <int D> struct BinShape;
template <> struct BinShape<1> { static constexpr int B0 = 512, B1 = 1, B2 = 1; };
template <> struct BinShape<3> { static constexpr int B0 = 4, B1 = 4, B2 = 8; };

void bin_shape(int d, int W, int B[3]) {
    if (d == 1) { B[0] = BinShape<1>::B0; B[1] = 1; B[2] = 1; }
    else if (d == 2) { B[0] = strip_bx(W); B[1] = kStripBy; B[2] = 1; }
    else { B[0] = BinShape<3>::B0; B[1] = BinShape<3>::B1; B[2] = BinShape<3>::B2; }
}

template <int D, int W>
struct SubGrid {
    static constexpr int S0 = BinShape<D>::B0 + W - 1;
    static constexpr int S1 = D > 1 ? BinShape<D>::B1 + W - 1 : 1;
    static constexpr int S2 = D > 2 ? BinShape<D>::B2 + W - 1 : 1;
    static constexpr int CELLS = S0 * S1 * S2;
};

// Window weights of one coordinate for the W = 2m taps starting at cell f - (m-1).
template <int W, typename T>
__device__ __forceinline__ void tap_weights(T u, T beta, T knorm, int& f, T (&w)[W]) {
    const T m = T(W / 2);
    T fl = floor(u);
    f = int(fl);
    T frac = u - fl;
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = kb_window<T>(frac + T(W / 2 - 1 - k), m, beta, knorm);
}

template <int D, int W, typename T>
__global__ void __launch_bounds__(256) k_spread(SpreadArgs a) {
    using SG = SubGrid<D, W>;
    constexpr int NC = SG::CELLS;
    const int B[3] = {BinShape<D>::B0, BinShape<D>::B1, BinShape<D>::B2};
    const int S[3] = {SG::S0, SG::S1, SG::S2};
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sub = reinterpret_cast<T*>(smem_raw);

    const int s = blockIdx.x;
    const int bin = a.sub_bin[s];
    const int start = a.sub_start[s];
    const int cnt = a.sub_count[s];
    int bc[3] = {0, 0, 0};
    {
        int rem = bin;
        for (int t = D - 1; t >= 0; --t) { bc[t] = rem % a.nb[t]; rem /= a.nb[t]; }
    }
    for (int c = threadIdx.x; c < NC; c += blockDim.x) sub[c] = T(0);
    __syncthreads();

    const T beta = T(a.beta), knorm = T(a.knorm);
    const T* c0 = static_cast<const T*>(a.coord[0]);
    const T* c1 = static_cast<const T*>(a.coord[1]);
    const T* c2 = static_cast<const T*>(a.coord[2]);
    // Points of a bin are sorted by cell, so neighbouring points share taps.
    // Interleave: slot q (lane q % 32 of group q / 32) takes point
    // (q % 32) * G + q / 32, so the 32 lanes of a warp add into cells far apart
    // instead of serializing on the same shared-memory addresses.
    const int G = (cnt + 31) / 32;
    for (int q = threadIdx.x; q < 32 * G; q += blockDim.x) {
        const int qi = (q & 31) * G + (q >> 5);
        if (qi >= cnt) continue;
        const int p = start + qi;
        const T val = T(a.w[p]);
        T w0[W], w1[W], w2[W];
        int f0 = 0, f1 = 0, f2 = 0;
        tap_weights<W, T>(c0[p], beta, knorm, f0, w0);
        const int l0 = f0 - bc[0] * B[0];
        if (D == 1) {
#pragma unroll
            for (int i = 0; i < W; ++i) atomicAdd(&sub[l0 + i], val * w0[i]);
            continue;
        }
        tap_weights<W, T>(c1[p], beta, knorm, f1, w1);
        const int l1 = f1 - bc[1] * B[1];
        if (D == 2) {
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const T v0 = val * w0[i];
                T* row = sub + (l0 + i) * SG::S1 + l1;
#pragma unroll
                for (int j = 0; j < W; ++j) atomicAdd(row + j, v0 * w1[j]);
            }
            continue;
        }
        tap_weights<W, T>(c2[p], beta, knorm, f2, w2);
        const int l2 = f2 - bc[2] * B[2];
#pragma unroll 1
        for (int i = 0; i < W; ++i) {
            const T v0 = val * w0[i];
#pragma unroll 2
            for (int j = 0; j < W; ++j) {
                const T v1 = v0 * w1[j];
                T* row = sub + ((l0 + i) * SG::S1 + (l1 + j)) * SG::S2 + l2;
#pragma unroll
                for (int k = 0; k < W; ++k) atomicAdd(row + k, v1 * w2[k]);
            }
        }
    }
    __syncthreads();

    T* grid = static_cast<T*>(a.grid);
    const int n = a.n_os;
    int org[3];
    for (int t = 0; t < D; ++t) org[t] = bc[t] * B[t] - (W / 2 - 1);
    for (int c = threadIdx.x; c < NC; c += blockDim.x) {
        const T v = sub[c];
        if (v == T(0)) continue;
        int loc[3] = {0, 0, 0};
        int rem = c;
        for (int t = D - 1; t >= 0; --t) { loc[t] = rem % S[t]; rem /= S[t]; }
        int64_t gi = 0;
        bool ok = true;
        for (int t = 0; t < D; ++t) {
            const int g = org[t] + loc[t];
            ok = ok && (g >= 0) && (g < n);
            gi = gi * n + g;
        }
        if (ok) atomicAdd(&grid[gi], v);
    }
}

template <int D, int W, typename T>
__global__ void __launch_bounds__(256) k_interp(InterpArgs a, Epilogue e) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double sq = 0.0, bad = 0.0, dot = 0.0;
    if (i < a.n) {
        const T beta = T(a.beta), knorm = T(a.knorm);
        const T* grid = static_cast<const T*>(a.grid);
        const int64_t n = a.n_os;
        T w0[W], w1[W], w2[W];
        int f0 = 0, f1 = 0, f2 = 0;
        tap_weights<W, T>(static_cast<const T*>(a.coord[0])[i], beta, knorm, f0, w0);
        const int64_t g0 = f0 - (W / 2 - 1);
        T acc = T(0);
        if (D == 1) {
#pragma unroll
            for (int k = 0; k < W; ++k) acc += __ldg(grid + g0 + k) * w0[k];
        } else {
            tap_weights<W, T>(static_cast<const T*>(a.coord[1])[i], beta, knorm, f1, w1);
            const int64_t g1 = f1 - (W / 2 - 1);
            if (D == 2) {
#pragma unroll
                for (int r = 0; r < W; ++r) {
                    const T* row = grid + (g0 + r) * n + g1;
                    T s = T(0);
#pragma unroll
                    for (int k = 0; k < W; ++k) s += __ldg(row + k) * w1[k];
                    acc += s * w0[r];
                }
            } else {
                tap_weights<W, T>(static_cast<const T*>(a.coord[2])[i], beta, knorm, f2, w2);
                const int64_t g2 = f2 - (W / 2 - 1);
#pragma unroll 1
                for (int r = 0; r < W; ++r) {
                    T sr = T(0);
#pragma unroll 2
                    for (int q = 0; q < W; ++q) {
                        const T* row = grid + ((g0 + r) * n + (g1 + q)) * n + g2;
                        T s = T(0);
#pragma unroll
                        for (int k = 0; k < W; ++k) s += __ldg(row + k) * w2[k];
                        sr += s * w1[q];
                    }
                    acc += sr * w0[r];
                }
            }
        }
        epi_point(e, i, double(acc), sq, bad, dot);
    }
    epi_finish(e, sq, bad, dot);
}

// ------------------------------------------------------------------ dispatch

template <int D, int W, typename T>
static cudaError_t spread_one(const SpreadArgs& a, cudaStream_t s) {
    constexpr size_t bytes = size_t(SubGrid<D, W>::CELLS) * sizeof(T);
    static unsigned long long configured = 0ull;   // one bit per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(configured & (1ull << (dev & 63)))) {   // the 48 KB default also counts static shared memory
        cudaError_t err = cudaFuncSetAttribute(k_spread<D, W, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(bytes));
        if (err != cudaSuccess) return err;
        configured |= (1ull << (dev & 63));
    }
    if (a.nsub == 0) return cudaSuccess;
    k_spread<D, W, T><<<a.nsub, 256, bytes, s>>>(a);
    return cudaGetLastError();
}

template <int D, typename T>
static cudaError_t spread_w(int W, const SpreadArgs& a, cudaStream_t s) {
    switch (W) {
        case 4: return spread_one<D, 4, T>(a, s);
        case 6: return spread_one<D, 6, T>(a, s);
        case 8: return spread_one<D, 8, T>(a, s);
        case 10: return spread_one<D, 10, T>(a, s);
        case 12: return spread_one<D, 12, T>(a, s);
        case 14: return spread_one<D, 14, T>(a, s);
        case 16: return spread_one<D, 16, T>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_spread(int d, int W, const SpreadArgs& a, cudaStream_t s) {
    if (column_kernels(d, W)) return launch_spread3<T>(W, a, s);
    switch (d) {
        case 1: return spread_w<1, T>(W, a, s);
        case 2: return launch_spread2<T>(W, a, s);
        case 3: return spread_w<3, T>(W, a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
int interp_blocks(int64_t n) { return int((n + 255) / 256); }

template <int D, int W, typename T>
static cudaError_t interp_one(const InterpArgs& a, const Epilogue& e, int64_t* launches, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_interp<D, W, T><<<interp_blocks<T>(a.n), 256, 0, s>>>(a, e);
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <int D, typename T>
static cudaError_t interp_w(int W, const InterpArgs& a, const Epilogue& e, int64_t* l, cudaStream_t s) {
    switch (W) {
        case 4: return interp_one<D, 4, T>(a, e, l, s);
        case 6: return interp_one<D, 6, T>(a, e, l, s);
        case 8: return interp_one<D, 8, T>(a, e, l, s);
        case 10: return interp_one<D, 10, T>(a, e, l, s);
        case 12: return interp_one<D, 12, T>(a, e, l, s);
        case 14: return interp_one<D, 14, T>(a, e, l, s);
        case 16: return interp_one<D, 16, T>(a, e, l, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_interp(int d, int W, const InterpArgs& a, const Epilogue& e, int64_t* launches,
                          cudaStream_t s) {
    if (column_kernels(d, W)) {
        if (launches && a.ncols > 0) ++*launches;
        return launch_interp3<T>(W, a, e, s);
    }
    switch (d) {
        case 1: return interp_w<1, T>(W, a, e, launches, s);
        case 2:
            if (launches && a.nstasks > 0) ++*launches;
            return launch_interp2<T>(W, a, e, s);
        case 3: return interp_w<3, T>(W, a, e, launches, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_spread<float>(int, int, const SpreadArgs&, cudaStream_t);
template cudaError_t launch_spread<double>(int, int, const SpreadArgs&, cudaStream_t);
template cudaError_t launch_interp<float>(int, int, const InterpArgs&, const Epilogue&, int64_t*, cudaStream_t);
template cudaError_t launch_interp<double>(int, int, const InterpArgs&, const Epilogue&, int64_t*, cudaStream_t);
template int interp_blocks<float>(int64_t);
template int interp_blocks<double>(int64_t);

}  // namespace sk
