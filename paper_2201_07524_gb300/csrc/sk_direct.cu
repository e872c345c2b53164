// Plain direct summation t_i = sum_j w_j exp(-||x_i - y_j||^r / eps)
// (Eqs. (matexp), (matexpt)) on the GPU: the O(n m) baseline the fast
// summation is measured against.  Sources are staged through shared memory
// in tiles; each thread owns two targets.  In FP32 the kernel values and the
// per-tile partial sums are FP32 and the tiles are combined in FP64.
#include "sk_internal.cuh"

namespace sk {

constexpr int kDirectTile = 1024;
constexpr int kDirectPerThread = 2;

template <typename T, int RK>
__device__ __forceinline__ T kernel_value(T d2, T coef, T r);

// r = 2: exp(-coef d^2)
template <> __device__ __forceinline__ float kernel_value<float, 2>(float d2, float coef, float) {
    return exp2f(-coef * d2);
}
template <> __device__ __forceinline__ double kernel_value<double, 2>(double d2, double coef, double) {
    return exp(-coef * d2);
}
// r = 1: exp(-coef d)
template <> __device__ __forceinline__ float kernel_value<float, 1>(float d2, float coef, float) {
    return exp2f(-coef * sqrtf(d2));
}
template <> __device__ __forceinline__ double kernel_value<double, 1>(double d2, double coef, double) {
    return exp(-coef * sqrt(d2));
}
// general r: exp(-coef d^r)
template <> __device__ __forceinline__ float kernel_value<float, 0>(float d2, float coef, float r) {
    return exp2f(-coef * powf(d2, 0.5f * r));
}
template <> __device__ __forceinline__ double kernel_value<double, 0>(double d2, double coef, double r) {
    return exp(-coef * pow(d2, 0.5 * r));
}

template <int D, typename T, int RK>
__global__ void __launch_bounds__(256) k_direct(DirectArgs a, Epilogue e) {
    __shared__ T sc[D][kDirectTile];
    __shared__ T sw[kDirectTile];
    // FP32 evaluates exp2, so fold log2(e) into the coefficient.
    const T coef = sizeof(T) == 4 ? T(a.coef * 1.4426950408889634) : T(a.coef);
    const T r = T(a.r);
    const int64_t base = int64_t(blockIdx.x) * blockDim.x * kDirectPerThread + threadIdx.x;
    T xt[kDirectPerThread][D];
    double acc[kDirectPerThread];
#pragma unroll
    for (int q = 0; q < kDirectPerThread; ++q) {
        const int64_t i = base + int64_t(q) * blockDim.x;
        acc[q] = 0.0;
#pragma unroll
        for (int t = 0; t < D; ++t) xt[q][t] = i < a.nt ? static_cast<const T*>(a.tcoord[t])[i] : T(0);
    }
    for (int64_t j0 = 0; j0 < a.ns; j0 += kDirectTile) {
        const int cnt = int(a.ns - j0 < int64_t(kDirectTile) ? a.ns - j0 : int64_t(kDirectTile));
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
#pragma unroll
            for (int t = 0; t < D; ++t) sc[t][j] = static_cast<const T*>(a.scoord[t])[j0 + j];
            sw[j] = T(a.w[j0 + j]);
        }
        __syncthreads();
        T part[kDirectPerThread];
#pragma unroll
        for (int q = 0; q < kDirectPerThread; ++q) part[q] = T(0);
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
            const T wj = sw[j];
#pragma unroll
            for (int q = 0; q < kDirectPerThread; ++q) {
                T d2 = T(0);
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    const T dd = xt[q][t] - sc[t][j];
                    d2 += dd * dd;
                }
                part[q] += wj * kernel_value<T, RK>(d2, coef, r);
            }
        }
#pragma unroll
        for (int q = 0; q < kDirectPerThread; ++q) acc[q] += double(part[q]);
    }
    double sq = 0.0, bad = 0.0, dot = 0.0;
#pragma unroll
    for (int q = 0; q < kDirectPerThread; ++q) {
        const int64_t i = base + int64_t(q) * blockDim.x;
        if (i < a.nt) epi_point(e, i, acc[q], sq, bad, dot);
    }
    epi_finish(e, sq, bad, dot);
}

template <typename T>
int direct_blocks(int64_t nt) {
    const int64_t per = 256 * kDirectPerThread;
    return int((nt + per - 1) / per);
}

template <int D, typename T>
static cudaError_t direct_d(const DirectArgs& a, const Epilogue& e, cudaStream_t s) {
    const int blocks = direct_blocks<T>(a.nt);
    if (a.r == 2.0)
        k_direct<D, T, 2><<<blocks, 256, 0, s>>>(a, e);
    else if (a.r == 1.0)
        k_direct<D, T, 1><<<blocks, 256, 0, s>>>(a, e);
    else
        k_direct<D, T, 0><<<blocks, 256, 0, s>>>(a, e);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_direct(int d, const DirectArgs& a, const Epilogue& e, int64_t* launches, cudaStream_t s) {
    if (a.nt == 0) return cudaSuccess;
    if (launches) ++*launches;
    switch (d) {
        case 1: return direct_d<1, T>(a, e, s);
        case 2: return direct_d<2, T>(a, e, s);
        case 3: return direct_d<3, T>(a, e, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_direct<float>(int, const DirectArgs&, const Epilogue&, int64_t*, cudaStream_t);
template cudaError_t launch_direct<double>(int, const DirectArgs&, const Epilogue&, int64_t*, cudaStream_t);
template int direct_blocks<float>(int64_t);
template int direct_blocks<double>(int64_t);

}  // namespace sk
