// FP32 issue-rate microbenchmark: the measured denominator of the roofline
// of the kernels that are bound by FP32 arithmetic (spreading, interpolation).
//
// Every thread runs kChains independent FMA chains a = a * b + c (scalar
// FFMA, or packed FFMA2 on float2 pairs), so the FMA pipes never wait on a
// chain's latency; the grid fills every SM to its resident-thread limit.
// Work = blocks * threads * iters * chains FMAs (twice that for the packed
// form), 2 flops each, over the kernel's CUDA-event time.
#include <cuda_runtime.h>

#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__device__ float g_peak_sink;

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(int iters, float b, float c) {
    float s = 0.f;
    if constexpr (PACKED) {
        float2 acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = make_float2(float(threadIdx.x) * 1e-3f + k, float(k) * 0.5f);
        const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll 4
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = __ffma2_rn(acc[k], bb, cc);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k].x + acc[k].y;
    } else {
        float acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = float(threadIdx.x) * 1e-3f + k;
#pragma unroll 4
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fmaf(acc[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k];
    }
    // never true for the values used; keeps the chains from being removed
    if (s == -1.2345e-30f) g_peak_sink = s;
}

struct Events {
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~Events() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace
}  // namespace sk

extern "C" int sk_fp32_peak(int packed, int iters, double* tflops, int* sms, void* stream) {
    using namespace sk;
    if (!tflops || iters < 1 || (packed != 0 && packed != 1)) return SK_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SK_ERR_CUDA;
    }
    const void* fn = packed ? reinterpret_cast<const void*>(&k_fma_chains<true>)
                            : reinterpret_cast<const void*>(&k_fma_chains<false>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPeakThreads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return SK_ERR_CUDA;
    }
    const unsigned blocks = unsigned(nsm * per_sm);
    const float b = 0.999999f, c = 1e-6f;
    Events t;
    if (cudaEventCreate(&t.ev[0]) != cudaSuccess || cudaEventCreate(&t.ev[1]) != cudaSuccess) {
        cudaGetLastError();
        return SK_ERR_CUDA;
    }
    // one untimed launch (clocks up, code loaded), then the timed one
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1 && cudaEventRecord(t.ev[0], s) != cudaSuccess) break;
        if (packed)
            k_fma_chains<true><<<blocks, kPeakThreads, 0, s>>>(iters, b, c);
        else
            k_fma_chains<false><<<blocks, kPeakThreads, 0, s>>>(iters, b, c);
        if (rep == 1) cudaEventRecord(t.ev[1], s);
    }
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(t.ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, t.ev[0], t.ev[1]) != cudaSuccess || !(ms > 0.f)) {
        cudaGetLastError();
        return SK_ERR_CUDA;
    }
    const double fmas = double(blocks) * kPeakThreads * double(iters) * kChains * (packed ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (double(ms) * 1e-3) / 1e12;
    if (sms) *sms = nsm;
    return SK_OK;
}
