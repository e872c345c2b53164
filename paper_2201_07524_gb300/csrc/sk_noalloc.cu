// A kernel product that allocates no device memory.
//
// Every other entry point works on a plan, and building a plan calls
// cudaMalloc.  Some callers cannot do that: code that runs inside a framework
// whose memory pool already owns the device memory (a second allocator would
// fail or fragment it), services that must not allocate after start-up because
// an allocation may synchronize the device, and code that hands the library
// only the buffers it owns.  sk_direct_residual_noalloc serves them: it
// evaluates t = K v by direct sums (the variant of the direct-summation kernel
// with the fused FP64 residual reduction) and keeps its reduction scratch in a
// fixed file-scope device array instead of plan memory.
//
// Limits and sharing: the array holds the partial sums of at most
// kNoAllocMaxBlocks blocks of kNoAllocTargetsPerBlock targets, so n is at most
// 2,097,152; larger n is rejected.  The array exists once per GPU that loads
// the library and lives until the process exits.  Every call shares it, so
// calls whose kernels overlap on the GPU (different streams, or different host
// threads on one device) race and give wrong sums; serialize them.
#include <cstdint>
#include <mutex>

#include "sk_internal.cuh"

namespace sk {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPerThread = 2;
constexpr int kNoAllocTargetsPerBlock = kNoAllocThreads * kNoAllocPerThread;
constexpr int kNoAllocMaxBlocks = 4096;
constexpr int kNoAllocTile = 1024;
constexpr int kNoAllocTicketDoubles = 32;   // 256 bytes in front of the partials hold the ticket

// [ticket (256 B)][per-block partials: 2 doubles per block]
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocTicketDoubles + 2 * kNoAllocMaxBlocks];

template <int D, int RK>
__global__ void __launch_bounds__(kNoAllocThreads)
k_direct_residual_noalloc(const double* __restrict__ x, const double* __restrict__ u, const double* __restrict__ a,
                          int64_t n, const double* __restrict__ y, const double* __restrict__ v, int64_t m,
                          float coef, float r, double* __restrict__ t_out, double* __restrict__ stats,
                          double* __restrict__ scratch) {
    __shared__ double sy[D][kNoAllocTile];
    __shared__ float sv[kNoAllocTile];
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
    double* partial = scratch + kNoAllocTicketDoubles;

    const int64_t base = int64_t(blockIdx.x) * kNoAllocTargetsPerBlock + threadIdx.x;
    double xt[kNoAllocPerThread][D];
    double acc[kNoAllocPerThread];
#pragma unroll
    for (int q = 0; q < kNoAllocPerThread; ++q) {
        const int64_t i = base + int64_t(q) * kNoAllocThreads;
        acc[q] = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) xt[q][c] = i < n ? x[i * D + c] : 0.0;
    }
    for (int64_t j0 = 0; j0 < m; j0 += kNoAllocTile) {
        const int cnt = int(m - j0 < int64_t(kNoAllocTile) ? m - j0 : int64_t(kNoAllocTile));
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += kNoAllocThreads) {
#pragma unroll
            for (int c = 0; c < D; ++c) sy[c][j] = y[(j0 + j) * D + c];
            sv[j] = float(v[j0 + j]);
        }
        __syncthreads();
        float part[kNoAllocPerThread];
#pragma unroll
        for (int q = 0; q < kNoAllocPerThread; ++q) part[q] = 0.f;
        for (int j = 0; j < cnt; ++j) {
#pragma unroll
            for (int q = 0; q < kNoAllocPerThread; ++q) {
                double d2 = 0.0;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const double dd = xt[q][c] - sy[c][j];
                    d2 += dd * dd;
                }
                const float f2 = float(d2);
                float e;
                if (RK == 2)
                    e = exp2f(-coef * f2);
                else if (RK == 1)
                    e = exp2f(-coef * sqrtf(f2));
                else
                    e = exp2f(-coef * powf(f2, 0.5f * r));
                part[q] += sv[j] * e;
            }
        }
#pragma unroll
        for (int q = 0; q < kNoAllocPerThread; ++q) acc[q] += double(part[q]);
    }
    double sq = 0.0, dot = 0.0;
#pragma unroll
    for (int q = 0; q < kNoAllocPerThread; ++q) {
        const int64_t i = base + int64_t(q) * kNoAllocThreads;
        if (i < n) {
            t_out[i] = acc[q];
            const double ut = u[i] * acc[q];
            const double res = ut - a[i];
            sq += res * res;
            dot += ut;
        }
    }
    // block sums, then the last block to finish adds the partials in block order
    __shared__ double red[2][kNoAllocThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sq = warp_sum(sq);
    dot = warp_sum(dot);
    if (lane == 0) { red[0][wid] = sq; red[1][wid] = dot; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < kNoAllocThreads / 32; ++w) { s0 += red[0][w]; s1 += red[1][w]; }
        partial[2 * blockIdx.x] = s0;
        partial[2 * blockIdx.x + 1] = s1;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            s0 += ((volatile double*)partial)[2 * b];
            s1 += ((volatile double*)partial)[2 * b + 1];
        }
        stats[0] = s0;
        stats[1] = s1;
        *ticket = 0u;
    }
}

// True when p is memory the kernel may read on the current device: device
// memory of that device, or managed memory.  Device memory of another GPU is
// refused: without peer access a kernel that reads it faults.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// True when the byte ranges [p, p + pn) and [q, q + qn) share a byte.
bool overlaps(const void* p, size_t pn, const void* q, size_t qn) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(q);
    return a < b + qn && b < a + pn;
}

// Device address of g_noalloc_scratch on device `dev` (the current device),
// looked up once per device: the first call on a device does this set-up, so
// that call has to come before any stream capture.  The address is kept for
// the life of the process; a device reset (cudaDeviceReset, or a reset of the
// primary context) after that first call is not supported, because the
// library's module, and the array with it, may then sit at another address.
cudaError_t scratch_address(int dev, double** out) {
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = static_cast<double*>(p);
    }
    *out = addr[dev];
    return cudaSuccess;
}

// The status codes carry the reason; msg documents it at the call site.
int fail(int code, const char* /*msg*/) { return code; }

template <int D>
cudaError_t launch(int rk, const double* x, const double* u, const double* a, int64_t n, const double* y,
                   const double* v, int64_t m, float coef, float r, double* t_out, double* stats, double* scratch,
                   unsigned blocks, cudaStream_t s) {
    if (rk == 2)
        k_direct_residual_noalloc<D, 2><<<blocks, kNoAllocThreads, 0, s>>>(x, u, a, n, y, v, m, coef, r, t_out, stats,
                                                                         scratch);
    else if (rk == 1)
        k_direct_residual_noalloc<D, 1><<<blocks, kNoAllocThreads, 0, s>>>(x, u, a, n, y, v, m, coef, r, t_out, stats,
                                                                         scratch);
    else
        k_direct_residual_noalloc<D, 0><<<blocks, kNoAllocThreads, 0, s>>>(x, u, a, n, y, v, m, coef, r, t_out, stats,
                                                                         scratch);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sk

extern "C" int sk_direct_residual_noalloc(int d, int64_t n, const double* x, const double* u, const double* a,
                                          int64_t m, const double* y, const double* v, double eps, double r,
                                          double* t_out, double* stats_out, void* stream) {
    using namespace sk;
    if (d < 1 || d > 3 || n < 1 || m < 1) return fail(SK_ERR_ARG, "d must be 1..3 and n, m >= 1");
    if (!(eps > 0.0) || !std::isfinite(eps) || !(r >= 1.0) || !std::isfinite(r))
        return fail(SK_ERR_ARG, "eps must be > 0 and r >= 1");
    if (n > int64_t(kNoAllocMaxBlocks) * kNoAllocTargetsPerBlock)
        return fail(SK_ERR_TOO_LARGE, "n exceeds the fixed scratch of sk_direct_residual_noalloc (n <= 2097152)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SK_ERR_CUDA, cudaGetErrorString(e));
    }
    const void* ptrs[7] = {x, u, a, y, v, t_out, stats_out};
    for (const void* p : ptrs)
        if (!p || !on_device(p, dev))
            return fail(SK_ERR_ARG, "all arrays must be device memory of the current device (or managed)");
    // outputs may not share memory with any input or with each other: other
    // blocks still read the inputs while t_out is written
    const size_t nb = size_t(n) * sizeof(double), mb = size_t(m) * sizeof(double);
    const void* in_p[5] = {x, u, a, y, v};
    const size_t in_n[5] = {nb * size_t(d), nb, nb, mb * size_t(d), mb};
    for (int k = 0; k < 5; ++k)
        if (overlaps(t_out, nb, in_p[k], in_n[k]) || overlaps(stats_out, 2 * sizeof(double), in_p[k], in_n[k]))
            return fail(SK_ERR_ARG, "t_out and stats_out must not overlap an input");
    if (overlaps(t_out, nb, stats_out, 2 * sizeof(double)))
        return fail(SK_ERR_ARG, "t_out and stats_out must not overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SK_ERR_CUDA, cudaGetErrorString(e));
    }
    // the ticket must start at zero; an earlier call leaves it at zero, but a
    // call that was cut short may not have
    e = cudaMemsetAsync(scratch, 0, kNoAllocTicketDoubles * sizeof(double), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SK_ERR_CUDA, cudaGetErrorString(e));
    }
    const int rk = r == 2.0 ? 2 : (r == 1.0 ? 1 : 0);
    const float coef = float(1.4426950408889634 / eps);   // exp(-z/eps) = exp2(-z log2(e) / eps)
    const unsigned blocks = unsigned((n + kNoAllocTargetsPerBlock - 1) / kNoAllocTargetsPerBlock);
    switch (d) {
        case 1: e = launch<1>(rk, x, u, a, n, y, v, m, coef, float(r), t_out, stats_out, scratch, blocks, s); break;
        case 2: e = launch<2>(rk, x, u, a, n, y, v, m, coef, float(r), t_out, stats_out, scratch, blocks, s); break;
        default: e = launch<3>(rk, x, u, a, n, y, v, m, coef, float(r), t_out, stats_out, scratch, blocks, s); break;
    }
    if (e != cudaSuccess) return fail(SK_ERR_CUDA, cudaGetErrorString(e));
    return SK_OK;
}
