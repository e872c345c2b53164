// Near-field correction for kernels that are not smooth at y = 0 (r not an
// even integer; Remark "Arithmetic complexity": r = 1 needs near-field
// regularization).  The fast summation uses the regularized kernel K_R, which
// equals the even polynomial K_I for rho < eps_I; adding
//     t_i += sum_{j : |x_i - y_j| < eps_I} v_j (K(rho_ij) - K_I(rho_ij))
// restores the exact kernel near 0.
//
// Both clouds carry a second cell list at plan time: cubic cells of side
// h >= eps_I / K (K = 2, or 4 when the cells at K = 2 would hold 256 points
// or more on average) over the unit torus, so every neighbour of a
// point lies within K cells of its own along each axis.  Of those (2K+1)^d
// cells only the ones whose closest approach to the target cell,
// h sqrt(sum_t max(|o_t| - 1, 0)^2) for offset o, is below eps_I can hold a
// pair; along the last axis (the fastest in the cell order) the kept cells
// of each row form one contiguous source range.  One block takes one
// non-empty target cell; the sources of those rows are staged through shared
// memory in tiles;
// its 512 work items cover the cell's targets, several copies per target when
// the cell holds few.  Partial sums are FP32 per tile and FP64 across tiles.
#include <type_traits>

#include "sk_internal.cuh"

namespace sk {

constexpr int kNearTile = 512;   // sources staged per tile
constexpr int kNearPerThread = 2;   // 512 work items per block pass
constexpr int kNearThreads = 256;

// Cell of each point in the near-field cell list (coordinates in grid units).
template <typename T>
__global__ void k_near_keys(const T* __restrict__ u0, const T* __restrict__ u1, const T* __restrict__ u2, int64_t n,
                            int d, double inv_cell, int nc, int* __restrict__ key, int* __restrict__ count) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T* u[3] = {u0, u1, u2};
    int k = 0;
    for (int t = 0; t < d; ++t) {
        int c = int(floor(double(u[t][i]) * inv_cell));
        c = c < 0 ? 0 : (c >= nc ? nc - 1 : c);
        k = k * nc + c;
    }
    key[i] = k;
    atomicAdd(&count[k], 1);
}

// Near-field order: idx[pos] = the point's index in the NFFT sort order, and
// its coordinates copied into near-field order.
template <typename T>
__global__ void k_near_scatter(const int* __restrict__ key, int64_t n, const int* __restrict__ start,
                               int* __restrict__ cursor, int* __restrict__ idx) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    idx[start[k] + atomicAdd(&cursor[k], 1)] = int(i);
}

template <typename T>
__global__ void k_near_gather(const int* __restrict__ idx, int64_t n, int d, const T* __restrict__ u0,
                              const T* __restrict__ u1, const T* __restrict__ u2, T* __restrict__ o0,
                              T* __restrict__ o1, T* __restrict__ o2) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = idx[i];
    o0[i] = u0[p];
    if (d > 1) o1[i] = u1[p];
    if (d > 2) o2[i] = u2[p];
}

// Non-empty cells of a count array.
__global__ void k_count_nonempty(const int* __restrict__ count, int ncells, int* __restrict__ nonempty) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncells && count[c] > 0) atomicAdd(nonempty, 1);
}

// Non-empty cells of the list (one block task each).
__global__ void k_near_tasks(const int* __restrict__ start, int ncells, int* __restrict__ tasks,
                             int* __restrict__ ntasks) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    if (start[c + 1] > start[c]) tasks[atomicAdd(ntasks, 1)] = c;
}

// FP32 plans take the hardware's approximate base-2 exponential and
// reciprocal square root (PTX ex2.approx / rsqrt.approx, relative error about
// 2^-22): a pair's term then carries an error of a few 1e-7 of K, below the
// FP32 fast summation's own.  FP64 plans use the full-precision functions.
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float exp2_pair(float x) { return ex2_fast(x); }
__device__ __forceinline__ double exp2_pair(double x) { return exp2(x); }
__device__ __forceinline__ float rsqrt_pair(float x) { return rsqrt_fast(x); }
__device__ __forceinline__ double rsqrt_pair(double x) { return rsqrt(x); }

// Per-pair correction v (K(rho) - K_I(rho)) for |du|^2 = d2 < r2max (else 0).
// Everything here is FP32 (or FP64 for FP64 plans); the parameters were
// converted once per thread.  For r = 1 the distance is d2 * rsqrt(d2).
template <typename T, bool R1, int NP>
__device__ __forceinline__ T pair_term(T d2, T w, T r2max, T inv_r2, T kc, T half_r, const T (&ki)[kMaxP]) {
    T rho_r;
    if (R1) {
        rho_r = d2 > T(0) ? d2 * rsqrt_pair(d2) : T(0);
    } else {
        rho_r = pow(d2, half_r);
    }
    const T kv = exp2_pair(-kc * rho_r);
    const T s = d2 * inv_r2;
    T kin = ki[NP - 1];
#pragma unroll
    for (int k = NP - 2; k >= 0; --k) kin = fma(kin, s, ki[k]);
    return d2 < r2max ? w * (kv - kin) : T(0);
}

// The same correction for a thread's two FP32 targets against one source,
// in packed FP32x2 arithmetic (one instruction for both pairs, the
// exponential and reciprocal square root per pair).
template <bool R1, int NP>
__device__ __forceinline__ float2 pair_terms2(float2 d2, float w, float r2max, float inv_r2, float kc, float half_r,
                                              const float (&ki)[kMaxP]) {
    float2 rho;
    if (R1) {
        rho.x = d2.x > 0.f ? rsqrt_fast(d2.x) : 0.f;
        rho.y = d2.y > 0.f ? rsqrt_fast(d2.y) : 0.f;
        rho = __fmul2_rn(rho, d2);
    } else {
        rho.x = powf(d2.x, half_r);
        rho.y = powf(d2.y, half_r);
    }
    const float2 arg = __fmul2_rn(rho, make_float2(-kc, -kc));
    const float2 kv = make_float2(ex2_fast(arg.x), ex2_fast(arg.y));
    const float2 s = __fmul2_rn(d2, make_float2(inv_r2, inv_r2));
    float2 kin = make_float2(ki[NP - 1], ki[NP - 1]);
#pragma unroll
    for (int k = NP - 2; k >= 0; --k) kin = __ffma2_rn(kin, s, make_float2(ki[k], ki[k]));
    float2 t = __fmul2_rn(__ffma2_rn(kin, make_float2(-1.f, -1.f), kv), make_float2(w, w));
    t.x = d2.x < r2max ? t.x : 0.f;
    t.y = d2.y < r2max ? t.y : 0.f;
    return t;
}

// NP: polynomial length of K_I (the plan's p; kMaxP covers every p with zero padding).
// A pass over a cell's targets has 512 work items (kNearThreads threads x
// kNearPerThread): `slots` target slots (the pass's targets rounded up to a
// power of two >= 32) times `copies` = 512 / slots copies, copy c taking the
// staged sources j = c, c + copies, ...; the copies' sums are combined in
// shared memory.  A sparse cell so keeps every lane busy with real pairs.
// Thread t holds slots t % per + q per (per = slots / kNearPerThread) of copy
// t / per.
template <int D, typename T, bool R1, int NP, int K>
__global__ void __launch_bounds__(kNearThreads) k_nearfield(NearArgs a) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double4>::type;
    constexpr int kItems = kNearThreads * kNearPerThread;
    __shared__ V src[kNearTile];   // (x, y, z, w) of the staged sources
    __shared__ double red[kItems];
    const int cell = a.tasks[blockIdx.x];
    int cc[3] = {0, 0, 0};
    {
        int rem = cell;
        for (int t = D - 1; t >= 0; --t) { cc[t] = rem % a.nc; rem /= a.nc; }
    }
    const int ts = a.t_start[cell], te = a.t_start[cell + 1];
    const T* tc[3] = {static_cast<const T*>(a.t_coord[0]), static_cast<const T*>(a.t_coord[1]),
                      static_cast<const T*>(a.t_coord[2])};
    const T* scd[3] = {static_cast<const T*>(a.s_coord[0]), static_cast<const T*>(a.s_coord[1]),
                       static_cast<const T*>(a.s_coord[2])};
    // parameters in the working precision, once
    const T r2max = T(a.r2max), inv_r2 = T(a.inv_r2), half_r = T(0.5 * a.r);
    const T kc = T(a.kcoef * 1.4426950408889634);    // exp(-x) = exp2(-x log2 e)
    T ki[kMaxP];
#pragma unroll
    for (int k = 0; k < kMaxP; ++k) ki[k] = k < a.p ? T(a.ki[k]) : T(0);
    // outer axes: 0 and 1 for D = 3, 0 for D = 2, none for D = 1
    const int r0 = D == 3 ? K : 0, r1 = D >= 2 ? K : 0;
    for (int tb = ts; tb < te; tb += kItems) {
        const int rem = min(kItems, te - tb);
        int slots = 32;
        while (slots < rem) slots <<= 1;
        const int copies = kItems / slots;
        // a thread's kNearPerThread slots share one copy, so each staged source
        // it reads serves all of them
        const int per = slots / kNearPerThread;          // threads per copy
        const int copy = threadIdx.x / per;
        T xt[kNearPerThread][3];
        int slot[kNearPerThread];
        double acc[kNearPerThread];
#pragma unroll
        for (int q = 0; q < kNearPerThread; ++q) {
            slot[q] = threadIdx.x % per + q * per;
            const int i = tb + slot[q];
            const bool ok = slot[q] < rem;
            acc[q] = 0.0;
#pragma unroll
            for (int t = 0; t < 3; ++t) xt[q][t] = (t < D && ok) ? tc[t][i] : (t < D ? T(1e18) : T(0));
        }
        for (int o0 = -r0; o0 <= r0; ++o0)
            for (int o1 = -r1; o1 <= r1; ++o1) {
                // the row of cells along the last axis at outer offsets (o0, o1)
                int m2 = 0, row = 0;
                bool inside = true;
                if (D == 3) {
                    const int c0 = cc[0] + o0, c1 = cc[1] + o1;
                    inside = c0 >= 0 && c0 < a.nc && c1 >= 0 && c1 < a.nc;
                    m2 = max(abs(o0) - 1, 0) * max(abs(o0) - 1, 0) + max(abs(o1) - 1, 0) * max(abs(o1) - 1, 0);
                    row = (c0 * a.nc + c1) * a.nc;
                } else if (D == 2) {
                    const int c0 = cc[0] + o1;
                    inside = c0 >= 0 && c0 < a.nc;
                    m2 = max(abs(o1) - 1, 0) * max(abs(o1) - 1, 0);
                    row = c0 * a.nc;
                }
                if (!inside || m2 >= K * K) continue;
                int mz = 0;   // largest gap (in cells) along the last axis with m2 + gap^2 < K^2
                while ((mz + 1) * (mz + 1) + m2 < K * K) ++mz;
                const int cl = cc[D - 1];
                const int zl = max(0, cl - 1 - mz), zh = min(a.nc - 1, cl + 1 + mz);
                const int ss = a.s_start[row + zl], se = a.s_start[row + zh + 1];
                for (int s0 = ss; s0 < se; s0 += kNearTile) {
                    const int cnt = min(kNearTile, se - s0);
                    __syncthreads();
                    for (int j = threadIdx.x; j < cnt; j += kNearThreads) {
                        V v;
                        v.x = scd[0][s0 + j];
                        v.y = D > 1 ? scd[1][s0 + j] : T(0);
                        v.z = D > 2 ? scd[2][s0 + j] : T(0);
                        v.w = T(a.w[a.s_idx[s0 + j]]);
                        src[j] = v;
                    }
                    __syncthreads();
                    T part[kNearPerThread];
#pragma unroll
                    for (int q = 0; q < kNearPerThread; ++q) part[q] = T(0);
                    if constexpr (std::is_same<T, float>::value && kNearPerThread % 2 == 0) {
                        constexpr int H = kNearPerThread / 2;
                        float2 X0[H], X1[H], X2[H], part2[H];
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            X0[h] = make_float2(xt[2 * h][0], xt[2 * h + 1][0]);
                            X1[h] = make_float2(xt[2 * h][1], xt[2 * h + 1][1]);
                            X2[h] = make_float2(xt[2 * h][2], xt[2 * h + 1][2]);
                            part2[h] = make_float2(0.f, 0.f);
                        }
#pragma unroll 2
                        for (int j = copy; j < cnt; j += copies) {
                            const V sv = src[j];
                            float2 d2[H];
                            bool near = false;
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                const float2 dx = __fadd2_rn(X0[h], make_float2(-sv.x, -sv.x));
                                const float2 dy = __fadd2_rn(X1[h], make_float2(-sv.y, -sv.y));
                                const float2 dz = __fadd2_rn(X2[h], make_float2(-sv.z, -sv.z));
                                d2[h] = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                                near = near || d2[h].x < r2max || d2[h].y < r2max;
                            }
                            if (!__any_sync(__activemask(), near)) continue;
#pragma unroll
                            for (int h = 0; h < H; ++h)
                                part2[h] = __fadd2_rn(part2[h],
                                                      pair_terms2<R1, NP>(d2[h], sv.w, r2max, inv_r2, kc, half_r, ki));
                        }
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            part[2 * h] = part2[h].x;
                            part[2 * h + 1] = part2[h].y;
                        }
                    } else {
#pragma unroll 2
                    for (int j = copy; j < cnt; j += copies) {
                        const V sv = src[j];
                        T d2[kNearPerThread];
                        bool near = false;
#pragma unroll
                        for (int q = 0; q < kNearPerThread; ++q) {
                            const T dx = xt[q][0] - sv.x, dy = xt[q][1] - sv.y, dz = xt[q][2] - sv.z;
                            d2[q] = fma(dx, dx, fma(dy, dy, dz * dz));
                            near = near || d2[q] < r2max;
                        }
                        // a source no lane of the warp is close to costs only its distances
                        if (!__any_sync(__activemask(), near)) continue;
#pragma unroll
                        for (int q = 0; q < kNearPerThread; ++q)
                            part[q] += pair_term<T, R1, NP>(d2[q], sv.w, r2max, inv_r2, kc, half_r, ki);
                    }
                    }
#pragma unroll
                    for (int q = 0; q < kNearPerThread; ++q) acc[q] += double(part[q]);
                }
            }
        // combine the copies of each target slot (deterministic order)
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kNearPerThread; ++q) red[copy * slots + slot[q]] = acc[q];
        __syncthreads();
        for (int sl = threadIdx.x; sl < rem; sl += kNearThreads) {
            double t = 0.0;
            for (int c = 0; c < copies; ++c) t += red[c * slots + sl];
            a.out[a.t_idx[tb + sl]] = t;
        }
    }
}

// ------------------------------------------------------------------ launchers
template <typename T>
void launch_near_keys(void* const u[3], int64_t n, int d, double inv_cell, int nc, int* key, int* count,
                      cudaStream_t s) {
    k_near_keys<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(static_cast<const T*>(u[0]), static_cast<const T*>(u[1]),
                                                             static_cast<const T*>(u[2]), n, d, inv_cell, nc, key,
                                                             count);
}

void launch_near_scatter(const int* key, int64_t n, const int* start, int* cursor, int* idx, cudaStream_t s) {
    k_near_scatter<float><<<unsigned((n + 255) / 256), 256, 0, s>>>(key, n, start, cursor, idx);
}

template <typename T>
void launch_near_gather(const int* idx, int64_t n, int d, void* const u[3], void* const o[3], cudaStream_t s) {
    k_near_gather<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(
        idx, n, d, static_cast<const T*>(u[0]), static_cast<const T*>(u[1]), static_cast<const T*>(u[2]),
        static_cast<T*>(o[0]), static_cast<T*>(o[1]), static_cast<T*>(o[2]));
}

void launch_count_nonempty(const int* count, int ncells, int* nonempty, cudaStream_t s) {
    k_count_nonempty<<<unsigned((ncells + 255) / 256), 256, 0, s>>>(count, ncells, nonempty);
}

void launch_near_tasks(const int* start, int ncells, int* tasks, int* ntasks, cudaStream_t s) {
    k_near_tasks<<<unsigned((ncells + 255) / 256), 256, 0, s>>>(start, ncells, tasks, ntasks);
}

template <typename T>
cudaError_t launch_nearfield(int d, const NearArgs& a, int ntasks, cudaStream_t s) {
    if (ntasks == 0) return cudaSuccess;
    const bool r1 = a.r == 1.0;
    const bool p8 = a.p == 8;
#define SK_NF(DD, R, NP)                                                              \
    if (a.sub == 4)                                                                   \
        k_nearfield<DD, T, R, NP, 4><<<ntasks, kNearThreads, 0, s>>>(a);              \
    else                                                                              \
        k_nearfield<DD, T, R, NP, 2><<<ntasks, kNearThreads, 0, s>>>(a)
#define SK_NF_D(DD)                                  \
    if (r1 && p8) SK_NF(DD, true, 8);                 \
    else if (r1) SK_NF(DD, true, kMaxP);              \
    else if (p8) SK_NF(DD, false, 8);                 \
    else SK_NF(DD, false, kMaxP);
    switch (d) {
        case 1: SK_NF_D(1); break;
        case 2: SK_NF_D(2); break;
        default: SK_NF_D(3); break;
    }
#undef SK_NF_D
#undef SK_NF
    return cudaGetLastError();
}

template void launch_near_keys<float>(void* const[3], int64_t, int, double, int, int*, int*, cudaStream_t);
template void launch_near_keys<double>(void* const[3], int64_t, int, double, int, int*, int*, cudaStream_t);
template void launch_near_gather<float>(const int*, int64_t, int, void* const[3], void* const[3], cudaStream_t);
template void launch_near_gather<double>(const int*, int64_t, int, void* const[3], void* const[3], cudaStream_t);
template cudaError_t launch_nearfield<float>(int, const NearArgs&, int, cudaStream_t);
template cudaError_t launch_nearfield<double>(int, const NearArgs&, int, cudaStream_t);

}  // namespace sk
