// Tensor-core (tcgen05) interpolation for FP32 plans, 3-D and (further down)
// 2-D: the NFFT step of Eq. (fastsum) that evaluates the grid at the target
// points.
//
// Points are sorted by bin (4 x 4 x 8 cells).  Every window of a point of a
// bin lies in the bin's box of X x Y x Z grid cells (X = Y = 3 + W,
// Z = 7 + W), and the interpolated value of a point p is
//
//     t_p = sum_i wx_p[i] sum_j wy_p[j] H[p, (i, j)],
//     H[p, (i, j)] = sum_k wz_p[k] g[i, j, k],
//
// with the point's window weights placed at its offsets in the box (zero
// elsewhere).  For the 128 points of a tile and all X*Y rows (i, j) of the
// box, H is one product of a 128 x KZ matrix (each point's z-weights) with
// the transpose of an X*Y x KZ matrix (the box, z contiguous as in the grid):
// a dense contraction for the tensor core.  One thread issues it
// (tcgen05.mma kind::tf32, M = 128, N = X*Y rounded up to 16, K = KZ), the
// accumulator lands in tensor memory with one lane per point, and each thread
// reads its point's lane (tcgen05.ld) and finishes the two outer sums with its
// own x- and y-weights in FP32, then runs the FP64 epilogue (Eq. (S1) update,
// residual terms).
//
// Precision: kind::tf32 reads 10 mantissa bits of each operand, so each
// operand is split into hi (its TF32 part) and lo (the FP32 remainder) and H
// is accumulated from hi*hi + hi*lo + lo*hi.  The dropped lo*lo term is below
// 2^-20 of each product, so H carries FP32 accuracy.
//
// Operands sit in shared memory in the K-major layout without swizzling:
// core matrices of 8 rows x 16 bytes (4 values of K), LBO = 128 bytes between
// core matrices along K, SBO = KZ/4 * 128 bytes between groups of 8 rows.
// Work: tasks are runs of up to kTcRunPts points of one bin (most points
// first) taken from a global queue by persistent blocks of 128 threads (one
// point per thread and tile); a block loads its task's box once and runs one
// MMA group per tile of 128 points.  Tensor memory is shared by the blocks of
// an SM, so the launch pads its shared memory to keep at most 512 / columns
// blocks on an SM.  Every wait on the MMA's completion is bounded: a wait that
// gives up (on any lane of a warp) sets bit 2 of the epilogue's status word,
// the warp skips that tile's tensor-memory loads, and the block stops after
// the tile.  Before releasing its tensor memory the block waits once more
// (bounded) for the MMA group; if that wait gives up too, the columns are
// released all the same, because a kernel may not exit holding tensor memory:
// an MMA that is still running could then write into columns another block
// allocates next, and the solve that reported the timeout is not meaningful.
#include <algorithm>
#include <cstdint>

#include "sk_internal.cuh"
#include "sk_device.cuh"

namespace sk {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte
// units (bits 0-13, 16-29, 32-45), descriptor version 1 (bits 46-47), base
// offset 0, no swizzling (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t(lbo >> 4) << 16) | (uint64_t(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A
// and B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// The mbarrier arrives once every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the completion of the barrier's phase with parity `phase`, giving
// up after about a second (the global timer) or 2^24 tries, whichever comes
// first; an MMA group completes in microseconds.
constexpr unsigned long long kTcWaitNs = 1000000000ull;
constexpr int kTcWaitTries = 1 << 24;
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    const uint32_t addr = smem_addr(bar);
    unsigned long long t0 = 0;
    for (int it = 0; it < kTcWaitTries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(addr), "r"(phase)
            : "memory");
        if (done) return true;
        if ((it & 255) == 0) {
            const unsigned long long now = global_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > kTcWaitNs) return false;
        }
    }
    return false;
}

// 32 consecutive columns of this warp's 32 lanes: v[c] = column col0 + c of
// the thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

// TF32 part of v (the 10 mantissa bits the tensor core reads) and the rest.
__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); }

// ------------------------------------------------------------ shapes
template <int W>
struct Tc3 {
    static constexpr int M_W = W / 2;
    static constexpr int X = 3 + W, Y = 3 + W;           // box rows along x and y (bin 4 cells + W - 1)
    static constexpr int NR = X * Y;                     // rows (i, j) of the box
    static constexpr int N = (NR + 15) / 16 * 16;        // MMA N (multiple of 16 for M = 128)
    static constexpr int NCH = (N + 31) / 32;            // 32-column tensor-memory loads
    static constexpr int ZLEAD = 4;                      // the box starts at z0 - 4 (16-byte aligned)
    static constexpr int KZ = (12 + M_W + 7) / 8 * 8;    // z entries z0-4 .. z0+7+m, in whole MMA K steps of 8
    static constexpr int KC = KZ / 4;                    // 16-byte chunks per operand row
    static constexpr int LBO = 128, SBO = KC * 128;
    static constexpr int A_BYTES = 16 * SBO;             // 128 rows (points)
    static constexpr int B_BYTES = (N / 8) * SBO;        // N rows (box rows)
    static constexpr int OPERANDS = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int COLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));   // tensor-memory columns
    static constexpr int BLOCKS_PER_SM = (512 / COLS) > 8 ? 8 : 512 / COLS;
    static_assert(M_W >= 2 && M_W <= 5, "box shapes for m = 2..5");
    static_assert(NCH * 32 >= N && N <= 256, "N");
};

// ------------------------------------------------------------ interpolation
template <int W>
__global__ void __launch_bounds__(128) k_interp3_tc(InterpArgs a, Epilogue e) {
    using S = Tc3<W>;
    constexpr int m = S::M_W;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* a_hi = smem_raw;
    unsigned char* a_lo = a_hi + S::A_BYTES;
    unsigned char* b_hi = a_lo + S::A_BYTES;
    unsigned char* b_lo = b_hi + S::B_BYTES;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int task, abort_flag;
    __shared__ unsigned warps_done;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // box rows NR..N-1 stay zero for the whole launch
    for (int q = tid; q < 2 * S::B_BYTES / 16; q += 128) reinterpret_cast<float4*>(b_hi)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (warp == 0) tc_alloc(&tmem_slot, S::COLS);
    if (tid == 0) {
        mbar_init(&bar, 1);
        warps_done = 0u;
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = tmem + (uint32_t(warp * 32) << 16);
    constexpr uint32_t idesc = tc_idesc_tf32(128, S::N);
    const float* c0 = static_cast<const float*>(a.coord[0]);
    const float* c1 = static_cast<const float*>(a.coord[1]);
    const float* c2 = static_cast<const float*>(a.coord[2]);
    const float* grid = static_cast<const float*>(a.grid);
    const int n = a.n_os;
    uint32_t phase = 0;
    bool failed = false;
    double sq = 0.0, bad = 0.0, dot = 0.0;
    for (;;) {
        if (tid == 0) task = int(atomicAdd(a.queue, 1u));
        __syncthreads();
        const int t = task;
        if (t >= a.nttasks || abort_flag) break;
        const int bin = a.ttasks[3 * t], start = a.ttasks[3 * t + 1], end = a.ttasks[3 * t + 2];
        const int bz = bin % a.nb[2], by = (bin / a.nb[2]) % a.nb[1], bx = bin / (a.nb[2] * a.nb[1]);
        const int x0 = bx * 4, y0 = by * 4, z0 = bz * 8;
        // the box: rows (x0 - (m-1) + i, y0 - (m-1) + j), z from z0 - 4; zero
        // outside the grid.  All of a thread's loads are issued before its stores.
        {
            constexpr int LOADS = (S::NR * S::KC + 127) / 128;
            float4 v[LOADS];
#pragma unroll
            for (int l = 0; l < LOADS; ++l) {
                const int q = tid + 128 * l;
                const int r = q / S::KC, c = q - r * S::KC;
                const int i = r / S::Y, j = r - i * S::Y;
                const int xr = x0 - (m - 1) + i, yr = y0 - (m - 1) + j, zc = z0 - S::ZLEAD + 4 * c;
                v[l] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < S::NR * S::KC && xr >= 0 && xr < n && yr >= 0 && yr < n && zc >= 0 && zc + 4 <= n)
                    v[l] = __ldg(reinterpret_cast<const float4*>(grid + (int64_t(xr) * n + yr) * n + zc));
            }
#pragma unroll
            for (int l = 0; l < LOADS; ++l) {
                const int q = tid + 128 * l;
                if (q >= S::NR * S::KC) continue;
                const int r = q / S::KC, c = q - r * S::KC;
                const float4 h = make_float4(tf32_hi(v[l].x), tf32_hi(v[l].y), tf32_hi(v[l].z), tf32_hi(v[l].w));
                const int off = (r >> 3) * S::SBO + c * S::LBO + (r & 7) * 16;
                *reinterpret_cast<float4*>(b_hi + off) = h;
                *reinterpret_cast<float4*>(b_lo + off) =
                    make_float4(v[l].x - h.x, v[l].y - h.y, v[l].z - h.z, v[l].w - h.w);
            }
        }
        unsigned char* row_hi = a_hi + (tid >> 3) * S::SBO + (tid & 7) * 16;
        unsigned char* row_lo = a_lo + (tid >> 3) * S::SBO + (tid & 7) * 16;
        for (int base = start; base < end; base += 128) {
            const int p = base + tid;
            const bool ok = p < end;
            // only the z-weights feed the MMA; the x- and y-weights are evaluated
            // while it runs
            float wz[W];
            int k0 = 0;
            EpiPrefetch ep;
            ep.load(e, p, ok);
            const float ux = ok ? c0[p] : 0.f, uy = ok ? c1[p] : 0.f;
            if (ok) {
                int fz;
                window_poly<W, float>(c2[p], a.wp, 1.f, fz, wz);
                k0 = min(max(fz - z0 + S::ZLEAD - (m - 1), 0), S::KZ - W);
            } else {
#pragma unroll
                for (int k = 0; k < W; ++k) wz[k] = 0.f;
            }
            // the point's operand row, its W z-weights from entry k0, as whole
            // 16-byte chunks: the weights shifted by k0 mod 4 (selects) fill
            // NU chunks from chunk k0 / 4, the other chunks are zero.  Chunk
            // stores keep the warp's lanes on distinct banks, where single
            // values stored at a per-thread offset collide.
            {
                constexpr int NU = (W + 3 + 3) / 4;
                const int sh = k0 & 3, c0 = k0 >> 2;
                float u[4 * NU];
#pragma unroll
                for (int j = 0; j < 4 * NU; ++j) {
                    float v = 0.f;
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (j - t >= 0 && j - t < W) v = sh == t ? wz[j - t >= 0 && j - t < W ? j - t : 0] : v;
                    u[j] = v;
                }
#pragma unroll
                for (int r = 0; r < NU; ++r) {
                    if (c0 + r < S::KC) {
                        const float4 h = make_float4(tf32_hi(u[4 * r]), tf32_hi(u[4 * r + 1]), tf32_hi(u[4 * r + 2]),
                                                     tf32_hi(u[4 * r + 3]));
                        *reinterpret_cast<float4*>(row_hi + (c0 + r) * S::LBO) = h;
                        *reinterpret_cast<float4*>(row_lo + (c0 + r) * S::LBO) =
                            make_float4(u[4 * r] - h.x, u[4 * r + 1] - h.y, u[4 * r + 2] - h.z, u[4 * r + 3] - h.w);
                    }
                }
#pragma unroll
                for (int c = 0; c < S::KC; ++c) {
                    if (c < c0 || c >= c0 + NU) {
                        *reinterpret_cast<float4*>(row_hi + c * S::LBO) = make_float4(0.f, 0.f, 0.f, 0.f);
                        *reinterpret_cast<float4*>(row_lo + c * S::LBO) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (abort_flag) break;
            if (tid == 0 && !a.inject) {
                tc_fence_after();
                const uint32_t ah = smem_addr(a_hi), al = smem_addr(a_lo), bh = smem_addr(b_hi), bl = smem_addr(b_lo);
#pragma unroll
                for (int s = 0; s < S::KZ / 8; ++s) {
                    const uint32_t o = uint32_t(s * 2 * S::LBO);
                    tc_mma_tf32(tmem, tc_desc(ah + o, S::LBO, S::SBO), tc_desc(bh + o, S::LBO, S::SBO), idesc, s > 0);
                    tc_mma_tf32(tmem, tc_desc(ah + o, S::LBO, S::SBO), tc_desc(bl + o, S::LBO, S::SBO), idesc, 1u);
                    tc_mma_tf32(tmem, tc_desc(al + o, S::LBO, S::SBO), tc_desc(bh + o, S::LBO, S::SBO), idesc, 1u);
                }
                tc_commit(&bar);
            }
            float wx[W], wy[W];
            int dx = 0, dy = 0;
            if (ok) {
                int fx, fy;
                window_poly<W, float>(ux, a.wp, 1.f, fx, wx);
                window_poly<W, float>(uy, a.wp, 1.f, fy, wy);
                dx = min(max(fx - x0, 0), 3);
                dy = min(max(fy - y0, 0), 3);
            } else {
#pragma unroll
                for (int k = 0; k < W; ++k) wx[k] = wy[k] = 0.f;
            }
            // padded weights over the box rows (zero outside the point's window)
            float wxf[S::X], wyf[S::Y];
#pragma unroll
            for (int i = 0; i < S::X; ++i) {
                float vx = 0.f, vy = 0.f;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int q = i - s;
                    if (q >= 0 && q < W) {
                        vx = dx == s ? wx[q] : vx;
                        vy = dy == s ? wy[q] : vy;
                    }
                }
                wxf[i] = vx;
                wyf[i] = vy;
            }
            // warp-uniform: a warp whose wait gave up on any lane skips the
            // (warp-collective) tensor-memory loads of this tile
            const bool done = __all_sync(0xffffffffu, mbar_wait(&bar, phase));
            phase ^= 1u;
            if (!done) {
                failed = true;
                abort_flag = 1;
                if (e.status) atomicOr(e.status, 4);
            }
            tc_fence_after();
            float rs[S::X];
#pragma unroll
            for (int i = 0; i < S::X; ++i) rs[i] = 0.f;
#pragma unroll
            for (int ch = 0; ch < S::NCH; ++ch) {
                if (failed) break;
                float h[32];
                tmem_ld32(tlane + uint32_t(ch * 32), h);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int nn = ch * 32 + jj;
                    if (nn < S::NR) rs[nn / S::Y] = fmaf(wyf[nn % S::Y], h[jj], rs[nn / S::Y]);
                }
            }
            float tv = 0.f;
#pragma unroll
            for (int i = 0; i < S::X; ++i) tv = fmaf(wxf[i], rs[i], tv);
            if (ok && !failed) epi_point_pre32(e, p, tv, ep.q, ep.a, sq, bad, dot);
            tc_fence_before();
        }
    }
    // a block that gave up waits once more (bounded) for its last MMA group
    // before releasing the tensor memory
    if (failed) mbar_wait(&bar, phase ^ 1u);
    queue_leave(a.queue, lane);
    epi_finish_warps(e, sq, bad, dot, &warps_done);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, S::COLS);
}


// ------------------------------------------------------------ 2-D interpolation
// The same contraction for 2-D plans.  A bin is a strip of 33 - W x-cells by
// 8 y-cells, so its box is exactly 32 x-rows by 24 y-entries (from y0 - 8,
// 16-byte aligned, to y0 + 15, past the last tap y0 + 7 + m for m <= 8):
// H = Wy Gᵀ is one 128 x 32 x 24 product per tile (N = 32 box rows, 32
// tensor-memory columns).  The point's x-offset in the strip spans 33 - W
// values, too many for register selects, so each thread parks its 32 H
// values in its own row of the A operand (free once the MMA has completed)
// and reads back the W of its window.
template <int W>
struct Tc2 {
    static constexpr int M_W = W / 2;
    static constexpr int BX = 33 - W;            // x-cells of a strip bin
    static constexpr int N = 32;                 // box x-rows
    static constexpr int YLEAD = 8;              // the box starts at y0 - 8
    static constexpr int KY = 24;                // y entries
    static constexpr int KC = KY / 4;
    static constexpr int LBO = 128, SBO = KC * 128;
    static constexpr int A_BYTES = 16 * SBO;
    static constexpr int B_BYTES = (N / 8) * SBO;
    static constexpr int OPERANDS = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int COLS = 32;
    static constexpr int BLOCKS_PER_SM = 8;
    static_assert(M_W >= 2 && M_W <= 8, "window widths 4..16");
    static_assert(2 * KC >= N / 4, "a thread's operand row holds its N results");
};

// A point's A-operand row in the 2-D kernel: its W y-weights from entry K0,
// zeros elsewhere, as whole 16-byte chunks (hi and lo parts).  The offset K0
// is a compile-time constant here: the points of a warp share their y-cell
// almost always (a bin's points are sorted y-cell first), so the dispatch
// below costs one branch per warp, and the chunk stores put the warp's lanes
// on distinct banks, where stores of single values at a per-thread offset
// collide.
template <int W, int KC, int K0>
__device__ __forceinline__ void tc2_row_at(unsigned char* row_hi, unsigned char* row_lo, const float (&wy)[W]) {
#pragma unroll
    for (int c = 0; c < KC; ++c) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 4 * c + q - K0;
            v[q] = (k >= 0 && k < W) ? wy[k >= 0 && k < W ? k : 0] : 0.f;
        }
        const float4 h = make_float4(tf32_hi(v[0]), tf32_hi(v[1]), tf32_hi(v[2]), tf32_hi(v[3]));
        *reinterpret_cast<float4*>(row_hi + c * 128) = h;
        *reinterpret_cast<float4*>(row_lo + c * 128) = make_float4(v[0] - h.x, v[1] - h.y, v[2] - h.z, v[3] - h.w);
    }
}

template <int W, int KC, int K0, int KMAX>
__device__ __forceinline__ void tc2_row(int k0, unsigned char* row_hi, unsigned char* row_lo, const float (&wy)[W]) {
    if constexpr (K0 < KMAX) {
        if (k0 != K0) {
            tc2_row<W, KC, K0 + 1, KMAX>(k0, row_hi, row_lo, wy);
            return;
        }
    }
    tc2_row_at<W, KC, K0>(row_hi, row_lo, wy);
}

template <int W>
__global__ void __launch_bounds__(128) k_interp2_tc(InterpArgs a, Epilogue e) {
    using S = Tc2<W>;
    constexpr int m = S::M_W;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* a_hi = smem_raw;
    unsigned char* a_lo = a_hi + S::A_BYTES;
    unsigned char* b_hi = a_lo + S::A_BYTES;
    unsigned char* b_lo = b_hi + S::B_BYTES;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int task, abort_flag;
    __shared__ unsigned warps_done;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc_alloc(&tmem_slot, S::COLS);
    if (tid == 0) {
        mbar_init(&bar, 1);
        warps_done = 0u;
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = tmem + (uint32_t(warp * 32) << 16);
    constexpr uint32_t idesc = tc_idesc_tf32(128, S::N);
    const float* c0 = static_cast<const float*>(a.coord[0]);
    const float* c1 = static_cast<const float*>(a.coord[1]);
    const float* grid = static_cast<const float*>(a.grid);
    const int n = a.n_os;
    unsigned char* row_hi = a_hi + (tid >> 3) * S::SBO + (tid & 7) * 16;
    unsigned char* row_lo = a_lo + (tid >> 3) * S::SBO + (tid & 7) * 16;
    uint32_t phase = 0;
    bool failed = false;
    double sq = 0.0, bad = 0.0, dot = 0.0;
    for (;;) {
        if (tid == 0) task = int(atomicAdd(a.queue, 1u));
        __syncthreads();
        const int t = task;
        if (t >= a.nttasks || abort_flag) break;
        const int bin = a.ttasks[3 * t], start = a.ttasks[3 * t + 1], end = a.ttasks[3 * t + 2];
        const int x0 = (bin / a.nb[1]) * S::BX, y0 = (bin % a.nb[1]) * 8;
        // the box: rows x0 - (m-1) + i, y from y0 - 8; zero outside the grid
        {
            constexpr int LOADS = (S::N * S::KC + 127) / 128;
            float4 v[LOADS];
#pragma unroll
            for (int l = 0; l < LOADS; ++l) {
                const int q = tid + 128 * l;
                const int r = q / S::KC, c = q - r * S::KC;
                const int xr = x0 - (m - 1) + r, yc = y0 - S::YLEAD + 4 * c;
                v[l] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < S::N * S::KC && xr >= 0 && xr < n && yc >= 0 && yc + 4 <= n)
                    v[l] = __ldg(reinterpret_cast<const float4*>(grid + int64_t(xr) * n + yc));
            }
#pragma unroll
            for (int l = 0; l < LOADS; ++l) {
                const int q = tid + 128 * l;
                if (q >= S::N * S::KC) continue;
                const int r = q / S::KC, c = q - r * S::KC;
                const float4 h = make_float4(tf32_hi(v[l].x), tf32_hi(v[l].y), tf32_hi(v[l].z), tf32_hi(v[l].w));
                const int off = (r >> 3) * S::SBO + c * S::LBO + (r & 7) * 16;
                *reinterpret_cast<float4*>(b_hi + off) = h;
                *reinterpret_cast<float4*>(b_lo + off) =
                    make_float4(v[l].x - h.x, v[l].y - h.y, v[l].z - h.z, v[l].w - h.w);
            }
        }
        for (int base = start; base < end; base += 128) {
            const int p = base + tid;
            const bool ok = p < end;
            float wx[W], wy[W];
            int dx = 0, k0 = 0;
            EpiPrefetch ep;
            ep.load(e, p, ok);
            if (ok) {
                int fx, fy;
                window_poly<W, float>(c0[p], a.wp, 1.f, fx, wx);
                window_poly<W, float>(c1[p], a.wp, 1.f, fy, wy);
                dx = min(max(fx - x0, 0), S::BX - 1);
                k0 = min(max(fy - y0 + S::YLEAD - (m - 1), 0), S::KY - W);
            } else {
#pragma unroll
                for (int k = 0; k < W; ++k) wx[k] = wy[k] = 0.f;
            }
            static_assert(S::LBO == 128, "chunk stride of tc2_row_at");
            tc2_row<W, S::KC, 0, S::KY - W>(k0, row_hi, row_lo, wy);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (abort_flag) break;
            if (tid == 0 && !a.inject) {
                tc_fence_after();
                const uint32_t ah = smem_addr(a_hi), al = smem_addr(a_lo), bh = smem_addr(b_hi), bl = smem_addr(b_lo);
#pragma unroll
                for (int s2 = 0; s2 < S::KY / 8; ++s2) {
                    const uint32_t o = uint32_t(s2 * 2 * S::LBO);
                    tc_mma_tf32(tmem, tc_desc(ah + o, S::LBO, S::SBO), tc_desc(bh + o, S::LBO, S::SBO), idesc, s2 > 0);
                    tc_mma_tf32(tmem, tc_desc(ah + o, S::LBO, S::SBO), tc_desc(bl + o, S::LBO, S::SBO), idesc, 1u);
                    tc_mma_tf32(tmem, tc_desc(al + o, S::LBO, S::SBO), tc_desc(bh + o, S::LBO, S::SBO), idesc, 1u);
                }
                tc_commit(&bar);
            }
            // warp-uniform: a warp whose wait gave up on any lane skips the
            // (warp-collective) tensor-memory loads of this tile
            const bool done = __all_sync(0xffffffffu, mbar_wait(&bar, phase));
            phase ^= 1u;
            if (!done) {
                failed = true;
                abort_flag = 1;
                if (e.status) atomicOr(e.status, 4);
            }
            tc_fence_after();
            // the MMA has read the A operand, so the thread's own row of it (6
            // chunks of 4 in the hi part, 6 in the lo part) holds its 32 results:
            // element e in chunk e / 4, chunks 6 and 7 in the lo part
            if (!failed) {
                float h[32];
                tmem_ld32(tlane, h);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<float4*>((c < S::KC ? row_hi + c * S::LBO : row_lo + (c - S::KC) * S::LBO)) =
                        make_float4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3]);
            }
            float tv = 0.f;
#pragma unroll
            for (int q = 0; q < W; ++q) {
                const int el = dx + q, c = el >> 2;
                const unsigned char* at = c < S::KC ? row_hi + c * S::LBO : row_lo + (c - S::KC) * S::LBO;
                tv = fmaf(wx[q], *reinterpret_cast<const float*>(at + (el & 3) * 4), tv);
            }
            if (ok && !failed) epi_point_pre32(e, p, tv, ep.q, ep.a, sq, bad, dot);
            tc_fence_before();
        }
    }
    if (failed) mbar_wait(&bar, phase ^ 1u);
    queue_leave(a.queue, lane);
    epi_finish_warps(e, sq, bad, dot, &warps_done);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, S::COLS);
}

// ------------------------------------------------------------ launchers
struct TcLaunch {
    int smem = 0;     // dynamic shared memory per block
    int blocks = 0;   // resident blocks on the GPU
};

// Shared memory that keeps at most BLOCKS_PER_SM blocks on an SM (their
// tensor-memory columns fit its 512), and the launch's resident block count.
template <auto K, int OPERANDS, int BLOCKS_PER_SM>
static cudaError_t tc_config(TcLaunch& L) {
    int dev = 0, sms = 0, per_sm_smem = 0, reserved = 0, per_block_max = 0;
    cudaError_t err;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return err;
    if ((err = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
        return err;
    if ((err = cudaDeviceGetAttribute(&per_block_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return err;
    cudaFuncAttributes fa{};
    if ((err = cudaFuncGetAttributes(&fa, K)) != cudaSuccess) return err;
    // more than BLOCKS_PER_SM blocks must not fit: (BLOCKS_PER_SM + 1) * (smem + static + reserved) > per SM
    const int need = per_sm_smem / (BLOCKS_PER_SM + 1) + 1 - int(fa.sharedSizeBytes) - reserved;
    int smem = std::max(OPERANDS, need);
    smem = (smem + 127) / 128 * 128;
    if (smem + int(fa.sharedSizeBytes) > per_block_max) return cudaErrorInvalidConfiguration;
    if ((err = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return err;
    // the occupancy calculator reports one block per SM for kernels that
    // allocate tensor memory; the register and shared-memory limits decide
    int regs_per_sm = 0;
    if ((err = cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess)
        return err;
    const int by_regs = regs_per_sm / std::max(1, (fa.numRegs + 7) / 8 * 8 * 128);
    const int by_smem = per_sm_smem / (smem + int(fa.sharedSizeBytes) + reserved);
    const int per_sm = std::min(BLOCKS_PER_SM, std::min(by_regs, by_smem));
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    L.smem = smem;
    L.blocks = per_sm * sms;
    return cudaSuccess;
}

template <int D, int W>
static cudaError_t interp_tc_config(TcLaunch*& out) {
    static TcLaunch cfg[64];
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    TcLaunch& L = cfg[dev & 63];
    if (L.blocks == 0) {
        if constexpr (D == 3) {
            using S = Tc3<W>;
            err = tc_config<k_interp3_tc<W>, S::OPERANDS, S::BLOCKS_PER_SM>(L);
        } else {
            using S = Tc2<W>;
            err = tc_config<k_interp2_tc<W>, S::OPERANDS, S::BLOCKS_PER_SM>(L);
        }
        if (err != cudaSuccess) return err;
    }
    out = &L;
    return cudaSuccess;
}

template <int D, int W>
static cudaError_t interp_tc_one(const InterpArgs& a, const Epilogue& e, cudaStream_t s) {
    TcLaunch* L = nullptr;
    cudaError_t err = interp_tc_config<D, W>(L);
    if (err != cudaSuccess) return err;
    if (a.nttasks == 0) return cudaSuccess;
    const int blocks = std::max(1, std::min(L->blocks, a.nttasks));
    if constexpr (D == 3)
        k_interp3_tc<W><<<blocks, 128, L->smem, s>>>(a, e);
    else
        k_interp2_tc<W><<<blocks, 128, L->smem, s>>>(a, e);
    return cudaGetLastError();
}

template <int D, int W>
static int interp_tc_grid(int ntasks) {
    TcLaunch* L = nullptr;
    if (interp_tc_config<D, W>(L) != cudaSuccess || !L) return 0;
    return std::max(1, std::min(L->blocks, ntasks));
}

bool tc_supported(int d, int W, int precision_fp32) {
    return precision_fp32 && ((d == 3 && W >= 4 && W <= 10) || (d == 2 && W >= 4 && W <= 16));
}

#define SK_TC_CASES(FN, ...)                                    \
    if (d == 3) {                                               \
        switch (W) {                                            \
            case 4: return FN<3, 4>(__VA_ARGS__);               \
            case 6: return FN<3, 6>(__VA_ARGS__);               \
            case 8: return FN<3, 8>(__VA_ARGS__);               \
            case 10: return FN<3, 10>(__VA_ARGS__);             \
            default: break;                                     \
        }                                                       \
    } else if (d == 2) {                                        \
        switch (W) {                                            \
            case 4: return FN<2, 4>(__VA_ARGS__);               \
            case 6: return FN<2, 6>(__VA_ARGS__);               \
            case 8: return FN<2, 8>(__VA_ARGS__);               \
            case 10: return FN<2, 10>(__VA_ARGS__);             \
            case 12: return FN<2, 12>(__VA_ARGS__);             \
            case 14: return FN<2, 14>(__VA_ARGS__);             \
            case 16: return FN<2, 16>(__VA_ARGS__);             \
            default: break;                                     \
        }                                                       \
    }

cudaError_t launch_interp_tc(int d, int W, const InterpArgs& a, const Epilogue& e, cudaStream_t s) {
    SK_TC_CASES(interp_tc_one, a, e, s)
    return cudaErrorInvalidValue;
}

int interp_tc_blocks(int d, int W, int ntasks) {
    SK_TC_CASES(interp_tc_grid, ntasks)
    return 0;
}
#undef SK_TC_CASES

}  // namespace sk
