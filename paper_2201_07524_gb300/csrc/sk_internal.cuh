// Internal declarations shared by the translation units of the sk library.
//
// Data layout on the device (one plan):
//   * Each point cloud (X = sources x_i of K v's output side, Y = targets y_j)
//     is bin-sorted once at plan time.  Coordinates are stored SoA in grid
//     units u_t = n_os * z_t (z the torus coordinates), type T (float/double).
//     perm[i] maps the sorted position i to the caller's index.
//   * Marginals, scaling vectors and kernel sums are FP64 in sorted order.
//   * The oversampled grid g (n_os^d values of T, last axis contiguous) and two
//     complex spectra: A1 (real-to-complex half spectrum along the last axis)
//     and A2 (3-D only: axis 1 pruned to the 2h+1 kept frequencies).
//   * The multiplier table M = c_k b_k / prod_t psihat(k_t)^2 over the kept
//     frequencies, last axis halved (k_d in 0..h), type T.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../include/sk.h"

namespace sk {

constexpr int kMaxP = 12;            // smoothness limit of the regularized kernel
constexpr int kFftElems = 4096;      // complex elements per FFT block (P pencils x n)
constexpr int kSpreadMaxPts = 1024;  // points per spreading subproblem

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Parameters of the regularized kernel K_R in torus coordinates.
struct KernelParams {
    double eps_s;   // eps * scale^r
    double r;
    double L;       // 1/2 - eps_B
    double eps_I;   // near-field radius (used iff nearfield)
    int p;
    int nearfield;
    double kb[2 * kMaxP - 1];   // K_B(rho) = sum kb[i] tau^i, tau = (rho - L)/(1/2 - L)
    double ki[kMaxP];           // K_I(rho) = sum ki[q] (rho/eps_I)^(2q)
};

struct Cloud {
    int64_t n = 0;
    void* coord[3] = {nullptr, nullptr, nullptr};  // T*, sorted grid coordinates
    int* perm = nullptr;        // sorted -> caller index
    double* marg = nullptr;     // sorted marginal (a or b)
    double* scal = nullptr;     // sorted scaling vector (u or v)
    double* t = nullptr;        // sorted kernel sums of the last product into this cloud
    double* work = nullptr;     // sorted scratch (gathered weights)
    double* stage = nullptr;    // caller-order scratch for host<->device staging
    int* bin_start = nullptr;   // CSR over bins, nbins + 1
    int* sub_start = nullptr;   // spreading subproblems
    int* sub_count = nullptr;
    int* sub_bin = nullptr;
    int nsub = 0;
};

// What the interpolation / direct-sum kernels do with each kernel sum t_i.
enum EpiMode { EPI_APPLY = 0, EPI_UPDATE = 1, EPI_RESID = 2 };

struct Epilogue {
    int mode = EPI_APPLY;
    int64_t n = 0;
    const int* perm = nullptr;   // APPLY: out[perm[i]] = t_i
    double* out = nullptr;
    double* t_store = nullptr;   // UPDATE / RESID: t_store[i] = t_i
    const double* marg = nullptr;
    double* scal = nullptr;      // UPDATE: scal[i] = marg[i] / t_i; RESID: read only
    double* partial = nullptr;   // 3 doubles per block
    unsigned* ticket = nullptr;  // zero between launches; the last block resets it
    double* result = nullptr;    // [0] sum (scal_old t - marg)^2, [1] bad count, [2] sum scal_old t
    int* status = nullptr;       // bit 0 set when some t_i <= 0 or not finite (UPDATE)
};

struct SpreadArgs {
    const void* coord[3];
    const double* w;       // sorted weights
    const int* sub_start;
    const int* sub_count;
    const int* sub_bin;
    int nsub;
    int n_os;
    int nb[3];             // bins per dimension
    int B;                 // bin side in cells
    double beta;           // Kaiser-Bessel shape
    double knorm;          // m / sinh(beta m): normalizes the window to 1 at 0
    void* grid;            // T*, n_os^d, zeroed by the caller
};

struct InterpArgs {
    const void* coord[3];
    int64_t n;
    int n_os;
    double beta, knorm;
    const void* grid;
};

struct DirectArgs {
    const void* tcoord[3];   // targets (sorted grid coordinates)
    int64_t nt;
    const void* scoord[3];   // sources
    const double* w;         // sorted source weights
    int64_t ns;
    double coef;             // 1 / (eps_s * n_os^r): K = exp(-coef * |du|^r)
    double r;
};

// FFT pipeline description (per precision the plan uses).
struct FftPlan {
    int d = 0;
    int n = 0;          // n_os
    int log2n = 0;
    int h = 0;          // N/2
    void* grid = nullptr;     // T*
    void* A1 = nullptr;       // Cplx<T>*
    void* A2 = nullptr;       // Cplx<T>*, 3-D only
    void* A3 = nullptr;       // Cplx<T>*, stage entry points only
    void* mult = nullptr;     // T*
    void* tw = nullptr;       // Cplx<T>*, n/2 twiddles exp(-2 pi i k / n)
    const double* psihat = nullptr;  // 2h+1 values psihat_n(k/n), k = -h..h (FP64)
};

// ----------------------------------------------------------------- launchers
template <typename T> cudaError_t launch_spread(int d, int W, const SpreadArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_interp(int d, int W, const InterpArgs& a, const Epilogue& e,
                                                int64_t* launches, cudaStream_t s);
template <typename T> int interp_blocks(int64_t n);
template <typename T> cudaError_t launch_fft_convolve(const FftPlan& f, cudaStream_t s, int64_t* launches);
template <typename T> cudaError_t launch_fft_adjoint(const FftPlan& f, double* fhat, cudaStream_t s,
                                                     int64_t* launches);
template <typename T> cudaError_t launch_fft_forward(const FftPlan& f, const double* fhat, cudaStream_t s,
                                                     int64_t* launches);
template <typename T> cudaError_t launch_direct(int d, const DirectArgs& a, const Epilogue& e,
                                                int64_t* launches, cudaStream_t s);
template <typename T> int direct_blocks(int64_t nt);

// ----------------------------------------------------------- device helpers
#ifdef __CUDACC__

// Kaiser-Bessel window in grid units, normalized to 1 at 0 (Plonka et al. Ch. 7):
// psi(x) = sinh(beta sqrt(m^2 - x^2)) / sqrt(m^2 - x^2) * m / sinh(beta m), |x| <= m.
template <typename T>
__device__ __forceinline__ T kb_window(T x, T m, T beta, T knorm) {
    T z2 = m * m - x * x;
    if (z2 <= T(0)) return (z2 == T(0)) ? beta * knorm : T(0);
    T z = sqrt(z2);
    return sinh(beta * z) / z * knorm;
}

// Weight of frequency k in {-h..h}^d when the real part of a sum over
// I_N = {-h..h-1}^d is written as a sum over {-h..h}^d of Hermitian terms:
// Re sum_{I_N} = sum_k (1/2)(1[k in I_N] + 1[-k in I_N]) (.).
__host__ __device__ __forceinline__ double re_weight(const int* k, int d, int h) {
    bool in_pos = true, in_neg = true;
    for (int t = 0; t < d; ++t) {
        in_pos = in_pos && (k[t] != h);
        in_neg = in_neg && (k[t] != -h);
    }
    return 0.5 * (double(in_pos) + double(in_neg));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-point FP64 epilogue (Eq. (S1) update and Eq. (Error) residual terms).
__device__ __forceinline__ void epi_point(const Epilogue& e, int64_t i, double t,
                                          double& sq, double& bad, double& dot) {
    if (e.mode == EPI_APPLY) {
        e.out[e.perm[i]] = t;
        return;
    }
    double q = e.scal[i];
    double a = e.marg[i];
    double r = q * t - a;
    sq += r * r;
    dot += q * t;
    e.t_store[i] = t;
    if (e.mode == EPI_UPDATE) {
        double qn = a / t;
        if (!(t > 0.0) || !isfinite(qn)) bad += 1.0;
        e.scal[i] = qn;
    }
}

// Block reduction of the three epilogue sums, then a deterministic
// last-block-done reduction over the per-block partials.
__device__ __forceinline__ void epi_finish(const Epilogue& e, double sq, double bad, double dot) {
    if (e.mode == EPI_APPLY) return;
    __shared__ double red[3][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sq = warp_sum(sq);
    bad = warp_sum(bad);
    dot = warp_sum(dot);
    if (lane == 0) { red[0][wid] = sq; red[1][wid] = bad; red[2][wid] = dot; }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (wid == 0) {
        sq = lane < nw ? red[0][lane] : 0.0;
        bad = lane < nw ? red[1][lane] : 0.0;
        dot = lane < nw ? red[2][lane] : 0.0;
        sq = warp_sum(sq);
        bad = warp_sum(bad);
        dot = warp_sum(dot);
        if (lane == 0) {
            e.partial[3 * blockIdx.x + 0] = sq;
            e.partial[3 * blockIdx.x + 1] = bad;
            e.partial[3 * blockIdx.x + 2] = dot;
            __threadfence();
            unsigned tk = atomicAdd(e.ticket, 1u);
            last = (tk == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        s0 += ((volatile double*)e.partial)[3 * b + 0];
        s1 += ((volatile double*)e.partial)[3 * b + 1];
        s2 += ((volatile double*)e.partial)[3 * b + 2];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    __syncthreads();
    if (lane == 0) { red[0][wid] = s0; red[1][wid] = s1; red[2][wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < nw; ++w) { a0 += red[0][w]; a1 += red[1][w]; a2 += red[2][w]; }
        e.result[0] = a0;
        e.result[1] = a1;
        e.result[2] = a2;
        if (a1 > 0.0 && e.status) atomicOr(e.status, 1);
        *e.ticket = 0u;
    }
}

#endif  // __CUDACC__

}  // namespace sk
