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
constexpr int kSpreadMaxPts = 1024;  // points per spreading subproblem
constexpr int kTaskMaxPts = 4096;    // points per column task before a bin is split
constexpr int kTaskMaxPts2 = 2048;   // the same for the 2-D column kernel (finer tasks balance its strip bins)

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

// The regularized kernel K_R at distance rho (torus units): K_I below eps_I
// when near-field regularization is on, the exact kernel exp(-rho^r / eps_s)
// up to L, the boundary polynomial K_B beyond (constant past 1/2).
__host__ __device__ inline double kr_value(double rho, const KernelParams& kp) {
    double v = 0.0;
    if (kp.nearfield && rho < kp.eps_I) {
        const double s2 = (rho * rho) / (kp.eps_I * kp.eps_I);
        for (int q = kp.p - 1; q >= 0; --q) v = v * s2 + kp.ki[q];
    } else if (rho <= kp.L) {
        v = exp(-pow(rho, kp.r) / kp.eps_s);
    } else {
        const double tau = (fmin(rho, 0.5) - kp.L) / (0.5 - kp.L);
        for (int i = 2 * kp.p - 2; i >= 0; --i) v = v * tau + kp.kb[i];
    }
    return v;
}

struct Cloud {
    int64_t n = 0;
    void* coord[3] = {nullptr, nullptr, nullptr};  // T*, sorted grid coordinates
    int* perm = nullptr;        // sorted -> caller index
    double* marg = nullptr;     // sorted marginal (a or b)
    double* scal = nullptr;     // sorted scaling vector (u or v)
    double* t = nullptr;        // sorted kernel sums of the last product into this cloud
    double* work = nullptr;     // sorted scratch (gathered weights)
    double* stage = nullptr;    // caller-order scratch for host<->device staging
    int* key_start = nullptr;   // CSR over sort keys (bin, cell in bin), nkeys + 1
    int* bin_start = nullptr;   // CSR over bins, nbins + 1
    int* tasks = nullptr;       // column tasks (3-D)
    int ntasks = 0;
    int* cols = nullptr;        // non-empty (bin, column) pairs, bin * columns + column, most points first (3-D)
    int ncols = 0;
    int* stasks = nullptr;      // 2-D strip tasks (bin, first point, end point), most points first
    int nstasks = 0;
    int* ttasks = nullptr;      // tensor-core interpolation runs (bin, first point, end point), most points first
    int nttasks = 0;
    // near-field cell list (only when the kernel needs near-field correction)
    int* nf_start = nullptr;    // CSR over near-field cells
    int* nf_idx = nullptr;      // near-field position -> sorted index
    void* nf_coord[3] = {nullptr, nullptr, nullptr};   // T*, coordinates in near-field order
    int* nf_tasks = nullptr;    // non-empty near-field cells
    int nf_ntasks = 0;
    double* nf_corr = nullptr;  // correction of the last product into this cloud (sorted order)
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
    const int* perm = nullptr;   // APPLY: out[perm[i]] = t_i (out[i] = t_i when null)
    double* out = nullptr;
    double* t_store = nullptr;   // UPDATE / RESID: t_store[i] = t_i
    const double* marg = nullptr;
    double* scal = nullptr;      // UPDATE: scal[i] = marg[i] / t_i; RESID: read only
    const double* add = nullptr; // if set, t_i += add[i] before anything else (near-field correction)
    double* partial = nullptr;   // 3 doubles per block
    unsigned* ticket = nullptr;  // zero between launches; the last block resets it
    double* result = nullptr;    // [0] sum (scal_old t - marg)^2, [1] bad count, [2] sum scal_old t
    int* status = nullptr;       // bit 0 set when some t_i <= 0 or not finite (UPDATE); bit 2 when a
                                 // bounded wait of a tensor-core kernel gave up
    // log domain (Alg. 4): scal holds the dual variables beta; t_i is the sum
    // with the source weights exp((gamma_j - shift) / eps - 1/2), shift = *shift
    int log_domain = 0;
    int fp32_logs = 0;           // logs and exps of FP32-accurate sums in FP32 (FP32 plans)
    double eps = 0.0, lam = 0.0; // eps and 1 / eps
    const double* shift = nullptr;
};

// Piecewise-polynomial form of the Kaiser-Bessel window (the Horner scheme of
// Barnett, Magland and af Klinteberg's FINUFFT): on each of its W = 2m unit
// intervals the window, as a function of s = 2 frac - 1 in [-1, 1], is
// replaced by its Chebyshev interpolant of degree 8 (FP32) or 14 (FP64),
// written in monomials of s.  Tap k of a point with fractional offset frac is
// psi(frac + m - 1 - k) ~ sum_i c[k][i] s^i.  The interpolation error is below
// 7e-8 (degree 8, m = 2), 7e-9 (degree 8, m >= 4) and 1e-14 (degree 14) of
// the window's peak; FP32 rounding of the evaluation is ~6e-8.
constexpr int kPolyDeg32 = 8;
constexpr int kPolyDeg64 = 14;
struct WindowPoly {
    float c32[16][kPolyDeg32 + 1];
    double c64[16][kPolyDeg64 + 1];
};

struct SpreadArgs {
    const void* coord[3];
    const double* w;       // sorted weights
    const int* sub_start;  // subproblems of the per-point kernel
    const int* sub_count;
    const int* sub_bin;
    int nsub;
    const int* key_start;  // CSR over sort keys (bin, cell in bin)
    const int* tasks;      // column tasks: (bin, first column, end column)
    int ntasks;
    int n_os;
    int nb[3];             // bins per dimension
    double beta;           // Kaiser-Bessel shape
    double knorm;          // m / sinh(beta m): normalizes the window to 1 at 0
    void* grid;            // T*, n_os^d, zeroed by the caller
    WindowPoly wp;
};

struct InterpArgs {
    const void* coord[3];
    int64_t n;
    const int* key_start;
    const int* tasks;
    int ntasks;
    const int* cols;       // 3-D column queue: (bin, column) codes, most points first
    int ncols;
    const int* stasks;     // 2-D strip tasks: (bin, first point, end point), most points first
    int nstasks;
    const int* ttasks;     // tensor-core runs: (bin, first point, end point), most points first
    int nttasks;
    int inject;            // test hook: 1 = the tensor-core kernels skip their MMA, so its bounded wait runs out
    unsigned* queue;       // [0] next queue entry, [1] warps finished; zero between launches
    int nb[3];
    int n_os;
    double beta, knorm;
    const void* grid;
    WindowPoly wp;
};

struct NearArgs {
    const void* t_coord[3];   // targets in near-field order (T, grid units)
    const int* t_start;       // CSR over near-field cells of the targets
    const int* t_idx;         // near-field position -> sorted target index
    const void* s_coord[3];   // sources in near-field order
    const int* s_start;
    const int* s_idx;
    const double* w;          // source weights in sorted order
    const int* tasks;         // non-empty target cells
    int nc;                   // near-field cells per dimension
    int sub;                  // cells per eps_I (2 or 4)
    double r2max;             // (n_os eps_I)^2: squared near-field radius in grid units
    double inv_r2;            // 1 / r2max
    double kcoef;             // K = exp(-kcoef |du|^r) with kcoef = 1 / (eps_s n_os^r)
    double r;
    int p;
    double ki[kMaxP];         // K_I = sum_q ki[q] (|du|^2 / r2max)^q
    double* out;              // correction per target, sorted order
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
    void* grid = nullptr;     // T*, spreading target; zero outside the band, zeroed again by the first pass
    void* grid_out = nullptr; // T*, written by the last pass inside the band, read by interpolation
    int lo[3] = {0, 0, 0};    // band: cells lo[t]..hi[t] (inclusive) hold every point's window taps
    int hi[3] = {0, 0, 0};
    void* A1 = nullptr;       // Cplx<T>*
    void* A2 = nullptr;       // Cplx<T>*, 3-D only
    void* A3 = nullptr;       // Cplx<T>*, stage entry points only
    void* mult = nullptr;     // T*
    void* tw = nullptr;       // Cplx<T>*, the stage twiddle rows (fft_twiddle_rows<T>(n) entries)
    const double* psihat = nullptr;  // 2h+1 values psihat_n(k/n), k = -h..h (FP64)
    bool planes = false;      // 3-D FP32: the grid-side passes by thread-block-cluster planes (three launches)
    bool pdl = true;          // the plane path's three launches use programmatic dependent launch
};

// ----------------------------------------------------------------- launchers
template <typename T> cudaError_t launch_spread(int d, int W, const SpreadArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_interp(int d, int W, const InterpArgs& a, const Epilogue& e,
                                                int64_t* launches, cudaStream_t s);
template <typename T> int interp_blocks(int64_t n);
template <typename T> cudaError_t launch_spread3(int W, const SpreadArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_interp3(int W, const InterpArgs& a, const Epilogue& e, cudaStream_t s);
template <typename T> int interp3_blocks(int W, int ncols);
template <typename T> cudaError_t launch_spread2(int W, const SpreadArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_interp2(int W, const InterpArgs& a, const Epilogue& e, cudaStream_t s);
template <typename T> int strip2_blocks(int W, int ntasks);
constexpr int kStripMaxPts = 128;   // points per 2-D strip task
inline int strip_bx(int W) { return 33 - W; }   // x-cells of a 2-D strip: its window spans 32 rows
constexpr int kStripBy = 8;         // y-cells of a 2-D strip
bool column_kernels(int d, int W);
// Tensor-core (tcgen05) interpolation of FP32 plans, 2-D and 3-D (sk_tc.cu):
// tasks are runs of at most kTcRunPts points of one bin in InterpArgs::ttasks.
constexpr int kTcRunPts = 512;
bool tc_supported(int d, int W, int precision_fp32);
cudaError_t launch_interp_tc(int d, int W, const InterpArgs& a, const Epilogue& e, cudaStream_t s);
int interp_tc_blocks(int d, int W, int ntasks);
void bin_shape(int d, int W, int B[3]);
template <typename T> cudaError_t launch_fft_convolve(const FftPlan& f, cudaStream_t s, int64_t* launches);
bool fft_planes_supported(const FftPlan& f, bool fp32);
template <typename T> int fft_twiddle_rows(int n);
template <typename T> cudaError_t launch_twiddle_rows(void* rows, int n, cudaStream_t s);
template <typename T> cudaError_t launch_fft_adjoint(const FftPlan& f, double* fhat, cudaStream_t s,
                                                     int64_t* launches);
template <typename T> cudaError_t launch_fft_forward(const FftPlan& f, const double* fhat, cudaStream_t s,
                                                     int64_t* launches);
template <typename T> void launch_near_keys(void* const u[3], int64_t n, int d, double inv_cell, int nc, int* key,
                                            int* count, cudaStream_t s);
void launch_near_scatter(const int* key, int64_t n, const int* start, int* cursor, int* idx, cudaStream_t s);
template <typename T> void launch_near_gather(const int* idx, int64_t n, int d, void* const u[3], void* const o[3],
                                              cudaStream_t s);
void launch_near_tasks(const int* start, int ncells, int* tasks, int* ntasks, cudaStream_t s);
void launch_count_nonempty(const int* count, int ncells, int* nonempty, cudaStream_t s);
template <typename T> cudaError_t launch_nearfield(int d, const NearArgs& a, int ntasks, cudaStream_t s);
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

// a / t in FP64 for t > 0 in the FP32 normal range (tf = float(t)): the FP32
// reciprocal r (relative error below 2^-23) gives q = a r, and one Newton
// correction of the quotient, q + r (a - t q), squares that error (below
// 2^-45 relative, far under the error of the kernel sums t).  Four FP64
// operations instead of a full IEEE division, whose FP64 cost dominates on
// this GPU; outside that range it divides.
__device__ __forceinline__ double div_newton(double a, double t, float tf) {
    if (!(tf >= 1.17549435e-38f) || !(tf <= 3.0e38f)) return a / t;
    const double r = double(__frcp_rn(tf));
    const double q = a * r;
    return fma(r, fma(-t, q, a), q);
}

// log v for v > 0 in the FP32 normal range, split as e ln 2 + log(m) with
// v = m 2^e, m in [1/2, 1): the FP32 logarithm of m carries an absolute error
// of about 6e-8 whatever the size of log v.
__device__ __forceinline__ double log_split(float v) {
    int ex = 0;
    const float mant = frexpf(v, &ex);
    return double(ex) * 0.69314718055994530942 + double(logf(mant));
}

// Log-domain update (Alg. 4 with the first-order condition of Eq. (11)):
// beta_new = eps (log a - log t + 1/2) with t = exp(lam shift) t', and the
// residual of the old state u_old t - a = a (exp(lam (beta_old - beta_new)) - 1)
// (u_new t = a exactly).  RESID: u t = exp(lam (beta + shift) - 1/2) t'.
__device__ __forceinline__ void epi_point_log(const Epilogue& e, int64_t i, double t, double q, double a,
                                              double& sq, double& bad, double& dot) {
    const double sh = *e.shift;
    if (e.mode == EPI_UPDATE) {
        const float tf = float(t);
        if (!(tf >= 1.17549435e-38f && tf <= 3.0e38f)) bad += 1.0;
        double bn, r;
        if (!(a > 0.0)) {           // a point without mass: beta = -inf, no residual
            bn = -INFINITY;
            r = 0.0;
        } else if (e.fp32_logs) {
            bn = e.eps * (log_split(float(a)) - log_split(tf) + 0.5) - sh;
            r = a * double(expm1f(float(e.lam * (q - bn))));
        } else {
            bn = e.eps * (log(a) - log(t) + 0.5) - sh;
            r = a * expm1(e.lam * (q - bn));
        }
        sq = fma(r, r, sq);
        e.scal[i] = bn;
    } else {
        const double ut = a > 0.0 ? exp(e.lam * (q + sh) - 0.5) * t : 0.0;
        const double r = ut - a;
        sq = fma(r, r, sq);
        dot += ut;
        e.t_store[i] = t;
    }
}

// Per-point FP64 epilogue (Eq. (S1) update and Eq. (Error) residual terms).
// UPDATE: sq += (u_old t - a)^2 and u = a / t (the residual of the state before
// the update; the sum u_old t and the kernel sums are not needed inside the
// iteration).  RESID: sq, dot += u t, and t itself, for the final report.
__device__ __forceinline__ void epi_point(const Epilogue& e, int64_t i, double t,
                                          double& sq, double& bad, double& dot) {
    if (e.add) t += e.add[i];
    if (e.mode == EPI_APPLY) {
        e.out[e.perm ? e.perm[i] : i] = t;
        return;
    }
    const double q = e.scal[i];
    const double a = e.marg[i];
    if (e.log_domain) {
        epi_point_log(e, i, t, q, a, sq, bad, dot);
        return;
    }
    const double r = fma(q, t, -a);
    sq = fma(r, r, sq);
    if (e.mode == EPI_UPDATE) {
        const float tf = float(t);
        if (!(tf >= 1.17549435e-38f && tf <= 3.0e38f)) bad += 1.0;
        e.scal[i] = div_newton(a, t, tf);
    } else {
        dot = fma(q, t, dot);
        e.t_store[i] = t;
    }
}

// The epilogue's per-point inputs (old scaling value and marginal), loaded one
// batch ahead of their use.
struct EpiPrefetch {
    double q = 0.0, a = 0.0;
    __device__ __forceinline__ void load(const Epilogue& e, int64_t i, bool ok) {
        if (ok && e.mode != EPI_APPLY) {
            q = e.scal[i];
            a = e.marg[i];
        }
    }
};

// epi_point with the scaling value and marginal already loaded.
__device__ __forceinline__ void epi_point_pre(const Epilogue& e, int64_t i, double t, double q, double a,
                                              double& sq, double& bad, double& dot) {
    if (e.add) t += e.add[i];
    if (e.mode == EPI_APPLY) {
        e.out[e.perm ? e.perm[i] : i] = t;
        return;
    }
    if (e.log_domain) {
        epi_point_log(e, i, t, q, a, sq, bad, dot);
        return;
    }
    const double r = fma(q, t, -a);
    sq = fma(r, r, sq);
    if (e.mode == EPI_UPDATE) {
        const float tf = float(t);
        if (!(tf >= 1.17549435e-38f && tf <= 3.0e38f)) bad += 1.0;
        e.scal[i] = div_newton(a, t, tf);
    } else {
        dot = fma(q, t, dot);
        e.t_store[i] = t;
    }
}

// The same for a kernel sum computed in FP32 (tv): without a near-field term
// to add, the update's FP32 seed is tv itself, so the sum is converted to FP64
// once and never back (bit-identical to epi_point_pre(e, i, double(tv), ...)).
__device__ __forceinline__ void epi_point_pre32(const Epilogue& e, int64_t i, float tv, double q, double a,
                                                double& sq, double& bad, double& dot) {
    if (e.add || e.mode == EPI_APPLY || e.log_domain) {
        epi_point_pre(e, i, double(tv), q, a, sq, bad, dot);
        return;
    }
    const double t = double(tv);
    const double r = fma(q, t, -a);
    sq = fma(r, r, sq);
    if (e.mode == EPI_UPDATE) {
        if (!(tv >= 1.17549435e-38f && tv <= 3.0e38f)) bad += 1.0;
        e.scal[i] = div_newton(a, t, tv);
    } else {
        dot = fma(q, t, dot);
        e.t_store[i] = t;
    }
}

// Reduction of the epilogue sums without a block-wide barrier: each warp adds
// its sums into the block's shared slots; the last warp of the block to
// arrive writes the block partial and takes part in the grid-wide
// last-block-done reduction (deterministic order over blocks).
// `warps_done` is a shared counter the kernel sets to 0 before its first
// __syncthreads.
__device__ __forceinline__ void epi_finish_warps(const Epilogue& e, double sq, double bad, double dot,
                                                 unsigned* warps_done) {
    if (e.mode == EPI_APPLY) return;
    __shared__ double wsum[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned nw = (blockDim.x + 31) >> 5;
    sq = warp_sum(sq);
    bad = warp_sum(bad);
    dot = warp_sum(dot);
    bool last_warp = false;
    if (lane == 0) {
        wsum[0][wid] = sq;
        wsum[1][wid] = bad;
        wsum[2][wid] = dot;
        __threadfence_block();
        last_warp = atomicAdd(warps_done, 1u) == nw - 1;
    }
    last_warp = __shfl_sync(0xffffffffu, last_warp, 0);
    if (!last_warp) return;
    __threadfence_block();
    double b0 = 0.0, b1 = 0.0, b2 = 0.0;
    if (lane < int(nw)) {
        b0 = ((volatile double*)wsum[0])[lane];
        b1 = ((volatile double*)wsum[1])[lane];
        b2 = ((volatile double*)wsum[2])[lane];
    }
    // block sum in warp order (lanes are warps), then the grid step
    b0 = warp_sum(b0);
    b1 = warp_sum(b1);
    b2 = warp_sum(b2);
    bool last = false;
    if (lane == 0) {
        e.partial[3 * blockIdx.x + 0] = b0;
        e.partial[3 * blockIdx.x + 1] = b1;
        e.partial[3 * blockIdx.x + 2] = b2;
        __threadfence();
        last = atomicAdd(e.ticket, 1u) == gridDim.x - 1;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) {
        s0 += ((volatile double*)e.partial)[3 * b + 0];
        s1 += ((volatile double*)e.partial)[3 * b + 1];
        s2 += ((volatile double*)e.partial)[3 * b + 2];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) {
        e.result[0] = s0;
        e.result[1] = s1;
        e.result[2] = s2;
        if (s1 > 0.0 && e.status) atomicOr(e.status, 1);
        *e.ticket = 0u;
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
