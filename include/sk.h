/*
 * sk.h -- C ABI of the GB300 library for NFFT-accelerated Sinkhorn.
 *
 * Method: Lakshmanan, Pichler, Potts, "Nonequispaced Fast Fourier Transform
 * Boost for the Sinkhorn Algorithm".  Sinkhorn's iteration (Alg. 1, Eq. (S1))
 * alternates the scaling updates u = a ./ (K v) and v = b ./ (K^T u) with the
 * Gibbs kernel K_ij = exp(-||x_i - y_j||^r / eps) (the paper's exp(-lambda d^r)
 * with eps = 1/lambda).  Alg. 3 replaces both kernel-vector products by the
 * NFFT-based fast summation of Eq. (fastsum): spread the source weights onto
 * an oversampled grid with a Kaiser-Bessel window (adjoint NFFT), FFT,
 * multiply by the Fourier coefficients b_k of the regularized kernel
 * (Eq. (ansatz_NFFT)), inverse FFT, interpolate at the targets (NFFT).
 *
 * Conventions shared by every entry point:
 *  - Status: every int-returning call returns SK_OK (0) or one SK_ERR_* code;
 *    no C++ exception crosses this boundary.  sk_error_string() names a code.
 *  - Pointers: every double array argument may be device memory or host memory
 *    (pageable or pinned); the library asks the CUDA runtime which it is and
 *    copies host arrays itself.  Inputs are read-only and owned by the caller.
 *    Outputs are written in the caller's original point order.
 *  - Points: x is n-by-d and y is m-by-d, row-major (point i at x[i*d .. i*d+d-1]).
 *  - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *    All work is ordered after prior work on that stream; calls that return
 *    host values (sk_solve with a result, sk_init, the state getters)
 *    synchronize with it before returning.
 *  - Threading: a plan is not re-entrant.  Distinct plans may be used from
 *    different host threads and streams concurrently.
 */
#ifndef SK_H
#define SK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum {
    SK_OK = 0,
    SK_ERR_ARG = 1,           /* invalid argument (sizes, dims, parameters, NULL) */
    SK_ERR_DOMAIN = 2,        /* non-finite coordinates, or a point that falls outside the grid */
    SK_ERR_WEIGHTS = 3,       /* weights negative / non-finite / not summing to 1 */
    SK_ERR_NOMEM = 4,         /* device allocation failed */
    SK_ERR_UNDERFLOW = 5,     /* a kernel sum K v or K^T u was <= 0 or not finite */
    SK_ERR_NOT_CONVERGED = 6, /* tol > 0 and max_iter reached with ||E|| > tol */
    SK_ERR_TIMEOUT = 7,       /* reserved for bounded device waits */
    SK_ERR_CUDA = 8,          /* a CUDA runtime call failed */
    SK_ERR_UNSUPPORTED = 9,   /* valid request the library does not implement for this plan */
    SK_ERR_TOO_LARGE = 10     /* size beyond the fixed scratch of sk_direct_residual_noalloc */
};

enum { SK_FP32 = 0, SK_FP64 = 1 };          /* precision of spreading / FFT / interpolation */
enum { SK_METHOD_NFFT = 0, SK_METHOD_DIRECT = 1 };
enum { SK_DOMAIN_SCALING = 0, SK_DOMAIN_LOG = 1 };   /* state of the iteration: Alg. 3 or Alg. 4 */
enum { SK_KERNELS_SIMT = 0, SK_KERNELS_TENSOR = 1 };   /* interpolation on CUDA cores or tensor cores */
enum { SK_FFT_PASSES = 0, SK_FFT_PLANES = 1 };         /* 3-D FFT: five pass launches or three with cluster planes */
enum { SK_FAULT_NONE = 0, SK_FAULT_TC_WAIT = 1 };      /* sk_inject_fault (test hook) */
enum { SK_SET_X = 0, SK_SET_Y = 1 };        /* which point cloud a stage entry point acts on */

typedef struct sk_plan sk_plan;

/*
 * Parameters of the fast summation (Sec. 4.1).  The paper leaves all of them
 * open; sk_default_params() fills in the values this library is tested with.
 *   N        bandwidth: Fourier coefficients b_k for k in I_N = {-N/2..N/2-1}^d
 *            (Eq. (ansatz_NFFT)); even, >= 8.  N <= 0: chosen by sk_init once
 *            the geometry is known, as the smallest power of two >= 16 whose
 *            Fourier tail of the regularized kernel (one-dimensional slice) is
 *            below 1e-6 / d (SK_FP32) or 1e-10 / d (SK_FP64) of K(0).
 *   sigma    oversampling; the FFT grid has n_os = sigma*N points per dimension,
 *            which must be a power of two, 16 <= n_os <= 1024 (4096 for d = 1).
 *   m_w      Kaiser-Bessel window cutoff: 2*m_w taps per dimension, 2 <= m_w <= 8,
 *            n_os >= 4*(m_w+1).  m_w <= 0: the smallest m whose window error
 *            estimate 4 pi (1-1/sigma)^(1/4) exp(-2 pi m sqrt(1-1/sigma)) meets
 *            the same target (at most 5 in 3-D).
 *   p        smoothness of the regularized kernel: the boundary polynomial K_B and
 *            the near-field polynomial K_I match p-1 derivatives, 2 <= p <= 12.
 *   eps_B    width of the boundary region (torus units): L = 1/2 - eps_B, 0 < eps_B < 1/2.
 *   eps_I    near-field radius (torus units), used only when K is not smooth at 0
 *            (r not an even integer; Remark "Arithmetic complexity"): pairs closer
 *            than eps_I are summed directly with the exact kernel, the rest by the
 *            fast summation of the regularized kernel; 0 < eps_I < 1/2 - eps_B.
 *            eps_I <= 0 selects 16 / (3 N), which kept the fast-summation error
 *            below 1e-6 (d <= 2) and 5e-6 (d = 3) in the tested range with p = 8;
 *            the cost of the direct part grows like eps_I^d.
 *   precision SK_FP32 or SK_FP64 for spreading, FFT and interpolation; the scaling
 *            updates, residuals and objective are always FP64.
 *   user_geometry 0: the plan picks center = midpoint of the bounding box of
 *            x and y and scale = (1/4 - eps_B/2) / R with R the largest distance
 *            to that center; 1: use `center` and `scale` as given.  Torus
 *            coordinates are z = scale * (x - center) + 1/2.
 */
typedef struct {
    int N;
    double sigma;
    int m_w;
    int p;
    double eps_B;
    double eps_I;
    int precision;
    int user_geometry;
    double center[3];
    double scale;
} sk_nfft_params;

/* Summary of a solve (Alg. 3 result line, with 1/lambda = eps). */
typedef struct {
    double s;            /* eps (1 + <a,log u> + <b,log v> - sum_j v_j (K^T u)_j) */
    double s_upper;      /* s + eps (H(a) + H(b))  (the paper's upper bound s~_NFFT) */
    double err_row;      /* ||u .* (K v) - a||_2 of the returned state   (Eq. (Error)) */
    double err_col;      /* ||v .* (K^T u) - b||_2 of the returned state (Eq. (Error)) */
    double marg_err;     /* err_row + err_col */
    int iters;           /* iterations performed by this call (1 iteration = 2 half-steps) */
    int total_iters;     /* iterations since sk_init or the last sk_set_state */
} sk_result;

/* Geometry and sizes a plan settled on. */
typedef struct {
    int d;
    int64_t n, m;
    int N, n_os, m_w, p, precision, nearfield;
    double eps, r, eps_scaled;   /* eps_scaled = eps * scale^r: the kernel in torus coordinates */
    double center[3], scale, eps_B, eps_I;
    int n_subproblems_x, n_subproblems_y;   /* work items of the per-point spreading kernels (1-D; 3-D with m_w > 5) */
    int64_t device_bytes;        /* device memory the plan holds */
    int tensor_cores;            /* 1: interpolation runs on tensor cores (sk_set_kernels) */
    int fft_planes;              /* 1: the 3-D FFT runs as three launches with cluster planes (sk_set_fft) */
} sk_info;

/* Text for a status code (static storage, never NULL). */
const char* sk_error_string(int status);

/* Where the calling thread's last SK_ERR_CUDA / SK_ERR_NOMEM came from (source
 * line and the CUDA runtime's message); "" if none.  Thread-local storage. */
const char* sk_last_error(void);

/* Fill *prm with the defaults: N=64, sigma=2, m_w=4, p=8, eps_B=0.1, eps_I=0
 * (automatic), SK_FP32, automatic geometry.  Returns SK_ERR_ARG if prm is NULL. */
int sk_default_params(sk_nfft_params* prm);

/*
 * Build a plan for the problem (x, a) -> (y, b) with Gibbs kernel
 * exp(-||x-y||^r / eps) (Alg. 3 inputs: support nodes, probability vectors,
 * regularization).  Validates: d in {1,2,3}; n, m >= 1; eps > 0; r >= 1;
 * finite coordinates; weights >= 0 with |sum - 1| <= 1e-9 (SK_ERR_WEIGHTS).
 * Copies, scales and bin-sorts the points into plan-owned device buffers,
 * computes the coefficient table b_k / psi_hat(k)^2 on the device, and sets
 * u = 1_n, v = 1_m (the Set line of Alg. 1).  prm == NULL means defaults.
 * The caller may free x, a, y, b when this returns.  On failure *out is NULL.
 */
int sk_init(sk_plan** out, int d, int64_t n, const double* x, const double* a,
            int64_t m, const double* y, const double* b, double eps, double r,
            const sk_nfft_params* prm, void* stream);

/* Release everything the plan owns (NULL is a no-op). */
void sk_destroy(sk_plan* plan);

/* Choose how products are evaluated: SK_METHOD_NFFT (Eq. (fastsum), default)
 * or SK_METHOD_DIRECT (the plain O(n m) sums of Eqs. (matexp)/(matexpt), FP32
 * kernel values with FP64 accumulation across tiles). */
int sk_set_method(sk_plan* plan, int method);

/*
 * Choose the form of the iteration.  SK_DOMAIN_SCALING (default): Alg. 3, the
 * state is the scaling vectors u, v.  SK_DOMAIN_LOG: Alg. 4, the state is the
 * dual variables beta = eps (log u + 1/2), gamma = eps (log v + 1/2) of
 * Eq. (11), updated by its first-order condition
 *   beta_i = eps (log a_i - log t_i + 1/2),  t_i = sum_j k_ij exp(gamma_j / eps - 1/2)
 * (the update printed in Alg. 4 leaves out the + 1/2; with it the value is
 * the one of Alg. 3 at the same plan).  Each half-step forms its weights as
 * exp((gamma_j - max gamma) / eps - 1/2) <= e^(-1/2), so no weight leaves the
 * FP32 range however large the potentials grow (the scaling form's u, v leave
 * it for small eps); the kernel sums themselves keep their own range.  The
 * current state is converted (u = exp(beta / eps - 1/2) back, which can
 * overflow to inf); sk_get_state / sk_set_state / sk_solve's u_out, v_out
 * then carry beta, gamma.  sk_grad works in either domain.
 * Errors: SK_ERR_ARG for a NULL plan or an unknown domain.
 */
int sk_set_domain(sk_plan* plan, int domain);

/*
 * Choose how the interpolation step of Eq. (fastsum) (the NFFT: the grid at the
 * target points) runs.  SK_KERNELS_TENSOR (the default where supported: SK_FP32
 * plans with d = 3 and 2 <= m_w <= 5, or d = 2): per bin (4 x 4 x 8 cells in
 * 3-D, a strip of 33 - 2 m_w by 8 cells in 2-D) the contraction of the bin's
 * window box with the last-axis weights of 128 points at a time is one
 * tensor-core product (tcgen05, TF32 operands split into high and low parts,
 * three products, FP32 accumulation); the other axes' weights are applied per
 * point on the CUDA cores.  SK_KERNELS_SIMT: CUDA cores only.  Both meet the
 * FP32 accuracy of the plan; their sums differ by rounding.
 * Errors: SK_ERR_ARG for a NULL plan or an unknown value; SK_ERR_UNSUPPORTED
 * for SK_KERNELS_TENSOR on a plan it does not support (nothing changes).
 * A tensor-core wait that gives up (bounded) makes sk_solve / sk_solve_batch
 * return SK_ERR_TIMEOUT when they read results back.
 */
int sk_set_kernels(sk_plan* plan, int kernels);

/*
 * Choose how the FFT part of a 3-D product (Eq. (fastsum): the transform of the
 * spread grid, the multiply by the kernel's Fourier coefficients, the inverse
 * transform) is launched.  SK_FFT_PASSES: one launch per axis pass -- r2c along
 * z, forward y, the axis-0 pass with the multiply, inverse y, c2r along z.
 * SK_FFT_PLANES (the default where supported: SK_FP32 plans with d = 3 and
 * n_os = 64, 128 or 256): the two passes on each side of the axis-0 pass run
 * per x-plane in one launch, a thread-block cluster per plane exchanging the
 * plane through distributed shared memory -- three launches.  Both compute the
 * same transforms in the same order of operations per pencil.
 * Errors: SK_ERR_ARG for a NULL plan or an unknown value; SK_ERR_UNSUPPORTED
 * for SK_FFT_PLANES on a plan it does not support (nothing changes).
 */
int sk_set_fft(sk_plan* plan, int form);

/*
 * Autotuner for the interpolation kernels: times one product K v (three
 * repetitions after a warm-up, CUDA events on the plan's stream, the current
 * v as weights, output into plan scratch) with each kernel kind the plan
 * supports and keeps the faster, as sk_set_kernels would.  The plan's state
 * (u, v, iteration count) is unchanged.  chosen (host, optional) receives the
 * SK_KERNELS_* value kept.  Plans with one kind only, or in SK_METHOD_DIRECT,
 * keep their current choice.  Synchronizes the stream.
 * Errors: SK_ERR_ARG for a NULL plan; SK_ERR_CUDA.
 */
int sk_autotune(sk_plan* plan, int* chosen, void* stream);

/*
 * Test hook for the failure path of the tensor-core kernels.  With
 * SK_FAULT_TC_WAIT the plan's tensor-core interpolation skips its MMA group,
 * so the bounded wait for the group's completion (about a second) runs out:
 * the kernel sets its status bit, stops, releases its tensor memory and
 * returns, the GPU context stays usable, and sk_solve / sk_solve_batch return
 * SK_ERR_TIMEOUT when they read results back (the state of that solve is not
 * meaningful).  SK_FAULT_NONE restores normal operation.  Nothing faults or
 * hangs either way.
 * Errors: SK_ERR_ARG for a NULL plan or an unknown kind; SK_ERR_UNSUPPORTED
 * for SK_FAULT_TC_WAIT when the plan does not interpolate on tensor cores.
 */
int sk_inject_fault(sk_plan* plan, int kind);

/*
 * One kernel-vector product (Eqs. (matexp), (matexpt)):
 *   transpose = 0:  out[i] = sum_j K(x_i, y_j) in[j]   (in: m values, out: n values)
 *   transpose = 1:  out[j] = sum_i K(x_i, y_j) in[i]   (in: n values, out: m values)
 * Uses the plan's method.  Does not touch the plan's scaling vectors.
 */
int sk_kernel_apply(sk_plan* plan, int transpose, const double* in, double* out, void* stream);

/*
 * Run Sinkhorn iterations (Alg. 3) from the plan's current state.  One
 * iteration is the odd half-step u = a ./ (K v) followed by the even half-step
 * v = b ./ (K^T u).  tol <= 0: exactly max_iter iterations, no host sync
 * unless res/u_out/v_out are requested.  tol > 0: stop as soon as the
 * row residual ||u .* K v - a|| (the only nonzero term of Eq. (Error) after a
 * v-update) is <= tol, checking every check_every iterations (<= 0 means 10);
 * returns SK_ERR_NOT_CONVERGED if max_iter is reached first (state and outputs
 * are still written).  u_out (n), v_out (m) may be NULL.  res may be NULL; if
 * given, the final residuals and the value s are computed (one extra K v
 * product) and written.  Returns SK_ERR_UNDERFLOW if any kernel sum was <= 0 or
 * not finite.
 */
int sk_solve(sk_plan* plan, int max_iter, double tol, int check_every,
             double* u_out, double* v_out, sk_result* res, void* stream);

/*
 * Solve `count` independent plans together: one Sinkhorn iteration (Alg. 3)
 * of every plan is captured once into a single CUDA graph, the plans'
 * iterations as parallel branches (they share no memory), and the graph is
 * replayed max_iter times, so the kernels of small problems run side by side
 * on the GPU.  Each plan's state, iteration count and results then are those
 * of sk_solve(plan, max_iter, 0, ...).  results[count] (host) may be NULL;
 * if given, each plan's final residuals and value are computed as sk_solve
 * does.  Fixed iteration count (no tolerance).  All plans on one device,
 * none twice, none with stage timing on (else SK_ERR_ARG, nothing run).
 * Returns SK_ERR_UNDERFLOW if results were requested and a plan saw a
 * non-positive kernel sum.  Synchronizes `stream`.
 */
int sk_solve_batch(sk_plan* const* plans, int count, int max_iter, sk_result* results, void* stream);

/*
 * Gradient of the value with respect to the weights and the positions, at the
 * plan's current scaling vectors (Prop. "dual representation", Eqs. (13),
 * (27)): the gradient of the dual function Eq. (27) with u, v held fixed,
 *   grad_a[i] = eps (1/2 + log u_i)           (the dual variable beta_i)
 *   grad_b[j] = eps (1/2 + log v_j)           (gamma_j)
 *   grad_x[i] = sum_j pi_ij dC_ij/dx_i,  grad_y[j] = sum_i pi_ij dC_ij/dy_j,
 * with pi = diag(u) K diag(v) (Eq. (pi*)) and C_ij = ||x_i - y_j||^r.  After
 * Sinkhorn has converged (u, v maximize Eq. (14)) this is the gradient of the
 * value s returned by sk_solve (envelope theorem).  The weight gradient is
 * defined up to adding c to grad_a and -c to grad_b (sum a = sum b).
 * For r = 2 the position gradients use d + 1 fast summations per side:
 *   grad_x[i] = 2 u_i (x_i (K v)_i - (K (v y))_i), with the plan's method.
 * Layout: grad_a (n), grad_b (m), grad_x (n x d row-major), grad_y (m x d),
 * caller point order, host or device memory; any may be NULL (skipped).
 * Errors: SK_ERR_ARG for a NULL plan; SK_ERR_UNSUPPORTED if grad_x or grad_y
 * is requested and r != 2 (other r need the fast summation of a different
 * kernel); nothing is written then.  Synchronizes the plan's stream.
 */
int sk_grad(sk_plan* plan, double* grad_a, double* grad_b, double* grad_x, double* grad_y,
            void* stream);

/*
 * Sinkhorn divergence (Remark "Entropy bias and Sinkhorn divergence"; its
 * NFFT form after Alg. 3): sd = s(P, P~) - s(P, P) / 2 - s(P~, P~) / 2.
 * Builds and solves three plans with the arguments of sk_init and sk_solve
 * (the same params, max_iter and tol for each), then destroys them.
 * host_out[4] (host memory) receives sd, s(P, P~), s(P, P), s(P~, P~).
 * grad_a (n), grad_b (m), grad_x (n x d), grad_y (m x d), each optional
 * (NULL), host or device memory, caller order, receive the gradient of sd:
 * the sk_grad gradients of the three terms at their final states, the self
 * terms contributing both their source and target sides (every point of
 * s(P, P) is both).  Positions need r = 2 (else SK_ERR_UNSUPPORTED, nothing
 * written).  Returns the first error of sk_init / sk_solve / sk_grad
 * (nothing written then), SK_ERR_NOMEM if the gradient buffers cannot be
 * allocated, or SK_ERR_NOT_CONVERGED if a solve with tol > 0 reached
 * max_iter (values written), else SK_OK.  Synchronizes `stream`.
 */
int sk_divergence(int d, int64_t n, const double* x, const double* a, int64_t m, const double* y,
                  const double* b, double eps, double r, const sk_nfft_params* prm, int max_iter,
                  double tol, double* host_out, double* grad_a, double* grad_b, double* grad_x,
                  double* grad_y, void* stream);

/* Copy the scaling vectors out (caller order; either pointer may be NULL) and the
 * iteration count. Synchronizes. */
int sk_get_state(sk_plan* plan, double* u, double* v, int* iters);

/* Replace the scaling vectors (caller order).  u == NULL and v == NULL resets
 * both to ones.  iters sets the iteration counter. */
int sk_set_state(sk_plan* plan, const double* u, const double* v, int iters);

/* Geometry, sizes and memory of a plan. */
int sk_plan_info(const sk_plan* plan, sk_info* info);

/* ----------------------------------------------------- stage entry points --
 * These expose single steps of the fast summation for testing and profiling.
 */

/* The coefficients b_k, k in I_N, of the regularized kernel in torus
 * coordinates (Eq. (ansatz_NFFT)); out holds N^d doubles, entry
 * [(k_1+N/2) ... (k_d+N/2)] row-major.  Host or device pointer. */
int sk_fourier_coefficients(sk_plan* plan, double* out, void* stream);

/* Adjoint NFFT of weights w on cloud `set` (inner sum of Eq. (fastsum)):
 * fhat[k] = sum_j w_j exp(-2 pi i k.z_j), k in {-N/2..N/2}^d, z the torus
 * coordinates; fhat holds (N+1)^d complex values as interleaved (re, im)
 * doubles, row-major with index k_t + N/2.  Uses spreading, FFT and the
 * window deconvolution of the plan's precision. */
int sk_adjoint_nfft(sk_plan* plan, int set, const double* w, double* fhat, void* stream);

/* NFFT on cloud `set` (outer sum of Eq. (fastsum)) of a Hermitian coefficient
 * array (fhat[-k] = conj(fhat[k]); layout as in sk_adjoint_nfft):
 * f_j = Re sum_{k in I_N} fhat[k] exp(2 pi i k.z_j), computed as
 * sum_{k in {-N/2..N/2}^d} c_k fhat[k] exp(2 pi i k.z_j) with
 * c_k = (1[k in I_N] + 1[-k in I_N]) / 2.  The kernel products use the same
 * real part of the paper's sum over I_N. */
int sk_nfft(sk_plan* plan, int set, const double* fhat, double* f, void* stream);

/* ------------------------------------------------ sharded products ---------
 * One product split over several plans (for example one per GPU) by the
 * linearity of the inner sum of Eq. (fastsum): every plan holds a shard of the
 * sources and of the targets, all plans share one torus geometry (params with
 * user_geometry = 1 and the same center, scale, N, sigma, m_w, p, eps_B, eps,
 * r), each computes the spectrum of its own sources, the spectra are summed
 * across the plans (an all-reduce), and each plan evaluates the product at its
 * own targets from the sum:
 *   (K w)_i = Re sum_{k in I_N} b_k (sum over shards of spec_k) exp(2 pi i k.z_i).
 * The near-field correction of kernels that are not smooth at 0 (r not an
 * even integer) is not part of this split; such plans are refused
 * (SK_ERR_UNSUPPORTED).
 *
 * sk_spectrum: the adjoint NFFT (inner sum of Eq. (fastsum)) of weights w
 * (caller order) on cloud `set`, spec[k] = sum_j w_j exp(-2 pi i k.z_j) for
 * k in {-N/2..N/2}^d, as in sk_adjoint_nfft: (N+1)^d complex values,
 * interleaved (re, im) doubles, row-major with index k_t + N/2.
 * sk_apply_spectrum: out (caller order, n or m values) = the outer sum above
 * at the points of cloud `set`, for a Hermitian spec (spec[-k] = conj
 * spec[k]; every sum of sk_spectrum outputs is one).  Both: host or device
 * pointers; SK_ERR_ARG for NULL arguments or an unknown set.
 */
int sk_spectrum(sk_plan* plan, int set, const double* w, double* spec, void* stream);
int sk_apply_spectrum(sk_plan* plan, int set, const double* spec, double* out, void* stream);

/* Per-stage device times.  enable = 1 turns on CUDA-event timing of every
 * stage on the plan's stream (and disables graph replay); enable = 0 turns it
 * off.  ms_out (may be NULL) receives SK_NSTAGES accumulated milliseconds,
 * counts_out (may be NULL) the number of launches timed per stage; both are
 * reset after reading. */
enum { SK_STAGE_SPREAD = 0, SK_STAGE_FFT = 1, SK_STAGE_INTERP = 2, SK_STAGE_OTHER = 3,
       SK_STAGE_DIRECT = 4, SK_STAGE_NEAR = 5, SK_NSTAGES = 6 };
int sk_stage_times(sk_plan* plan, int enable, double* ms_out, int64_t* counts_out);

/* Number of kernels this plan has launched (graph replays count every kernel node). */
int64_t sk_launch_count(const sk_plan* plan);

/* -------------------------------------------------------- measurement ------
 * FP32 arithmetic rate of the current device, measured: every thread of a grid
 * that fills every SM runs 8 independent FMA chains for `iters` steps
 * (packed = 0: scalar FP32 FMAs; packed = 1: packed FMAs on float2 pairs, two
 * per instruction), timed with CUDA events on `stream` after one untimed
 * launch.  *tflops receives 2 flops x FMAs / time in TFLOP/s; *sms (may be
 * NULL) the device's SM count.  It is the denominator of the roofline of the
 * kernels bound by FP32 arithmetic.  Synchronizes `stream`.
 * Errors: SK_ERR_ARG (tflops NULL, iters < 1, packed not 0 or 1); SK_ERR_CUDA.
 */
int sk_fp32_peak(int packed, int iters, double* tflops, int* sms, void* stream);

/* ---------------------------------------------- no-allocation entry point --
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory (code running under a framework whose memory pool
 * already owns the GPU's memory, services that must not allocate after
 * start-up because cudaMalloc can synchronize the device, callers that hand
 * the library only buffers they own).  It needs no plan and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Computes, by direct FP32 kernel evaluation with FP64 accumulation across
 * 1024-source tiles (the direct method of sk_set_method),
 *   t_out[i]     = sum_j v_j exp(-||x_i - y_j||^r / eps)
 *   stats_out[0] = sum_i (u_i t_out[i] - a_i)^2
 *   stats_out[1] = sum_i u_i t_out[i]
 * x: n-by-d, y: m-by-d row-major; u, a: n; v: m; t_out: n; stats_out: 2.
 * Every pointer must be device memory of the current device (or managed
 * memory), else SK_ERR_ARG.  t_out and stats_out may not overlap an input or
 * each other (other blocks still read the inputs while t_out is written),
 * else SK_ERR_ARG.  The call is asynchronous on `stream`.
 *
 * Scratch: the per-block partial sums live in one file-scope device array of
 * 64 KB + 256 B, present on every GPU that loads the library until the process
 * exits.  It bounds n <= 2,097,152 (4096 blocks of 512 targets); larger n
 * returns SK_ERR_TOO_LARGE before any GPU work.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and keeps it,
 * so make the first call on each device before any stream capture, and do not
 * reset the device after it (the array may then move).  All calls share the
 * array: calls whose kernels overlap on the GPU (concurrent streams or host
 * threads on one device) race and return wrong sums, so serialize them. */
int sk_direct_residual_noalloc(int d, int64_t n, const double* x, const double* u, const double* a,
                               int64_t m, const double* y, const double* v, double eps, double r,
                               double* t_out, double* stats_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SK_H */
