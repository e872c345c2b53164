// C ABI of the library (include/sk.h): plan construction, the two half-steps
// of Sinkhorn's iteration (Alg. 3) as sequences of device kernels, CUDA-graph
// replay of an iteration, and the stage entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sk_internal.cuh"
#include "sk_plan_kernels.cuh"

using namespace sk;

struct sk_plan {
    int d = 0;
    int64_t n = 0, m = 0;
    double eps = 0, r = 0;
    sk_nfft_params prm{};
    int precision = SK_FP32;
    int method = SK_METHOD_NFFT;
    int domain = SK_DOMAIN_SCALING;
    int near_sub = 2;           // near-field cells per eps_I (2, or 4 for dense clouds)
    bool tc_ok = false;         // the tensor-core (tcgen05) interpolation supports this plan
    bool tc = false;            // ... and is selected
    int inject = 0;             // SK_FAULT_* test hook (sk_inject_fault)
    double* shift = nullptr;    // log domain: max of the Y ([0]) and X ([1]) dual variables
    int N = 0, h = 0, n_os = 0, log2n = 0, W = 0, B[3] = {1, 1, 1}, nb[3] = {1, 1, 1}, nbins = 0, bvol = 1;
    int64_t nkeys = 0;
    double beta = 0, knorm = 0;
    double center[3] = {0, 0, 0}, scale = 1, eps_s = 0;
    int nearfield = 0;
    KernelParams kp{};
    WindowPoly wp{};
    Cloud X, Y;
    FftPlan fft;
    size_t grid_elems = 0;
    double* bk = nullptr;       // N^d FP64
    double* spec_tmp = nullptr; // (N+1)^d complex FP64 scratch of sk_apply_spectrum (allocated on first use)
    double* psihat = nullptr;   // 2h+1 FP64
    double* partial = nullptr;  // reduction partials
    int partial_blocks = 0;
    unsigned* ticket = nullptr;
    double* stats = nullptr;    // slots of 3 doubles
    int* status = nullptr;
    double* pinned = nullptr;   // host pinned readback area
    double Ha = 0, Hb = 0;      // entropies of a and b
    cudaStream_t ps = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_kernels = 0;
    bool timing = false;
    // stage timing: pairs of events around each stage, either recorded as
    // the stages are launched (eager) or captured into the timed graph
    struct EventPool {
        std::vector<cudaEvent_t> ev;   // pairs
        std::vector<int> stage;
        size_t used = 0;
    };
    EventPool eager, graph_ev;
    EventPool* pool = &eager;
    cudaGraphExec_t gexec_timed = nullptr;   // one iteration with its stage events
    int64_t graph_kernels_timed = 0;
    double stage_ms[SK_NSTAGES] = {0};
    int64_t stage_cnt[SK_NSTAGES] = {0};
    int iters = 0;
    int64_t launches = 0;
    std::vector<void*> allocs;
    int64_t bytes = 0;
    int device = 0;
};

namespace {

enum Slot { SLOT_ROW = 0, SLOT_COL = 1, SLOT_RES_ROW = 2, SLOT_RES_COL = 3, SLOT_LOG = 4, NSLOTS = 6 };

struct Fail {
    int code;
};

thread_local char g_last_error[256] = "";

[[noreturn]] void cuda_fail(cudaError_t e, int line) {
    std::snprintf(g_last_error, sizeof(g_last_error), "sk_api.cu:%d: %s", line, cudaGetErrorString(e));
    cudaGetLastError();
    throw Fail{e == cudaErrorMemoryAllocation ? SK_ERR_NOMEM : SK_ERR_CUDA};
}

#define CK(x)                                     \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) cuda_fail(e_, __LINE__); \
    } while (0)

inline unsigned nblk(int64_t n, int t = 256) { return unsigned((n + t - 1) / t); }

void* dalloc(sk_plan* P, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{SK_ERR_NOMEM};
    }
    P->allocs.push_back(p);
    P->bytes += int64_t(bytes);
    return p;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of a caller array of `count` doubles: the pointer itself if it is
// device memory, else `staging` after an async host-to-device copy.
const double* device_view(sk_plan* P, const double* p, int64_t count, double* staging) {
    if (is_device_ptr(p)) return p;
    CK(cudaMemcpyAsync(staging, p, size_t(count) * sizeof(double), cudaMemcpyHostToDevice, P->ps));
    return staging;
}

void enter(sk_plan* P, void* stream) {
    CK(cudaSetDevice(P->device));
    CK(cudaEventRecord(P->ev_in, static_cast<cudaStream_t>(stream)));
    CK(cudaStreamWaitEvent(P->ps, P->ev_in, 0));
}

void leave(sk_plan* P, void* stream) {
    CK(cudaEventRecord(P->ev_out, P->ps));
    CK(cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), P->ev_out, 0));
}

// ------------------------------------------------------------ stage timing
// Inside a capture the stage events become event-record nodes of the graph
// (external records), so they are recorded, with timestamps, on every replay.
unsigned stage_record_flags(const sk_plan* P) {
    return P->pool == &P->graph_ev ? cudaEventRecordExternal : cudaEventRecordDefault;
}

int stage_begin(sk_plan* P, int stage) {
    if (!P->timing) return -1;
    sk_plan::EventPool& q = *P->pool;
    if (q.used * 2 + 2 > q.ev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            q.ev.push_back(e);
        }
        q.stage.resize(q.ev.size() / 2);
    }
    const int idx = int(q.used++);
    q.stage[idx] = stage;
    CK(cudaEventRecordWithFlags(q.ev[2 * idx], P->ps, stage_record_flags(P)));
    return idx;
}

void stage_end(sk_plan* P, int idx) {
    if (idx < 0) return;
    CK(cudaEventRecordWithFlags(P->pool->ev[2 * idx + 1], P->ps, stage_record_flags(P)));
}

// Adds the recorded stage intervals of a pool to the totals.
void pool_resolve(sk_plan* P, sk_plan::EventPool& q, bool keep) {
    if (q.used == 0) return;
    CK(cudaStreamSynchronize(P->ps));
    for (size_t k = 0; k < q.used; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, q.ev[2 * k], q.ev[2 * k + 1]));
        P->stage_ms[q.stage[k]] += ms;
        P->stage_cnt[q.stage[k]] += 1;
    }
    if (!keep) q.used = 0;
}

void stage_resolve(sk_plan* P) { pool_resolve(P, P->eager, false); }

// ------------------------------------------------------------ host math
// Derivatives 0..p-1 of K(rho) = exp(g(rho)), g = -rho^r / eps, at rho0, from
// f^(k+1) = sum_j binom(k, j) g^(j+1) f^(k-j).
void kernel_derivatives(double rho0, double eps, double r, int p, double* f) {
    double g[kMaxP + 1];
    g[0] = -std::pow(rho0, r) / eps;
    for (int j = 1; j <= p; ++j) {
        double fall = 1.0;
        for (int q = 0; q < j; ++q) fall *= (r - q);
        g[j] = -fall * std::pow(rho0, r - j) / eps;
    }
    f[0] = std::exp(g[0]);
    for (int k = 0; k + 1 < p; ++k) {
        double s = 0.0, binom = 1.0;
        for (int j = 0; j <= k; ++j) {
            s += binom * g[j + 1] * f[k - j];
            binom = binom * double(k - j) / double(j + 1);
        }
        f[k + 1] = s;
    }
}

// Solve A x = b (size k <= 2 kMaxP) by Gaussian elimination with partial pivoting.
bool solve_dense(int k, double* A, double* b) {
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int r = c + 1; r < k; ++r)
            if (std::fabs(A[r * k + c]) > std::fabs(A[piv * k + c])) piv = r;
        if (A[piv * k + c] == 0.0) return false;
        if (piv != c) {
            for (int j = 0; j < k; ++j) std::swap(A[c * k + j], A[piv * k + j]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < k; ++r) {
            const double f = A[r * k + c] / A[c * k + c];
            for (int j = c; j < k; ++j) A[r * k + j] -= f * A[c * k + j];
            b[r] -= f * b[c];
        }
    }
    for (int c = k - 1; c >= 0; --c) {
        double s = b[c];
        for (int j = c + 1; j < k; ++j) s -= A[c * k + j] * b[j];
        b[c] = s / A[c * k + c];
    }
    return true;
}

double falling(int e, int j) {  // e! / (e - j)!
    double v = 1.0;
    for (int q = 0; q < j; ++q) v *= double(e - q);
    return v;
}

// Two-point Taylor boundary polynomial in tau = (rho - L)/(1/2 - L): value and
// derivatives 0..p-1 of K at rho = L, derivatives 1..p-1 zero at rho = 1/2.
bool boundary_coefficients(KernelParams& kp) {
    const int p = kp.p;
    const double delta = 0.5 - kp.L;
    double f[kMaxP];
    kernel_derivatives(kp.L, kp.eps_s, kp.r, p, f);
    double fact = 1.0;
    for (int j = 0; j < p; ++j) {
        if (j > 0) fact *= j;
        kp.kb[j] = f[j] * std::pow(delta, j) / fact;
    }
    const int q = p - 1;
    if (q == 0) return true;
    double A[kMaxP * kMaxP], rhs[kMaxP];
    for (int row = 0; row < q; ++row) {
        const int order = row + 1;
        double s = 0.0;
        for (int e = order; e < p; ++e) s += kp.kb[e] * falling(e, order);
        rhs[row] = -s;
        for (int c = 0; c < q; ++c) A[row * q + c] = falling(p + c, order);
    }
    if (!solve_dense(q, A, rhs)) return false;
    for (int c = 0; c < q; ++c) kp.kb[p + c] = rhs[c];
    return true;
}

// Near-field polynomial sum_q ki[q] (rho/eps_I)^(2q) matching derivatives
// 0..p-1 of K at rho = eps_I.
bool nearfield_coefficients(KernelParams& kp) {
    const int p = kp.p;
    double f[kMaxP];
    kernel_derivatives(kp.eps_I, kp.eps_s, kp.r, p, f);
    double A[kMaxP * kMaxP], rhs[kMaxP];
    for (int j = 0; j < p; ++j) {
        rhs[j] = f[j] * std::pow(kp.eps_I, j);
        for (int q = 0; q < p; ++q) A[j * p + q] = (2 * q >= j) ? falling(2 * q, j) : 0.0;
    }
    if (!solve_dense(p, A, rhs)) return false;
    for (int q = 0; q < p; ++q) kp.ki[q] = rhs[q];
    return true;
}

bool even_integer(double r) { return std::floor(r) == r && (int64_t(r) % 2 == 0); }

// Kaiser-Bessel window in grid units, normalized to 1 at 0 (host, FP64).
double kb_host(double x, int m, double beta, double knorm) {
    const double z2 = double(m) * m - x * x;
    if (z2 < 0.0) return 0.0;
    if (z2 == 0.0) return beta * knorm;
    const double z = std::sqrt(z2);
    return std::sinh(beta * z) / z * knorm;
}

// Chebyshev interpolant of degree `deg` of f on [-1, 1], in monomials of s.
template <typename F>
void chebyshev_monomials(F f, int deg, double* c) {
    const int np = deg + 1;
    double vals[32], a[32];
    for (int i = 0; i < np; ++i) vals[i] = f(std::cos(M_PI * (i + 0.5) / np));
    for (int j = 0; j < np; ++j) {
        double acc = 0.0;
        for (int i = 0; i < np; ++i) acc += vals[i] * std::cos(M_PI * j * (i + 0.5) / np);
        a[j] = (j == 0 ? 1.0 : 2.0) * acc / np;
    }
    // T_j in monomials: T_0 = 1, T_1 = s, T_{j+1} = 2 s T_j - T_{j-1}
    double tm1[32] = {0}, t0[32] = {0}, t1[32] = {0};
    for (int i = 0; i <= deg; ++i) c[i] = 0.0;
    t0[0] = 1.0;
    for (int i = 0; i <= deg; ++i) c[i] += a[0] * t0[i];
    if (deg >= 1) {
        t1[1] = 1.0;
        for (int i = 0; i <= deg; ++i) c[i] += a[1] * t1[i];
    }
    for (int j = 2; j <= deg; ++j) {
        double tn[32] = {0};
        for (int i = 0; i <= deg; ++i) tn[i] = (i > 0 ? 2.0 * t1[i - 1] : 0.0) - t0[i];
        for (int i = 0; i <= deg; ++i) c[i] += a[j] * tn[i];
        for (int i = 0; i <= deg; ++i) { tm1[i] = t0[i]; t0[i] = t1[i]; t1[i] = tn[i]; }
    }
}

// Piecewise-polynomial window: tap k of a point with fractional offset frac is
// psi(frac + m - 1 - k), approximated in s = 2 frac - 1 (see WindowPoly).
void window_polynomials(int m, double beta, double knorm, WindowPoly& wp) {
    std::memset(&wp, 0, sizeof(wp));
    for (int k = 0; k < 2 * m; ++k) {
        auto f = [&](double s) { return kb_host(0.5 * (s + 1.0) + m - 1 - k, m, beta, knorm); };
        double c[32];
        chebyshev_monomials(f, kPolyDeg32, c);
        for (int i = 0; i <= kPolyDeg32; ++i) wp.c32[k][i] = float(c[i]);
        chebyshev_monomials(f, kPolyDeg64, c);
        for (int i = 0; i <= kPolyDeg64; ++i) wp.c64[k][i] = c[i];
    }
}

// ------------------------------------------------------------ reductions
// Reduce a partial table of `nf` fields with the given ops to host doubles.
void combine_to_host(sk_plan* P, int nblocks, int nf, const int* ops, double* host) {
    double* out = P->stats + 3 * NSLOTS;   // scratch after the slots
    k_combine<<<1, 32 * nf, 0, P->ps>>>(P->partial, nblocks, nf, ops[0], nf > 1 ? ops[1] : 0, nf > 2 ? ops[2] : 0,
                                   nf > 3 ? ops[3] : 0, nf > 4 ? ops[4] : 0, nf > 5 ? ops[5] : 0,
                                   nf > 6 ? ops[6] : 0, out);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(P->pinned, out, size_t(nf) * sizeof(double), cudaMemcpyDeviceToHost, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    std::memcpy(host, P->pinned, size_t(nf) * sizeof(double));
}

constexpr int kRedBlocks = 256;

// ------------------------------------------------------------ point clouds
// Exclusive scan into out[0..n] through the multi-block scan, with its scratch
// taken from the stream-ordered pool.
void scan_ints(sk_plan* P, const int* in, int* out, int n) {
    int* scratch = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&scratch), size_t(scan_scratch_ints(n)) * sizeof(int), P->ps));
    launch_scan_exclusive(in, out, n, scratch, P->ps);
    CK(cudaGetLastError());
    CK(cudaFreeAsync(scratch, P->ps));
}

int read_int(sk_plan* P, const int* dev) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, dev, sizeof(int), cudaMemcpyDeviceToHost, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    return v;
}

// Runs of at most `run` consecutive points of one bin (bin CSR `bs`), most
// points first, so the workers that take the last tasks take short ones;
// uploaded as (bin, first point, end point) triples.
int* upload_runs(sk_plan* P, const std::vector<int>& bs, int run, int& count) {
    std::vector<int> tk;
    for (int b = 0; b + 1 < int(bs.size()); ++b)
        for (int s0 = bs[b]; s0 < bs[b + 1]; s0 += run) {
            tk.push_back(b);
            tk.push_back(s0);
            tk.push_back(std::min(bs[b + 1], s0 + run));
        }
    const int nt = int(tk.size() / 3);
    std::vector<int> order(nt);
    for (int i = 0; i < nt; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
        return tk[3 * p + 2] - tk[3 * p + 1] > tk[3 * q + 2] - tk[3 * q + 1];
    });
    std::vector<int> sorted(tk.size());
    for (int i = 0; i < nt; ++i)
        for (int k = 0; k < 3; ++k) sorted[3 * i + k] = tk[3 * order[i] + k];
    count = nt;
    int* d = static_cast<int*>(dalloc(P, size_t(3 * std::max(nt, 1)) * sizeof(int)));
    if (nt > 0) CK(cudaMemcpyAsync(d, sorted.data(), sorted.size() * sizeof(int), cudaMemcpyHostToDevice, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    return d;
}

// The column queue of the CUDA-core 3-D interpolation for one cloud: every
// non-empty (bin, column) pair, most points first, so the warps that take the
// last entries take short ones.
void build_column_queue(sk_plan* P, Cloud& c) {
    const int ncol = P->B[0] * P->B[1];
    const int64_t npairs = int64_t(P->nbins) * ncol;
    int* cnt_d = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&cnt_d), size_t(npairs) * sizeof(int), P->ps));
    k_col_counts<<<unsigned((npairs + 255) / 256), 256, 0, P->ps>>>(c.key_start, P->nbins, P->bvol, ncol, P->B[2],
                                                                    cnt_d);
    CK(cudaGetLastError());
    std::vector<int> cnt(static_cast<size_t>(npairs));
    CK(cudaMemcpyAsync(cnt.data(), cnt_d, cnt.size() * sizeof(int), cudaMemcpyDeviceToHost, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    CK(cudaFreeAsync(cnt_d, P->ps));
    std::vector<int> cols;
    for (int64_t i = 0; i < npairs; ++i)
        if (cnt[i] > 0) cols.push_back(int(i));
    std::stable_sort(cols.begin(), cols.end(), [&](int p, int q) { return cnt[p] > cnt[q]; });
    c.ncols = int(cols.size());
    c.cols = static_cast<int*>(dalloc(P, size_t(std::max(c.ncols, 1)) * sizeof(int)));
    if (c.ncols > 0)
        CK(cudaMemcpyAsync(c.cols, cols.data(), cols.size() * sizeof(int), cudaMemcpyHostToDevice, P->ps));
    CK(cudaStreamSynchronize(P->ps));
}

// Both clouds' column queues and the reduction partials the CUDA-core 3-D
// interpolation needs, for a plan that turns to it after sk_init (a no-op when
// they exist or the plan has no column kernels).  Not during a capture: the
// callers are sk_set_kernels and sk_autotune.
template <typename T>
void ensure_column_queues(sk_plan* P) {
    if (!column_kernels(P->d, P->W) || P->X.cols) return;
    build_column_queue(P, P->X);
    build_column_queue(P, P->Y);
    const int need = interp3_blocks<T>(P->W, std::max(P->X.ncols, P->Y.ncols));
    if (need > P->partial_blocks) {
        P->partial_blocks = need;
        P->partial = static_cast<double*>(dalloc(P, size_t(need) * 8 * sizeof(double)));
    }
}

template <typename T>
void build_cloud(sk_plan* P, Cloud& c, const double* xdev, const double* wdev, int64_t n) {
    c.n = n;
    // the cloud's arrays in one allocation (each start 256-byte aligned): one
    // cudaMalloc instead of a dozen, which is most of a plan build's host time
    const size_t sizes[11] = {size_t(n) * sizeof(T), size_t(n) * sizeof(T), size_t(n) * sizeof(T),
                              size_t(n) * sizeof(int), size_t(n) * sizeof(double), size_t(n) * sizeof(double),
                              size_t(n) * sizeof(double), size_t(n) * sizeof(double), size_t(n) * sizeof(double),
                              size_t(P->nkeys + 1) * sizeof(int), size_t(P->nbins + 1) * sizeof(int)};
    size_t off[11], arena = 0;
    for (int k = 0; k < 11; ++k) {
        off[k] = arena;
        arena += (k < 3 && k >= P->d) ? 0 : (sizes[k] + 255) / 256 * 256;
    }
    unsigned char* base = static_cast<unsigned char*>(dalloc(P, arena));
    for (int t = 0; t < P->d; ++t) c.coord[t] = base + off[t];
    c.perm = reinterpret_cast<int*>(base + off[3]);
    c.marg = reinterpret_cast<double*>(base + off[4]);
    c.scal = reinterpret_cast<double*>(base + off[5]);
    c.t = reinterpret_cast<double*>(base + off[6]);
    c.work = reinterpret_cast<double*>(base + off[7]);
    c.stage = reinterpret_cast<double*>(base + off[8]);
    c.key_start = reinterpret_cast<int*>(base + off[9]);
    c.bin_start = reinterpret_cast<int*>(base + off[10]);

    // temporaries
    T* uo[3] = {nullptr, nullptr, nullptr};
    T* us[3] = {nullptr, nullptr, nullptr};
    void* tmp_u = nullptr;
    int *key = nullptr, *count = nullptr, *cursor = nullptr, *nsub = nullptr, *suboff = nullptr;
    CK(cudaMallocAsync(&tmp_u, size_t(n) * 3 * sizeof(T), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&key), size_t(n) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&count), size_t(P->nkeys) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&cursor), size_t(P->nkeys) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&nsub), size_t(P->nbins) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&suboff), size_t(P->nbins + 1) * sizeof(int), P->ps));
    for (int t = 0; t < 3; ++t) {
        uo[t] = static_cast<T*>(tmp_u) + size_t(t) * n;
        us[t] = t < P->d ? static_cast<T*>(c.coord[t]) : uo[t];
    }
    CK(cudaMemsetAsync(count, 0, size_t(P->nkeys) * sizeof(int), P->ps));
    CK(cudaMemsetAsync(cursor, 0, size_t(P->nkeys) * sizeof(int), P->ps));
    launch_prepare_points<T>(xdev, n, P->d, P->center, P->scale, P->n_os, P->B, P->nb, P->prm.m_w, uo, key, count,
                             P->status, P->ps);
    CK(cudaGetLastError());
    scan_ints(P, count, c.key_start, int(P->nkeys));
    k_scatter_perm<<<nblk(n), 256, 0, P->ps>>>(key, n, c.key_start, cursor, c.perm);
    CK(cudaGetLastError());
    launch_gather_points<T>(c.perm, n, P->d, uo, us, P->ps);
    CK(cudaGetLastError());
    k_gather<<<nblk(n), 256, 0, P->ps>>>(wdev, c.perm, n, c.marg);
    CK(cudaGetLastError());
    k_bin_starts<<<nblk(P->nbins + 1), 256, 0, P->ps>>>(c.key_start, P->nbins, P->bvol, c.bin_start);
    CK(cudaGetLastError());

    // subproblems of the per-point spreading kernel
    k_count_subs<<<nblk(P->nbins), 256, 0, P->ps>>>(c.bin_start, P->nbins, kSpreadMaxPts, nsub);
    CK(cudaGetLastError());
    scan_ints(P, nsub, suboff, P->nbins);
    const int total = read_int(P, suboff + P->nbins);
    c.nsub = total;
    c.sub_start = static_cast<int*>(dalloc(P, size_t(std::max(total, 1)) * sizeof(int)));
    c.sub_count = static_cast<int*>(dalloc(P, size_t(std::max(total, 1)) * sizeof(int)));
    c.sub_bin = static_cast<int*>(dalloc(P, size_t(std::max(total, 1)) * sizeof(int)));
    k_fill_subs<<<nblk(P->nbins), 256, 0, P->ps>>>(c.bin_start, suboff, P->nbins, kSpreadMaxPts, c.sub_start,
                                                  c.sub_count, c.sub_bin);
    CK(cudaGetLastError());

    // column tasks of the column spreading kernels (3-D: the B0 x B1 cell
    // columns of a bin; 2-D: the B0 x-cells of a strip bin)
    if (column_kernels(P->d, P->W) || P->d == 2) {
        const int ncol = P->d == 3 ? P->B[0] * P->B[1] : P->B[0];
        k_count_tasks<<<nblk(P->nbins), 256, 0, P->ps>>>(c.bin_start, P->nbins,
                                                         P->d == 3 ? kTaskMaxPts : kTaskMaxPts2, ncol, nsub);
        CK(cudaGetLastError());
        scan_ints(P, nsub, suboff, P->nbins);
        c.ntasks = read_int(P, suboff + P->nbins);
        c.tasks = static_cast<int*>(dalloc(P, size_t(3 * std::max(c.ntasks, 1)) * sizeof(int)));
        k_fill_tasks<<<nblk(P->nbins), 256, 0, P->ps>>>(suboff, P->nbins, ncol, c.tasks);
        CK(cudaGetLastError());
        // heaviest tasks first (longest-processing-time order), so the blocks
        // that start last are the short ones
        std::vector<int> tk(size_t(3) * c.ntasks), bs(size_t(P->nbins) + 1);
        CK(cudaMemcpyAsync(tk.data(), c.tasks, tk.size() * sizeof(int), cudaMemcpyDeviceToHost, P->ps));
        CK(cudaMemcpyAsync(bs.data(), c.bin_start, bs.size() * sizeof(int), cudaMemcpyDeviceToHost, P->ps));
        CK(cudaStreamSynchronize(P->ps));
        std::vector<int> order(c.ntasks);
        std::vector<double> load(c.ntasks);
        for (int i = 0; i < c.ntasks; ++i) {
            order[i] = i;
            const int b = tk[3 * i];
            load[i] = double(bs[b + 1] - bs[b]) * (tk[3 * i + 2] - tk[3 * i + 1]) / ncol;
        }
        std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return load[p] > load[q]; });
        std::vector<int> sorted(tk.size());
        for (int i = 0; i < c.ntasks; ++i)
            for (int k = 0; k < 3; ++k) sorted[3 * i + k] = tk[3 * order[i] + k];
        CK(cudaMemcpyAsync(c.tasks, sorted.data(), sorted.size() * sizeof(int), cudaMemcpyHostToDevice, P->ps));
        CK(cudaStreamSynchronize(P->ps));
    }
    // the CUDA-core interpolation's column queue, only where that kernel is
    // the plan's choice from the start (it is built on first use otherwise)
    if (column_kernels(P->d, P->W) && !P->tc) build_column_queue(P, c);
    // Run tasks: 2-D strips (one warp per task): at most kStripMaxPts points,
    // and small clouds take shorter runs (down to one batch of 32) so that
    // their tasks still reach every SM; tensor-core interpolation (one block
    // per task): at most kTcRunPts, whole tiles of 128.
    if (P->d == 2 || P->tc_ok) {
        int dev = 0, sms = 1;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        std::vector<int> bs(size_t(P->nbins) + 1);
        CK(cudaMemcpyAsync(bs.data(), c.bin_start, bs.size() * sizeof(int), cudaMemcpyDeviceToHost, P->ps));
        CK(cudaStreamSynchronize(P->ps));
        if (P->d == 2) {
            const int64_t per_warp = (n + int64_t(sms) * 8 - 1) / (int64_t(sms) * 8);
            const int run = int(std::min<int64_t>(kStripMaxPts, std::max<int64_t>(32, (per_warp + 31) / 32 * 32)));
            c.stasks = upload_runs(P, bs, run, c.nstasks);
        }
        if (P->tc_ok) c.ttasks = upload_runs(P, bs, kTcRunPts, c.nttasks);
    }
    k_fill<<<nblk(n), 256, 0, P->ps>>>(c.scal, n, 1.0);
    CK(cudaGetLastError());
    CK(cudaFreeAsync(tmp_u, P->ps));
    CK(cudaFreeAsync(key, P->ps));
    CK(cudaFreeAsync(count, P->ps));
    CK(cudaFreeAsync(cursor, P->ps));
    CK(cudaFreeAsync(nsub, P->ps));
    CK(cudaFreeAsync(suboff, P->ps));
}

// Near-field cell list of one cloud: cubic cells of side 1/nc >= eps_I / kNearSub
// over the unit torus (so all pairs closer than eps_I lie within kNearSub
// cells of a point's own along every axis; the kernel prunes the cells that
// cannot hold such a pair), the cloud in that order, and its non-empty cells.
int near_cells_per_dim(const sk_plan* P) { return std::max(1, int(std::floor(P->near_sub / P->prm.eps_I))); }

// Non-empty near-field cells of cloud c at the plan's current cell size.
template <typename T>
int near_occupied_cells(sk_plan* P, Cloud& c) {
    const int nc = near_cells_per_dim(P);
    int ncells = 1;
    for (int t = 0; t < P->d; ++t) ncells *= nc;
    int *key = nullptr, *count = nullptr, *nonempty = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&key), size_t(c.n) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&count), size_t(ncells) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&nonempty), sizeof(int), P->ps));
    CK(cudaMemsetAsync(count, 0, size_t(ncells) * sizeof(int), P->ps));
    CK(cudaMemsetAsync(nonempty, 0, sizeof(int), P->ps));
    launch_near_keys<T>(c.coord, c.n, P->d, double(nc) / P->n_os, nc, key, count, P->ps);
    CK(cudaGetLastError());
    launch_count_nonempty(count, ncells, nonempty, P->ps);
    CK(cudaGetLastError());
    const int occ = read_int(P, nonempty);
    CK(cudaFreeAsync(key, P->ps));
    CK(cudaFreeAsync(count, P->ps));
    CK(cudaFreeAsync(nonempty, P->ps));
    return occ;
}

// Cells per eps_I of the near-field lists: 4 (finer cells, fewer pairs outside
// eps_I examined) when the cells at 2 would hold 256 points or more on average,
// else 2 (a block's target slots are filled in units of 32).
template <typename T>
void choose_near_sub(sk_plan* P) {
    P->near_sub = 2;
    const int occ = near_occupied_cells<T>(P, P->X) + near_occupied_cells<T>(P, P->Y);
    if (occ > 0 && double(P->X.n + P->Y.n) / occ >= 256.0) P->near_sub = 4;
}

template <typename T>
void build_near(sk_plan* P, Cloud& c) {
    const int nc = near_cells_per_dim(P);
    int ncells = 1;
    for (int t = 0; t < P->d; ++t) ncells *= nc;
    const int64_t n = c.n;
    c.nf_start = static_cast<int*>(dalloc(P, size_t(ncells + 1) * sizeof(int)));
    c.nf_idx = static_cast<int*>(dalloc(P, size_t(n) * sizeof(int)));
    for (int t = 0; t < P->d; ++t) c.nf_coord[t] = dalloc(P, size_t(n) * sizeof(T));
    c.nf_tasks = static_cast<int*>(dalloc(P, size_t(ncells) * sizeof(int)));
    c.nf_corr = static_cast<double*>(dalloc(P, size_t(n) * sizeof(double)));
    int *key = nullptr, *count = nullptr, *cursor = nullptr, *ntask = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&key), size_t(n) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&count), size_t(ncells) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&cursor), size_t(ncells) * sizeof(int), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&ntask), sizeof(int), P->ps));
    CK(cudaMemsetAsync(count, 0, size_t(ncells) * sizeof(int), P->ps));
    CK(cudaMemsetAsync(cursor, 0, size_t(ncells) * sizeof(int), P->ps));
    CK(cudaMemsetAsync(ntask, 0, sizeof(int), P->ps));
    launch_near_keys<T>(c.coord, n, P->d, double(nc) / P->n_os, nc, key, count, P->ps);
    CK(cudaGetLastError());
    scan_ints(P, count, c.nf_start, ncells);
    launch_near_scatter(key, n, c.nf_start, cursor, c.nf_idx, P->ps);
    CK(cudaGetLastError());
    launch_near_gather<T>(c.nf_idx, n, P->d, c.coord, c.nf_coord, P->ps);
    CK(cudaGetLastError());
    launch_near_tasks(c.nf_start, ncells, c.nf_tasks, ntask, P->ps);
    CK(cudaGetLastError());
    c.nf_ntasks = read_int(P, ntask);
    CK(cudaFreeAsync(key, P->ps));
    CK(cudaFreeAsync(count, P->ps));
    CK(cudaFreeAsync(cursor, P->ps));
    CK(cudaFreeAsync(ntask, P->ps));
}

template <typename T>
void build_tables(sk_plan* P) {
    const int d = P->d, N = P->N, h = P->h;
    int64_t nN = 1;
    for (int t = 0; t < d; ++t) nN *= N;
    P->bk = static_cast<double*>(dalloc(P, size_t(nN) * sizeof(double)));
    double* tmp = nullptr;
    double* costab = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&tmp), size_t(nN) * sizeof(double), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&costab), size_t(N) * sizeof(double), P->ps));
    k_cos_table<<<nblk(N), 256, 0, P->ps>>>(costab, N);
    CK(cudaGetLastError());
    // samples -> d cosine passes, ping-ponging so the result ends in P->bk
    double* bufs[2] = {P->bk, tmp};
    int cur = (d % 2 == 0) ? 0 : 1;
    k_sample_kernel<<<nblk(nN), 256, 0, P->ps>>>(bufs[cur], N, d, P->kp);
    CK(cudaGetLastError());
    for (int axis = 0; axis < d; ++axis) {
        k_cos_dft_axis<<<nblk(nN), 256, 0, P->ps>>>(bufs[cur], bufs[1 - cur], N, d, axis, costab);
        CK(cudaGetLastError());
        cur = 1 - cur;
    }
    // now bufs[cur] == P->bk holds N^d * b_k
    P->psihat = static_cast<double*>(dalloc(P, size_t(2 * h + 1) * sizeof(double)));
    k_window_transform<<<nblk(2 * h + 1), 256, 0, P->ps>>>(P->psihat, h, P->n_os, P->prm.m_w, P->beta);
    CK(cudaGetLastError());
    int64_t mtotal = h + 1;
    for (int t = 0; t < d - 1; ++t) mtotal *= (2 * h + 1);
    P->fft.mult = dalloc(P, size_t(mtotal) * sizeof(T));
    const double inv_norm = 1.0 / double(nN);
    launch_build_mult<T>(static_cast<T*>(P->fft.mult), d, h, P->bk, inv_norm, P->psihat, mtotal, P->ps);
    CK(cudaGetLastError());
    // keep b_k itself (normalized) for sk_fourier_coefficients
    k_scale<<<nblk(nN), 256, 0, P->ps>>>(P->bk, nN, inv_norm);
    CK(cudaGetLastError());
    CK(cudaFreeAsync(tmp, P->ps));
    CK(cudaFreeAsync(costab, P->ps));
    // twiddles
    P->fft.tw = dalloc(P, size_t(std::max(1, fft_twiddle_rows<T>(P->n_os))) * sizeof(typename Cplx<T>::type));
    CK(launch_twiddle_rows<T>(P->fft.tw, P->n_os, P->ps));
    CK(cudaGetLastError());
}

template <typename T>
void build_grid(sk_plan* P) {
    using C = typename Cplx<T>::type;
    const int64_t n = P->n_os, H = P->h + 1, K = 2 * P->h + 1;
    FftPlan& f = P->fft;
    f.d = P->d;
    f.n = P->n_os;
    f.log2n = P->log2n;
    f.h = P->h;
    f.psihat = P->psihat;
    if (P->d == 1) {
        P->grid_elems = size_t(2 * n);
        f.A1 = dalloc(P, size_t(2 * H) * sizeof(C));
        f.A3 = nullptr;
    } else if (P->d == 2) {
        P->grid_elems = size_t(n * n);
        f.A1 = dalloc(P, size_t(n * H) * sizeof(C));
        f.A3 = dalloc(P, size_t(K * H) * sizeof(C));
    } else {
        P->grid_elems = size_t(n * n * n);
        f.A1 = dalloc(P, size_t(n * n * H) * sizeof(C));
        f.A2 = dalloc(P, size_t(n * K * H) * sizeof(C));
        f.A3 = dalloc(P, size_t(K * K * H) * sizeof(C));
    }
    f.grid = dalloc(P, P->grid_elems * sizeof(T));
    f.grid_out = dalloc(P, P->grid_elems * sizeof(T));
    CK(cudaMemsetAsync(f.grid, 0, P->grid_elems * sizeof(T), P->ps));
    CK(cudaMemsetAsync(f.grid_out, 0, P->grid_elems * sizeof(T), P->ps));
    // the spectra are zero outside the band between products (see sk_fft.cu)
    if (P->d == 1) {
        CK(cudaMemsetAsync(f.A1, 0, size_t(2 * H) * sizeof(C), P->ps));
    } else if (P->d == 2) {
        CK(cudaMemsetAsync(f.A1, 0, size_t(n * H) * sizeof(C), P->ps));
    } else {
        CK(cudaMemsetAsync(f.A1, 0, size_t(n * n * H) * sizeof(C), P->ps));
        CK(cudaMemsetAsync(f.A2, 0, size_t(n * K * H) * sizeof(C), P->ps));
    }
    // band of cells holding every point's window taps, from both clouds
    int* bounds = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&bounds), 6 * sizeof(int), P->ps));
    k_init_bounds<<<1, 32, 0, P->ps>>>(bounds);
    CK(cudaGetLastError());
    launch_cell_bounds<T>(P->X.coord, P->X.n, P->d, bounds, P->ps);
    launch_cell_bounds<T>(P->Y.coord, P->Y.n, P->d, bounds, P->ps);
    CK(cudaGetLastError());
    int hb[6];
    CK(cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    CK(cudaFreeAsync(bounds, P->ps));
    const int m = P->prm.m_w;
    for (int t = 0; t < 3; ++t) {
        if (t < P->d) {
            f.lo[t] = std::max(0, hb[t] - (m - 1));
            f.hi[t] = std::min(P->n_os - 1, hb[3 + t] + m);
        } else {
            f.lo[t] = 0;
            f.hi[t] = 0;
        }
    }
    f.planes = fft_planes_supported(f, sizeof(T) == 4);
}

template <typename T>
void prepare_kernels(sk_plan* P) {
    SpreadArgs a{};
    a.nsub = 0;
    a.ntasks = 0;
    CK(launch_spread<T>(P->d, P->W, a, P->ps));
    if (column_kernels(P->d, P->W)) {
        InterpArgs ia{};
        ia.ncols = 0;
        CK(launch_interp3<T>(P->W, ia, Epilogue{}, P->ps));
    }
    if (P->d == 2) {
        InterpArgs ia{};
        ia.nstasks = 0;
        CK(launch_interp2<T>(P->W, ia, Epilogue{}, P->ps));
    }
    if (P->tc_ok) {
        InterpArgs ia{};
        ia.nttasks = 0;
        CK(launch_interp_tc(P->d, P->W, ia, Epilogue{}, P->ps));
    }
    CK(launch_fft_convolve<T>(P->fft, P->ps, nullptr));   // runs once on the zero grid
}

// ------------------------------------------------------------ products
Epilogue make_epilogue(sk_plan* P, int mode, Cloud& dst, int slot, double* out) {
    Epilogue e;
    e.mode = mode;
    e.n = dst.n;
    e.perm = dst.perm;
    e.out = out;
    e.t_store = dst.t;
    e.marg = dst.marg;
    e.scal = dst.scal;
    e.partial = P->partial;
    e.ticket = P->ticket;
    e.result = P->stats + 3 * slot;
    e.status = P->status;
    e.log_domain = P->domain == SK_DOMAIN_LOG ? 1 : 0;
    e.fp32_logs = P->precision == SK_FP32 ? 1 : 0;
    e.eps = P->eps;
    e.lam = 1.0 / P->eps;
    e.shift = P->shift;
    return e;
}

// Log domain: the weights exp((g_j - shift) / eps - 1/2) of cloud c's dual
// variables g into c.work, shift = max g stored at P->shift[slot].
const double* log_weights(sk_plan* P, Cloud& c, int slot) {
    k_block_max<<<kRedBlocks, 256, 0, P->ps>>>(c.scal, c.n, P->partial);
    CK(cudaGetLastError());
    k_log_weights<<<kRedBlocks, 256, 0, P->ps>>>(c.scal, c.n, P->partial, kRedBlocks, 1.0 / P->eps,
                                                   P->precision == SK_FP32 ? 1 : 0, c.work, P->shift + slot);
    CK(cudaGetLastError());
    P->launches += 2;
    return c.work;
}

// The weights of a product from cloud c: its scaling vector, or in the log
// domain the shifted exponentials of its dual variables (slot 0 for Y, 1 for X).
const double* source_weights(sk_plan* P, Cloud& c, int slot, Epilogue& e) {
    if (P->domain != SK_DOMAIN_LOG) return c.scal;
    e.shift = P->shift + slot;
    return log_weights(P, c, slot);
}

template <typename T>
void spread_into_grid(sk_plan* P, const Cloud& src, const double* w) {
    // the grid is zero here: the first FFT pass zeroes what spreading wrote
    SpreadArgs a{};
    for (int t = 0; t < 3; ++t) a.coord[t] = src.coord[t];
    a.w = w;
    a.sub_start = src.sub_start;
    a.sub_count = src.sub_count;
    a.sub_bin = src.sub_bin;
    a.nsub = src.nsub;
    a.key_start = src.key_start;
    a.tasks = src.tasks;
    a.ntasks = src.ntasks;
    a.n_os = P->n_os;
    for (int t = 0; t < 3; ++t) a.nb[t] = P->nb[t];
    a.beta = P->beta;
    a.knorm = P->knorm;
    a.grid = P->fft.grid;
    a.wp = P->wp;
    const int st = stage_begin(P, SK_STAGE_SPREAD);
    CK(launch_spread<T>(P->d, P->W, a, P->ps));
    if ((column_kernels(P->d, P->W) || P->d == 2 ? src.ntasks : src.nsub) > 0) ++P->launches;
    stage_end(P, st);
}

template <typename T>
void interp_from_grid(sk_plan* P, Cloud& dst, const Epilogue& e) {
    InterpArgs a{};
    for (int t = 0; t < 3; ++t) a.coord[t] = dst.coord[t];
    a.n = dst.n;
    a.key_start = dst.key_start;
    a.tasks = dst.tasks;
    a.ntasks = dst.ntasks;
    for (int t = 0; t < 3; ++t) a.nb[t] = P->nb[t];
    a.n_os = P->n_os;
    a.beta = P->beta;
    a.knorm = P->knorm;
    a.cols = dst.cols;
    a.ncols = dst.ncols;
    a.stasks = dst.stasks;
    a.nstasks = dst.nstasks;
    a.ttasks = dst.ttasks;
    a.nttasks = dst.nttasks;
    a.inject = P->inject == SK_FAULT_TC_WAIT ? 1 : 0;
    a.queue = P->ticket + 2;
    a.grid = P->fft.grid_out;
    a.wp = P->wp;
    int st = stage_begin(P, SK_STAGE_INTERP);
    if (P->tc && std::is_same<T, float>::value) {
        if (a.nttasks > 0) ++P->launches;
        CK(launch_interp_tc(P->d, P->W, a, e, P->ps));
    } else {
        CK(launch_interp<T>(P->d, P->W, a, e, &P->launches, P->ps));
    }
    stage_end(P, st);
}

// One product into `dst` from `src` with sorted source weights `w`.
template <typename T>
void product(sk_plan* P, Cloud& src, const double* w, Cloud& dst, const Epilogue& e) {
    if (P->method == SK_METHOD_DIRECT) {
        DirectArgs a{};
        for (int t = 0; t < 3; ++t) { a.tcoord[t] = dst.coord[t]; a.scoord[t] = src.coord[t]; }
        a.nt = dst.n;
        a.w = w;
        a.ns = src.n;
        a.coef = 1.0 / (P->eps_s * std::pow(double(P->n_os), P->r));
        a.r = P->r;
        int st = stage_begin(P, SK_STAGE_DIRECT);
        CK(launch_direct<T>(P->d, a, e, &P->launches, P->ps));
        stage_end(P, st);
        return;
    }
    Epilogue ee = e;
    if (P->nearfield) {
        // direct sums over pairs closer than eps_I, added to t in the epilogue
        NearArgs na{};
        for (int t = 0; t < 3; ++t) { na.t_coord[t] = dst.nf_coord[t]; na.s_coord[t] = src.nf_coord[t]; }
        na.t_start = dst.nf_start;
        na.t_idx = dst.nf_idx;
        na.s_start = src.nf_start;
        na.s_idx = src.nf_idx;
        na.w = w;
        na.tasks = dst.nf_tasks;
        na.nc = near_cells_per_dim(P);
        na.sub = P->near_sub;
        const double rg = P->n_os * P->prm.eps_I;
        na.r2max = rg * rg;
        na.inv_r2 = 1.0 / (rg * rg);
        na.kcoef = 1.0 / (P->eps_s * std::pow(double(P->n_os), P->r));
        na.r = P->r;
        na.p = P->kp.p;
        for (int q = 0; q < kMaxP; ++q) na.ki[q] = P->kp.ki[q];
        na.out = dst.nf_corr;
        const int st = stage_begin(P, SK_STAGE_NEAR);
        CK(launch_nearfield<T>(P->d, na, dst.nf_ntasks, P->ps));
        if (dst.nf_ntasks > 0) ++P->launches;
        stage_end(P, st);
        ee.add = dst.nf_corr;
    }
    spread_into_grid<T>(P, src, w);
    int st = stage_begin(P, SK_STAGE_FFT);
    CK(launch_fft_convolve<T>(P->fft, P->ps, &P->launches));
    stage_end(P, st);
    interp_from_grid<T>(P, dst, ee);
}

// Average time (ms) of `reps` products K v of the plan with its current
// interpolation kernels: weights = the current v, output into scratch.
template <typename T>
double time_products(sk_plan* P, int reps) {
    Epilogue e = make_epilogue(P, EPI_APPLY, P->X, 0, P->X.stage);
    product<T>(P, P->Y, P->Y.scal, P->X, e);   // warm-up
    struct Events {   // released on every exit, including a failed CUDA call
        cudaEvent_t ev[2] = {nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t v : ev)
                if (v) cudaEventDestroy(v);
        }
    } t;
    CK(cudaEventCreate(&t.ev[0]));
    CK(cudaEventCreate(&t.ev[1]));
    CK(cudaEventRecord(t.ev[0], P->ps));
    for (int r = 0; r < reps; ++r) product<T>(P, P->Y, P->Y.scal, P->X, e);
    CK(cudaEventRecord(t.ev[1], P->ps));
    CK(cudaEventSynchronize(t.ev[1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t.ev[0], t.ev[1]));
    return double(ms) / reps;
}


template <typename T>
void iteration(sk_plan* P) {
    // odd half-step: u = a ./ (K v)  (log domain: beta = eps (log a - log t + 1/2))
    Epilogue e1 = make_epilogue(P, EPI_UPDATE, P->X, SLOT_ROW, nullptr);
    const double* w1 = source_weights(P, P->Y, 0, e1);
    product<T>(P, P->Y, w1, P->X, e1);
    // even half-step: v = b ./ (K^T u)
    Epilogue e2 = make_epilogue(P, EPI_UPDATE, P->Y, SLOT_COL, nullptr);
    const double* w2 = source_weights(P, P->X, 1, e2);
    product<T>(P, P->X, w2, P->Y, e2);
}

void run_iteration(sk_plan* P) {
    if (P->precision == SK_FP32)
        iteration<float>(P);
    else
        iteration<double>(P);
}

void destroy_graph(sk_plan* P) {
    if (P->gexec) {
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
    }
    if (P->gexec_timed) {
        cudaGraphExecDestroy(P->gexec_timed);
        P->gexec_timed = nullptr;
    }
}

// One iteration captured into a graph; with stage timing on, the stage events
// are captured too (as event-record nodes of their own pool).
void capture_iteration(sk_plan* P, cudaGraphExec_t* out, int64_t* kernels) {
    const int64_t before = P->launches;
    if (P->timing) {
        P->graph_ev.used = 0;
        P->pool = &P->graph_ev;
    }
    CK(cudaStreamBeginCapture(P->ps, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t g = nullptr;
    try {
        run_iteration(P);
    } catch (...) {
        cudaStreamEndCapture(P->ps, &g);
        if (g) cudaGraphDestroy(g);
        P->launches = before;
        P->pool = &P->eager;
        throw;
    }
    P->pool = &P->eager;
    CK(cudaStreamEndCapture(P->ps, &g));
    *kernels = P->launches - before;
    P->launches = before;
    cudaError_t e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e);
}

// Iterations by graph replay.  With stage timing on, the replayed graph
// holds the stage events, which are read after every replay.
void iterate(sk_plan* P, int k) {
    for (int i = 0; i < k; ++i) {
        if (P->timing) {
            if (!P->gexec_timed) capture_iteration(P, &P->gexec_timed, &P->graph_kernels_timed);
            CK(cudaGraphLaunch(P->gexec_timed, P->ps));
            P->launches += P->graph_kernels_timed;
            pool_resolve(P, P->graph_ev, true);
        } else {
            if (!P->gexec) capture_iteration(P, &P->gexec, &P->graph_kernels);
            CK(cudaGraphLaunch(P->gexec, P->ps));
            P->launches += P->graph_kernels;
        }
        ++P->iters;
    }
}

double read_slot(sk_plan* P, int slot, int field) {
    CK(cudaMemcpyAsync(P->pinned, P->stats + 3 * slot + field, sizeof(double), cudaMemcpyDeviceToHost, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    return P->pinned[0];
}

int read_status(sk_plan* P) {
    int st = 0;
    CK(cudaMemcpyAsync(P->pinned, P->status, sizeof(int), cudaMemcpyDeviceToHost, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    std::memcpy(&st, P->pinned, sizeof(int));
    return st;
}

void clear_status(sk_plan* P) { CK(cudaMemsetAsync(P->status, 0, sizeof(int), P->ps)); }

// sum_i a_i log u_i; in the log domain lam sum_i a_i beta_i - 1/2 (sum a = 1).
double sum_marg_log(sk_plan* P, const Cloud& c) {
    const int as_is = P->domain == SK_DOMAIN_LOG ? 1 : 0;
    k_sum_marg_log<<<kRedBlocks, 256, 0, P->ps>>>(c.marg, c.scal, c.n, as_is, P->partial);
    CK(cudaGetLastError());
    ++P->launches;
    const int ops[1] = {0};
    double v = 0.0;
    combine_to_host(P, kRedBlocks, 1, ops, &v);
    ++P->launches;
    return as_is ? v / P->eps - 0.5 : v;
}

template <typename T>
void final_report(sk_plan* P, sk_result* res) {
    Epilogue e1 = make_epilogue(P, EPI_RESID, P->X, SLOT_RES_ROW, nullptr);
    const double* w1 = source_weights(P, P->Y, 0, e1);
    product<T>(P, P->Y, w1, P->X, e1);
    Epilogue e2 = make_epilogue(P, EPI_RESID, P->Y, SLOT_RES_COL, nullptr);
    const double* w2 = source_weights(P, P->X, 1, e2);
    product<T>(P, P->X, w2, P->Y, e2);
    CK(cudaMemcpyAsync(P->pinned, P->stats, sizeof(double) * 3 * NSLOTS, cudaMemcpyDeviceToHost, P->ps));
    CK(cudaStreamSynchronize(P->ps));
    double st[3 * NSLOTS];
    std::memcpy(st, P->pinned, sizeof(st));
    const double row2 = st[3 * SLOT_RES_ROW + 0], uKv = st[3 * SLOT_RES_ROW + 2];
    const double col2 = st[3 * SLOT_RES_COL + 0];
    const double la = sum_marg_log(P, P->X), lb = sum_marg_log(P, P->Y);
    res->s = P->eps * (1.0 + la + lb - uKv);
    res->s_upper = res->s + P->eps * (P->Ha + P->Hb);
    res->err_row = std::sqrt(row2);
    res->err_col = std::sqrt(col2);
    res->marg_err = res->err_row + res->err_col;
    res->total_iters = P->iters;
}

// The dual variables of one cloud's marginal constraint, eps (1/2 + log u),
// into a caller buffer (host or device) in caller order.
void dual_variable_out(sk_plan* P, const Cloud& c, double* out) {
    const bool host = !is_device_ptr(out);
    k_dual_variable<<<nblk(c.n), 256, 0, P->ps>>>(c.scal, c.perm, c.n, P->eps, P->domain == SK_DOMAIN_LOG ? 1 : 0,
                                                  host ? c.stage : out);
    CK(cudaGetLastError());
    ++P->launches;
    if (host) {
        CK(cudaMemcpyAsync(out, c.stage, size_t(c.n) * sizeof(double), cudaMemcpyDeviceToHost, P->ps));
        CK(cudaStreamSynchronize(P->ps));
    }
}

// Gradient of the dual function Eq. (27) with respect to the positions of
// cloud `dst` for r = 2, at the plan's current scaling vectors:
//   grad_i = sum_j pi_ij 2 (x_i - y_j) = 2 u_i (x_i (K v)_i - (K (v y))_i),
// with coordinates taken relative to the plan's centre.  d + 1 products
// from `src` (weights v and v (y_t - c_t)); out is n x d row-major, caller order.
template <typename T>
void position_gradient(sk_plan* P, Cloud& src, Cloud& dst, double* out) {
    const int d = P->d;
    const int64_t n = dst.n;
    const bool host = !is_device_ptr(out);
    double *t0 = nullptr, *tt = nullptr, *w = nullptr, *g = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&t0), size_t(n) * sizeof(double), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&tt), size_t(n) * sizeof(double), P->ps));
    CK(cudaMallocAsync(reinterpret_cast<void**>(&w), size_t(src.n) * sizeof(double), P->ps));
    if (host) CK(cudaMallocAsync(reinterpret_cast<void**>(&g), size_t(n) * d * sizeof(double), P->ps));
    double* gdst = host ? g : out;
    const double inv_nos = 1.0 / P->n_os, inv_s = 1.0 / P->scale;
    Epilogue e = make_epilogue(P, EPI_APPLY, dst, 0, t0);
    e.perm = nullptr;   // sorted order
    const int slot = &src == &P->Y ? 0 : 1;
    const double* ws = source_weights(P, src, slot, e);     // v, or the log domain's shifted weights
    const double* log_shift = P->domain == SK_DOMAIN_LOG ? P->shift + slot : nullptr;
    product<T>(P, src, ws, dst, e);
    for (int t = 0; t < d; ++t) {
        launch_weighted_coord<T>(ws, src.coord[t], src.n, inv_nos, inv_s, w, P->ps);
        CK(cudaGetLastError());
        ++P->launches;
        Epilogue et = make_epilogue(P, EPI_APPLY, dst, 0, tt);
        et.perm = nullptr;
        product<T>(P, src, w, dst, et);
        launch_position_gradient<T>(dst.scal, dst.coord[t], t0, tt, dst.perm, n, d, t, inv_nos, inv_s, log_shift,
                                    1.0 / P->eps, gdst, P->ps);
        CK(cudaGetLastError());
        ++P->launches;
    }
    if (host) {
        CK(cudaMemcpyAsync(out, g, size_t(n) * d * sizeof(double), cudaMemcpyDeviceToHost, P->ps));
        CK(cudaStreamSynchronize(P->ps));
    }
    CK(cudaFreeAsync(t0, P->ps));
    CK(cudaFreeAsync(tt, P->ps));
    CK(cudaFreeAsync(w, P->ps));
    if (g) CK(cudaFreeAsync(g, P->ps));
}

void write_out(sk_plan* P, const Cloud& c, const double* sorted, double* out) {
    if (!out) return;
    if (is_device_ptr(out)) {
        k_scatter<<<nblk(c.n), 256, 0, P->ps>>>(sorted, c.perm, c.n, out);
        CK(cudaGetLastError());
        ++P->launches;
    } else {
        k_scatter<<<nblk(c.n), 256, 0, P->ps>>>(sorted, c.perm, c.n, c.stage);
        CK(cudaGetLastError());
        ++P->launches;
        CK(cudaMemcpyAsync(out, c.stage, size_t(c.n) * sizeof(double), cudaMemcpyDeviceToHost, P->ps));
        CK(cudaStreamSynchronize(P->ps));
    }
}

void read_in(sk_plan* P, const Cloud& c, const double* in, double* sorted) {
    const double* src = device_view(P, in, c.n, c.stage);
    k_gather<<<nblk(c.n), 256, 0, P->ps>>>(src, c.perm, c.n, sorted);
    CK(cudaGetLastError());
    ++P->launches;
}

int fail_code(const Fail& f) { return f.code; }

}  // namespace

// ====================================================================== ABI

extern "C" {

const char* sk_last_error(void) { return g_last_error; }

const char* sk_error_string(int status) {
    switch (status) {
        case SK_OK: return "ok";
        case SK_ERR_ARG: return "invalid argument";
        case SK_ERR_DOMAIN: return "coordinates not finite or outside the grid";
        case SK_ERR_WEIGHTS: return "weights negative, not finite or not summing to 1";
        case SK_ERR_NOMEM: return "device allocation failed";
        case SK_ERR_UNDERFLOW: return "a kernel sum was <= 0 or not finite";
        case SK_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case SK_ERR_TIMEOUT: return "bounded device wait ran out";
        case SK_ERR_CUDA: return "CUDA runtime error";
        case SK_ERR_UNSUPPORTED: return "not supported for this plan";
        case SK_ERR_TOO_LARGE: return "size exceeds the fixed scratch of the no-allocation entry point (n <= 2097152)";
        default: return "unknown status";
    }
}

int sk_default_params(sk_nfft_params* prm) {
    if (!prm) return SK_ERR_ARG;
    std::memset(prm, 0, sizeof(*prm));
    prm->N = 64;
    prm->sigma = 2.0;
    prm->m_w = 4;
    prm->p = 8;
    prm->eps_B = 0.1;
    prm->eps_I = 0.0;
    prm->precision = SK_FP32;
    prm->user_geometry = 0;
    prm->scale = 1.0;
    return SK_OK;
}

// ------------------------------------------------------------ parameter choice
// Accuracy targets of the automatic choices, relative to K(0) = 1: below the
// rounding of the kernel sums in each precision.
double auto_target(int precision) { return precision == SK_FP32 ? 1e-6 : 1e-10; }

// Window cutoff m for the target: the Kaiser-Bessel window's error with
// oversampling sigma decays like 4 pi (1 - 1/sigma)^(1/4) exp(-2 pi m sqrt(1 - 1/sigma))
// (the window's error estimate, Plonka et al. Ch. 7).  3-D plans stop at m = 5,
// the widest window of the column kernels.
int choose_cutoff(int d, double sigma, int precision) {
    const double q = 1.0 - 1.0 / sigma;
    const double m = std::log(4.0 * M_PI * std::pow(q, 0.25) / auto_target(precision)) / (2.0 * M_PI * std::sqrt(q));
    return std::max(2, std::min(d == 3 ? 5 : 8, int(std::ceil(m))));
}

// Bandwidth N: the smallest power of two from 16 for which the Fourier tail of
// the regularized kernel, sum over |k| >= N/2 of |c_k| for its slice
// rho -> K_R(|rho|) along one axis (Eq. (ansatz_NFFT)'s coefficients in one
// dimension, from 2048 samples), stays below target / d.
int choose_bandwidth(double eps_s, double r, int d, const sk_nfft_params& p, bool auto_I, bool nearfield) {
    KernelParams kp{};
    kp.eps_s = eps_s;
    kp.r = r;
    kp.L = 0.5 - p.eps_B;
    kp.p = p.p;
    kp.nearfield = nearfield ? 1 : 0;
    kp.eps_I = p.eps_I;
    const int nmax = d == 1 ? 2048 : 512;
    if (!boundary_coefficients(kp)) return 64;
    const int M = 2048;
    std::vector<double> ct(M), f(M), c(M / 2 + 1);
    for (int l = 0; l < M; ++l) ct[l] = std::cos(2.0 * M_PI * l / M);
    const double target = auto_target(p.precision) / d;
    int spectrum_for = -1;   // the N whose eps_I the spectrum was computed with (near field only)
    for (int N = 16; N <= nmax; N *= 2) {
        if (spectrum_for < 0 || (nearfield && auto_I)) {
            if (nearfield) {
                if (auto_I) kp.eps_I = 16.0 / (3.0 * N);
                if (!(kp.eps_I < kp.L) || !nearfield_coefficients(kp)) continue;
            }
            for (int l = 0; l < M; ++l) f[l] = kr_value(std::fabs(double(l - M / 2) / M), kp);
            for (int k = 0; k <= M / 2; ++k) {
                double acc = 0.0;
                for (int l = 0; l < M; ++l) acc += f[l] * ct[(int64_t(k) * l) % M];
                c[k] = acc / M;
            }
            spectrum_for = N;
        }
        double tail = 0.0;
        for (int k = N / 2; k <= M / 2; ++k) tail += 2.0 * std::fabs(c[k]);
        if (tail <= target) return N;
    }
    return nmax;
}

static int validate_params(int d, const sk_nfft_params& p, int& n_os, int& log2n) {
    if (p.N < 8 || (p.N % 2) != 0) return SK_ERR_ARG;
    if (!(p.sigma > 1.0) || !std::isfinite(p.sigma)) return SK_ERR_ARG;
    const double nd = p.sigma * p.N;
    n_os = int(std::lround(nd));
    if (std::fabs(nd - n_os) > 1e-9) return SK_ERR_ARG;
    if (n_os < 16 || (n_os & (n_os - 1)) != 0) return SK_ERR_ARG;
    if (n_os > (d == 1 ? 4096 : 1024)) return SK_ERR_ARG;
    if (p.N > n_os / 2) return SK_ERR_ARG;
    log2n = 0;
    while ((1 << log2n) < n_os) ++log2n;
    if (p.m_w < 2 || p.m_w > 8) return SK_ERR_ARG;
    if (n_os < 4 * (p.m_w + 1)) return SK_ERR_ARG;
    if (p.p < 2 || p.p > kMaxP) return SK_ERR_ARG;
    if (!(p.eps_B > 0.0 && p.eps_B < 0.5)) return SK_ERR_ARG;
    if (p.precision != SK_FP32 && p.precision != SK_FP64) return SK_ERR_ARG;
    if (p.user_geometry && !(p.scale > 0.0 && std::isfinite(p.scale))) return SK_ERR_ARG;
    return SK_OK;
}

int sk_init(sk_plan** out, int d, int64_t n, const double* x, const double* a, int64_t m, const double* y,
            const double* b, double eps, double r, const sk_nfft_params* prm, void* stream) {
    if (!out) return SK_ERR_ARG;
    *out = nullptr;
    if (d < 1 || d > 3 || n < 1 || m < 1 || n > INT32_MAX / 2 || m > INT32_MAX / 2) return SK_ERR_ARG;
    if (!x || !a || !y || !b) return SK_ERR_ARG;
    if (!(eps > 0.0) || !std::isfinite(eps) || !(r >= 1.0) || !std::isfinite(r)) return SK_ERR_ARG;
    sk_nfft_params p;
    if (prm)
        p = *prm;
    else
        sk_default_params(&p);
    // N <= 0 or m_w <= 0: chosen once the geometry is known (choose_bandwidth,
    // choose_cutoff); placeholders let every other parameter be checked now
    const bool auto_N = p.N <= 0, auto_m = p.m_w <= 0, auto_I = !(p.eps_I > 0.0);
    if (auto_N) p.N = 64;
    if (auto_m) p.m_w = 4;
    int n_os = 0, log2n = 0;
    int rc = validate_params(d, p, n_os, log2n);
    if (rc != SK_OK) return rc;
    const bool nearfield = !even_integer(r);
    if (auto_I) p.eps_I = 16.0 / (3.0 * p.N);   // automatic near-field radius
    if (nearfield && !(p.eps_I < 0.5 - p.eps_B)) return SK_ERR_ARG;

    sk_plan* P = new (std::nothrow) sk_plan();
    if (!P) return SK_ERR_NOMEM;
    try {
        CK(cudaGetDevice(&P->device));
        P->d = d;
        P->n = n;
        P->m = m;
        P->eps = eps;
        P->r = r;
        P->nearfield = nearfield ? 1 : 0;

        CK(cudaStreamCreateWithFlags(&P->ps, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
        CK(cudaMallocHost(reinterpret_cast<void**>(&P->pinned), 64 * sizeof(double)));
        enter(P, stream);

        const int64_t nmax = std::max(n, m);
        P->partial_blocks = std::max<int64_t>(interp_blocks<double>(nmax), kRedBlocks);
        P->partial = static_cast<double*>(dalloc(P, size_t(P->partial_blocks) * 8 * sizeof(double)));
        P->ticket = static_cast<unsigned*>(dalloc(P, sizeof(unsigned) * 8));   // [0] reductions, [2..3] interpolation queue
        P->stats = static_cast<double*>(dalloc(P, sizeof(double) * (3 * NSLOTS + 8)));
        P->status = static_cast<int*>(dalloc(P, sizeof(int) * 4));
        P->shift = static_cast<double*>(dalloc(P, sizeof(double) * 2));
        CK(cudaMemsetAsync(P->shift, 0, sizeof(double) * 2, P->ps));
        CK(cudaMemsetAsync(P->ticket, 0, sizeof(unsigned) * 8, P->ps));
        CK(cudaMemsetAsync(P->stats, 0, sizeof(double) * (3 * NSLOTS + 8), P->ps));
        CK(cudaMemsetAsync(P->status, 0, sizeof(int) * 4, P->ps));

        // inputs on the device (staged through temporaries if on the host)
        double *xd = nullptr, *yd = nullptr, *ad = nullptr, *bd = nullptr;
        const bool xdev = is_device_ptr(x), ydev = is_device_ptr(y), adev = is_device_ptr(a), bdev = is_device_ptr(b);
        std::vector<void*> tmps;
        auto stage_in = [&](const double* src, bool dev, int64_t cnt) -> const double* {
            if (dev) return src;
            double* dst = nullptr;
            CK(cudaMallocAsync(reinterpret_cast<void**>(&dst), size_t(cnt) * sizeof(double), P->ps));
            tmps.push_back(dst);
            CK(cudaMemcpyAsync(dst, src, size_t(cnt) * sizeof(double), cudaMemcpyHostToDevice, P->ps));
            return dst;
        };
        const double* xs = stage_in(x, xdev, n * d);
        const double* ys = stage_in(y, ydev, m * d);
        const double* as = stage_in(a, adev, n);
        const double* bs = stage_in(b, bdev, m);
        (void)xd;
        (void)yd;
        (void)ad;
        (void)bd;

        // validation: finite coordinates, bounding box; weights
        const int bounds_ops[7] = {1, 1, 1, 2, 2, 2, 0};
        double bx[7], by[7];
        k_point_bounds<<<kRedBlocks, 256, 0, P->ps>>>(xs, n, d, P->partial);
        CK(cudaGetLastError());
        combine_to_host(P, kRedBlocks, 7, bounds_ops, bx);
        k_point_bounds<<<kRedBlocks, 256, 0, P->ps>>>(ys, m, d, P->partial);
        CK(cudaGetLastError());
        combine_to_host(P, kRedBlocks, 7, bounds_ops, by);
        if (bx[6] > 0 || by[6] > 0) throw Fail{SK_ERR_DOMAIN};
        const int wops[4] = {0, 1, 0, 0};
        double wa[4], wb[4];
        k_weight_stats<<<kRedBlocks, 256, 0, P->ps>>>(as, n, P->partial);
        CK(cudaGetLastError());
        combine_to_host(P, kRedBlocks, 4, wops, wa);
        k_weight_stats<<<kRedBlocks, 256, 0, P->ps>>>(bs, m, P->partial);
        CK(cudaGetLastError());
        combine_to_host(P, kRedBlocks, 4, wops, wb);
        if (wa[2] > 0 || wb[2] > 0 || wa[1] < 0 || wb[1] < 0 || std::fabs(wa[0] - 1.0) > 1e-9 ||
            std::fabs(wb[0] - 1.0) > 1e-9)
            throw Fail{SK_ERR_WEIGHTS};
        P->Ha = wa[3];
        P->Hb = wb[3];

        // geometry
        if (p.user_geometry) {
            for (int t = 0; t < 3; ++t) P->center[t] = t < d ? p.center[t] : 0.0;
            P->scale = p.scale;
        } else {
            for (int t = 0; t < 3; ++t)
                P->center[t] = t < d ? 0.5 * (std::min(bx[t], by[t]) + std::max(bx[3 + t], by[3 + t])) : 0.0;
            const int rops[1] = {2};
            double rx = 0, ry = 0;
            k_point_radius<<<kRedBlocks, 256, 0, P->ps>>>(xs, n, d, P->center[0], P->center[1], P->center[2],
                                                           P->partial);
            CK(cudaGetLastError());
            combine_to_host(P, kRedBlocks, 1, rops, &rx);
            k_point_radius<<<kRedBlocks, 256, 0, P->ps>>>(ys, m, d, P->center[0], P->center[1], P->center[2],
                                                           P->partial);
            CK(cudaGetLastError());
            combine_to_host(P, kRedBlocks, 1, rops, &ry);
            const double R = std::sqrt(std::max(rx, ry));
            P->scale = R > 0.0 ? (0.25 - 0.5 * p.eps_B) / R : 1.0;
        }
        P->eps_s = eps * std::pow(P->scale, r);
        if (auto_N || auto_m) {
            if (auto_m) p.m_w = choose_cutoff(d, p.sigma, p.precision);
            if (auto_N) p.N = choose_bandwidth(P->eps_s, r, d, p, auto_I, nearfield);
            if (auto_I) p.eps_I = 16.0 / (3.0 * p.N);
            if (validate_params(d, p, n_os, log2n) != SK_OK) throw Fail{SK_ERR_ARG};
            if (nearfield && !(p.eps_I < 0.5 - p.eps_B)) throw Fail{SK_ERR_ARG};
        }
        P->prm = p;
        P->precision = p.precision;
        P->N = p.N;
        P->h = p.N / 2;
        P->n_os = n_os;
        P->log2n = log2n;
        P->W = 2 * p.m_w;
        bin_shape(d, P->W, P->B);
        P->tc_ok = tc_supported(d, P->W, P->precision == SK_FP32);
        P->tc = P->tc_ok;
        P->nbins = 1;
        P->bvol = 1;
        for (int t = 0; t < 3; ++t) {
            P->nb[t] = t < d ? (n_os + P->B[t] - 1) / P->B[t] : 1;
            P->nbins *= P->nb[t];
            P->bvol *= t < d ? P->B[t] : 1;
        }
        P->nkeys = int64_t(P->nbins) * P->bvol;
        P->beta = M_PI * (2.0 - 1.0 / p.sigma);
        P->knorm = double(p.m_w) / std::sinh(P->beta * p.m_w);
        window_polynomials(p.m_w, P->beta, P->knorm, P->wp);

        // kernel parameters in torus coordinates
        P->kp.eps_s = P->eps_s;
        P->kp.r = r;
        P->kp.L = 0.5 - p.eps_B;
        P->kp.eps_I = p.eps_I;
        P->kp.p = p.p;
        P->kp.nearfield = P->nearfield;
        if (!boundary_coefficients(P->kp)) throw Fail{SK_ERR_ARG};
        if (P->nearfield && !nearfield_coefficients(P->kp)) throw Fail{SK_ERR_ARG};

        if (P->precision == SK_FP32) {
            build_cloud<float>(P, P->X, xs, as, n);
            build_cloud<float>(P, P->Y, ys, bs, m);
            if (P->nearfield) {
                choose_near_sub<float>(P);
                build_near<float>(P, P->X);
                build_near<float>(P, P->Y);
            }
            build_tables<float>(P);
            build_grid<float>(P);
        } else {
            build_cloud<double>(P, P->X, xs, as, n);
            build_cloud<double>(P, P->Y, ys, bs, m);
            if (P->nearfield) {
                choose_near_sub<double>(P);
                build_near<double>(P, P->X);
                build_near<double>(P, P->Y);
            }
            build_tables<double>(P);
            build_grid<double>(P);
        }
        for (void* t : tmps) CK(cudaFreeAsync(t, P->ps));
        // opt the kernels this plan uses into their shared-memory sizes now, so
        // no attribute call happens while an iteration is being captured
        if (P->precision == SK_FP32)
            prepare_kernels<float>(P);
        else
            prepare_kernels<double>(P);
        // the strip and column kernels reduce one partial per block
        if (P->d == 2) {
            const int nt = std::max(P->X.nstasks, P->Y.nstasks);
            const int need = P->precision == SK_FP32 ? strip2_blocks<float>(P->W, nt) : strip2_blocks<double>(P->W, nt);
            if (need > P->partial_blocks) {
                P->partial_blocks = need;
                P->partial = static_cast<double*>(dalloc(P, size_t(need) * 8 * sizeof(double)));
            }
        }
        if (P->tc_ok) {
            const int need = interp_tc_blocks(P->d, P->W, std::max(P->X.nttasks, P->Y.nttasks));
            if (need <= 0) throw Fail{SK_ERR_CUDA};
            if (need > P->partial_blocks) {
                P->partial_blocks = need;
                P->partial = static_cast<double*>(dalloc(P, size_t(need) * 8 * sizeof(double)));
            }
        }
        if (column_kernels(P->d, P->W)) {
            const int ncols = std::max(P->X.ncols, P->Y.ncols);
            const int need = std::max(std::max(P->X.ntasks, P->Y.ntasks),
                                      P->precision == SK_FP32 ? interp3_blocks<float>(P->W, ncols)
                                                              : interp3_blocks<double>(P->W, ncols));
            if (need > P->partial_blocks) {
                P->partial_blocks = need;
                P->partial = static_cast<double*>(dalloc(P, size_t(need) * 8 * sizeof(double)));
            }
        }
        const int st = read_status(P);
        if (st & 2) throw Fail{SK_ERR_DOMAIN};
        leave(P, stream);
        CK(cudaStreamSynchronize(P->ps));
    } catch (const Fail& f) {
        cudaStreamSynchronize(P->ps);
        cudaGetLastError();
        sk_destroy(P);
        return fail_code(f);
    }
    *out = P;
    return SK_OK;
}

void sk_destroy(sk_plan* P) {
    if (!P) return;
    cudaSetDevice(P->device);
    if (P->ps) cudaStreamSynchronize(P->ps);
    destroy_graph(P);
    for (void* p : P->allocs) cudaFree(p);
    for (cudaEvent_t e : P->eager.ev) cudaEventDestroy(e);
    for (cudaEvent_t e : P->graph_ev.ev) cudaEventDestroy(e);
    if (P->pinned) cudaFreeHost(P->pinned);
    if (P->ev_in) cudaEventDestroy(P->ev_in);
    if (P->ev_out) cudaEventDestroy(P->ev_out);
    if (P->ps) cudaStreamDestroy(P->ps);
    delete P;
}

int sk_set_method(sk_plan* P, int method) {
    if (!P || (method != SK_METHOD_NFFT && method != SK_METHOD_DIRECT)) return SK_ERR_ARG;
    if (method != P->method) {
        destroy_graph(P);
        P->method = method;
    }
    return SK_OK;
}

int sk_set_kernels(sk_plan* P, int kernels) {
    if (!P || (kernels != SK_KERNELS_SIMT && kernels != SK_KERNELS_TENSOR)) return SK_ERR_ARG;
    if (kernels == SK_KERNELS_TENSOR && !P->tc_ok) return SK_ERR_UNSUPPORTED;
    const bool tc = kernels == SK_KERNELS_TENSOR;
    if (!tc) {
        try {
            if (P->precision == SK_FP32)
                ensure_column_queues<float>(P);
            else
                ensure_column_queues<double>(P);
        } catch (const Fail& f) {
            return fail_code(f);
        }
    }
    if (tc != P->tc) {
        destroy_graph(P);
        P->tc = tc;
    }
    return SK_OK;
}

int sk_set_fft(sk_plan* P, int form) {
    if (!P || (form != SK_FFT_PASSES && form != SK_FFT_PLANES)) return SK_ERR_ARG;
    const bool planes = form == SK_FFT_PLANES;
    if (planes && !fft_planes_supported(P->fft, P->precision == SK_FP32)) return SK_ERR_UNSUPPORTED;
    if (planes != P->fft.planes) {
        destroy_graph(P);
        P->fft.planes = planes;
    }
    return SK_OK;
}

int sk_autotune(sk_plan* P, int* chosen, void* stream) {
    if (!P) return SK_ERR_ARG;
    try {
        enter(P, stream);
        int best = P->tc ? SK_KERNELS_TENSOR : SK_KERNELS_SIMT;
        if (P->tc_ok && P->method == SK_METHOD_NFFT) {
            if (P->precision == SK_FP32)
                ensure_column_queues<float>(P);
            else
                ensure_column_queues<double>(P);
            const bool was = P->tc;
            const int64_t launches = P->launches;
            double ms[2] = {0.0, 0.0};
            for (int k = 0; k < 2; ++k) {
                P->tc = k == SK_KERNELS_TENSOR;
                ms[k] = P->precision == SK_FP32 ? time_products<float>(P, 3) : time_products<double>(P, 3);
            }
            P->launches = launches;   // tuning launches are not the caller's work
            best = ms[SK_KERNELS_TENSOR] <= ms[SK_KERNELS_SIMT] ? SK_KERNELS_TENSOR : SK_KERNELS_SIMT;
            P->tc = best == SK_KERNELS_TENSOR;
            if (P->tc != was) destroy_graph(P);
        }
        if (chosen) *chosen = best;
        leave(P, stream);
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int sk_inject_fault(sk_plan* P, int kind) {
    if (!P || (kind != SK_FAULT_NONE && kind != SK_FAULT_TC_WAIT)) return SK_ERR_ARG;
    if (kind == SK_FAULT_TC_WAIT && !P->tc) return SK_ERR_UNSUPPORTED;
    if (kind != P->inject) {
        destroy_graph(P);
        P->inject = kind;
    }
    return SK_OK;
}

int sk_set_domain(sk_plan* P, int domain) {
    if (!P || (domain != SK_DOMAIN_SCALING && domain != SK_DOMAIN_LOG)) return SK_ERR_ARG;
    if (domain == P->domain) return SK_OK;
    try {
        CK(cudaSetDevice(P->device));
        const int to_log = domain == SK_DOMAIN_LOG ? 1 : 0;
        k_convert_domain<<<nblk(P->X.n), 256, 0, P->ps>>>(P->X.scal, P->X.n, P->eps, to_log);
        CK(cudaGetLastError());
        k_convert_domain<<<nblk(P->Y.n), 256, 0, P->ps>>>(P->Y.scal, P->Y.n, P->eps, to_log);
        CK(cudaGetLastError());
        P->launches += 2;
        CK(cudaStreamSynchronize(P->ps));
        destroy_graph(P);
        P->domain = domain;
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int sk_kernel_apply(sk_plan* P, int transpose, const double* in, double* out, void* stream) {
    if (!P || !in || !out || (transpose != 0 && transpose != 1)) return SK_ERR_ARG;
    try {
        enter(P, stream);
        Cloud& src = transpose ? P->X : P->Y;
        Cloud& dst = transpose ? P->Y : P->X;
        read_in(P, src, in, src.work);
        const bool host_out = !is_device_ptr(out);
        Epilogue e = make_epilogue(P, EPI_APPLY, dst, 0, host_out ? dst.stage : out);
        if (P->precision == SK_FP32)
            product<float>(P, src, src.work, dst, e);
        else
            product<double>(P, src, src.work, dst, e);
        if (host_out) {
            CK(cudaMemcpyAsync(out, dst.stage, size_t(dst.n) * sizeof(double), cudaMemcpyDeviceToHost, P->ps));
            CK(cudaStreamSynchronize(P->ps));
        }
        leave(P, stream);
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int sk_solve(sk_plan* P, int max_iter, double tol, int check_every, double* u_out, double* v_out, sk_result* res,
             void* stream) {
    if (!P || max_iter < 0) return SK_ERR_ARG;
    int rc = SK_OK;
    try {
        enter(P, stream);
        clear_status(P);
        const int every = check_every > 0 ? check_every : 10;
        int done = 0;
        bool converged = false;
        if (tol > 0.0) {
            while (done < max_iter) {
                const int k = std::min(every, max_iter - done);
                iterate(P, k);
                done += k;
                const double row2 = read_slot(P, SLOT_ROW, 0);
                if (std::sqrt(row2) <= tol) {
                    converged = true;
                    break;
                }
            }
            if (!converged) rc = SK_ERR_NOT_CONVERGED;
        } else {
            iterate(P, max_iter);
            done = max_iter;
        }
        if (res) {
            std::memset(res, 0, sizeof(*res));
            if (P->precision == SK_FP32)
                final_report<float>(P, res);
            else
                final_report<double>(P, res);
            res->iters = done;
        }
        write_out(P, P->X, P->X.scal, u_out);
        write_out(P, P->Y, P->Y.scal, v_out);
        if (res || u_out || v_out || tol > 0.0) {
            const int st = read_status(P);
            if (st & 1) rc = SK_ERR_UNDERFLOW;
            if (st & 4) rc = SK_ERR_TIMEOUT;
        }
        leave(P, stream);
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return rc;
}

int sk_solve_batch(sk_plan* const* plans, int count, int max_iter, sk_result* results, void* stream) {
    if (!plans || count < 1 || max_iter < 0) return SK_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || plans[i]->timing) return SK_ERR_ARG;
        if (plans[i]->device != plans[0]->device) return SK_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return SK_ERR_ARG;
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaStream_t bs = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join(size_t(count), nullptr);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int rc = SK_OK;
    try {
        CK(cudaSetDevice(plans[0]->device));
        CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (auto& e : join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        // every plan's stream starts after the caller's work; statuses cleared
        for (int i = 0; i < count; ++i) {
            enter(plans[i], stream);
            clear_status(plans[i]);
        }
        std::vector<int64_t> kernels(size_t(count), 0);
        if (max_iter > 0) {
            // one iteration of every plan as parallel branches of one graph
            CK(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
            try {
                CK(cudaEventRecord(fork, bs));
                for (int i = 0; i < count; ++i) {
                    sk_plan* P = plans[i];
                    CK(cudaStreamWaitEvent(P->ps, fork, 0));
                    const int64_t before = P->launches;
                    run_iteration(P);
                    kernels[size_t(i)] = P->launches - before;
                    P->launches = before;
                    CK(cudaEventRecord(join[size_t(i)], P->ps));
                    CK(cudaStreamWaitEvent(bs, join[size_t(i)], 0));
                }
            } catch (...) {
                cudaStreamEndCapture(bs, &g);
                throw;
            }
            CK(cudaStreamEndCapture(bs, &g));
            CK(cudaGraphInstantiate(&ge, g, 0));
            // the replays start after every plan's preparation above
            for (int i = 0; i < count; ++i) {
                CK(cudaEventRecord(join[size_t(i)], plans[i]->ps));
                CK(cudaStreamWaitEvent(bs, join[size_t(i)], 0));
            }
            for (int k = 0; k < max_iter; ++k) CK(cudaGraphLaunch(ge, bs));
            CK(cudaEventRecord(fork, bs));
        }
        for (int i = 0; i < count; ++i) {
            sk_plan* P = plans[i];
            if (max_iter > 0) CK(cudaStreamWaitEvent(P->ps, fork, 0));
            P->iters += max_iter;
            P->launches += kernels[size_t(i)] * max_iter;
            if (results) {
                sk_result* res = results + i;
                std::memset(res, 0, sizeof(*res));
                if (P->precision == SK_FP32)
                    final_report<float>(P, res);
                else
                    final_report<double>(P, res);
                res->iters = max_iter;
                const int st = read_status(P);
                if (st & 1) rc = SK_ERR_UNDERFLOW;
                if (st & 4) rc = SK_ERR_TIMEOUT;
            }
            leave(P, stream);
        }
        CK(cudaStreamSynchronize(cs));
    } catch (const Fail& f) {
        rc = fail_code(f);
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    for (auto& e : join)
        if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (bs) {
        cudaStreamSynchronize(bs);
        cudaStreamDestroy(bs);
    }
    return rc;
}

int sk_grad(sk_plan* P, double* grad_a, double* grad_b, double* grad_x, double* grad_y, void* stream) {
    if (!P) return SK_ERR_ARG;
    if ((grad_x || grad_y) && P->r != 2.0) return SK_ERR_UNSUPPORTED;
    try {
        enter(P, stream);
        if (grad_a) dual_variable_out(P, P->X, grad_a);
        if (grad_b) dual_variable_out(P, P->Y, grad_b);
        if (P->precision == SK_FP32) {
            if (grad_x) position_gradient<float>(P, P->Y, P->X, grad_x);
            if (grad_y) position_gradient<float>(P, P->X, P->Y, grad_y);
        } else {
            if (grad_x) position_gradient<double>(P, P->Y, P->X, grad_x);
            if (grad_y) position_gradient<double>(P, P->X, P->Y, grad_y);
        }
        leave(P, stream);
        CK(cudaStreamSynchronize(P->ps));
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int sk_divergence(int d, int64_t n, const double* x, const double* a, int64_t m, const double* y, const double* b,
                  double eps, double r, const sk_nfft_params* prm, int max_iter, double tol, double* host_out,
                  double* grad_a, double* grad_b, double* grad_x, double* grad_y, void* stream) {
    if (!host_out || max_iter < 0 || d < 1 || d > 3 || n < 1 || m < 1) return SK_ERR_ARG;
    if ((grad_x || grad_y) && r != 2.0) return SK_ERR_UNSUPPORTED;
    const bool want_grad = grad_a || grad_b || grad_x || grad_y;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // s(P, P~), s(P, P), s(P~, P~): three plans, each solved like sk_solve
    const double* cx[3] = {x, x, y};
    const double* ca[3] = {a, a, b};
    const double* cy[3] = {y, x, y};
    const double* cb[3] = {b, a, b};
    const int64_t cn[3] = {n, n, m}, cm[3] = {m, n, m};
    double val[3] = {0.0, 0.0, 0.0};
    int worst = SK_OK;
    // device accumulators of the gradient (caller order) and one term's parts
    std::vector<void*> mem;
    auto dev = [&](int64_t count) -> double* {
        void* p = nullptr;
        if (cudaMalloc(&p, size_t(std::max<int64_t>(count, 1)) * sizeof(double)) != cudaSuccess) return nullptr;
        mem.push_back(p);
        return static_cast<double*>(p);
    };
    auto release = [&]() {
        for (void* p : mem) cudaFree(p);
        mem.clear();
    };
    double *acc_a = nullptr, *acc_b = nullptr, *acc_x = nullptr, *acc_y = nullptr;
    double *t1 = nullptr, *t2 = nullptr, *tx1 = nullptr, *tx2 = nullptr;
    if (want_grad) {
        const int64_t nm = std::max(n, m);
        acc_a = dev(n), acc_b = dev(m), acc_x = dev(n * d), acc_y = dev(m * d);
        t1 = dev(nm), t2 = dev(nm), tx1 = dev(nm * d), tx2 = dev(nm * d);
        if (!acc_a || !acc_b || !acc_x || !acc_y || !t1 || !t2 || !tx1 || !tx2) {
            release();
            return SK_ERR_NOMEM;
        }
    }
    for (int k = 0; k < 3; ++k) {
        sk_plan* P = nullptr;
        int st = sk_init(&P, d, cn[k], cx[k], ca[k], cm[k], cy[k], cb[k], eps, r, prm, stream);
        if (st != SK_OK) {
            release();
            return st;
        }
        sk_result res{};
        st = sk_solve(P, max_iter, tol, 0, nullptr, nullptr, &res, stream);
        if (st == SK_OK || st == SK_ERR_NOT_CONVERGED) {
            if (st == SK_ERR_NOT_CONVERGED) worst = st;
            val[k] = res.s;
            if (want_grad) {
                // s(P, P~) -> the accumulators; the self terms subtract half of
                // both sides' gradients (every point is source and target)
                const bool posg = grad_x || grad_y;
                if (k == 0)
                    st = sk_grad(P, acc_a, acc_b, posg ? acc_x : nullptr, posg ? acc_y : nullptr, stream);
                else
                    st = sk_grad(P, t1, t2, posg ? tx1 : nullptr, posg ? tx2 : nullptr, stream);
                if (st == SK_OK && k > 0) {
                    const int64_t c = cn[k];
                    k_sub_half_sum<<<unsigned((c + 255) / 256), 256, 0, cs>>>(k == 1 ? acc_a : acc_b, t1, t2, c);
                    if (posg)
                        k_sub_half_sum<<<unsigned((c * d + 255) / 256), 256, 0, cs>>>(k == 1 ? acc_x : acc_y, tx1,
                                                                                      tx2, c * d);
                    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(cs) != cudaSuccess)
                        st = SK_ERR_CUDA;
                }
            }
        }
        sk_destroy(P);
        if (st != SK_OK && st != SK_ERR_NOT_CONVERGED) {
            release();
            return st;
        }
    }
    int rc = worst;
    if (want_grad) {
        const double* src[4] = {acc_a, acc_b, acc_x, acc_y};
        double* dst[4] = {grad_a, grad_b, grad_x, grad_y};
        const int64_t cnt[4] = {n, m, n * d, m * d};
        for (int k = 0; k < 4; ++k)
            if (dst[k] && cudaMemcpyAsync(dst[k], src[k], size_t(cnt[k]) * sizeof(double), cudaMemcpyDefault, cs) !=
                              cudaSuccess)
                rc = SK_ERR_CUDA;
        if (cudaStreamSynchronize(cs) != cudaSuccess) rc = SK_ERR_CUDA;
        release();
        if (rc == SK_ERR_CUDA) return rc;
    }
    host_out[0] = val[0] - 0.5 * (val[1] + val[2]);
    host_out[1] = val[0];
    host_out[2] = val[1];
    host_out[3] = val[2];
    return rc;
}

int sk_get_state(sk_plan* P, double* u, double* v, int* iters) {
    if (!P) return SK_ERR_ARG;
    try {
        CK(cudaSetDevice(P->device));
        write_out(P, P->X, P->X.scal, u);
        write_out(P, P->Y, P->Y.scal, v);
        CK(cudaStreamSynchronize(P->ps));
        if (iters) *iters = P->iters;
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int sk_set_state(sk_plan* P, const double* u, const double* v, int iters) {
    if (!P || iters < 0) return SK_ERR_ARG;
    try {
        CK(cudaSetDevice(P->device));
        if (u)
            read_in(P, P->X, u, P->X.scal);
        else if (!v)
            k_fill<<<nblk(P->X.n), 256, 0, P->ps>>>(P->X.scal, P->X.n, 1.0);
        if (v)
            read_in(P, P->Y, v, P->Y.scal);
        else if (!u)
            k_fill<<<nblk(P->Y.n), 256, 0, P->ps>>>(P->Y.scal, P->Y.n, 1.0);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(P->ps));
        P->iters = iters;
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int sk_plan_info(const sk_plan* P, sk_info* info) {
    if (!P || !info) return SK_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->d = P->d;
    info->n = P->n;
    info->m = P->m;
    info->N = P->N;
    info->n_os = P->n_os;
    info->m_w = P->prm.m_w;
    info->p = P->prm.p;
    info->precision = P->precision;
    info->nearfield = P->nearfield;
    info->eps = P->eps;
    info->r = P->r;
    info->eps_scaled = P->eps_s;
    for (int t = 0; t < 3; ++t) info->center[t] = P->center[t];
    info->scale = P->scale;
    info->eps_B = P->prm.eps_B;
    info->eps_I = P->prm.eps_I;
    info->n_subproblems_x = P->X.nsub;
    info->n_subproblems_y = P->Y.nsub;
    info->device_bytes = P->bytes;
    info->tensor_cores = P->tc ? 1 : 0;
    info->fft_planes = P->fft.planes ? 1 : 0;
    return SK_OK;
}

int sk_fourier_coefficients(sk_plan* P, double* out, void* stream) {
    if (!P || !out) return SK_ERR_ARG;
    try {
        enter(P, stream);
        int64_t nN = 1;
        for (int t = 0; t < P->d; ++t) nN *= P->N;
        CK(cudaMemcpyAsync(out, P->bk, size_t(nN) * sizeof(double), cudaMemcpyDefault, P->ps));
        CK(cudaStreamSynchronize(P->ps));
        leave(P, stream);
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int sk_adjoint_nfft(sk_plan* P, int set, const double* w, double* fhat, void* stream) {
    if (!P || !w || !fhat || (set != SK_SET_X && set != SK_SET_Y)) return SK_ERR_ARG;
    try {
        enter(P, stream);
        Cloud& c = set == SK_SET_X ? P->X : P->Y;
        read_in(P, c, w, c.work);
        int64_t total = 1;
        for (int t = 0; t < P->d; ++t) total *= (2 * P->h + 1);
        const bool dev = is_device_ptr(fhat);
        double* dout = fhat;
        if (!dev) CK(cudaMallocAsync(reinterpret_cast<void**>(&dout), size_t(2 * total) * sizeof(double), P->ps));
        if (P->precision == SK_FP32) {
            spread_into_grid<float>(P, c, c.work);
            CK(launch_fft_adjoint<float>(P->fft, dout, P->ps, &P->launches));
        } else {
            spread_into_grid<double>(P, c, c.work);
            CK(launch_fft_adjoint<double>(P->fft, dout, P->ps, &P->launches));
        }
        if (!dev) {
            CK(cudaMemcpyAsync(fhat, dout, size_t(2 * total) * sizeof(double), cudaMemcpyDeviceToHost, P->ps));
            CK(cudaFreeAsync(dout, P->ps));
            CK(cudaStreamSynchronize(P->ps));
        }
        leave(P, stream);
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

namespace {
// The NFFT of a device-resident Hermitian coefficient array `din` at cloud c
// into f (host or device, caller order).
void nfft_device(sk_plan* P, Cloud& c, const double* din, double* f) {
    const bool host_out = !is_device_ptr(f);
    Epilogue e = make_epilogue(P, EPI_APPLY, c, 0, host_out ? c.stage : f);
    if (P->precision == SK_FP32) {
        CK(launch_fft_forward<float>(P->fft, din, P->ps, &P->launches));
        interp_from_grid<float>(P, c, e);
    } else {
        CK(launch_fft_forward<double>(P->fft, din, P->ps, &P->launches));
        interp_from_grid<double>(P, c, e);
    }
    if (host_out) {
        CK(cudaMemcpyAsync(f, c.stage, size_t(c.n) * sizeof(double), cudaMemcpyDeviceToHost, P->ps));
        CK(cudaStreamSynchronize(P->ps));
    }
}

int64_t spectrum_size(const sk_plan* P) {
    int64_t total = 1;
    for (int t = 0; t < P->d; ++t) total *= (2 * P->h + 1);
    return total;
}
}  // namespace

int sk_nfft(sk_plan* P, int set, const double* fhat, double* f, void* stream) {
    if (!P || !fhat || !f || (set != SK_SET_X && set != SK_SET_Y)) return SK_ERR_ARG;
    try {
        enter(P, stream);
        Cloud& c = set == SK_SET_X ? P->X : P->Y;
        const int64_t total = spectrum_size(P);
        const double* din = fhat;
        double* tmp = nullptr;
        if (!is_device_ptr(fhat)) {
            CK(cudaMallocAsync(reinterpret_cast<void**>(&tmp), size_t(2 * total) * sizeof(double), P->ps));
            CK(cudaMemcpyAsync(tmp, fhat, size_t(2 * total) * sizeof(double), cudaMemcpyHostToDevice, P->ps));
            din = tmp;
        }
        nfft_device(P, c, din, f);
        if (tmp) CK(cudaFreeAsync(tmp, P->ps));
        leave(P, stream);
    } catch (const Fail& f2) {
        return fail_code(f2);
    }
    return SK_OK;
}

int sk_spectrum(sk_plan* P, int set, const double* w, double* spec, void* stream) {
    if (P && P->nearfield) return SK_ERR_UNSUPPORTED;
    return sk_adjoint_nfft(P, set, w, spec, stream);
}

int sk_apply_spectrum(sk_plan* P, int set, const double* spec, double* out, void* stream) {
    if (!P || !spec || !out || (set != SK_SET_X && set != SK_SET_Y)) return SK_ERR_ARG;
    if (P->nearfield) return SK_ERR_UNSUPPORTED;
    try {
        enter(P, stream);
        Cloud& c = set == SK_SET_X ? P->X : P->Y;
        const int64_t total = spectrum_size(P);
        if (!P->spec_tmp) P->spec_tmp = static_cast<double*>(dalloc(P, size_t(2 * total) * sizeof(double)));
        const double* din = spec;
        if (!is_device_ptr(spec)) {
            CK(cudaMemcpyAsync(P->spec_tmp, spec, size_t(2 * total) * sizeof(double), cudaMemcpyHostToDevice,
                               P->ps));
            din = P->spec_tmp;
        }
        k_times_bk<<<nblk(total), 256, 0, P->ps>>>(din, P->bk, P->d, P->h, P->spec_tmp);
        CK(cudaGetLastError());
        ++P->launches;
        nfft_device(P, c, P->spec_tmp, out);
        leave(P, stream);
    } catch (const Fail& f2) {
        return fail_code(f2);
    }
    return SK_OK;
}

int sk_stage_times(sk_plan* P, int enable, double* ms_out, int64_t* counts_out) {
    if (!P || (enable != 0 && enable != 1)) return SK_ERR_ARG;
    try {
        CK(cudaSetDevice(P->device));
        stage_resolve(P);
        if (ms_out)
            for (int s = 0; s < SK_NSTAGES; ++s) ms_out[s] = P->stage_ms[s];
        if (counts_out)
            for (int s = 0; s < SK_NSTAGES; ++s) counts_out[s] = P->stage_cnt[s];
        for (int s = 0; s < SK_NSTAGES; ++s) {
            P->stage_ms[s] = 0.0;
            P->stage_cnt[s] = 0;
        }
        P->timing = enable == 1;
    } catch (const Fail& f) {
        return fail_code(f);
    }
    return SK_OK;
}

int64_t sk_launch_count(const sk_plan* P) { return P ? P->launches : -1; }

}  // extern "C"
