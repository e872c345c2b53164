// Plan-time and bookkeeping kernels: input validation reductions, scaling
// into the torus and bin sorting, the coefficient table of the regularized
// kernel (Eq. (ansatz_NFFT)), the window transform, twiddles, and the FP64
// gathers / scatters / reductions of the solver.
#include "sk_plan_kernels.cuh"

namespace sk {

// ------------------------------------------------------------ reductions
// Per-block partials of (min_t, max_t for t < d, count of non-finite values).
__global__ void k_point_bounds(const double* __restrict__ x, int64_t n, int d, double* __restrict__ partial) {
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    double bad = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        for (int t = 0; t < d; ++t) {
            const double v = x[i * d + t];
            if (!isfinite(v)) { bad += 1.0; continue; }
            mn[t] = fmin(mn[t], v);
            mx[t] = fmax(mx[t], v);
        }
    }
    __shared__ double s[7][256];
    for (int t = 0; t < 3; ++t) { s[t][threadIdx.x] = mn[t]; s[3 + t][threadIdx.x] = mx[t]; }
    s[6][threadIdx.x] = bad;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int t = 0; t < 3; ++t) {
                s[t][threadIdx.x] = fmin(s[t][threadIdx.x], s[t][threadIdx.x + w]);
                s[3 + t][threadIdx.x] = fmax(s[3 + t][threadIdx.x], s[3 + t][threadIdx.x + w]);
            }
            s[6][threadIdx.x] += s[6][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int f = 0; f < 7; ++f) partial[blockIdx.x * 7 + f] = s[f][0];
}

// Per-block partials of (max |x_i - c|^2).
__global__ void k_point_radius(const double* __restrict__ x, int64_t n, int d, double c0, double c1, double c2,
                               double* __restrict__ partial) {
    const double c[3] = {c0, c1, c2};
    double mx = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        double r2 = 0.0;
        for (int t = 0; t < d; ++t) {
            const double dd = x[i * d + t] - c[t];
            r2 += dd * dd;
        }
        mx = fmax(mx, r2);
    }
    __shared__ double s[256];
    s[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// Per-block partials of (sum w, min w, count non-finite, -sum w log w).
__global__ void k_weight_stats(const double* __restrict__ w, int64_t n, double* __restrict__ partial) {
    double sum = 0.0, mn = INFINITY, bad = 0.0, ent = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double v = w[i];
        if (!isfinite(v)) { bad += 1.0; continue; }
        sum += v;
        mn = fmin(mn, v);
        if (v > 0.0) ent -= v * log(v);
    }
    __shared__ double s[4][256];
    s[0][threadIdx.x] = sum;
    s[1][threadIdx.x] = mn;
    s[2][threadIdx.x] = bad;
    s[3][threadIdx.x] = ent;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            s[0][threadIdx.x] += s[0][threadIdx.x + k];
            s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + k]);
            s[2][threadIdx.x] += s[2][threadIdx.x + k];
            s[3][threadIdx.x] += s[3][threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int f = 0; f < 4; ++f) partial[blockIdx.x * 4 + f] = s[f][0];
}

// Per-block partial of sum_i marg_i log(scal_i).
// sum_i a_i log u_i (as_is = 0) or sum_i a_i scal_i (as_is = 1: scal holds
// log-domain dual variables), points without mass skipped.
__global__ void k_sum_marg_log(const double* __restrict__ marg, const double* __restrict__ scal, int64_t n,
                               int as_is, double* __restrict__ partial) {
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double a = marg[i];
        if (a > 0.0) acc += a * (as_is ? scal[i] : log(scal[i]));
    }
    __shared__ double s[256];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// Combine nblocks rows of nf fields; op[f] = 0 sum, 1 min, 2 max.  One block
// of 32 nf threads: warp f takes field f, each lane combines rows lane,
// lane + 32, ... (all its loads in flight at once), then the lanes combine in
// a fixed butterfly order, so the result does not depend on timing.
__global__ void k_combine(const double* __restrict__ partial, int nblocks, int nf, int op0, int op1, int op2,
                          int op3, int op4, int op5, int op6, double* __restrict__ out) {
    const int ops[7] = {op0, op1, op2, op3, op4, op5, op6};
    const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (f >= nf) return;
    const int op = ops[f];
    auto comb = [op](double a, double b) { return op == 0 ? a + b : (op == 1 ? fmin(a, b) : fmax(a, b)); };
    double acc = op == 0 ? 0.0 : (op == 1 ? INFINITY : -INFINITY);
    for (int b = lane; b < nblocks; b += 32) acc = comb(acc, partial[b * nf + f]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = comb(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) out[f] = acc;
}

// ------------------------------------------------------------ bin sorting
// Sort key of a point: its bin (bins of B[0] x .. x B[d-1] cells, last axis
// fastest) times the cells per bin, plus its cell inside the bin (last axis
// fastest; in 2-D the y cell is the major one).  Sorting by this key keeps
// every bin contiguous and, inside a 3-D bin, every column of cells along the
// last axis contiguous.
template <typename T>
__global__ void k_prepare_points(const double* __restrict__ x, int64_t n, int d, double c0, double c1, double c2,
                                 double scale, int n_os, int B0, int B1, int B2, int nb0, int nb1, int nb2, int m,
                                 T* __restrict__ u0, T* __restrict__ u1, T* __restrict__ u2,
                                 int* __restrict__ key, int* __restrict__ count, int* __restrict__ status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c[3] = {c0, c1, c2};
    const int nb[3] = {nb0, nb1, nb2};
    const int B[3] = {B0, B1, B2};
    T* u[3] = {u0, u1, u2};
    int bin = 0, loc = 0, bvol = 1, lx = 0;
    bool ok = true;
    for (int t = 0; t < d; ++t) {
        const double z = scale * (x[i * d + t] - c[t]) + 0.5;
        const T ut = T(double(n_os) * z);
        u[t][i] = ut;
        const T fl = floor(ut);
        int f = (fl > T(-1e9) && fl < T(1e9)) ? int(fl) : -1000000000;
        ok = ok && (f - (m - 1) >= 0) && (f + m <= n_os - 1);
        if (f < 0) f = 0;
        if (f > n_os - 1) f = n_os - 1;
        int bt = f / B[t];
        bt = bt >= nb[t] ? nb[t] - 1 : bt;
        bin = bin * nb[t] + bt;
        loc = loc * B[t] + (f - bt * B[t]);
        if (t == 0) lx = f - bt * B[t];
        bvol *= B[t];
    }
    // 2-D: inside a bin the y-cell is the major key (the strip kernels walk a
    // bin's points in y order); otherwise the last axis is fastest
    if (d == 2) loc = (loc - lx * B[1]) * B[0] + lx;
    if (!ok) atomicOr(status, 2);
    const int k = bin * bvol + loc;
    key[i] = k;
    atomicAdd(&count[k], 1);
}

// Exclusive scan of n ints into out[0..n] (out[n] = total) in three passes:
// per-block scans of kScanBlock elements, a scan of the block totals (one
// block), and the addition of the block offsets.
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanBlock = kScanThreads * kScanPerThread;

__global__ void k_scan_local(const int* __restrict__ in, int* __restrict__ out, int n, int* __restrict__ totals) {
    __shared__ int s[kScanThreads];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPerThread;
    int v[kScanPerThread];
    int sum = 0;
    for (int k = 0; k < kScanPerThread; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        sum += v[k];
    }
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const int add = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    int run = s[threadIdx.x] - sum;
    for (int k = 0; k < kScanPerThread; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) totals[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_totals(int* __restrict__ totals, int nblocks, int* __restrict__ grand) {
    __shared__ int s[kScanThreads];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
        const int i = b0 + threadIdx.x;
        const int v = i < nblocks ? totals[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < kScanThreads; off <<= 1) {
            const int add = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nblocks) totals[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ totals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += totals[i / kScanBlock];
}

void launch_scan_exclusive(const int* in, int* out, int n, int* scratch, cudaStream_t s) {
    const int nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_local<<<nb, kScanThreads, 0, s>>>(in, out, n, scratch);
    k_scan_totals<<<1, kScanThreads, 0, s>>>(scratch, nb, out + n);
    k_scan_add<<<unsigned((n + 255) / 256), 256, 0, s>>>(out, n, scratch);
}

int scan_scratch_ints(int n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

__global__ void k_scatter_perm(const int* __restrict__ key, int64_t n, const int* __restrict__ start,
                               int* __restrict__ cursor, int* __restrict__ perm) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    const int pos = start[k] + atomicAdd(&cursor[k], 1);
    perm[pos] = int(i);
}

template <typename T>
__global__ void k_gather_points(const int* __restrict__ perm, int64_t n, int d, const T* __restrict__ i0,
                                const T* __restrict__ i1, const T* __restrict__ i2, T* __restrict__ o0,
                                T* __restrict__ o1, T* __restrict__ o2) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = perm[i];
    o0[i] = i0[p];
    if (d > 1) o1[i] = i1[p];
    if (d > 2) o2[i] = i2[p];
}

// bin_start[b] = key_start[b * bvol], b = 0..nbins
__global__ void k_bin_starts(const int* __restrict__ key_start, int nbins, int bvol, int* __restrict__ bin_start) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b <= nbins) bin_start[b] = key_start[int64_t(b) * bvol];
}

__global__ void k_count_subs(const int* __restrict__ bin_start, int nbins, int maxpts, int* __restrict__ nsub) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int cnt = bin_start[b + 1] - bin_start[b];
    nsub[b] = (cnt + maxpts - 1) / maxpts;
}

__global__ void k_fill_subs(const int* __restrict__ bin_start, const int* __restrict__ sub_off, int nbins,
                            int maxpts, int* __restrict__ sub_start, int* __restrict__ sub_count,
                            int* __restrict__ sub_bin) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int s0 = bin_start[b], cnt = bin_start[b + 1] - s0;
    const int o = sub_off[b], ns = sub_off[b + 1] - o;
    for (int k = 0; k < ns; ++k) {
        sub_start[o + k] = s0 + k * maxpts;
        sub_count[o + k] = min(maxpts, cnt - k * maxpts);
        sub_bin[o + k] = b;
    }
}

// Column tasks of the 3-D column kernels: a non-empty bin with up to maxpts
// points is one task over all its ncol columns; a heavier bin is split into
// up to ncol tasks over equal ranges of its columns.
__global__ void k_count_tasks(const int* __restrict__ bin_start, int nbins, int maxpts, int ncol,
                              int* __restrict__ ntask) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int cnt = bin_start[b + 1] - bin_start[b];
    ntask[b] = cnt == 0 ? 0 : min(ncol, (cnt + maxpts - 1) / maxpts);
}

__global__ void k_fill_tasks(const int* __restrict__ ntask_off, int nbins, int ncol, int* __restrict__ task) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int o = ntask_off[b], nt = ntask_off[b + 1] - o;
    for (int k = 0; k < nt; ++k) {
        task[3 * (o + k) + 0] = b;
        task[3 * (o + k) + 1] = (k * ncol) / nt;
        task[3 * (o + k) + 2] = ((k + 1) * ncol) / nt;
    }
}

// Points in each (bin, column) pair of the 3-D column kernels: a column is the
// bz cells of one (x, y) cell position inside a bin, consecutive sort keys.
__global__ void k_col_counts(const int* __restrict__ key_start, int nbins, int bvol, int ncol, int bz,
                             int* __restrict__ count) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(nbins) * ncol) return;
    const int64_t k0 = (i / ncol) * bvol + (i % ncol) * bz;
    count[i] = key_start[k0 + bz] - key_start[k0];
}

// ------------------------------------------------------------ coefficient table
// K_R(l/N) for l in {-N/2..N/2-1}^d, stored at index l + N/2 per dimension.
__global__ void k_sample_kernel(double* __restrict__ out, int N, int d, KernelParams kp) {
    int64_t total = 1;
    for (int t = 0; t < d; ++t) total *= N;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int64_t rem = idx;
    double rho2 = 0.0;
    for (int t = d - 1; t >= 0; --t) {
        const int l = int(rem % N) - N / 2;
        rem /= N;
        const double y = double(l) / double(N);
        rho2 += y * y;
    }
    const double v = kr_value(sqrt(rho2), kp);
    out[idx] = v;
}

// One cosine-DFT pass along `axis` of an N^d array indexed by l + N/2:
// out[.. k ..] = sum_l in[.. l ..] cos(2 pi k l / N), k, l in -N/2..N/2-1.
// (The samples are even in every coordinate, so the sine part vanishes.)
__global__ void k_cos_dft_axis(const double* __restrict__ in, double* __restrict__ out, int N, int d, int axis,
                               const double* __restrict__ costab) {
    int64_t total = 1;
    for (int t = 0; t < d; ++t) total *= N;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int64_t stride = 1;
    for (int t = d - 1; t > axis; --t) stride *= N;
    const int ka = int((idx / stride) % N);
    const int64_t base = idx - int64_t(ka) * stride;
    const int k = ka - N / 2;
    double acc = 0.0;
    for (int la = 0; la < N; ++la) {
        const int l = la - N / 2;
        int j = (k * l) % N;
        if (j < 0) j += N;
        acc += in[base + int64_t(la) * stride] * costab[j];
    }
    out[idx] = acc;
}

__global__ void k_cos_table(double* __restrict__ c, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) c[j] = cospi(2.0 * double(j) / double(N));
}

// psihat_n(k / n_os) for k = -h..h: the Fourier transform of the window
// normalized to 1 at 0, pi m / sinh(beta m) * I_0(m sqrt(beta^2 - (2 pi k / n_os)^2)).
// I_0 by its power series sum_j ((x/2)^(2j)) / (j!)^2.
__global__ void k_window_transform(double* __restrict__ out, int h, int n_os, int m, double beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > 2 * h) return;
    const int k = i - h;
    const double w = 2.0 * M_PI * double(k) / double(n_os);
    const double arg = double(m) * sqrt(beta * beta - w * w);
    const double q = 0.25 * arg * arg;
    double term = 1.0, sum = 1.0;
    for (int j = 1; j < 400; ++j) {
        term *= q / (double(j) * double(j));
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    out[i] = M_PI * double(m) / sinh(beta * double(m)) * sum;
}

// M over the kept half spectrum: c_k b_k / prod_t psihat(k_t)^2, last axis k = 0..h,
// with c_k the weight of the real part of the sum over I_N (re_weight).
template <typename T>
__global__ void k_build_mult(T* __restrict__ M, int d, int h, const double* __restrict__ bk, double inv_norm,
                             const double* __restrict__ psihat) {
    const int K = 2 * h + 1, N = 2 * h;
    int64_t total = h + 1;
    for (int t = 0; t < d - 1; ++t) total *= K;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int k[3] = {0, 0, 0};
    int64_t rem = idx;
    k[d - 1] = int(rem % (h + 1));
    rem /= (h + 1);
    for (int t = d - 2; t >= 0; --t) { k[t] = int(rem % K) - h; rem /= K; }
    int64_t bi = 0;
    double c = inv_norm;
    for (int t = 0; t < d; ++t) {
        const int kt = k[t] == h ? -h : k[t];      // b is N-periodic: b_{N/2} = b_{-N/2}
        bi = bi * N + (kt + h);
        const double ph = psihat[k[t] + h];
        c /= ph * ph;
    }
    c *= re_weight(k, d, h);
    M[idx] = T(c * bk[bi]);
}

// ------------------------------------------------------------ vectors
__global__ void k_fill(double* __restrict__ p, int64_t n, double v) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_scale(double* __restrict__ p, int64_t n, double f) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) p[i] *= f;
}

// out[i] = in[perm[i]]: caller order -> sorted order
__global__ void k_gather(const double* __restrict__ in, const int* __restrict__ perm, int64_t n,
                         double* __restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[perm[i]];
}

// out[perm[i]] = in[i]: sorted order -> caller order
__global__ void k_scatter(const double* __restrict__ in, const int* __restrict__ perm, int64_t n,
                          double* __restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = in[i];
}

// Smallest and largest cell index per axis over the points (atomics on ints;
// out[0..2] start at INT_MAX, out[3..5] at INT_MIN).
template <typename T>
__global__ void k_cell_bounds(const T* __restrict__ u0, const T* __restrict__ u1, const T* __restrict__ u2,
                              int64_t n, int d, int* __restrict__ out) {
    const T* u[3] = {u0, u1, u2};
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        for (int t = 0; t < d; ++t) {
            const int f = int(floor(u[t][i]));
            mn[t] = min(mn[t], f);
            mx[t] = max(mx[t], f);
        }
    }
    for (int t = 0; t < d; ++t) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[t] = min(mn[t], __shfl_xor_sync(0xffffffffu, mn[t], o));
            mx[t] = max(mx[t], __shfl_xor_sync(0xffffffffu, mx[t], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&out[t], mn[t]);
            atomicMax(&out[3 + t], mx[t]);
        }
    }
}

__global__ void k_init_bounds(int* out) {
    if (threadIdx.x < 3) out[threadIdx.x] = INT_MAX;
    else if (threadIdx.x < 6) out[threadIdx.x] = INT_MIN;
}

// ------------------------------------------------------------ host launchers
template <typename T>
void launch_cell_bounds(void* const u[3], int64_t n, int d, int* out, cudaStream_t s) {
    k_cell_bounds<T><<<256, 256, 0, s>>>(static_cast<const T*>(u[0]), static_cast<const T*>(u[1]),
                                         static_cast<const T*>(u[2]), n, d, out);
}
template void launch_cell_bounds<float>(void* const[3], int64_t, int, int*, cudaStream_t);
template void launch_cell_bounds<double>(void* const[3], int64_t, int, int*, cudaStream_t);

template <typename T>
void launch_prepare_points(const double* x, int64_t n, int d, const double c[3], double scale, int n_os,
                           const int B[3], const int nb[3], int m, T* const u[3], int* key, int* count, int* status,
                           cudaStream_t s) {
    k_prepare_points<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(x, n, d, c[0], c[1], c[2], scale, n_os, B[0], B[1],
                                                                  B[2], nb[0], nb[1], nb[2], m, u[0], u[1], u[2], key,
                                                                  count, status);
}

template <typename T>
void launch_gather_points(const int* perm, int64_t n, int d, T* const in[3], T* const out[3], cudaStream_t s) {
    k_gather_points<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(perm, n, d, in[0], in[1], in[2], out[0], out[1],
                                                                 out[2]);
}

__global__ void k_times_bk(const double* __restrict__ spec, const double* __restrict__ bk, int d, int h,
                           double* __restrict__ out) {
    const int K = 2 * h + 1, N = 2 * h;
    int64_t total = 1;
    for (int t = 0; t < d; ++t) total *= K;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int64_t rem = idx, b = 0, stride = 1;
    for (int t = d - 1; t >= 0; --t) {
        int kt = int(rem % K) - h;
        rem /= K;
        if (kt == h) kt = -h;
        b += int64_t(kt + h) * stride;
        stride *= N;
    }
    const double f = bk[b];
    out[2 * idx] = spec[2 * idx] * f;
    out[2 * idx + 1] = spec[2 * idx + 1] * f;
}

template <typename T>
void launch_build_mult(T* M, int d, int h, const double* bk, double inv_norm, const double* psihat,
                       int64_t total, cudaStream_t s) {
    k_build_mult<T><<<unsigned((total + 255) / 256), 256, 0, s>>>(M, d, h, bk, inv_norm, psihat);
}


template void launch_prepare_points<float>(const double*, int64_t, int, const double[3], double, int, const int[3],
                                           const int[3], int, float* const[3], int*, int*, int*, cudaStream_t);
template void launch_prepare_points<double>(const double*, int64_t, int, const double[3], double, int, const int[3],
                                            const int[3], int, double* const[3], int*, int*, int*, cudaStream_t);
template void launch_gather_points<float>(const int*, int64_t, int, float* const[3], float* const[3], cudaStream_t);
template void launch_gather_points<double>(const int*, int64_t, int, double* const[3], double* const[3],
                                           cudaStream_t);
template void launch_build_mult<float>(float*, int, int, const double*, double, const double*, int64_t,
                                       cudaStream_t);
template void launch_build_mult<double>(double*, int, int, const double*, double, const double*, int64_t,
                                        cudaStream_t);

// ------------------------------------------------------------ log domain
// Per-block maxima of v (-inf for an empty block), for the shift of the
// log-domain weights.
__global__ void k_block_max(const double* __restrict__ v, int64_t n, double* __restrict__ partial) {
    double m = -INFINITY;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        m = fmax(m, v[i]);
    __shared__ double s[256];
    s[threadIdx.x] = m;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// Weights of a log-domain half-step: w_j = exp((g_j - shift) / eps - 1/2) with
// shift = max_j g_j (from the block maxima), so every weight is at most
// e^(-1/2) and none overflows; block 0 stores the shift for the epilogue.  FP32
// plans evaluate exp(x) as 2^k exp(x - k ln 2), the reduced argument in FP32.
__global__ void k_log_weights(const double* __restrict__ g, int64_t n, const double* __restrict__ partial,
                              int nparts, double lam, int fp32, double* __restrict__ w, double* __restrict__ shift) {
    __shared__ double s[256];
    double m = -INFINITY;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) m = fmax(m, partial[k]);
    s[threadIdx.x] = m;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + k]);
        __syncthreads();
    }
    const double sh = isfinite(s[0]) ? s[0] : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *shift = sh;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double x = lam * (g[i] - sh) - 0.5;
        double v;
        if (!(x > -745.0)) {
            v = 0.0;
        } else if (fp32) {
            const double k = rint(x * 1.4426950408889634);
            const float red = float(fma(-k, 0.69314718055994530942, x));
            v = double(ldexpf(expf(red), int(k)));
        } else {
            v = exp(x);
        }
        w[i] = v;
    }
}

// Conversion of a state between the domains: beta = eps (log u + 1/2)
// (to_log) or u = exp(beta / eps - 1/2), the substitution of Eq. (27).
__global__ void k_convert_domain(double* __restrict__ v, int64_t n, double eps, int to_log) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) v[i] = to_log ? eps * (log(v[i]) + 0.5) : exp(v[i] / eps - 0.5);
}

// ------------------------------------------------------------ gradient
// acc[i] -= (p[i] + q[i]) / 2: a self term's two sides in the divergence's gradient.
__global__ void k_sub_half_sum(double* __restrict__ acc, const double* __restrict__ p, const double* __restrict__ q,
                               int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) acc[i] -= 0.5 * (p[i] + q[i]);
}


// Dual variable of a marginal constraint from its scaling vector (or the
// dual variables themselves, as_is: the log domain), in caller order: beta_i = eps (1/2 + log u_i), the substitution alpha_i =
// exp(lambda beta_i - 1/2) of Eq. (27) inverted (lambda = 1 / eps).
__global__ void k_dual_variable(const double* __restrict__ scal, const int* __restrict__ perm, int64_t n, double eps,
                                int as_is, double* __restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = as_is ? scal[i] : eps * (0.5 + log(scal[i]));
}

// w_j = v_j (y_jt - c_t): a scaling vector times one coordinate relative to
// the plan's centre, from grid units u = n_os (s (y - c) + 1/2).
template <typename T>
__global__ void k_weighted_coord(const double* __restrict__ scal, const T* __restrict__ coord, int64_t n,
                                 double inv_nos, double inv_s, double* __restrict__ w) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) w[i] = scal[i] * ((double(coord[i]) * inv_nos - 0.5) * inv_s);
}

// Position gradient for r = 2, coordinate t, in caller order (row-major n x d):
// sum_j pi_ij 2 (x_it - y_jt) = 2 u_i ((x_it - c_t) (K v)_i - (K (v (y_t - c_t)))_i).
// In the log domain scal holds beta and the products were formed with the
// shifted weights, so the prefactor is u_i e^(lam shift) = exp(lam (beta_i + shift) - 1/2).
template <typename T>
__global__ void k_position_gradient(const double* __restrict__ scal, const T* __restrict__ coord,
                                    const double* __restrict__ t0, const double* __restrict__ tt,
                                    const int* __restrict__ perm, int64_t n, int d, int t, double inv_nos,
                                    double inv_s, const double* __restrict__ log_shift, double lam,
                                    double* __restrict__ grad) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xc = (double(coord[i]) * inv_nos - 0.5) * inv_s;
    const double u = log_shift ? exp(lam * (scal[i] + *log_shift) - 0.5) : scal[i];
    grad[int64_t(perm[i]) * d + t] = 2.0 * u * (xc * t0[i] - tt[i]);
}

template <typename T>
void launch_weighted_coord(const double* scal, const void* coord, int64_t n, double inv_nos, double inv_s, double* w,
                           cudaStream_t s) {
    k_weighted_coord<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(scal, static_cast<const T*>(coord), n, inv_nos, inv_s,
                                                                  w);
}

template <typename T>
void launch_position_gradient(const double* scal, const void* coord, const double* t0, const double* tt,
                              const int* perm, int64_t n, int d, int t, double inv_nos, double inv_s,
                              const double* log_shift, double lam, double* grad, cudaStream_t s) {
    k_position_gradient<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(scal, static_cast<const T*>(coord), t0, tt, perm,
                                                                     n, d, t, inv_nos, inv_s, log_shift, lam, grad);
}

template void launch_weighted_coord<float>(const double*, const void*, int64_t, double, double, double*, cudaStream_t);
template void launch_weighted_coord<double>(const double*, const void*, int64_t, double, double, double*, cudaStream_t);
template void launch_position_gradient<float>(const double*, const void*, const double*, const double*, const int*,
                                              int64_t, int, int, double, double, const double*, double, double*,
                                              cudaStream_t);
template void launch_position_gradient<double>(const double*, const void*, const double*, const double*, const int*,
                                               int64_t, int, int, double, double, const double*, double, double*,
                                               cudaStream_t);

}  // namespace sk
