// Batched pencil FFTs on the oversampled grid (the O(N log N) part of
// Eq. (fastsum)) and the pointwise multiply by the kernel's Fourier
// coefficients, written for shared memory:
//
//   * Every block loads P pencils of length n (P * n = kFftElems complex
//     values) into shared memory, runs a radix-2 FFT there and writes back.
//     Pencils are padded to n+1 elements so that the loads, which walk the
//     pencils in parallel, do not collide in shared-memory banks.
//   * The grid is real, so the first pass packs two real rows into one complex
//     FFT and splits the result into two half spectra (k = 0..h along the
//     contiguous axis); the last inverse pass does the reverse.
//   * Only the 2h+1 = N+1 frequencies -N/2..N/2 survive the multiply, so the
//     forward passes keep only those and the inverse passes start from them.
//   * The multiply by c_k b_k / psihat(k)^2 is fused into the pass along
//     axis 0: forward FFT, multiply, inverse FFT in one kernel.
//
// Convolution pipeline (n = n_os, h = N/2, grid g[x][y][z] with z contiguous):
//   3-D: r2c(z) -> fwd(y, keep 2h+1) -> [fwd(x) * M, inv(x)] -> inv(y) -> c2r(z)
//   2-D: r2c(y) -> [fwd(x) * M, inv(x)] -> c2r(y)
//   1-D: r2c(x) -> * M -> c2r(x)            (the grid carries a second, zero row)
#include "sk_internal.cuh"

namespace sk {

enum { FULL = 0, CENTERED = 1 };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

__device__ __forceinline__ int bitrev(int v, int log2n) { return int(__brev(unsigned(v)) >> (32 - log2n)); }

// Decimation in time: input in bit-reversed order, output in natural order.
template <typename T, bool INV>
__device__ void fft_dit(typename Cplx<T>::type* buf, int ns, int n, int log2n, int P,
                        const typename Cplx<T>::type* __restrict__ tw) {
    using C = typename Cplx<T>::type;
    const int half = n >> 1;
    const int total = P * half;
    for (int s = 0; s < log2n; ++s) {
        __syncthreads();
        const int hs = 1 << s;
        const int shift = log2n - 1 - s;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int p = b >> (log2n - 1);
            const int j = b & (half - 1);
            const int k = j & (hs - 1);
            const int i0 = ((j >> s) << (s + 1)) + k;
            C w = tw[k << shift];
            if (INV) w.y = -w.y;
            C* base = buf + p * ns;
            const C a = base[i0];
            const C t = cmul(w, base[i0 + hs]);
            base[i0].x = a.x + t.x;
            base[i0].y = a.y + t.y;
            base[i0 + hs].x = a.x - t.x;
            base[i0 + hs].y = a.y - t.y;
        }
    }
    __syncthreads();
}

// Decimation in frequency: input in natural order, output in bit-reversed order.
template <typename T, bool INV>
__device__ void fft_dif(typename Cplx<T>::type* buf, int ns, int n, int log2n, int P,
                        const typename Cplx<T>::type* __restrict__ tw) {
    using C = typename Cplx<T>::type;
    const int half = n >> 1;
    const int total = P * half;
    for (int s = log2n - 1; s >= 0; --s) {
        __syncthreads();
        const int hs = 1 << s;
        const int shift = log2n - 1 - s;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int p = b >> (log2n - 1);
            const int j = b & (half - 1);
            const int k = j & (hs - 1);
            const int i0 = ((j >> s) << (s + 1)) + k;
            C w = tw[k << shift];
            if (INV) w.y = -w.y;
            C* base = buf + p * ns;
            const C a = base[i0];
            const C c = base[i0 + hs];
            C dlt;
            dlt.x = a.x - c.x;
            dlt.y = a.y - c.y;
            base[i0].x = a.x + c.x;
            base[i0].y = a.y + c.y;
            base[i0 + hs] = cmul(dlt, w);
        }
    }
    __syncthreads();
}

// Two real rows (2q, 2q+1) of length n -> two half spectra of length h+1.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_r2c_rows(const T* __restrict__ g, typename Cplx<T>::type* __restrict__ out,
                                                      int64_t npairs, int n, int log2n, int h,
                                                      const typename Cplx<T>::type* __restrict__ tw) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int P = kFftElems >> log2n;
    const int ns = n + 1;
    const int64_t q0 = int64_t(blockIdx.x) * P;
    for (int e = threadIdx.x; e < P * n; e += blockDim.x) {
        const int p = e >> log2n;
        const int l = e & (n - 1);
        const int64_t q = q0 + p;
        C z;
        z.x = T(0);
        z.y = T(0);
        if (q < npairs) {
            z.x = g[(2 * q) * n + l];
            z.y = g[(2 * q + 1) * n + l];
        }
        buf[p * ns + bitrev(l, log2n)] = z;
    }
    fft_dit<T, false>(buf, ns, n, log2n, P, tw);
    const int H = h + 1;
    for (int e = threadIdx.x; e < P * H; e += blockDim.x) {
        const int p = e / H;
        const int k = e - p * H;
        const int64_t q = q0 + p;
        if (q >= npairs) continue;
        const C zk = buf[p * ns + k];
        const C zm = buf[p * ns + ((n - k) & (n - 1))];
        C A, Bv;
        A.x = (zk.x + zm.x) * T(0.5);
        A.y = (zk.y - zm.y) * T(0.5);
        Bv.x = (zk.y + zm.y) * T(0.5);
        Bv.y = (zm.x - zk.x) * T(0.5);
        out[(2 * q) * H + k] = A;
        out[(2 * q + 1) * H + k] = Bv;
    }
}

// Two half spectra (rows 2q, 2q+1) -> two real rows, by Hermitian completion.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_c2r_rows(const typename Cplx<T>::type* __restrict__ in, T* __restrict__ g,
                                                      int64_t npairs, int n, int log2n, int h,
                                                      const typename Cplx<T>::type* __restrict__ tw) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int P = kFftElems >> log2n;
    const int ns = n + 1;
    const int H = h + 1;
    const int64_t q0 = int64_t(blockIdx.x) * P;
    for (int e = threadIdx.x; e < P * n; e += blockDim.x) {
        const int p = e >> log2n;
        const int pos = e & (n - 1);
        const int64_t q = q0 + p;
        C z;
        z.x = T(0);
        z.y = T(0);
        if (q < npairs) {
            const int k = pos <= (n >> 1) ? pos : pos - n;
            if (k >= 0 && k <= h) {
                C A = in[(2 * q) * H + k];
                C Bv = in[(2 * q + 1) * H + k];
                if (k == 0) { A.y = T(0); Bv.y = T(0); }
                z.x = A.x - Bv.y;
                z.y = A.y + Bv.x;
            } else if (k < 0 && -k <= h) {
                const C A = in[(2 * q) * H - k];
                const C Bv = in[(2 * q + 1) * H - k];
                z.x = A.x + Bv.y;
                z.y = Bv.x - A.y;
            }
        }
        buf[p * ns + pos] = z;
    }
    fft_dif<T, true>(buf, ns, n, log2n, P, tw);
    for (int e = threadIdx.x; e < P * n; e += blockDim.x) {
        const int p = e >> log2n;
        const int l = e & (n - 1);
        const int64_t q = q0 + p;
        if (q >= npairs) continue;
        const C v = buf[p * ns + bitrev(l, log2n)];
        g[(2 * q) * n + l] = v.x;
        g[(2 * q + 1) * n + l] = v.y;
    }
}

// Pencils along the middle axis of an (O, L, I) array: element k of pencil
// q = o*I + i sits at (o*L + k)*I + i.  FULL keeps all n entries along the
// axis; CENTERED stores frequencies -h..h at positions 0..2h.
template <typename T, int INM, int OUTM, bool INV>
__global__ void __launch_bounds__(256) k_fft_axis(const typename Cplx<T>::type* __restrict__ in,
                                                  typename Cplx<T>::type* __restrict__ out, int64_t O, int64_t I,
                                                  int n, int log2n, int h,
                                                  const typename Cplx<T>::type* __restrict__ tw) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int P = kFftElems >> log2n;
    const int ns = n + 1;
    const int64_t Q = O * I;
    const int64_t q0 = int64_t(blockIdx.x) * P;
    const int Lin = INM == FULL ? n : 2 * h + 1;
    const int Lout = OUTM == FULL ? n : 2 * h + 1;
    if (INM == CENTERED) {
        for (int e = threadIdx.x; e < P * ns; e += blockDim.x) {
            buf[e].x = T(0);
            buf[e].y = T(0);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < P * Lin; e += blockDim.x) {
        const int k = e / P;
        const int pl = e - k * P;
        const int64_t q = q0 + pl;
        if (q >= Q) continue;
        const int64_t o = q / I, i = q - o * I;
        const int pos = INM == FULL ? k : ((k - h) & (n - 1));
        buf[pl * ns + bitrev(pos, log2n)] = in[(o * Lin + k) * I + i];
    }
    fft_dit<T, INV>(buf, ns, n, log2n, P, tw);
    for (int e = threadIdx.x; e < P * Lout; e += blockDim.x) {
        const int k = e / P;
        const int pl = e - k * P;
        const int64_t q = q0 + pl;
        if (q >= Q) continue;
        const int64_t o = q / I, i = q - o * I;
        const int pos = OUTM == FULL ? k : ((k - h) & (n - 1));
        out[(o * Lout + k) * I + i] = buf[pl * ns + pos];
    }
}

// Pencils along axis 0 of an (n, I) array: forward FFT, multiply the kept
// frequencies by M[(k+h)*I + q] and zero the rest, inverse FFT, in place.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_axis0_convolve(typename Cplx<T>::type* __restrict__ data, int64_t I,
                                                            int n, int log2n, int h, const T* __restrict__ mult,
                                                            const typename Cplx<T>::type* __restrict__ tw) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int P = kFftElems >> log2n;
    const int ns = n + 1;
    const int64_t q0 = int64_t(blockIdx.x) * P;
    for (int e = threadIdx.x; e < P * n; e += blockDim.x) {
        const int k = e / P;
        const int pl = e - k * P;
        const int64_t q = q0 + pl;
        C v;
        v.x = T(0);
        v.y = T(0);
        if (q < I) v = data[int64_t(k) * I + q];
        buf[pl * ns + bitrev(k, log2n)] = v;
    }
    fft_dit<T, false>(buf, ns, n, log2n, P, tw);
    for (int e = threadIdx.x; e < P * n; e += blockDim.x) {
        const int pos = e / P;
        const int pl = e - pos * P;
        const int64_t q = q0 + pl;
        const int k = pos <= (n >> 1) ? pos : pos - n;
        C& v = buf[pl * ns + pos];
        if (q < I && k >= -h && k <= h) {
            const T mv = mult[int64_t(k + h) * I + q];
            v.x *= mv;
            v.y *= mv;
        } else {
            v.x = T(0);
            v.y = T(0);
        }
    }
    fft_dif<T, true>(buf, ns, n, log2n, P, tw);
    for (int e = threadIdx.x; e < P * n; e += blockDim.x) {
        const int k = e / P;
        const int pl = e - k * P;
        const int64_t q = q0 + pl;
        if (q < I) data[int64_t(k) * I + q] = buf[pl * ns + bitrev(k, log2n)];
    }
}

// 1-D: multiply the half spectrum of row 0 by M[k], k = 0..h.
template <typename T>
__global__ void k_mult_half(typename Cplx<T>::type* __restrict__ A1, int h, const T* __restrict__ mult) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= h) {
        A1[k].x *= mult[k];
        A1[k].y *= mult[k];
    }
}

// Half spectrum S (dims (2h+1)^(d-1) x (h+1)) -> full Hermitian FP64 array over
// {-h..h}^d, divided by the window transform prod_t psihat(k_t).
template <typename T>
__global__ void k_extract_adjoint(const typename Cplx<T>::type* __restrict__ S, int d, int h,
                                  const double* __restrict__ psihat, double* __restrict__ out) {
    const int K = 2 * h + 1;
    int64_t total = 1;
    for (int t = 0; t < d; ++t) total *= K;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int k[3] = {0, 0, 0};
    int64_t rem = idx;
    for (int t = d - 1; t >= 0; --t) { k[t] = int(rem % K) - h; rem /= K; }
    const bool flip = k[d - 1] < 0;
    int64_t s = 0;
    double den = 1.0;
    for (int t = 0; t < d; ++t) {
        const int kt = flip ? -k[t] : k[t];
        s = (t == d - 1) ? s * (h + 1) + kt : s * K + (kt + h);
        den *= psihat[k[t] + h];
    }
    const double re = double(S[s].x), im = double(S[s].y);
    out[2 * idx] = re / den;
    out[2 * idx + 1] = (flip ? -im : im) / den;
}

// Hermitian FP64 array over {-h..h}^d -> half spectrum S with the weights c_k
// and the window deconvolution folded in.
template <typename T>
__global__ void k_fill_forward(const double* __restrict__ fhat, int d, int h, const double* __restrict__ psihat,
                               typename Cplx<T>::type* __restrict__ S) {
    const int K = 2 * h + 1;
    int64_t total = h + 1;
    for (int t = 0; t < d - 1; ++t) total *= K;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int k[3] = {0, 0, 0};
    int64_t rem = idx;
    k[d - 1] = int(rem % (h + 1));
    rem /= (h + 1);
    for (int t = d - 2; t >= 0; --t) { k[t] = int(rem % K) - h; rem /= K; }
    int64_t f = 0;
    double c = 1.0;
    for (int t = 0; t < d; ++t) {
        f = f * K + (k[t] + h);
        c /= psihat[k[t] + h];
    }
    c *= re_weight(k, d, h);
    S[idx].x = T(fhat[2 * f] * c);
    S[idx].y = T(fhat[2 * f + 1] * c);
}

// ------------------------------------------------------------------ launchers

template <typename T>
static size_t fft_smem_bytes(int n) {
    const int P = kFftElems / n;
    return size_t(P) * size_t(n + 1) * sizeof(typename Cplx<T>::type);
}

// Largest dynamic shared memory any FFT launch of this precision can use:
// P (n+1) complex values with P n = kFftElems and n >= 16.
template <typename T>
static size_t fft_smem_max() {
    return size_t(kFftElems + kFftElems / 16) * sizeof(typename Cplx<T>::type);
}

// Opt a kernel into its largest shared-memory size once per device (the cache
// is per kernel: K is the kernel itself, not its type).
template <typename T, auto K>
static cudaError_t ensure_smem() {
    const size_t bytes = fft_smem_max<T>();
    if (bytes <= 48 * 1024) return cudaSuccess;
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured & (1ull << (dev & 63))) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) configured |= (1ull << (dev & 63));
    return e;
}

#define SK_TRY(x)                                   \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

template <typename T>
static cudaError_t run_r2c(const FftPlan& f, int64_t nrows, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const size_t bytes = fft_smem_bytes<T>(f.n);
    SK_TRY((ensure_smem<T, k_fft_r2c_rows<T>>()));
    const int64_t npairs = nrows / 2;
    const int P = kFftElems / f.n;
    k_fft_r2c_rows<T><<<unsigned((npairs + P - 1) / P), 256, bytes, s>>>(
        static_cast<const T*>(f.grid), static_cast<C*>(f.A1), npairs, f.n, f.log2n, f.h,
        static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t run_c2r(const FftPlan& f, int64_t nrows, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const size_t bytes = fft_smem_bytes<T>(f.n);
    SK_TRY((ensure_smem<T, k_fft_c2r_rows<T>>()));
    const int64_t npairs = nrows / 2;
    const int P = kFftElems / f.n;
    k_fft_c2r_rows<T><<<unsigned((npairs + P - 1) / P), 256, bytes, s>>>(
        static_cast<const C*>(f.A1), static_cast<T*>(f.grid), npairs, f.n, f.log2n, f.h,
        static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T, int INM, int OUTM, bool INV>
static cudaError_t run_axis(const FftPlan& f, const void* in, void* out, int64_t O, int64_t I,
                            int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const size_t bytes = fft_smem_bytes<T>(f.n);
    SK_TRY((ensure_smem<T, k_fft_axis<T, INM, OUTM, INV>>()));
    const int P = kFftElems / f.n;
    const int64_t Q = O * I;
    k_fft_axis<T, INM, OUTM, INV><<<unsigned((Q + P - 1) / P), 256, bytes, s>>>(
        static_cast<const C*>(in), static_cast<C*>(out), O, I, f.n, f.log2n, f.h, static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t run_axis0_convolve(const FftPlan& f, void* data, int64_t I, int64_t* launches, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const size_t bytes = fft_smem_bytes<T>(f.n);
    SK_TRY((ensure_smem<T, k_fft_axis0_convolve<T>>()));
    const int P = kFftElems / f.n;
    k_fft_axis0_convolve<T><<<unsigned((I + P - 1) / P), 256, bytes, s>>>(
        static_cast<C*>(data), I, f.n, f.log2n, f.h, static_cast<const T*>(f.mult), static_cast<const C*>(f.tw));
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_convolve(const FftPlan& f, cudaStream_t s, int64_t* launches) {
    using C = typename Cplx<T>::type;
    const int64_t n = f.n, H = f.h + 1, K = 2 * f.h + 1;
    if (f.d == 1) {
        SK_TRY(run_r2c<T>(f, 2, launches, s));
        k_mult_half<T><<<unsigned((H + 255) / 256), 256, 0, s>>>(static_cast<C*>(f.A1), f.h,
                                                                 static_cast<const T*>(f.mult));
        if (launches) ++*launches;
        SK_TRY(cudaGetLastError());
        return run_c2r<T>(f, 2, launches, s);
    }
    if (f.d == 2) {
        SK_TRY(run_r2c<T>(f, n, launches, s));
        SK_TRY(run_axis0_convolve<T>(f, f.A1, H, launches, s));
        return run_c2r<T>(f, n, launches, s);
    }
    SK_TRY(run_r2c<T>(f, n * n, launches, s));
    SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A1, f.A2, n, H, launches, s)));
    SK_TRY(run_axis0_convolve<T>(f, f.A2, K * H, launches, s));
    SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A2, f.A1, n, H, launches, s)));
    return run_c2r<T>(f, n * n, launches, s);
}

template <typename T>
cudaError_t launch_fft_adjoint(const FftPlan& f, double* fhat, cudaStream_t s, int64_t* launches) {
    using C = typename Cplx<T>::type;
    const int64_t n = f.n, H = f.h + 1, K = 2 * f.h + 1;
    const void* S = nullptr;
    if (f.d == 1) {
        SK_TRY(run_r2c<T>(f, 2, launches, s));
        S = f.A1;
    } else if (f.d == 2) {
        SK_TRY(run_r2c<T>(f, n, launches, s));
        SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A1, f.A3, 1, H, launches, s)));
        S = f.A3;
    } else {
        SK_TRY(run_r2c<T>(f, n * n, launches, s));
        SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A1, f.A2, n, H, launches, s)));
        SK_TRY((run_axis<T, FULL, CENTERED, false>(f, f.A2, f.A3, 1, K * H, launches, s)));
        S = f.A3;
    }
    int64_t total = 1;
    for (int t = 0; t < f.d; ++t) total *= K;
    k_extract_adjoint<T><<<unsigned((total + 255) / 256), 256, 0, s>>>(static_cast<const C*>(S), f.d, f.h,
                                                                      f.psihat, fhat);
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_forward(const FftPlan& f, const double* fhat, cudaStream_t s, int64_t* launches) {
    using C = typename Cplx<T>::type;
    const int64_t n = f.n, H = f.h + 1, K = 2 * f.h + 1;
    void* S = f.d == 1 ? f.A1 : f.A3;
    int64_t total = H;
    for (int t = 0; t < f.d - 1; ++t) total *= K;
    if (f.d == 1) SK_TRY(cudaMemsetAsync(f.A1, 0, size_t(2 * H) * sizeof(C), s));
    k_fill_forward<T><<<unsigned((total + 255) / 256), 256, 0, s>>>(fhat, f.d, f.h, f.psihat, static_cast<C*>(S));
    if (launches) ++*launches;
    SK_TRY(cudaGetLastError());
    if (f.d == 1) return run_c2r<T>(f, 2, launches, s);
    if (f.d == 2) {
        SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A3, f.A1, 1, H, launches, s)));
        return run_c2r<T>(f, n, launches, s);
    }
    SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A3, f.A2, 1, K * H, launches, s)));
    SK_TRY((run_axis<T, CENTERED, FULL, true>(f, f.A2, f.A1, n, H, launches, s)));
    return run_c2r<T>(f, n * n, launches, s);
}

template cudaError_t launch_fft_convolve<float>(const FftPlan&, cudaStream_t, int64_t*);
template cudaError_t launch_fft_convolve<double>(const FftPlan&, cudaStream_t, int64_t*);
template cudaError_t launch_fft_adjoint<float>(const FftPlan&, double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_adjoint<double>(const FftPlan&, double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_forward<float>(const FftPlan&, const double*, cudaStream_t, int64_t*);
template cudaError_t launch_fft_forward<double>(const FftPlan&, const double*, cudaStream_t, int64_t*);

}  // namespace sk
