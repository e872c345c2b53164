// Device helpers shared by the spreading and interpolation kernels: the
// window weights (the Kaiser-Bessel window of the NFFT, one piecewise
// polynomial per tap, set up on the host by window_polynomials, evaluated by
// Horner's rule) and the global task queue of the persistent launches.
#pragma once

#include "sk_internal.cuh"

namespace sk {

template <typename T> struct PolyDeg;
template <> struct PolyDeg<float> { static constexpr int D = kPolyDeg32; };
template <> struct PolyDeg<double> { static constexpr int D = kPolyDeg64; };

template <typename T>
__device__ __forceinline__ T poly_coef(const WindowPoly& wp, int k, int i);
template <> __device__ __forceinline__ float poly_coef<float>(const WindowPoly& wp, int k, int i) {
    return wp.c32[k][i];
}
template <> __device__ __forceinline__ double poly_coef<double>(const WindowPoly& wp, int k, int i) {
    return wp.c64[k][i];
}

// The W window weights of one coordinate (taps starting at cell f - (m-1)),
// by Horner's rule on the piecewise polynomial; `scale` multiplies them.  The
// window is even, so tap W-1-k is tap k's polynomial at -s: with
// P_k(s) = E_k(s^2) + s O_k(s^2), w[k] = E + s O and w[W-1-k] = E - s O, one
// pair of taps for the cost of one polynomial.
template <int W, typename T>
__device__ __forceinline__ void window_poly(T u, const WindowPoly& wp, T scale, int& f, T* w) {
    constexpr int DEG = PolyDeg<T>::D;
    constexpr int DE = DEG / 2;          // even coefficients c0, c2, ..., c(2 DE)
    constexpr int DO = (DEG - 1) / 2;    // odd coefficients c1, c3, ..., c(2 DO + 1)
    const T fl = floor(u);
    f = int(fl);
    const T s = T(2) * (u - fl) - T(1);
    const T s2 = s * s;
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
        T e = poly_coef<T>(wp, k, 2 * DE);
#pragma unroll
        for (int j = DE - 1; j >= 0; --j) e = fma(e, s2, poly_coef<T>(wp, k, 2 * j));
        T o = poly_coef<T>(wp, k, 2 * DO + 1);
#pragma unroll
        for (int j = DO - 1; j >= 0; --j) o = fma(o, s2, poly_coef<T>(wp, k, 2 * j + 1));
        const T so = s * o;
        w[k] = (e + so) * scale;
        w[W - 1 - k] = (e - so) * scale;
    }
}

// Next entry of a persistent launch's task queue for this warp (lane 0 takes
// it; every lane gets it).
__device__ __forceinline__ int queue_take(unsigned* q, int lane) {
    unsigned c = 0u;
    if (lane == 0) c = atomicAdd(q, 1u);
    return int(__shfl_sync(0xffffffffu, c, 0));
}

// A warp that has left the queue loop signs off; the last warp of the grid
// resets the queue for the next launch (every other warp has already taken
// its last entry, which precedes its sign-off).
__device__ __forceinline__ void queue_leave(unsigned* q, int lane) {
    if (lane == 0) {
        __threadfence();
        const unsigned total = gridDim.x * (blockDim.x >> 5);
        if (atomicAdd(q + 1, 1u) == total - 1u) {
            q[0] = 0u;
            q[1] = 0u;
            __threadfence();
        }
    }
}

}  // namespace sk
