// Declarations of the plan-time and bookkeeping kernels (sk_plan_kernels.cu).
#pragma once

#include "sk_internal.cuh"

namespace sk {

void bin_shape(int d, int W, int B[3]);

__global__ void k_point_bounds(const double* x, int64_t n, int d, double* partial);
__global__ void k_point_radius(const double* x, int64_t n, int d, double c0, double c1, double c2, double* partial);
__global__ void k_weight_stats(const double* w, int64_t n, double* partial);
__global__ void k_sum_marg_log(const double* marg, const double* scal, int64_t n, int as_is, double* partial);
__global__ void k_combine(const double* partial, int nblocks, int nf, int op0, int op1, int op2, int op3, int op4,
                          int op5, int op6, double* out);

template <typename T>
void launch_prepare_points(const double* x, int64_t n, int d, const double c[3], double scale, int n_os,
                           const int B[3], const int nb[3], int m, T* const u[3], int* key, int* count, int* status,
                           cudaStream_t s);
void launch_scan_exclusive(const int* in, int* out, int n, int* scratch, cudaStream_t s);
int scan_scratch_ints(int n);
__global__ void k_scatter_perm(const int* key, int64_t n, const int* start, int* cursor, int* perm);
template <typename T>
void launch_gather_points(const int* perm, int64_t n, int d, T* const in[3], T* const out[3], cudaStream_t s);
__global__ void k_bin_starts(const int* key_start, int nbins, int bvol, int* bin_start);
__global__ void k_count_tasks(const int* bin_start, int nbins, int maxpts, int ncol, int* ntask);
__global__ void k_sub_half_sum(double* acc, const double* p, const double* q, int64_t n);
__global__ void k_dual_variable(const double* scal, const int* perm, int64_t n, double eps, int as_is, double* out);
template <typename T>
void launch_weighted_coord(const double* scal, const void* coord, int64_t n, double inv_nos, double inv_s, double* w,
                           cudaStream_t s);
template <typename T>
void launch_position_gradient(const double* scal, const void* coord, const double* t0, const double* tt,
                              const int* perm, int64_t n, int d, int t, double inv_nos, double inv_s,
                              const double* log_shift, double lam, double* grad, cudaStream_t s);
__global__ void k_block_max(const double* v, int64_t n, double* partial);
__global__ void k_log_weights(const double* g, int64_t n, const double* partial, int nparts, double lam, int fp32,
                              double* w, double* shift);
__global__ void k_convert_domain(double* v, int64_t n, double eps, int to_log);
__global__ void k_col_counts(const int* key_start, int nbins, int bvol, int ncol, int bz, int* count);
__global__ void k_fill_tasks(const int* ntask_off, int nbins, int ncol, int* task);
__global__ void k_count_subs(const int* bin_start, int nbins, int maxpts, int* nsub);
__global__ void k_fill_subs(const int* bin_start, const int* sub_off, int nbins, int maxpts, int* sub_start,
                            int* sub_count, int* sub_bin);

__global__ void k_sample_kernel(double* out, int N, int d, KernelParams kp);
__global__ void k_cos_dft_axis(const double* in, double* out, int N, int d, int axis, const double* costab);
__global__ void k_cos_table(double* c, int N);
__global__ void k_window_transform(double* out, int h, int n_os, int m, double beta);
template <typename T>
void launch_build_mult(T* M, int d, int h, const double* bk, double inv_norm, const double* psihat, int64_t total,
                       cudaStream_t s);

// spec[k] *= b_k over k in {-h..h}^d (interleaved complex, row-major with
// index k_t + h), b_k taken from the N^d table over I_N; the kernel is even in
// every coordinate, so b at k_t = +h is b at k_t = -h.
__global__ void k_times_bk(const double* spec, const double* bk, int d, int h, double* out);

__global__ void k_init_bounds(int* out);
template <typename T>
void launch_cell_bounds(void* const u[3], int64_t n, int d, int* out, cudaStream_t s);
__global__ void k_fill(double* p, int64_t n, double v);
__global__ void k_scale(double* p, int64_t n, double f);
__global__ void k_gather(const double* in, const int* perm, int64_t n, double* out);
__global__ void k_scatter(const double* in, const int* perm, int64_t n, double* out);

}  // namespace sk
