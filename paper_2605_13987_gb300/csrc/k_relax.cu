// Relaxation helpers (Abstract: third-order quasi-static PDE; Sec. 3 forward
// Euler, here its exact modal limit; Sec. 5 column resistance).  FP64.
#include "wt_internal.cuh"

namespace wt {

// Dense resistive-line matrix from its tridiagonal description: diag[i] and
// off[i] = conductance between nodes i and i+1 (0 across column boundaries).
__global__ void build_k_kernel(const double* __restrict__ diag, const double* __restrict__ off, int n,
                               double* __restrict__ K) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    int i = idx / n, j = idx % n;
    double v = 0.0;
    if (i == j) v = diag[i];
    else if (j == i + 1) v = off[i];
    else if (j == i - 1) v = off[j];
    K[idx] = v;
}
void build_k(cudaStream_t s, const double* diag, const double* off, int n, double* K) {
    size_t tot = (size_t)n * n;
    build_k_kernel<<<(tot + 255) / 256, 256, 0, s>>>(diag, off, n, K);
    WT_LAUNCH("build_k");
}

// E[k][t] = amp[k] exp(-mu[k] t_n)
__global__ void modal_factor_kernel(const double* __restrict__ amp, const double* __restrict__ mu, int n,
                                    const double* __restrict__ t, int nt, double* __restrict__ E) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * nt) return;
    int k = idx / nt, j = idx % nt;
    E[idx] = amp[k] * exp(-mu[k] * t[j]);
}
void modal_factors(cudaStream_t s, const double* amp, const double* mu, int n, const double* t, int nt, double* E) {
    size_t tot = (size_t)n * nt;
    modal_factor_kernel<<<(tot + 255) / 256, 256, 0, s>>>(amp, mu, n, t, nt, E);
    WT_LAUNCH("modal_factors");
}

// Q[i][t] += q_inf[i]
__global__ void add_col_vec_kernel(double* Q, int n, int nt, const double* __restrict__ v) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * nt) return;
    Q[idx] += v[idx / nt];
}
void add_column_vector(cudaStream_t s, double* Q, int n, int nt, const double* v) {
    size_t tot = (size_t)n * nt;
    add_col_vec_kernel<<<(tot + 255) / 256, 256, 0, s>>>(Q, n, nt, v);
    WT_LAUNCH("add_column_vector");
}

// dst[i] = (float)(scale * src[i])
__global__ void to_float_kernel(const double* __restrict__ src, size_t n, double scale, float* __restrict__ dst) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)(scale * src[i]);
}
void to_float(cudaStream_t s, const double* src, size_t n, double scale, float* dst) {
    if (!n) return;
    to_float_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, n, scale, dst);
    WT_LAUNCH("to_float");
}

__global__ void check_finite_kernel(const double* __restrict__ x, size_t n, int* d_err) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) atomicMax(d_err, (int)DERR_NAN);
}
void check_finite(cudaStream_t s, const double* x, size_t n, int* d_err) {
    if (!n) return;
    check_finite_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, d_err);
    WT_LAUNCH("check_finite");
}

}  // namespace wt
