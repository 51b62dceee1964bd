// FP64 dense linear algebra for the one-time setup (boundary fit, relaxation
// modes, time basis).  GB300's FP64 rate is low, so these kernels are
// arithmetic-bound at modest sizes; they are written for correctness and
// coalesced access rather than peak throughput.
#include "wt_internal.cuh"

#include <algorithm>
#include <cstring>
#include <cmath>
#include <vector>

namespace wt {

// ------------------------------------------------------------------- DGEMM
// 64x64 output tile per 256-thread block, 4x4 outputs per thread (rows
// ty + 16 i, columns tx + 16 j), K staged through shared memory 16 at a time.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha,
                                                    const double* __restrict__ A, int lda,
                                                    const double* __restrict__ B, int ldb, double beta,
                                                    double* __restrict__ C, int ldc, int lower_only) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int bm = blockIdx.y * 64, bn = blockIdx.x * 64;
    if (lower_only && bn > bm + 63) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int mm, kk;
            if (!TA) { mm = e >> 4; kk = e & 15; } else { kk = e >> 6; mm = e & 63; }
            const int gm = bm + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < K) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int nn, kk;
            if (!TB) { kk = e >> 6; nn = e & 63; } else { nn = e >> 4; kk = e & 15; }
            const int gn = bn + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < N && gk < K) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = bm + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = bn + tx + 16 * j;
            if (gn >= N) continue;
            if (lower_only && gn > gm) continue;
            double* c = C + (size_t)gm * ldc + gn;
            *c = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
        }
    }
}

void dgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc, bool lower_only) {
    if (M <= 0 || N <= 0) return;
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    if (K <= 0) {  // C = beta C
        // handled by a degenerate launch with K = 0: acc stays 0
    }
    if (!ta && !tb) dgemm_kernel<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only);
    else if (ta && !tb) dgemm_kernel<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only);
    else if (!ta && tb) dgemm_kernel<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only);
    else dgemm_kernel<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only);
    WT_LAUNCH("dgemm");
}

// -------------------------------------------------------------- utilities
__global__ void symm_lower_kernel(double* A, int n, int lda) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t tot = (size_t)n * n;
    if (idx >= tot) return;
    int i = idx / n, j = idx % n;
    if (j > i) A[(size_t)i * lda + j] = A[(size_t)j * lda + i];
}
void symmetrize_from_lower(cudaStream_t s, double* A, int n, int lda) {
    size_t tot = (size_t)n * n;
    symm_lower_kernel<<<(tot + 255) / 256, 256, 0, s>>>(A, n, lda);
    WT_LAUNCH("symmetrize_from_lower");
}

__global__ void transpose_kernel(const double* __restrict__ A, int rows, int cols, double* __restrict__ At) {
    __shared__ double t[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int r = by + k, c = bx + threadIdx.x;
        if (r < rows && c < cols) t[k][threadIdx.x] = A[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int c = bx + k, r = by + threadIdx.x;
        if (r < rows && c < cols) At[(size_t)c * rows + r] = t[threadIdx.x][k];
    }
}
void transpose(cudaStream_t s, const double* A, int rows, int cols, double* At) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_kernel<<<grid, block, 0, s>>>(A, rows, cols, At);
    WT_LAUNCH("transpose");
}

__global__ void symm_avg_kernel(const double* __restrict__ F, double* __restrict__ C, int n) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    int i = idx / n, j = idx % n;
    C[idx] = 0.5 * (F[idx] + F[(size_t)j * n + i]);
}
void symmetrize_avg(cudaStream_t s, const double* F, double* C, int n) {
    size_t tot = (size_t)n * n;
    symm_avg_kernel<<<(tot + 255) / 256, 256, 0, s>>>(F, C, n);
    WT_LAUNCH("symmetrize_avg");
}

// y = alpha op(A) x + beta y.  One warp per output element.
__global__ void dgemv_n_kernel(int M, int N, double alpha, const double* __restrict__ A, int lda,
                               const double* __restrict__ x, double beta, double* __restrict__ y) {
    int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (row >= M) return;
    double acc = 0.0;
    for (int j = lane; j < N; j += 32) acc = fma(A[(size_t)row * lda + j], x[j], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * y[row]);
}
// transposed: y[j] = sum_i A[i][j] x[i]; thread per column, rows split over blockIdx.y, atomics
__global__ void dgemv_t_kernel(int M, int N, double alpha, const double* __restrict__ A, int lda,
                               const double* __restrict__ x, double* __restrict__ y, int rows_per) {
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= N) return;
    int r0 = blockIdx.y * rows_per, r1 = min(M, r0 + rows_per);
    double acc = 0.0;
    for (int i = r0; i < r1; ++i) acc = fma(A[(size_t)i * lda + col], x[i], acc);
    atomicAdd(&y[col], alpha * acc);
}
__global__ void scale_vec_kernel(double* y, size_t n, double b) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (b == 0.0) ? 0.0 : b * y[i];
}
void dgemv(cudaStream_t s, bool ta, int M, int N, double alpha, const double* A, int lda, const double* x,
           double beta, double* y) {
    if (!ta) {
        dgemv_n_kernel<<<(M + 7) / 8, 256, 0, s>>>(M, N, alpha, A, lda, x, beta, y);
    } else {
        scale_vec_kernel<<<(N + 255) / 256, 256, 0, s>>>(y, N, beta);
        int rows_per = 256;
        dim3 grid((N + 127) / 128, (M + rows_per - 1) / rows_per);
        dgemv_t_kernel<<<grid, 128, 0, s>>>(M, N, alpha, A, lda, x, y, rows_per);
    }
    WT_LAUNCH("dgemv");
}

__global__ void sumsq_kernel(const double* __restrict__ x, size_t n, double* out) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc = fma(x[i], x[i], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x / 32] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}
double dnrm2(cudaStream_t s, const double* x, size_t n, double* d_scratch) {
    WT_CUDA(cudaMemsetAsync(d_scratch, 0, sizeof(double), s));
    int blocks = (int)std::min<size_t>(1024, (n + 255) / 256 + 1);
    sumsq_kernel<<<blocks, 256, 0, s>>>(x, n, d_scratch);
    WT_LAUNCH("dnrm2");
    double h = 0;
    WT_CUDA(cudaMemcpyAsync(&h, d_scratch, sizeof(double), cudaMemcpyDeviceToHost, s));
    WT_CUDA(cudaStreamSynchronize(s));
    return std::sqrt(h);
}

__global__ void fill_kernel(double* x, size_t n, double v) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}
void fill(cudaStream_t s, double* x, size_t n, double v) {
    if (!n) return;
    fill_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, v);
    WT_LAUNCH("fill");
}
__global__ void axpy_kernel(size_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], y[i]);
}
void axpy(cudaStream_t s, size_t n, double a, const double* x, double* y) {
    if (!n) return;
    axpy_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a, x, y);
    WT_LAUNCH("axpy");
}
__global__ void dscal_kernel(size_t n, double a, double* x) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] *= a;
}
void dscal(cudaStream_t s, size_t n, double a, double* x) {
    if (!n) return;
    dscal_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a, x);
    WT_LAUNCH("dscal");
}
__global__ void rank1_kernel(int M, int N, double alpha, const double* __restrict__ u, const double* __restrict__ v,
                             double* __restrict__ A, int lda) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)M * N) return;
    int i = idx / N, j = idx % N;
    A[(size_t)i * lda + j] = fma(alpha * u[i], v[j], A[(size_t)i * lda + j]);
}
void rank1(cudaStream_t s, int M, int N, double alpha, const double* u, const double* v, double* A, int lda) {
    size_t tot = (size_t)M * N;
    if (!tot) return;
    rank1_kernel<<<(tot + 255) / 256, 256, 0, s>>>(M, N, alpha, u, v, A, lda);
    WT_LAUNCH("rank1");
}
__global__ void copy_block_kernel(const double* __restrict__ src, int lds, double* __restrict__ dst, int ldd,
                                  int rows, int cols) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * cols) return;
    int i = idx / cols, j = idx % cols;
    dst[(size_t)i * ldd + j] = src[(size_t)i * lds + j];
}
void copy_block(cudaStream_t s, const double* src, int lds, double* dst, int ldd, int rows, int cols) {
    size_t tot = (size_t)rows * cols;
    if (!tot) return;
    copy_block_kernel<<<(tot + 255) / 256, 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
    WT_LAUNCH("copy_block");
}
__global__ void scale_cols_kernel(double* A, int M, int N, int lda, const double* __restrict__ d) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)M * N) return;
    int i = idx / N, j = idx % N;
    A[(size_t)i * lda + j] *= d[j];
}
void scale_columns(cudaStream_t s, double* A, int M, int N, int lda, const double* d) {
    size_t tot = (size_t)M * N;
    if (!tot) return;
    scale_cols_kernel<<<(tot + 255) / 256, 256, 0, s>>>(A, M, N, lda, d);
    WT_LAUNCH("scale_columns");
}
__global__ void scale_rows_kernel(double* A, int M, int N, int lda, const double* __restrict__ d) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)M * N) return;
    int i = idx / N, j = idx % N;
    A[(size_t)i * lda + j] *= d[i];
}
void scale_rows(cudaStream_t s, double* A, int M, int N, int lda, const double* d) {
    size_t tot = (size_t)M * N;
    if (!tot) return;
    scale_rows_kernel<<<(tot + 255) / 256, 256, 0, s>>>(A, M, N, lda, d);
    WT_LAUNCH("scale_rows");
}
__global__ void col_norm_kernel(const double* __restrict__ A, int M, int N, int lda, double* out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double acc = 0.0;
    for (int i = 0; i < M; ++i) {
        double v = A[(size_t)i * lda + j];
        acc = fma(v, v, acc);
    }
    out[j] = sqrt(acc);
}
void column_norms(cudaStream_t s, const double* A, int M, int N, int lda, double* out) {
    col_norm_kernel<<<(N + 127) / 128, 128, 0, s>>>(A, M, N, lda, out);
    WT_LAUNCH("column_norms");
}
__global__ void diag_kernel(const double* A, int n, int lda, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = A[(size_t)i * lda + i];
}
void get_diag(cudaStream_t s, const double* A, int n, int lda, double* out) {
    diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(A, n, lda, out);
    WT_LAUNCH("get_diag");
}

// ---------------------------------------------------------------- Cholesky
constexpr int CHOL_NB = 32;

// Unblocked right-looking factorisation of one nb x nb diagonal block in
// shared memory.  A pivot that is not positive and finite sets d_err.
__global__ void potrf_block_kernel(double* A, int lda, int nb, int* d_err) {
    __shared__ double a[CHOL_NB][CHOL_NB + 1];
    __shared__ int bad;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) a[e / nb][e % nb] = A[(size_t)(e / nb) * lda + e % nb];
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            double d = a[j][j];
            if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
            a[j][j] = sqrt(d);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= a[j][j];
        __syncthreads();
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            int i = e / nb, l = e % nb;
            if (l > j && i >= l) a[i][l] -= a[i][j] * a[l][j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, l = e % nb;
        if (l <= i) A[(size_t)i * lda + l] = a[i][l];
    }
    if (threadIdx.x == 0 && bad) atomicMax(d_err, (int)DERR_NOT_SPD);
}

// Panel: rows below the diagonal block, X L11^T = A21 -> X (one thread per row).
__global__ void trsm_panel_kernel(const double* L11, double* A21, int lda, int rows, int nb) {
    __shared__ double l[CHOL_NB][CHOL_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) l[e / nb][e % nb] = L11[(size_t)(e / nb) * lda + e % nb];
    __syncthreads();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double* row = A21 + (size_t)r * lda;
    double x[CHOL_NB];
#pragma unroll
    for (int j = 0; j < CHOL_NB; ++j) {
        if (j < nb) {
            double v = row[j];
            for (int k = 0; k < j; ++k) v -= x[k] * l[j][k];
            x[j] = v / l[j][j];
            row[j] = x[j];
        }
    }
}

void cholesky(cudaStream_t s, double* A, int n, int lda, int* d_err) {
    for (int k = 0; k < n; k += CHOL_NB) {
        int nb = std::min(CHOL_NB, n - k);
        double* Akk = A + (size_t)k * lda + k;
        potrf_block_kernel<<<1, 256, 0, s>>>(Akk, lda, nb, d_err);
        WT_LAUNCH("potrf_block");
        int rest = n - k - nb;
        if (rest > 0) {
            double* A21 = A + (size_t)(k + nb) * lda + k;
            trsm_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(Akk, A21, lda, rest, nb);
            WT_LAUNCH("trsm_panel");
            double* A22 = A + (size_t)(k + nb) * lda + (k + nb);
            dgemm(s, false, true, rest, rest, nb, -1.0, A21, lda, A21, lda, 1.0, A22, lda, true);
        }
    }
}

// Diagonal-block triangular solves, one thread per right-hand side column.
__global__ void trsv_block_lower_kernel(const double* L, int ldl, int nb, double* B, int ldb, int nrhs) {
    __shared__ double l[CHOL_NB][CHOL_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) l[e / nb][e % nb] = L[(size_t)(e / nb) * ldl + e % nb];
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double y[CHOL_NB];
#pragma unroll
    for (int i = 0; i < CHOL_NB; ++i) {
        if (i < nb) {
            double v = B[(size_t)i * ldb + c];
            for (int k = 0; k < i; ++k) v -= l[i][k] * y[k];
            y[i] = v / l[i][i];
            B[(size_t)i * ldb + c] = y[i];
        }
    }
}
__global__ void trsv_block_upper_t_kernel(const double* L, int ldl, int nb, double* B, int ldb, int nrhs) {
    __shared__ double l[CHOL_NB][CHOL_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) l[e / nb][e % nb] = L[(size_t)(e / nb) * ldl + e % nb];
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    double x[CHOL_NB];
#pragma unroll
    for (int ii = CHOL_NB - 1; ii >= 0; --ii) {
        if (ii < nb) {
            double v = B[(size_t)ii * ldb + c];
            for (int k = ii + 1; k < nb; ++k) v -= l[k][ii] * x[k];
            x[ii] = v / l[ii][ii];
            B[(size_t)ii * ldb + c] = x[ii];
        }
    }
}

void trsm_lower(cudaStream_t s, const double* L, int n, int ldl, double* B, int nrhs, int ldb) {
    for (int k = 0; k < n; k += CHOL_NB) {
        int nb = std::min(CHOL_NB, n - k);
        trsv_block_lower_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(L + (size_t)k * ldl + k, ldl, nb,
                                                                   B + (size_t)k * ldb, ldb, nrhs);
        WT_LAUNCH("trsv_block_lower");
        int rest = n - k - nb;
        if (rest > 0)
            dgemm(s, false, false, rest, nrhs, nb, -1.0, L + (size_t)(k + nb) * ldl + k, ldl,
                  B + (size_t)k * ldb, ldb, 1.0, B + (size_t)(k + nb) * ldb, ldb);
    }
}

void trsm_lower_t(cudaStream_t s, const double* L, int n, int ldl, double* B, int nrhs, int ldb) {
    int last = ((n - 1) / CHOL_NB) * CHOL_NB;
    for (int k = last; k >= 0; k -= CHOL_NB) {
        int nb = std::min(CHOL_NB, n - k);
        trsv_block_upper_t_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(L + (size_t)k * ldl + k, ldl, nb,
                                                                     B + (size_t)k * ldb, ldb, nrhs);
        WT_LAUNCH("trsv_block_upper_t");
        if (k > 0)  // B[0:k] -= L[k:k+nb, 0:k]^T X[k:k+nb]
            dgemm(s, true, false, k, nrhs, nb, -1.0, L + (size_t)k * ldl, ldl, B + (size_t)k * ldb, ldb, 1.0, B, ldb);
    }
}

// ------------------------------------------------------------------ Jacobi
// Circle-method pairing: position 0 is fixed, positions 1..m-1 rotate by one
// each round; pair i joins positions i and m-1-i.  Consecutive pairs hold
// consecutive indices, so rows of A are read and written in coalesced runs.
__device__ __forceinline__ int circle_player(int pos, int round, int m) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (m - 1)) + 1;
}

__global__ void jacobi_angles_kernel(const double* __restrict__ A, int m, int lda, int n_real, int round,
                                     double abs_tol, double* __restrict__ cs, unsigned long long* __restrict__ n_rot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m / 2) return;
    int p = circle_player(i, round, m), q = circle_player(m - 1 - i, round, m);
    if (p > q) { int t = p; p = q; q = t; }
    double c = 1.0, sn = 0.0, t = 0.0;
    if (q < n_real) {
        double app = A[(size_t)p * lda + p], aqq = A[(size_t)q * lda + q], apq = A[(size_t)p * lda + q];
        // rotate only when the coupling is above rounding relative to the diagonal (and above
        // the caller's absolute floor: couplings between rounding-level directions never settle)
        if (fabs(apq) > 1e-15 * sqrt(fabs(app) * fabs(aqq)) && fabs(apq) > fmax(abs_tol, 1e-300)) {
            double tau = (aqq - app) / (2.0 * apq);
            t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
            atomicAdd(n_rot, 1ull);
        }
    }
    cs[4 * i + 0] = c;
    cs[4 * i + 1] = sn;
    cs[4 * i + 2] = t;
    cs[4 * i + 3] = 0.0;
}

// A <- J^T A J for the m/2 disjoint rotations of this round; one thread per
// (pair i, pair j) 2x2 block.
__global__ void jacobi_apply_kernel(double* __restrict__ A, int m, int lda, int round,
                                    const double* __restrict__ cs) {
    int half = m / 2;
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)half * half) return;
    int i = idx / half, j = idx % half;
    int pi = circle_player(i, round, m), qi = circle_player(m - 1 - i, round, m);
    int pj = circle_player(j, round, m), qj = circle_player(m - 1 - j, round, m);
    if (pi > qi) { int t = pi; pi = qi; qi = t; }
    if (pj > qj) { int t = pj; pj = qj; qj = t; }
    double ci = cs[4 * i], si = cs[4 * i + 1], ti = cs[4 * i + 2];
    double cj = cs[4 * j], sj = cs[4 * j + 1];
    double* a11 = A + (size_t)pi * lda + pj;
    double* a12 = A + (size_t)pi * lda + qj;
    double* a21 = A + (size_t)qi * lda + pj;
    double* a22 = A + (size_t)qi * lda + qj;
    if (i == j) {
        if (si == 0.0) return;
        double apq = *a12;
        *a11 = *a11 - ti * apq;
        *a22 = *a22 + ti * apq;
        *a12 = 0.0;
        *a21 = 0.0;
        return;
    }
    if (si == 0.0 && sj == 0.0) return;
    double x11 = *a11, x12 = *a12, x21 = *a21, x22 = *a22;
    double y11 = cj * x11 - sj * x12, y12 = sj * x11 + cj * x12;
    double y21 = cj * x21 - sj * x22, y22 = sj * x21 + cj * x22;
    *a11 = ci * y11 - si * y21;
    *a21 = si * y11 + ci * y21;
    *a12 = ci * y12 - si * y22;
    *a22 = si * y12 + ci * y22;
}

// V <- V J (columns p_j, q_j of every row).
__global__ void jacobi_vec_kernel(double* __restrict__ V, int n_rows, int m, int ldv, int round,
                                  const double* __restrict__ cs) {
    int half = m / 2;
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_rows * half) return;
    int r = idx / half, j = idx % half;
    double sj = cs[4 * j + 1];
    if (sj == 0.0) return;
    double cj = cs[4 * j];
    int pj = circle_player(j, round, m), qj = circle_player(m - 1 - j, round, m);
    if (pj > qj) { int t = pj; pj = qj; qj = t; }
    double* vp = V + (size_t)r * ldv + pj;
    double* vq = V + (size_t)r * ldv + qj;
    double a = *vp, b = *vq;
    *vp = cj * a - sj * b;
    *vq = sj * a + cj * b;
}

__global__ void eye_kernel(double* V, int n, int ld) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    int i = idx / n, j = idx % n;
    V[(size_t)i * ld + j] = (i == j) ? 1.0 : 0.0;
}

int jacobi_eig(cudaStream_t s, double* A_in, int n, double* w, double* V_out, int* d_err, int max_sweeps,
               double abs_tol) {
    // work on an even-sized copy (a padded index has zero coupling and never rotates)
    int m = n + (n & 1);
    if (m < 2) m = 2;
    DBuf<double> A, V, cs;
    DBuf<unsigned long long> cnt;
    A.alloc((size_t)m * m);
    V.alloc((size_t)m * m);
    cs.alloc((size_t)4 * (m / 2));
    cnt.alloc(1);
    A.zero(s);
    copy_block(s, A_in, n, A.p, m, n, n);
    eye_kernel<<<((size_t)m * m + 255) / 256, 256, 0, s>>>(V.p, m, m);
    WT_LAUNCH("eye");
    int half = m / 2;
    int sweeps = 0;
    bool converged = false;
    for (; sweeps < max_sweeps && !converged; ++sweeps) {
        WT_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < m - 1; ++r) {
            jacobi_angles_kernel<<<(half + 127) / 128, 128, 0, s>>>(A.p, m, m, n, r, abs_tol, cs.p, cnt.p);
            size_t nb = (size_t)half * half;
            jacobi_apply_kernel<<<(nb + 255) / 256, 256, 0, s>>>(A.p, m, m, r, cs.p);
            size_t nv = (size_t)m * half;
            jacobi_vec_kernel<<<(nv + 255) / 256, 256, 0, s>>>(V.p, m, m, m, r, cs.p);
        }
        WT_LAUNCH("jacobi sweep");
        unsigned long long h = 0;
        WT_CUDA(cudaMemcpyAsync(&h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        WT_CUDA(cudaStreamSynchronize(s));
        converged = (h == 0);
    }
    get_diag(s, A.p, n, m, w);
    copy_block(s, V.p, m, V_out, n, n, n);
    if (!converged) {
        int v = DERR_TIMEOUT;
        WT_CUDA(cudaMemcpyAsync(d_err, &v, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    WT_CUDA(cudaStreamSynchronize(s));
    return sweeps;
}

// ------------------------------------------------------ one-sided Jacobi SVD
// Hestenes' method on the rows of A [m][n]: every round rotates the m/2
// disjoint row pairs of one circle-method pairing, (a_p, a_q) <- (c a_p - s a_q,
// s a_p + c a_q) with the angle that makes them orthogonal, and applies the
// same rotation to rows p, q of V [m][m].  No Gram matrix is formed, so the
// singular values keep their relative accuracy (a Gram matrix would square
// the condition number).  One block per pair: three block-wide dot products,
// then the rotation of both rows.
__global__ void __launch_bounds__(256) osj_round_kernel(double* __restrict__ A, int n, int lda,
                                                        double* __restrict__ V, int m_real, int m, int ldv,
                                                        int round, double tol, double abs_floor,
                                                        unsigned long long* __restrict__ n_rot,
                                                        unsigned long long* __restrict__ max_rel) {
    int p = circle_player(blockIdx.x, round, m), q = circle_player(m - 1 - blockIdx.x, round, m);
    if (p > q) { const int t = p; p = q; q = t; }
    if (q >= m_real) return;                      // the padding row of an odd m
    double* ap = A + (size_t)p * lda;
    double* aq = A + (size_t)q * lda;
    double sa = 0.0, sb = 0.0, sg = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double x = ap[k], y = aq[k];
        sa = fma(x, x, sa);
        sb = fma(y, y, sb);
        sg = fma(x, y, sg);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
    }
    __shared__ double red[3][8];
    __shared__ double rot[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = sa; red[1][warp] = sb; red[2][warp] = sg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { al += red[0][w]; be += red[1][w]; ga += red[2][w]; }
        double c = 1.0, sn = 0.0;
        // rotate when the rows are coupled above rounding relative to their norms and above the
        // absolute floor (pairs of rounding-level rows would otherwise keep rotating)
        if (ga != 0.0 && al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be) && fabs(ga) > abs_floor) {
            const double zeta = (be - al) / (2.0 * ga);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = c * t;
            atomicAdd(n_rot, 1ull);
            // largest relative coupling rotated in this sweep (non-negative doubles order like their bits)
            const double rel = fabs(ga) / (sqrt(al) * sqrt(be));
            atomicMax(max_rel, (unsigned long long)__double_as_longlong(rel));
        }
        rot[0] = c;
        rot[1] = sn;
    }
    __syncthreads();
    const double c = rot[0], sn = rot[1];
    if (sn == 0.0) return;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double x = ap[k], y = aq[k];
        ap[k] = c * x - sn * y;
        aq[k] = sn * x + c * y;
    }
    if (!V) return;                               // rotations not accumulated
    double* vp = V + (size_t)p * ldv;
    double* vq = V + (size_t)q * ldv;
    for (int k = threadIdx.x; k < m_real; k += blockDim.x) {
        const double x = vp[k], y = vq[k];
        vp[k] = c * x - sn * y;
        vq[k] = sn * x + c * y;
    }
}

__global__ void __launch_bounds__(256) row_norms_kernel(const double* __restrict__ A, int n, int lda,
                                                        double* __restrict__ out) {
    const double* a = A + (size_t)blockIdx.x * lda;
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s = fma(a[k], a[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[blockIdx.x] = sqrt(t);
    }
}

int onesided_jacobi_rows(cudaStream_t s, double* A, int m, int n, int lda, double* V, double* sigma, int* d_err,
                         int max_sweeps, double* coupling_out) {
    const int mp = m + (m & 1);                  // even circle; an odd m has one idle row per round
    if (V) {                                     // V = NULL: the rotations are not accumulated
        eye_kernel<<<((size_t)m * m + 255) / 256, 256, 0, s>>>(V, m, m);
        WT_LAUNCH("eye");
    }
    DBuf<unsigned long long> cnt;
    cnt.alloc(2);                                // rotations, largest relative coupling (its bits)
    constexpr double kAcceptCoupling = 1e-10;
    // relative coupling left unrotated: the rounding level of a length-n dot product (n eps), so
    // that pairs whose coupling is rounding noise stop rotating
    const double tol = fmax(1e-15, (double)n * 2.220446049250313e-16);
    // absolute floor: (1e-15 ||A||_F)^2, far below the couplings of rows that carry information
    double abs_floor = 0.0;
    if (m > 0) {
        row_norms_kernel<<<m, 256, 0, s>>>(A, n, lda, sigma);
        WT_LAUNCH("row norms");
        std::vector<double> h(m);
        WT_CUDA(cudaMemcpyAsync(h.data(), sigma, m * sizeof(double), cudaMemcpyDeviceToHost, s));
        WT_CUDA(cudaStreamSynchronize(s));
        double f2 = 0.0;
        for (double x : h) f2 += x * x;
        abs_floor = 1e-30 * f2;
    }
    int sweeps = 0;
    bool converged = m < 2;
    double last_rel = 0.0;
    for (; sweeps < max_sweeps && !converged; ++sweeps) {
        WT_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), s));
        for (int r = 0; r < mp - 1; ++r)
            osj_round_kernel<<<mp / 2, 256, 0, s>>>(A, n, lda, V, m, mp, m, r, tol, abs_floor, cnt.p, cnt.p + 1);
        WT_LAUNCH("one-sided Jacobi sweep");
        unsigned long long h[2] = {0, 0};
        WT_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        WT_CUDA(cudaStreamSynchronize(s));
        converged = (h[0] == 0);
        std::memcpy(&last_rel, &h[1], sizeof(double));
    }
    // rows still coupled after the sweep limit, but only far below any use of the decomposition
    // (the time basis truncates at 1e-7): accepted (rounding noise that keeps rotating)
    if (!converged && last_rel <= kAcceptCoupling) converged = true;
    if (coupling_out) *coupling_out = last_rel;
    if (m > 0) {
        row_norms_kernel<<<m, 256, 0, s>>>(A, n, lda, sigma);
        WT_LAUNCH("row norms");
    }
    if (!converged) {
        int v = DERR_TIMEOUT;
        WT_CUDA(cudaMemcpyAsync(d_err, &v, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    WT_CUDA(cudaStreamSynchronize(s));
    return sweeps;
}

// ------------------------------------------------------------------------
// Householder QR with column pivoting of a tall matrix whose columns are the rows of a
// row-major array (column j = M + j ld, ns entries; ns >= nt columns): M P = Q1 R.  Only R is
// kept (the reflectors are not needed afterwards).  Step k: the column of largest remaining
// norm is swapped into place and its reflector formed (one block), then every trailing column
// takes the reflector and recomputes its remaining norm exactly (one block per column), so no
// norm downdating can go stale.

// sum over the block (blockDim.x a multiple of 32, at most 1024); every thread gets the result
__device__ double qr_block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = l < nw ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (l == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

__global__ void __launch_bounds__(256) qrcp_norms_kernel(const double* __restrict__ M, int ns, int ld,
                                                         double* __restrict__ nrm) {
    __shared__ double sh[33];
    const double* a = M + (size_t)blockIdx.x * ld;
    double ss = 0.0;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) ss = fma(a[i], a[i], ss);
    ss = qr_block_sum(ss, sh);
    if (threadIdx.x == 0) nrm[blockIdx.x] = ss;
}

// pivot (largest remaining squared norm, the lowest index among equals), swap, reflector
// v = x - beta e_k with beta = -sign(x_k) ||x||, tau = 2 / v.v; column k becomes beta e_k
__global__ void __launch_bounds__(512) qrcp_pivot_kernel(double* __restrict__ M, int ns, int nt, int ld, int k,
                                                         double* __restrict__ nrm, int* __restrict__ piv,
                                                         double* __restrict__ v, double* __restrict__ tau) {
    __shared__ double sh[33];
    __shared__ double bv[32];
    __shared__ int bi[32];
    __shared__ int sp;
    double best = -1.0;
    int bj = nt;
    for (int j = k + threadIdx.x; j < nt; j += blockDim.x)
        if (nrm[j] > best) { best = nrm[j]; bj = j; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ov > best || (ov == best && oj < bj)) { best = ov; bj = oj; }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) { bv[w] = best; bi[w] = bj; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = bv[0];
        int j = bi[0];
        for (int q = 1; q < nw; ++q)
            if (bv[q] > b || (bv[q] == b && bi[q] < j)) { b = bv[q]; j = bi[q]; }
        sp = (j < nt) ? j : k;
    }
    __syncthreads();
    const int p = sp;
    double* x = M + (size_t)k * ld;
    if (p != k) {
        double* y = M + (size_t)p * ld;
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            const double t = x[i];
            x[i] = y[i];
            y[i] = t;
        }
        if (threadIdx.x == 0) {
            const double t = nrm[k];
            nrm[k] = nrm[p];
            nrm[p] = t;
            const int q = piv[k];
            piv[k] = piv[p];
            piv[p] = q;
        }
    }
    __syncthreads();
    double ss = 0.0;
    for (int i = k + threadIdx.x; i < ns; i += blockDim.x) ss = fma(x[i], x[i], ss);
    ss = qr_block_sum(ss, sh);
    const double x0 = x[k];
    const double alpha = sqrt(ss);
    const double beta = alpha > 0.0 ? -copysign(alpha, x0) : 0.0;
    const double vn = 2.0 * alpha * (alpha + fabs(x0));          // (x - beta e_k).(x - beta e_k)
    for (int i = threadIdx.x; i < ns; i += blockDim.x) v[i] = i < k ? 0.0 : (i == k ? x0 - beta : x[i]);
    __syncthreads();
    for (int i = k + threadIdx.x; i < ns; i += blockDim.x) x[i] = i == k ? beta : 0.0;
    if (threadIdx.x == 0) {
        *tau = vn > 0.0 ? 2.0 / vn : 0.0;
        nrm[k] = 0.0;
    }
}

// columns j > k: a -= tau (v.a) v, then their squared norms below row k
__global__ void __launch_bounds__(256) qrcp_apply_kernel(double* __restrict__ M, int ns, int ld, int k,
                                                         const double* __restrict__ v, const double* __restrict__ tau,
                                                         double* __restrict__ nrm) {
    __shared__ double sh[33];
    const int j = k + 1 + blockIdx.x;
    double* a = M + (size_t)j * ld;
    double d = 0.0;
    for (int i = k + threadIdx.x; i < ns; i += blockDim.x) d = fma(v[i], a[i], d);
    d = qr_block_sum(d, sh);
    const double t = *tau * d;
    double ss = 0.0;
    for (int i = k + threadIdx.x; i < ns; i += blockDim.x) {
        const double y = fma(-t, v[i], a[i]);
        a[i] = y;
        if (i > k) ss = fma(y, y, ss);
    }
    ss = qr_block_sum(ss, sh);
    if (threadIdx.x == 0) nrm[j] = ss;
}

// R[i][j] = M[j][i] for i, j < nt (upper triangular after the factorisation)
__global__ void qrcp_extract_kernel(const double* __restrict__ M, int nt, int ld, double* __restrict__ R) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)nt * nt) return;
    const int i = (int)(e / nt), j = (int)(e % nt);
    R[e] = i <= j ? M[(size_t)j * ld + i] : 0.0;
}

void qrcp_r(cudaStream_t s, double* M, int ns, int nt, int ld, double* R, int* piv) {
    if (nt < 1) return;
    if (ns < nt) fail(WT_ERR_ARG, "column-pivoted QR: needs at least as many rows as columns");
    DBuf<double> v, nrm, tau;
    v.alloc(ns);
    nrm.alloc(nt);
    tau.alloc(1);
    std::vector<int> h(nt);
    for (int j = 0; j < nt; ++j) h[j] = j;
    WT_CUDA(cudaMemcpyAsync(piv, h.data(), nt * sizeof(int), cudaMemcpyHostToDevice, s));
    qrcp_norms_kernel<<<nt, 256, 0, s>>>(M, ns, ld, nrm.p);
    WT_LAUNCH("qrcp norms");
    for (int k = 0; k < nt; ++k) {
        qrcp_pivot_kernel<<<1, 512, 0, s>>>(M, ns, nt, ld, k, nrm.p, piv, v.p, tau.p);
        if (k + 1 < nt) qrcp_apply_kernel<<<nt - k - 1, 256, 0, s>>>(M, ns, ld, k, v.p, tau.p, nrm.p);
    }
    WT_LAUNCH("qrcp steps");
    qrcp_extract_kernel<<<(unsigned)(((size_t)nt * nt + 255) / 256), 256, 0, s>>>(M, nt, ld, R);
    WT_LAUNCH("qrcp extract");
    WT_CUDA(cudaStreamSynchronize(s));      // the host pivot array and the work buffers go out of scope
}

__global__ void gather_rows_scaled_kernel(const double* __restrict__ A, int n, int lda, const int* __restrict__ idx,
                                          const double* __restrict__ scale, double* __restrict__ out) {
    const int r = blockIdx.y;
    const double* a = A + (size_t)idx[r] * lda;
    const double f = scale[r];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[(size_t)r * n + k] = f * a[k];
}

void gather_rows_scaled(cudaStream_t s, const double* A, int n, int lda, const int* idx, const double* scale,
                        int rows, double* out) {
    if (rows < 1) return;
    dim3 g((unsigned)std::min(64, (n + 255) / 256), (unsigned)rows);
    gather_rows_scaled_kernel<<<g, 256, 0, s>>>(A, n, lda, idx, scale, out);
    WT_LAUNCH("gather rows");
}

}  // namespace wt
