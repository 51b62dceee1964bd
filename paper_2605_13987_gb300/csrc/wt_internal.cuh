// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/wt.h"

namespace wt {

constexpr double kEps0 = 8.8541878128e-12;   // vacuum permittivity [F/m]
constexpr double kPi = 3.14159265358979323846;

// Device error words (ctx->d_err[i]); a kernel that detects a failure sets
// the word with atomicMax so the host sees the most severe code.
enum DeviceErr : int {
    DERR_NONE = 0,
    DERR_NOT_SPD = 1,        // non-positive pivot in a Cholesky factorisation
    DERR_NAN = 2,            // non-finite value
    DERR_TIMEOUT = 3,        // a bounded wait gave up
};

struct Status {
    wt_status code = WT_OK;
    std::string msg;
    bool ok() const { return code == WT_OK; }
};

// Throwing is confined to the library; the C entry points catch and convert.
struct Error {
    wt_status code;
    std::string msg;
};

[[noreturn]] void fail(wt_status code, const std::string& msg);

// Host-side fault injection: WT_FAULT is a comma-separated list of names
// (fit_singular, alloc, nan_q, queue_stall); each forces one error path.
inline bool fault_enabled(const char* name) {
    const char* env = std::getenv("WT_FAULT");
    if (!env) return false;
    const std::string list = std::string(",") + env + ",";
    return list.find(std::string(",") + name + ",") != std::string::npos;
}
void cuda_check(cudaError_t e, const char* what);
#define WT_CUDA(call) ::wt::cuda_check((call), #call)
#define WT_LAUNCH(what) ::wt::cuda_check(cudaGetLastError(), what)

// Let `kernel` take up to `bytes` of dynamic shared memory (fails if the
// device cannot).  The limit is raised to the device's opt-in maximum and
// never lowered: it is a per-function setting shared by every context and by
// launches already captured in CUDA graphs.
template <class K>
void allow_dyn_smem(K* kernel, size_t bytes) {
    int dev = 0, optin = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    cuda_check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "cudaDeviceGetAttribute");
    cudaFuncAttributes fa{};
    cuda_check(cudaFuncGetAttributes(&fa, kernel), "cudaFuncGetAttributes");
    const int room = optin - (int)fa.sharedSizeBytes;
    if ((long long)bytes > room) fail(WT_ERR_UNSUPPORTED, "kernel needs more shared memory than the device has");
    if (fa.maxDynamicSharedSizeBytes < room)
        cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, room),
                   "cudaFuncSetAttribute");
}

// Owning device buffer.
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        if (count == n && p) return;
        release();
        if (count == 0) return;
        if (fault_enabled("alloc")) fail(WT_ERR_OOM, "injected allocation failure (WT_FAULT=alloc)");
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            fail(WT_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
        }
        n = count;
    }
    void zero(cudaStream_t s) { if (n) WT_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
    void take(DBuf& o) {
        release();
        p = o.p;
        n = o.n;
        o.p = nullptr;
        o.n = 0;
    }
    void upload(const T* host, size_t count, cudaStream_t s) {
        alloc(count);
        if (count) WT_CUDA(cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void download(T* host, size_t count, cudaStream_t s) const {
        if (count) WT_CUDA(cudaMemcpyAsync(host, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
};

// ---------------------------------------------------------------- dense FP64
// Row-major matrices.  op(A) is M x K, op(B) is K x N, C is M x N.
void dgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
           const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
           bool lower_only = false);
void symmetrize_from_lower(cudaStream_t s, double* A, int n, int lda);
void symmetrize_avg(cudaStream_t s, const double* F, double* C, int n);   // C = (F + F^T)/2
void transpose(cudaStream_t s, const double* A, int rows, int cols, double* At);
// Lower Cholesky in place (upper triangle untouched).  Sets d_err on failure.
void cholesky(cudaStream_t s, double* A, int n, int lda, int* d_err);
// Solve L Y = B (lower) in place on B [n x nrhs].
void trsm_lower(cudaStream_t s, const double* L, int n, int ldl, double* B, int nrhs, int ldb);
// Solve L^T X = B in place on B.
void trsm_lower_t(cudaStream_t s, const double* L, int n, int ldl, double* B, int nrhs, int ldb);
// Symmetric eigendecomposition by parallel two-sided Jacobi: A (n x n,
// destroyed) -> eigenvalues w[n] (unsorted), eigenvectors V (n x n, columns).
// Returns the number of sweeps; sets d_err on non-convergence.  Couplings
// below abs_tol are not rotated (for rank-deficient Gram matrices, whose
// rounding-level directions would otherwise keep rotating).
int jacobi_eig(cudaStream_t s, double* A, int n, double* w, double* V, int* d_err, int max_sweeps = 40,
               double abs_tol = 0.0);
// Symmetric eigendecomposition by Householder tridiagonalisation, divide and conquer on the
// tridiagonal matrix and blocked back-transformation: A (n x n row-major, destroyed) ->
// eigenvalues w[n] (ascending), eigenvectors V (n x n, columns).  Sets d_err (DERR_TIMEOUT) if a
// leaf's QL iteration does not converge.
void sym_eig(cudaStream_t s, double* A, int n, double* w, double* V, int* d_err);
// Singular value decomposition of the rows of A [m][n] (row-major, destroyed)
// by one-sided (Hestenes) Jacobi: on return the rows of A are mutually
// orthogonal (row i = sigma_i u_i^T), V [m][m] holds the accumulated rotations
// (A_in = V^T A_out; V = NULL: not accumulated) and sigma[m] the row norms (unsorted).  Returns the number
// of sweeps; sets d_err (DERR_TIMEOUT) when max_sweeps do not converge (unless the largest
// relative coupling still rotated in the last sweep is below 1e-10; coupling_out returns it).
int onesided_jacobi_rows(cudaStream_t s, double* A, int m, int n, int lda, double* V, double* sigma, int* d_err,
                         int max_sweeps = 40, double* coupling_out = nullptr);
// Householder QR with column pivoting, M P = Q1 R, of the ns x nt matrix whose column j is row j of
// the row-major array M [nt][ld] (ns >= nt; M is destroyed): R [nt][nt] row-major upper triangular,
// piv[i] (device) = the column of M that became column i.  Only R and P are formed.
void qrcp_r(cudaStream_t s, double* M, int ns, int nt, int ld, double* R, int* piv);
// out[r][n] = scale[r] * A[idx[r]][:]  (idx, scale: device arrays of `rows`)
void gather_rows_scaled(cudaStream_t s, const double* A, int n, int lda, const int* idx, const double* scale,
                        int rows, double* out);
// y = alpha * A x + beta * y  (A row-major M x N, or its transpose)
void dgemv(cudaStream_t s, bool ta, int M, int N, double alpha, const double* A, int lda,
           const double* x, double beta, double* y);
double dnrm2(cudaStream_t s, const double* x, size_t n, double* d_scratch);
void fill(cudaStream_t s, double* x, size_t n, double v);
void axpy(cudaStream_t s, size_t n, double a, const double* x, double* y);
void dscal(cudaStream_t s, size_t n, double a, double* x);
// A[i][j] += alpha * u[i] * v[j]
void rank1(cudaStream_t s, int M, int N, double alpha, const double* u, const double* v, double* A, int lda);
void copy_block(cudaStream_t s, const double* src, int lds, double* dst, int ldd, int rows, int cols);
void scale_columns(cudaStream_t s, double* A, int M, int N, int lda, const double* d);
void scale_rows(cudaStream_t s, double* A, int M, int N, int lda, const double* d);
void column_norms(cudaStream_t s, const double* A, int M, int N, int lda, double* out);
void get_diag(cudaStream_t s, const double* A, int n, int lda, double* out);

// One tensor-core expansion H[t][c][p] = sum_m W[t][m] E[c][m][p] (FP32).
struct ExpandJob {
    const float* E;      // [3][r_pad][npts], 16-byte aligned
    int r_pad;           // 32
    int r;               // rows in use (rows >= r of E may hold anything)
    const float* W;      // [nt][32]
    int nt;
    size_t npts;
    float* H;            // [nt][3][npts]
};
bool expand_tc_available();
int expand_tc_max_jobs();
void expand_tc(cudaStream_t s, const float* E, int r_pad, int r, const float* W, int nt, size_t npts, float* H,
               int* d_err);
// Several expansions in one persistent launch (at most max_ctas CTAs, 0 = one
// per SM; nch = time samples per accumulator chunk: 64, 128 or 256; nepi =
// epilogue warps: 8, 12 or 16; vec = floats per store: 4, 2 or 1).
void expand_tc_jobs(cudaStream_t s, const ExpandJob* jobs, int n_jobs, int max_ctas, int nch, int* d_err,
                    int nepi = 8, int vec = 4);

}  // namespace wt
