// Fundamental-solution tables and the fit matrix (Abstract: fundamental
// solutions impose the boundary conditions; Sec. 3: point charges adjusted
// in magnitude; |k|^2 spectral division).  FP64.
//
// Band-limited periodic Green's function with a mirror image in z:
//   Phi(t; s) = pref sum_k exp(i k_perp.(t - s)_perp) [e^{i kz (tz - sz)} + e^{i kz (tz + sz)}] / |k|^2
//             = 2 pref sum_{mz >= 0} w(mz) L(dxy, kz) cos(kz tz) cos(kz sz),
//   L(dxy, kz) = sum_{mx, my >= 0} wx wy cos(kx dx) cos(ky dy) / |k|^2   (k = 0 excluded),
// w = 1 for index 0 and 2 otherwise (the +- mode pairs).
#include "wt_internal.cuh"

namespace wt {

// T[mx][my][mz] = 1 / |k|^2 for mx < Nx/2, my < Ny/2, mz < Nz; 0 at the origin.
__global__ void invk2_kernel(int hx, int hy, int nz, double Lx, double Ly, double Lz, double* T) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t tot = (size_t)hx * hy * nz;
    if (idx >= tot) return;
    int mz = idx % nz;
    int my = (idx / nz) % hy;
    int mx = idx / ((size_t)nz * hy);
    double kx = 2.0 * kPi * mx / Lx, ky = 2.0 * kPi * my / Ly, kz = kPi * mz / Lz;
    double k2 = kx * kx + ky * ky + kz * kz;
    T[idx] = k2 > 0.0 ? 1.0 / k2 : 0.0;
}

// One block per lateral offset (combo); threads over mz.
__global__ void lateral_table_kernel(const double* __restrict__ dxy, int hx, int hy, int nz, double Lx, double Ly,
                                     const double* __restrict__ T, double* __restrict__ Lout) {
    extern __shared__ double sh[];
    double* cx = sh;
    double* cy = sh + hx;
    const int combo = blockIdx.x;
    const double dx = dxy[2 * combo], dy = dxy[2 * combo + 1];
    for (int m = threadIdx.x; m < hx; m += blockDim.x) cx[m] = (m ? 2.0 : 1.0) * cospi(2.0 * m * dx / Lx);
    for (int m = threadIdx.x; m < hy; m += blockDim.x) cy[m] = (m ? 2.0 : 1.0) * cospi(2.0 * m * dy / Ly);
    __syncthreads();
    for (int mz = threadIdx.x; mz < nz; mz += blockDim.x) {
        double acc = 0.0;
        for (int mx = 0; mx < hx; ++mx) {
            double inner = 0.0;
            const double* t = T + (size_t)mx * hy * nz + mz;
            for (int my = 0; my < hy; ++my) inner = fma(cy[my], t[(size_t)my * nz], inner);
            acc = fma(cx[mx], inner, acc);
        }
        Lout[(size_t)combo * nz + mz] = acc;
    }
}

// cos(pi m z / Lz) tables: C[i][m] for heights z[i].
__global__ void cos_table_kernel(const double* __restrict__ z, int n, int nz, double Lz, double* __restrict__ C) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * nz) return;
    int i = idx / nz, m = idx % nz;
    C[idx] = cospi((double)m * z[i] / Lz);
}

// Block description for P assembly: P[row0 + p][col0 + j] for p < nrow, j < ncol.
struct PBlock {
    int row0, nrow, col0, ncol;
    int ct0;      // first row of the collocation cos table
    int cs0;      // first row of the source cos table
    int combo;    // lateral table row
};

// P_block = 2 pref Ct diag(w L) Cs^T, tiled 64x64 with K = mz staged 16 at a time.
__global__ void __launch_bounds__(256) pblock_kernel(const PBlock* __restrict__ blocks, const double* __restrict__ Ct,
                                                     const double* __restrict__ Cs, const double* __restrict__ Lt,
                                                     int nz, double pref2, double* __restrict__ P, int ldp) {
    const PBlock B = blocks[blockIdx.z];
    const int bm = blockIdx.y * 64, bn = blockIdx.x * 64;
    if (bm >= B.nrow || bn >= B.ncol) return;
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    const double* L = Lt + (size_t)B.combo * nz;
    for (int k0 = 0; k0 < nz; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int mm = e >> 4, kk = e & 15;
            int gm = bm + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < B.nrow && gk < nz) v = Ct[(size_t)(B.ct0 + gm) * nz + gk] * (gk ? 2.0 : 1.0) * L[gk];
            As[kk][mm] = v;
            int gn = bn + mm;
            double u = 0.0;
            if (gn < B.ncol && gk < nz) u = Cs[(size_t)(B.cs0 + gn) * nz + gk];
            Bs[kk][mm] = u;
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
        int gm = bm + ty + 16 * i;
        if (gm >= B.nrow) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = bn + tx + 16 * j;
            if (gn >= B.ncol) continue;
            P[(size_t)(B.row0 + gm) * ldp + B.col0 + gn] = pref2 * acc[i][j];
        }
    }
}

// Rt[j][k] = sum over the collocation rows i that interpolate node j of
// S[i][j] * A[i][k]  (CSC lists of S).  Thread per (j, k).
__global__ void ats_kernel(const double* __restrict__ A, int lda, int ncolA, const int* __restrict__ sp,
                           const int* __restrict__ si, const double* __restrict__ sw, double* __restrict__ Rt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (k >= ncolA) return;
    double acc = 0.0;
    for (int e = sp[j]; e < sp[j + 1]; ++e) acc = fma(sw[e], A[(size_t)si[e] * lda + k], acc);
    Rt[(size_t)j * ncolA + k] = acc;
}

// Res[i][j] += S[i][j] using the CSC lists (each (i, j) appears once).
__global__ void add_s_kernel(double* __restrict__ R, int ldr, int ns, const int* __restrict__ sp,
                             const int* __restrict__ si, const double* __restrict__ sw, double scale) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    for (int e = sp[j]; e < sp[j + 1]; ++e) R[(size_t)si[e] * ldr + j] += scale * sw[e];
}

__global__ void set_column_kernel(double* A, int M, int lda, int col, double v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) A[(size_t)i * lda + col] = v;
}

// ------------------------------------------------------------ host wrappers
void green_invk2(cudaStream_t s, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz, double* T) {
    size_t tot = (size_t)(Nx / 2) * (Ny / 2) * Nz;
    invk2_kernel<<<(tot + 255) / 256, 256, 0, s>>>(Nx / 2, Ny / 2, Nz, Lx, Ly, Lz, T);
    WT_LAUNCH("invk2");
}
void green_lateral(cudaStream_t s, const double* dxy, int n_combo, int Nx, int Ny, int Nz, double Lx, double Ly,
                   const double* T, double* L) {
    size_t sh = (size_t)(Nx / 2 + Ny / 2) * sizeof(double);
    lateral_table_kernel<<<n_combo, 256, sh, s>>>(dxy, Nx / 2, Ny / 2, Nz, Lx, Ly, T, L);
    WT_LAUNCH("lateral_table");
}
void green_cos_table(cudaStream_t s, const double* z, int n, int Nz, double Lz, double* C) {
    size_t tot = (size_t)n * Nz;
    cos_table_kernel<<<(tot + 255) / 256, 256, 0, s>>>(z, n, Nz, Lz, C);
    WT_LAUNCH("cos_table");
}
void green_pblocks(cudaStream_t s, const void* blocks, int n_blocks, int max_rows, int max_cols, const double* Ct,
                   const double* Cs, const double* L, int Nz, double pref, double* P, int ldp) {
    dim3 grid((max_cols + 63) / 64, (max_rows + 63) / 64, n_blocks);
    pblock_kernel<<<grid, 256, 0, s>>>(static_cast<const PBlock*>(blocks), Ct, Cs, L, Nz, 2.0 * pref, P, ldp);
    WT_LAUNCH("pblock");
}
size_t pblock_size() { return sizeof(PBlock); }
void pack_pblock(void* dst, int row0, int nrow, int col0, int ncol, int ct0, int cs0, int combo) {
    PBlock* b = static_cast<PBlock*>(dst);
    *b = PBlock{row0, nrow, col0, ncol, ct0, cs0, combo};
}
void fit_ats(cudaStream_t s, const double* A, int lda, int nrow, int ncol, const int* sp, const int* si,
             const double* sw, int ns, double* Rt) {
    (void)nrow;
    dim3 grid((ncol + 127) / 128, ns);
    ats_kernel<<<grid, 128, 0, s>>>(A, lda, ncol, sp, si, sw, Rt);
    WT_LAUNCH("ats");
}
void fit_add_s(cudaStream_t s, double* R, int ldr, int ns, const int* sp, const int* si, const double* sw,
               double scale) {
    add_s_kernel<<<(ns + 127) / 128, 128, 0, s>>>(R, ldr, ns, sp, si, sw, scale);
    WT_LAUNCH("add_s");
}
void set_column(cudaStream_t s, double* A, int M, int lda, int col, double v) {
    set_column_kernel<<<(M + 255) / 256, 256, 0, s>>>(A, M, lda, col, v);
    WT_LAUNCH("set_column");
}

}  // namespace wt
