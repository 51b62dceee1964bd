// Tangent-linear kernels of the derivative of Eq. 1 currents with respect to
// the column resistivity, radius and the lateral scale (pitch).  FP64.
#include "wt_internal.cuh"

namespace wt {

// Derivative lateral tables, one block per (target lateral position, source
// column) combination, threads over mz.  With dx, dy the lateral offset,
// (ux, uy) the collocation point's radial unit vector and r the radius:
//   mode 0 (radius):  dL/dr   = sum wx wy [-kx sin(kx dx) cos(ky dy) ux - ky cos(kx dx) sin(ky dy) uy] / |k|^2
//   mode 1 (scale):   dL/dlam - 2 L, with
//          dL/dlam = sum wx wy [kx r ux sin(kx dx) cos(ky dy) + ky r uy cos(kx dx) sin(ky dy)] / |k|^2
//                  + sum wx wy 2 (kx^2 + ky^2) cos(kx dx) cos(ky dy) / |k|^4
// (-2 L: the prefactor 1/(eps V') scales as lambda^-2).  k = 0 excluded.
__global__ void lateral_dtable_kernel(const double* __restrict__ dxy, const double* __restrict__ uxy, int hx, int hy,
                                      int nz, double Lx, double Ly, double Lz, double radius, int mode,
                                      double* __restrict__ out) {
    extern __shared__ double sh[];
    double* cx = sh;
    double* sx = cx + hx;
    double* cy = sx + hx;
    double* sy = cy + hy;
    const int combo = blockIdx.x;
    const double dx = dxy[2 * combo], dy = dxy[2 * combo + 1];
    const double ux = uxy[2 * combo], uy = uxy[2 * combo + 1];
    for (int m = threadIdx.x; m < hx; m += blockDim.x) sincospi(2.0 * m * dx / Lx, &sx[m], &cx[m]);
    for (int m = threadIdx.x; m < hy; m += blockDim.x) sincospi(2.0 * m * dy / Ly, &sy[m], &cy[m]);
    __syncthreads();
    for (int mz = threadIdx.x; mz < nz; mz += blockDim.x) {
        const double kz = kPi * mz / Lz;
        double acc = 0.0;
        for (int mx = 0; mx < hx; ++mx) {
            const double kx = 2.0 * kPi * mx / Lx;
            const double wx = mx ? 2.0 : 1.0;
            for (int my = 0; my < hy; ++my) {
                const double ky = 2.0 * kPi * my / Ly;
                const double kp2 = kx * kx + ky * ky;
                const double k2 = kp2 + kz * kz;
                if (k2 <= 0.0) continue;
                const double w = wx * (my ? 2.0 : 1.0);
                const double ik2 = 1.0 / k2;
                if (mode == 0) {
                    acc -= w * (kx * sx[mx] * cy[my] * ux + ky * cx[mx] * sy[my] * uy) * ik2;
                } else {
                    const double cc = cx[mx] * cy[my];
                    acc += w * ((kx * radius * ux * sx[mx] * cy[my] + ky * radius * uy * cx[mx] * sy[my]) * ik2 +
                                2.0 * kp2 * cc * ik2 * ik2 - 2.0 * cc * ik2);
                }
            }
        }
        out[(size_t)combo * nz + mz] = acc;
    }
}

void green_lateral_deriv(cudaStream_t s, const double* dxy, const double* uxy, int n_combo, int Nx, int Ny, int Nz,
                         double Lx, double Ly, double Lz, double radius, int mode, double* out) {
    size_t sh = (size_t)(Nx + Ny) * sizeof(double);
    lateral_dtable_kernel<<<n_combo, 256, sh, s>>>(dxy, uxy, Nx / 2, Ny / 2, Nz, Lx, Ly, Lz, radius, mode, out);
    WT_LAUNCH("lateral_dtable");
}

// inv[k][l] = 1/(mu_k - mu_l) for well separated pairs, 0 on the diagonal and
// for near-degenerate pairs (handled by the limit form in modal_tangent).
__global__ void inv_gap_kernel(const double* __restrict__ mu, int n, double* __restrict__ inv) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    int k = idx / n, l = idx % n;
    const double d = mu[k] - mu[l];
    const double scale = fmax(fabs(mu[k]), fabs(mu[l]));
    inv[idx] = (k != l && fabs(d) > 1e-9 * scale) ? 1.0 / d : 0.0;
}
void modal_inv_gap(cudaStream_t s, const double* mu, int n, double* inv) {
    size_t tot = (size_t)n * n;
    inv_gap_kernel<<<(tot + 255) / 256, 256, 0, s>>>(mu, n, inv);
    WT_LAUNCH("inv_gap");
}

// out[k][t] = sum_l Om[k][l] amp[l] F_kl(t_n) + E[k][t] c[k], with E[k][t] = exp(-mu_k t_n) and the
// divided difference F_kl(t) = (E_k - E_l)/(mu_k - mu_l), F_kk = -t E_k, near-degenerate pairs
// -t (E_k + E_l)/2.  (Daleckii-Krein derivative of the matrix exponential.)  One block per k,
// threads over t; the row of Om * amp and of the inverse gaps sit in shared memory.
__global__ void modal_tangent_kernel(const double* __restrict__ Om, const double* __restrict__ amp,
                                     const double* __restrict__ inv, const double* __restrict__ E,
                                     const double* __restrict__ t, const double* __restrict__ c, int n, int nt,
                                     double* __restrict__ out) {
    extern __shared__ double sh[];
    double* ma = sh;
    double* iv = sh + n;
    const int k = blockIdx.x;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        ma[l] = Om[(size_t)k * n + l] * amp[l];
        iv[l] = inv[(size_t)k * n + l];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        const double ek = E[(size_t)k * nt + j], tj = t[j];
        double acc = 0.0;
        for (int l = 0; l < n; ++l) {
            const double el = E[(size_t)l * nt + j];
            double f;
            if (l == k) f = -tj * ek;
            else if (iv[l] != 0.0) f = (ek - el) * iv[l];
            else f = -tj * 0.5 * (ek + el);
            acc = fma(ma[l], f, acc);
        }
        out[(size_t)k * nt + j] = acc + ek * c[k];
    }
}
void modal_tangent(cudaStream_t s, const double* Om, const double* amp, const double* inv, const double* E,
                   const double* t, const double* c, int n, int nt, double* out) {
    size_t sh = 2 * (size_t)n * sizeof(double);
    if (sh > 200 * 1024) fail(WT_ERR_UNSUPPORTED, "modal tangent: too many modes for shared memory");
    allow_dyn_smem(modal_tangent_kernel, sh);
    modal_tangent_kernel<<<n, 256, sh, s>>>(Om, amp, inv, E, t, c, n, nt, out);
    WT_LAUNCH("modal_tangent");
}

// Omega[k][l] = Sh[k][l] - Ah[k][l] mu[l]
__global__ void omega_kernel(const double* __restrict__ Sh, const double* __restrict__ Ah,
                             const double* __restrict__ mu, int n, double* __restrict__ Om) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    const int l = idx % n;
    Om[idx] = Sh[idx] - (Ah ? Ah[idx] * mu[l] : 0.0);
}
void modal_omega(cudaStream_t s, const double* Sh, const double* Ah, const double* mu, int n, double* Om) {
    size_t tot = (size_t)n * n;
    omega_kernel<<<(tot + 255) / 256, 256, 0, s>>>(Sh, Ah, mu, n, Om);
    WT_LAUNCH("omega");
}

// Q[i][t] = sum over the rows: Q += phi[i] (every t)
__global__ void add_row_const_kernel(double* Q, int n, int nt, const double* __restrict__ phi) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * nt) return;
    Q[idx] += phi[idx / nt];
}
void add_row_const(cudaStream_t s, double* Q, int n, int nt, const double* phi) {
    size_t tot = (size_t)n * nt;
    add_row_const_kernel<<<(tot + 255) / 256, 256, 0, s>>>(Q, n, nt, phi);
    WT_LAUNCH("add_row_const");
}

// partial[b] = sum over a slice of i * di (FP64 accumulation of FP32 currents)
__global__ void dot_f32_kernel(const float* __restrict__ a, const float* __restrict__ b, size_t n, double* out) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc = fma((double)a[i], (double)b[i], acc);
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
__global__ void dot_f64_kernel(const double* __restrict__ a, const double* __restrict__ b, size_t n, double* out) {
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
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
double dot_f64(cudaStream_t s, const double* a, const double* b, size_t n, double* d_scratch) {
    WT_CUDA(cudaMemsetAsync(d_scratch, 0, sizeof(double), s));
    if (n) {
        int blocks = (int)std::min<size_t>(1024, (n + 255) / 256);
        dot_f64_kernel<<<blocks, 256, 0, s>>>(a, b, n, d_scratch);
        WT_LAUNCH("dot_f64");
    }
    double h = 0;
    WT_CUDA(cudaMemcpyAsync(&h, d_scratch, sizeof(double), cudaMemcpyDeviceToHost, s));
    WT_CUDA(cudaStreamSynchronize(s));
    return h;
}

double dot_f32(cudaStream_t s, const float* a, const float* b, size_t n, double* d_scratch) {
    WT_CUDA(cudaMemsetAsync(d_scratch, 0, sizeof(double), s));
    if (n) {
        int blocks = (int)std::min<size_t>(1024, (n + 255) / 256);
        dot_f32_kernel<<<blocks, 256, 0, s>>>(a, b, n, d_scratch);
        WT_LAUNCH("dot_f32");
    }
    double h = 0;
    WT_CUDA(cudaMemcpyAsync(&h, d_scratch, sizeof(double), cudaMemcpyDeviceToHost, s));
    WT_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace wt
