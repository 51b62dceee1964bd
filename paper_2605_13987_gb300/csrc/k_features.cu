// Signal-shape features of sampled waveforms (Eq. 1 currents or shaped
// signals) and their first-order sensitivities, for the geometry scans of
// Sec. 5, where sensor variants (bias-electrode diameter, thickness) are
// compared by the shape of their signals.  Per waveform x_m at
// tau_m = t0 + m dt:
//   A       x_k, k the first index of the largest |x_m|; s = sign(A), y = s x
//   t_peak  tau_k + dt delta, delta the vertex of the parabola through k-1, k, k+1
//   Q       dt sum_m x_m
//   t_f     leading-edge crossing of l = f y_k (f = lo, hi, cfd): j the last
//           index below k with y_j < l, linear interpolation between j, j+1;
//           tau_0 when there is none.
// The decisions k and j are taken in FP32 (|x|, s x exact, l one rounded
// product, exact comparisons); the features are evaluated in FP64.  For a
// tangent waveform dx the sensitivities are the derivatives at fixed
// decisions.  One warp per waveform.
#include "wt_internal.cuh"

namespace wt {

constexpr int kNF = WT_N_FEATURES;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_max_int(int v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(256) features_kernel(const float* __restrict__ x, const float* __restrict__ dx,
                                                       int n_dir, int n_tracks, int n, double t0, double dt,
                                                       float3 fr, double* __restrict__ f, double* __restrict__ df) {
    const int tr = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (tr >= n_tracks) return;                          // whole warps leave together
    const float* row = x + (size_t)tr * n;
    // first index of the largest |x|
    float best = -1.f;
    int bi = n;
    double sum = 0.0;
    for (int m = lane; m < n; m += 32) {
        const float v = row[m];
        const float a = fabsf(v);
        if (a > best) { best = a; bi = m; }
        sum += (double)v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    sum = warp_sum(sum);
    const int k = bi < n ? bi : 0;                       // every sample NaN: no maximum (features unspecified)
    const float A = row[k];
    const float s = A < 0.f ? -1.f : 1.f;
    const float yk = s * A;
    const float lv[3] = {__fmul_rn(fr.x, yk), __fmul_rn(fr.y, yk), __fmul_rn(fr.z, yk)};
    int jl[3] = {-1, -1, -1};
    for (int m = lane; m < k; m += 32) {
        const float y = s * row[m];
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (y < lv[q]) jl[q] = m;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) jl[q] = warp_max_int(jl[q]);
    const double sd = (double)s;
    auto Y = [&](int m) { return sd * (double)row[m]; };
    const double fq[3] = {(double)fr.x, (double)fr.y, (double)fr.z};
    if (lane == 0) {
        double* o = f + (size_t)tr * kNF;
        double delta = 0.0;
        if (k > 0 && k < n - 1) {
            const double den = Y(k - 1) - 2.0 * Y(k) + Y(k + 1);
            if (den != 0.0) delta = (Y(k - 1) - Y(k + 1)) / (2.0 * den);
        }
        o[0] = (double)A;
        o[1] = t0 + dt * ((double)k + delta);
        o[2] = dt * sum;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int j = jl[q];
            o[3 + q] = j < 0 ? t0 : t0 + dt * ((double)j + ((double)lv[q] - Y(j)) / (Y(j + 1) - Y(j)));
        }
    }
    for (int d = 0; d < n_dir; ++d) {
        const float* drow = dx + ((size_t)d * n_tracks + tr) * n;
        double dsum = 0.0;
        for (int m = lane; m < n; m += 32) dsum += (double)drow[m];
        dsum = warp_sum(dsum);
        if (lane == 0) {
            auto dY = [&](int m) { return sd * (double)drow[m]; };
            double* o = df + ((size_t)d * n_tracks + tr) * kNF;
            double dpk = 0.0;
            if (k > 0 && k < n - 1) {
                const double den = Y(k - 1) - 2.0 * Y(k) + Y(k + 1);
                if (den != 0.0) {
                    const double num = Y(k - 1) - Y(k + 1);
                    const double dnum = dY(k - 1) - dY(k + 1);
                    const double dden = dY(k - 1) - 2.0 * dY(k) + dY(k + 1);
                    dpk = dt * (dnum * den - num * dden) / (2.0 * den * den);
                }
            }
            o[0] = (double)drow[k];
            o[1] = dpk;
            o[2] = dt * dsum;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int j = jl[q];
                double v = 0.0;
                if (j >= 0) {
                    const double dd = Y(j + 1) - Y(j);
                    v = dt * ((fq[q] * dY(k) - dY(j)) * dd - ((double)lv[q] - Y(j)) * (dY(j + 1) - dY(j))) / (dd * dd);
                }
                o[3 + q] = v;
            }
        }
    }
}

void features_launch(cudaStream_t s, const float* x, int n_tracks, int n, double t0, double dt, float lo, float hi,
                     float cfd, const float* dx, int n_dir, double* f, double* df) {
    if (n_tracks > 0) {
        const int blocks = (int)(((size_t)n_tracks * 32 + 255) / 256);
        features_kernel<<<blocks, 256, 0, s>>>(x, dx, n_dir, n_tracks, n, t0, dt, make_float3(lo, hi, cfd), f, df);
    }
    WT_LAUNCH("features");
}

// y += x (FP32), for summing current tangents.
__global__ void add_f32_kernel(size_t n, const float* __restrict__ x, float* __restrict__ y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}
void add_f32(cudaStream_t s, size_t n, const float* x, float* y) {
    if (!n) return;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    add_f32_kernel<<<blocks, 256, 0, s>>>(n, x, y);
    WT_LAUNCH("add_f32");
}

}  // namespace wt
