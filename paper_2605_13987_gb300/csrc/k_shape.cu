// Front-end shaping of Eq. 1 currents: CR-(RC)^n impulse response of unit
// area, h(t) = (t / tau)^n e^(-t / tau) / (n! tau), convolved on the output
// grid by the rectangle rule, v_m = G sum_k h(k dt) dt i_(m-k) + sigma w_m
// (the paper names the electronics' response as a step of the signal chain
// without a transfer function; this is its parameterised form).
#include "wt_internal.cuh"

namespace wt {

// One block per track: the taps (FP64) and the track's currents sit in shared
// memory; threads over output samples, FP64 accumulation.
__global__ void shape_kernel(const float* __restrict__ cur, int n_out, int n_taps, double dt, double tau, int order,
                             double scale, double noise_rms, const float* __restrict__ noise, float* __restrict__ v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* taps = reinterpret_cast<double*>(smem_raw);
    float* row = reinterpret_cast<float*>(taps + n_taps);
    const size_t tr = blockIdx.x;
    for (int k = threadIdx.x; k < n_taps; k += blockDim.x) {
        const double x = k * dt / tau;
        taps[k] = scale * pow(x, (double)order) * exp(-x);        // scale = G dt / (n! tau)
    }
    for (int m = threadIdx.x; m < n_out; m += blockDim.x) row[m] = cur[tr * n_out + m];
    __syncthreads();
    for (int m = threadIdx.x; m < n_out; m += blockDim.x) {
        double acc = 0.0;
        const int kmax = min(m, n_taps - 1);
        for (int k = 0; k <= kmax; ++k) acc = fma(taps[k], (double)row[m - k], acc);
        if (noise) acc += noise_rms * (double)noise[tr * n_out + m];
        v[tr * n_out + m] = (float)acc;
    }
}

void shape_launch(cudaStream_t s, const float* cur, int n_tracks, int n_out, double dt, double tau, int order,
                  double gain, double noise_rms, const float* noise, float* v) {
    // taps beyond t = (order + 60) tau are below e^-50 of the peak and are dropped
    const double span = (order + 60.0) * tau / dt;
    const int n_taps = (int)std::max(1.0, std::min((double)n_out, std::ceil(span)));
    const size_t sh = (size_t)n_taps * sizeof(double) + (size_t)n_out * sizeof(float);
    allow_dyn_smem(shape_kernel, sh);
    double fact = 1.0;
    for (int k = 2; k <= order; ++k) fact *= k;
    const double scale = gain * dt / (fact * tau);
    if (n_tracks > 0)
        shape_kernel<<<n_tracks, 256, sh, s>>>(cur, n_out, n_taps, dt, tau, order, scale, noise_rms, noise, v);
    WT_LAUNCH("shape");
}

}  // namespace wt
