// Dense expansion of the FP32 basis fields over time (plain FP32 FMA form):
//   H[t][c][p] = sum_m W[t][m] E[c][m][p]
// One thread per grid point holds that point's r basis values; the time
// coefficients sit in shared memory.  Reference form of the tensor-core
// expansion kernel, kept for cross-checks.
#include "wt_internal.cuh"

namespace wt {

template <int R>
__global__ void __launch_bounds__(256) expand_simt_kernel(const float* __restrict__ E, const float* __restrict__ W,
                                                         int nt, int ldw, size_t npts, float* __restrict__ H) {
    extern __shared__ float ws[];
    for (int e = threadIdx.x; e < nt * R; e += blockDim.x) ws[e] = W[(size_t)(e / R) * ldw + (e % R)];
    __syncthreads();
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (p >= npts) return;
    float e[R];
#pragma unroll
    for (int m = 0; m < R; ++m) e[m] = E[((size_t)c * R + m) * npts + p];
    for (int t = 0; t < nt; ++t) {
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < R; ++m) acc = fmaf(ws[t * R + m], e[m], acc);
        H[((size_t)t * 3 + c) * npts + p] = acc;
    }
}

void expand_simt(cudaStream_t s, const float* E, int r_pad, const float* W, int nt, int ldw, size_t npts, float* H) {
    dim3 grid((unsigned)((npts + 255) / 256), 3);
    size_t sh = (size_t)nt * r_pad * sizeof(float);
    if (r_pad == 32) {
        allow_dyn_smem(expand_simt_kernel<32>, sh);
        expand_simt_kernel<32><<<grid, 256, sh, s>>>(E, W, nt, ldw, npts, H);
    } else if (r_pad == 64) {
        allow_dyn_smem(expand_simt_kernel<64>, sh);
        expand_simt_kernel<64><<<grid, 256, sh, s>>>(E, W, nt, ldw, npts, H);
    } else {
        fail(WT_ERR_UNSUPPORTED, "expansion rank must be padded to 32 or 64");
    }
    WT_LAUNCH("expand_simt");
}

}  // namespace wt
