// FP32 z pass of the bulk extension (see k_fft32.cu): cosine and sine series
// along z, one register-FFT length per template instance.
#include "k_fft32_common.cuh"

namespace wt {

// Cosine (W_x, W_y) or sine (W_z) series along z at the cell centres,
//   cos: f(z_n) = X_0 + 2 sum_{m>0} X_m cos(pi m (2n+1) / 2N)
//   sin: f(z_n) = sum_{m>0} S_m sin(pi m (2n+1) / 2N),        N = Nz,
// for LB (x, y) lines per block, two real lines (a, b) per complex N-point
// warp FFT (Makhoul's reordering of the DCT-III):
//   Y_m = (c_m - i c_{N-m}) e^{i pi m / 2N},  c = X^a + i X^b,  c_N = 0,
//   y = sum_m Y_m e^{2 pi i m k / N}  (Hermitian per line: y^a + i y^b),
//   f(z_{2k}) = y_k,  f(z_{2k+1}) = y_{N-1-k}.
// The sine series is the cosine series of the reversed coefficients
// (X'_m = S_{N-m}) with signs (-1)^n: Y_m = (c_{N-m} - i c_m) e^{i pi m / 2N}
// and f(z_n) = (-1)^n y_n / 2 after the same reordering.
// Lines L = y Nx + x of the plane kernel's layout; output in H's point
// order (x Ny + y) Nz + z, staged per line pair for coalesced stores.
// grid (ceil(Nx Ny / LB), 3, nb).
// Skewed index of coefficient m in a staged line pair: a gap every R entries
// makes the per-lane chunk stride R + 1, so the reads are free of bank conflicts.
__device__ __forceinline__ int zskew(int m, int R) { return m + m / R; }

template <int RZ, int LB>
__global__ void __launch_bounds__(256, RZ <= 8 ? 3 : 2) f32_zpass_kernel(GridDev g, const float* __restrict__ R,
                                                        const C2<float>* __restrict__ twz,
                                                        const C2<float>* __restrict__ zsh, float* __restrict__ out,
                                                        size_t out_sb, size_t out_sc, ZLines zl) {
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.Nx, ny = g.Ny, nz = g.Nz;
    const size_t nxy = (size_t)nx * zl.ys;      // staged lines: rows y0 .. y0 + ys - 1 of each plane
    const int comp = blockIdx.y, b = blockIdx.z;
    const size_t L0 = (size_t)blockIdx.x * LB;
    const int S = zpass_pitch(nz, RZ);                                      // odd pair pitch
    C2<float>* cs = reinterpret_cast<C2<float>*>(smem_raw);                 // [LB/2][S]
    C2<float>* tw = cs + (size_t)(LB / 2) * S;                              // [nz]
    C2<float>* zs = tw + nz;                                                // [zskew(nz-1)+1], skewed
    for (int e = threadIdx.x; e < nz; e += blockDim.x) {
        tw[e] = twz[e];
        zs[zskew(e, RZ)] = zsh[e];          // read at m = j1 + RZ gl: the skew spreads the banks
    }
    if (nxy % 4 == 0) {
        // thread t stages lines 4 (t % (LB / 4)) .. + 3 (two line pairs) of rows t / (LB / 4) + k:
        // one 16-byte load per row, two 8-byte stores
        constexpr int TPR = LB / 4, MS = 256 / TPR;
        const int l4 = 4 * (threadIdx.x % TPR), m0 = threadIdx.x / TPR;
        const bool lin = L0 + l4 < nxy;                  // nxy and L0 are multiples of 4: all four or none
        const float4* sp = reinterpret_cast<const float4*>(R + ((size_t)b * 3 + comp) * nz * nxy + L0 + l4);
        const size_t rs = nxy / 4;
        C2<float>* d0 = cs + (size_t)(l4 >> 1) * S;
        C2<float>* d1 = d0 + S;
#pragma unroll 8
        for (int m = m0; m < nz; m += MS) {
            const float4 v = lin ? __ldg(sp + (size_t)m * rs) : make_float4(0.f, 0.f, 0.f, 0.f);
            d0[zskew(m, RZ)] = C2<float>{v.x, v.y};
            d1[zskew(m, RZ)] = C2<float>{v.z, v.w};
        }
    } else {
        // thread t stages line t % LB for rows t / LB + k (256 / LB); loads batched ahead of the stores
        constexpr int MS = 256 / LB;
        const int l = threadIdx.x % LB, m0 = threadIdx.x / LB;
        const bool lin = L0 + l < nxy;
        const float* sp = R + ((size_t)b * 3 + comp) * nz * nxy + L0 + l;
        float* dst = reinterpret_cast<float*>(cs) + 2 * (size_t)(l >> 1) * S + (l & 1);
#pragma unroll 8
        for (int m = m0; m < nz; m += MS) dst[2 * zskew(m, RZ)] = lin ? sp[(size_t)m * nxy] : 0.f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = nz / RZ, G = 32 / W, grp = lane / W, gl = lane % W;
    const int k2 = warp_fft_k2(gl, W);
    const bool sine = comp == 2;
    LaneTw<RZ> lt;
    lane_twiddles<RZ>(tw, gl, W, false, lt);
    float* ob = out + (size_t)b * out_sb + (size_t)comp * out_sc;
    for (int base = warp * G; base < LB / 2; base += 8 * G) {
        const int f = base + grp;                 // lines 2f, 2f+1 of this block
        const bool act = f < LB / 2;              // groups past the block's pairs only join the shuffles
        C2<float>* cf = cs + (size_t)(act ? f : 0) * S;
        C2<float> v[RZ];
#pragma unroll
        for (int j1 = 0; j1 < RZ; ++j1) {
            const int m = j1 + RZ * gl;
            const C2<float> cm = act ? cf[zskew(m, RZ)] : C2<float>{0.f, 0.f};
            const C2<float> cr = (act && m) ? cf[zskew(nz - m, RZ)] : C2<float>{0.f, 0.f};
            const C2<float> p = sine ? cr : cm, q = sine ? cm : cr;     // Y = (p - i q) e^{i pi m / 2N}
            v[j1] = cmul(C2<float>{p.x + q.y, p.y - q.x}, zs[zskew(m, RZ)]);
        }
        warp_fft_t<RZ>(v, gl, W, lt, tw);
        __syncwarp();                             // every lane of the group has read its inputs
        if (act)
#pragma unroll
            for (int k1 = 0; k1 < RZ; ++k1) {
                const int j = k2 + W * k1;
                const int z = 2 * j < nz ? 2 * j : 2 * nz - 2 * j - 1;
                C2<float> y = v[k1];
                if (sine) {
                    const float sg = (z & 1) ? -0.5f : 0.5f;
                    y = {sg * y.x, sg * y.y};
                }
                cf[z + (z >> 4)] = y;             // z order with a gap every 16: conflict-free both ways
            }
        __syncwarp();
        if (!act) continue;
        const size_t La = L0 + 2 * f, Lb = La + 1;
        const size_t pa = ((La % nx) * ny + zl.y0 + La / nx) * (size_t)nz;
        const size_t pb = ((Lb % nx) * ny + zl.y0 + Lb / nx) * (size_t)nz;
        if (Lb < nxy) {
            for (int z = gl; z < nz; z += W) {      // one 64-bit read per lane feeds both lines
                const C2<float> y = cf[z + (z >> 4)];
                ob[pa + z] = y.x;
                ob[pb + z] = y.y;
            }
        } else if (La < nxy) {
            for (int z = gl; z < nz; z += W) ob[pa + z] = cf[z + (z >> 4)].x;
        }
    }
}

void zpass_allow(int r, size_t sz) {
    switch (r) {
#define WT_CASE(R) case R: { \
        allow_dyn_smem(f32_zpass_kernel<R, 16>, sz); \
        allow_dyn_smem(f32_zpass_kernel<R, 32>, sz); \
        allow_dyn_smem(f32_zpass_kernel<R, 64>, sz); break; }
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
        default: fail(WT_ERR_UNSUPPORTED, "register-FFT length not compiled in");
    }
}

void zpass_launch(int r, int lb, dim3 gz, cudaStream_t s, const GridDev& g, const float* R, const C2<float>* tz,
                  const C2<float>* zz, float* out, size_t out_sb, size_t out_sc, ZLines zl) {
    const size_t sz = zpass_smem(g, lb, r);
    switch (r) {
#define WT_CASE(RR) case RR: \
        if (lb == 16) f32_zpass_kernel<RR, 16><<<gz, 256, sz, s>>>(g, R, tz, zz, out, out_sb, out_sc, zl); \
        else if (lb == 32) f32_zpass_kernel<RR, 32><<<gz, 256, sz, s>>>(g, R, tz, zz, out, out_sb, out_sc, zl); \
        else f32_zpass_kernel<RR, 64><<<gz, 256, sz, s>>>(g, R, tz, zz, out, out_sb, out_sc, zl); \
        break;
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
        default: fail(WT_ERR_UNSUPPORTED, "register-FFT length not compiled in");
    }
    WT_LAUNCH("f32_zpass");
}

}  // namespace wt
