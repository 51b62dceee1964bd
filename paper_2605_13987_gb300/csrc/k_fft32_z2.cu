// FP32 z pass of the bulk extension, two-pass shared-memory form for
// Nz = A B with A in {8, 16} lanes per line pair and B built from the factors
// 2, 3, 5, 7 (Nz = 64, 96, 128, 160, 192, 224, 256, 384): the same cosine
// and sine series as the register-FFT z pass (k_fft32_z.cu, Makhoul's
// reordering of the DCT-III with two real lines per complex FFT), with the
// N-point FFT split as
//   X[c + B d] = sum_a w_A^{a d} w_N^{a c} sum_b Y[a + A b] w_B^{b c}:
// pass 1, lane a of a line's A lanes: one B-point DFT in registers, the
// twiddles w_N^{a c}, the results to shared memory; pass 2: the B columns'
// A-point DFTs shared out over the A lanes (ceil(B / A) per lane).  Register
// DFTs with compile-time twiddles; no shuffles.
#include "k_fft32_common.cuh"

namespace wt {

// Staged-pair pitch (complex): inputs (N), the pass-1 matrix A (B + 1) and
// the z-ordered outputs (N + 8); = 1 mod 16, so that the staging stores, the
// column reads and the two output halves fall into distinct banks.
__host__ __device__ constexpr int zpass2_pitch(int A, int B) {
    const int n = A * B + (A > 8 ? A : 8);
    return ((n + 15) / 16) * 16 + 1;
}
size_t zpass2_smem(int A, int B, int lb) {
    // staged pairs, e^{i pi m / 2N} and the per-lane twiddles w_N^{a c} ([c][a])
    return ((size_t)(lb / 2) * zpass2_pitch(A, B) + 2 * (size_t)A * B) * sizeof(C2<float>);
}

// blocks per SM the kernel is compiled for (register budget): four for DFTs up to 16 points (64
// registers, no spills; shared memory allows four at 32 lines per block), two for the larger ones
__host__ __device__ constexpr int zpass2_min_blocks(int A, int B) { return B > 16 ? 2 : 4; }

template <int A, int B, int LB>
__global__ void __launch_bounds__(256, zpass2_min_blocks(A, B)) f32_zpass2_kernel(GridDev g, const float* __restrict__ R,
                                                            const C2<float>* __restrict__ twz,
                                                            const C2<float>* __restrict__ zsh, float* __restrict__ out,
                                                            size_t out_sb, size_t out_sc, ZLines zl) {
    constexpr int N = A * B, S = zpass2_pitch(A, B), G = 32 / A, NP = LB / 2;
    constexpr int RC = (B + A - 1) / A;          // pass-2 columns per lane
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.Nx, ny = g.Ny;
    const size_t nxy = (size_t)nx * zl.ys;      // staged lines: rows y0 .. y0 + ys - 1 of each plane
    const int comp = blockIdx.y, b = blockIdx.z;
    const size_t L0 = (size_t)blockIdx.x * LB;
    C2<float>* cs = reinterpret_cast<C2<float>*>(smem_raw);                 // [NP][S]
    C2<float>* zs = cs + (size_t)NP * S;                                    // [N]
    C2<float>* tl = zs + N;                                                 // [B][A]: w_N^{a c} at c A + a
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        zs[e] = zsh[e];
        const int c = e / A, a = e % A;
        tl[e] = twz[a * c];                                                 // a c < N
    }
    if (nxy % 4 == 0) {
        // thread t stages lines 4 (t % (LB / 4)) .. + 3 of rows t / (LB / 4) + k (256 / (LB / 4)): one
        // 16-byte load per row (four lines, two line pairs), two 8-byte stores into the pairs' rows;
        // the loads of a batch are all in flight before the first store
        constexpr int TPR = LB / 4, MS = 256 / TPR;
        const int l4 = 4 * (threadIdx.x % TPR), m0 = threadIdx.x / TPR;
        const bool lin = L0 + l4 < nxy;                  // nxy and L0 are multiples of 4: all four or none
        const float4* sp = reinterpret_cast<const float4*>(R + ((size_t)b * 3 + comp) * N * nxy + L0 + l4);
        const size_t rs = nxy / 4;
        C2<float>* d0 = cs + (size_t)(l4 >> 1) * S;
        C2<float>* d1 = d0 + S;
#pragma unroll 8
        for (int m = m0; m < N; m += MS) {
            const float4 v = lin ? __ldg(sp + (size_t)m * rs) : make_float4(0.f, 0.f, 0.f, 0.f);
            d0[m] = C2<float>{v.x, v.y};
            d1[m] = C2<float>{v.z, v.w};
        }
    } else {
        // thread t stages line t % LB for rows t / LB + k (256 / LB)
        constexpr int MS = 256 / LB;
        const int l = threadIdx.x % LB, m0 = threadIdx.x / LB;
        const bool lin = L0 + l < nxy;
        const float* sp = R + ((size_t)b * 3 + comp) * N * nxy + L0 + l;
        float* dst = reinterpret_cast<float*>(cs) + 2 * (size_t)(l >> 1) * S + (l & 1);
#pragma unroll 16
        for (int m = m0; m < N; m += MS) dst[2 * m] = lin ? sp[(size_t)m * nxy] : 0.f;
    }
    __syncthreads();
    if constexpr (LB >= 32) {
        // the staged rows are scratch that only this block reads: invalidate their L2 lines so that
        // the slab never goes back to DRAM (whole 128-byte lines inside the slab row only; the
        // host enables this when every row starts on a 128-byte boundary)
        if (zl.discard) {
            constexpr int SEG = LB / 32;
            const float* base = R + ((size_t)b * 3 + comp) * N * nxy + L0;
            for (int e = threadIdx.x; e < N * SEG; e += blockDim.x) {
                const int m = e / SEG, q = e - m * SEG;
                if (L0 + (size_t)(q + 1) * 32 <= nxy)
                    asm volatile("discard.global.L2 [%0], 128;" ::"l"(base + (size_t)m * nxy + q * 32) : "memory");
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / A, gl = lane % A;
    const bool sine = comp == 2;
    float* ob = out + (size_t)b * out_sb + (size_t)comp * out_sc;
    for (int base = warp * G; base < NP; base += 8 * G) {
        const int f = base + grp;                 // lines 2f, 2f+1 of this block
        const bool act = f < NP;
        C2<float>* cf = cs + (size_t)(act ? f : 0) * S;
        // pass 1: Y_m = (p - i q) e^{i pi m / 2N} at m = gl + A j, then the B-point DFT over j
        C2<float> v[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int m = gl + A * j;
            const C2<float> cm = act ? cf[m] : C2<float>{0.f, 0.f};
            const C2<float> cr = (act && m) ? cf[N - m] : C2<float>{0.f, 0.f};
            const C2<float> p = sine ? cr : cm, q = sine ? cm : cr;
            v[j] = cmul(C2<float>{p.x + q.y, p.y - q.x}, zs[m]);
        }
        __syncwarp();                             // every lane has read its inputs before the matrix overwrites them
        reg_dft_k<B>(v);
#pragma unroll
        for (int c = 1; c < B; ++c) v[c] = cmul(v[c], tl[c * A + gl]);
        if (act)
#pragma unroll
            for (int c = 0; c < B; ++c) cf[gl * (B + 1) + c] = v[c];
        __syncwarp();
        // pass 2: column c = gl + A r (< B), A-point DFT over a -> X[c + B d]
        C2<float> o[RC * A];
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const bool col = act && gl + A * r < B;
            C2<float> u[A];
#pragma unroll
            for (int a = 0; a < A; ++a) u[a] = col ? cf[a * (B + 1) + gl + A * r] : C2<float>{0.f, 0.f};
            reg_dft_c<A>(u);
#pragma unroll
            for (int d = 0; d < A; ++d) o[r * A + d] = u[d];
        }
        __syncwarp();                             // the matrix is read before the outputs overwrite it
        // X[j] belongs at z = 2j (j < N/2, d < A/2) or z = 2N - 1 - 2j; stored even z at z/2,
        // odd z at N/2 + 8 + (z - 1)/2; the sine series takes (-1)^z / 2
        if (act)
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                if (gl + A * r >= B) break;
#pragma unroll
                for (int d = 0; d < A; ++d) {
                    const int j = gl + A * r + B * d;
                    C2<float> y = o[r * A + d];
                    if (sine) {
                        const float sg = (2 * d < A) ? 0.5f : -0.5f;
                        y = {sg * y.x, sg * y.y};
                    }
                    cf[(2 * d < A) ? j : N / 2 + 8 + (N - 1 - j)] = y;
                }
            }
        __syncwarp();
        if (!act) continue;
        const size_t La = L0 + 2 * f, Lb = La + 1;
        const size_t pa = ((La % nx) * ny + zl.y0 + La / nx) * (size_t)N;
        const size_t pb = ((Lb % nx) * ny + zl.y0 + Lb / nx) * (size_t)N;
        if (Lb < nxy) {
            // lane takes z = 2 h and 2 h + 1: two 64-bit reads (the even and the odd half) feed one
            // 8-byte store per line, each warp store a whole 128-byte line segment
            for (int h = gl; h < N / 2; h += A) {
                const C2<float> ev = cf[h], od = cf[N / 2 + 8 + h];
                *reinterpret_cast<float2*>(ob + pa + 2 * h) = make_float2(ev.x, od.x);
                *reinterpret_cast<float2*>(ob + pb + 2 * h) = make_float2(ev.y, od.y);
            }
        } else if (La < nxy) {
            for (int z = gl; z < N; z += A) ob[pa + z] = cf[(z & 1) ? N / 2 + 8 + (z >> 1) : (z >> 1)].x;
        }
    }
}

// Two-pass forms compiled in: (A, B) for Nz = 64, 96, 128, 160, 192, 224, 256, 384.
#define WT_FOR_EACH_Z2(X) X(8, 8) X(8, 12) X(8, 16) X(8, 20) X(8, 24) X(16, 14) X(16, 16) X(16, 24)

static bool z2_shape(int nz, int* A, int* B) {
    switch (nz) {
        case 64: *A = 8; break;
        case 96: *A = 8; break;
        case 128: *A = 8; break;
        case 160: *A = 8; break;
        case 192: *A = 8; break;
        case 224: *A = 16; break;
        case 256: *A = 16; break;
        case 384: *A = 16; break;
        default: return false;
    }
    *B = nz / *A;
    return true;
}
bool zpass2_supported(int nz) {
    int A, B;
    return z2_shape(nz, &A, &B);
}

void zpass2_allow(int nz) {
    int A, B;
    if (!z2_shape(nz, &A, &B))
        fail(WT_ERR_UNSUPPORTED, "two-pass z FFT needs Nz in {64, 96, 128, 160, 192, 224, 256, 384}");
    const size_t sz = zpass2_smem(A, B, 64);
#define WT_CASE(AA, BB) \
    if (A == AA && B == BB) { \
        allow_dyn_smem(f32_zpass2_kernel<AA, BB, 16>, sz); \
        allow_dyn_smem(f32_zpass2_kernel<AA, BB, 32>, sz); \
        allow_dyn_smem(f32_zpass2_kernel<AA, BB, 64>, sz); \
    }
    WT_FOR_EACH_Z2(WT_CASE)
#undef WT_CASE
}

void zpass2_launch(int lb, dim3 gz, cudaStream_t s, const GridDev& g, const float* R, const C2<float>* tz,
                   const C2<float>* zz, float* out, size_t out_sb, size_t out_sc, ZLines zl) {
    int A, B;
    if (!z2_shape(g.Nz, &A, &B))
        fail(WT_ERR_UNSUPPORTED, "two-pass z FFT needs Nz in {64, 96, 128, 160, 192, 224, 256, 384}");
    const size_t sz = zpass2_smem(A, B, lb);
#define WT_CASE(AA, BB) \
    if (A == AA && B == BB) { \
        if (lb == 16) f32_zpass2_kernel<AA, BB, 16><<<gz, 256, sz, s>>>(g, R, tz, zz, out, out_sb, out_sc, zl); \
        else if (lb == 32) f32_zpass2_kernel<AA, BB, 32><<<gz, 256, sz, s>>>(g, R, tz, zz, out, out_sb, out_sc, zl); \
        else f32_zpass2_kernel<AA, BB, 64><<<gz, 256, sz, s>>>(g, R, tz, zz, out, out_sb, out_sc, zl); \
    }
    WT_FOR_EACH_Z2(WT_CASE)
#undef WT_CASE
    WT_LAUNCH("f32_zpass2");
}

}  // namespace wt
