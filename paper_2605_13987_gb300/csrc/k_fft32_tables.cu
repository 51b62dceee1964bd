// FP32 basis fields from per-column lateral tables.
//
// Sec. 3 builds the potential from rescaled and translated chunks of the
// fundamental solution.  In the spectral form used here every column c
// contributes, for each z mode k_z and field component a, a lateral field
//
//   T_c[a][k_z](x, y) = IFFT_2D( multiplier_a(k) e^{-i (k_x x_c + k_y y_c)} )
//
// that depends on the geometry only (grid, column position), not on the
// charges.  A basis charge vector b enters only through its column
// z-transforms Z[b][c][k_z], so the per-plane fields that the z pass turns
// into basis fields are the linear combination
//
//   R[b][a][k_z](x, y) = sum_c Z[b][c][k_z] T_c[a][k_z](x, y),
//
// the same sum that the deposit forms in the spectral domain, moved after
// the lateral transform.  The tables are built once per context with the
// deposit and plane kernels (a unit z-transform per column); an extension then
// needs this combination and the z pass only.  The combination runs over
// slabs of y rows (the autotuner picks their height): a small slab's planes
// stay in L2 for the z pass; larger ones go through DRAM but take fewer,
// longer launches.
#include "k_fft32_common.cuh"

#include <type_traits>

namespace wt {

// Coefficients of the combination in the order a block reads them: ZcT[k_z][c][b] (32 per column,
// zero for b >= r) from the column transforms Zc[b][c][k_z].
__global__ void combine_coeffs_kernel(const float* __restrict__ Zc, int r, int n_cols, int Nz,
                                      float* __restrict__ ZcT) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)Nz * n_cols * 32) return;
    const int b = (int)(e % 32);
    const size_t q = e / 32;
    const int c = (int)(q % n_cols), kz = (int)(q / n_cols);
    ZcT[e] = b < r ? Zc[((size_t)b * n_cols + c) * Nz + kz] : 0.f;
}

constexpr int kCombineCC = 8;      // columns per asynchronous copy group
constexpr int kCombineStages = 3;  // copy groups in flight
constexpr int kCombineMinBlocks = 5;   // resident blocks per SM the register budget allows

// One block of 128 threads per (line chunk, k_z, component); each thread takes VEC
// consecutive lines and accumulates RB basis vectors in registers.  A thread's table values
// T[c][a][k_z][its lines] arrive by asynchronous copies in groups of kCombineCC columns,
// kCombineStages groups in flight, into shared memory that only this thread reads back, so
// the column loop overlaps the copies of later columns and needs no barrier; the coefficients
// ZcT[k_z][c][0..RB) are staged once per block, contiguous, as [c][RB].
// T: [n_cols][3][Nz][nxy] (plane layout [y][x]); ZcT: [Nz][n_cols][32];
// R: [r][3][Nz][nl], line j of the slab = line off + j of the plane.
template <int RB, int VEC>
__global__ void __launch_bounds__(128, kCombineMinBlocks) column_combine_kernel(const float* __restrict__ T,
                                                             const float* __restrict__ ZcT, int r, int n_cols,
                                                             int Nz, size_t nxy, size_t off, int nl,
                                                             float* __restrict__ R) {
    using V = typename std::conditional<VEC == 4, float4, typename std::conditional<VEC == 2, float2, float>::type>::type;
    constexpr int LPB = 128 * VEC;                    // lines per block
    constexpr int CC = kCombineCC, NS = kCombineStages;
    extern __shared__ __align__(16) float smem[];
    float* zs = smem;                                 // [n_cols][RB]
    V* ts = reinterpret_cast<V*>(smem + n_cols * RB); // [NS][CC][128] vectors of VEC lines
    const int kz = blockIdx.y, comp = blockIdx.z;
    const float* zrow = ZcT + (size_t)kz * n_cols * 32;
    for (int e = threadIdx.x; e < n_cols * RB; e += blockDim.x) zs[e] = zrow[(e / RB) * 32 + e % RB];
    const int j0 = blockIdx.x * LPB;
    const int j = j0 + threadIdx.x * VEC;
    const bool act = j < nl;                          // nl is a multiple of VEC
    const size_t cstride = (size_t)3 * Nz * nxy;
    const float* tp = T + ((size_t)comp * Nz + kz) * nxy + off + (act ? j : 0);
    const int ngroups = (n_cols + CC - 1) / CC;
    // group g: columns g CC .. into stage g % NS; every thread commits one (possibly empty) group
    // per call so that the group counts stay uniform
    auto issue = [&](int g) {
        if (act && g < ngroups) {
            V* dst0 = ts + (size_t)(g % NS) * CC * 128 + threadIdx.x;
            const int c1 = min(n_cols, (g + 1) * CC);
            for (int c = g * CC; c < c1; ++c) {
                const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(dst0 + (c - g * CC) * 128));
                const float* src = tp + c * cstride;
                if constexpr (sizeof(V) == 16)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
                else if constexpr (sizeof(V) == 8)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int g = 0; g < NS - 1; ++g) issue(g);
    __syncthreads();                                  // zs staged
    float acc[RB][VEC];
#pragma unroll
    for (int b = 0; b < RB; ++b)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[b][v] = 0.f;
    for (int g = 0; g < ngroups; ++g) {
        issue(g + NS - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");   // group g has landed
        if (!act) continue;
        const V* tg = ts + (size_t)(g % NS) * CC * 128 + threadIdx.x;
        const float* zg = zs + g * CC * RB;
        // one column: RB x VEC FMAs from one table vector and RB broadcast coefficients
        auto column = [&](const V q, const float* zc) {
            const float* t = reinterpret_cast<const float*>(&q);
            const float4* z4 = reinterpret_cast<const float4*>(zc);
#pragma unroll
            for (int b4 = 0; b4 < RB / 4; ++b4) {
                const float4 z = z4[b4];
                const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[4 * b4 + i][v] = fmaf(zz[i], t[v], acc[4 * b4 + i][v]);
            }
        };
        if ((g + 1) * CC <= n_cols) {
#pragma unroll
            for (int cc = 0; cc < CC; ++cc) column(tg[cc * 128], zg + cc * RB);   // a full group, unrolled
        } else {
            for (int cc = 0; cc < n_cols - g * CC; ++cc) column(tg[cc * 128], zg + cc * RB);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!act) return;
    float* rp = R + ((size_t)comp * Nz + kz) * nl + j;
    const size_t bstride = (size_t)3 * Nz * nl;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        if (b >= r) break;
        V o;
        float* of = reinterpret_cast<float*>(&o);
#pragma unroll
        for (int v = 0; v < VEC; ++v) of[v] = acc[b][v];
        *reinterpret_cast<V*>(rp + b * bstride) = o;
    }
}

template <int RB, int VEC>
static void combine_launch(cudaStream_t s, const float* T, const float* Zc, int r, int n_cols, int Nz, size_t nxy,
                           size_t off, int nl, float* R) {
    const size_t sh = ((size_t)n_cols * RB + (size_t)kCombineStages * kCombineCC * 128 * VEC) * sizeof(float);
    allow_dyn_smem(column_combine_kernel<RB, VEC>, sh);
    dim3 gd((unsigned)((nl + 128 * VEC - 1) / (128 * VEC)), (unsigned)Nz, 3);
    column_combine_kernel<RB, VEC><<<gd, 128, sh, s>>>(T, Zc, r, n_cols, Nz, nxy, off, nl, R);
}

void combine_coeffs(cudaStream_t s, const float* Zc, int r, int n_cols, int Nz, float* ZcT) {
    const size_t n = (size_t)Nz * n_cols * 32;
    if (!n) return;
    combine_coeffs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Zc, r, n_cols, Nz, ZcT);
    WT_LAUNCH("combine_coeffs");
}

void column_combine(cudaStream_t s, const float* T, const float* Zc, int r, int n_cols, int Nz, size_t nxy,
                    size_t off, int nl, float* R, bool one_line) {
    if (r < 1 || r > 32) fail(WT_ERR_ARG, "column combination: rank must be 1..32");
    if (n_cols < 1 || n_cols > 96) fail(WT_ERR_UNSUPPORTED, "the lateral tables take 1 to 96 columns");
    // vectors of VEC lines when every line chunk starts aligned to them
    const uintptr_t al = reinterpret_cast<uintptr_t>(T) | reinterpret_cast<uintptr_t>(R);
    // (one_line: one line per thread, fewer registers and more resident warps)
    const bool v4 = !one_line && (off % 4 == 0) && (nl % 4 == 0) && (nxy % 4 == 0) && (al % 16 == 0);
    const bool v2 = !one_line && (off % 2 == 0) && (nl % 2 == 0) && (nxy % 2 == 0) && (al % 8 == 0);
    if (r <= 8) {
        if (v4) combine_launch<8, 4>(s, T, Zc, r, n_cols, Nz, nxy, off, nl, R);
        else combine_launch<8, 1>(s, T, Zc, r, n_cols, Nz, nxy, off, nl, R);
    } else if (r <= 16) {
        if (v4) combine_launch<16, 4>(s, T, Zc, r, n_cols, Nz, nxy, off, nl, R);
        else combine_launch<16, 1>(s, T, Zc, r, n_cols, Nz, nxy, off, nl, R);
    } else {
        if (v2) combine_launch<32, 2>(s, T, Zc, r, n_cols, Nz, nxy, off, nl, R);
        else combine_launch<32, 1>(s, T, Zc, r, n_cols, Nz, nxy, off, nl, R);
    }
    WT_LAUNCH("column_combine");
}

}  // namespace wt
