// Shared pieces of the FP32 spectral kernels (plane and z passes live in
// their own translation units so that their many register-FFT instances
// compile in parallel).
#pragma once
#include "k_fft.cuh"
#include "fft_core.cuh"
#include "warp_fft.cuh"

namespace wt {

// Register-FFT lengths compiled in: elements per lane R = N / W.
#define WT_FOR_EACH_R(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(12) X(14) X(15) X(16) X(24)

// Two-pass y transforms of Ny = ny2 in {64, 128}: ny2 = A B with A = 8 lanes per row; each
// row holds the A x B exchange matrix (skewed, no padding).
__host__ __device__ constexpr int plane_y2_a(int ny2) { return ny2 == 256 ? 16 : 8; }
// odd row pitch (complex units, Ny + 1 entries; = 1 mod 16 for the power-of-two Ny of the
// two-pass forms)
__host__ __device__ constexpr int plane_ldp_of(int ny, int /*ny2*/) { return (ny + 1) | 1; }
inline size_t plane_smem(const GridDev& g, int ny2 = 0) {
    const int nxh = g.Nx / 2 + 1;
    return ((size_t)nxh * plane_ldp_of(g.Ny, ny2) + g.Ny + g.Nx + ny2) * sizeof(C2<float>);
}
// (Ny, elements per lane of the x transforms) compiled with two-pass y transforms: 16 or 32 lanes per x
// line (a 256 x 256 plane does not fit one block's shared memory on either y path)
#define WT_FOR_EACH_Y2(X) X(64, 2) X(64, 4) X(128, 4) X(128, 8)
// Row pitch of a staged z line pair: room for the skewed inputs and the skewed outputs.
__host__ __device__ __forceinline__ int zpass_pitch(int nz, int R) {
    const int a = (nz - 1) + (nz - 1) / R + 1, b = (nz - 1) + ((nz - 1) >> 4) + 1;
    return (a > b ? a : b) | 1;
}
inline size_t zpass_smem(const GridDev& g, int lb, int R) {
    const size_t S = (size_t)zpass_pitch(g.Nz, R);
    // staged pairs, the twiddle table (nz) and the skewed phase table (nz + nz / R)
    return ((size_t)(lb / 2) * S + 2 * (size_t)g.Nz + (size_t)g.Nz / R + 1) * sizeof(C2<float>);
}

// Lines of a z pass: the staged planes hold rows y0 .. y0 + ys - 1 (every x) of each k_z plane,
// laid out [y - y0][x]; the outputs go to H's point order (x Ny + y) Nz + z of the full grid.
struct ZLines {
    int ys, y0;
    int discard;    // two-pass z pass: drop the staged rows' L2 lines once read (no write-back)
};

// Launchers (k_fft32_plane.cu, k_fft32_z.cu): dispatch on the register-FFT length.
// r = 0 with ny2: the two-pass x transforms as well
void plane_allow(int r, int ny2, size_t smem);
bool plane_y2_supported(int ny, int r);
void plane_launch(int r, bool xdirect, int ny2, dim3 grid, cudaStream_t s, const GridDev& g, const C2<float>* rho,
                  const C2<float>* twy, const C2<float>* twx, float* R, int mode);
void zpass_allow(int r, size_t smem);
void zpass_launch(int r, int lb, dim3 grid, cudaStream_t s, const GridDev& g, const float* R, const C2<float>* twz,
                  const C2<float>* zsh, float* out, size_t out_sb, size_t out_sc, ZLines zl);
// Two-pass shared-memory z FFT (k_fft32_z2.cu), Nz in {64, 96, 128, 160, 192, 224, 256, 384}.
bool zpass2_supported(int nz);
size_t zpass2_smem(int A, int B, int lb);
void zpass2_allow(int nz);
void zpass2_launch(int lb, dim3 grid, cudaStream_t s, const GridDev& g, const float* R, const C2<float>* twz,
                   const C2<float>* zsh, float* out, size_t out_sb, size_t out_sc, ZLines zl);

}  // namespace wt
