// Batched pseudo-spectral extension: charge vectors -> field components on
// the voxel grid.  Templated on the arithmetic type (float: fast path basis
// fields; double: plain FP64 path).
#pragma once
#include "wt_internal.cuh"

namespace wt {

struct FftPlan {
    int N;
    int ns;
    int r[16];
};
FftPlan make_plan(int N);   // radices 4, 2, 3, 5, 7; fails for other prime factors

struct GridDev {
    int Nx, Ny, Nz;
    double Lx, Ly, Lz;
    double pref;            // 1 / (eps V')
};

// Per-context spectral machinery for one precision.
template <class T>
struct Spectral {
    GridDev g{};
    int n_cols = 0;
    FftPlan pz{}, py{}, px{};
    DBuf<double> col_xy;          // [n_cols][2]
    DBuf<T> tw_z, tw_y, tw_x;     // interleaved complex twiddles e^{+2 pi i k / N}
    void init(const GridDev& gd, const std::vector<double>& xy, cudaStream_t s);
    // Zc [nb][n_cols][Nz] (column z-transforms of nb charge vectors) ->
    // out[b * out_sb + c * out_sc + (x Ny + y) Nz + z], c = 0..2.
    // G is a scratch buffer of nb * 3 * (Nx/2+1) * Ny * Nz complex T.
    void fields(const T* Zc, int nb, T* G, T* out, size_t out_sb, size_t out_sc, cudaStream_t s) const;
    size_t scratch_elems(int nb) const { return (size_t)nb * 3 * (g.Nx / 2 + 1) * g.Ny * g.Nz * 2; }
};

// Column z-transform of charge vectors: Zc[b][c][mz] = sum_{j in c} q[b][j] 2 cos(pi mz z_j / Lz).
// q: [nb][n_src] (double), zcos [n_src][Nz] = 2 cos(pi mz z_j / Lz), col_off [n_cols+1].
template <class T>
void column_ztransform(cudaStream_t s, const double* q, int nb, int n_src, int ldq, const double* zcos,
                       const int* col_off, int n_cols, int Nz, T* Zc);
void column_cos_table(cudaStream_t s, const double* zsrc, int n_src, int Nz, double Lz, double* zcos);

}  // namespace wt

namespace wt {

// FP32 basis-field path: deposit -> per-k_z-plane lateral inverse FFT ->
// z cosine/sine series, written z-contiguous in the H point order.
struct Fast32 {
    GridDev g{};
    int n_cols = 0;
    int rxy = 0, rz = 0;           // register-FFT elements per lane (lateral, z); lanes per line = N / R
    bool xdirect = false;          // x transforms store from registers (else staged for coalescing)
    bool zsm = false;              // z pass: two-pass shared-memory FFT (else the register FFT of rz)
    bool ysm = false;              // y transforms: two-pass shared-memory FFT (rxy then serves x only)
    bool xsm = false;              // x transforms two-pass as well (with ysm; rxy, xdirect unused)
    DBuf<float> tw_y, tw_x, tw_z;
    DBuf<float> phx, phy, zsh;     // complex tables
    void init(const GridDev& gd, const std::vector<double>& xy, cudaStream_t s);
    // register-FFT shapes: the elements per lane that give a power-of-two lane count 4..32
    static std::vector<int> radix_options(int N);
    void set_radix(int r_xy, int r_z, bool z_two_pass = false, bool y_two_pass = false, bool x_two_pass = false);
    static bool z_two_pass_supported(int Nz);
    static bool y_two_pass_supported(int Ny, int r_xy);
    // rho scratch: nb * Nz * (Nx/2+1) * Ny complex; R scratch: nb * 3 * Nz * Nx * Ny real.
    size_t rho_elems(int nb) const { return (size_t)nb * g.Nz * (g.Nx / 2 + 1) * g.Ny * 2; }
    size_t r_elems(int nb) const { return (size_t)nb * 3 * g.Nz * g.Nx * g.Ny; }
    // mode 0: the field, 1: its lateral-scale derivative; lb: (x, y) lines per z-pass block (16, 32, 64)
    void fields(const float* Zc, int nb, float* rho, float* R, float* out, size_t out_sb, size_t out_sc,
                cudaStream_t s, int mode = 0, int lb = 32) const;
    // deposit and plane passes only: R [nb][3][Nz][Ny][Nx] (plane layout [y][x])
    void lateral(const float* Zc, int nb, float* rho, float* R, cudaStream_t s, int mode = 0) const;
    // z pass of rows y0 .. y0 + ys - 1: R [nb][3][Nz][ys][Nx] -> out[b * out_sb + c * out_sc + (x Ny + y) Nz + z]
    // discard: with the two-pass z pass, invalidate the consumed rows of R in L2 (R is scratch;
    // needs Nx ys a multiple of 32, R 128-byte aligned and lb >= 32, else ignored)
    void zlines(const float* R, int nb, int y0, int ys, float* out, size_t out_sb, size_t out_sc, cudaStream_t s,
                int lb, bool discard = false) const;
};

// R[b][a][kz][j] = sum_c Zc[b][c][kz] T[c][a][kz][off + j] for j < nl, b < r <= 32: the planes of the
// per-column lateral tables T [n_cols][3][Nz][nxy] combined by the basis vectors' column z-transforms,
// read as ZcT [Nz][n_cols][32] (combine_coeffs).
void column_combine(cudaStream_t s, const float* T, const float* ZcT, int r, int n_cols, int Nz, size_t nxy,
                    size_t off, int nl, float* R, bool one_line = false);
// ZcT[kz][c][b] = Zc[b][c][kz] for b < r, 0 for r <= b < 32 (Zc: [r][n_cols][Nz]).
void combine_coeffs(cudaStream_t s, const float* Zc, int r, int n_cols, int Nz, float* ZcT);

}  // namespace wt
