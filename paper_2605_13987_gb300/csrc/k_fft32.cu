// FP32 basis fields of the bulk extension (Abstract; Sec. 1 discrete Fourier
// transforms; Sec. 3 |k|^2 spectral division), three kernels per batch of
// charge vectors, all FP32 (the phases come from FP64-built tables):
//   deposit: rho^[b][mz][mx][my] = sum_c e^{-i kx x_c} e^{-i ky y_c} Zc[b][c][mz]
//   plane:   for one (b, component, mz): multiply by the component's factor
//            (-i k_a w / |k|^2, or 2 kz / |k|^2 for W_z), inverse FFT along y,
//            half-spectrum -> real inverse FFT along x; R[b][c][mz][x][y]
//   zpass:   cosine (W_x, W_y) or sine (W_z) series along z, two real lines
//            packed in one length-2Nz complex FFT; out[b][c][x][y][z].
#include "k_fft32_common.cuh"

namespace wt {

__global__ void f32_tables_kernel(const double* __restrict__ xy, int n_cols, int nxh, int ny, int nz, double Lx,
                                  double Ly, float* __restrict__ phx, float* __restrict__ phy,
                                  float* __restrict__ zsh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double sn, cs;
    if (i < n_cols * nxh) {
        const int c = i / nxh, mx = i % nxh;
        sincospi(-2.0 * mx * xy[2 * c] / Lx, &sn, &cs);
        phx[2 * i] = (float)cs;
        phx[2 * i + 1] = (float)sn;
    }
    if (i < n_cols * ny) {
        const int c = i / ny, my = i % ny;
        const int mys = my < ny / 2 ? my : my - ny;
        sincospi(-2.0 * mys * xy[2 * c + 1] / Ly, &sn, &cs);
        phy[2 * i] = (float)cs;
        phy[2 * i + 1] = (float)sn;
    }
    if (i < nz) {
        sincospi((double)i / (2.0 * nz), &sn, &cs);
        zsh[2 * i] = (float)cs;
        zsh[2 * i + 1] = (float)sn;
    }
}

// rho^ planes; grid (Nz, nb, F32_DEP_SPLIT): each block takes a slice of the
// m_x rows 0 <= m_x < Nx/2 of one plane (the x Nyquist row is never read: the
// plane pass keeps it zero), warps over 4-row x 64-column tiles, lanes over m_y.
// Shared tables: px[c][mx] = e^{-i kx x_c} (the block's rows),
// qy[c][my] = e^{-i ky y_c} Zc[b][c][mz].
constexpr int F32_DEP_SPLIT = 4;
__host__ __device__ inline int deposit_rows(int nx) {          // rows per block, a multiple of 4
    return (((nx / 2 + F32_DEP_SPLIT - 1) / F32_DEP_SPLIT) + 3) & ~3;
}
__global__ void f32_deposit_kernel(GridDev g, int n_cols, const C2<float>* __restrict__ phx,
                                   const C2<float>* __restrict__ phy, const float* __restrict__ Zc,
                                   C2<float>* __restrict__ rho) {
    extern __shared__ unsigned char smem_raw[];
    const int mz = blockIdx.x, b = blockIdx.y;
    const int nxh = g.Nx / 2 + 1, nxq = g.Nx / 2, ny = g.Ny;
    const int rows = deposit_rows(g.Nx);
    const int mx0 = blockIdx.z * rows, mx1 = min(nxq, mx0 + rows);
    if (mx0 >= mx1) return;
    const int nr = mx1 - mx0;
    C2<float>* px = reinterpret_cast<C2<float>*>(smem_raw);        // [n_cols][rows]
    C2<float>* qy = px + (size_t)n_cols * rows;                      // [n_cols][ny]
    for (int e = threadIdx.x; e < n_cols * rows; e += blockDim.x) {
        const int c = e / rows, r = e - c * rows;
        px[e] = r < nr ? phx[c * nxh + mx0 + r] : C2<float>{0.f, 0.f};
    }
    for (int e = threadIdx.x; e < n_cols * ny; e += blockDim.x) {
        const float z = Zc[((size_t)b * n_cols + e / ny) * g.Nz + mz];
        const C2<float> p = phy[e];
        qy[e] = {p.x * z, p.y * z};
    }
    __syncthreads();
    C2<float>* out = rho + ((size_t)b * g.Nz + mz) * nxh * ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // register tiles of 4 rows x 2 columns per lane (64-column chunks): per column 4 broadcast
    // loads of px (zero past the block's rows) and 2 loads of qy feed 8 complex multiply-adds
    const int n_rq = (nr + 3) / 4, n_ch = (ny + 63) / 64;
    for (int item = warp; item < n_rq * n_ch; item += nw) {
        const int r = 4 * (item / n_ch), my = (item % n_ch) * 64 + lane;
        const bool c0 = my < ny, c1 = my + 32 < ny;
        C2<float> a[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i][0] = a[i][1] = C2<float>{0.f, 0.f};
        const C2<float>* pr = px + r;
        const C2<float>* qm = qy + my;
#pragma unroll 3
        for (int c = 0; c < n_cols; ++c) {
            const C2<float> q0 = c0 ? qm[c * ny] : C2<float>{0.f, 0.f};
            const C2<float> q1 = c1 ? qm[c * ny + 32] : C2<float>{0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const C2<float> p = pr[c * rows + i];
                a[i][0] = {fmaf(p.x, q0.x, fmaf(-p.y, q0.y, a[i][0].x)), fmaf(p.x, q0.y, fmaf(p.y, q0.x, a[i][0].y))};
                a[i][1] = {fmaf(p.x, q1.x, fmaf(-p.y, q1.y, a[i][1].x)), fmaf(p.x, q1.y, fmaf(p.y, q1.x, a[i][1].y))};
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (r + i >= nr) break;
            C2<float>* o = out + (size_t)(mx0 + r + i) * ny + my;
            if (c0) o[0] = a[i][0];
            if (c1) o[32] = a[i][1];
        }
    }
}

__global__ void f32_twiddle_kernel(float* tw, int N) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double sn, cs;
    sincospi(2.0 * (double)k / (double)N, &sn, &cs);
    tw[2 * k] = (float)cs;
    tw[2 * k + 1] = (float)sn;
}

static size_t deposit_smem(const GridDev& g, int n_cols) {
    return (size_t)n_cols * (deposit_rows(g.Nx) + g.Ny) * sizeof(C2<float>);
}


static bool supported_r(int r) {
    switch (r) {
#define WT_CASE(R) case R:
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
        return true;
        default: return false;
    }
}

void Fast32::init(const GridDev& gd, const std::vector<double>& xy, cudaStream_t s) {
    g = gd;
    n_cols = (int)xy.size() / 2;
    if (g.Nx != g.Ny) fail(WT_ERR_UNSUPPORTED, "the FP32 fast path needs Nx == Ny");
    int w;
    warp_fft_shape(g.Nx, &w, &rxy);
    warp_fft_shape(g.Nz, &w, &rz);
    if (!supported_r(rxy) || !supported_r(rz))
        fail(WT_ERR_UNSUPPORTED, "FFT length not covered by the register FFT (N / W in {1..10, 12, 14, 15, 16, 24})");
    const int nxh = g.Nx / 2 + 1;
    DBuf<double> dxy;
    dxy.upload(xy.data(), xy.size(), s);
    phx.alloc(2 * (size_t)n_cols * nxh);
    phy.alloc(2 * (size_t)n_cols * g.Ny);
    zsh.alloc(2 * (size_t)g.Nz);
    const int n = std::max(n_cols * std::max(nxh, g.Ny), g.Nz);
    f32_tables_kernel<<<(n + 127) / 128, 128, 0, s>>>(dxy.p, n_cols, nxh, g.Ny, g.Nz, g.Lx, g.Ly, phx.p, phy.p,
                                                      zsh.p);
    tw_y.alloc(2 * (size_t)g.Ny);
    tw_x.alloc(2 * (size_t)g.Nx);
    tw_z.alloc(2 * (size_t)g.Nz);
    f32_twiddle_kernel<<<(g.Ny + 127) / 128, 128, 0, s>>>(tw_y.p, g.Ny);
    f32_twiddle_kernel<<<(g.Nx + 127) / 128, 128, 0, s>>>(tw_x.p, g.Nx);
    f32_twiddle_kernel<<<(g.Nz + 127) / 128, 128, 0, s>>>(tw_z.p, g.Nz);
    WT_LAUNCH("fast32 tables");
    const size_t sd = deposit_smem(g, n_cols);
    if (sd > 227 * 1024) fail(WT_ERR_UNSUPPORTED, "too many columns for the FP32 deposit kernel");
    allow_dyn_smem(f32_deposit_kernel, sd);
    set_radix(rxy, rz);
    WT_CUDA(cudaStreamSynchronize(s));
}

std::vector<int> Fast32::radix_options(int N) {
    std::vector<int> out;
    for (int w = 32; w >= 4; w >>= 1)
        if (N % w == 0 && supported_r(N / w)) out.push_back(N / w);
    return out;
}

bool Fast32::z_two_pass_supported(int Nz) { return zpass2_supported(Nz); }
bool Fast32::y_two_pass_supported(int Ny, int r_xy) { return plane_y2_supported(Ny, r_xy); }

void Fast32::set_radix(int r_xy, int r_z, bool z_two_pass, bool y_two_pass, bool x_two_pass) {
    if (g.Nx % r_xy || g.Nz % r_z || !supported_r(r_xy) || !supported_r(r_z))
        fail(WT_ERR_ARG, "register-FFT length does not divide the grid");
    int w = g.Nx / r_xy, wz = g.Nz / r_z;
    if ((w & (w - 1)) || w > 32 || (wz & (wz - 1)) || wz > 32)
        fail(WT_ERR_ARG, "lanes per FFT line must be a power of two up to 32");
    const int ny2 = y_two_pass ? g.Ny : 0;
    if (x_two_pass && !(y_two_pass && g.Nx == g.Ny && plane_y2_supported(g.Ny, 0)))
        fail(WT_ERR_UNSUPPORTED, "two-pass x transforms need the two-pass y transforms and Nx = Ny in {64, 128}");
    if (y_two_pass && !x_two_pass && !plane_y2_supported(g.Ny, r_xy))
        fail(WT_ERR_UNSUPPORTED, "two-pass y transforms need Ny in {64, 128} and 16 or 32 lanes per x line");
    const size_t sp = plane_smem(g, ny2), sz = zpass_smem(g, 64, r_z);
    if (sp > 227 * 1024 || sz > 227 * 1024) fail(WT_ERR_UNSUPPORTED, "grid too large for the FP32 plane kernels");
    plane_allow(x_two_pass ? 0 : r_xy, ny2, sp);
    zpass_allow(r_z, sz);
    if (z_two_pass) zpass2_allow(g.Nz);           // fails for lengths it does not cover
    rxy = r_xy;
    rz = r_z;
    zsm = z_two_pass;
    ysm = y_two_pass;
    xsm = x_two_pass;
}

void Fast32::lateral(const float* Zc, int nb, float* rho, float* R, cudaStream_t s, int mode) const {
    C2<float>* rc = reinterpret_cast<C2<float>*>(rho);
    dim3 gd(g.Nz, nb, F32_DEP_SPLIT);
    f32_deposit_kernel<<<gd, 256, deposit_smem(g, n_cols), s>>>(g, n_cols, reinterpret_cast<const C2<float>*>(phx.p),
                                                                reinterpret_cast<const C2<float>*>(phy.p), Zc, rc);
    WT_LAUNCH("f32_deposit");
    dim3 gp(g.Nz, 3, nb);
    const C2<float>* ty = reinterpret_cast<const C2<float>*>(tw_y.p);
    const C2<float>* tx = reinterpret_cast<const C2<float>*>(tw_x.p);
    plane_launch(xsm ? 0 : rxy, xdirect, ysm ? g.Ny : 0, gp, s, g, rc, ty, tx, R, mode);
}

void Fast32::zlines(const float* R, int nb, int y0, int ys, float* out, size_t out_sb, size_t out_sc, cudaStream_t s,
                    int lb, bool discard) const {
    if (lb != 16 && lb != 32 && lb != 64) fail(WT_ERR_ARG, "z-pass lines per block must be 16, 32 or 64");
    if (y0 < 0 || ys < 1 || y0 + ys > g.Ny) fail(WT_ERR_ARG, "z-pass rows out of range");
    const size_t nl = (size_t)g.Nx * ys;
    dim3 gz((unsigned)((nl + lb - 1) / lb), 3, nb);
    const C2<float>* tz = reinterpret_cast<const C2<float>*>(tw_z.p);
    const C2<float>* zz = reinterpret_cast<const C2<float>*>(zsh.p);
    const bool disc = discard && zsm && lb >= 32 && nl % 32 == 0 && reinterpret_cast<uintptr_t>(R) % 128 == 0;
    const ZLines zl{ys, y0, disc ? 1 : 0};
    if (zsm) zpass2_launch(lb, gz, s, g, R, tz, zz, out, out_sb, out_sc, zl);
    else zpass_launch(rz, lb, gz, s, g, R, tz, zz, out, out_sb, out_sc, zl);
}

void Fast32::fields(const float* Zc, int nb, float* rho, float* R, float* out, size_t out_sb, size_t out_sc,
                    cudaStream_t s, int mode, int lb) const {
    lateral(Zc, nb, rho, R, s, mode);
    zlines(R, nb, 0, g.Ny, out, out_sb, out_sc, s, lb);
}

}  // namespace wt
