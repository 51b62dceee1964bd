// FP32 basis fields of the bulk extension (Abstract; Sec. 1 discrete Fourier
// transforms; Sec. 3 |k|^2 spectral division), three kernels per batch of
// charge vectors, all FP32 (the phases come from FP64-built tables):
//   deposit: rho^[b][mz][mx][my] = sum_c e^{-i kx x_c} e^{-i ky y_c} Zc[b][c][mz]
//   plane:   for one (b, component, mz): multiply by the component's factor
//            (-i k_a w / |k|^2, or 2 kz / |k|^2 for W_z), inverse FFT along y,
//            half-spectrum -> real inverse FFT along x; R[b][c][mz][x][y]
//   zpass:   cosine (W_x, W_y) or sine (W_z) series along z, two real lines
//            packed in one length-2Nz complex FFT; out[b][c][x][y][z].
#include "k_fft.cuh"
#include "fft_core.cuh"

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

// rho^ planes; grid (Nz, nb), threads over (mx, my)
__global__ void f32_deposit_kernel(GridDev g, int n_cols, const C2<float>* __restrict__ phx,
                                   const C2<float>* __restrict__ phy, const float* __restrict__ Zc,
                                   C2<float>* __restrict__ rho) {
    extern __shared__ float zc_s[];
    const int mz = blockIdx.x, b = blockIdx.y;
    const int nxh = g.Nx / 2 + 1;
    for (int c = threadIdx.x; c < n_cols; c += blockDim.x) zc_s[c] = Zc[((size_t)b * n_cols + c) * g.Nz + mz];
    __syncthreads();
    C2<float>* out = rho + ((size_t)b * g.Nz + mz) * nxh * g.Ny;
    for (int e = threadIdx.x; e < nxh * g.Ny; e += blockDim.x) {
        const int mx = e / g.Ny, my = e % g.Ny;
        C2<float> acc = {0.f, 0.f};
        for (int c = 0; c < n_cols; ++c) {
            const C2<float> p = cmul(phx[c * nxh + mx], phy[c * g.Ny + my]);
            acc.x = fmaf(p.x, zc_s[c], acc.x);
            acc.y = fmaf(p.y, zc_s[c], acc.y);
        }
        out[e] = acc;
    }
}

constexpr int F32_NL = 16;   // lines per FFT batch in the plane kernel

// grid (Nz, 3, nb)
__global__ void __launch_bounds__(256) f32_plane_kernel(GridDev g, const C2<float>* __restrict__ rho, FftPlan py,
                                                        FftPlan px, const C2<float>* __restrict__ twy,
                                                        const C2<float>* __restrict__ twx, float* __restrict__ R) {
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.Nx, ny = g.Ny, nz = g.Nz, nxh = nx / 2 + 1;
    const int mz = blockIdx.x, comp = blockIdx.y, b = blockIdx.z;
    const int ldp = ny + 1;
    const int nmax = nx > ny ? nx : ny;
    C2<float>* P = reinterpret_cast<C2<float>*>(smem_raw);            // [nxh][ldp]
    C2<float>* A = P + (size_t)nxh * ldp;                             // [F32_NL][nmax]
    C2<float>* B = A + (size_t)F32_NL * nmax;
    float* Rout = R + (((size_t)b * 3 + comp) * nz + mz) * nx * ny;
    if (comp == 2 && mz == 0) {       // the sine series has no k_z = 0 term
        for (int e = threadIdx.x; e < nx * ny; e += blockDim.x) Rout[e] = 0.f;
        return;
    }
    const float kz = (float)(kPi * mz / g.Lz);
    const float ckx = (float)(2.0 * kPi / g.Lx), cky = (float)(2.0 * kPi / g.Ly);
    const float pref = (float)g.pref;
    const C2<float>* rp = rho + ((size_t)b * nz + mz) * nxh * ny;
    for (int e = threadIdx.x; e < nxh * ny; e += blockDim.x) {
        const int mx = e / ny, my = e % ny;
        const int mys = my < ny / 2 ? my : my - ny;
        C2<float> v = {0.f, 0.f};
        if (mx != nx / 2 && my != ny / 2) {
            const float kx = ckx * mx, ky = cky * mys;
            const float k2 = kx * kx + ky * ky + kz * kz;
            if (k2 > 0.f) {
                const C2<float> r = rp[e];
                const float gk = pref / k2 * (mx ? 2.f : 1.f);     // x half-spectrum fold
                // cosine components carry no w(m_z) here: the z pass builds
                // d_m = C e, d_{2N-m} = C e*, which already sums the +-k_z pair
                if (comp == 0) { const float f = kx * gk; v = {r.y * f, -r.x * f}; }
                else if (comp == 1) { const float f = ky * gk; v = {r.y * f, -r.x * f}; }
                else { const float f = 2.f * kz * gk; v = {r.x * f, r.y * f}; }
            }
        }
        P[mx * ldp + my] = v;
    }
    __syncthreads();
    // inverse FFT along y for every mx row
    for (int r0 = 0; r0 < nxh; r0 += F32_NL) {
        const int nl = min(F32_NL, nxh - r0);
        for (int e = threadIdx.x; e < nl * ny; e += blockDim.x) A[(e / ny) * nmax + e % ny] = P[(r0 + e / ny) * ldp + e % ny];
        __syncthreads();
        C2<float>* res = fft_lines<float>(A, B, nmax, nl, py, twy);
        for (int e = threadIdx.x; e < nl * ny; e += blockDim.x) P[(r0 + e / ny) * ldp + e % ny] = res[(e / ny) * nmax + e % ny];
        __syncthreads();
    }
    // half spectrum along x -> real, F32_NL consecutive y at a time
    for (int y0 = 0; y0 < ny; y0 += F32_NL) {
        const int nl = min(F32_NL, ny - y0);
        for (int e = threadIdx.x; e < nl * nx; e += blockDim.x) {
            const int l = e / nx, mx = e % nx;
            A[l * nmax + mx] = mx < nx / 2 ? P[mx * ldp + y0 + l] : C2<float>{0.f, 0.f};
        }
        __syncthreads();
        C2<float>* res = fft_lines<float>(A, B, nmax, nl, px, twx);
        for (int e = threadIdx.x; e < nl * nx; e += blockDim.x) {
            const int x = e / nl, l = e % nl;
            Rout[(size_t)x * ny + y0 + l] = res[l * nmax + x].x;
        }
        __syncthreads();
    }
}

constexpr int F32_LB = 16;   // (x, y) lines per z-pass block

// grid (Nx*Ny / F32_LB, 3, nb)
__global__ void __launch_bounds__(256) f32_zpass_kernel(GridDev g, const float* __restrict__ R, FftPlan pz,
                                                        const C2<float>* __restrict__ twz,
                                                        const C2<float>* __restrict__ zsh, float* __restrict__ out,
                                                        size_t out_sb, size_t out_sc) {
    extern __shared__ unsigned char smem_raw[];
    const int nz = g.Nz, n2 = 2 * nz;
    const size_t nxy = (size_t)g.Nx * g.Ny;
    const int comp = blockIdx.y, b = blockIdx.z;
    const size_t L0 = (size_t)blockIdx.x * F32_LB;
    float* in = reinterpret_cast<float*>(smem_raw);                      // [nz][F32_LB]
    C2<float>* A = reinterpret_cast<C2<float>*>(in + (size_t)nz * F32_LB);   // [F32_LB/2][n2]
    C2<float>* Bf = A + (size_t)(F32_LB / 2) * n2;
    const float* src = R + ((size_t)b * 3 + comp) * nz * nxy + L0;
    for (int e = threadIdx.x; e < nz * F32_LB; e += blockDim.x) {
        const int m = e / F32_LB, l = e % F32_LB;
        in[e] = (L0 + l < nxy) ? src[(size_t)m * nxy + l] : 0.f;
    }
    __syncthreads();
    // pack lines (2p, 2p+1) as real and imaginary parts; build the length-2Nz sequence
    for (int e = threadIdx.x; e < (F32_LB / 2) * nz; e += blockDim.x) {
        const int p = e / nz, m = e % nz;
        C2<float>* d = A + (size_t)p * n2;
        const C2<float> c = {in[m * F32_LB + 2 * p], in[m * F32_LB + 2 * p + 1]};
        const C2<float> ez = zsh[m];
        const C2<float> ezc = {ez.x, -ez.y};
        if (comp < 2) {            // cosine series
            if (m == 0) { d[0] = c; d[nz] = {0.f, 0.f}; }
            else { d[m] = cmul(c, ez); d[n2 - m] = cmul(c, ezc); }
        } else {                   // sine series: d_m = C e/(2i), d_{2N-m} = -C ec/(2i)
            if (m == 0) { d[0] = {0.f, 0.f}; d[nz] = {0.f, 0.f}; }
            else {
                const C2<float> t1 = cmul(c, ez), t2 = cmul(c, ezc);
                d[m] = {0.5f * t1.y, -0.5f * t1.x};
                d[n2 - m] = {-0.5f * t2.y, 0.5f * t2.x};
            }
        }
    }
    __syncthreads();
    C2<float>* res = fft_lines<float>(A, Bf, n2, F32_LB / 2, pz, twz);
    float* o = out + (size_t)b * out_sb + (size_t)comp * out_sc + L0 * nz;
    for (int e = threadIdx.x; e < F32_LB * nz; e += blockDim.x) {
        const int l = e / nz, z = e % nz;
        if (L0 + l < nxy) {
            const C2<float> v = res[(size_t)(l >> 1) * n2 + z];
            o[(size_t)l * nz + z] = (l & 1) ? v.y : v.x;
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

static size_t plane_smem(const GridDev& g) {
    const int nxh = g.Nx / 2 + 1, nmax = g.Nx > g.Ny ? g.Nx : g.Ny;
    return ((size_t)nxh * (g.Ny + 1) + 2 * (size_t)F32_NL * nmax) * sizeof(C2<float>);
}
static size_t zpass_smem(const GridDev& g) {
    return (size_t)g.Nz * F32_LB * sizeof(float) + 2 * (size_t)(F32_LB / 2) * 2 * g.Nz * sizeof(C2<float>);
}

void Fast32::init(const GridDev& gd, const std::vector<double>& xy, cudaStream_t s) {
    g = gd;
    n_cols = (int)xy.size() / 2;
    py = make_plan(g.Ny);
    px = make_plan(g.Nx);
    pz = make_plan(2 * g.Nz);
    const int nxh = g.Nx / 2 + 1;
    DBuf<double> dxy;
    dxy.upload(xy.data(), xy.size(), s);
    phx.alloc(2 * (size_t)n_cols * nxh);
    phy.alloc(2 * (size_t)n_cols * g.Ny);
    zsh.alloc(2 * (size_t)g.Nz);
    const int n = std::max(n_cols * std::max(nxh, g.Ny), g.Nz);
    f32_tables_kernel<<<(n + 127) / 128, 128, 0, s>>>(dxy.p, n_cols, nxh, g.Ny, g.Nz, g.Lx, g.Ly, phx.p, phy.p,
                                                      zsh.p);
    tw_y.alloc(2 * (size_t)py.N);
    tw_x.alloc(2 * (size_t)px.N);
    tw_z.alloc(2 * (size_t)pz.N);
    f32_twiddle_kernel<<<(py.N + 127) / 128, 128, 0, s>>>(tw_y.p, py.N);
    f32_twiddle_kernel<<<(px.N + 127) / 128, 128, 0, s>>>(tw_x.p, px.N);
    f32_twiddle_kernel<<<(pz.N + 127) / 128, 128, 0, s>>>(tw_z.p, pz.N);
    WT_LAUNCH("fast32 tables");
    const size_t sp = plane_smem(g), sz = zpass_smem(g);
    if (sp > 227 * 1024 || sz > 227 * 1024) fail(WT_ERR_UNSUPPORTED, "grid too large for the FP32 plane kernels");
    WT_CUDA(cudaFuncSetAttribute(f32_plane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp));
    WT_CUDA(cudaFuncSetAttribute(f32_zpass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz));
    WT_CUDA(cudaStreamSynchronize(s));
}

void Fast32::fields(const float* Zc, int nb, float* rho, float* R, float* out, size_t out_sb, size_t out_sc,
                    cudaStream_t s) const {
    C2<float>* rc = reinterpret_cast<C2<float>*>(rho);
    dim3 gd(g.Nz, nb);
    f32_deposit_kernel<<<gd, 256, n_cols * sizeof(float), s>>>(g, n_cols, reinterpret_cast<const C2<float>*>(phx.p),
                                                               reinterpret_cast<const C2<float>*>(phy.p), Zc, rc);
    WT_LAUNCH("f32_deposit");
    dim3 gp(g.Nz, 3, nb);
    f32_plane_kernel<<<gp, 256, plane_smem(g), s>>>(g, rc, py, px, reinterpret_cast<const C2<float>*>(tw_y.p),
                                                    reinterpret_cast<const C2<float>*>(tw_x.p), R);
    WT_LAUNCH("f32_plane");
    const size_t nxy = (size_t)g.Nx * g.Ny;
    dim3 gz((unsigned)((nxy + F32_LB - 1) / F32_LB), 3, nb);
    f32_zpass_kernel<<<gz, 256, zpass_smem(g), s>>>(g, R, pz, reinterpret_cast<const C2<float>*>(tw_z.p),
                                                    reinterpret_cast<const C2<float>*>(zsh.p), out, out_sb, out_sc);
    WT_LAUNCH("f32_zpass");
}

}  // namespace wt
