// Pseudo-spectral bulk extension (Abstract; Sec. 1 discrete Fourier
// transforms; Sec. 3 spectra divided by |k|^2): for a charge vector on the
// column axes,
//   rho^(k)   = sum_c exp(-i k_perp . x_c) Zc(k_z),  Zc = sum_j q_j 2 cos(k_z z_j)
//   W_x, W_y  = pref sum_k (-i k_a) rho^ / |k|^2 w(m_z) cos(k_z z) exp(i k_perp . x)
//   W_z       = pref sum_k rho^ 2 k_z / |k|^2 sin(k_z z) exp(i k_perp . x)
// (w = 1 for m_z = 0, 2 otherwise; the +-k_z pairs of the mirrored box).
// Three passes over a half-spectrum array G[b][c][mx][my][z] (mx = 0..Nx/2):
//   Z: deposit + |k|^2 division + (-ik) + z cosine/sine series, done as one
//      length-2Nz complex FFT per line in shared memory;
//   Y: inverse complex FFT along y;
//   X: half-spectrum -> real inverse FFT along x, written to the output layout.
// FFTs are Stockham autosort, mixed radix (4, 2, 3, 5, 7), in shared memory.
#include "k_fft.cuh"
#include "fft_core.cuh"

#include <cmath>

namespace wt {

FftPlan make_plan(int N) {
    FftPlan p{};
    p.N = N;
    int n = N;
    const int rad[5] = {4, 2, 3, 5, 7};
    for (int k = 0; k < 5; ++k) {
        while (n % rad[k] == 0) {
            if (p.ns >= 16) fail(WT_ERR_UNSUPPORTED, "FFT length has too many factors");
            p.r[p.ns++] = rad[k];
            n /= rad[k];
        }
    }
    if (n != 1) fail(WT_ERR_UNSUPPORTED, "FFT length " + std::to_string(N) + " has a prime factor above 7");
    return p;
}

template <class T>
__global__ void twiddle_kernel(T* tw, int N) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double sn, cs;
    sincospi(2.0 * (double)k / (double)N, &sn, &cs);
    tw[2 * k] = (T)cs;
    tw[2 * k + 1] = (T)sn;
}

// ------------------------------------------------------------------ pass Z
template <class T>
__global__ void pass_z_kernel(GridDev g, int n_cols, const double* __restrict__ col_xy, const T* __restrict__ Zc,
                              C2<T>* __restrict__ G, FftPlan pl, const C2<T>* __restrict__ tw) {
    extern __shared__ unsigned char smem_raw[];
    const int nz = g.Nz, n2 = 2 * g.Nz;
    const int nxh = g.Nx / 2 + 1;
    C2<T>* buf = reinterpret_cast<C2<T>*>(smem_raw);          // 3 lines of n2
    C2<T>* scr = buf + 3 * n2;
    C2<T>* ph = scr + 3 * n2;                                 // n_cols phases
    const int line = blockIdx.x;                              // mx * Ny + my
    const int b = blockIdx.y;
    const int mx = line / g.Ny, my = line % g.Ny;
    const int mys = my < g.Ny / 2 ? my : my - g.Ny;
    const bool zero_line = (mx == g.Nx / 2) || (my == g.Ny / 2);
    for (int c = threadIdx.x; c < n_cols; c += blockDim.x) {
        double sn, cs;
        // exp(-i (kx x_c + ky y_c)), kx x_c = 2 pi mx x_c / Lx
        sincospi(-2.0 * (mx * col_xy[2 * c] / g.Lx + mys * col_xy[2 * c + 1] / g.Ly), &sn, &cs);
        ph[c] = {(T)cs, (T)sn};
    }
    __syncthreads();
    const double kx = 2.0 * kPi * mx / g.Lx, ky = 2.0 * kPi * mys / g.Ly;
    const T* zc = Zc + (size_t)b * n_cols * nz;
    for (int m = threadIdx.x; m < nz; m += blockDim.x) {
        C2<T> rho = {(T)0, (T)0};
        if (!zero_line)
            for (int c = 0; c < n_cols; ++c) {
                const T z = zc[(size_t)c * nz + m];
                rho.x += ph[c].x * z;
                rho.y += ph[c].y * z;
            }
        const double kz = kPi * m / g.Lz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double gk = (k2 > 0.0 && !zero_line) ? g.pref / k2 : 0.0;
        // shift factor exp(+i pi m / (2 Nz)) of the half-sample grid offset
        double sn, cs;
        sincospi((double)m / (double)n2, &sn, &cs);
        const C2<T> e = {(T)cs, (T)sn};
        const C2<T> ec = {(T)cs, (T)(-sn)};
        // W_x, W_y coefficients: -i k_a rho^ gk w; W_z: rho^ 2 kz gk
        const T wx = (T)(kx * gk), wy = (T)(ky * gk), wz = (T)(2.0 * kz * gk);
        const C2<T> cx = {rho.y * wx, -rho.x * wx};       // -i * rho * (kx gk)
        const C2<T> cy = {rho.y * wy, -rho.x * wy};
        const C2<T> cz = {rho.x * wz, rho.y * wz};
        if (m == 0) {
            buf[0] = cx;   // cosine series: d_0 = C(0)
            buf[n2] = cy;
            buf[2 * n2] = {(T)0, (T)0};
            buf[nz] = {(T)0, (T)0};
            buf[n2 + nz] = {(T)0, (T)0};
            buf[2 * n2 + nz] = {(T)0, (T)0};
        } else {
            // cosine (w = 2): d_m = C e, d_{2N-m} = C ec  (the 1/2 cancels w)
            buf[m] = cmul(cx, e);
            buf[n2 - m] = cmul(cx, ec);
            buf[n2 + m] = cmul(cy, e);
            buf[n2 + n2 - m] = cmul(cy, ec);
            // sine: d_m = C e / (2i), d_{2N-m} = -C ec / (2i)
            const C2<T> t1 = cmul(cz, e), t2 = cmul(cz, ec);
            buf[2 * n2 + m] = {t1.y * (T)0.5, -t1.x * (T)0.5};
            buf[2 * n2 + n2 - m] = {-t2.y * (T)0.5, t2.x * (T)0.5};
        }
    }
    __syncthreads();
    C2<T>* res = fft_lines<T>(buf, scr, n2, 3, pl, tw);
    const size_t plane = (size_t)nxh * g.Ny * nz;
    for (int e = threadIdx.x; e < 3 * nz; e += blockDim.x) {
        const int c = e / nz, z = e % nz;
        G[((size_t)b * 3 + c) * plane + (size_t)line * nz + z] = res[c * n2 + z];
    }
}

// ------------------------------------------------------------------ pass Y
constexpr int ZC = 16;   // z values per block in the lateral passes

template <class T>
__global__ void pass_y_kernel(GridDev g, C2<T>* __restrict__ G, FftPlan pl, const C2<T>* __restrict__ tw) {
    extern __shared__ unsigned char smem_raw[];
    const int ny = g.Ny, nz = g.Nz, ld = ny + 1;
    C2<T>* buf = reinterpret_cast<C2<T>*>(smem_raw);
    C2<T>* scr = buf + ZC * ld;
    const int z0 = blockIdx.x * ZC;
    const int mx = blockIdx.y;
    const int bc = blockIdx.z;                     // b * 3 + c
    const int nxh = g.Nx / 2 + 1;
    const int nzc = min(ZC, nz - z0);
    C2<T>* base = G + ((size_t)bc * nxh + mx) * ny * nz + z0;
    for (int e = threadIdx.x; e < ny * ZC; e += blockDim.x) {
        const int my = e / ZC, l = e % ZC;
        if (l < nzc) buf[l * ld + my] = base[(size_t)my * nz + l];
        else buf[l * ld + my] = {(T)0, (T)0};
    }
    __syncthreads();
    C2<T>* res = fft_lines<T>(buf, scr, ld, ZC, pl, tw);
    for (int e = threadIdx.x; e < ny * ZC; e += blockDim.x) {
        const int y = e / ZC, l = e % ZC;
        if (l < nzc) base[(size_t)y * nz + l] = res[l * ld + y];
    }
}

// ------------------------------------------------------------------ pass X
template <class T, class OutT>
__global__ void pass_x_kernel(GridDev g, const C2<T>* __restrict__ G, FftPlan pl, const C2<T>* __restrict__ tw,
                              OutT* __restrict__ out, size_t out_sb, size_t out_sc) {
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.Nx, ny = g.Ny, nz = g.Nz, ld = nx + 1;
    const int nxh = nx / 2 + 1;
    C2<T>* buf = reinterpret_cast<C2<T>*>(smem_raw);
    C2<T>* scr = buf + ZC * ld;
    const int z0 = blockIdx.x * ZC;
    const int y = blockIdx.y;
    const int bc = blockIdx.z;
    const int b = bc / 3, c = bc % 3;
    const int nzc = min(ZC, nz - z0);
    const C2<T>* base = G + (size_t)bc * nxh * ny * nz + (size_t)y * nz + z0;
    for (int e = threadIdx.x; e < nx * ZC; e += blockDim.x) {
        const int mx = e / ZC, l = e % ZC;
        C2<T> v = {(T)0, (T)0};
        if (l < nzc && mx < nx / 2) {
            v = base[(size_t)mx * ny * nz + l];
            if (mx > 0) { v.x *= (T)2; v.y *= (T)2; }
        }
        buf[l * ld + mx] = v;
    }
    __syncthreads();
    C2<T>* res = fft_lines<T>(buf, scr, ld, ZC, pl, tw);
    OutT* o = out + (size_t)b * out_sb + (size_t)c * out_sc + (size_t)y * nz + z0;
    for (int e = threadIdx.x; e < nx * ZC; e += blockDim.x) {
        const int x = e / ZC, l = e % ZC;
        if (l < nzc) o[(size_t)x * ny * nz + l] = (OutT)res[l * ld + x].x;
    }
}

// --------------------------------------------------- column z-transforms
__global__ void column_cos_kernel(const double* __restrict__ zsrc, int n_src, int Nz, double Lz,
                                  double* __restrict__ zcos) {
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_src * Nz) return;
    const int j = idx / Nz, m = idx % Nz;
    zcos[idx] = 2.0 * cospi((double)m * zsrc[j] / Lz);
}
void column_cos_table(cudaStream_t s, const double* zsrc, int n_src, int Nz, double Lz, double* zcos) {
    const size_t tot = (size_t)n_src * Nz;
    column_cos_kernel<<<(tot + 255) / 256, 256, 0, s>>>(zsrc, n_src, Nz, Lz, zcos);
    WT_LAUNCH("column_cos_table");
}

template <class T>
__global__ void column_z_kernel(const double* __restrict__ q, int ldq, const double* __restrict__ zcos,
                                const int* __restrict__ col_off, int n_cols, int Nz, T* __restrict__ Zc) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y, b = blockIdx.z;
    if (m >= Nz) return;
    double acc = 0.0;
    const double* qb = q + (size_t)b * ldq;
    for (int j = col_off[c]; j < col_off[c + 1]; ++j) acc = fma(qb[j], zcos[(size_t)j * Nz + m], acc);
    Zc[((size_t)b * n_cols + c) * Nz + m] = (T)acc;
}

template <class T>
void column_ztransform(cudaStream_t s, const double* q, int nb, int n_src, int ldq, const double* zcos,
                       const int* col_off, int n_cols, int Nz, T* Zc) {
    (void)n_src;
    dim3 grid((Nz + 127) / 128, n_cols, nb);
    column_z_kernel<T><<<grid, 128, 0, s>>>(q, ldq, zcos, col_off, n_cols, Nz, Zc);
    WT_LAUNCH("column_ztransform");
}

template <class T>
void Spectral<T>::init(const GridDev& gd, const std::vector<double>& xy, cudaStream_t s) {
    g = gd;
    n_cols = (int)xy.size() / 2;
    pz = make_plan(2 * g.Nz);
    py = make_plan(g.Ny);
    px = make_plan(g.Nx);
    col_xy.upload(xy.data(), xy.size(), s);
    tw_z.alloc(2 * (size_t)pz.N);
    tw_y.alloc(2 * (size_t)py.N);
    tw_x.alloc(2 * (size_t)px.N);
    twiddle_kernel<T><<<(pz.N + 127) / 128, 128, 0, s>>>(tw_z.p, pz.N);
    twiddle_kernel<T><<<(py.N + 127) / 128, 128, 0, s>>>(tw_y.p, py.N);
    twiddle_kernel<T><<<(px.N + 127) / 128, 128, 0, s>>>(tw_x.p, px.N);
    WT_LAUNCH("twiddles");
    size_t smz = (size_t)(6 * 2 * g.Nz) * sizeof(C2<T>) + (size_t)n_cols * sizeof(C2<T>);
    size_t smy = (size_t)2 * ZC * (g.Ny + 1) * sizeof(C2<T>);
    size_t smx = (size_t)2 * ZC * (g.Nx + 1) * sizeof(C2<T>);
    allow_dyn_smem(pass_z_kernel<T>, smz);
    allow_dyn_smem(pass_y_kernel<T>, smy);
    allow_dyn_smem(pass_x_kernel<T, T>, smx);
}

template <class T>
void Spectral<T>::fields(const T* Zc, int nb, T* G, T* out, size_t out_sb, size_t out_sc, cudaStream_t s) const {
    const int nxh = g.Nx / 2 + 1;
    C2<T>* Gc = reinterpret_cast<C2<T>*>(G);
    size_t smz = (size_t)(6 * 2 * g.Nz) * sizeof(C2<T>) + (size_t)n_cols * sizeof(C2<T>);
    size_t smy = (size_t)2 * ZC * (g.Ny + 1) * sizeof(C2<T>);
    size_t smx = (size_t)2 * ZC * (g.Nx + 1) * sizeof(C2<T>);
    dim3 gz(nxh * g.Ny, nb);
    pass_z_kernel<T><<<gz, 256, smz, s>>>(g, n_cols, col_xy.p, Zc, Gc, pz, reinterpret_cast<const C2<T>*>(tw_z.p));
    WT_LAUNCH("pass_z");
    dim3 gy((g.Nz + ZC - 1) / ZC, nxh, nb * 3);
    pass_y_kernel<T><<<gy, 256, smy, s>>>(g, Gc, py, reinterpret_cast<const C2<T>*>(tw_y.p));
    WT_LAUNCH("pass_y");
    dim3 gx((g.Nz + ZC - 1) / ZC, g.Ny, nb * 3);
    pass_x_kernel<T, T><<<gx, 256, smx, s>>>(g, Gc, px, reinterpret_cast<const C2<T>*>(tw_x.p), out, out_sb, out_sc);
    WT_LAUNCH("pass_x");
}

template struct Spectral<float>;
template struct Spectral<double>;
template void column_ztransform<float>(cudaStream_t, const double*, int, int, int, const double*, const int*, int,
                                       int, float*);
template void column_ztransform<double>(cudaStream_t, const double*, int, int, int, const double*, const int*, int,
                                        int, double*);

}  // namespace wt
