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
#include "warp_fft.cuh"

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
// m_x rows of one plane (warps over rows, lanes over m_y).  Shared tables:
// px[c][mx] = e^{-i kx x_c} (the block's rows), qy[c][my] = e^{-i ky y_c} Zc[b][c][mz].
constexpr int F32_DEP_SPLIT = 4;
__global__ void f32_deposit_kernel(GridDev g, int n_cols, const C2<float>* __restrict__ phx,
                                   const C2<float>* __restrict__ phy, const float* __restrict__ Zc,
                                   C2<float>* __restrict__ rho) {
    extern __shared__ unsigned char smem_raw[];
    const int mz = blockIdx.x, b = blockIdx.y;
    const int nxh = g.Nx / 2 + 1, ny = g.Ny;
    const int rows = (nxh + F32_DEP_SPLIT - 1) / F32_DEP_SPLIT;
    const int mx0 = blockIdx.z * rows, mx1 = min(nxh, mx0 + rows);
    if (mx0 >= mx1) return;
    const int nr = mx1 - mx0;
    C2<float>* px = reinterpret_cast<C2<float>*>(smem_raw);        // [n_cols][rows]
    C2<float>* qy = px + (size_t)n_cols * rows;                      // [n_cols][ny]
    for (int e = threadIdx.x; e < n_cols * nr; e += blockDim.x) {
        const int c = e / nr, r = e - c * nr;
        px[c * rows + r] = phx[c * nxh + mx0 + r];
    }
    for (int e = threadIdx.x; e < n_cols * ny; e += blockDim.x) {
        const float z = Zc[((size_t)b * n_cols + e / ny) * g.Nz + mz];
        const C2<float> p = phy[e];
        qy[e] = {p.x * z, p.y * z};
    }
    __syncthreads();
    C2<float>* out = rho + ((size_t)b * g.Nz + mz) * nxh * ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < nr; r += nw)
        for (int my = lane; my < ny; my += 32) {
            C2<float> acc = {0.f, 0.f};
            for (int c = 0; c < n_cols; ++c) {
                const C2<float> a = px[c * rows + r], q = qy[c * ny + my];
                acc.x = fmaf(a.x, q.x, fmaf(-a.y, q.y, acc.x));
                acc.y = fmaf(a.x, q.y, fmaf(a.y, q.x, acc.y));
            }
            out[(size_t)(mx0 + r) * ny + my] = acc;
        }
}

// One (k_z plane, component, charge vector) per block: component factor,
// inverse FFT along y for every m_x row, then half spectrum -> real along x.
// Warp FFTs in registers; the plane stays in shared memory.
// Output R[b][c][mz][y][x].  grid (Nz, 3, nb).
// mode 0: the field; mode 1: its derivative with respect to the lateral scale
// lambda (Lx, Ly, column and grid positions scale together): the multiplier
// times (-3 + 2 k_perp^2/|k|^2) for W_x, W_y and (-2 + 2 k_perp^2/|k|^2) for W_z.
template <int RY, int RX>
__global__ void __launch_bounds__(256, RX <= 5 ? 3 : 2) f32_plane_kernel(GridDev g, const C2<float>* __restrict__ rho,
                                                        const C2<float>* __restrict__ twy,
                                                        const C2<float>* __restrict__ twx, float* __restrict__ R,
                                                        int mode) {
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.Nx, ny = g.Ny, nz = g.Nz, nxh = nx / 2 + 1;
    const int mz = blockIdx.x, comp = blockIdx.y, b = blockIdx.z;
    const int ldp = (ny + 1) | 1;                              // odd pitch: conflict-free column reads
    C2<float>* P = reinterpret_cast<C2<float>*>(smem_raw);     // [nxh][ldp]
    C2<float>* ty = P + (size_t)nxh * ldp;                     // [ny]
    C2<float>* tx = ty + ny;                                   // [nx]
    float* Rout = R + (((size_t)b * 3 + comp) * nz + mz) * nx * ny;
    if (comp == 2 && mz == 0) {       // the sine series has no k_z = 0 term
        for (int e = threadIdx.x; e < nx * ny; e += blockDim.x) Rout[e] = 0.f;
        return;
    }
    for (int e = threadIdx.x; e < ny; e += blockDim.x) ty[e] = twy[e];
    for (int e = threadIdx.x; e < nx; e += blockDim.x) tx[e] = twx[e];
    const float kz = (float)(kPi * mz / g.Lz);
    const float ckx = (float)(2.0 * kPi / g.Lx), cky = (float)(2.0 * kPi / g.Ly);
    const float pref = (float)g.pref;
    const C2<float>* rp = rho + ((size_t)b * nz + mz) * nxh * ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warps over m_x rows, lanes over m_y (no index division); FP32 fast division: the path's
    // tolerance is far above its 2-ulp error
    for (int mx = warp; mx < nxh; mx += 8) {
        const float kx = ckx * mx;
        const float fold = mx ? 2.f : 1.f;                        // x half-spectrum fold
        const C2<float>* rrow = rp + (size_t)mx * ny;
        C2<float>* prow = P + (size_t)mx * ldp;
#pragma unroll 4
        for (int my = lane; my < ny; my += 32) {
            const int mys = my < ny / 2 ? my : my - ny;
            C2<float> v = {0.f, 0.f};
            if (mx != nx / 2 && my != ny / 2) {
                const float ky = cky * mys;
                const float kp2 = kx * kx + ky * ky;
                const float k2 = kp2 + kz * kz;
                if (k2 > 0.f) {
                    const C2<float> r = rrow[my];
                    float gk = __fdividef(pref * fold, k2);
                    if (mode == 1) gk *= (comp < 2 ? -3.f : -2.f) + __fdividef(2.f * kp2, k2);
                    // the z pass's cosine series carries the factor 2 of the +-k_z pair itself
                    if (comp == 0) { const float f = kx * gk; v = {r.y * f, -r.x * f}; }
                    else if (comp == 1) { const float f = ky * gk; v = {r.y * f, -r.x * f}; }
                    else { const float f = 2.f * kz * gk; v = {r.x * f, r.y * f}; }
                }
            }
            prow[my] = v;
        }
    }
    __syncthreads();
    const int Wy = ny / RY;
    {   // y: nxh lines of length ny (decimation in time: lanes read consecutive elements).  Lane gl
        // ends with Y[k + RY bitrev(gl)] and writes it back at row position gl + Wy k (consecutive
        // lanes, no bank conflicts): Y[y] sits at column sigma(y) = bitrev(y / RY) + Wy (y % RY).
        const int W = Wy, G = 32 / W, grp = lane / W, gl = lane % W;
        LaneTw<RY> lt;
        lane_twiddles<RY>(ty, gl, W, true, lt);
        for (int base = warp * G; base < nxh; base += 8 * G) {
            const int mx = base + grp;
            const bool act = mx < nxh;
            C2<float> v[RY];
#pragma unroll
            for (int j = 0; j < RY; ++j) v[j] = act ? P[mx * ldp + gl + W * j] : C2<float>{0.f, 0.f};
            warp_fft_dit_t<RY>(v, gl, W, lt, ty);
            if (act)
#pragma unroll
                for (int k = 0; k < RY; ++k) P[mx * ldp + gl + W * k] = v[k];
        }
    }
    __syncthreads();
    {   // x: ny real lines of length nx from the half spectrum, two lines (y = 2p, 2p + 1) per
        // complex FFT: Z[m] = A'[m] + i B'[m] with the Hermitian completions A'[0] = Re a[0],
        // A'[m] = a[m] / 2, A'[nx - m] = conj(a[m]) / 2 (0 < m < nx/2; a carries the x fold
        // factor 2), A'[nx/2] = 0, so that FFT(Z) = out_a + i out_b.  Decimation in time reads
        // consecutive rows per lane; the two output lines are staged in the pair's own columns
        // of P for coalesced stores.
        const int W = nx / RX, G = 32 / W, grp = lane / W, gl = lane % W;
        const int k2 = warp_fft_k2(gl, W);
        const int nxq = nx / 2;
        LaneTw<RX> lt;
        lane_twiddles<RX>(tx, gl, W, true, lt);
        for (int base = warp * G; base < ny / 2; base += 8 * G) {
            const int pp = base + grp;
            const bool act = pp < ny / 2;
            const int ya = 2 * pp, yb = ya + 1;
            const int ca = warp_fft_k2(ya / RY, Wy) + Wy * (ya % RY);     // columns sigma(ya), sigma(yb)
            const int cb = warp_fft_k2(yb / RY, Wy) + Wy * (yb % RY);
            C2<float> v[RX];
#pragma unroll
            for (int j = 0; j < RX; ++j) {
                const int mx = gl + W * j;
                C2<float> z = {0.f, 0.f};
                if (act) {
                    if (mx == 0) {
                        z = {P[ca].x, P[cb].x};
                    } else if (mx < nxq) {
                        const C2<float> a = P[mx * ldp + ca], bb = P[mx * ldp + cb];
                        z = {0.5f * (a.x - bb.y), 0.5f * (a.y + bb.x)};          // (a + i b) / 2
                    } else if (mx > nxq) {
                        const C2<float> a = P[(nx - mx) * ldp + ca], bb = P[(nx - mx) * ldp + cb];
                        z = {0.5f * (a.x + bb.y), 0.5f * (bb.x - a.y)};          // (conj a + i conj b) / 2
                    }
                }
                v[j] = z;
            }
            warp_fft_dit_t<RX>(v, gl, W, lt, tx);
            // the pair's own two columns of P (read only by this lane group, now consumed) hold the
            // two output lines: x -> float (x & 1) of P[x / 2][y]
            __syncwarp();
            if (act)
#pragma unroll
                for (int k = 0; k < RX; ++k) {
                    const int x = k + RX * k2;
                    reinterpret_cast<float*>(&P[(x >> 1) * ldp + ca])[x & 1] = v[k].x;
                    reinterpret_cast<float*>(&P[(x >> 1) * ldp + cb])[x & 1] = v[k].y;
                }
            __syncwarp();
            if (act) {
                float* ra = Rout + (size_t)ya * nx;
                for (int x = gl; x < nx; x += W) {
                    ra[x] = reinterpret_cast<const float*>(&P[(x >> 1) * ldp + ca])[x & 1];
                    ra[nx + x] = reinterpret_cast<const float*>(&P[(x >> 1) * ldp + cb])[x & 1];
                }
            }
        }
    }
}

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
// Row pitch of a staged line pair: room for the skewed inputs and the skewed outputs.
__host__ __device__ __forceinline__ int zpass_pitch(int nz, int R) {
    const int a = (nz - 1) + (nz - 1) / R + 1, b = (nz - 1) + ((nz - 1) >> 4) + 1;
    return (a > b ? a : b) | 1;
}

template <int RZ, int LB>
__global__ void __launch_bounds__(256, RZ <= 8 ? 3 : 2) f32_zpass_kernel(GridDev g, const float* __restrict__ R,
                                                        const C2<float>* __restrict__ twz,
                                                        const C2<float>* __restrict__ zsh, float* __restrict__ out,
                                                        size_t out_sb, size_t out_sc) {
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.Nx, ny = g.Ny, nz = g.Nz;
    const size_t nxy = (size_t)nx * ny;
    const int comp = blockIdx.y, b = blockIdx.z;
    const size_t L0 = (size_t)blockIdx.x * LB;
    const int S = zpass_pitch(nz, RZ);                                      // odd pair pitch
    C2<float>* cs = reinterpret_cast<C2<float>*>(smem_raw);                 // [LB/2][S]
    C2<float>* tw = cs + (size_t)(LB / 2) * S;                              // [nz]
    C2<float>* zs = tw + nz;                                                // [nz]
    for (int e = threadIdx.x; e < nz; e += blockDim.x) {
        tw[e] = twz[e];
        zs[e] = zsh[e];
    }
    {   // thread t stages line t % LB for rows t / LB + k (256 / LB); loads batched ahead of the stores
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
            v[j1] = cmul(C2<float>{p.x + q.y, p.y - q.x}, zs[m]);
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
        const size_t pa = ((La % nx) * ny + La / nx) * (size_t)nz;
        const size_t pb = ((Lb % nx) * ny + Lb / nx) * (size_t)nz;
        if (La < nxy)
            for (int z = gl; z < nz; z += W) ob[pa + z] = cf[z + (z >> 4)].x;
        if (Lb < nxy)
            for (int z = gl; z < nz; z += W) ob[pb + z] = cf[z + (z >> 4)].y;
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

static int plane_ldp(const GridDev& g) { return (g.Ny + 1) | 1; }     // odd row pitch (complex units)
static size_t plane_smem(const GridDev& g) {
    const int nxh = g.Nx / 2 + 1;
    int W, R;
    warp_fft_shape(g.Nx, &W, &R);
    (void)W;
    return ((size_t)nxh * plane_ldp(g) + g.Ny + g.Nx) * sizeof(C2<float>);
}
static size_t zpass_smem(const GridDev& g, int lb, int R) {
    const size_t S = (size_t)zpass_pitch(g.Nz, R);
    return ((size_t)(lb / 2) * S + 2 * (size_t)g.Nz) * sizeof(C2<float>);
}
static size_t deposit_smem(const GridDev& g, int n_cols) {
    const int rows = (g.Nx / 2 + 1 + F32_DEP_SPLIT - 1) / F32_DEP_SPLIT;
    return (size_t)n_cols * (rows + g.Ny) * sizeof(C2<float>);
}

// Register-FFT lengths compiled in: elements per lane R = N / W.
#define WT_FOR_EACH_R(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(12) X(14) X(15) X(16) X(24)

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

void Fast32::set_radix(int r_xy, int r_z) {
    if (g.Nx % r_xy || g.Nz % r_z || !supported_r(r_xy) || !supported_r(r_z))
        fail(WT_ERR_ARG, "register-FFT length does not divide the grid");
    int w = g.Nx / r_xy, wz = g.Nz / r_z;
    if ((w & (w - 1)) || w > 32 || (wz & (wz - 1)) || wz > 32)
        fail(WT_ERR_ARG, "lanes per FFT line must be a power of two up to 32");
    const size_t sp = plane_smem(g), sz = zpass_smem(g, 64, r_z);
    if (sp > 227 * 1024 || sz > 227 * 1024) fail(WT_ERR_UNSUPPORTED, "grid too large for the FP32 plane kernels");
    switch (r_xy) {
#define WT_CASE(R) case R: { allow_dyn_smem(f32_plane_kernel<R, R>, sp); break; }
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
    }
    switch (r_z) {
#define WT_CASE(R) case R: { \
        allow_dyn_smem(f32_zpass_kernel<R, 16>, sz); \
        allow_dyn_smem(f32_zpass_kernel<R, 32>, sz); \
        allow_dyn_smem(f32_zpass_kernel<R, 64>, sz); break; }
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
    }
    rxy = r_xy;
    rz = r_z;
}

void Fast32::fields(const float* Zc, int nb, float* rho, float* R, float* out, size_t out_sb, size_t out_sc,
                    cudaStream_t s, int mode, int lb) const {
    if (lb != 16 && lb != 32 && lb != 64) fail(WT_ERR_ARG, "z-pass lines per block must be 16, 32 or 64");
    C2<float>* rc = reinterpret_cast<C2<float>*>(rho);
    dim3 gd(g.Nz, nb, F32_DEP_SPLIT);
    f32_deposit_kernel<<<gd, 256, deposit_smem(g, n_cols), s>>>(g, n_cols, reinterpret_cast<const C2<float>*>(phx.p),
                                                                reinterpret_cast<const C2<float>*>(phy.p), Zc, rc);
    WT_LAUNCH("f32_deposit");
    dim3 gp(g.Nz, 3, nb);
    const C2<float>* ty = reinterpret_cast<const C2<float>*>(tw_y.p);
    const C2<float>* tx = reinterpret_cast<const C2<float>*>(tw_x.p);
    switch (rxy) {
#define WT_CASE(RR) case RR: f32_plane_kernel<RR, RR><<<gp, 256, plane_smem(g), s>>>(g, rc, ty, tx, R, mode); break;
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
    }
    WT_LAUNCH("f32_plane");
    const size_t nxy = (size_t)g.Nx * g.Ny;
    dim3 gz((unsigned)((nxy + lb - 1) / lb), 3, nb);
    const C2<float>* tz = reinterpret_cast<const C2<float>*>(tw_z.p);
    const C2<float>* zz = reinterpret_cast<const C2<float>*>(zsh.p);
    switch (rz) {
#define WT_CASE(RR) case RR: \
        if (lb == 16) f32_zpass_kernel<RR, 16><<<gz, 256, zpass_smem(g, lb, RR), s>>>(g, R, tz, zz, out, out_sb, out_sc); \
        else if (lb == 32) f32_zpass_kernel<RR, 32><<<gz, 256, zpass_smem(g, lb, RR), s>>>(g, R, tz, zz, out, out_sb, out_sc); \
        else f32_zpass_kernel<RR, 64><<<gz, 256, zpass_smem(g, lb, RR), s>>>(g, R, tz, zz, out, out_sb, out_sc); \
        break;
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
    }
    WT_LAUNCH("f32_zpass");
}

}  // namespace wt
