// FP32 plane pass of the bulk extension (see k_fft32.cu): the per-k_z-plane
// lateral inverse FFT, one register-FFT length per template instance.
#include "k_fft32_common.cuh"

namespace wt {

// One (k_z plane, component, charge vector) per block: component factor,
// inverse FFT along y for every m_x row, then half spectrum -> real along x.
// Warp FFTs in registers; the plane stays in shared memory.
// Output R[b][c][mz][y][x].  grid (Nz, 3, nb).
// mode 0: the field; mode 1: its derivative with respect to the lateral scale
// lambda (Lx, Ly, column and grid positions scale together): the multiplier
// times (-3 + 2 k_perp^2/|k|^2) for W_x, W_y and (-2 + 2 k_perp^2/|k|^2) for W_z.
template <int RY, int RX, bool XDIRECT>
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
    const int Wy = ny / RY;
    __syncthreads();                                           // twiddle tables
    {   // multiplier and y transform, row by row from global memory: nxh lines of length ny
        // (decimation in time: lanes read consecutive elements).  Lane gl ends with
        // Y[k + RY bitrev(gl)] and writes it at row position gl + Wy k (consecutive lanes, no
        // bank conflicts): Y[y] sits at column sigma(y) = bitrev(y / RY) + Wy (y % RY).
        // FP32 fast division: the path's tolerance is far above its 2-ulp error.
        const int W = Wy, G = 32 / W, grp = lane / W, gl = lane % W;
        LaneTw<RY> lt;
        lane_twiddles<RY>(ty, gl, W, true, lt);
        // the next row's rho^ values are loaded while the current row is transformed
        C2<float> raw[RY];
        auto load_row = [&](int base_) {
            const int mx_ = base_ + grp;
            const bool live_ = mx_ < nxh && mx_ != nx / 2;
            const C2<float>* rrow = rp + (size_t)(live_ ? mx_ : 0) * ny;
#pragma unroll
            for (int j = 0; j < RY; ++j) raw[j] = live_ ? rrow[gl + W * j] : C2<float>{0.f, 0.f};
        };
        if (warp * G < nxh) load_row(warp * G);
        for (int base = warp * G; base < nxh; base += 8 * G) {
            const int mx = base + grp;
            const bool act = mx < nxh;
            const bool live = act && mx != nx / 2;                 // the x Nyquist row stays zero
            const float kx = ckx * mx;
            const float fold = mx ? 2.f : 1.f;                     // x half-spectrum fold
            C2<float> v[RY];
#pragma unroll
            for (int j = 0; j < RY; ++j) {
                const int my = gl + W * j;
                const int mys = my < ny / 2 ? my : my - ny;
                const float ky = cky * mys;
                const float kp2 = kx * kx + ky * ky;
                const float k2 = kp2 + kz * kz;
                C2<float> e = {0.f, 0.f};
                if (live && my != ny / 2 && k2 > 0.f) {
                    const C2<float> r = raw[j];
                    float gk = __fdividef(pref * fold, k2);
                    if (mode == 1) gk *= (comp < 2 ? -3.f : -2.f) + __fdividef(2.f * kp2, k2);
                    // the z pass's cosine series carries the factor 2 of the +-k_z pair itself
                    if (comp == 0) { const float f = kx * gk; e = {r.y * f, -r.x * f}; }
                    else if (comp == 1) { const float f = ky * gk; e = {r.y * f, -r.x * f}; }
                    else { const float f = 2.f * kz * gk; e = {r.x * f, r.y * f}; }
                }
                v[j] = e;
            }
            if (base + 8 * G < nxh) load_row(base + 8 * G);
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
            if constexpr (XDIRECT) {
                // straight from registers: lane gl holds x = k + RX bitrev(gl); the partial lines
                // of the RX stores per row merge in L2
                if (act) {
                    float* ra = Rout + (size_t)ya * nx;
#pragma unroll
                    for (int k = 0; k < RX; ++k) {
                        ra[k + RX * k2] = v[k].x;
                        ra[nx + k + RX * k2] = v[k].y;
                    }
                }
                continue;
            }
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

void plane_allow(int r, size_t sp) {
    switch (r) {
#define WT_CASE(R) case R: { allow_dyn_smem(f32_plane_kernel<R, R, false>, sp); \
                                allow_dyn_smem(f32_plane_kernel<R, R, true>, sp); break; }
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
        default: fail(WT_ERR_UNSUPPORTED, "register-FFT length not compiled in");
    }
}

void plane_launch(int r, bool xdirect, dim3 gp, cudaStream_t s, const GridDev& g, const C2<float>* rc,
                  const C2<float>* ty, const C2<float>* tx, float* R, int mode) {
    const size_t sp = plane_smem(g);
    switch (r) {
#define WT_CASE(RR) case RR: \
        if (xdirect) f32_plane_kernel<RR, RR, true><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode); \
        else f32_plane_kernel<RR, RR, false><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode); \
        break;
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
        default: fail(WT_ERR_UNSUPPORTED, "register-FFT length not compiled in");
    }
    WT_LAUNCH("f32_plane");
}

}  // namespace wt
