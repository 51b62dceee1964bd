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
// NY2 = 0: y transforms by the register FFT of RY elements per lane; NY2 = Ny
// in {64, 128}: two-pass shared-memory y transforms (as in the z pass), Y[y]
// stored at column y.  X2 (with NY2 = Nx = Ny): the x transforms two-pass as
// well, their exchange matrix in the pair's own two columns, stores from
// registers (RX and XDIRECT unused).
template <int RY, int RX, bool XDIRECT, int NY2, bool X2 = false>
__global__ void __launch_bounds__(256, RX <= 5 ? 3 : 2) f32_plane_kernel(GridDev g, const C2<float>* __restrict__ rho,
                                                        const C2<float>* __restrict__ twy,
                                                        const C2<float>* __restrict__ twx, float* __restrict__ R,
                                                        int mode) {
    constexpr int YA = plane_y2_a(NY2), YB = NY2 ? NY2 / YA : 1;
    extern __shared__ unsigned char smem_raw[];
    const int nx = g.Nx, ny = g.Ny, nz = g.Nz, nxh = nx / 2 + 1, nxq = nx / 2;
    const int mz = blockIdx.x, comp = blockIdx.y, b = blockIdx.z;
    const int ldp = plane_ldp_of(ny, NY2);                     // odd pitch: conflict-free column reads
    C2<float>* P = reinterpret_cast<C2<float>*>(smem_raw);     // [nxh][ldp]
    C2<float>* ty = P + (size_t)nxh * ldp;                     // [ny]
    C2<float>* tx = ty + ny;                                   // [nx]
    C2<float>* tl = tx + nx;                                   // [YB][YA]: w_ny^{a c} (two-pass y)
    float* Rout = R + (((size_t)b * 3 + comp) * nz + mz) * nx * ny;
    if (comp == 2 && mz == 0) {       // the sine series has no k_z = 0 term
        for (int e = threadIdx.x; e < nx * ny; e += blockDim.x) Rout[e] = 0.f;
        return;
    }
    for (int e = threadIdx.x; e < ny; e += blockDim.x) ty[e] = twy[e];
    for (int e = threadIdx.x; e < nx; e += blockDim.x) tx[e] = twx[e];
    if constexpr (NY2 != 0)
        for (int e = threadIdx.x; e < NY2; e += blockDim.x) tl[e] = twy[(e % YA) * (e / YA)];
    const float kz = (float)(kPi * mz / g.Lz);
    const float ckx = (float)(2.0 * kPi / g.Lx), cky = (float)(2.0 * kPi / g.Ly);
    const float pref = (float)g.pref;
    const C2<float>* rp = rho + ((size_t)b * nz + mz) * nxh * ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Wy = ny / RY;
    // spectral multiplier of element m_y of row m_x (live: a row that carries data)
    // FP32 fast division: the path's tolerance is far above its 2-ulp error.
    auto mult = [&](C2<float> r, int my, float kx, float fold, bool live) {
        const int mys = my < ny / 2 ? my : my - ny;
        const float ky = cky * mys;
        const float kp2 = kx * kx + ky * ky;
        const float k2 = kp2 + kz * kz;
        C2<float> e = {0.f, 0.f};
        if (live && my != ny / 2 && k2 > 0.f) {
            float gk = __fdividef(pref * fold, k2);
            if (mode == 1) gk *= (comp < 2 ? -3.f : -2.f) + __fdividef(2.f * kp2, k2);
            // the z pass's cosine series carries the factor 2 of the +-k_z pair itself
            if (comp == 0) { const float f = kx * gk; e = {r.y * f, -r.x * f}; }
            else if (comp == 1) { const float f = ky * gk; e = {r.y * f, -r.x * f}; }
            else { const float f = 2.f * kz * gk; e = {r.x * f, r.y * f}; }
        }
        return e;
    };
    __syncthreads();                                           // twiddle tables
    if constexpr (NY2 == 0) {
        // multiplier and y transform, row by row from global memory: rows 0 <= m_x < nx/2 of
        // length ny (the x Nyquist row m_x = nx/2 is zero and the x transforms never read it;
        // decimation in time: lanes read consecutive elements).  Lane gl ends with
        // Y[k + RY bitrev(gl)] and writes it at row position gl + Wy k (consecutive lanes, no
        // bank conflicts): Y[y] sits at column sigma(y) = bitrev(y / RY) + Wy (y % RY).
        const int W = Wy, G = 32 / W, grp = lane / W, gl = lane % W;
        LaneTw<RY> lt;
        lane_twiddles<RY>(ty, gl, W, true, lt);
        // the next row's rho^ values are loaded while the current row is transformed
        C2<float> raw[RY];
        auto load_row = [&](int base_) {
            const int mx_ = base_ + grp;
            const bool live_ = mx_ < nxq;
            const C2<float>* rrow = rp + (size_t)(live_ ? mx_ : 0) * ny;
#pragma unroll
            for (int j = 0; j < RY; ++j) raw[j] = live_ ? rrow[gl + W * j] : C2<float>{0.f, 0.f};
        };
        if (warp * G < nxq) load_row(warp * G);
        for (int base = warp * G; base < nxq; base += 8 * G) {
            const int mx = base + grp;
            const bool act = mx < nxq;
            const float kx = ckx * mx;
            const float fold = mx ? 2.f : 1.f;                     // x half-spectrum fold
            C2<float> v[RY];
#pragma unroll
            for (int j = 0; j < RY; ++j) v[j] = mult(raw[j], gl + W * j, kx, fold, act);
            if (base + 8 * G < nxq) load_row(base + 8 * G);
            warp_fft_dit_t<RY>(v, gl, W, lt, ty);
            if (act)
#pragma unroll
                for (int k = 0; k < RY; ++k) P[mx * ldp + gl + W * k] = v[k];
        }
    } else {
        // two-pass y transforms, Ny = YA YB: lane a of a row's YA lanes takes m_y = a + YA j
        // (a YB-point DFT over j, twiddles w_ny^{a c}, the matrix to the row's own
        // storage, entry (a, c) at a YB + ((a + c) mod YB)), then YB / YA YA-point DFTs per
        // lane; Y[y] at column y.  The four rows of a warp are 8 apart: with the pitch = 1
        // mod 16 the two rows of a half-warp fall into disjoint bank halves.
        // (no prefetch of the next row here: the YB inputs would double the live registers)
        static_assert(YA == 8, "the row mapping assumes 8 lanes per line");
        const int grp = lane / YA, gl = lane % YA;
        for (int k0 = 0; k0 < nxq; k0 += 32) {
            const int mx = k0 + warp + 8 * grp;
            const bool act = mx < nxq;
            const float kx = ckx * mx;
            const float fold = mx ? 2.f : 1.f;
            const C2<float>* rrow = rp + (size_t)(act ? mx : 0) * ny;
            C2<float> v[YB];
#pragma unroll
            for (int j = 0; j < YB; ++j) v[j] = act ? rrow[gl + YA * j] : C2<float>{0.f, 0.f};
#pragma unroll
            for (int j = 0; j < YB; ++j) v[j] = mult(v[j], gl + YA * j, kx, fold, act);
            C2<float>* row = P + (size_t)(act ? mx : 0) * ldp;
            reg_dft_c<YB>(v);
#pragma unroll
            for (int c = 1; c < YB; ++c) v[c] = cmul(v[c], tl[c * YA + gl]);
            if (act)
#pragma unroll
                for (int c = 0; c < YB; ++c) row[gl * YB + ((gl + c) & (YB - 1))] = v[c];
            __syncwarp();
            C2<float> o[YB];
#pragma unroll
            for (int r = 0; r < YB / YA; ++r) {
                C2<float> u[YA];
#pragma unroll
                for (int a = 0; a < YA; ++a)
                    u[a] = act ? row[a * YB + ((a + gl + YA * r) & (YB - 1))] : C2<float>{0.f, 0.f};
                reg_dft_c<YA>(u);
#pragma unroll
                for (int d = 0; d < YA; ++d) o[r * YA + d] = u[d];
            }
            __syncwarp();                         // the matrix is read before the outputs overwrite it
            if (act)
#pragma unroll
                for (int r = 0; r < YB / YA; ++r)
#pragma unroll
                    for (int d = 0; d < YA; ++d) row[gl + YA * r + YB * d] = o[r * YA + d];
        }
    }
    __syncthreads();
    if constexpr (X2) {
        // two-pass x transforms of Nx = YA YB, two real lines (ya, yb) per complex FFT with the
        // Hermitian completion of the register path below; pass 1 reads the pair's columns, then
        // holds the YA x YB exchange matrix there: entry (a, c) at slot s = 8 c + ((a + c) mod 8)
        // < Nx, row s mod (Nx/2) of column ya (s < Nx/2) or yb (rows 0..Nx/2 - 1 of both
        // columns; the plane has Nx/2 + 1 rows).  The pairs of a half-warp are 4 apart
        // (columns 8 apart): disjoint bank halves.
        static_assert(YA == 8, "the pair mapping assumes 8 lanes per line");
        const int grp = lane / YA, gl = lane % YA;
        for (int k0 = 0; k0 < ny / 2; k0 += 32) {
            const int pp = k0 + 16 * (warp >> 2) + (warp & 3) + 4 * grp;
            const bool act = pp < ny / 2;
            const int ya = 2 * pp, yb = ya + 1;
            const int ca = act ? ya : 0, cb = act ? yb : 0;
            C2<float> v[YB];
#pragma unroll
            for (int j = 0; j < YB; ++j) {
                const int mx = gl + YA * j;
                C2<float> z = {0.f, 0.f};
                if (act) {
                    if (mx == 0) {
                        z = {P[ca].x, P[cb].x};
                    } else if (mx < nxq) {
                        const C2<float> a = P[mx * ldp + ca], bb = P[mx * ldp + cb];
                        z = {0.5f * (a.x - bb.y), 0.5f * (a.y + bb.x)};
                    } else if (mx > nxq) {
                        const C2<float> a = P[(nx - mx) * ldp + ca], bb = P[(nx - mx) * ldp + cb];
                        z = {0.5f * (a.x + bb.y), 0.5f * (bb.x - a.y)};
                    }
                }
                v[j] = z;
            }
            __syncwarp();                         // the pair's columns are read before they hold the matrix
            reg_dft_c<YB>(v);
#pragma unroll
            for (int c = 1; c < YB; ++c) v[c] = cmul(v[c], tl[c * YA + gl]);
            auto slot = [&](int a, int c) -> C2<float>& {
                const int sl = 8 * c + ((a + c) & 7);
                return P[(sl & (nxq - 1)) * ldp + (sl < nxq ? ca : cb)];     // nx a power of two
            };
            if (act)
#pragma unroll
                for (int c = 0; c < YB; ++c) slot(gl, c) = v[c];
            __syncwarp();
            C2<float> o[YB];
#pragma unroll
            for (int r = 0; r < YB / YA; ++r) {
                C2<float> u[YA];
#pragma unroll
                for (int a = 0; a < YA; ++a) u[a] = act ? slot(a, gl + YA * r) : C2<float>{0.f, 0.f};
                reg_dft_c<YA>(u);
#pragma unroll
                for (int d = 0; d < YA; ++d) o[r * YA + d] = u[d];
            }
            if (act) {
                float* ra = Rout + (size_t)ya * nx;
#pragma unroll
                for (int r = 0; r < YB / YA; ++r)
#pragma unroll
                    for (int d = 0; d < YA; ++d) {
                        const int x = gl + YA * r + YB * d;
                        ra[x] = o[r * YA + d].x;
                        ra[nx + x] = o[r * YA + d].y;
                    }
            }
        }
    } else
    {   // x: ny real lines of length nx from the half spectrum, two lines (y = 2p, 2p + 1) per
        // complex FFT: Z[m] = A'[m] + i B'[m] with the Hermitian completions A'[0] = Re a[0],
        // A'[m] = a[m] / 2, A'[nx - m] = conj(a[m]) / 2 (0 < m < nx/2; a carries the x fold
        // factor 2), A'[nx/2] = 0, so that FFT(Z) = out_a + i out_b.  Decimation in time reads
        // consecutive rows per lane; the two output lines are staged in the pair's own columns
        // of P for coalesced stores.
        const int W = nx / RX, G = 32 / W, grp = lane / W, gl = lane % W;
        const int k2 = warp_fft_k2(gl, W);
        LaneTw<RX> lt;
        lane_twiddles<RX>(tx, gl, W, true, lt);
        for (int base = warp * G; base < ny / 2; base += 8 * G) {
            const int pp = base + grp;
            const bool act = pp < ny / 2;
            const int ya = 2 * pp, yb = ya + 1;
            // columns of Y[ya], Y[yb]: sigma(y) after the register y FFT, y after the two-pass one
            const int ca = NY2 ? ya : warp_fft_k2(ya / RY, Wy) + Wy * (ya % RY);
            const int cb = NY2 ? yb : warp_fft_k2(yb / RY, Wy) + Wy * (yb % RY);
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

void plane_allow(int r, int ny2, size_t sp) {
    if (ny2) {
        if (r == 0) {                         // two-pass x transforms as well
            if (ny2 == 64) { allow_dyn_smem(f32_plane_kernel<2, 2, true, 64, true>, sp); return; }
            if (ny2 == 128) { allow_dyn_smem(f32_plane_kernel<4, 4, true, 128, true>, sp); return; }
        }
#define WT_CASE(NN, RR) \
        if (ny2 == NN && r == RR) { allow_dyn_smem(f32_plane_kernel<RR, RR, false, NN>, sp); \
                                    allow_dyn_smem(f32_plane_kernel<RR, RR, true, NN>, sp); return; }
        WT_FOR_EACH_Y2(WT_CASE)
#undef WT_CASE
        fail(WT_ERR_UNSUPPORTED, "two-pass y transforms: Ny in {64, 128} with 16 or 32 lanes per x line");
    }
    switch (r) {
#define WT_CASE(R) case R: { allow_dyn_smem(f32_plane_kernel<R, R, false, 0>, sp); \
                                allow_dyn_smem(f32_plane_kernel<R, R, true, 0>, sp); break; }
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
        default: fail(WT_ERR_UNSUPPORTED, "register-FFT length not compiled in");
    }
}

bool plane_y2_supported(int ny, int r) {
    if (r == 0) return ny == 64 || ny == 128;     // with two-pass x transforms
#define WT_CASE(NN, RR) if (ny == NN && r == RR) return true;
    WT_FOR_EACH_Y2(WT_CASE)
#undef WT_CASE
    return false;
}

void plane_launch(int r, bool xdirect, int ny2, dim3 gp, cudaStream_t s, const GridDev& g, const C2<float>* rc,
                  const C2<float>* ty, const C2<float>* tx, float* R, int mode) {
    const size_t sp = plane_smem(g, ny2);
    if (ny2) {
        if (r == 0) {                         // two-pass x transforms as well
            if (ny2 == 64) f32_plane_kernel<2, 2, true, 64, true><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode);
            else if (ny2 == 128) f32_plane_kernel<4, 4, true, 128, true><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode);
            else fail(WT_ERR_UNSUPPORTED, "two-pass x transforms: Nx = Ny in {64, 128}");
            WT_LAUNCH("f32_plane");
            return;
        }
#define WT_CASE(NN, RR) \
        if (ny2 == NN && r == RR) { \
            if (xdirect) f32_plane_kernel<RR, RR, true, NN><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode); \
            else f32_plane_kernel<RR, RR, false, NN><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode); \
            WT_LAUNCH("f32_plane"); return; }
        WT_FOR_EACH_Y2(WT_CASE)
#undef WT_CASE
        fail(WT_ERR_UNSUPPORTED, "two-pass y transforms: Ny in {64, 128} with 16 or 32 lanes per x line");
    }
    switch (r) {
#define WT_CASE(RR) case RR: \
        if (xdirect) f32_plane_kernel<RR, RR, true, 0><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode); \
        else f32_plane_kernel<RR, RR, false, 0><<<gp, 256, sp, s>>>(g, rc, ty, tx, R, mode); \
        break;
        WT_FOR_EACH_R(WT_CASE)
#undef WT_CASE
        default: fail(WT_ERR_UNSUPPORTED, "register-FFT length not compiled in");
    }
    WT_LAUNCH("f32_plane");
}

}  // namespace wt
