// Exact FP64 point evaluation of the field (the band-limited spectral sum of
// the bulk extension, Abstract / Sec. 1, at arbitrary points):
//   W_x(p) = pref sum_c sum_mz w(mz) Zc(mz) cos(kz z_p) Lx(p - x_c; kz)
//   W_y(p) = pref sum_c sum_mz w(mz) Zc(mz) cos(kz z_p) Ly(p - x_c; kz)
//   W_z(p) = pref sum_c sum_mz Zc(mz) 2 kz sin(kz z_p) L0(p - x_c; kz)
// with the lateral sums over all (kx, ky) of the band:
//   Lx = sum kx sin(kx dx) cos(ky dy)/|k|^2, Ly = sum ky cos(kx dx) sin(ky dy)/|k|^2,
//   L0 = sum cos(kx dx) cos(ky dy)/|k|^2  (k = 0 excluded).
#include "wt_internal.cuh"

namespace wt {

// Lat[p][c][mz][3] for one point per block.x, one column per block.y.
__global__ void sample_lateral_kernel(const double* __restrict__ pts, const double* __restrict__ col_xy, int n_cols,
                                      int hx, int hy, int nz, double Lx, double Ly, const double* __restrict__ T,
                                      double* __restrict__ Lat) {
    extern __shared__ double sh[];
    double* cx = sh;
    double* sx = cx + hx;
    double* cy = sx + hx;
    double* sy = cy + hy;
    const int p = blockIdx.x, c = blockIdx.y;
    const double dx = pts[3 * p] - col_xy[2 * c], dy = pts[3 * p + 1] - col_xy[2 * c + 1];
    for (int m = threadIdx.x; m < hx; m += blockDim.x) sincospi(2.0 * m * dx / Lx, &sx[m], &cx[m]);
    for (int m = threadIdx.x; m < hy; m += blockDim.x) sincospi(2.0 * m * dy / Ly, &sy[m], &cy[m]);
    __syncthreads();
    for (int mz = threadIdx.x; mz < nz; mz += blockDim.x) {
        double ax = 0.0, ay = 0.0, a0 = 0.0;
        for (int mx = 0; mx < hx; ++mx) {
            const double kx = 2.0 * kPi * mx / Lx;
            const double wxx = mx ? 2.0 : 1.0;
            double iy_c = 0.0, iy_s = 0.0;   // sum_my wy cy T, sum_my wy ky sy T
            const double* t = T + (size_t)mx * hy * nz + mz;
            for (int my = 0; my < hy; ++my) {
                const double tv = t[(size_t)my * nz];
                const double wy = my ? 2.0 : 1.0;
                iy_c = fma(wy * cy[my], tv, iy_c);
                iy_s = fma(2.0 * (2.0 * kPi * my / Ly) * sy[my], tv, iy_s);
            }
            ax = fma(2.0 * kx * sx[mx], iy_c, ax);   // +-kx pairs; mx = 0 gives 0
            ay = fma(wxx * cx[mx], iy_s, ay);
            a0 = fma(wxx * cx[mx], iy_c, a0);
        }
        double* o = Lat + (((size_t)p * n_cols + c) * nz + mz) * 3;
        o[0] = ax;
        o[1] = ay;
        o[2] = a0;
    }
}

// out[t][p][a] from Zc[t][c][mz] and Lat.  Thread per (t, p).
__global__ void sample_contract_kernel(const double* __restrict__ pts, const double* __restrict__ Lat,
                                       const double* __restrict__ Zc, int n_pts, int n_t, int n_cols, int nz,
                                       double Lz, double pref, double* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_pts * n_t) return;
    const int t = idx / n_pts, p = idx % n_pts;
    const double z = pts[3 * p + 2];
    double wx = 0.0, wy = 0.0, wz = 0.0;
    for (int c = 0; c < n_cols; ++c) {
        const double* zc = Zc + ((size_t)t * n_cols + c) * nz;
        const double* lat = Lat + ((size_t)p * n_cols + c) * nz * 3;
        for (int mz = 0; mz < nz; ++mz) {
            double sn, cs;
            sincospi((double)mz * z / Lz, &sn, &cs);
            const double kz = kPi * mz / Lz;
            const double w = mz ? 2.0 : 1.0;
            const double a = zc[mz];
            wx = fma(w * a * cs, lat[3 * mz], wx);
            wy = fma(w * a * cs, lat[3 * mz + 1], wy);
            wz = fma(2.0 * kz * a * sn, lat[3 * mz + 2], wz);
        }
    }
    double* o = out + ((size_t)t * n_pts + p) * 3;
    o[0] = pref * wx;
    o[1] = pref * wy;
    o[2] = pref * wz;
}

void sample_lateral(cudaStream_t s, const double* pts, int n_pts, const double* col_xy, int n_cols, int Nx, int Ny,
                    int Nz, double Lx, double Ly, const double* T, double* Lat) {
    dim3 grid(n_pts, n_cols);
    size_t sh = (size_t)(Nx + Ny) * sizeof(double);
    sample_lateral_kernel<<<grid, 128, sh, s>>>(pts, col_xy, n_cols, Nx / 2, Ny / 2, Nz, Lx, Ly, T, Lat);
    WT_LAUNCH("sample_lateral");
}
void sample_contract(cudaStream_t s, const double* pts, const double* Lat, const double* Zc, int n_pts, int n_t,
                     int n_cols, int Nz, double Lz, double pref, double* out) {
    int tot = n_pts * n_t;
    sample_contract_kernel<<<(tot + 127) / 128, 128, 0, s>>>(pts, Lat, Zc, n_pts, n_t, n_cols, Nz, Lz, pref, out);
    WT_LAUNCH("sample_contract");
}

}  // namespace wt
