// Carrier drift in the static field (the paper's Fig. 2 field with its carrier
// transport, here a constant-mobility drift that produces Eq. 1 tracks):
// dx/dt = s mu E(x), explicit midpoint steps in FP64 on the trilinear
// interpolation of the FP32 field (grid points (i hx, j hy, (k + 1/2) hz);
// x, y periodic; z clamped to the first and last planes, as in Eq. 1).  Each
// step records its midpoint and velocity; a carrier stops after the step that
// ends inside a column (nearest periodic image) or outside 0 <= z <= Lz.
#include "wt_internal.cuh"

namespace wt {

struct DriftColumn {
    double x, y, r2, z0, z1;
};

__device__ __forceinline__ void drift_interp(const float* __restrict__ E, int Nx, int Ny, int Nz, double ihx,
                                             double ihy, double ihz, double px, double py, double pz, double* out) {
    const size_t npts = (size_t)Nx * Ny * Nz;
    const double fx = px * ihx, fy = py * ihy;
    double fz = pz * ihz - 0.5;
    fz = fz < 0.0 ? 0.0 : (fz > Nz - 1.0 ? Nz - 1.0 : fz);
    const double flx = floor(fx), fly = floor(fy);
    const int k0 = min((int)floor(fz), Nz - 2);
    const double wx = fx - flx, wy = fy - fly, wz = fz - k0;
    const int i0 = (((long long)flx % Nx) + Nx) % Nx, j0 = (((long long)fly % Ny) + Ny) % Ny;
    const int i1 = (i0 + 1) % Nx, j1 = (j0 + 1) % Ny;
    const size_t a00 = ((size_t)i0 * Ny + j0) * Nz + k0, a01 = ((size_t)i0 * Ny + j1) * Nz + k0;
    const size_t a10 = ((size_t)i1 * Ny + j0) * Nz + k0, a11 = ((size_t)i1 * Ny + j1) * Nz + k0;
    for (int c = 0; c < 3; ++c) {
        const float* e = E + c * npts;
        const double v00 = (1 - wz) * e[a00] + wz * e[a00 + 1], v01 = (1 - wz) * e[a01] + wz * e[a01 + 1];
        const double v10 = (1 - wz) * e[a10] + wz * e[a10 + 1], v11 = (1 - wz) * e[a11] + wz * e[a11 + 1];
        out[c] = (1 - wx) * ((1 - wy) * v00 + wy * v01) + wx * ((1 - wy) * v10 + wy * v11);
    }
}

__global__ void drift_kernel(const float* __restrict__ E, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                             const DriftColumn* __restrict__ cols, int n_cols, const double* __restrict__ x0,
                             const double* __restrict__ smu, int n, int n_steps, double dt, float* __restrict__ X,
                             float* __restrict__ Y, float* __restrict__ Z, float* __restrict__ VX,
                             float* __restrict__ VY, float* __restrict__ VZ) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const double ihx = Nx / Lx, ihy = Ny / Ly, ihz = Nz / Lz;
    double p[3] = {x0[3 * (size_t)a], x0[3 * (size_t)a + 1], x0[3 * (size_t)a + 2]};
    const double s = smu[a];
    bool alive = true;
    for (int m = 0; m < n_steps; ++m) {
        const size_t o = (size_t)a * n_steps + m;
        if (!alive) {
            X[o] = (float)p[0]; Y[o] = (float)p[1]; Z[o] = (float)p[2];
            VX[o] = 0.f; VY[o] = 0.f; VZ[o] = 0.f;
            continue;
        }
        double k1[3], k2[3], pm[3];
        drift_interp(E, Nx, Ny, Nz, ihx, ihy, ihz, p[0], p[1], p[2], k1);
        for (int c = 0; c < 3; ++c) pm[c] = p[c] + 0.5 * dt * s * k1[c];
        drift_interp(E, Nx, Ny, Nz, ihx, ihy, ihz, pm[0], pm[1], pm[2], k2);
        for (int c = 0; c < 3; ++c) k2[c] *= s;
        X[o] = (float)(pm[0] - Lx * floor(pm[0] / Lx));
        Y[o] = (float)(pm[1] - Ly * floor(pm[1] / Ly));
        Z[o] = (float)pm[2];
        VX[o] = (float)k2[0]; VY[o] = (float)k2[1]; VZ[o] = (float)k2[2];
        for (int c = 0; c < 3; ++c) p[c] += dt * k2[c];
        p[0] -= Lx * floor(p[0] / Lx);
        p[1] -= Ly * floor(p[1] / Ly);
        if (p[2] < 0.0 || p[2] > Lz) alive = false;
        for (int k = 0; k < n_cols && alive; ++k) {
            double dx = p[0] - cols[k].x + 0.5 * Lx, dy = p[1] - cols[k].y + 0.5 * Ly;
            dx = dx - Lx * floor(dx / Lx) - 0.5 * Lx;
            dy = dy - Ly * floor(dy / Ly) - 0.5 * Ly;
            if (dx * dx + dy * dy < cols[k].r2 && p[2] >= cols[k].z0 && p[2] <= cols[k].z1) alive = false;
        }
    }
    if (!alive) {}   // the last position stays as recorded
}

void drift_launch(cudaStream_t s, const float* E, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                  const std::vector<double>& colspec, const double* x0, const double* smu, int n, int n_steps,
                  double dt, float* X, float* Y, float* Z, float* VX, float* VY, float* VZ) {
    const int n_cols = (int)colspec.size() / 5;
    DBuf<double> dcols;
    dcols.upload(colspec.data(), colspec.size(), s);
    drift_kernel<<<(n + 127) / 128, 128, 0, s>>>(E, Nx, Ny, Nz, Lx, Ly, Lz,
                                                 reinterpret_cast<const DriftColumn*>(dcols.p), n_cols, x0, smu, n,
                                                 n_steps, dt, X, Y, Z, VX, VY, VZ);
    WT_LAUNCH("drift");
    WT_CUDA(cudaStreamSynchronize(s));     // the column table is freed on return
}

}  // namespace wt
