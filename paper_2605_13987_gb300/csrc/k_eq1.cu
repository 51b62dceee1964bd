// Eq. 1 (Ramo-Shockley-Riegler convolution) against carrier tracks, direct
// form on the stored FP32 field H[t][c][x][y][z]:
//   Q(tau_m) = sum_{m' <= m, m' < n_steps} W(x_m', (m - m' + 1/2) dt) . v_m' dt
//   i(tau_m) = -(q / V_w) (Q(tau_m) - Q(tau_{m-1})) / dt
// W between grid points: trilinear (periodic x, y; z clamped to the first and
// last grid planes); between time samples: linear in t, W(0) = 0, held after
// the last sample.  One block per track: the dot products W(x_m', t_n) . v_m'
// at the time samples are staged in shared memory for a chunk of steps, then
// every output time accumulates its lags: the FP64 field in FP64; the FP32
// field as current increments, FP32 within a chunk and FP64 across chunks.
#include "wt_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

namespace wt {

struct Eq1Lag {
    int n;          // lower time sample
    float w0, w1;   // weights of samples n and n+1
};
// FP64 weights, for the FP64 field of the loss
struct Eq1Lag64 {
    int n;
    double w0, w1;
};

constexpr int EQ1_MC = 16;   // track steps per chunk

// Current increments of one chunk of track steps (FP32 field): for output m,
//   D(m) = Q(tau_m) - Q(tau_{m-1}) = sum_j [g_j(m - m'_j) - g_j(m - m'_j - 1)] dt,
// g_j(L) = W(x_j, (L + 1/2) dt) . v_j (linear in time between the staged samples f[j][n],
// g_j(-1) = 0), summed in FP32 over the chunk's steps (at most EQ1_MC terms, each a difference of
// neighbouring lags, so nothing large cancels) and carried across chunks in FP64: one FP64
// addition per output and chunk instead of FP64 products per lag (GB300's FP64 rate is low).
__device__ __forceinline__ float eq1_interp(const float* __restrict__ fj, int nt, Eq1Lag lg) {
    return fmaf(lg.w0, fj[lg.n], lg.w1 * fj[min(lg.n + 1, nt - 1)]);
}
// f: [mc][nt] (nt: the row stride, also the clamp of sample n + 1); outputs m < c0 take nothing
// from this chunk, so the threads start at c0.
__device__ __forceinline__ void eq1_increments(const float* __restrict__ f, int nt, int mc, int c0, int n_out,
                                               const Eq1Lag* __restrict__ lags, double* __restrict__ D) {
    for (int m = c0 + threadIdx.x; m < n_out; m += blockDim.x) {
        const int jmax = min(mc - 1, m - c0);
        if (jmax < 0) continue;
        // step j sees lag L = m - c0 - j; the entry of lag L - 1 is the next step's entry of lag L
        int L = m - c0;
        Eq1Lag hi = lags[L];
        float d = 0.f;
        for (int j = 0; j <= jmax; ++j, --L) {
            const float* fj = f + j * nt;
            const float g_hi = eq1_interp(fj, nt, hi);
            if (L == 0) {
                d += g_hi;
                break;
            }
            const Eq1Lag lo = lags[L - 1];
            d += g_hi - eq1_interp(fj, nt, lo);
            hi = lo;
        }
        D[m] += (double)d;
    }
}

// T: field type; L: lag table entry; TO: current type
template <class T, class L, class TO>
// nu: time samples the lag table reads (samples n >= nu are never staged)
__global__ void __launch_bounds__(256) eq1_kernel(const T* __restrict__ H, int Nx, int Ny, int Nz, int nt, int nu,
                                                  T inv_hx, T inv_hy, T inv_hz,
                                                  const float* __restrict__ X, const float* __restrict__ Y,
                                                  const float* __restrict__ Z, const float* __restrict__ VX,
                                                  const float* __restrict__ VY, const float* __restrict__ VZ,
                                                  const float* __restrict__ qtrack, float qconst, int n_steps,
                                                  int n_out, double dt, double inv_vw,
                                                  const L* __restrict__ lags, TO* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* f = reinterpret_cast<T*>(smem_raw);                               // [EQ1_MC][nt]
    double* Q = reinterpret_cast<double*>(smem_raw + (((size_t)EQ1_MC * nt * sizeof(T) + 15) & ~(size_t)15));   // [n_out]
    const int tr = blockIdx.x;
    const size_t npts = (size_t)Nx * Ny * Nz;
    for (int m = threadIdx.x; m < n_out; m += blockDim.x) Q[m] = 0.0;
    for (int c0 = 0; c0 < n_steps; c0 += EQ1_MC) {
        const int mc = min(EQ1_MC, n_steps - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < mc * nu; e += blockDim.x) {
            const int j = e / nu, n = e % nu;
            const size_t s = (size_t)tr * n_steps + c0 + j;
            const T vx = VX[s], vy = VY[s], vz = VZ[s];
            T acc = 0;
            if (vx != 0 || vy != 0 || vz != 0) {
                const T one = 1;
                const T fx = (T)X[s] * inv_hx, fy = (T)Y[s] * inv_hy;
                T fz = (T)Z[s] * inv_hz - (T)0.5;
                fz = fz < (T)0 ? (T)0 : (fz > (T)(Nz - 1) ? (T)(Nz - 1) : fz);
                const T flx = floor(fx), fly = floor(fy);
                int k0 = min((int)floor(fz), Nz - 2);
                const T wx = fx - flx, wy = fy - fly, wz = fz - (T)k0;
                int i0 = ((int)flx % Nx + Nx) % Nx, j0 = ((int)fly % Ny + Ny) % Ny;
                const int i1 = (i0 + 1) % Nx, j1 = (j0 + 1) % Ny;
                const T* hb = H + (size_t)n * 3 * npts;
                T w[3] = {0, 0, 0};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T* h = hb + (size_t)c * npts;
                    const size_t a00 = ((size_t)i0 * Ny + j0) * Nz + k0, a01 = ((size_t)i0 * Ny + j1) * Nz + k0;
                    const size_t a10 = ((size_t)i1 * Ny + j0) * Nz + k0, a11 = ((size_t)i1 * Ny + j1) * Nz + k0;
                    const T v00 = (one - wz) * h[a00] + wz * h[a00 + 1];
                    const T v01 = (one - wz) * h[a01] + wz * h[a01 + 1];
                    const T v10 = (one - wz) * h[a10] + wz * h[a10 + 1];
                    const T v11 = (one - wz) * h[a11] + wz * h[a11 + 1];
                    w[c] = (one - wx) * ((one - wy) * v00 + wy * v01) + wx * ((one - wy) * v10 + wy * v11);
                }
                acc = w[0] * vx + w[1] * vy + w[2] * vz;
            }
            f[j * nt + n] = acc;
        }
        __syncthreads();
        if constexpr (std::is_same<T, float>::value) {
            // FP32 field: increments D(m) = Q(tau_m) - Q(tau_{m-1}) over dt, accumulated in Q
            eq1_increments(f, nt, mc, c0, n_out, lags, Q);
        } else {
            for (int m = threadIdx.x; m < n_out; m += blockDim.x) {
                double q = 0.0;
                const int jmax = min(mc - 1, m - c0);
                for (int j = 0; j <= jmax; ++j) {
                    const L lg = lags[m - (c0 + j)];
                    q += (double)lg.w0 * (double)f[j * nt + lg.n] +
                         (double)lg.w1 * (double)f[j * nt + min(lg.n + 1, nt - 1)];
                }
                Q[m] += q * dt;
            }
        }
    }
    __syncthreads();
    const float qc = qtrack ? qtrack[tr] : qconst;
    for (int m = threadIdx.x; m < n_out; m += blockDim.x) {
        // FP32 field: Q holds the increments already (the dt of Q and of the derivative cancel)
        const double dq = std::is_same<T, float>::value ? Q[m] * dt : Q[m] - (m ? Q[m - 1] : 0.0);
        out[(size_t)tr * n_out + m] = (TO)(-(double)qc * inv_vw * dq / dt);
    }
}

template <class T, class L, class TO>
static void eq1_launch_t(cudaStream_t s, const T* H, int Nx, int Ny, int Nz, int nt, double Lx, double Ly, double Lz,
                         const float* x, const float* y, const float* z, const float* vx, const float* vy,
                         const float* vz, const float* q, float qconst, int n_tracks, int n_steps, int n_out,
                         double dt, double v_w, const void* lags, int nu, TO* out) {
    if (nu < 1 || nu > nt) fail(WT_ERR_ARG, "eq1: bad count of time samples in use");
    size_t sh = (((size_t)EQ1_MC * nt * sizeof(T) + 15) & ~(size_t)15) + (size_t)n_out * sizeof(double);
    if (sh > 200 * 1024) fail(WT_ERR_UNSUPPORTED, "eq1: n_t or n_out too large for shared memory");
    allow_dyn_smem(eq1_kernel<T, L, TO>, sh);
    eq1_kernel<T, L, TO><<<n_tracks, 256, sh, s>>>(H, Nx, Ny, Nz, nt, nu, (T)(Nx / Lx), (T)(Ny / Ly), (T)(Nz / Lz), x, y,
                                                   z, vx, vy, vz, q, qconst, n_steps, n_out, dt, 1.0 / v_w,
                                                   static_cast<const L*>(lags), out);
    WT_LAUNCH("eq1");
}
void eq1_launch(cudaStream_t s, const float* H, int Nx, int Ny, int Nz, int nt, double Lx, double Ly, double Lz,
                const float* x, const float* y, const float* z, const float* vx, const float* vy, const float* vz,
                const float* q, float qconst, int n_tracks, int n_steps, int n_out, double dt, double v_w,
                const void* lags, int nu, float* out) {
    eq1_launch_t<float, Eq1Lag, float>(s, H, Nx, Ny, Nz, nt, Lx, Ly, Lz, x, y, z, vx, vy, vz, q, qconst, n_tracks,
                                       n_steps, n_out, dt, v_w, lags, nu, out);
}
// FP64 field (plain path): interpolation, time weights and currents in FP64 (lags: FP64 table).
void eq1_launch64(cudaStream_t s, const double* H, int Nx, int Ny, int Nz, int nt, double Lx, double Ly, double Lz,
                  const float* x, const float* y, const float* z, const float* vx, const float* vy, const float* vz,
                  const float* q, float qconst, int n_tracks, int n_steps, int n_out, double dt, double v_w,
                  const void* lags, int nu, double* out) {
    eq1_launch_t<double, Eq1Lag64, double>(s, H, Nx, Ny, Nz, nt, Lx, Ly, Lz, x, y, z, vx, vy, vz, q, qconst,
                                           n_tracks, n_steps, n_out, dt, v_w, lags, nu, out);
}
// Eq. 1 straight from the rank-r form of the FP32 field, H[t][c][p] = sum_m W[t][m] E[c][m][p]
// (the representation the tensor-core expansion writes out): the staged dot products are
// W(x_j, t_n) . v_j = sum_m W[t_n][m] (E_m(x_j) . v_j), the interpolation being linear, so per
// track step the r basis fields are interpolated once instead of the field at every time
// sample (r x 24 gathers from E instead of n_t x 24 from H).  Lags, accumulation and currents
// as in eq1_kernel.  The basis fields are read point-major, Ep[p][c][32] (eq1_point_major): one
// warp per track step, a lane per basis field, so that each of the 24 corner-component reads is
// one 128-byte line, and the two z neighbours of a corner are adjacent lines.
// f[j][n] = sum_m W[t_n][m] sv[m][j] for n < nu, j < mc: NB time samples (nq apart, so that a warp
// reads consecutive words of Wt) by four steps per thread; Wt rows hold NB nq >= nu samples, the
// ones past nu zero.
template <int NB>
__device__ __forceinline__ void eq1_stage_product(const float* __restrict__ sv, const float* __restrict__ Wt, int r,
                                                  int nq, int nu, int mc, float* __restrict__ f) {
    const int ng = (mc + 3) >> 2, ldw = NB * nq;
    for (int e = threadIdx.x; e < nq * ng; e += blockDim.x) {
        const int n0 = e % nq, j0 = 4 * (e / nq);
        float acc[NB][4] = {};
        for (int m = 0; m < r; ++m) {
            const float4 s4 = *reinterpret_cast<const float4*>(sv + m * EQ1_MC + j0);
            const float* wr = Wt + (size_t)m * ldw + n0;
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const float wv = wr[i * nq];
                acc[i][0] = fmaf(wv, s4.x, acc[i][0]);
                acc[i][1] = fmaf(wv, s4.y, acc[i][1]);
                acc[i][2] = fmaf(wv, s4.z, acc[i][2]);
                acc[i][3] = fmaf(wv, s4.w, acc[i][3]);
            }
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int n = n0 + i * nq;
            if (n >= nu) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < mc) f[(j0 + q) * nu + n] = acc[i][q];
        }
    }
}

__global__ void __launch_bounds__(256) eq1_basis_kernel(const float* __restrict__ Ep, int r,
                                                        const float* __restrict__ W32, int Nx, int Ny, int Nz,
                                                        int nt, int nu, float inv_hx, float inv_hy,
                                                        float inv_hz,
                                                        const float* __restrict__ X, const float* __restrict__ Y,
                                                        const float* __restrict__ Z, const float* __restrict__ VX,
                                                        const float* __restrict__ VY, const float* __restrict__ VZ,
                                                        const float* __restrict__ qtrack, float qconst, int n_steps,
                                                        int n_out, double dt, double inv_vw, int nb,
                                                        bool stage_lags, const Eq1Lag* __restrict__ lags,
                                                        float* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sv = reinterpret_cast<float*>(smem_raw);                          // [32][EQ1_MC] (basis-major)
    float* Wt = sv + 32 * EQ1_MC;                                            // [r][ldw]
    const int nq = (nu + nb - 1) / nb, ldw = nb * nq;                        // Wt row: nu samples, zero-padded
    float* f = Wt + (size_t)r * ldw;                                         // [EQ1_MC][nu]
    double* Q = reinterpret_cast<double*>(smem_raw + ((((size_t)r * ldw + EQ1_MC * 32 + (size_t)EQ1_MC * nu) *
                                                        sizeof(float) + 15) & ~(size_t)15));   // [n_out]
    Eq1Lag* ls = reinterpret_cast<Eq1Lag*>(Q + n_out);                       // [n_out] when staged
    if (stage_lags)
        for (int m = threadIdx.x; m < n_out; m += blockDim.x) ls[m] = lags[m];
    const Eq1Lag* lg = stage_lags ? ls : lags;
    const int tr = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int e = threadIdx.x; e < r * ldw; e += blockDim.x) {
        const int m = e / ldw, n = e - m * ldw;
        Wt[e] = n < nu ? W32[(size_t)n * 32 + m] : 0.f;
    }
    for (int m = threadIdx.x; m < n_out; m += blockDim.x) Q[m] = 0.0;
    for (int c0 = 0; c0 < n_steps; c0 += EQ1_MC) {
        const int mc = min(EQ1_MC, n_steps - c0);
        __syncthreads();
        for (int j = warp; j < mc; j += nwarps) {
            const size_t s = (size_t)tr * n_steps + c0 + j;
            const float vx = VX[s], vy = VY[s], vz = VZ[s];
            float acc = 0.f;
            if (vx != 0.f || vy != 0.f || vz != 0.f) {
                const float fx = X[s] * inv_hx, fy = Y[s] * inv_hy;
                float fz = Z[s] * inv_hz - 0.5f;
                fz = fz < 0.f ? 0.f : (fz > (float)(Nz - 1) ? (float)(Nz - 1) : fz);
                const float flx = floorf(fx), fly = floorf(fy);
                const int k0 = min((int)floorf(fz), Nz - 2);
                const float wx = fx - flx, wy = fy - fly, wz = fz - (float)k0;
                const int i0 = ((int)flx % Nx + Nx) % Nx, j0 = ((int)fly % Ny + Ny) % Ny;
                const int i1 = (i0 + 1) % Nx, j1 = (j0 + 1) % Ny;
                // 96 floats per point; the z neighbour is the next point
                const float* p00 = Ep + (((size_t)i0 * Ny + j0) * Nz + k0) * 96 + lane;
                const float* p01 = Ep + (((size_t)i0 * Ny + j1) * Nz + k0) * 96 + lane;
                const float* p10 = Ep + (((size_t)i1 * Ny + j0) * Nz + k0) * 96 + lane;
                const float* p11 = Ep + (((size_t)i1 * Ny + j1) * Nz + k0) * 96 + lane;
                float w[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int o = 32 * c;
                    const float v00 = (1.f - wz) * __ldg(p00 + o) + wz * __ldg(p00 + 96 + o);
                    const float v01 = (1.f - wz) * __ldg(p01 + o) + wz * __ldg(p01 + 96 + o);
                    const float v10 = (1.f - wz) * __ldg(p10 + o) + wz * __ldg(p10 + 96 + o);
                    const float v11 = (1.f - wz) * __ldg(p11 + o) + wz * __ldg(p11 + 96 + o);
                    w[c] = (1.f - wx) * ((1.f - wy) * v00 + wy * v01) + wx * ((1.f - wy) * v10 + wy * v11);
                }
                acc = w[0] * vx + w[1] * vy + w[2] * vz;
            }
            sv[lane * EQ1_MC + j] = lane < r ? acc : 0.f;
        }
        __syncthreads();
        switch (nb) {
            case 1: eq1_stage_product<1>(sv, Wt, r, nq, nu, mc, f); break;
            case 2: eq1_stage_product<2>(sv, Wt, r, nq, nu, mc, f); break;
            case 3: eq1_stage_product<3>(sv, Wt, r, nq, nu, mc, f); break;
            default: eq1_stage_product<4>(sv, Wt, r, nq, nu, mc, f); break;
        }
        __syncthreads();
        eq1_increments(f, nu, mc, c0, n_out, lg, Q);
    }
    __syncthreads();
    const float qc = qtrack ? qtrack[tr] : qconst;
    for (int m = threadIdx.x; m < n_out; m += blockDim.x)
        out[(size_t)tr * n_out + m] = (float)(-(double)qc * inv_vw * Q[m]);
}

// Point-major copy of the basis fields for eq1_basis_kernel: Ep[p][c][m] = E[c][m][p] for m < r, 0 for
// r <= m < 32 (E: [3][32][npts], rows m >= r need not be written).  A block moves a tile of 32 points x
// 96 rows through shared memory: coalesced 128-byte row reads, one contiguous 12 KB write.
__global__ void __launch_bounds__(256) eq1_point_major_kernel(const float* __restrict__ E, int r, size_t npts,
                                                              float* __restrict__ Ep) {
    __shared__ float tile[96][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t ntiles = (npts + 31) / 32;
    for (size_t tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const size_t p0 = tb * 32;
        const size_t p = p0 + lane;
        for (int row = warp; row < 96; row += 8) {
            const int m = row & 31;
            tile[row][lane] = (m < r && p < npts) ? __ldg(E + (size_t)row * npts + p) : 0.f;
        }
        __syncthreads();
        const int np = (int)min((size_t)32, npts - p0);
        float* o = Ep + p0 * 96;
        for (int e = threadIdx.x; e < np * 96; e += 256) o[e] = tile[e % 96][e / 96];
        __syncthreads();
    }
}

void eq1_point_major(cudaStream_t s, const float* E, int r, size_t npts, float* Ep) {
    if (npts == 0) return;
    int dev = 0, num_sms = 0;
    WT_CUDA(cudaGetDevice(&dev));
    WT_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t ntiles = (npts + 31) / 32;
    const int grid = (int)std::min<size_t>(ntiles, (size_t)num_sms * 8);
    eq1_point_major_kernel<<<grid, 256, 0, s>>>(E, r, npts, Ep);
    WT_LAUNCH("eq1_point_major");
}

void eq1_basis_launch(cudaStream_t s, const float* Ep, int r, const float* W32, int Nx, int Ny, int Nz, int nt,
                      double Lx, double Ly, double Lz, const float* x, const float* y, const float* z,
                      const float* vx, const float* vy, const float* vz, const float* q, float qconst, int n_tracks,
                      int n_steps, int n_out, double dt, double v_w, const void* lags, int nu, float* out) {
    if (r < 1 || r > 32) fail(WT_ERR_ARG, "eq1: basis rank out of range");
    if (nu < 1 || nu > nt) fail(WT_ERR_ARG, "eq1: bad count of time samples in use");
    // time samples per thread in the staged product: the fewest that keep the (samples / nb) x
    // (steps / 4) items within one pass of the 256 threads
    const int nb = std::min(4, std::max(1, (nu + 63) / 64));
    const size_t ldw = (size_t)nb * ((nu + nb - 1) / nb);
    const size_t base = ((((size_t)r * ldw + EQ1_MC * 32 + (size_t)EQ1_MC * nu) * sizeof(float) + 15) & ~(size_t)15) +
                        (size_t)n_out * sizeof(double);
    // the lag table goes into shared memory beside the rest when it is small (12 B per output)
    const bool stage_lags = (size_t)n_out * sizeof(Eq1Lag) <= 16384;
    const size_t sh = base + (stage_lags ? (size_t)n_out * sizeof(Eq1Lag) : 0);
    if (sh > 200 * 1024) fail(WT_ERR_UNSUPPORTED, "eq1: n_t or n_out too large for shared memory");
    allow_dyn_smem(eq1_basis_kernel, sh);
    if (n_tracks > 0)
        eq1_basis_kernel<<<n_tracks, 256, sh, s>>>(Ep, r, W32, Nx, Ny, Nz, nt, nu, (float)(Nx / Lx), (float)(Ny / Ly),
                                                   (float)(Nz / Lz), x, y, z, vx, vy, vz, q, qconst, n_steps, n_out,
                                                   dt, 1.0 / v_w, nb, stage_lags, static_cast<const Eq1Lag*>(lags),
                                                   out);
    WT_LAUNCH("eq1_basis");
}

size_t eq1_lag_size() { return sizeof(Eq1Lag); }
void eq1_pack_lag(void* dst, int n, float w0, float w1) { *static_cast<Eq1Lag*>(dst) = Eq1Lag{n, w0, w1}; }
size_t eq1_lag64_size() { return sizeof(Eq1Lag64); }
void eq1_pack_lag64(void* dst, int n, double w0, double w1) { *static_cast<Eq1Lag64*>(dst) = Eq1Lag64{n, w0, w1}; }

// ------------------------------------------------------------------------
// Allocation-free variant (wt_eq1_noalloc).  The per-call lag table lives in
// this fixed device array instead of a cudaMalloc'd buffer; every GPU that
// loads the library holds it (12 B x WT_EQ1_NOALLOC_MAX_OUT = 192 KB) until the
// process exits.  The limit is the one the header documents.
constexpr int kEq1NoAllocMaxOut = WT_EQ1_NOALLOC_MAX_OUT;
static __device__ __align__(256) Eq1Lag g_eq1_lag_scratch[kEq1NoAllocMaxOut];

// Lag table on the device from the relaxation's time samples: same rule as
// the host-built table of eq1_launch's callers (linear in t, 0 at t = 0,
// held after the last sample).  Every entry is overwritten on each call.
__global__ void eq1_lag_table_kernel(const double* __restrict__ t, int nt, double dt, int n_out,
                                     Eq1Lag* __restrict__ lags) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_out) return;
    const double L = (k + 0.5) * dt;
    int n0 = 0;
    double w0 = 0.0, w1 = 0.0;
    if (L <= t[0]) { n0 = 0; w0 = L / t[0]; }
    else if (L >= t[nt - 1]) { n0 = nt - 1; w0 = 1.0; }
    else {
        int lo = 0, hi = nt - 1;           // t[lo] <= L < t[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (t[mid] <= L) lo = mid; else hi = mid;
        }
        n0 = lo;
        const double f = (L - t[lo]) / (t[lo + 1] - t[lo]);
        w0 = 1.0 - f;
        w1 = f;
    }
    lags[k] = Eq1Lag{n0, (float)w0, (float)w1};
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
// Device address of the scratch per device, and the id of the CUDA context it
// was looked up in: a context created anew on the device (after a
// cudaDeviceReset, say) reloads the module, so the address is looked up again.
struct ScratchAddr {
    Eq1Lag* p = nullptr;
    unsigned long long ctx_id = 0;
};
ScratchAddr g_noalloc_addr[kMaxDevices];

// id of the current CUDA context (unique for the life of the process), through
// the runtime's driver entry points (no libcuda link)
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    if (!get_cur || !get_id) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        WT_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 4000, cudaEnableDefault, &qa));
        WT_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb));
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            fail(WT_ERR_CUDA, "cuCtxGetCurrent / cuCtxGetId unavailable");
        get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(a);
        get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(b);
    }
    CUcontext cx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&cx) != CUDA_SUCCESS || !cx || get_id(cx, &id) != CUDA_SUCCESS)
        fail(WT_ERR_CUDA, "no current CUDA context for the allocation-free scratch");
    return id;
}
}  // namespace

// The caller's device is current.  Resolves the scratch address on the first
// call in this device's current context (the symbol's host-side name is not a
// device address); later calls in the same context reuse it.
void eq1_noalloc_launch(cudaStream_t s, int device, const float* H, int Nx, int Ny, int Nz, const double* d_times,
                        int nt, double Lx, double Ly, double Lz, const float* x, const float* y, const float* z,
                        const float* vx, const float* vy, const float* vz, const float* q, float qconst,
                        int n_tracks, int n_steps, int n_out, double dt, double v_w, int nu, float* out) {
    if (n_out > kEq1NoAllocMaxOut)
        fail(WT_ERR_ARG, "n_out " + std::to_string(n_out) + " exceeds the allocation-free limit of " +
                             std::to_string(kEq1NoAllocMaxOut));
    if (device < 0 || device >= kMaxDevices) fail(WT_ERR_UNSUPPORTED, "device index beyond the scratch table");
    Eq1Lag* lags = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        const unsigned long long id = current_context_id();
        ScratchAddr& a = g_noalloc_addr[device];
        if (!a.p || a.ctx_id != id) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_eq1_lag_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                fail(WT_ERR_CUDA, std::string("cudaGetSymbolAddress(eq1 scratch): ") + cudaGetErrorString(e));
            }
            a.p = static_cast<Eq1Lag*>(p);
            a.ctx_id = id;
        }
        lags = a.p;
    }
    eq1_lag_table_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(d_times, nt, dt, n_out, lags);
    WT_LAUNCH("eq1_lag_table");
    eq1_launch(s, H, Nx, Ny, Nz, nt, Lx, Ly, Lz, x, y, z, vx, vy, vz, q, qconst, n_tracks, n_steps, n_out, dt, v_w,
               lags, nu, out);
}

}  // namespace wt
