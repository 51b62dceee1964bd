// Symmetric eigendecomposition for the relaxation modes (the quasi-static
// relaxation of Sec. 3, solved exactly through its modes): FP64 throughout.
//
//   1. Householder tridiagonalisation Y = Q T Q^T, one reflector per column:
//      H_k = I - tau_k u_k u_k^T with u_k = [0 (k + 1 entries); v_k],
//      v_k[0] = 1.  Per step: the reflector (one block), p = tau A22 v (one
//      warp per row), w = p - (tau p.v / 2) v (one block), and the rank-two
//      update A22 -= v w^T + w v^T, both products rounded before the sum so
//      that A stays exactly symmetric.  v_k is kept in row k of A.
//   2. Divide and conquer on T (Cuppen's splitting): T = diag(T1', T2') +
//      |rho| s s^T with rho the coupling at the split, s = [e_last; sign(rho)
//      e_first] and T1', T2' the halves with |rho| taken off the touching
//      diagonal entries.  Leaves (<= 32 rows) by implicit QL with Wilkinson
//      shifts, one warp each.  A merge turns the halves' eigen-
//      decompositions into that of D + r z z^T (r = 2|rho|, |z| = 1):
//      deflation of negligible z entries and of close pairs of D (a Givens
//      rotation zeroes one z entry), the roots of the secular equation
//      1 + r sum_i z_i^2 / (d_i - lambda) = 0 (one thread per root, each root
//      held as the offset tau from its nearer pole so that every difference
//      d_i - lambda is formed without cancellation), the update vector
//      recomputed from the roots by Loewner's formula (Gu and Eisenstat), so
//      that the eigenvectors z^_i / (d_i - lambda_j) come out orthogonal to
//      working precision, and one GEMM per merge for the new eigenvectors.
//   3. Back-transformation V = H_0 H_1 ... H_{n-3} Z in blocks of 32
//      reflectors (compact WY form I - W T W^T, three GEMMs per block).
#include "wt_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace wt {

namespace {

constexpr int kLeaf = 32;       // largest leaf of the divide-and-conquer tree
constexpr int kWyBlock = 32;    // reflectors per back-transformation block
constexpr double kEps = 2.220446049250313e-16;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (blockDim.x a multiple of 32); every thread gets the result.
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        t = warp_sum(t);
        if (l == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// ------------------------------------------------------ tridiagonalisation
// Reflector of step k from x = A[k][k+1 ..] (row k equals column k): H x = beta e_0.
__global__ void __launch_bounds__(1024) trd_house_kernel(double* A, int n, int k, double* vk, double* d, double* e,
                                                        double* tau) {
    __shared__ double sh[33];
    const int m = n - k - 1;
    double* row = A + (size_t)k * n + k + 1;
    double ss = 0.0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) ss = fma(row[i], row[i], ss);
    ss = block_sum(ss, sh);
    const double x0 = row[0];
    double t = 0.0, beta = x0, scale = 0.0;
    if (ss > 0.0) {
        beta = -copysign(sqrt(fma(x0, x0, ss)), x0);
        t = (beta - x0) / beta;
        scale = 1.0 / (x0 - beta);
    }
    __syncthreads();                      // x0 read everywhere before row[0] is replaced
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double v = i == 0 ? 1.0 : row[i] * scale;
        vk[i] = v;
        row[i] = v;
    }
    if (threadIdx.x == 0) {
        d[k] = A[(size_t)k * n + k];
        e[k] = beta;
        tau[k] = t;
    }
}

// p = tau A22 v, one warp per row of the trailing block.
__global__ void __launch_bounds__(256) trd_symv_kernel(const double* __restrict__ A, int n, int k,
                                                      const double* __restrict__ v, const double* __restrict__ tau,
                                                      double* __restrict__ p) {
    const int m = n - k - 1;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= m) return;
    const double* row = A + (size_t)(k + 1 + i) * n + k + 1;
    double acc = 0.0;
    for (int j = lane; j < m; j += 32) acc = fma(row[j], v[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) p[i] = tau[k] * acc;
}

// w = p - (tau (p . v) / 2) v, in place on p (one block).
__global__ void __launch_bounds__(1024) trd_w_kernel(int n, int k, const double* __restrict__ v,
                                                    const double* __restrict__ tau, double* __restrict__ p) {
    __shared__ double sh[33];
    const int m = n - k - 1;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s = fma(p[i], v[i], s);
    s = block_sum(s, sh);
    const double a = 0.5 * tau[k] * s;
    for (int i = threadIdx.x; i < m; i += blockDim.x) p[i] = fma(-a, v[i], p[i]);
}

// A22 -= v w^T + w v^T; four rows per block row.
__global__ void __launch_bounds__(256) trd_syr2_kernel(double* __restrict__ A, int n, int k,
                                                      const double* __restrict__ v, const double* __restrict__ w) {
    const int m = n - k - 1;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double vj = v[j], wj = w[j];
    const int i1 = min(m, (int)blockIdx.y * 4 + 4);
    for (int i = blockIdx.y * 4; i < i1; ++i) {
        double* a = A + (size_t)(k + 1 + i) * n + k + 1 + j;
        const double t = __dadd_rn(__dmul_rn(v[i], wj), __dmul_rn(w[i], vj));
        *a = __dsub_rn(*a, t);
    }
}

__global__ void trd_tail_kernel(const double* A, int n, double* d, double* e, double* tau) {
    if (threadIdx.x) return;
    if (n >= 2) {
        d[n - 2] = A[(size_t)(n - 2) * n + n - 2];
        e[n - 2] = A[(size_t)(n - 2) * n + n - 1];
        tau[n - 2] = 0.0;
    }
    d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
    e[n - 1] = 0.0;
    tau[n - 1] = 0.0;
}

// Small matrices (n <= kSmallTrd) in one block: the same four steps per column on a copy of A in
// shared memory (rows of pitch n), then A (reflectors in its rows), d, e, tau written back.
constexpr int kSmallTrd = 96;
__global__ void __launch_bounds__(1024) trd_small_kernel(double* A, int n, double* d, double* e, double* tau) {
    extern __shared__ double sm[];
    double* a = sm;                       // [n][n]
    double* v = a + (size_t)n * n;        // [n]
    double* p = v + n;                    // [n]
    __shared__ double red[33];
    __shared__ double par[3];             // tau, beta, scale
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) a[i] = A[i];
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double* row = a + (size_t)k * n + k + 1;
        double ss = 0.0;
        for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) ss = fma(row[i], row[i], ss);
        ss = block_sum(ss, red);
        if (threadIdx.x == 0) {
            const double x0 = row[0];
            double t = 0.0, beta = x0, scale = 0.0;
            if (ss > 0.0) {
                beta = -copysign(sqrt(fma(x0, x0, ss)), x0);
                t = (beta - x0) / beta;
                scale = 1.0 / (x0 - beta);
            }
            par[0] = t;
            par[1] = beta;
            par[2] = scale;
            d[k] = a[(size_t)k * n + k];
            e[k] = beta;
            tau[k] = t;
        }
        __syncthreads();
        const double t = par[0], scale = par[2];
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double vi = i == 0 ? 1.0 : row[i] * scale;
            v[i] = vi;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) row[i] = v[i];
        // p = tau A22 v, one thread per row
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double* r = a + (size_t)(k + 1 + i) * n + k + 1;
            double acc = 0.0;
            for (int j = 0; j < m; ++j) acc = fma(r[j], v[j], acc);
            p[i] = t * acc;
        }
        __syncthreads();
        double sv = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) sv = fma(p[i], v[i], sv);
        sv = block_sum(sv, red);
        const double al = 0.5 * t * sv;
        for (int i = threadIdx.x; i < m; i += blockDim.x) p[i] = fma(-al, v[i], p[i]);
        __syncthreads();
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int i = idx / m, j = idx % m;
            double* x = a + (size_t)(k + 1 + i) * n + k + 1 + j;
            *x = __dsub_rn(*x, __dadd_rn(__dmul_rn(v[i], p[j]), __dmul_rn(p[i], v[j])));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (n >= 2) {
            d[n - 2] = a[(size_t)(n - 2) * n + n - 2];
            e[n - 2] = a[(size_t)(n - 2) * n + n - 1];
            tau[n - 2] = 0.0;
        }
        d[n - 1] = a[(size_t)(n - 1) * n + n - 1];
        e[n - 1] = 0.0;
        tau[n - 1] = 0.0;
    }
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) A[i] = a[i];
}

// ------------------------------------------------------- divide and conquer
// Take |rho| off the diagonal entries on both sides of every split (one thread, in order).
__global__ void dc_split_kernel(double* d, const double* e, const int* splits, int n_splits) {
    if (threadIdx.x || blockIdx.x) return;
    for (int q = 0; q < n_splits; ++q) {
        const int s = splits[q];
        const double a = fabs(e[s - 1]);
        d[s - 1] -= a;
        d[s] -= a;
    }
}

// One warp per leaf: implicit QL with Wilkinson shifts (lane 0 runs the recurrence and records
// each sweep's rotations), all lanes rotate their rows of the leaf's eigenvector matrix.
// Output sorted ascending: lam[l0 + j], Q[(l0 + i) n + l0 + j].
__global__ void __launch_bounds__(128) dc_leaf_kernel(const double* __restrict__ d, const double* __restrict__ e,
                                                      const int* __restrict__ starts, int n_leaves, int n,
                                                      double* __restrict__ lam, double* __restrict__ Q, int* err) {
    __shared__ double Zs[4][kLeaf][kLeaf + 1];
    __shared__ double dd[4][kLeaf], ee[4][kLeaf], rc[4][kLeaf], rs[4][kLeaf];
    __shared__ int ctl[4][4];
    __shared__ int perm[4][kLeaf];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int leaf = blockIdx.x * 4 + w;
    if (leaf >= n_leaves) return;
    const int l0 = starts[leaf], K = starts[leaf + 1] - l0;
    double (*Z)[kLeaf + 1] = Zs[w];
    for (int j = 0; j < K; ++j) Z[lane][j] = (lane == j) ? 1.0 : 0.0;
    if (lane < K) {
        dd[w][lane] = d[l0 + lane];
        ee[w][lane] = lane < K - 1 ? e[l0 + lane] : 0.0;
    }
    __syncwarp();
    for (int l = 0; l < K; ++l) {
        int iter = 0;
        while (true) {
            if (lane == 0) {
                double* D = dd[w];
                double* E = ee[w];
                int m = l;
                for (; m < K - 1; ++m) {
                    const double s = fabs(D[m]) + fabs(D[m + 1]);
                    if (fabs(E[m]) <= kEps * s) break;
                }
                int lo = 0, hi = -1, done = (m == l);
                if (!done && ++iter > 60) {
                    atomicMax(err, (int)DERR_TIMEOUT);
                    done = 1;
                }
                if (!done) {
                    double g = (D[l + 1] - D[l]) / (2.0 * E[l]);
                    double r = hypot(g, 1.0);
                    g = D[m] - D[l] + E[l] / (g + copysign(r, g));
                    double s = 1.0, c = 1.0, p = 0.0;
                    int i = m - 1;
                    bool under = false;
                    for (; i >= l; --i) {
                        const double f = s * E[i], b = c * E[i];
                        r = hypot(f, g);
                        E[i + 1] = r;
                        if (r == 0.0) {
                            D[i + 1] -= p;
                            E[m] = 0.0;
                            under = true;
                            break;
                        }
                        s = f / r;
                        c = g / r;
                        g = D[i + 1] - p;
                        r = (D[i] - g) * s + 2.0 * c * b;
                        p = s * r;
                        D[i + 1] = g + p;
                        g = c * r - b;
                        rc[w][i] = c;
                        rs[w][i] = s;
                    }
                    if (!under) {
                        D[l] -= p;
                        E[l] = g;
                        E[m] = 0.0;
                    }
                    lo = under ? i + 1 : l;
                    hi = m - 1;
                }
                ctl[w][0] = done;
                ctl[w][1] = lo;
                ctl[w][2] = hi;
            }
            __syncwarp();
            const int done = ctl[w][0], lo = ctl[w][1], hi = ctl[w][2];
            if (done) break;
            if (lane < K)
                for (int i = hi; i >= lo; --i) {
                    const double c = rc[w][i], s = rs[w][i];
                    const double f = Z[lane][i + 1];
                    Z[lane][i + 1] = s * Z[lane][i] + c * f;
                    Z[lane][i] = c * Z[lane][i] - s * f;
                }
            __syncwarp();
        }
        __syncwarp();
    }
    if (lane == 0) {                      // ascending order (selection sort, K <= 32)
        for (int j = 0; j < K; ++j) perm[w][j] = j;
        for (int j = 0; j < K; ++j) {
            int b = j;
            for (int q = j + 1; q < K; ++q)
                if (dd[w][perm[w][q]] < dd[w][perm[w][b]]) b = q;
            const int t = perm[w][j];
            perm[w][j] = perm[w][b];
            perm[w][b] = t;
        }
    }
    __syncwarp();
    if (lane < K) {
        lam[l0 + lane] = dd[w][perm[w][lane]];
        for (int j = 0; j < K; ++j) Q[(size_t)(l0 + lane) * n + l0 + j] = Z[lane][perm[w][j]];
    }
}

// Per-merge scratch, all arrays indexed from the node's first row l.
struct DcWork {
    int* perm;        // sorted position -> index in the node (0 .. K-1)
    int* fcol;        // sorted position -> column of the gathered matrix ([non-deflated | deflated])
    int* rot_p;       // Givens rotations on gathered columns, in order
    int* rot_i;
    double* rot_c;
    double* rot_s;
    double* ds;       // sorted (and rotated) diagonal; deflated eigenvalues at their sorted positions
    double* delta;    // non-deflated poles (ascending), [Kp]
    double* zeta;     // their update vector entries
    int* org;         // root j: index of its pole of origin
    double* tau;      // root j: lambda_j - delta[org_j]
    double* zh;       // Loewner update vector
    double* root;     // lambda_j
    double* defl_val; // deflated eigenvalues in gathered-column order (column Kp + q)
    int* oper;        // final order: output column j <- gathered column oper[j]
    double* lam_out;
    int* node_kp;     // per node
    int* node_nrot;
    double* node_r;
};

struct DcNode {
    int l, mid, r;
};

// One block per merge node: the rank-one update vector, the merged order, deflation (thread 0,
// sequential over the sorted entries) and the compaction of the non-deflated poles.
__global__ void __launch_bounds__(256) dc_prep_kernel(const DcNode* __restrict__ nodes, const double* __restrict__ e,
                                                      const double* __restrict__ lamA, const double* __restrict__ QA,
                                                      int n, DcWork W, double* zbuf) {
    const DcNode nd = nodes[blockIdx.x];
    const int l = nd.l, K = nd.r - nd.l, K1 = nd.mid - nd.l;
    const double rho = e[nd.mid - 1];
    const double sg = rho < 0.0 ? -1.0 : 1.0;
    const double inv_sqrt2 = 0.70710678118654752440;
    double* z = zbuf + l;
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        z[i] = inv_sqrt2 * (i < K1 ? QA[(size_t)(nd.mid - 1) * n + l + i] : sg * QA[(size_t)nd.mid * n + l + i]);
    __syncthreads();
    if (threadIdx.x) return;
    const double r = 2.0 * fabs(rho);
    int* perm = W.perm + l;
    double* ds = W.ds + l;
    // merge the two ascending halves
    {
        int a = 0, b = K1, q = 0;
        while (a < K1 || b < K) {
            const bool ta = b >= K || (a < K1 && lamA[l + a] <= lamA[l + b]);
            perm[q++] = ta ? a++ : b++;
        }
    }
    double dmax = 0.0;
    for (int q = 0; q < K; ++q) {
        ds[q] = lamA[l + perm[q]];
        dmax = fmax(dmax, fabs(ds[q]));
    }
    const double tol = 8.0 * kEps * fmax(dmax, r);
    // deflation: zs kept in zbuf at sorted positions from here on (reuse: z is read through perm)
    double* zs = W.zh + l;                 // scratch until the Loewner pass overwrites it
    for (int q = 0; q < K; ++q) zs[q] = z[perm[q]];
    unsigned char* flag = reinterpret_cast<unsigned char*>(W.fcol + l);   // temporary: 1 = deflated
    for (int q = 0; q < K; ++q) flag[q] = 0;
    int nrot = 0, p = -1;
    for (int q = 0; q < K; ++q) {
        if (r * fabs(zs[q]) <= tol) {
            flag[q] = 1;
            continue;
        }
        if (p >= 0) {
            const double x = zs[p], y = zs[q];
            const double t = hypot(x, y);
            const double c = y / t, s = x / t;
            const double off = c * s * (ds[p] - ds[q]);
            if (fabs(off) <= tol) {
                const double a = ds[p], b = ds[q];
                ds[p] = c * c * a + s * s * b;
                ds[q] = s * s * a + c * c * b;
                zs[p] = 0.0;
                zs[q] = t;
                flag[p] = 1;
                W.rot_p[l + nrot] = p;
                W.rot_i[l + nrot] = q;
                W.rot_c[l + nrot] = c;
                W.rot_s[l + nrot] = s;
                ++nrot;
            }
        }
        p = q;
    }
    // compaction: non-deflated first (ascending), then deflated
    int kp = 0;
    for (int q = 0; q < K; ++q)
        if (!flag[q]) ++kp;
    int a = 0, b = kp;
    double* delta = W.delta + l;
    double* zeta = W.zeta + l;
    double* dv = W.defl_val + l;
    // flag lives in fcol's storage: read it all before fcol is written
    for (int q = 0; q < K; ++q) {
        if (!flag[q]) {
            delta[a] = ds[q];
            zeta[a] = zs[q];
            W.org[l + q] = a++;          // temporary: sorted position -> gathered column
        } else {
            dv[b - kp] = ds[q];
            W.org[l + q] = b++;
        }
    }
    for (int q = 0; q < K; ++q) W.fcol[l + q] = W.org[l + q];
    W.node_kp[blockIdx.x] = kp;
    W.node_nrot[blockIdx.x] = nrot;
    W.node_r[blockIdx.x] = r;
}

// f(tau) = 1 + r sum_i zeta_i^2 / ((delta_i - delta_org) - tau) and its derivative, summed by the
// 32 lanes of a warp (lane k takes the poles k, k + 32, ...).  The xor butterfly gives every lane
// the same bits, so the iteration that uses them stays uniform across the warp.
__device__ __forceinline__ void secular_f(const double* __restrict__ delta, const double* __restrict__ zeta, int kp,
                                          double dorg, double r, double tau, double* f, double* fp) {
    double s = 0.0, sp = 0.0;
    for (int i = threadIdx.x & 31; i < kp; i += 32) {
        const double q = 1.0 / ((delta[i] - dorg) - tau);
        const double z2 = zeta[i] * zeta[i];
        s = fma(z2, q, s);
        sp = fma(z2 * q, q, sp);
    }
    s = warp_sum(s);
    sp = warp_sum(sp);
    *f = fma(r, s, 1.0);
    *fp = r * sp;
}

// One warp per root (eight per block): bracket between the poles, Newton steps kept inside the
// bracket, else bisection; stops when the bracket is at the rounding level of tau.
__global__ void __launch_bounds__(256) dc_secular_kernel(const DcNode* __restrict__ nodes, DcWork W) {
    const DcNode nd = nodes[blockIdx.y];
    const int l = nd.l, kp = W.node_kp[blockIdx.y];
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= kp) return;                 // whole warps leave together
    const double r = W.node_r[blockIdx.y];
    const double* delta = W.delta + l;
    const double* zeta = W.zeta + l;
    int org;
    double lo, hi;
    if (j < kp - 1) {
        const double gap = delta[j + 1] - delta[j];
        double f, fp;
        secular_f(delta, zeta, kp, delta[j], r, 0.5 * gap, &f, &fp);
        if (f > 0.0) { org = j; lo = 0.0; hi = 0.5 * gap; }
        else { org = j + 1; lo = -0.5 * gap; hi = 0.0; }
    } else {
        double zz = 0.0;
        for (int i = threadIdx.x & 31; i < kp; i += 32) zz = fma(zeta[i], zeta[i], zz);
        zz = warp_sum(zz);
        org = j;
        lo = 0.0;
        hi = r * zz;
    }
    const double dorg = delta[org];
    double t = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double f, fp;
        secular_f(delta, zeta, kp, dorg, r, t, &f, &fp);
        if (f == 0.0) { lo = hi = t; break; }
        if (f > 0.0) hi = t; else lo = t;
        const double w = hi - lo;
        if (w <= 4.0 * kEps * fmax(fabs(lo), fabs(hi))) break;
        double tn = t - f / fp;
        if (!(tn > lo && tn < hi) || (fabs(tn - t) > 0.5 * w && it > 2)) tn = 0.5 * (lo + hi);
        // converged: the step is at the rounding level of tau (Newton may otherwise alternate
        // between neighbouring values until the iteration limit)
        if (fabs(tn - t) <= 2.0 * kEps * fabs(t)) { t = tn; break; }
        t = tn;
    }
    if ((threadIdx.x & 31) == 0) {
        W.org[l + j] = org;
        W.tau[l + j] = t;
        W.root[l + j] = dorg + t;
    }
}

// Loewner's formula: zh_i^2 = (lambda_last - delta_i) / r  prod_{j < i} (lambda_j - delta_i) / (delta_j - delta_i)
//                              prod_{i <= j < last} (lambda_j - delta_i) / (delta_{j+1} - delta_i)
__global__ void __launch_bounds__(128) dc_loewner_kernel(const DcNode* __restrict__ nodes, DcWork W) {
    const DcNode nd = nodes[blockIdx.y];
    const int l = nd.l, kp = W.node_kp[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kp) return;
    const double r = W.node_r[blockIdx.y];
    const double* delta = W.delta + l;
    const int* org = W.org + l;
    const double* tau = W.tau + l;
    const double di = delta[i];
    double acc = ((delta[org[kp - 1]] - di) + tau[kp - 1]) / r;
    for (int j = 0; j < kp - 1; ++j) {
        const double num = (delta[org[j]] - di) + tau[j];
        const double den = j < i ? delta[j] - di : delta[j + 1] - di;
        acc *= num / den;
    }
    W.zh[l + i] = copysign(sqrt(fmax(acc, 0.0)), W.zeta[l + i]);
}

// Eigenvectors of D + r z z^T: column j = zh / (delta - lambda_j), normalised; written as rows of
// WT (WT[j][i]) for the GEMM.  One warp per root.
__global__ void __launch_bounds__(256) dc_vec_kernel(const DcNode* __restrict__ nodes, DcWork W, int n,
                                                     double* __restrict__ WT) {
    const DcNode nd = nodes[blockIdx.y];
    const int l = nd.l, kp = W.node_kp[blockIdx.y];
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= kp) return;
    const double* delta = W.delta + l;
    const double* zh = W.zh + l;
    const double dorg = delta[W.org[l + j]], t = W.tau[l + j];
    double ss = 0.0;
    for (int i = lane; i < kp; i += 32) {
        const double v = zh[i] / ((delta[i] - dorg) - t);
        ss = fma(v, v, ss);
    }
    ss = warp_sum(ss);
    const double inv = 1.0 / sqrt(ss);
    double* row = WT + (size_t)(l + j) * n + l;
    for (int i = lane; i < kp; i += 32) row[i] = inv * (zh[i] / ((delta[i] - dorg) - t));
}

// Gathered eigenvector matrix of the halves: G[row][fcol[q]] = QA[row][l + perm[q]], then the
// deflation rotations on its columns, in order.  One thread per row of the node.
__global__ void __launch_bounds__(128) dc_gather_kernel(const DcNode* __restrict__ nodes, DcWork W, int n,
                                                        const double* __restrict__ QA, double* __restrict__ G) {
    const DcNode nd = nodes[blockIdx.y];
    const int l = nd.l, K = nd.r - nd.l;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= K) return;
    const double* src = QA + (size_t)(l + row) * n + l;
    double* dst = G + (size_t)(l + row) * n + l;
    for (int q = 0; q < K; ++q) dst[W.fcol[l + q]] = src[W.perm[l + q]];
    const int nrot = W.node_nrot[blockIdx.y];
    for (int k = 0; k < nrot; ++k) {
        const int cp = W.fcol[l + W.rot_p[l + k]], ci = W.fcol[l + W.rot_i[l + k]];
        const double c = W.rot_c[l + k], s = W.rot_s[l + k];
        const double a = dst[cp], b = dst[ci];
        dst[cp] = c * a - s * b;
        dst[ci] = s * a + c * b;
    }
}

// Final order of a node's eigenvalues: roots (ascending) merged with the deflated values
// (insertion-sorted first: they arrive nearly in order).  Thread 0 per node.
__global__ void dc_order_kernel(const DcNode* __restrict__ nodes, DcWork W) {
    if (threadIdx.x) return;
    const DcNode nd = nodes[blockIdx.x];
    const int l = nd.l, K = nd.r - nd.l, kp = W.node_kp[blockIdx.x];
    const int nd_ = K - kp;
    double* dv = W.defl_val + l;
    int* idx = W.perm + l;                 // reused: deflated order (column offsets)
    for (int q = 0; q < nd_; ++q) idx[q] = q;
    for (int q = 1; q < nd_; ++q) {
        const int x = idx[q];
        const double v = dv[x];
        int p = q - 1;
        while (p >= 0 && dv[idx[p]] > v) {
            idx[p + 1] = idx[p];
            --p;
        }
        idx[p + 1] = x;
    }
    const double* root = W.root + l;
    int a = 0, b = 0, o = 0;
    while (a < kp || b < nd_) {
        const bool tr = b >= nd_ || (a < kp && root[a] <= dv[idx[b]]);
        if (tr) {
            W.lam_out[l + o] = root[a];
            W.oper[l + o] = a++;
        } else {
            W.lam_out[l + o] = dv[idx[b]];
            W.oper[l + o] = kp + idx[b++];
        }
        ++o;
    }
}

// QB[row][l + j] = X[row][l + oper[j]], one thread per (row, column chunk).
__global__ void __launch_bounds__(256) dc_permute_kernel(const DcNode* __restrict__ nodes, DcWork W, int n,
                                                         const double* __restrict__ X, double* __restrict__ QB,
                                                         double* __restrict__ lamB) {
    const DcNode nd = nodes[blockIdx.z];
    const int l = nd.l, K = nd.r - nd.l;
    const int j = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y;
    if (j >= K || row >= K) return;
    QB[(size_t)(l + row) * n + l + j] = X[(size_t)(l + row) * n + l + W.oper[l + j]];
    if (row == 0) lamB[l + j] = W.lam_out[l + j];
}

// ------------------------------------------------------- back-transformation
// Rows j of Wt (nb x n): u_{k0 + j} (zeros up to column k0 + j, then v_k from row k0 + j of A).
__global__ void wy_rows_kernel(const double* __restrict__ A, int n, int k0, int nb, double* __restrict__ Wt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (c >= n || j >= nb) return;
    const int k = k0 + j;
    Wt[(size_t)j * n + c] = c <= k ? 0.0 : A[(size_t)k * n + c];
}

// T (nb x nb, upper) of H_{k0} ... H_{k0+nb-1} = I - W T W^T from S = Wt Wt^T:
// T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] S[0:j, j].  One thread.
__global__ void wy_t_kernel(const double* __restrict__ S, const double* __restrict__ tau, int k0, int nb,
                            double* __restrict__ T) {
    if (threadIdx.x || blockIdx.x) return;
    for (int i = 0; i < nb * nb; ++i) T[i] = 0.0;
    for (int j = 0; j < nb; ++j) {
        const double tj = tau[k0 + j];
        for (int i = 0; i < j; ++i) {
            double acc = 0.0;
            for (int q = i; q < j; ++q) acc = fma(T[i * nb + q], S[q * nb + j], acc);
            T[i * nb + j] = -tj * acc;
        }
        T[j * nb + j] = tj;
    }
}

}  // namespace

// Eigendecomposition of the symmetric A (n x n row-major, destroyed): w ascending, V columns.
void sym_eig(cudaStream_t s, double* A, int n, double* w, double* V, int* d_err) {
    if (n <= 0) return;
    DBuf<double> d, e, tau, vk, p;
    d.alloc(n);
    e.alloc(n);
    tau.alloc(n);
    vk.alloc(n);
    p.alloc(n);
    // 1. tridiagonalisation (small matrices in one block)
    if (n <= kSmallTrd) {
        const size_t sh = ((size_t)n * n + 2 * (size_t)n) * sizeof(double);
        allow_dyn_smem(trd_small_kernel, sh);
        trd_small_kernel<<<1, 1024, sh, s>>>(A, n, d.p, e.p, tau.p);
    } else {
        for (int k = 0; k + 2 < n; ++k) {
            const int m = n - k - 1;
            trd_house_kernel<<<1, 1024, 0, s>>>(A, n, k, vk.p, d.p, e.p, tau.p);
            trd_symv_kernel<<<(m + 7) / 8, 256, 0, s>>>(A, n, k, vk.p, tau.p, p.p);
            trd_w_kernel<<<1, 1024, 0, s>>>(n, k, vk.p, tau.p, p.p);
            trd_syr2_kernel<<<dim3((m + 255) / 256, (m + 3) / 4), 256, 0, s>>>(A, n, k, vk.p, p.p);
        }
        trd_tail_kernel<<<1, 32, 0, s>>>(A, n, d.p, e.p, tau.p);
    }
    WT_LAUNCH("tridiagonalisation");
    vk.release();
    p.release();

    // 2. divide and conquer: tree by halving, leaves <= kLeaf rows
    std::vector<int> leaves;            // starts, plus n
    std::vector<std::vector<DcNode>> levels;
    std::vector<int> splits;
    struct Item { int l, r, depth; };
    std::vector<Item> stack{{0, n, 0}};
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        if (it.r - it.l <= kLeaf) {
            leaves.push_back(it.l);
            continue;
        }
        const int mid = it.l + (it.r - it.l) / 2;
        if ((int)levels.size() <= it.depth) levels.resize(it.depth + 1);
        levels[it.depth].push_back({it.l, mid, it.r});
        splits.push_back(mid);
        stack.push_back({it.l, mid, it.depth + 1});
        stack.push_back({mid, it.r, it.depth + 1});
    }
    std::sort(leaves.begin(), leaves.end());
    const int n_leaves = (int)leaves.size();
    leaves.push_back(n);
    DBuf<double> lamA, lamB, QA, QB, G;
    lamA.alloc(n);
    lamB.alloc(n);
    QA.alloc((size_t)n * n);
    QA.zero(s);
    if (!splits.empty()) {
        DBuf<int> dsp;
        dsp.upload(splits.data(), splits.size(), s);
        dc_split_kernel<<<1, 32, 0, s>>>(d.p, e.p, dsp.p, (int)splits.size());
        WT_LAUNCH("dc_split");
        WT_CUDA(cudaStreamSynchronize(s));
    }
    {
        DBuf<int> dst;
        dst.upload(leaves.data(), leaves.size(), s);
        dc_leaf_kernel<<<(n_leaves + 3) / 4, 128, 0, s>>>(d.p, e.p, dst.p, n_leaves, n, lamA.p, QA.p, d_err);
        WT_LAUNCH("dc_leaf");
        WT_CUDA(cudaStreamSynchronize(s));
    }
    if (!levels.empty()) {
        QB.alloc((size_t)n * n);
        G.alloc((size_t)n * n);
        QB.zero(s);
        DBuf<int> ibuf;
        DBuf<double> fbuf;
        ibuf.alloc((size_t)n * 8);
        fbuf.alloc((size_t)n * 12);
        DBuf<double> WT, zbuf;
        WT.alloc((size_t)n * n);
        zbuf.alloc(n);
        const size_t nn = n;
        DcWork Wk{};
        Wk.perm = ibuf.p;
        Wk.fcol = ibuf.p + nn;
        Wk.rot_p = ibuf.p + 2 * nn;
        Wk.rot_i = ibuf.p + 3 * nn;
        Wk.org = ibuf.p + 4 * nn;
        Wk.oper = ibuf.p + 5 * nn;
        Wk.node_kp = ibuf.p + 6 * nn;
        Wk.node_nrot = ibuf.p + 7 * nn;
        Wk.rot_c = fbuf.p;
        Wk.rot_s = fbuf.p + nn;
        Wk.ds = fbuf.p + 2 * nn;
        Wk.delta = fbuf.p + 3 * nn;
        Wk.zeta = fbuf.p + 4 * nn;
        Wk.tau = fbuf.p + 5 * nn;
        Wk.zh = fbuf.p + 6 * nn;
        Wk.root = fbuf.p + 7 * nn;
        Wk.defl_val = fbuf.p + 8 * nn;
        Wk.lam_out = fbuf.p + 9 * nn;
        Wk.node_r = fbuf.p + 10 * nn;
        DBuf<DcNode> dnodes;
        double *qa = QA.p, *qb = QB.p, *la = lamA.p, *lb = lamB.p;
        for (int lev = (int)levels.size() - 1; lev >= 0; --lev) {
            const std::vector<DcNode>& nodes = levels[lev];
            const int nn_ = (int)nodes.size();
            dnodes.upload(nodes.data(), nodes.size(), s);
            int kmax = 0;
            for (const DcNode& nd : nodes) kmax = std::max(kmax, nd.r - nd.l);
            dc_prep_kernel<<<nn_, 256, 0, s>>>(dnodes.p, e.p, la, qa, n, Wk, zbuf.p);
            WT_LAUNCH("dc_prep");
            dc_secular_kernel<<<dim3((kmax + 7) / 8, nn_), 256, 0, s>>>(dnodes.p, Wk);
            WT_LAUNCH("dc_secular");
            dc_loewner_kernel<<<dim3((kmax + 127) / 128, nn_), 128, 0, s>>>(dnodes.p, Wk);
            WT_LAUNCH("dc_loewner");
            dc_vec_kernel<<<dim3((kmax + 7) / 8, nn_), 256, 0, s>>>(dnodes.p, Wk, n, WT.p);
            WT_LAUNCH("dc_vec");
            dc_gather_kernel<<<dim3((kmax + 127) / 128, nn_), 128, 0, s>>>(dnodes.p, Wk, n, qa, G.p);
            WT_LAUNCH("dc_gather");
            std::vector<int> kp(nn_);
            WT_CUDA(cudaMemcpyAsync(kp.data(), Wk.node_kp, nn_ * sizeof(int), cudaMemcpyDeviceToHost, s));
            WT_CUDA(cudaStreamSynchronize(s));
            for (int q = 0; q < nn_; ++q) {
                const DcNode& nd = nodes[q];
                const int K = nd.r - nd.l, k1 = kp[q];
                const size_t off = (size_t)nd.l * n + nd.l;
                if (k1 > 0) dgemm(s, false, true, K, k1, k1, 1.0, G.p + off, n, WT.p + off, n, 0.0, qa + off, n);
                if (K > k1) copy_block(s, G.p + off + k1, n, qa + off + k1, n, K, K - k1);
            }
            dc_order_kernel<<<nn_, 32, 0, s>>>(dnodes.p, Wk);
            WT_LAUNCH("dc_order");
            dc_permute_kernel<<<dim3((kmax + 255) / 256, kmax, nn_), 256, 0, s>>>(dnodes.p, Wk, n, qa, qb, lb);
            WT_LAUNCH("dc_permute");
            // rows and eigenvalues of the leaves/nodes not merged at this level carry over
            WT_CUDA(cudaStreamSynchronize(s));
            std::swap(qa, qb);
            std::swap(la, lb);
            // untouched blocks: copy the ones that did not take part (nodes of shallower leaves)
            std::vector<char> cov(n, 0);
            for (const DcNode& nd : nodes)
                for (int i = nd.l; i < nd.r; ++i) cov[i] = 1;
            for (int i = 0; i < n;) {
                if (cov[i]) { ++i; continue; }
                int j = i;
                while (j < n && !cov[j]) ++j;
                copy_block(s, qb + (size_t)i * n + i, n, qa + (size_t)i * n + i, n, j - i, j - i);
                WT_CUDA(cudaMemcpyAsync(la + i, lb + i, (j - i) * sizeof(double), cudaMemcpyDeviceToDevice, s));
                i = j;
            }
        }
        if (qa != QA.p) {
            copy_block(s, qa, n, QA.p, n, n, n);
            WT_CUDA(cudaMemcpyAsync(lamA.p, la, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
    }
    WT_CUDA(cudaMemcpyAsync(w, lamA.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    QB.release();
    G.release();

    // 3. back-transformation: V = H_0 ... H_{n-3} Z, blocks of reflectors from the last one down
    double* Z = QA.p;
    const int nref = std::max(0, n - 2);
    if (nref > 0) {
        DBuf<double> Wt, S, T, Y, Y2;
        Wt.alloc((size_t)kWyBlock * n);
        S.alloc((size_t)kWyBlock * kWyBlock);
        T.alloc((size_t)kWyBlock * kWyBlock);
        Y.alloc((size_t)kWyBlock * n);
        Y2.alloc((size_t)kWyBlock * n);
        const int nblk = (nref + kWyBlock - 1) / kWyBlock;
        for (int bi = nblk - 1; bi >= 0; --bi) {
            const int k0 = bi * kWyBlock, nb = std::min(kWyBlock, nref - k0);
            const int m = n - k0 - 1;           // rows k0 + 1 .. n - 1
            wy_rows_kernel<<<dim3((n + 255) / 256, nb), 256, 0, s>>>(A, n, k0, nb, Wt.p);
            WT_LAUNCH("wy_rows");
            dgemm(s, false, true, nb, nb, m, 1.0, Wt.p + k0 + 1, n, Wt.p + k0 + 1, n, 0.0, S.p, nb);
            wy_t_kernel<<<1, 32, 0, s>>>(S.p, tau.p, k0, nb, T.p);
            WT_LAUNCH("wy_t");
            dgemm(s, false, false, nb, n, m, 1.0, Wt.p + k0 + 1, n, Z + (size_t)(k0 + 1) * n, n, 0.0, Y.p, n);
            dgemm(s, false, false, nb, n, nb, 1.0, T.p, nb, Y.p, n, 0.0, Y2.p, n);
            dgemm(s, true, false, m, n, nb, -1.0, Wt.p + k0 + 1, n, Y2.p, n, 1.0, Z + (size_t)(k0 + 1) * n, n);
        }
    }
    copy_block(s, Z, n, V, n, n, n);
    WT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace wt
