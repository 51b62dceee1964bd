// C ABI entry points and the host-side orchestration of the library:
// geometry and layout (host, FP64), boundary fit and relaxation (GPU FP64),
// bulk extension (GPU FP32 fast path / FP64 plain path).
#include "wt_internal.cuh"
#include "k_fft.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

namespace wt {

// kernels defined in other translation units
void green_invk2(cudaStream_t, int, int, int, double, double, double, double*);
void green_lateral(cudaStream_t, const double*, int, int, int, int, double, double, const double*, double*);
void green_cos_table(cudaStream_t, const double*, int, int, double, double*);
void green_pblocks(cudaStream_t, const void*, int, int, int, const double*, const double*, const double*, int, double,
                   double*, int);
size_t pblock_size();
void pack_pblock(void*, int, int, int, int, int, int, int);
void fit_ats(cudaStream_t, const double*, int, int, int, const int*, const int*, const double*, int, double*);
void fit_add_s(cudaStream_t, double*, int, int, const int*, const int*, const double*, double);
void set_column(cudaStream_t, double*, int, int, int, double);
void build_k(cudaStream_t, const double*, const double*, int, double*);
void modal_factors(cudaStream_t, const double*, const double*, int, const double*, int, double*);
void add_column_vector(cudaStream_t, double*, int, int, const double*);
void to_float(cudaStream_t, const double*, size_t, double, float*);
void check_finite(cudaStream_t, const double*, size_t, int*);
void expand_simt(cudaStream_t, const float*, int, const float*, int, int, size_t, float*);
void sample_lateral(cudaStream_t, const double*, int, const double*, int, int, int, int, double, double,
                    const double*, double*);
void sample_contract(cudaStream_t, const double*, const double*, const double*, int, int, int, int, double, double,
                     double*);
void eq1_launch(cudaStream_t, const float*, int, int, int, int, double, double, double, const float*, const float*,
                const float*, const float*, const float*, const float*, const float*, float, int, int, int, double,
                double, const void*, int, float*);
size_t eq1_lag_size();
void eq1_launch64(cudaStream_t, const double*, int, int, int, int, double, double, double, const float*, const float*,
                  const float*, const float*, const float*, const float*, const float*, float, int, int, int, double,
                  double, const void*, int, double*);
void green_lateral_deriv(cudaStream_t, const double*, const double*, int, int, int, int, double, double, double, double,
                         int, double*);
void modal_inv_gap(cudaStream_t, const double*, int, double*);
void modal_tangent(cudaStream_t, const double*, const double*, const double*, const double*, const double*,
                   const double*, int, int, double*);
void modal_omega(cudaStream_t, const double*, const double*, const double*, int, double*);
void add_row_const(cudaStream_t, double*, int, int, const double*);
double dot_f32(cudaStream_t, const float*, const float*, size_t, double*);
void eq1_noalloc_launch(cudaStream_t, int, const float*, int, int, int, const double*, int, double, double, double,
                        const float*, const float*, const float*, const float*, const float*, const float*,
                        const float*, float, int, int, int, double, double, int, float*);
void eq1_pack_lag(void*, int, float, float);
size_t eq1_lag64_size();
void eq1_pack_lag64(void*, int, double, double);
double dot_f64(cudaStream_t, const double*, const double*, size_t, double*);
void shape_launch(cudaStream_t, const float*, int, int, double, double, int, double, double, const float*, float*);
void eq1_point_major(cudaStream_t, const float*, int, size_t, float*);
void eq1_basis_launch(cudaStream_t, const float*, int, const float*, int, int, int, int, double, double, double,
                      const float*, const float*, const float*, const float*, const float*, const float*,
                      const float*, float, int, int, int, double, double, const void*, int, float*);
void features_launch(cudaStream_t, const float*, int, int, double, double, float, float, float, const float*, int,
                     double*, double*);
void add_f32(cudaStream_t, size_t, const float*, float*);
void drift_launch(cudaStream_t, const float*, int, int, int, double, double, double, const std::vector<double>&,
                  const double*, const double*, int, int, double, float*, float*, float*, float*, float*, float*);

void fail(wt_status code, const std::string& msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(WT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

using clk = std::chrono::steady_clock;
static double secs(clk::time_point a) { return std::chrono::duration<double>(clk::now() - a).count(); }

}  // namespace wt

using namespace wt;

struct wt_ctx {
    int dev = 0;
    cudaStream_t s = nullptr;
    cudaStream_t s_copy = nullptr;   // device-to-host copies of host-buffer extensions
    wt_grid grid{};
    std::vector<wt_column> cols;
    std::vector<std::vector<double>> rho_prof;   // per column: node resistivities (empty: uniform)
    wt_fit_opts opts{};
    std::string err;
    int stage = 0;                   // 0 created, 1 fitted, 2 relaxed
    // layout (host)
    int ns = 0, nc = 0;
    std::vector<int> col_off, colloc_off;
    std::vector<double> src_z;
    std::vector<double> phi_dc;
    // S as CSC lists: node j -> (collocation row, weight)
    std::vector<int> s_ptr, s_idx;
    std::vector<double> s_w;
    double pref = 0;
    // device, fit results
    DBuf<int> d_err;
    DBuf<double> d_scr;
    DBuf<double> Cn;                 // ns x ns capacitance
    DBuf<double> offset;             // ns: potential offset per node potential
    // relaxation
    std::vector<double> times;
    DBuf<double> d_times, mu, qinf, Qt;   // Qt [nt][ns]
    DBuf<double> Vm, amp;                 // modes (n1 x n1), amplitudes (n1)
    DBuf<double> hv;                      // Householder vector
    double beta = 0;
    int rank = 0, r_pad = 0;
    DBuf<double> Ub;                      // [r][ns] basis charge vectors
    DBuf<float> W32;                      // [nt][r_pad] time coefficients
    // spectral
    DBuf<double> d_zsrc;
    DBuf<double> zcos;                   // [ns][Nz] 2 cos(pi m z_j / Lz)
    DBuf<int> d_col_off;
    Fast32 sp32;
    Spectral<double> sp64;
    bool sp_ready = false;
    DBuf<float> Zc32, rho32, R32, E32;
    DBuf<float> Ep32;                // point-major copy of E32 for Eq. 1 from the rank-r form
    DBuf<float> ZcT32;               // column transforms as the table combination reads them
    // per-column lateral tables of the FP32 path ([n_cols][3][Nz][Ny][Nx], geometry only; built once)
    // and the slab buffer of the combined planes ([32][3][Nz][ys][Nx])
    DBuf<float> T32, Rsl;
    bool t32_ready = false;
    DBuf<double> Zc64, G64;
    DBuf<float> stage32;
    DBuf<double> stage64;
    wt_info info{};
    // kept from the fit for the derivative (wt_eq1_loss_grad)
    DBuf<double> fitA, fitD, fitL, fitY;      // scaled fit matrix, column scales, Cholesky factor, scaled solution
    std::vector<double> f_dxy, f_uxy, f_hzc;  // lateral offsets / radial directions per combo, collocation heights
    std::vector<int> f_ctoff;
    std::vector<unsigned char> f_blocks;
    int f_ncombo = 0, f_maxrows = 0, f_maxcols = 0;
    std::vector<double> k_diag, k_off, k_k1;  // resistive lines
    // stage timing (wt_set_timing)
    bool timing = false;
    bool use_tc = true;          // WT_EXPAND=simt selects the FP32 FMA expansion
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_noalloc = nullptr;    // last wt_eq1_noalloc call, on the caller's stream
    bool noalloc_pending = false;
    bool ev_recorded = false;
    int last_launches = 0;
    double grad_ms[6] = {0, 0, 0, 0, 0, 0};   // stages of the last timed loss derivative
    // launch shapes of the FP32 path (autotuned by wt_batch_run): charge vectors per spectral
    // launch, (x, y) lines per z-pass block, time samples per expansion accumulator chunk
    int tune_nb = 1, tune_lb = 32, tune_nch = 256, tune_nepi = 8, tune_vec = 4;
    int tune_ys = 0;                 // > 0: basis fields from the lateral tables, y slabs of tune_ys rows
    int tune_tf = 0;                 // table path flags: 1 slabs pipelined on two streams, 2 L2 discard,
                                     // 4 one line per thread in the combination
    cudaStream_t s_aux = nullptr;    // second stream of the pipelined table path
    cudaEvent_t ev_tc[2] = {nullptr, nullptr}, ev_tz[2] = {nullptr, nullptr}, ev_fork = nullptr;
    bool tuned = false;              // launch shapes chosen (first FP32 extension or batch)
    // identity and state counter, for the captured graphs of wt_batch_run
    unsigned long long uid = 0, version = 0;
    // version for which E32 holds the basis fields of this relaxation (0: anything else)
    unsigned long long e32_stamp = 0;
    std::vector<std::unique_ptr<struct BatchPlan>> plans;
    ~wt_ctx();
};

namespace {

thread_local std::string g_create_err;

template <class F>
wt_status run(wt_ctx* ctx, const char* fn, F&& body) {
    try {
        if (ctx) {
            cudaError_t e = cudaSetDevice(ctx->dev);
            if (e != cudaSuccess) fail(WT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
        }
        body();
        if (ctx) ctx->err.clear();
        return WT_OK;
    } catch (const Error& e) {
        if (ctx) ctx->err = std::string(fn) + ": " + e.msg;
        else g_create_err = std::string(fn) + ": " + e.msg;
        return e.code;
    } catch (const std::exception& e) {
        if (ctx) ctx->err = std::string(fn) + ": " + e.what();
        return WT_ERR_CUDA;
    }
}

int read_err(wt_ctx* c) {
    int h = 0;
    WT_CUDA(cudaMemcpyAsync(&h, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    WT_CUDA(cudaStreamSynchronize(c->s));
    return h;
}
void clear_err(wt_ctx* c) { WT_CUDA(cudaMemsetAsync(c->d_err.p, 0, sizeof(int), c->s)); }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Empty when [p, p + bytes) is device memory of device `dev` inside one
// allocation (or managed memory); otherwise why not.  The allocation's extent
// comes from cuMemGetAddressRange (through the runtime's driver entry point).
std::string device_span_problem(const void* p, size_t bytes, int dev) {
    if (!p) return "NULL buffer";
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) { cudaGetLastError(); return "not device memory"; }
    if (a.type == cudaMemoryTypeManaged) return "";
    if (a.type != cudaMemoryTypeDevice) return "not device memory";
    if (a.device != dev) return "device memory of device " + std::to_string(a.device) + ", the context is on " +
                                std::to_string(dev);
    static PFN_cuMemGetAddressRange_v3020 range = nullptr;
    if (!range) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        WT_CUDA(cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 3020, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !f) fail(WT_ERR_CUDA, "cuMemGetAddressRange unavailable");
        range = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(f);
    }
    CUdeviceptr base = 0;
    size_t size = 0;
    if (range(&base, &size, reinterpret_cast<CUdeviceptr>(p)) != CUDA_SUCCESS) return "not device memory";
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p);
    if (lo + bytes > (uintptr_t)base + size)
        return "buffer too small: " + std::to_string(bytes) + " bytes needed, " +
               std::to_string((uintptr_t)base + size - lo) + " in its allocation";
    return "";
}

void validate_geometry(const wt_ctx* c) {
    const wt_grid& g = c->grid;
    if (c->cols.empty()) fail(WT_ERR_GEOMETRY, "no columns");
    for (size_t i = 0; i < c->cols.size(); ++i) {
        const wt_column& k = c->cols[i];
        if (!(k.z0 >= 0.0 && k.z1 > k.z0 && k.z1 <= g.Lz * (1 + 1e-12)))
            fail(WT_ERR_GEOMETRY, "column " + std::to_string(i) + " z range outside the sensor");
        if (!(k.radius > 0.0) || !(k.resistivity > 0.0) || k.n_sources < 1)
            fail(WT_ERR_GEOMETRY, "column " + std::to_string(i) + ": radius, resistivity and n_sources must be > 0");
        if (!std::isfinite(k.x) || !std::isfinite(k.y)) fail(WT_ERR_NAN, "non-finite column position");
    }
    for (size_t i = 0; i < c->cols.size(); ++i)
        for (size_t j = i + 1; j < c->cols.size(); ++j) {
            double dx = c->cols[i].x - c->cols[j].x, dy = c->cols[i].y - c->cols[j].y;
            dx -= g.Lx * std::round(dx / g.Lx);
            dy -= g.Ly * std::round(dy / g.Ly);
            if (std::hypot(dx, dy) <= c->cols[i].radius + c->cols[j].radius)
                fail(WT_ERR_GEOMETRY, "columns " + std::to_string(i) + " and " + std::to_string(j) + " overlap");
        }
}

void build_layout(wt_ctx* c) {
    const int ncol = (int)c->cols.size();
    const int n_az = c->opts.n_az, n_h = c->opts.n_h;
    c->col_off.assign(ncol + 1, 0);
    c->colloc_off.assign(ncol + 1, 0);
    c->src_z.clear();
    for (int k = 0; k < ncol; ++k) {
        const wt_column& col = c->cols[k];
        const int m = col.n_sources;
        const double dz = (col.z1 - col.z0) / m;
        for (int j = 0; j < m; ++j) c->src_z.push_back(col.z0 + (j + 0.5) * dz);
        c->col_off[k + 1] = c->col_off[k] + m;
        c->colloc_off[k + 1] = c->colloc_off[k] + n_az * n_h * m;
    }
    c->ns = c->col_off[ncol];
    c->nc = c->colloc_off[ncol];
    // S: collocation height -> linear interpolation between the bracketing nodes
    std::vector<std::vector<std::pair<int, double>>> lists(c->ns);
    for (int k = 0; k < ncol; ++k) {
        const wt_column& col = c->cols[k];
        const int m = col.n_sources, nh = n_h * m;
        const double dz = (col.z1 - col.z0) / m;
        for (int a = 0; a < n_az; ++a)
            for (int p = 0; p < nh; ++p) {
                const int row = c->colloc_off[k] + a * nh + p;
                const double zc = col.z0 + (p + 0.5) * (col.z1 - col.z0) / nh;
                const double u = (zc - col.z0) / dz - 0.5;
                const int off = c->col_off[k];
                if (u <= 0.0) lists[off].push_back({row, 1.0});
                else if (u >= m - 1) lists[off + m - 1].push_back({row, 1.0});
                else {
                    const int j = (int)std::floor(u);
                    const double f = u - j;
                    lists[off + j].push_back({row, 1.0 - f});
                    if (f != 0.0) lists[off + j + 1].push_back({row, f});
                }
            }
    }
    c->s_ptr.assign(c->ns + 1, 0);
    c->s_idx.clear();
    c->s_w.clear();
    for (int j = 0; j < c->ns; ++j) {
        for (auto& e : lists[j]) { c->s_idx.push_back(e.first); c->s_w.push_back(e.second); }
        c->s_ptr[j + 1] = (int)c->s_idx.size();
    }
    c->phi_dc.assign(c->ns, 0.0);
    for (int k = 0; k < ncol; ++k)
        if (c->cols[k].driven)
            for (int j = c->col_off[k]; j < c->col_off[k + 1]; ++j) c->phi_dc[j] = c->opts.v_w;
}

// H M H for symmetric M (n x n, in place), H = I - beta v v^T.
void householder_two_sided(wt_ctx* c, double* M, int n) {
    DBuf<double> u;
    u.alloc(n);
    dgemv(c->s, false, n, n, 1.0, M, n, c->hv.p, 0.0, u.p);
    std::vector<double> hu(n), hv(n);
    u.download(hu.data(), n, c->s);
    c->hv.download(hv.data(), n, c->s);
    WT_CUDA(cudaStreamSynchronize(c->s));
    double gamma = 0;
    for (int i = 0; i < n; ++i) gamma += hv[i] * hu[i];
    std::vector<double> w(n);
    for (int i = 0; i < n; ++i) w[i] = c->beta * hu[i] - 0.5 * c->beta * c->beta * gamma * hv[i];
    DBuf<double> dw;
    dw.upload(w.data(), n, c->s);
    rank1(c->s, n, n, -1.0, c->hv.p, dw.p, M, n);
    rank1(c->s, n, n, -1.0, dw.p, c->hv.p, M, n);
    WT_CUDA(cudaStreamSynchronize(c->s));
}

void do_fit(wt_ctx* c) {
    auto t0 = clk::now();
    validate_geometry(c);
    build_layout(c);
    const wt_grid& g = c->grid;
    const int ncol = (int)c->cols.size(), ns = c->ns, nc = c->nc;
    const int n_az = c->opts.n_az;
    const double eps = kEps0 * g.eps_r;
    const double vol = g.Lx * g.Ly * 2.0 * g.Lz;
    c->pref = 1.0 / (eps * vol);
    cudaStream_t s = c->s;
    clear_err(c);

    // --- S2: fundamental-solution tables and the fit matrix P
    DBuf<double> T, L, dxy, Ct, Cs, zc_all, zs_all, P;
    T.alloc((size_t)(g.Nx / 2) * (g.Ny / 2) * g.Nz);
    green_invk2(s, g.Nx, g.Ny, g.Nz, g.Lx, g.Ly, g.Lz, T.p);
    const int n_tg = ncol * n_az;                  // target lateral groups
    std::vector<double> hdxy, huxy;
    for (int k = 0; k < ncol; ++k)
        for (int a = 0; a < n_az; ++a) {
            const double th = c->opts.az0 + 2.0 * kPi * a / n_az;
            const double tx = c->cols[k].x + c->cols[k].radius * std::cos(th);
            const double ty = c->cols[k].y + c->cols[k].radius * std::sin(th);
            for (int k2 = 0; k2 < ncol; ++k2) {
                hdxy.push_back(tx - c->cols[k2].x);
                hdxy.push_back(ty - c->cols[k2].y);
                huxy.push_back(std::cos(th));
                huxy.push_back(std::sin(th));
            }
        }
    const int n_combo = n_tg * ncol;
    dxy.upload(hdxy.data(), hdxy.size(), s);
    L.alloc((size_t)n_combo * g.Nz);
    green_lateral(s, dxy.p, n_combo, g.Nx, g.Ny, g.Nz, g.Lx, g.Ly, T.p, L.p);
    T.release();
    // cos tables: collocation heights per column (n_h M_c each), source heights
    std::vector<double> hzc;
    std::vector<int> ct_off(ncol + 1, 0);
    for (int k = 0; k < ncol; ++k) {
        const wt_column& col = c->cols[k];
        const int nh = c->opts.n_h * col.n_sources;
        for (int p = 0; p < nh; ++p) hzc.push_back(col.z0 + (p + 0.5) * (col.z1 - col.z0) / nh);
        ct_off[k + 1] = ct_off[k] + nh;
    }
    zc_all.upload(hzc.data(), hzc.size(), s);
    zs_all.upload(c->src_z.data(), ns, s);
    Ct.alloc(hzc.size() * g.Nz);
    Cs.alloc((size_t)ns * g.Nz);
    green_cos_table(s, zc_all.p, (int)hzc.size(), g.Nz, g.Lz, Ct.p);
    green_cos_table(s, zs_all.p, ns, g.Nz, g.Lz, Cs.p);
    std::vector<unsigned char> blocks(pblock_size() * (size_t)n_combo);
    int max_rows = 0, max_cols = 0;
    for (int k = 0; k < ncol; ++k)
        for (int a = 0; a < n_az; ++a)
            for (int k2 = 0; k2 < ncol; ++k2) {
                const int tg = k * n_az + a;
                const int nh = c->opts.n_h * c->cols[k].n_sources;
                const int row0 = c->colloc_off[k] + a * nh;
                pack_pblock(blocks.data() + pblock_size() * (size_t)(tg * ncol + k2), row0, nh, c->col_off[k2],
                            c->cols[k2].n_sources, ct_off[k], c->col_off[k2], tg * ncol + k2);
                max_rows = std::max(max_rows, nh);
                max_cols = std::max(max_cols, c->cols[k2].n_sources);
            }
    c->f_dxy = hdxy;
    c->f_uxy = huxy;
    c->f_hzc = hzc;
    c->f_ctoff = ct_off;
    c->f_blocks = blocks;
    c->f_ncombo = n_combo;
    c->f_maxrows = max_rows;
    c->f_maxcols = max_cols;
    DBuf<unsigned char> dblocks;
    dblocks.upload(blocks.data(), blocks.size(), s);
    P.alloc((size_t)nc * ns);
    green_pblocks(s, dblocks.p, n_combo, max_rows, max_cols, Ct.p, Cs.p, L.p, g.Nz, c->pref, P.p, ns);
    Ct.release(); Cs.release(); L.release();

    // --- S3: neutral basis (Householder), offset column, column scaling
    std::vector<double> hv(ns, 1.0);
    hv[0] += std::sqrt((double)ns);
    double vtv = 0;
    for (double x : hv) vtv += x * x;
    c->beta = 2.0 / vtv;
    c->hv.upload(hv.data(), ns, s);
    DBuf<double> w, dcol;
    w.alloc(nc);
    dgemv(s, false, nc, ns, 1.0, P.p, ns, c->hv.p, 0.0, w.p);
    rank1(s, nc, ns, -c->beta, w.p, c->hv.p, P.p, ns);     // P H
    set_column(s, P.p, nc, ns, 0, 1.0);                     // A = [1 | P B]
    w.release();
    dcol.alloc(ns);
    column_norms(s, P.p, nc, ns, ns, dcol.p);
    std::vector<double> hd(ns);
    dcol.download(hd.data(), ns, s);
    WT_CUDA(cudaStreamSynchronize(s));
    double max_sq = 0;
    for (int k = 0; k < ns; ++k) {
        if (!(hd[k] > 0.0) || !std::isfinite(hd[k])) fail(WT_ERR_ILL_CONDITIONED, "zero or non-finite fit column");
        if (k > 0) max_sq = std::max(max_sq, hd[k] * hd[k]);
        hd[k] = 1.0 / hd[k];
    }
    dcol.upload(hd.data(), ns, s);
    scale_columns(s, P.p, nc, ns, ns, dcol.p);               // A_s = A D

    // normal matrix G = A_s^T A_s (+ ridge on the charge part)
    DBuf<double> G, R, Y;
    G.alloc((size_t)ns * ns);
    dgemm(s, true, false, ns, ns, nc, 1.0, P.p, ns, P.p, ns, 0.0, G.p, ns, true);
    symmetrize_from_lower(s, G.p, ns, ns);
    if (c->opts.tikhonov > 0.0) {
        std::vector<double> ridge(ns, 0.0);
        for (int k = 1; k < ns; ++k) ridge[k] = c->opts.tikhonov * max_sq * hd[k] * hd[k];
        DBuf<double> dr;
        dr.upload(ridge.data(), ns, s);
        // G[k][k] += ridge[k]: a rank-1 of diagonal form via a strided axpy
        DBuf<double> diag;
        diag.alloc(ns);
        get_diag(s, G.p, ns, ns, diag.p);
        axpy(s, ns, 1.0, dr.p, diag.p);
        copy_block(s, diag.p, 1, G.p, ns + 1, ns, 1);
    }
    // right-hand sides R = A_s^T S
    DBuf<int> sp, si;
    DBuf<double> sw;
    sp.upload(c->s_ptr.data(), c->s_ptr.size(), s);
    si.upload(c->s_idx.data(), c->s_idx.size(), s);
    sw.upload(c->s_w.data(), c->s_w.size(), s);
    R.alloc((size_t)ns * ns);
    Y.alloc((size_t)ns * ns);
    fit_ats(s, P.p, ns, nc, ns, sp.p, si.p, sw.p, ns, Y.p);   // Y = R^T
    transpose(s, Y.p, ns, ns, R.p);
    // --- S4: Cholesky and solves, one step of corrected semi-normal equations
    cholesky(s, G.p, ns, ns, c->d_err.p);
    if (fault_enabled("fit_singular")) {      // injected: as if the factorisation met a non-positive pivot
        const int v = DERR_NOT_SPD;
        WT_CUDA(cudaMemcpyAsync(c->d_err.p, &v, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    if (read_err(c)) fail(WT_ERR_NOT_SPD, "normal matrix of the fit is not positive definite (rank-deficient fit)");
    copy_block(s, R.p, ns, Y.p, ns, ns, ns);
    trsm_lower(s, G.p, ns, ns, Y.p, ns, ns);
    trsm_lower_t(s, G.p, ns, ns, Y.p, ns, ns);
    // Corrected semi-normal equations: dY = G^-1 A_s^T (S - A_s Y).  Its two products cost
    // 4 nc ns^2 flops, most of the fit; dY is linear in the right-hand sides, so its action on
    // eight random +-1 combinations Z (dY Z, from S Z and Y Z at 8/ns of the cost) estimates
    // ||dY|| / ||Y||, and the full step runs only when that exceeds kRefineSkip, a tenth of the
    // FP64 path's accuracy bound (1e-10): the normal equations alone err by about cond(A_s)^2 eps.
    constexpr double kRefineSkip = 1e-11;
    bool refine = c->opts.refine == 1;
    double correction = 0.0;
    if (!refine) {
        constexpr int kp = 8;
        std::vector<double> hz((size_t)ns * kp), hsz((size_t)nc * kp, 0.0);
        unsigned long long st = 0x9E3779B97F4A7C15ull;            // fixed seed: reproducible fits
        for (double& v : hz) {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            v = (st >> 63) ? 1.0 : -1.0;
        }
        for (int j = 0; j < ns; ++j)
            for (int e = c->s_ptr[j]; e < c->s_ptr[j + 1]; ++e)
                for (int k = 0; k < kp; ++k) hsz[(size_t)c->s_idx[e] * kp + k] += c->s_w[e] * hz[(size_t)j * kp + k];
        DBuf<double> Z, Yz, Rz, Cz;
        Z.upload(hz.data(), hz.size(), s);
        Rz.upload(hsz.data(), hsz.size(), s);                    // S Z
        Yz.alloc((size_t)ns * kp);
        Cz.alloc((size_t)ns * kp);
        dgemm(s, false, false, ns, kp, ns, 1.0, Y.p, ns, Z.p, kp, 0.0, Yz.p, kp);
        dgemm(s, false, false, nc, kp, ns, -1.0, P.p, ns, Yz.p, kp, 1.0, Rz.p, kp);
        dgemm(s, true, false, ns, kp, nc, 1.0, P.p, ns, Rz.p, kp, 0.0, Cz.p, kp);
        trsm_lower(s, G.p, ns, ns, Cz.p, kp, kp);
        trsm_lower_t(s, G.p, ns, ns, Cz.p, kp, kp);
        const double ny = dnrm2(s, Yz.p, (size_t)ns * kp, c->d_scr.p);
        const double nd = dnrm2(s, Cz.p, (size_t)ns * kp, c->d_scr.p);
        correction = ny > 0.0 ? nd / ny : INFINITY;
        refine = !(correction <= kRefineSkip);
    }
    if (refine) {
        DBuf<double> Res;
        Res.alloc((size_t)nc * ns);
        dgemm(s, false, false, nc, ns, ns, -1.0, P.p, ns, Y.p, ns, 0.0, Res.p, ns);
        fit_add_s(s, Res.p, ns, ns, sp.p, si.p, sw.p, 1.0);
        dgemm(s, true, false, ns, ns, nc, 1.0, P.p, ns, Res.p, ns, 0.0, R.p, ns);
        trsm_lower(s, G.p, ns, ns, R.p, ns, ns);
        trsm_lower_t(s, G.p, ns, ns, R.p, ns, ns);
        const double ny = dnrm2(s, Y.p, (size_t)ns * ns, c->d_scr.p);
        correction = ny > 0.0 ? dnrm2(s, R.p, (size_t)ns * ns, c->d_scr.p) / ny : INFINITY;
        axpy(s, (size_t)ns * ns, 1.0, R.p, Y.p);
    }
    c->info.fit_correction = correction;
    c->info.fit_refined = refine ? 1 : 0;
    // DC boundary residual || A_s (Y phi) - S phi || / || S phi ||
    {
        DBuf<double> dphi, yphi, r;
        dphi.upload(c->phi_dc.data(), ns, s);
        yphi.alloc(ns);
        r.alloc(nc);
        dgemv(s, false, ns, ns, 1.0, Y.p, ns, dphi.p, 0.0, yphi.p);
        dgemv(s, false, nc, ns, 1.0, P.p, ns, yphi.p, 0.0, r.p);
        std::vector<double> hr(nc), sphi(nc, 0.0);
        r.download(hr.data(), nc, s);
        WT_CUDA(cudaStreamSynchronize(s));
        for (int j = 0; j < ns; ++j)
            for (int e = c->s_ptr[j]; e < c->s_ptr[j + 1]; ++e) sphi[c->s_idx[e]] += c->s_w[e] * c->phi_dc[j];
        double num = 0, den = 0;
        for (int i = 0; i < nc; ++i) { num += (hr[i] - sphi[i]) * (hr[i] - sphi[i]); den += sphi[i] * sphi[i]; }
        c->info.boundary_residual = den > 0 ? std::sqrt(num / den) : 0.0;
    }
    // condition estimate from the Cholesky diagonal of the scaled normal matrix
    {
        DBuf<double> dg;
        dg.alloc(ns);
        get_diag(s, G.p, ns, ns, dg.p);
        std::vector<double> h(ns);
        dg.download(h.data(), ns, s);
        WT_CUDA(cudaStreamSynchronize(s));
        double mx = 0, mn = 1e300;
        for (double x : h) { mx = std::max(mx, std::fabs(x)); mn = std::min(mn, std::fabs(x)); }
        c->info.cond_estimate = mn > 0 ? mx / mn : INFINITY;
    }
    // keep the factors for the derivative of the fit (scaled A, D, Cholesky factor, scaled solution)
    c->fitY.alloc((size_t)ns * ns);
    copy_block(s, Y.p, ns, c->fitY.p, ns, ns, ns);
    c->fitL.take(G);
    c->fitA.take(P);
    // X = D Y; offsets = row 0; F = H [0; X_1:]
    scale_rows(s, Y.p, ns, ns, ns, dcol.p);
    c->offset.alloc(ns);
    copy_block(s, Y.p, ns, c->offset.p, ns, 1, ns);
    fill(s, Y.p, ns, 0.0);
    DBuf<double> u;
    u.alloc(ns);
    dgemv(s, true, ns, ns, 1.0, Y.p, ns, c->hv.p, 0.0, u.p);
    rank1(s, ns, ns, -c->beta, c->hv.p, u.p, Y.p, ns);      // F in Y
    c->Cn.alloc((size_t)ns * ns);
    symmetrize_avg(s, Y.p, c->Cn.p, ns);
    transpose(s, Y.p, ns, ns, R.p);
    double nF = dnrm2(s, Y.p, (size_t)ns * ns, c->d_scr.p);
    axpy(s, (size_t)ns * ns, -1.0, Y.p, R.p);
    double nA = dnrm2(s, R.p, (size_t)ns * ns, c->d_scr.p);
    c->info.asymmetry = nF > 0 ? nA / nF : 0.0;
    check_finite(s, c->Cn.p, (size_t)ns * ns, c->d_err.p);
    if (read_err(c)) fail(WT_ERR_NAN, "non-finite capacitance");
    c->fitD.take(dcol);
    c->info.n_columns = ncol;
    c->info.n_sources = ns;
    c->info.n_colloc = nc;
    c->info.fit_seconds = secs(t0);
}

// Q [ns][nt] = q(t_n) = q_inf + Cn H [0; V (amp * exp(-mu t_n))] for device times.
void charges_at(wt_ctx* c, const double* d_t, int nt, double* Q) {
    cudaStream_t s = c->s;
    const int ns = c->ns, n1 = ns - 1;
    DBuf<double> E, Zf, vz;
    E.alloc((size_t)n1 * nt);
    modal_factors(s, c->amp.p, c->mu.p, n1, d_t, nt, E.p);
    Zf.alloc((size_t)ns * nt);
    Zf.zero(s);
    dgemm(s, false, false, n1, nt, n1, 1.0, c->Vm.p, n1, E.p, nt, 0.0, Zf.p + nt, nt);
    vz.alloc(nt);
    dgemv(s, true, ns, nt, 1.0, Zf.p, nt, c->hv.p, 0.0, vz.p);
    rank1(s, ns, nt, -c->beta, c->hv.p, vz.p, Zf.p, nt);
    dgemm(s, false, false, ns, nt, ns, 1.0, c->Cn.p, ns, Zf.p, nt, 0.0, Q, nt);
    add_column_vector(s, Q, ns, nt, c->qinf.p);
}

// Time basis of a charge history Q [ns][nt] for the FP32 path: the singular
// value decomposition Q = sum_i sigma_i u_i v_i^T by one-sided Jacobi (no Gram
// matrix: the small singular values keep their relative accuracy).  When
// ns >= nt the Jacobi runs on the rows of R from a column-pivoted QR,
// Q P = Q1 R (Drmac and Veselic's preconditioning: rows of length nt instead
// of ns, and a few sweeps instead of twenty for the nearly parallel samples of
// a relaxation): rotated to orthogonal rows S_k = sigma_k w_k^T, R's rows give
// v_k[P_i] = w_k[i], and u_k = Q v_k / sigma_k.  Otherwise it runs on the rows
// of Q^T directly.  Then the smallest rank r <= 32 whose truncation error in every
// time sample, ||q(t_n) - sum_{i<r} sigma_i u_i v_i[n]|| / ||q(t_n)||, is at
// most kTruncTarget (the FP32 rounding level).  The error is exact from the
// decomposition: the squared tail sum_{i>=r} (sigma_i v_i[n])^2, summed from
// the smallest term up.  Samples whose charge is below kTruncFloor of the
// largest one are measured against that floor (tangent histories can vanish
// at some times).  Outputs: basis charge vectors Ub [r][ns] (unit norm),
// FP32 coefficients W32 [nt][32] = sigma_m v_m[n], r, and the largest
// per-sample truncation at r (trunc_out).
constexpr double kTruncTarget = 1e-7;
constexpr double kTruncLimit = 1e-6;     // the FP32 field paths refuse a basis truncated beyond this
constexpr double kTruncFloor = 1e-6;
void compress_history(wt_ctx* c, const double* Q, int nt, DBuf<double>& Ub, DBuf<float>& W32, int& rank_out,
                      double& trunc_out) {
    cudaStream_t s = c->s;
    const int ns = c->ns;
    const bool pre = ns >= nt;                    // column-pivoted QR first
    DBuf<double> A, V, sig, Rm;
    DBuf<int> dpiv;
    A.alloc((size_t)nt * ns);
    transpose(s, Q, ns, nt, A.p);                 // rows = time samples (the columns of Q)
    sig.alloc(nt);
    if (pre) {
        Rm.alloc((size_t)nt * nt);
        dpiv.alloc(nt);
        qrcp_r(s, A.p, ns, nt, ns, Rm.p, dpiv.p);
        A.release();
    } else {
        V.alloc((size_t)nt * nt);
    }
    clear_err(c);
    double coupling = 0.0;
    const int sweeps = pre ? onesided_jacobi_rows(s, Rm.p, nt, nt, nt, nullptr, sig.p, c->d_err.p, 40, &coupling)
                           : onesided_jacobi_rows(s, A.p, nt, ns, ns, V.p, sig.p, c->d_err.p, 40, &coupling);
    if (read_err(c)) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "one-sided Jacobi (time basis) did not converge: %d sweeps, relative coupling %.3e still rotated",
                      sweeps, coupling);
        fail(WT_ERR_TIMEOUT, msg);
    }
    std::vector<double> hs(nt), hv((size_t)nt * nt);
    sig.download(hs.data(), nt, s);
    if (pre) {
        // hv[k][P_i] = S[k][i] / sigma_k: the coefficient of u_k in sample P_i over sigma_k
        std::vector<double> hS((size_t)nt * nt);
        std::vector<int> hp(nt);
        Rm.download(hS.data(), hS.size(), s);
        dpiv.download(hp.data(), nt, s);
        WT_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nt; ++k) {
            const double inv = hs[k] > 0.0 ? 1.0 / hs[k] : 0.0;
            for (int i = 0; i < nt; ++i) hv[(size_t)k * nt + hp[i]] = hS[(size_t)k * nt + i] * inv;
        }
    } else {
        V.download(hv.data(), (size_t)nt * nt, s);
        WT_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<int> ord(nt);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hs[a] > hs[b]; });
    // per-sample squared norms and suffix (tail) sums, smallest terms first
    auto term = [&](int j, int n) {
        const double x = hs[ord[j]] * hv[(size_t)ord[j] * nt + n];
        return x * x;
    };
    std::vector<double> norm2(nt, 0.0);
    for (int n = 0; n < nt; ++n)
        for (int j = nt - 1; j >= 0; --j) norm2[n] += term(j, n);
    double nmax = 0.0;
    for (double v : norm2) nmax = std::max(nmax, std::sqrt(v));
    const int r_cap = std::min(fault_enabled("rank_cap") ? 4 : 32, nt);    // WT_FAULT=rank_cap: the guard's test
    // worst per-sample truncation for every r <= r_cap
    std::vector<double> worst(r_cap + 1, 0.0);
    std::vector<double> tail(nt, 0.0);
    for (int j = nt - 1; j >= 0; --j) {
        for (int n = 0; n < nt; ++n) tail[n] += term(j, n);
        if (j <= r_cap) {
            double w = 0.0;
            for (int n = 0; n < nt; ++n)
                w = std::max(w, std::sqrt(tail[n]) / std::max(std::sqrt(norm2[n]), kTruncFloor * nmax));
            worst[j] = nmax > 0 ? w : 0.0;
        }
    }
    int r = 1;
    while (r < r_cap && worst[r] > kTruncTarget) ++r;
    if (r < r_cap && hs[ord[r]] <= 0.0) r = std::max(1, r);
    rank_out = r;
    trunc_out = r < nt ? worst[r] : 0.0;
    const int rp = 32;
    std::vector<double> coef((size_t)nt * rp, 0.0), scale(r);
    std::vector<int> idx(r);
    for (int m = 0; m < r; ++m) {
        const double sg = hs[ord[m]];
        idx[m] = ord[m];
        scale[m] = sg > 0 ? 1.0 / sg : 0.0;
        for (int n = 0; n < nt; ++n) coef[(size_t)n * rp + m] = sg * hv[(size_t)ord[m] * nt + n];
    }
    DBuf<int> didx;
    DBuf<double> dscale, dcoef;
    Ub.alloc((size_t)r * ns);
    if (pre) {
        // u_m = Q v_m / sigma_m: Ub [r][ns] = (V_r / sigma) Q^T
        std::vector<double> vr((size_t)r * nt);
        for (int m = 0; m < r; ++m)
            for (int n = 0; n < nt; ++n) vr[(size_t)m * nt + n] = hv[(size_t)idx[m] * nt + n] * scale[m];
        DBuf<double> dvr;
        dvr.upload(vr.data(), vr.size(), s);
        dgemm(s, false, true, r, ns, nt, 1.0, dvr.p, nt, Q, nt, 0.0, Ub.p, ns);
        WT_CUDA(cudaStreamSynchronize(s));
    } else {
        didx.upload(idx.data(), r, s);
        dscale.upload(scale.data(), r, s);
        gather_rows_scaled(s, A.p, ns, ns, didx.p, dscale.p, r, Ub.p);
    }
    dcoef.upload(coef.data(), coef.size(), s);
    W32.alloc(coef.size());
    to_float(s, dcoef.p, coef.size(), 1.0, W32.p);
    WT_CUDA(cudaStreamSynchronize(s));
}

// The FP32 field paths expand the relaxation's time basis: refuse one that cannot carry the
// FP32 accuracy (a charge history that needs more than 32 basis vectors).
void require_fp32_basis(const wt_ctx* c) {
    if (c->info.trunc_rel > kTruncLimit)
        fail(WT_ERR_ACCURACY, "the charge history needs a time basis of rank > 32: the rank-32 basis leaves " +
                                  std::to_string(c->info.trunc_rel) +
                                  " relative error in a time sample (limit 1e-6); use WT_FP64");
}

void do_relax(wt_ctx* c, const double* t, int nt) {
    auto t0 = clk::now();
    ++c->version;
    cudaStream_t s = c->s;
    const int ns = c->ns, n1 = ns - 1;
    if (n1 < 1) fail(WT_ERR_GEOMETRY, "need at least two sources");
    clear_err(c);
    c->times.assign(t, t + nt);
    // resistive lines (Sec. 5): G_seg = pi r^2 / (rho Delta), terminal 2 G_seg
    // node j is the centre of a cell of height dz and resistivity rho_j: neighbours are joined
    // through two half cells, the terminal node reaches the electrode end through one
    std::vector<double> diag(ns, 0.0), off(ns, 0.0), k1(ns, 0.0);
    for (size_t k = 0; k < c->cols.size(); ++k) {
        const wt_column& col = c->cols[k];
        const int m = col.n_sources, o = c->col_off[k];
        const double dz = (col.z1 - col.z0) / m;
        const double area = kPi * col.radius * col.radius;
        auto rho = [&](int j) { return c->rho_prof[k].empty() ? col.resistivity : c->rho_prof[k][j]; };
        for (int j = 0; j + 1 < m; ++j) {
            const double gs = area / (0.5 * (rho(j) + rho(j + 1)) * dz);
            off[o + j] = gs;
            diag[o + j] -= gs;
            diag[o + j + 1] -= gs;
        }
        const int jl = col.terminal_top ? m - 1 : 0;
        const double gt = area / (0.5 * rho(jl) * dz);
        diag[o + jl] -= gt;
        k1[o + jl] = -gt;                   // K 1: only the terminal leak survives
    }
    c->k_diag = diag;
    c->k_off = off;
    c->k_k1 = k1;
    double s1 = 0;
    for (double x : k1) s1 += x;
    DBuf<double> dd, doff, dk1, K, Am, Sm;
    dd.upload(diag.data(), ns, s);
    doff.upload(off.data(), ns, s);
    dk1.upload(k1.data(), ns, s);
    K.alloc((size_t)ns * ns);
    build_k(s, dd.p, doff.p, ns, K.p);
    rank1(s, ns, ns, -1.0 / s1, dk1.p, dk1.p, K.p, ns);     // K~ = K - K1 1^T K / (1^T K 1)
    // reduced pencil on the neutral subspace: Am = (H Cn H)[1:,1:], Sm = -(H K~ H)[1:,1:]
    DBuf<double> HC;
    HC.alloc((size_t)ns * ns);
    copy_block(s, c->Cn.p, ns, HC.p, ns, ns, ns);
    householder_two_sided(c, HC.p, ns);
    householder_two_sided(c, K.p, ns);
    Am.alloc((size_t)n1 * n1);
    Sm.alloc((size_t)n1 * n1);
    copy_block(s, HC.p + ns + 1, ns, Am.p, n1, n1, n1);
    copy_block(s, K.p + ns + 1, ns, Sm.p, n1, n1, n1);
    HC.release();
    K.release();
    dscal(s, (size_t)n1 * n1, -1.0, Sm.p);                  // Sm = -B^T K~ B
    {
        DBuf<double> tmp;
        tmp.alloc((size_t)n1 * n1);
        symmetrize_avg(s, Am.p, tmp.p, n1);
        copy_block(s, tmp.p, n1, Am.p, n1, n1, n1);
        symmetrize_avg(s, Sm.p, tmp.p, n1);
        copy_block(s, tmp.p, n1, Sm.p, n1, n1, n1);
    }
    // Cholesky of the capacitance pencil side
    cholesky(s, Am.p, n1, n1, c->d_err.p);
    if (read_err(c)) fail(WT_ERR_NOT_SPD, "fitted capacitance is not positive definite on the neutral subspace");
    // Shat = L^-1 Sm L^-T (symmetric positive definite)
    DBuf<double> Y, Yt;
    Y.alloc((size_t)n1 * n1);
    Yt.alloc((size_t)n1 * n1);
    copy_block(s, Sm.p, n1, Y.p, n1, n1, n1);
    trsm_lower(s, Am.p, n1, n1, Y.p, n1, n1);
    transpose(s, Y.p, n1, n1, Yt.p);
    trsm_lower(s, Am.p, n1, n1, Yt.p, n1, n1);
    symmetrize_avg(s, Yt.p, Y.p, n1);
    c->mu.alloc(n1);
    DBuf<double> U;
    U.alloc((size_t)n1 * n1);
    // modes: tridiagonalisation + divide and conquer; WT_EIGEN=jacobi selects the two-sided
    // Jacobi solver instead (a cross-check)
    const char* eig_env = std::getenv("WT_EIGEN");
    if (eig_env && std::string(eig_env) == "jacobi") {
        jacobi_eig(s, Y.p, n1, c->mu.p, U.p, c->d_err.p);
        if (read_err(c)) fail(WT_ERR_TIMEOUT, "Jacobi eigensolver did not converge");
    } else {
        sym_eig(s, Y.p, n1, c->mu.p, U.p, c->d_err.p);
        if (read_err(c)) fail(WT_ERR_TIMEOUT, "tridiagonal QL iteration did not converge");
    }
    trsm_lower_t(s, Am.p, n1, n1, U.p, n1, n1);              // V = L^-T U
    Y.release(); Yt.release(); Sm.release();
    std::vector<double> hmu(n1);
    c->mu.download(hmu.data(), n1, s);
    WT_CUDA(cudaStreamSynchronize(s));
    double mn = 1e300, mx = -1e300;
    for (double x : hmu) { mn = std::min(mn, x); mx = std::max(mx, x); }
    if (!(mn > 0.0)) fail(WT_ERR_NOT_SPD, "non-positive relaxation rate (resistive pencil not definite)");
    c->info.mu_min = mn;
    c->info.mu_max = mx;
    // q_inf = Cn phi_DC; amplitudes amp = V^T B^T (-q_inf)
    DBuf<double> dphi, g;
    dphi.upload(c->phi_dc.data(), ns, s);
    c->qinf.alloc(ns);
    dgemv(s, false, ns, ns, 1.0, c->Cn.p, ns, dphi.p, 0.0, c->qinf.p);
    std::vector<double> hq(ns), hv(ns);
    c->qinf.download(hq.data(), ns, s);
    c->hv.download(hv.data(), ns, s);
    WT_CUDA(cudaStreamSynchronize(s));
    double vq = 0;
    for (int i = 0; i < ns; ++i) vq += hv[i] * hq[i];
    std::vector<double> hg(n1);
    for (int i = 1; i < ns; ++i) hg[i - 1] = -(hq[i] - c->beta * hv[i] * vq);
    g.upload(hg.data(), n1, s);
    c->amp.alloc(n1);
    dgemv(s, true, n1, n1, 1.0, U.p, n1, g.p, 0.0, c->amp.p);
    c->Vm.alloc((size_t)n1 * n1);
    copy_block(s, U.p, n1, c->Vm.p, n1, n1, n1);
    U.release();
    // q(t_n) = q_inf + Cn H [0; V (amp * exp(-mu t_n))]
    // an allocation-free Eq. 1 call may still read the previous time samples on its own stream
    if (c->noalloc_pending) {
        WT_CUDA(cudaStreamWaitEvent(s, c->ev_noalloc, 0));
        c->noalloc_pending = false;
    }
    if (!c->ev_noalloc) WT_CUDA(cudaEventCreateWithFlags(&c->ev_noalloc, cudaEventDisableTiming));
    c->d_times.upload(t, nt, s);
    DBuf<double> Q;
    Q.alloc((size_t)ns * nt);
    charges_at(c, c->d_times.p, nt, Q.p);
    c->Qt.alloc((size_t)nt * ns);
    transpose(s, Q.p, ns, nt, c->Qt.p);
    if (fault_enabled("nan_q")) fill(s, c->Qt.p, 1, std::nan(""));     // injected non-finite charge
    check_finite(s, c->Qt.p, (size_t)nt * ns, c->d_err.p);
    if (read_err(c)) fail(WT_ERR_NAN, "non-finite charges");
    // S5b: time basis of the charge history (Gram matrix + Jacobi)
    c->r_pad = 32;
    compress_history(c, Q.p, nt, c->Ub, c->W32, c->rank, c->info.trunc_rel);
    c->info.n_t = nt;
    c->info.rank = c->rank;
    c->info.relax_seconds = secs(t0);
}

void ensure_spectral(wt_ctx* c) {
    if (c->sp_ready) return;
    const wt_grid& g = c->grid;
    GridDev gd{g.Nx, g.Ny, g.Nz, g.Lx, g.Ly, g.Lz, c->pref};
    std::vector<double> xy;
    for (auto& col : c->cols) { xy.push_back(col.x); xy.push_back(col.y); }
    c->sp32.init(gd, xy, c->s);
    c->sp64.init(gd, xy, c->s);
    c->d_zsrc.upload(c->src_z.data(), c->ns, c->s);
    c->d_col_off.upload(c->col_off.data(), c->col_off.size(), c->s);
    c->zcos.alloc((size_t)c->ns * g.Nz);
    column_cos_table(c->s, c->d_zsrc.p, c->ns, g.Nz, g.Lz, c->zcos.p);
    WT_CUDA(cudaStreamSynchronize(c->s));
    c->sp_ready = true;
}

// FP32 fast path for a basis of charge vectors Ub [r][ns] and coefficients
// W32 [nt][32]: column transforms, basis fields (mode 0: the field, 1: its
// lateral-scale derivative) and the expansion into out [nt][3][npts].
// host_out != NULL: out is a device staging buffer; the expansion runs in time chunks and each
// chunk is copied to host_out on the context's copy stream while the next one is computed.
// Basis fields E32[c][m][p] (m < r) of the charge vectors Ub (column transform and the
// spectral passes), at the context's launch shapes.  Marks E32 as the relaxation's own fields
// when Ub is the context's basis (mode 0), as anything else otherwise.
// Bytes of the lateral tables of a context, and whether they are worth holding: at most 16 GiB and
// a quarter of the device memory free now.
size_t tables_bytes(const wt_ctx* c) {
    const wt_grid& g = c->grid;
    return c->cols.size() * (size_t)3 * g.Nz * g.Nx * g.Ny * sizeof(float);
}
bool tables_fit(const wt_ctx* c) {
    if (c->t32_ready) return true;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return false; }
    const size_t b = tables_bytes(c);
    return b <= ((size_t)16 << 30) && b <= fr / 4 && c->cols.size() <= 96;
}

// The lateral tables T_c (Sec. 3's fundamental-solution chunks in spectral form): the deposit and
// plane passes of one unit column z-transform per column, at the context's FFT shapes.
void build_tables(wt_ctx* c) {
    if (c->t32_ready) return;
    const wt_grid& g = c->grid;
    const int ncol = (int)c->cols.size();
    const size_t nxy = (size_t)g.Nx * g.Ny;
    cudaStream_t s = c->s;
    c->T32.alloc((size_t)ncol * 3 * g.Nz * nxy);
    std::vector<float> unit((size_t)ncol * ncol * g.Nz, 0.f);     // [k][c][kz] = (c == k)
    for (int k = 0; k < ncol; ++k)
        for (int z = 0; z < g.Nz; ++z) unit[((size_t)k * ncol + k) * g.Nz + z] = 1.f;
    DBuf<float> Zu;
    Zu.upload(unit.data(), unit.size(), s);
    c->rho32.alloc(c->sp32.rho_elems(std::max(1, c->tune_nb)));
    for (int k = 0; k < ncol; ++k)
        c->sp32.lateral(Zu.p + (size_t)k * ncol * g.Nz, 1, c->rho32.p, c->T32.p + (size_t)k * 3 * g.Nz * nxy, s, 0);
    WT_CUDA(cudaStreamSynchronize(s));
    c->t32_ready = true;
}

// Basis fields of Zc [r][n_cols][Nz] from the lateral tables: per slab of ys y rows, the
// combination of the tables' planes (into the L2-sized slab buffer) and the z pass.
// Slab buffers of the table path: one, or two for the pipelined form.
size_t slab_elems(const wt_ctx* c) { return (size_t)32 * 3 * c->grid.Nz * c->grid.Nx * c->tune_ys; }
void alloc_slabs(wt_ctx* c) {
    c->Rsl.alloc(slab_elems(c) * ((c->tune_tf & 1) ? 2 : 1));
    c->ZcT32.alloc((size_t)c->grid.Nz * c->cols.size() * 32);
}

// The second stream and the events of the pipelined table path (created once per context).
void ensure_aux(wt_ctx* c) {
    if (c->s_aux) return;
    WT_CUDA(cudaStreamCreateWithFlags(&c->s_aux, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        WT_CUDA(cudaEventCreateWithFlags(&c->ev_tc[k], cudaEventDisableTiming));
        WT_CUDA(cudaEventCreateWithFlags(&c->ev_tz[k], cudaEventDisableTiming));
    }
    WT_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
}

void spectral_tables(wt_ctx* c, const float* Zc, int r, cudaStream_t s) {
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz, nxy = (size_t)g.Nx * g.Ny;
    const int ncol = (int)c->cols.size(), ys = c->tune_ys;
    const bool pipe = c->tune_tf & 1, disc = c->tune_tf & 2;
    alloc_slabs(c);
    combine_coeffs(s, Zc, r, ncol, g.Nz, c->ZcT32.p);
    if (!pipe) {
        for (int y0 = 0; y0 < g.Ny; y0 += ys) {
            const int yn = std::min(ys, g.Ny - y0);
            column_combine(s, c->T32.p, c->ZcT32.p, r, ncol, g.Nz, nxy, (size_t)y0 * g.Nx, g.Nx * yn, c->Rsl.p,
                           c->tune_tf & 4);
            c->sp32.zlines(c->Rsl.p, r, y0, yn, c->E32.p, npts, (size_t)32 * npts, s, c->tune_lb, disc);
        }
        return;
    }
    // combination of slab k + 1 (stream s) overlaps the z pass of slab k (second stream); two slab
    // buffers, each reused once the z pass two slabs back has read it
    ensure_aux(c);
    const size_t se = slab_elems(c);
    WT_CUDA(cudaEventRecord(c->ev_fork, s));
    WT_CUDA(cudaStreamWaitEvent(c->s_aux, c->ev_fork, 0));
    int k = 0;
    for (int y0 = 0; y0 < g.Ny; y0 += ys, ++k) {
        const int yn = std::min(ys, g.Ny - y0), bi = k & 1;
        float* R = c->Rsl.p + bi * se;
        if (k >= 2) WT_CUDA(cudaStreamWaitEvent(s, c->ev_tz[bi], 0));
        column_combine(s, c->T32.p, c->ZcT32.p, r, ncol, g.Nz, nxy, (size_t)y0 * g.Nx, g.Nx * yn, R, c->tune_tf & 4);
        WT_CUDA(cudaEventRecord(c->ev_tc[bi], s));
        WT_CUDA(cudaStreamWaitEvent(c->s_aux, c->ev_tc[bi], 0));
        c->sp32.zlines(R, r, y0, yn, c->E32.p, npts, (size_t)32 * npts, c->s_aux, c->tune_lb, disc);
        WT_CUDA(cudaEventRecord(c->ev_tz[bi], c->s_aux));
    }
    for (int q = 0; q < std::min(k, 2); ++q) WT_CUDA(cudaStreamWaitEvent(s, c->ev_tz[q], 0));
}
bool use_tables(const wt_ctx* c, int mode) { return mode == 0 && c->tune_ys > 0 && c->t32_ready; }

void basis_fields32(wt_ctx* c, const double* Ub, int r, cudaStream_t s, int mode, int* launches, bool timing) {
    if (Ub == c->Ub.p) require_fp32_basis(c);
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int ncol = (int)c->cols.size();
    const int rp = 32;
    const int nb = c->tune_nb;      // charge vectors per spectral launch (1 keeps the intermediates in L2)
    const bool tc = c->use_tc && expand_tc_available();
    c->Zc32.alloc((size_t)rp * ncol * g.Nz);
    c->rho32.alloc(c->sp32.rho_elems(nb));
    c->R32.alloc(c->sp32.r_elems(nb));
    c->E32.alloc((size_t)3 * rp * npts);
    c->e32_stamp = 0;
    // the tensor-core expansion reads only the r rows in use; the FMA one reads all 32
    if (!tc && r < rp) WT_CUDA(cudaMemsetAsync(c->E32.p, 0, c->E32.n * sizeof(float), s));
    column_ztransform<float>(s, Ub, r, c->ns, c->ns, c->zcos.p, c->d_col_off.p, ncol, g.Nz, c->Zc32.p);
    *launches += 1;
    if (timing) WT_CUDA(cudaEventRecord(c->ev[1], s));
    if (use_tables(c, mode)) {
        spectral_tables(c, c->Zc32.p, r, s);
        *launches += 1 + 2 * ((g.Ny + c->tune_ys - 1) / c->tune_ys);
    } else {
        for (int m0 = 0; m0 < r; m0 += nb) {
            const int b = std::min(nb, r - m0);
            c->sp32.fields(c->Zc32.p + (size_t)m0 * ncol * g.Nz, b, c->rho32.p, c->R32.p,
                           c->E32.p + (size_t)m0 * npts, npts, (size_t)rp * npts, s, mode, c->tune_lb);
            *launches += 3;
        }
    }
    if (timing) WT_CUDA(cudaEventRecord(c->ev[2], s));
    if (mode == 0 && Ub == c->Ub.p && r == c->rank) c->e32_stamp = c->version;
}

void extend32_basis(wt_ctx* c, const double* Ub, int r, const float* W32, int nt, float* out, cudaStream_t s, int mode,
                    int* launches, bool timing, float* host_out = nullptr) {
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int rp = 32;
    const bool tc = c->use_tc && expand_tc_available();
    basis_fields32(c, Ub, r, s, mode, launches, timing);
    if (host_out) {
        // about 2 GB of H per chunk (whole 32-sample tiles): copies overlap the later chunks' expansion
        const size_t per_t = 3 * npts * sizeof(float);
        int tc_n = (int)std::max<size_t>(1, ((size_t)2 << 30) / per_t);
        tc_n = std::max(32, tc_n / 32 * 32);
        cudaEvent_t ev;
        WT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        for (int t0 = 0; t0 < nt; t0 += tc_n) {
            const int n = std::min(tc_n, nt - t0);
            float* o = out + (size_t)t0 * 3 * npts;
            if (tc) {
                ExpandJob jb{c->E32.p, rp, r, W32 + (size_t)t0 * rp, n, npts, o};
                expand_tc_jobs(s, &jb, 1, 0, c->tune_nch, c->d_err.p, c->tune_nepi, c->tune_vec);
            } else {
                expand_simt(s, c->E32.p, rp, W32 + (size_t)t0 * rp, n, rp, npts, o);
            }
            *launches += 1;
            WT_CUDA(cudaEventRecord(ev, s));
            WT_CUDA(cudaStreamWaitEvent(c->s_copy, ev, 0));
            WT_CUDA(cudaMemcpyAsync(host_out + (size_t)t0 * 3 * npts, o, (size_t)n * per_t, cudaMemcpyDeviceToHost,
                                    c->s_copy));
        }
        cudaEventDestroy(ev);
        if (timing) WT_CUDA(cudaEventRecord(c->ev[3], s));
        WT_CUDA(cudaStreamSynchronize(c->s_copy));
        return;
    }
    if (tc) {
        ExpandJob jb{c->E32.p, rp, r, W32, nt, npts, out};
        expand_tc_jobs(s, &jb, 1, 0, c->tune_nch, c->d_err.p, c->tune_nepi, c->tune_vec);
    } else {
        expand_simt(s, c->E32.p, rp, W32, nt, rp, npts, out);
    }
    *launches += 1;
    if (timing) WT_CUDA(cudaEventRecord(c->ev[3], s));
}

// FP64 plain path: one spectral transform per time sample into out [nt][3][npts].
void extend64(wt_ctx* c, double* out, cudaStream_t s, int* launches) {
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int nt = (int)c->times.size(), ncol = (int)c->cols.size();
    const int nb = 4;
    c->Zc64.alloc((size_t)nb * ncol * g.Nz);
    c->G64.alloc(c->sp64.scratch_elems(nb));
    for (int t0 = 0; t0 < nt; t0 += nb) {
        const int b = std::min(nb, nt - t0);
        column_ztransform<double>(s, c->Qt.p + (size_t)t0 * c->ns, b, c->ns, c->ns, c->zcos.p, c->d_col_off.p, ncol,
                                  g.Nz, c->Zc64.p);
        c->sp64.fields(c->Zc64.p, b, c->G64.p, out + (size_t)t0 * 3 * npts, 3 * npts, npts, s);
        *launches += 4;
    }
}

void tune_context(wt_ctx* c, float* H);

void do_extend(wt_ctx* c, wt_precision prec, void* H, size_t bytes, cudaStream_t us) {
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int nt = (int)c->times.size();
    const size_t esz = prec == WT_FP64 ? 8 : 4;
    const size_t need = (size_t)nt * 3 * npts * esz;
    if (!H) fail(WT_ERR_ARG, "H is NULL");
    if (bytes < need) fail(WT_ERR_ARG, "H_bytes too small: need " + std::to_string(need));
    ensure_spectral(c);
    const bool dev = is_device_ptr(H);
    cudaStream_t s = us;
    if (!dev) {  // compute into an internal buffer on the context stream, then copy out
        s = c->s;
        if (prec == WT_FP64) c->stage64.alloc((size_t)nt * 3 * npts);
        else c->stage32.alloc((size_t)nt * 3 * npts);
    }
    const int ncol = (int)c->cols.size();
    if (c->timing) {
        for (int k = 0; k < 4; ++k)
            if (!c->ev[k]) WT_CUDA(cudaEventCreate(&c->ev[k]));
        WT_CUDA(cudaEventRecord(c->ev[0], s));
    }
    int launches = 0;
    if (prec == WT_FP64) {
        double* out = dev ? static_cast<double*>(H) : c->stage64.p;
        extend64(c, out, s, &launches);
        if (c->timing) {
            WT_CUDA(cudaEventRecord(c->ev[1], s));
            WT_CUDA(cudaEventRecord(c->ev[2], s));
            WT_CUDA(cudaEventRecord(c->ev[3], s));
        }
    } else {
        float* out = dev ? static_cast<float*>(H) : c->stage32.p;
        if (!c->tuned) {
            // first FP32 extension: pick the launch shapes, writing trial results into out, after
            // the caller's pending work on its stream and before this extension
            cudaEvent_t e;
            WT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            WT_CUDA(cudaEventRecord(e, s));
            WT_CUDA(cudaStreamWaitEvent(c->s, e, 0));
            cudaEventDestroy(e);
            tune_context(c, out);
            if (c->timing) WT_CUDA(cudaEventRecord(c->ev[0], s));
        }
        extend32_basis(c, c->Ub.p, c->rank, c->W32.p, nt, out, s, 0, &launches, c->timing,
                       dev ? nullptr : static_cast<float*>(H));
    }
    c->last_launches = launches;
    c->ev_recorded = c->timing;
    if (!dev && prec == WT_FP32) {           // copied out chunk by chunk above; synchronous: report now
        const int e = read_err(c);
        if (e) {
            clear_err(c);
            fail(e == DERR_TIMEOUT ? WT_ERR_TIMEOUT : WT_ERR_NAN, "device-side failure during the extension");
        }
        return;
    }
    if (!dev) {
        const void* src = prec == WT_FP64 ? (const void*)c->stage64.p : (const void*)c->stage32.p;
        WT_CUDA(cudaMemcpyAsync(H, src, need, cudaMemcpyDeviceToHost, s));
        WT_CUDA(cudaStreamSynchronize(s));
    }
    if (!dev) {       // synchronous: report a device-side failure now (device H: at wt_sync)
        const int e = read_err(c);
        if (e) {
            clear_err(c);
            fail(e == DERR_TIMEOUT ? WT_ERR_TIMEOUT : WT_ERR_NAN, "device-side failure during the extension");
        }
    }
}


void do_sample(wt_ctx* c, const double* xyz, int n, const double* t, int nt, double* out) {
    ensure_spectral(c);
    cudaStream_t s = c->s;
    const wt_grid& g = c->grid;
    const int ns = c->ns, ncol = (int)c->cols.size();
    for (int i = 0; i < nt; ++i)
        if (!(t[i] >= 0.0) || !std::isfinite(t[i])) fail(WT_ERR_ARG, "sample times must be finite and >= 0");
    for (int i = 0; i < 3 * n; ++i)
        if (!std::isfinite(xyz[i])) fail(WT_ERR_NAN, "non-finite sample point");
    DBuf<double> dt_, Q, Qt, Zc, T, Lat, pts, o;
    dt_.upload(t, nt, s);
    Q.alloc((size_t)ns * nt);
    charges_at(c, dt_.p, nt, Q.p);
    Qt.alloc((size_t)nt * ns);
    transpose(s, Q.p, ns, nt, Qt.p);
    Zc.alloc((size_t)nt * ncol * g.Nz);
    column_ztransform<double>(s, Qt.p, nt, ns, ns, c->zcos.p, c->d_col_off.p, ncol, g.Nz, Zc.p);
    T.alloc((size_t)(g.Nx / 2) * (g.Ny / 2) * g.Nz);
    green_invk2(s, g.Nx, g.Ny, g.Nz, g.Lx, g.Ly, g.Lz, T.p);
    const int chunk = 512;
    Lat.alloc((size_t)std::min(n, chunk) * ncol * g.Nz * 3);
    o.alloc((size_t)nt * std::min(n, chunk) * 3);
    std::vector<double> hbuf;
    for (int p0 = 0; p0 < n; p0 += chunk) {
        const int np = std::min(chunk, n - p0);
        pts.upload(xyz + 3 * (size_t)p0, 3 * (size_t)np, s);
        sample_lateral(s, pts.p, np, c->sp64.col_xy.p, ncol, g.Nx, g.Ny, g.Nz, g.Lx, g.Ly, T.p, Lat.p);
        sample_contract(s, pts.p, Lat.p, Zc.p, np, nt, ncol, g.Nz, g.Lz, c->pref, o.p);
        hbuf.resize((size_t)nt * np * 3);
        o.download(hbuf.data(), hbuf.size(), s);
        WT_CUDA(cudaStreamSynchronize(s));
        for (int tt = 0; tt < nt; ++tt)
            std::memcpy(out + ((size_t)tt * n + p0) * 3, hbuf.data() + (size_t)tt * np * 3, sizeof(double) * np * 3);
    }
}

// Lag table of Eq. 1: (k + 1/2) dt -> bracketing samples and weights (linear
// in t; 0 at t = 0; held after the last sample).
// Returns the count of time samples the table reads (samples n0 and n0 + 1 of every lag; n0 grows
// with the lag), so that the kernels stage no sample beyond it.
int build_lags(wt_ctx* c, double dt, int n_out, DBuf<unsigned char>& dlag, cudaStream_t s, bool f64 = false) {
    const int nt = (int)c->times.size();
    int n0_max = 0;
    const size_t esz = f64 ? eq1_lag64_size() : eq1_lag_size();
    std::vector<unsigned char> lag(esz * (size_t)n_out);
    const std::vector<double>& ts = c->times;
    for (int k = 0; k < n_out; ++k) {
        const double L = (k + 0.5) * dt;
        int n0 = 0;
        double w0 = 0, w1 = 0;
        if (L <= ts.front()) { n0 = 0; w0 = L / ts.front(); }
        else if (L >= ts.back()) { n0 = nt - 1; w0 = 1.0; }
        else {
            n0 = (int)(std::upper_bound(ts.begin(), ts.end(), L) - ts.begin()) - 1;
            const double f = (L - ts[n0]) / (ts[n0 + 1] - ts[n0]);
            w0 = 1.0 - f;
            w1 = f;
        }
        if (f64) eq1_pack_lag64(lag.data() + esz * k, n0, w0, w1);
        else eq1_pack_lag(lag.data() + esz * k, n0, (float)w0, (float)w1);
        n0_max = std::max(n0_max, n0);
    }
    dlag.upload(lag.data(), lag.size(), s);
    return std::min(nt, n0_max + 2);
}
// The same count for a table built on the device by the same rule (the allocation-free call),
// from the longest lag, with one sample of margin.
int lag_samples_used(const std::vector<double>& ts, double dt, int n_out) {
    const int nt = (int)ts.size();
    const double L = (n_out - 0.5) * dt;
    int n0 = 0;
    if (L >= ts.back()) n0 = nt - 1;
    else if (L > ts.front()) n0 = (int)(std::upper_bound(ts.begin(), ts.end(), L) - ts.begin()) - 1;
    return std::min(nt, n0 + 3);
}

struct TrackDev {
    const float *x, *y, *z, *vx, *vy, *vz, *q;
    float qconst;
    int n_tracks, n_steps, n_out;
    double dt;
};

void check_tracks(const wt_tracks* tr) {
    if (!tr) fail(WT_ERR_ARG, "NULL tracks");
    if (tr->n_tracks < 0 || tr->n_steps < 1 || tr->n_out < 1 || !(tr->dt > 0.0))
        fail(WT_ERR_ARG, "bad track sizes or dt");
}

// Device view of the tracks; host arrays are copied into `keep`.
TrackDev stage_tracks(wt_ctx* c, const wt_tracks* tr, DBuf<float> (&keep)[7], cudaStream_t s) {
    if (!tr->x || !tr->y || !tr->z || !tr->vx || !tr->vy || !tr->vz) fail(WT_ERR_ARG, "NULL track array");
    const size_t nts = (size_t)tr->n_tracks * tr->n_steps;
    const float* arr[7] = {tr->x, tr->y, tr->z, tr->vx, tr->vy, tr->vz, tr->q};
    if (!is_device_ptr(tr->x)) {
        for (int k = 0; k < 6; ++k) { keep[k].upload(arr[k], nts, s); arr[k] = keep[k].p; }
        if (tr->q) { keep[6].upload(tr->q, tr->n_tracks, s); arr[6] = keep[6].p; }
    }
    return TrackDev{arr[0], arr[1], arr[2], arr[3], arr[4], arr[5], tr->q ? arr[6] : nullptr, (float)tr->charge,
                    tr->n_tracks, tr->n_steps, tr->n_out, tr->dt};
}

// h64: FP64 field, FP64 lag weights and FP64 currents (out is double*); else all FP32 (float*).
void eq1_run(wt_ctx* c, const void* H, bool h64, const TrackDev& t, void* out, cudaStream_t s,
             const float* vz_override = nullptr) {
    const wt_grid& g = c->grid;
    const int nt = (int)c->times.size();
    DBuf<unsigned char> dlag;
    const int nu = build_lags(c, t.dt, t.n_out, dlag, s, h64);
    const float* vz = vz_override ? vz_override : t.vz;
    if (h64)
        eq1_launch64(s, static_cast<const double*>(H), g.Nx, g.Ny, g.Nz, nt, g.Lx, g.Ly, g.Lz, t.x, t.y, t.z, t.vx,
                     t.vy, vz, t.q, t.qconst, t.n_tracks, t.n_steps, t.n_out, t.dt, c->opts.v_w, dlag.p, nu,
                     static_cast<double*>(out));
    else
        eq1_launch(s, static_cast<const float*>(H), g.Nx, g.Ny, g.Nz, nt, g.Lx, g.Ly, g.Lz, t.x, t.y, t.z, t.vx, t.vy,
                   vz, t.q, t.qconst, t.n_tracks, t.n_steps, t.n_out, t.dt, c->opts.v_w, dlag.p, nu,
                   static_cast<float*>(out));
    WT_CUDA(cudaStreamSynchronize(s));   // the lag table is freed on return
}

void do_eq1(wt_ctx* c, const void* H, const wt_tracks* tr, float* iout, cudaStream_t us) {
    check_tracks(tr);
    if (tr->n_tracks == 0) return;     // nothing to convolve; no pointer is read
    if (!H || !iout) fail(WT_ERR_ARG, "NULL argument");
    if (!is_device_ptr(H)) fail(WT_ERR_ARG, "H must be device memory (FP32 output of wt_extend)");
    const bool dev_in = is_device_ptr(tr->x);
    const bool dev_out = is_device_ptr(iout);
    cudaStream_t s = (dev_in && dev_out) ? us : c->s;
    DBuf<float> keep[7];
    const TrackDev td = stage_tracks(c, tr, keep, s);
    DBuf<float> dout;
    float* o = iout;
    if (!dev_out) { dout.alloc((size_t)tr->n_tracks * tr->n_out); o = dout.p; }
    eq1_run(c, H, false, td, o, s);
    if (!dev_out) {
        dout.download(iout, (size_t)tr->n_tracks * tr->n_out, s);
        WT_CUDA(cudaStreamSynchronize(s));
    }
}

// Eq. 1 from the rank-r form of the FP32 field (the context's basis fields E32 and time
// coefficients W32), without writing H; the basis fields are computed when E32 does not hold
// them already.
void eq1_basis_run(wt_ctx* c, const float* E, int r, const float* W32, const TrackDev& t, float* out, cudaStream_t s,
                   const float* vz_override = nullptr) {
    const wt_grid& g = c->grid;
    const int nt = (int)c->times.size();
    DBuf<unsigned char> dlag;
    const int nu = build_lags(c, t.dt, t.n_out, dlag, s, false);
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    c->Ep32.alloc(npts * 96);
    eq1_point_major(s, E, r, npts, c->Ep32.p);
    eq1_basis_launch(s, c->Ep32.p, r, W32, g.Nx, g.Ny, g.Nz, nt, g.Lx, g.Ly, g.Lz, t.x, t.y, t.z, t.vx, t.vy,
                     vz_override ? vz_override : t.vz, t.q, t.qconst, t.n_tracks, t.n_steps, t.n_out, t.dt,
                     c->opts.v_w, dlag.p, nu, out);
    WT_CUDA(cudaStreamSynchronize(s));   // the lag table is freed on return
}

void ensure_base_fields(wt_ctx* c, cudaStream_t s) {
    ensure_spectral(c);
    if (c->e32_stamp == c->version && c->E32.p) return;
    int launches = 0;
    basis_fields32(c, c->Ub.p, c->rank, s, 0, &launches, false);
}

void do_eq1_direct(wt_ctx* c, const wt_tracks* tr, float* iout, cudaStream_t us) {
    check_tracks(tr);
    if (tr->n_tracks == 0) return;
    if (!iout) fail(WT_ERR_ARG, "NULL argument");
    const bool dev_in = is_device_ptr(tr->x);
    const bool dev_out = is_device_ptr(iout);
    cudaStream_t s = c->s;
    if (dev_in && dev_out && us != s) {       // after the caller's pending work on its stream
        cudaEvent_t ev;
        WT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        WT_CUDA(cudaEventRecord(ev, us));
        WT_CUDA(cudaStreamWaitEvent(s, ev, 0));
        cudaEventDestroy(ev);
    }
    DBuf<float> keep[7];
    const TrackDev td = stage_tracks(c, tr, keep, s);
    ensure_base_fields(c, s);
    DBuf<float> dout;
    float* o = iout;
    if (!dev_out) { dout.alloc((size_t)tr->n_tracks * tr->n_out); o = dout.p; }
    eq1_basis_run(c, c->E32.p, c->rank, c->W32.p, td, o, s);
    if (!dev_out) {
        dout.download(iout, (size_t)tr->n_tracks * tr->n_out, s);
        WT_CUDA(cudaStreamSynchronize(s));
    }
    if (read_err(c)) fail(WT_ERR_TIMEOUT, "device wait timed out");
}

// H M (right Householder product) for M rows x ns, in place.
void house_right(wt_ctx* c, double* M, int rows) {
    DBuf<double> w;
    w.alloc(rows);
    dgemv(c->s, false, rows, c->ns, 1.0, M, c->ns, c->hv.p, 0.0, w.p);
    rank1(c->s, rows, c->ns, -c->beta, w.p, c->hv.p, M, c->ns);
}
// H M (left Householder product) for M ns x cols, in place.
void house_left(wt_ctx* c, double* M, int cols) {
    DBuf<double> u;
    u.alloc(cols);
    dgemv(c->s, true, c->ns, cols, 1.0, M, cols, c->hv.p, 0.0, u.p);
    rank1(c->s, c->ns, cols, -c->beta, c->hv.p, u.p, M, cols);
}

double do_loss(wt_ctx* c, wt_precision prec, const wt_tracks* tr) {
    check_tracks(tr);
    ensure_spectral(c);
    cudaStream_t s = c->s;
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int nt = (int)c->times.size();
    if (tr->n_tracks == 0) return 0.0;
    DBuf<float> keep[7];
    const TrackDev td = stage_tracks(c, tr, keep, s);
    int launches = 0;
    const size_t nI = (size_t)tr->n_tracks * tr->n_out;
    double sum;
    if (prec == WT_FP64) {
        c->stage64.alloc((size_t)nt * 3 * npts);
        extend64(c, c->stage64.p, s, &launches);
        DBuf<double> I;
        I.alloc(nI);
        eq1_run(c, c->stage64.p, true, td, I.p, s);
        sum = dot_f64(s, I.p, I.p, nI, c->d_scr.p);
    } else {
        // FP32 field in its rank-r form: no H is written
        ensure_base_fields(c, s);
        DBuf<float> I;
        I.alloc(nI);
        eq1_basis_run(c, c->E32.p, c->rank, c->W32.p, td, I.p, s);
        sum = dot_f32(s, I.p, I.p, nI, c->d_scr.p);
    }
    if (read_err(c)) fail(WT_ERR_TIMEOUT, "device wait timed out");
    return sum / (double)nI;
}

// Derivative of L = mean i^2 with respect to [readout resistivity scale, bias
// resistivity scale, radius, lateral scale], tangent-linear through the fit,
// the relaxation modes, the extension and Eq. 1 (see include/wt.h).
// Per-segment derivative of the resistive line along a relative node-resistivity
// perturbation delta (rho_j -> rho_j (1 + eps delta_j)): dd, doff, dk1 as K's diag,
// off-diagonal and K 1 (conductances ~ 1 / (rho_j + rho_j+1), terminal ~ 1 / rho_t).
void kline_direction(const wt_ctx* c, const double* delta, std::vector<double>& dd, std::vector<double>& doff,
                     std::vector<double>& dk1) {
    const int ns = c->ns;
    dd.assign(ns, 0.0);
    doff.assign(ns, 0.0);
    dk1.assign(ns, 0.0);
    for (size_t k = 0; k < c->cols.size(); ++k) {
        const wt_column& col = c->cols[k];
        const int m = col.n_sources, o = c->col_off[k];
        auto rho = [&](int j) { return c->rho_prof[k].empty() ? col.resistivity : c->rho_prof[k][j]; };
        for (int j = 0; j + 1 < m; ++j) {
            const double g = c->k_off[o + j];
            const double dg = -g * (rho(j) * delta[o + j] + rho(j + 1) * delta[o + j + 1]) / (rho(j) + rho(j + 1));
            doff[o + j] = dg;
            dd[o + j] -= dg;
            dd[o + j + 1] -= dg;
        }
        const int jt = o + (col.terminal_top ? m - 1 : 0);
        const double dgt = c->k_k1[jt] * delta[jt];      // k1 = -g_t, so d g_t = -g_t delta_t = k1 delta_t
        dd[jt] -= dgt;                                   // K_tt holds -g_t, K 1 at t is -g_t
        dk1[jt] = -dgt;
    }
}

// I_out ([n_tracks][n_out]) and dI_out ([4][n_tracks][n_out]), device, optional: the currents and their
// tangents (parameters 0..3 only).
// CUDA events at the stage boundaries of one loss derivative (timing on): the time between a mark and
// the previous one goes to the stage the later mark names.
struct StageClock {
    cudaStream_t s = nullptr;
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> stage;
    void mark(int k) {
        if (!on) return;
        cudaEvent_t e;
        WT_CUDA(cudaEventCreate(&e));
        WT_CUDA(cudaEventRecord(e, s));
        ev.push_back(e);
        stage.push_back(k);
    }
    void finish(double* ms, int n) {
        if (!on || ev.empty()) return;
        WT_CUDA(cudaEventSynchronize(ev.back()));
        for (int k = 0; k < n; ++k) ms[k] = 0.0;
        for (size_t i = 1; i < ev.size(); ++i) {
            float t = 0.f;
            WT_CUDA(cudaEventElapsedTime(&t, ev[i - 1], ev[i]));
            if (stage[i] >= 0 && stage[i] < n) ms[stage[i]] += t;
        }
    }
    ~StageClock() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

void do_loss_grad(wt_ctx* c, const wt_tracks* tr, double* loss, double* grad, const double* delta = nullptr,
                  float* I_out = nullptr, float* dI_out = nullptr) {
    check_tracks(tr);
    if (c->opts.tikhonov > 0.0) fail(WT_ERR_UNSUPPORTED, "the derivative assumes an unregularised fit");
    ensure_spectral(c);
    cudaStream_t s = c->s;
    const wt_grid& g = c->grid;
    const int ns = c->ns, n1 = ns - 1, nc = c->nc, ncol = (int)c->cols.size();
    const int nt = (int)c->times.size();
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int n_out_params = delta ? 1 : 4;
    for (int k = 0; k < n_out_params; ++k) grad[k] = 0.0;
    *loss = 0.0;
    if (tr->n_tracks == 0) return;
    DBuf<float> keep[7];
    const TrackDev td = stage_tracks(c, tr, keep, s);
    const size_t nI = (size_t)tr->n_tracks * tr->n_out;
    int launches = 0;
    clear_err(c);
    c->info.grad_trunc_rel = 0.0;
    StageClock clock;
    clock.s = s;
    clock.on = c->timing;
    for (double& v : c->grad_ms) v = 0.0;
    clock.mark(-1);
    // base field and currents
    c->stage32.alloc((size_t)nt * 3 * npts);
    extend32_basis(c, c->Ub.p, c->rank, c->W32.p, nt, c->stage32.p, s, 0, &launches, false);
    DBuf<float> I, dI;
    I.alloc(nI);
    dI.alloc(nI);
    eq1_run(c, c->stage32.p, false, td, I.p, s);
    if (I_out) WT_CUDA(cudaMemcpyAsync(I_out, I.p, nI * sizeof(float), cudaMemcpyDeviceToDevice, s));
    *loss = dot_f32(s, I.p, I.p, nI, c->d_scr.p) / (double)nI;
    const double gscale = 2.0 / (double)nI;
    clock.mark(0);

    // shared pieces: fit residual, modal factors, inverse gaps, potentials Phi(t)
    DBuf<int> sp, si;
    DBuf<double> sw, Rs, E, AE, ones, invg, Phi, dphi;
    sp.upload(c->s_ptr.data(), c->s_ptr.size(), s);
    si.upload(c->s_idx.data(), c->s_idx.size(), s);
    sw.upload(c->s_w.data(), c->s_w.size(), s);
    Rs.alloc((size_t)nc * ns);
    dgemm(s, false, false, nc, ns, ns, -1.0, c->fitA.p, ns, c->fitY.p, ns, 0.0, Rs.p, ns);
    fit_add_s(s, Rs.p, ns, ns, sp.p, si.p, sw.p, 1.0);
    std::vector<double> h1(n1, 1.0);
    ones.upload(h1.data(), n1, s);
    E.alloc((size_t)n1 * nt);
    modal_factors(s, ones.p, c->mu.p, n1, c->d_times.p, nt, E.p);
    AE.alloc((size_t)n1 * nt);
    modal_factors(s, c->amp.p, c->mu.p, n1, c->d_times.p, nt, AE.p);
    invg.alloc((size_t)n1 * n1);
    modal_inv_gap(s, c->mu.p, n1, invg.p);
    Phi.alloc((size_t)ns * nt);
    Phi.zero(s);
    dgemm(s, false, false, n1, nt, n1, 1.0, c->Vm.p, n1, AE.p, nt, 0.0, Phi.p + nt, nt);
    house_left(c, Phi.p, nt);
    dphi.upload(c->phi_dc.data(), ns, s);
    add_row_const(s, Phi.p, ns, nt, dphi.p);
    // tables for the derivative of the fit matrix
    DBuf<double> zc_all, zs_all, Ct, Cs, ddxy, duxy, Ld;
    DBuf<unsigned char> dblocks;
    zc_all.upload(c->f_hzc.data(), c->f_hzc.size(), s);
    zs_all.upload(c->src_z.data(), ns, s);
    Ct.alloc(c->f_hzc.size() * g.Nz);
    Cs.alloc((size_t)ns * g.Nz);
    green_cos_table(s, zc_all.p, (int)c->f_hzc.size(), g.Nz, g.Lz, Ct.p);
    green_cos_table(s, zs_all.p, ns, g.Nz, g.Lz, Cs.p);
    ddxy.upload(c->f_dxy.data(), c->f_dxy.size(), s);
    dblocks.upload(c->f_blocks.data(), c->f_blocks.size(), s);
    Ld.alloc((size_t)c->f_ncombo * g.Nz);
    DBuf<float> dH, zeros;
    dH.alloc((size_t)nt * 3 * npts);
    zeros.alloc((size_t)td.n_tracks * td.n_steps);
    zeros.zero(s);
    clock.mark(1);
    DBuf<double> dCn, dKt, T, tmp, dP, Sh, Ah, Om, Mm, cm, dz, dQ, dQq, dgv, dqi;
    // parameters 0..3 (s_R, s_B, r, lambda), or 4: the node-resistivity direction delta
    const int p_first = delta ? 4 : 0, p_last = delta ? 4 : 3;
    for (int p = p_first; p <= p_last; ++p) {
        const bool has_dc = p == 2 || p == 3, has_dk = p != 3;
        // ---- fit tangent: dC_n
        if (has_dc) {
            std::vector<double> uxy(c->f_uxy);
            if (p == 3) {      // lateral scale: the radial offset r_c (ux, uy) of the target column
                const int n_az = c->opts.n_az;
                for (int cb = 0; cb < c->f_ncombo; ++cb) {
                    const int k = (cb / ncol) / n_az;
                    uxy[2 * cb] *= c->cols[k].radius;
                    uxy[2 * cb + 1] *= c->cols[k].radius;
                }
            }
            duxy.upload(uxy.data(), uxy.size(), s);
            green_lateral_deriv(s, ddxy.p, duxy.p, c->f_ncombo, g.Nx, g.Ny, g.Nz, g.Lx, g.Ly, g.Lz, 1.0, p - 2, Ld.p);
            dP.alloc((size_t)nc * ns);
            green_pblocks(s, dblocks.p, c->f_ncombo, c->f_maxrows, c->f_maxcols, Ct.p, Cs.p, Ld.p, g.Nz, c->pref,
                          dP.p, ns);
            house_right(c, dP.p, nc);
            set_column(s, dP.p, nc, ns, 0, 0.0);
            scale_columns(s, dP.p, nc, ns, ns, c->fitD.p);                    // dA_s
            // T = dA_s^T R - (A_s^T dA_s) Y: the collocation-long contraction A_s^T dA_s once, then
            // the N_s-long product with Y (4 N_c N_s^2 + 2 N_s^3 flop instead of 6 N_c N_s^2 for
            // A_s^T (dA_s Y))
            tmp.alloc((size_t)ns * ns);
            dgemm(s, true, false, ns, ns, nc, 1.0, c->fitA.p, ns, dP.p, ns, 0.0, tmp.p, ns);
            T.alloc((size_t)ns * ns);
            dgemm(s, false, false, ns, ns, ns, -1.0, tmp.p, ns, c->fitY.p, ns, 0.0, T.p, ns);
            dgemm(s, true, false, ns, ns, nc, 1.0, dP.p, ns, Rs.p, ns, 1.0, T.p, ns);
            trsm_lower(s, c->fitL.p, ns, ns, T.p, ns, ns);
            trsm_lower_t(s, c->fitL.p, ns, ns, T.p, ns, ns);
            scale_rows(s, T.p, ns, ns, ns, c->fitD.p);                        // dX
            fill(s, T.p, ns, 0.0);
            house_left(c, T.p, ns);                                          // dF
            dCn.alloc((size_t)ns * ns);
            symmetrize_avg(s, T.p, dCn.p, ns);
            clock.mark(2);
        }
        // ---- resistive-line tangent: dK~
        if (has_dk) {
            std::vector<double> dd(ns, 0.0), doff(ns, 0.0), dk1(ns, 0.0);
            if (p == 4) {
                kline_direction(c, delta, dd, doff, dk1);
            } else {
                for (int k = 0; k < ncol; ++k) {
                    const wt_column& col = c->cols[k];
                    double f = 0.0;
                    if (p == 0 && col.terminal_top) f = -1.0;        // G ~ 1/rho: dG/ds = -G
                    if (p == 1 && !col.terminal_top) f = -1.0;
                    if (p == 2) f = 2.0 / col.radius;                  // G ~ r^2
                    for (int j = c->col_off[k]; j < c->col_off[k + 1]; ++j) {
                        dd[j] = f * c->k_diag[j];
                        doff[j] = f * c->k_off[j];
                        dk1[j] = f * c->k_k1[j];
                    }
                }
            }
            double s1 = 0, ds1 = 0;
            for (int j = 0; j < ns; ++j) { s1 += c->k_k1[j]; ds1 += dk1[j]; }
            DBuf<double> d_dd, d_doff, d_dk1, d_k1;
            d_dd.upload(dd.data(), ns, s);
            d_doff.upload(doff.data(), ns, s);
            d_dk1.upload(dk1.data(), ns, s);
            d_k1.upload(c->k_k1.data(), ns, s);
            dKt.alloc((size_t)ns * ns);
            build_k(s, d_dd.p, d_doff.p, ns, dKt.p);
            rank1(s, ns, ns, -1.0 / s1, d_dk1.p, d_k1.p, dKt.p, ns);
            rank1(s, ns, ns, -1.0 / s1, d_k1.p, d_dk1.p, dKt.p, ns);
            rank1(s, ns, ns, ds1 / (s1 * s1), d_k1.p, d_k1.p, dKt.p, ns);
            WT_CUDA(cudaStreamSynchronize(s));
        }
        // ---- modal tangent: Omega = V^T dS_m V - V^T dA_m V diag(mu)
        tmp.alloc((size_t)n1 * n1);
        Om.alloc((size_t)n1 * n1);
        Sh.alloc((size_t)n1 * n1);
        Sh.zero(s);
        if (has_dk) {
            householder_two_sided(c, dKt.p, ns);
            dgemm(s, false, false, n1, n1, n1, -1.0, dKt.p + ns + 1, ns, c->Vm.p, n1, 0.0, tmp.p, n1);   // dS_m V
            dgemm(s, true, false, n1, n1, n1, 1.0, c->Vm.p, n1, tmp.p, n1, 0.0, Sh.p, n1);
        }
        Ah.alloc((size_t)n1 * n1);
        Ah.zero(s);
        if (has_dc) {
            DBuf<double> HC;
            HC.alloc((size_t)ns * ns);
            copy_block(s, dCn.p, ns, HC.p, ns, ns, ns);
            householder_two_sided(c, HC.p, ns);
            dgemm(s, false, false, n1, n1, n1, 1.0, HC.p + ns + 1, ns, c->Vm.p, n1, 0.0, tmp.p, n1);
            dgemm(s, true, false, n1, n1, n1, 1.0, c->Vm.p, n1, tmp.p, n1, 0.0, Ah.p, n1);
        }
        modal_omega(s, Sh.p, has_dc ? Ah.p : nullptr, c->mu.p, n1, Om.p);
        // c_mod = V^T dg - Ah amp, dg = -(H dq_inf)[1:], dq_inf = dC_n phi_DC
        cm.alloc(n1);
        cm.zero(s);
        if (has_dc) {
            dqi.alloc(ns);
            dgemv(s, false, ns, ns, 1.0, dCn.p, ns, dphi.p, 0.0, dqi.p);
            house_left(c, dqi.p, 1);
            dgemv(s, true, n1, n1, -1.0, c->Vm.p, n1, dqi.p + 1, 0.0, cm.p);
            dgemv(s, false, n1, n1, -1.0, Ah.p, n1, c->amp.p, 1.0, cm.p);
        }
        dz.alloc((size_t)n1 * nt);
        modal_tangent(s, Om.p, c->amp.p, invg.p, E.p, c->d_times.p, cm.p, n1, nt, dz.p);
        // dQ = C_n H [0; V dzeta] + dC_n Phi      [ns][nt]
        dQ.alloc((size_t)ns * nt);
        dQ.zero(s);
        dgemm(s, false, false, n1, nt, n1, 1.0, c->Vm.p, n1, dz.p, nt, 0.0, dQ.p + nt, nt);
        house_left(c, dQ.p, nt);
        dQq.alloc((size_t)ns * nt);
        dgemm(s, false, false, ns, nt, ns, 1.0, c->Cn.p, ns, dQ.p, nt, 0.0, dQq.p, nt);
        if (has_dc) dgemm(s, false, false, ns, nt, ns, 1.0, dCn.p, ns, Phi.p, nt, 1.0, dQq.p, nt);
        check_finite(s, dQq.p, (size_t)ns * nt, c->d_err.p);
        clock.mark(3);
        // field and current tangents
        DBuf<double> dUb;
        DBuf<float> dW;
        int dr = 0;
        double dtr = 0.0;
        compress_history(c, dQq.p, nt, dUb, dW, dr, dtr);
        clock.mark(4);
        c->info.grad_trunc_rel = std::max(c->info.grad_trunc_rel, dtr);
        extend32_basis(c, dUb.p, dr, dW.p, nt, dH.p, s, 0, &launches, false);
        eq1_run(c, dH.p, false, td, dI.p, s);
        float* dIo = (dI_out && p < 4) ? dI_out + (size_t)p * nI : nullptr;
        if (dIo) WT_CUDA(cudaMemcpyAsync(dIo, dI.p, nI * sizeof(float), cudaMemcpyDeviceToDevice, s));
        double acc = dot_f32(s, I.p, dI.p, nI, c->d_scr.p);
        if (p == 3) {
            // derivative of the field operator itself, and of the lateral velocities
            extend32_basis(c, c->Ub.p, c->rank, c->W32.p, nt, dH.p, s, 1, &launches, false);
            eq1_run(c, dH.p, false, td, dI.p, s);
            acc += dot_f32(s, I.p, dI.p, nI, c->d_scr.p);
            if (dIo) add_f32(s, nI, dI.p, dIo);
            eq1_run(c, c->stage32.p, false, td, dI.p, s, zeros.p);
            acc += dot_f32(s, I.p, dI.p, nI, c->d_scr.p);
            if (dIo) add_f32(s, nI, dI.p, dIo);
        }
        grad[p - p_first] = gscale * acc;
        clock.mark(5);
        if (read_err(c)) fail(WT_ERR_NAN, "non-finite or timed-out tangent");
    }
    clock.finish(c->grad_ms, 6);
}

}  // namespace

// ---------------------------------------------------------------- batched FP32 path
// One entry per context of a captured batch: what the graph's nodes point at.
struct BatchEntry {
    wt_ctx* c;
    unsigned long long uid, version;
    const void* H;
    const void *E, *Zc, *rho, *R, *Ub, *W, *T, *Rsl;
    int nb, lb, rxy, rz, xd, tp, ys, tf;
    bool operator==(const BatchEntry& o) const {
        return c == o.c && uid == o.uid && version == o.version && H == o.H && E == o.E && Zc == o.Zc &&
               rho == o.rho && R == o.R && Ub == o.Ub && W == o.W && T == o.T && Rsl == o.Rsl && nb == o.nb &&
               lb == o.lb && rxy == o.rxy && rz == o.rz && xd == o.xd && tp == o.tp && ys == o.ys && tf == o.tf;
    }
};

struct BatchPlan {
    std::vector<BatchEntry> ents;
    int nch = 256, nepi = 8, vec = 4;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long last_use = 0;
    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

wt_ctx::~wt_ctx() = default;

namespace {

struct TuneResult {
    int nb, lb, nch, nepi, rxy, rz, xd, tp, vec;   // tp: two-pass FFTs, bits: 1 z pass, 2 y, 4 x transforms
    double spectral_ms, expand_ms;
    int ys;                                         // > 0: lateral tables, y slabs of ys rows
    int tf;                                         // table path flags (pipelined slabs, L2 discard)
};
using TuneKey = std::tuple<int, int, int, int, int, int>;   // device, Nx, Ny, Nz, n_t, columns
std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune;
std::atomic<unsigned long long> g_plan_clock{0};

TuneKey tune_key(const wt_ctx* c) {
    return TuneKey{c->dev, c->grid.Nx, c->grid.Ny, c->grid.Nz, (int)c->times.size(), (int)c->cols.size()};
}

// Buffers of the FP32 path at the context's launch shapes.
void alloc_fast32(wt_ctx* c) {
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    c->Zc32.alloc((size_t)32 * c->cols.size() * g.Nz);
    c->rho32.alloc(c->sp32.rho_elems(c->tune_nb));
    c->R32.alloc(c->sp32.r_elems(c->tune_nb));
    c->E32.alloc((size_t)3 * 32 * npts);
}

// Spectral passes (deposit, plane, z) of all basis vectors of one context.
void spectral_all(wt_ctx* c, cudaStream_t s) {
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int ncol = (int)c->cols.size();
    if (use_tables(c, 0)) {
        spectral_tables(c, c->Zc32.p, c->rank, s);
        return;
    }
    for (int m0 = 0; m0 < c->rank; m0 += c->tune_nb) {
        const int b = std::min(c->tune_nb, c->rank - m0);
        c->sp32.fields(c->Zc32.p + (size_t)m0 * ncol * g.Nz, b, c->rho32.p, c->R32.p, c->E32.p + (size_t)m0 * npts,
                       npts, (size_t)32 * npts, s, 0, c->tune_lb);
    }
}

template <class F>
float time_min(cudaStream_t s, int reps, F&& f) {
    cudaEvent_t a, b;
    WT_CUDA(cudaEventCreate(&a));
    WT_CUDA(cudaEventCreate(&b));
    f();                                    // warm-up
    float best = 1e30f;
    for (int i = 0; i < reps; ++i) {
        WT_CUDA(cudaEventRecord(a, s));
        f();
        WT_CUDA(cudaEventRecord(b, s));
        WT_CUDA(cudaEventSynchronize(b));
        float ms = 0;
        WT_CUDA(cudaEventElapsedTime(&ms, a, b));
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Autotuner: times every candidate launch shape of the FP32 path on this
// context (its own basis vectors, writing into H; the minimum of 3 runs, 5 for
// the expansion) and keeps the fastest: the FFT forms (register-FFT lanes,
// two-pass y / x / z transforms, direct or staged x stores), then spectral
// batch nb in {1, 2, 4} x z-pass lines per block in {16, 32, 64}, then the
// expansion's time chunk {64, 128, 256} x epilogue warps {8, 12, 16} x store
// width {4, 2, 1}.  Results are cached per (device, grid, n_t) for the process.
TuneResult autotune(wt_ctx* c, float* H) {
    c->e32_stamp = 0;                       // trial shapes overwrite the basis fields
    // WT_LAUNCH_SHAPES = "nb,lb,nch,nepi,r_xy,r_z,x_direct[,two_pass[,store_vec[,table_rows[,table_flags]]]]"
    // fixes the shapes without timing (reproducible profiling runs); the values are checked like tuned ones
    if (const char* env = std::getenv("WT_LAUNCH_SHAPES")) {
        TuneResult t{};
        const int nread = std::sscanf(env, "%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d", &t.nb, &t.lb, &t.nch, &t.nepi,
                                      &t.rxy, &t.rz, &t.xd, &t.tp, &t.vec, &t.ys, &t.tf);
        if (nread < 8) t.tp = 0;
        if (nread < 9) t.vec = 4;
        if (nread < 10) t.ys = 0;
        if (nread < 11) t.tf = 0;
        if (t.tf < 0 || t.tf > 7) fail(WT_ERR_ARG, "WT_LAUNCH_SHAPES: table flags must be 0..7");
        if (t.ys < 0 || t.ys > c->grid.Ny) fail(WT_ERR_ARG, "WT_LAUNCH_SHAPES: table rows must be 0..Ny");
        if (t.ys > 0 && !tables_fit(c)) t.ys = 0;
        if (nread < 7 || (t.vec != 1 && t.vec != 2 && t.vec != 4) || (t.nb != 1 && t.nb != 2 && t.nb != 4) ||
            (t.lb != 16 && t.lb != 32 && t.lb != 64) || (t.nch != 64 && t.nch != 128 && t.nch != 256) ||
            (t.nepi != 8 && t.nepi != 12 && t.nepi != 16) || t.tp < 0 || t.tp > 7)
            fail(WT_ERR_ARG,
                 "WT_LAUNCH_SHAPES must be nb,lb,nch,nepi,r_xy,r_z,x_direct[,two_pass[,store_vec]] with valid values");
        c->sp32.set_radix(t.rxy, t.rz, t.tp & 1, t.tp & 2, t.tp & 4);   // checks the FFT lengths
        t.xd = t.xd ? 1 : 0;
        t.spectral_ms = t.expand_ms = 0.0;
        return t;
    }
    // the process cache of timed results (the environment's fixed shapes above take precedence)
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(tune_key(c));
        if (it != g_tune.end()) return it->second;
    }
    cudaStream_t s = c->s;
    const wt_grid& g = c->grid;
    const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
    const int ncol = (int)c->cols.size(), nt = (int)c->times.size();
    TuneResult best{1, 32, 256, 8, c->sp32.rxy, c->sp32.rz, 0, 0, 4, 1e30, 1e30, 0, 0};
    c->tune_ys = 0;
    c->tune_tf = 0;
    c->tune_nb = 1;
    c->tune_lb = 32;
    alloc_fast32(c);
    column_ztransform<float>(s, c->Ub.p, c->rank, c->ns, c->ns, c->zcos.p, c->d_col_off.p, ncol, g.Nz, c->Zc32.p);
    // register-FFT shapes (lanes per line) of the plane and z passes, and the two-pass z FFT
    {
        std::vector<std::pair<int, int>> zopts, xyopts;   // (elements per lane, two-pass)
        for (int rz : Fast32::radix_options(g.Nz)) zopts.push_back({rz, 0});
        if (Fast32::z_two_pass_supported(g.Nz)) zopts.push_back({c->sp32.rz, 1});
        for (int rxy : Fast32::radix_options(g.Nx)) {
            xyopts.push_back({rxy, 0});
            if (Fast32::y_two_pass_supported(g.Ny, rxy)) xyopts.push_back({rxy, 2});
        }
        if (g.Nx == g.Ny && Fast32::y_two_pass_supported(g.Ny, 0)) xyopts.push_back({c->sp32.rxy, 6});
        double best_ms = 1e30;
        for (int xd : {0, 1})
            for (const auto& xo : xyopts)
                for (const auto& zo : zopts) {
                    c->sp32.set_radix(xo.first, zo.first, zo.second, xo.second & 2, xo.second & 4);
                    c->sp32.xdirect = xd;
                    const float ms = time_min(s, 3, [&] { spectral_all(c, s); });
                    if (ms < best_ms) {
                        best_ms = ms;
                        best.rxy = xo.first;
                        best.rz = zo.first;
                        best.tp = zo.second | xo.second;
                        best.xd = xd;
                    }
                }
        c->sp32.set_radix(best.rxy, best.rz, best.tp & 1, best.tp & 2, best.tp & 4);
        c->sp32.xdirect = best.xd;
    }
    for (int nb : {1, 2, 4}) {
        if (nb > 1 && nb > c->rank) break;
        c->tune_nb = nb;
        alloc_fast32(c);
        for (int lb : {16, 32, 64}) {
            c->tune_lb = lb;
            const float ms = time_min(s, 3, [&] { spectral_all(c, s); });
            if (ms < best.spectral_ms) { best.spectral_ms = ms; best.nb = nb; best.lb = lb; }
        }
    }
    c->tune_nb = best.nb;
    c->tune_lb = best.lb;
    alloc_fast32(c);
    // the lateral tables (built once per context, at the FFT shapes chosen above): slabs of
    // 1 .. 32 y rows x z-pass lines per block x {one stream, slabs pipelined on two} x {slab kept,
    // slab's L2 lines dropped after its z pass} x {vectors of lines, one line per thread in the
    // combination}, against the per-basis passes' best time
    if (tables_fit(c)) {
        build_tables(c);
        const int lb0 = best.lb;
        for (int ys : {1, 2, 4, 8, 16, 32}) {
            if (ys > g.Ny) break;
            c->tune_ys = ys;
            for (int tf = 0; tf < 8; ++tf) {
                if ((tf & 2) && !(c->sp32.zsm && (g.Nx * ys) % 32 == 0)) continue;   // discard needs whole lines
                c->tune_tf = tf;
                for (int lb : {16, 32, 64}) {
                    if ((tf & 2) && lb < 32) continue;
                    c->tune_lb = lb;
                    const float ms = time_min(s, 3, [&] { spectral_all(c, s); });
                    if (ms < best.spectral_ms) { best.spectral_ms = ms; best.ys = ys; best.lb = lb; best.tf = tf; }
                }
            }
        }
        c->tune_ys = best.ys;
        c->tune_tf = best.ys ? best.tf : 0;
        c->tune_lb = best.ys ? best.lb : lb0;
        if (!best.ys) {                      // not faster here: give the memory back
            c->T32.release();
            c->Rsl.release();
            c->t32_ready = false;
        }
    }
    spectral_all(c, s);
    for (int vec : {4, 2, 1})
        for (int nepi : {8, 12, 16})
            for (int nch : {64, 128, 256}) {
                ExpandJob jb{c->E32.p, 32, c->rank, c->W32.p, nt, npts, H};
                const float ms = time_min(s, 5, [&] { expand_tc_jobs(s, &jb, 1, 0, nch, c->d_err.p, nepi, vec); });
                if (ms < best.expand_ms) {
                    best.expand_ms = ms;
                    best.nch = nch;
                    best.nepi = nepi;
                    best.vec = vec;
                }
            }
    if (read_err(c)) fail(WT_ERR_TIMEOUT, "device wait timed out while tuning");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[tune_key(c)] = best;
    return best;
}

void apply_tuning(wt_ctx* c, const TuneResult& t) {
    c->tune_nb = t.nb;
    c->tune_lb = t.lb;
    c->tune_nch = t.nch;
    c->tune_nepi = t.nepi;
    c->tune_vec = t.vec;
    c->sp32.set_radix(t.rxy, t.rz, t.tp & 1, t.tp & 2, t.tp & 4);
    c->sp32.xdirect = t.xd;
    c->tune_ys = (t.ys > 0 && tables_fit(c)) ? t.ys : 0;
    c->tune_tf = c->tune_ys ? t.tf : 0;
    alloc_fast32(c);
    if (c->tune_ys) build_tables(c);         // the tables of this context (geometry only; kept)
    c->tuned = true;
}

void tune_context(wt_ctx* c, float* H) { apply_tuning(c, autotune(c, H)); }

BatchEntry entry_of(wt_ctx* c, const void* H) {
    if (c->tune_ys) alloc_slabs(c);   // captured by address
    if (c->tune_ys && (c->tune_tf & 1)) ensure_aux(c);   // the second stream exists before any capture
    return BatchEntry{c, c->uid, c->version, H, c->E32.p, c->Zc32.p, c->rho32.p, c->R32.p, c->Ub.p, c->W32.p,
                      c->T32.p, c->Rsl.p, c->tune_nb, c->tune_lb, c->sp32.rxy, c->sp32.rz, (int)c->sp32.xdirect,
                      (int)c->sp32.zsm | ((int)c->sp32.ysm << 1) | ((int)c->sp32.xsm << 2), c->tune_ys,
                      c->tune_tf};
}

// Records the whole batch (column transforms, spectral passes of every
// context, one persistent expansion launch per 64 contexts) as a CUDA graph.
void capture_batch(BatchPlan& P, wt_ctx* const* ctxs, int n, float* const* H) {
    cudaStream_t cs = ctxs[0]->s;
    WT_CUDA(cudaStreamSynchronize(cs));
    WT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        std::vector<ExpandJob> jobs;
        for (int i = 0; i < n; ++i) {
            wt_ctx* c = ctxs[i];
            const wt_grid& g = c->grid;
            const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
            const int ncol = (int)c->cols.size();
            column_ztransform<float>(cs, c->Ub.p, c->rank, c->ns, c->ns, c->zcos.p, c->d_col_off.p, ncol, g.Nz,
                                     c->Zc32.p);
            spectral_all(c, cs);
            jobs.push_back(ExpandJob{c->E32.p, 32, c->rank, c->W32.p, (int)c->times.size(), npts, H[i]});
        }
        const int mj = expand_tc_max_jobs();
        for (int j0 = 0; j0 < n; j0 += mj)
            expand_tc_jobs(cs, jobs.data() + j0, std::min(mj, n - j0), 0, P.nch, ctxs[0]->d_err.p, P.nepi, P.vec);
    } catch (...) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        if (junk) cudaGraphDestroy(junk);
        cudaGetLastError();
        throw;
    }
    WT_CUDA(cudaStreamEndCapture(cs, &P.graph));
    WT_CUDA(cudaGraphInstantiate(&P.exec, P.graph, 0));
}

void do_batch(wt_ctx* const* ctxs, int n, wt_precision prec, void* const* H, cudaStream_t us) {
    wt_ctx* c0 = ctxs[0];
    for (int i = 0; i < n; ++i) {
        wt_ctx* c = ctxs[i];
        if (!c) fail(WT_ERR_ARG, "NULL context in the batch");
        if (c->stage < 2) fail(WT_ERR_STATE, "every context of a batch must be relaxed");
        if (c->dev != c0->dev) fail(WT_ERR_ARG, "all contexts of a batch must be on one device");
        if (!H[i] || !is_device_ptr(H[i])) fail(WT_ERR_ARG, "batch outputs must be device memory");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == c) fail(WT_ERR_ARG, "a context appears twice in the batch");
    }
    if (prec == WT_FP64) {       // plain path: one extension after the other
        for (int i = 0; i < n; ++i) {
            const wt_grid& g = ctxs[i]->grid;
            const size_t need = ctxs[i]->times.size() * 3 * (size_t)g.Nx * g.Ny * g.Nz * sizeof(double);
            do_extend(ctxs[i], WT_FP64, H[i], need, us);
        }
        return;
    }
    if (!expand_tc_available()) fail(WT_ERR_UNSUPPORTED, "the batched path needs the tensor-core expansion");
    // launch shapes: tuned once per (grid, n_t), then every context at its shape's values
    std::map<TuneKey, TuneResult> shapes;
    for (int i = 0; i < n; ++i) {
        wt_ctx* c = ctxs[i];
        ensure_spectral(c);
        const TuneKey k = tune_key(c);
        if (!shapes.count(k)) shapes[k] = autotune(c, static_cast<float*>(H[i]));
        apply_tuning(c, shapes[k]);
    }
    // one (time chunk, epilogue warps, store width) for the shared expansion launch: the one most
    // of the grid points asked for
    std::map<std::tuple<int, int, int>, double> votes;
    for (int i = 0; i < n; ++i) {
        const wt_grid& g = ctxs[i]->grid;
        votes[{ctxs[i]->tune_nch, ctxs[i]->tune_nepi, ctxs[i]->tune_vec}] += (double)g.Nx * g.Ny * g.Nz;
    }
    int nch = 256, nepi = 8, vec = 4;
    double top = -1;
    for (auto& v : votes)
        if (v.second > top) {
            top = v.second;
            std::tie(nch, nepi, vec) = v.first;
        }
    std::vector<BatchEntry> want;
    for (int i = 0; i < n; ++i) want.push_back(entry_of(ctxs[i], H[i]));
    BatchPlan* plan = nullptr;
    for (auto& p : c0->plans)
        if (p->nch == nch && p->nepi == nepi && p->vec == vec && p->ents == want) plan = p.get();
    if (!plan) {
        auto P = std::make_unique<BatchPlan>();
        P->ents = want;
        P->nch = nch;
        P->nepi = nepi;
        P->vec = vec;
        capture_batch(*P, ctxs, n, reinterpret_cast<float* const*>(H));
        if (c0->plans.size() >= 4) {         // keep the four most recently used graphs
            auto old = std::min_element(c0->plans.begin(), c0->plans.end(),
                                        [](const auto& a, const auto& b) { return a->last_use < b->last_use; });
            c0->plans.erase(old);
        }
        c0->plans.push_back(std::move(P));
        plan = c0->plans.back().get();
    }
    plan->last_use = ++g_plan_clock;
    for (int i = 0; i < n; ++i) ctxs[i]->e32_stamp = 0;     // written by the graph on the caller's stream
    // the graph runs on the caller's stream after the contexts' own pending work
    cudaEvent_t ev;
    WT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    for (int i = 0; i < n; ++i) {
        WT_CUDA(cudaEventRecord(ev, ctxs[i]->s));
        WT_CUDA(cudaStreamWaitEvent(us, ev, 0));
    }
    cudaEventDestroy(ev);
    WT_CUDA(cudaGraphLaunch(plan->exec, us));
}

}  // namespace

extern "C" {

wt_status wt_create(wt_ctx** out, const wt_grid* grid, int cuda_device) {
    return run(nullptr, "wt_create", [&] {
        if (!out || !grid) fail(WT_ERR_ARG, "NULL argument");
        *out = nullptr;
        const wt_grid& g = *grid;
        if (!(g.Lx > 0 && g.Ly > 0 && g.Lz > 0) || g.Nx < 4 || g.Ny < 4 || g.Nz < 2 || !(g.eps_r > 0))
            fail(WT_ERR_ARG, "grid sizes must be positive (Nx, Ny >= 4, Nz >= 2)");
        if ((g.Nx & 1) || (g.Ny & 1)) fail(WT_ERR_ARG, "Nx and Ny must be even");
        if (g.zbc != WT_Z_MIRROR) fail(WT_ERR_UNSUPPORTED, "only the mirror z boundary is implemented");
        make_plan(2 * g.Nz);
        make_plan(g.Nx);
        make_plan(g.Ny);
        int ndev = 0;
        WT_CUDA(cudaGetDeviceCount(&ndev));
        if (cuda_device < 0 || cuda_device >= ndev) fail(WT_ERR_ARG, "no such CUDA device");
        WT_CUDA(cudaSetDevice(cuda_device));
        wt_ctx* c = new wt_ctx();
        c->dev = cuda_device;
        static std::atomic<unsigned long long> next_uid{1};
        c->uid = next_uid++;
        if (const char* e = std::getenv("WT_EXPAND")) c->use_tc = std::strcmp(e, "simt") != 0;
        c->grid = g;
        c->info.Nx = g.Nx;
        c->info.Ny = g.Ny;
        c->info.Nz = g.Nz;
        try {
            WT_CUDA(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
            WT_CUDA(cudaStreamCreateWithFlags(&c->s_copy, cudaStreamNonBlocking));
            c->d_err.alloc(16);
            c->d_err.zero(c->s);
            c->d_scr.alloc(16);
        } catch (...) {
            if (c->s) cudaStreamDestroy(c->s);
            if (c->s_copy) cudaStreamDestroy(c->s_copy);
            delete c;
            throw;
        }
        *out = c;
    });
}

wt_status wt_add_columns(wt_ctx* ctx, const wt_column* cols, int n) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_add_columns", [&] {
        if (ctx->stage != 0) fail(WT_ERR_STATE, "columns must be added before wt_fit");
        if (n < 0 || (n > 0 && !cols)) fail(WT_ERR_ARG, "bad column array");
        for (int i = 0; i < n; ++i) {
            ctx->cols.push_back(cols[i]);
            ctx->rho_prof.emplace_back();
        }
    });
}

wt_status wt_fit(wt_ctx* ctx, const wt_fit_opts* opts, double* cond_out) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_fit", [&] {
        if (ctx->stage != 0) fail(WT_ERR_STATE, "wt_fit already called");
        wt_fit_opts o{4, 2, 0.0, 1.0, 0.0, 0};
        if (opts) o = *opts;
        if (o.n_az < 1 || o.n_h < 1 || !(o.tikhonov >= 0) || !(o.v_w != 0) || !std::isfinite(o.az0) ||
            (o.refine != 0 && o.refine != 1))
            fail(WT_ERR_ARG, "bad fit options");
        ctx->opts = o;
        do_fit(ctx);
        ctx->stage = 1;
        if (cond_out) *cond_out = ctx->info.cond_estimate;
    });
}

wt_status wt_relax(wt_ctx* ctx, const double* t, int n_t) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_relax", [&] {
        if (ctx->stage < 1) fail(WT_ERR_STATE, "wt_relax needs wt_fit first");
        if (!t || n_t < 1) fail(WT_ERR_ARG, "need at least one time sample");
        for (int i = 0; i < n_t; ++i) {
            if (!(t[i] > 0.0) || !std::isfinite(t[i])) fail(WT_ERR_ARG, "times must be finite and > 0");
            if (i && !(t[i] > t[i - 1])) fail(WT_ERR_ARG, "times must increase");
        }
        do_relax(ctx, t, n_t);
        ctx->stage = 2;
    });
}

wt_status wt_extend(wt_ctx* ctx, wt_precision prec, void* H, size_t H_bytes, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_extend", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_extend needs wt_relax first");
        if (prec != WT_FP32 && prec != WT_FP64) fail(WT_ERR_ARG, "bad precision");
        do_extend(ctx, prec, H, H_bytes, static_cast<cudaStream_t>(stream));
    });
}

wt_status wt_sample_H(wt_ctx* ctx, const double* xyz, int n, const double* t, int n_t, double* out) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_sample_H", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_sample_H needs wt_relax first");
        if (n < 0 || n_t < 0 || (n && !xyz) || (n_t && !t) || (n && n_t && !out)) fail(WT_ERR_ARG, "bad arguments");
        if (n == 0 || n_t == 0) return;
        do_sample(ctx, xyz, n, t, n_t, out);
    });
}

wt_status wt_eq1(wt_ctx* ctx, const void* H, const wt_tracks* tracks, float* i, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_eq1", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_eq1 needs wt_relax first");
        do_eq1(ctx, H, tracks, i, static_cast<cudaStream_t>(stream));
    });
}

wt_status wt_eq1_noalloc(wt_ctx* ctx, const float* H, const wt_tracks* tr, float* i, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_eq1_noalloc", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_eq1_noalloc needs wt_relax first");
        if (!tr) fail(WT_ERR_ARG, "NULL tracks");
        if (tr->n_tracks < 0 || tr->n_steps < 1 || tr->n_out < 1 || !(tr->dt > 0.0))
            fail(WT_ERR_ARG, "bad track sizes or dt");
        if (tr->n_tracks == 0) return;
        const wt_grid& g = ctx->grid;
        // every buffer: device memory of the context's device, large enough for what the kernels touch
        const size_t nts = (size_t)tr->n_tracks * tr->n_steps;
        const size_t need[9] = {ctx->times.size() * 3 * (size_t)g.Nx * g.Ny * g.Nz * sizeof(float),
                                (size_t)tr->n_tracks * tr->n_out * sizeof(float),
                                nts * sizeof(float), nts * sizeof(float), nts * sizeof(float),
                                nts * sizeof(float), nts * sizeof(float), nts * sizeof(float),
                                (size_t)tr->n_tracks * sizeof(float)};
        const void* ptrs[9] = {H, i, tr->x, tr->y, tr->z, tr->vx, tr->vy, tr->vz, tr->q};
        const char* names[9] = {"H", "i", "x", "y", "z", "vx", "vy", "vz", "q"};
        for (int k = 0; k < 9; ++k) {
            if (k == 8 && !tr->q) continue;
            const std::string why = device_span_problem(ptrs[k], need[k], ctx->dev);
            if (!why.empty())
                fail(WT_ERR_ARG, std::string(names[k]) + ": " + why +
                                     " (every buffer must be device memory of the context's device)");
        }
        const cudaStream_t us = static_cast<cudaStream_t>(stream);
        eq1_noalloc_launch(us, ctx->dev, H, g.Nx, g.Ny, g.Nz, ctx->d_times.p,
                           (int)ctx->times.size(), g.Lx, g.Ly, g.Lz, tr->x, tr->y, tr->z, tr->vx, tr->vy, tr->vz,
                           tr->q, (float)tr->charge, tr->n_tracks, tr->n_steps, tr->n_out, tr->dt, ctx->opts.v_w,
                           lag_samples_used(ctx->times, tr->dt, tr->n_out), i);
        // the call reads the relaxation's time samples on the caller's stream: a later wt_relax
        // waits for this event before it rewrites them (the event was created by wt_relax)
        WT_CUDA(cudaEventRecord(ctx->ev_noalloc, us));
        ctx->noalloc_pending = true;
    });
}

wt_status wt_eq1_loss(wt_ctx* ctx, wt_precision prec, const wt_tracks* tracks, double* loss) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_eq1_loss", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_eq1_loss needs wt_relax first");
        if (!loss) fail(WT_ERR_ARG, "NULL output");
        if (prec != WT_FP32 && prec != WT_FP64) fail(WT_ERR_ARG, "bad precision");
        *loss = do_loss(ctx, prec, tracks);
    });
}

wt_status wt_eq1_loss_grad(wt_ctx* ctx, const wt_tracks* tracks, double* loss, double* grad) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_eq1_loss_grad", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_eq1_loss_grad needs wt_relax first");
        if (!loss || !grad) fail(WT_ERR_ARG, "NULL output");
        do_loss_grad(ctx, tracks, loss, grad);
    });
}

wt_status wt_batch_run(wt_ctx* const* ctxs, int n, wt_precision prec, void* const* H, void* stream) {
    if (!ctxs || n < 1 || !H || !ctxs[0]) return WT_ERR_ARG;
    return run(ctxs[0], "wt_batch_run", [&] {
        if (prec != WT_FP32 && prec != WT_FP64) fail(WT_ERR_ARG, "bad precision");
        do_batch(ctxs, n, prec, H, static_cast<cudaStream_t>(stream));
    });
}

wt_status wt_get_tuning(wt_ctx* ctx, wt_tuning* out) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_get_tuning", [&] {
        if (!out) fail(WT_ERR_ARG, "NULL output");
        out->nb = ctx->tune_nb;
        out->lb = ctx->tune_lb;
        out->nch = ctx->tune_nch;
        out->nepi = ctx->tune_nepi;
        out->r_xy = ctx->sp_ready ? ctx->sp32.rxy : 0;
        out->r_z = ctx->sp_ready ? ctx->sp32.rz : 0;
        out->x_direct = ctx->sp_ready ? (int)ctx->sp32.xdirect : 0;
        out->two_pass = ctx->sp_ready ? (int)ctx->sp32.zsm | ((int)ctx->sp32.ysm << 1) | ((int)ctx->sp32.xsm << 2) : 0;
        out->store_vec = ctx->tune_vec;
        out->table_rows = ctx->tune_ys;
        out->table_flags = ctx->tune_tf;
    });
}

wt_status wt_set_resistivity_profile(wt_ctx* ctx, int column, const double* rho, int n) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_set_resistivity_profile", [&] {
        if (column < 0 || column >= (int)ctx->cols.size()) fail(WT_ERR_ARG, "no such column");
        if (!rho) {
            ctx->rho_prof[column].clear();
            return;
        }
        if (n != ctx->cols[column].n_sources) fail(WT_ERR_ARG, "the profile needs one value per source node");
        for (int j = 0; j < n; ++j)
            if (!(rho[j] > 0.0) || !std::isfinite(rho[j])) fail(WT_ERR_ARG, "resistivities must be finite and > 0");
        ctx->rho_prof[column].assign(rho, rho + n);
    });
}

wt_status wt_eq1_loss_grad_profile(wt_ctx* ctx, const wt_tracks* tracks, const double* delta, double* loss,
                                   double* dL) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_eq1_loss_grad_profile", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_eq1_loss_grad_profile needs wt_relax first");
        if (!delta || !loss || !dL) fail(WT_ERR_ARG, "NULL argument");
        for (int j = 0; j < ctx->ns; ++j)
            if (!std::isfinite(delta[j])) fail(WT_ERR_ARG, "non-finite direction");
        do_loss_grad(ctx, tracks, loss, dL, delta);
    });
}

wt_status wt_static_field(wt_ctx* ctx, const double* phi_cols, wt_precision prec, void* E, size_t E_bytes,
                          void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_static_field", [&] {
        if (ctx->stage < 1) fail(WT_ERR_STATE, "wt_static_field needs wt_fit first");
        if (!phi_cols || !E) fail(WT_ERR_ARG, "NULL argument");
        if (prec != WT_FP32 && prec != WT_FP64) fail(WT_ERR_ARG, "bad precision");
        const wt_grid& g = ctx->grid;
        const size_t npts = (size_t)g.Nx * g.Ny * g.Nz;
        const size_t need = 3 * npts * (prec == WT_FP64 ? 8 : 4);
        if (E_bytes < need) fail(WT_ERR_ARG, "E_bytes too small: need " + std::to_string(need));
        if (!is_device_ptr(E)) fail(WT_ERR_ARG, "E must be device memory");
        ensure_spectral(ctx);
        cudaStream_t s = ctx->s;
        const int ns = ctx->ns, ncol = (int)ctx->cols.size();
        // every node of a column at its electrode's potential; q = C_n phi
        std::vector<double> phi(ns);
        for (int k = 0; k < ncol; ++k) {
            if (!std::isfinite(phi_cols[k])) fail(WT_ERR_ARG, "non-finite potential");
            for (int j = ctx->col_off[k]; j < ctx->col_off[k + 1]; ++j) phi[j] = phi_cols[k];
        }
        DBuf<double> dphi, q;
        dphi.upload(phi.data(), ns, s);
        q.alloc(ns);
        dgemv(s, false, ns, ns, 1.0, ctx->Cn.p, ns, dphi.p, 0.0, q.p);
        // order after the caller's pending work on its stream, then back
        cudaEvent_t ev;
        WT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        WT_CUDA(cudaEventRecord(ev, static_cast<cudaStream_t>(stream)));
        WT_CUDA(cudaStreamWaitEvent(s, ev, 0));
        if (prec == WT_FP64) {
            ctx->Zc64.alloc((size_t)4 * ncol * g.Nz);
            ctx->G64.alloc(ctx->sp64.scratch_elems(4));
            column_ztransform<double>(s, q.p, 1, ns, ns, ctx->zcos.p, ctx->d_col_off.p, ncol, g.Nz, ctx->Zc64.p);
            ctx->sp64.fields(ctx->Zc64.p, 1, ctx->G64.p, static_cast<double*>(E), 0, npts, s);
        } else {
            ctx->Zc32.alloc((size_t)32 * ncol * g.Nz);
            ctx->rho32.alloc(ctx->sp32.rho_elems(ctx->tune_nb));
            ctx->R32.alloc(ctx->sp32.r_elems(ctx->tune_nb));
            column_ztransform<float>(s, q.p, 1, ns, ns, ctx->zcos.p, ctx->d_col_off.p, ncol, g.Nz, ctx->Zc32.p);
            ctx->sp32.fields(ctx->Zc32.p, 1, ctx->rho32.p, ctx->R32.p, static_cast<float*>(E), 0, npts, s, 0,
                             ctx->tune_lb);
        }
        WT_CUDA(cudaEventRecord(ev, s));
        WT_CUDA(cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), ev, 0));
        WT_CUDA(cudaStreamSynchronize(s));
        cudaEventDestroy(ev);
    });
}

wt_status wt_drift(wt_ctx* ctx, const float* E, const double* x0, const double* smu, int n, int n_steps, double dt,
                   float* x, float* y, float* z, float* vx, float* vy, float* vz, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_drift", [&] {
        if (n < 0 || n_steps < 1 || !(dt > 0.0)) fail(WT_ERR_ARG, "bad sizes or dt");
        if (n == 0) return;
        const void* ptrs[10] = {E, x0, smu, x, y, z, vx, vy, vz, nullptr};
        for (int k = 0; k < 9; ++k)
            if (!ptrs[k] || !is_device_ptr(ptrs[k])) fail(WT_ERR_ARG, "every array of wt_drift must be device memory");
        std::vector<double> cs;
        for (const wt_column& c : ctx->cols) {
            cs.push_back(c.x);
            cs.push_back(c.y);
            cs.push_back(c.radius * c.radius);
            cs.push_back(c.z0);
            cs.push_back(c.z1);
        }
        const wt_grid& g = ctx->grid;
        drift_launch(static_cast<cudaStream_t>(stream), E, g.Nx, g.Ny, g.Nz, g.Lx, g.Ly, g.Lz, cs, x0, smu, n, n_steps,
                     dt, x, y, z, vx, vy, vz);
    });
}

wt_status wt_shape(wt_ctx* ctx, const float* i, int n_tracks, int n_out, double dt, const wt_shaper* sh,
                   const float* noise, float* v, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_shape", [&] {
        if (!sh || n_tracks < 0 || n_out < 1 || !(dt > 0.0)) fail(WT_ERR_ARG, "bad sizes or dt");
        if (!(sh->tau > 0.0) || sh->order < 0 || sh->order > 20 || !std::isfinite(sh->gain) ||
            !std::isfinite(sh->noise_rms))
            fail(WT_ERR_ARG, "bad shaper parameters (tau > 0, 0 <= order <= 20)");
        if (n_tracks == 0) return;
        if (!i || !v || !is_device_ptr(i) || !is_device_ptr(v) || (noise && !is_device_ptr(noise)))
            fail(WT_ERR_ARG, "currents, noise and output must be device memory");
        if ((size_t)n_out * 12 > 200 * 1024) fail(WT_ERR_UNSUPPORTED, "n_out too large for one block's shared memory");
        shape_launch(static_cast<cudaStream_t>(stream), i, n_tracks, n_out, dt, sh->tau, sh->order, sh->gain,
                     sh->noise_rms, noise, v);
    });
}

wt_status wt_eq1_direct(wt_ctx* ctx, const wt_tracks* tracks, float* i, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_eq1_direct", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_eq1_direct needs wt_relax first");
        do_eq1_direct(ctx, tracks, i, static_cast<cudaStream_t>(stream));
    });
}

wt_status wt_eq1_tangents(wt_ctx* ctx, const wt_tracks* tracks, float* i, float* di, double* loss, double* grad) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_eq1_tangents", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "wt_eq1_tangents needs wt_relax first");
        if (!tracks) fail(WT_ERR_ARG, "NULL tracks");
        if ((i && !is_device_ptr(i)) || (di && !is_device_ptr(di)))
            fail(WT_ERR_ARG, "current and tangent outputs must be device memory");
        double l = 0.0, g[4];
        do_loss_grad(ctx, tracks, &l, g, nullptr, i, di);
        WT_CUDA(cudaStreamSynchronize(ctx->s));
        if (loss) *loss = l;
        if (grad)
            for (int k = 0; k < 4; ++k) grad[k] = g[k];
    });
}

wt_status wt_features(wt_ctx* ctx, const float* x, int n_tracks, int n, double t0, double dt,
                      const wt_feature_opts* opts, const float* dx, int n_dir, double* f, double* df, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_features", [&] {
        const wt_feature_opts o = opts ? *opts : wt_feature_opts{0.1f, 0.9f, 0.5f};
        auto frac_ok = [](float v) { return v > 0.f && v <= 1.f; };
        if (n_tracks < 0 || n < 1 || n_dir < 0 || !(dt > 0.0) || !std::isfinite(t0))
            fail(WT_ERR_ARG, "bad sizes, dt or t0");
        if (!frac_ok(o.lo) || !frac_ok(o.hi) || !frac_ok(o.cfd)) fail(WT_ERR_ARG, "fractions must lie in (0, 1]");
        if (n_tracks == 0) return;
        if (!x || !f || !is_device_ptr(x) || !is_device_ptr(f)) fail(WT_ERR_ARG, "x and f must be device memory");
        if (n_dir > 0 && (!dx || !df || !is_device_ptr(dx) || !is_device_ptr(df)))
            fail(WT_ERR_ARG, "dx and df must be device memory when n_dir > 0");
        features_launch(static_cast<cudaStream_t>(stream), x, n_tracks, n, t0, dt, o.lo, o.hi, o.cfd, dx, n_dir, f,
                        df);
    });
}

wt_status wt_sync(wt_ctx* ctx, void* stream) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_sync", [&] {
        WT_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
        WT_CUDA(cudaStreamSynchronize(ctx->s_copy));
        const int e = read_err(ctx);          // synchronises the context's stream
        if (e) {
            clear_err(ctx);
            WT_CUDA(cudaStreamSynchronize(ctx->s));
            fail(e == DERR_TIMEOUT ? WT_ERR_TIMEOUT : e == DERR_NOT_SPD ? WT_ERR_NOT_SPD : WT_ERR_NAN,
                 "device-side failure in earlier asynchronous work on this context");
        }
    });
}

wt_status wt_get_charges(wt_ctx* ctx, double* q) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_get_charges", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "no charges before wt_relax");
        if (!q) fail(WT_ERR_ARG, "NULL output");
        ctx->Qt.download(q, ctx->times.size() * (size_t)ctx->ns, ctx->s);
        WT_CUDA(cudaStreamSynchronize(ctx->s));
    });
}

wt_status wt_get_capacitance(wt_ctx* ctx, double* cn) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_get_capacitance", [&] {
        if (ctx->stage < 1) fail(WT_ERR_STATE, "no capacitance before wt_fit");
        if (!cn) fail(WT_ERR_ARG, "NULL output");
        ctx->Cn.download(cn, (size_t)ctx->ns * ctx->ns, ctx->s);
        WT_CUDA(cudaStreamSynchronize(ctx->s));
    });
}

wt_status wt_get_modes(wt_ctx* ctx, double* mu) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_get_modes", [&] {
        if (ctx->stage < 2) fail(WT_ERR_STATE, "no modes before wt_relax");
        if (!mu) fail(WT_ERR_ARG, "NULL output");
        ctx->mu.download(mu, ctx->ns - 1, ctx->s);
        WT_CUDA(cudaStreamSynchronize(ctx->s));
    });
}

wt_status wt_get_info(wt_ctx* ctx, wt_info* info) {
    if (!ctx || !info) return WT_ERR_ARG;
    *info = ctx->info;
    return WT_OK;
}

wt_status wt_set_timing(wt_ctx* ctx, int enable) {
    if (!ctx) return WT_ERR_ARG;
    ctx->timing = enable != 0;
    return WT_OK;
}

wt_status wt_get_grad_timing(wt_ctx* ctx, double* ms6) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_get_grad_timing", [&] {
        if (!ms6) fail(WT_ERR_ARG, "NULL output");
        for (int k = 0; k < 6; ++k) ms6[k] = ctx->grad_ms[k];
    });
}

wt_status wt_get_timing(wt_ctx* ctx, double* ms3, int* n_launches) {
    if (!ctx) return WT_ERR_ARG;
    return run(ctx, "wt_get_timing", [&] {
        if (!ms3) fail(WT_ERR_ARG, "NULL output");
        if (!ctx->ev_recorded) fail(WT_ERR_STATE, "no timed wt_extend (call wt_set_timing(ctx, 1) first)");
        for (int k = 1; k < 4; ++k) {
            WT_CUDA(cudaEventSynchronize(ctx->ev[k]));
            float ms = 0.f;
            WT_CUDA(cudaEventElapsedTime(&ms, ctx->ev[k - 1], ctx->ev[k]));
            ms3[k - 1] = ms;
        }
        if (n_launches) *n_launches = ctx->last_launches;
    });
}

const char* wt_last_error(const wt_ctx* ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

void wt_destroy(wt_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    if (ctx->s) cudaStreamSynchronize(ctx->s);
    cudaStream_t s = ctx->s, s2 = ctx->s_copy;
    if (s2) cudaStreamSynchronize(s2);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->s_aux) {
        cudaStreamSynchronize(ctx->s_aux);
        for (int k = 0; k < 2; ++k) {
            cudaEventDestroy(ctx->ev_tc[k]);
            cudaEventDestroy(ctx->ev_tz[k]);
        }
        cudaEventDestroy(ctx->ev_fork);
        cudaStreamDestroy(ctx->s_aux);
    }
    if (ctx->ev_noalloc) {
        cudaEventSynchronize(ctx->ev_noalloc);
        cudaEventDestroy(ctx->ev_noalloc);
    }
    delete ctx;
    if (s) cudaStreamDestroy(s);
    if (s2) cudaStreamDestroy(s2);
}

}  // extern "C"
