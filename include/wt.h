/*
 * wt.h -- C ABI of the GB300 weighting-field library.
 *
 * Computes the time-dependent weighting field H(x, t) of a 3D diamond sensor
 * with resistive graphitised column electrodes (arXiv 2605.13987), and the
 * Ramo-Shockley-Riegler induced current of Eq. 1 from it.
 *
 * Method (the paper prints only Eq. 1 and the resistance formula of Sec. 5;
 * the rest is its Abstract / Sec. 1 / Sec. 3 description):
 *   - point sources ("fundamental solutions", Abstract; Sec. 3) on each column
 *     axis, their magnitudes fitted to the electrode boundary values;
 *   - the quasi-static third-order PDE (Abstract) reduced to resistive lines
 *     coupled through the fitted capacitance, relaxed in time exactly in
 *     FP64 (Sec. 3 describes forward-Euler steps; the exact modal exponential
 *     is their dt -> 0 limit);
 *   - a pseudo-spectral extension into the bulk (Abstract; Sec. 1 "discrete
 *     Fourier transforms"; Sec. 3 spectra multiplied/divided by |k|^2) at
 *     every time sample.
 *
 * Units: SI (m, s, Ohm*m, F, C, V).  Grid points: x_i = i Lx/Nx,
 * y_j = j Ly/Ny, z_k = (k + 1/2) Lz/Nz.  Lateral boundaries are periodic; z is
 * mirrored at 0 and Lz (Neumann).  Spectral modes: |m_x| <= Nx/2 - 1,
 * |m_y| <= Ny/2 - 1 (Nyquist dropped), k_z = pi m_z / Lz, m_z = 0..Nz-1.
 *
 * H layout in memory: H[t][c][x][y][z], z fastest, c = 0,1,2 the field
 * components (V/m), t the time samples given to wt_relax.  H stores
 * W = -grad(psi) of the step response to V_w applied at t = 0 on the driven
 * readout; Eq. 1's impulse response is its time derivative (see wt_eq1).
 *
 * Conventions.  Every call returns a wt_status; nothing aborts or prints.
 * wt_last_error() gives the message of the last failed call on a context.
 * The caller owns every buffer it passes; the library owns the context and
 * its internal device workspaces (allocated with cudaMalloc on the
 * context's device).  Calls must come in order: create -> add_columns ->
 * fit -> relax -> extend / sample_H / eq1; an out-of-order call returns
 * WT_ERR_STATE.  A context is not thread-safe; use one per host thread.
 */
#ifndef WT_H
#define WT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wt_ctx wt_ctx;

typedef enum {
    WT_OK = 0,
    WT_ERR_ARG = 1,              /* bad argument: NULL, size, range */
    WT_ERR_GEOMETRY = 2,         /* overlapping columns, column outside the sensor */
    WT_ERR_ILL_CONDITIONED = 3,  /* fit matrix too ill-conditioned for FP64 */
    WT_ERR_NOT_SPD = 4,          /* fitted capacitance not positive definite */
    WT_ERR_OOM = 5,              /* device allocation failed */
    WT_ERR_CUDA = 6,             /* CUDA runtime error */
    WT_ERR_TIMEOUT = 7,          /* a bounded device wait gave up */
    WT_ERR_STATE = 8,            /* call out of order */
    WT_ERR_NAN = 9,              /* non-finite input or intermediate */
    WT_ERR_UNSUPPORTED = 10,     /* size or option this build does not handle */
    WT_ERR_ACCURACY = 11         /* the FP32 path cannot reach its accuracy for this charge history
                                    (its time basis would need rank > 32): use WT_FP64 */
} wt_status;

typedef enum { WT_FP32 = 0, WT_FP64 = 1 } wt_precision;
/* z boundary of the sensor box: a mirror (Neumann) plane at z = 0 and at z = Lz,
 * the diamond slab between its two faces (the box is periodic in x and y, a
 * tile of a pixel matrix).  A box periodic in z as well (a stack of sensors
 * with no faces) is not part of this library. */
typedef enum { WT_Z_MIRROR = 0 } wt_zbc;

/* Sensor box and voxel grid.  Nx, Ny even; eps_r = relative permittivity
 * (5.7 for diamond; the columns take the same value). */
typedef struct {
    double Lx, Ly, Lz;
    int Nx, Ny, Nz;
    double eps_r;
    int zbc;                     /* wt_zbc: WT_Z_MIRROR (any other value gives WT_ERR_UNSUPPORTED) */
} wt_grid;

/* One graphitised column: axis at (x, y), spanning z0..z1, radius, and
 * resistivity [Ohm*m] (Sec. 5: R = 4 rho L / (pi d^2)).  terminal_top = 1
 * puts the terminal at z1 (readout), 0 at z0 (bias).  driven = 1 holds the
 * terminal at V_w (the readout whose weighting field is computed); all other
 * terminals are at 0.  n_sources point sources sit on the axis at
 * z0 + (j + 1/2)(z1 - z0)/n_sources. */
typedef struct {
    double x, y, z0, z1, radius, resistivity;
    int terminal_top;
    int driven;
    int n_sources;
} wt_column;

/* Boundary fit: n_h * n_sources collocation heights times n_az azimuths
 * (az0 + 2 pi a / n_az) per column, on the column surface.  tikhonov >= 0
 * is a relative ridge weight (0 = plain least squares).  v_w = weighting
 * potential (Eq. 1: 1 V).  refine: the least-squares solve is Cholesky on
 * the normal equations, corrected by one step of the semi-normal equations
 * (the residual taken in the collocation space) either always (1) or (0,
 * the default) only when the correction, probed on eight random
 * combinations of the right-hand sides, exceeds 1e-11 of the solution
 * (wt_info.fit_correction, wt_info.fit_refined). */
typedef struct {
    int n_az, n_h;
    double tikhonov;
    double v_w;
    double az0;
    int refine;
} wt_fit_opts;

/* Carrier tracks for Eq. 1, [track][step] float32 arrays, positions in m,
 * velocities in m/s, time step dt [s].  Pointers may be device or host
 * memory.  q: optional per-track charge [C] (NULL: every track has
 * `charge`).  n_out output times tau_m = m dt, m = 0..n_out-1. */
typedef struct {
    int n_tracks, n_steps, n_out;
    double dt, charge;
    const float *x, *y, *z, *vx, *vy, *vz;
    const float *q;
} wt_tracks;

/* Diagnostics of a context after wt_fit / wt_relax. */
typedef struct {
    int n_columns, n_sources, n_colloc, n_t;
    int rank;                    /* time-basis rank of the FP32 path (0 before relax) */
    double cond_estimate;        /* 2-norm condition estimate of the column-scaled fit matrix */
    double boundary_residual;    /* ||P q + c - S phi_DC|| / ||S phi_DC|| of the DC state */
    double asymmetry;            /* ||F - F^T|| / ||F|| (Green reciprocity) */
    double trunc_rel;            /* largest relative truncation error of one time sample of the
                                    charge history in the FP32 path's rank-`rank` time basis,
                                    ||q(t_n) - q_r(t_n)|| / ||q(t_n)|| (exact, from its SVD) */
    double mu_min, mu_max;       /* relaxation rates [1/s] */
    double fit_seconds, relax_seconds;
    double grad_trunc_rel;       /* largest relative truncation of the charge tangents in the
                                    last wt_eq1_loss_grad (rank-32 time bases) */
    int Nx, Ny, Nz;              /* the context's grid (H holds n_t x 3 x Nx x Ny x Nz values) */
    double fit_correction;       /* relative size of the semi-normal-equations correction of the fit
                                    (the full one when applied, else the probe's estimate) */
    int fit_refined;             /* 1 when the fit applied the correction */
} wt_info;

/* Create a context on CUDA device `cuda_device` for the given grid.
 * Fails with WT_ERR_ARG for non-positive sizes or odd Nx/Ny, and
 * WT_ERR_UNSUPPORTED for a z boundary this build does not implement. */
wt_status wt_create(wt_ctx** out, const wt_grid* grid, int cuda_device);

/* Append n columns (host array).  Geometry is validated at wt_fit. */
wt_status wt_add_columns(wt_ctx* ctx, const wt_column* cols, int n);

/* Boundary fit (Abstract; Sec. 3 point charges adjusted in magnitude),
 * FP64 on the GPU: the fit matrix P of the band-limited fundamental
 * solution at the collocation points, the neutral least-squares fit
 * q = F phi with one free potential offset (normal equations with column
 * scaling, one step of residual correction), capacitance C_n = (F + F^T)/2.
 * cond_estimate_out (may be NULL) receives the condition estimate.
 * Synchronous.  Errors: WT_ERR_GEOMETRY, WT_ERR_NOT_SPD (the normal
 * matrix or the capacitance is not positive definite), WT_ERR_ILL_CONDITIONED. */
wt_status wt_fit(wt_ctx* ctx, const wt_fit_opts* opts, double* cond_estimate_out);

/* Relaxation in time (Abstract: third-order quasi-static PDE; Sec. 3
 * forward-Euler iteration, here its exact limit), FP64 on the GPU:
 * C_n dphi/dt = K phi + b with the resistive lines of Sec. 5, solved by
 * the generalised symmetric eigenproblem on the neutral subspace (Cholesky
 * reduction, Householder tridiagonalisation, divide and conquer; the
 * environment variable WT_EIGEN=jacobi selects a two-sided Jacobi solver
 * instead, a cross-check; wt_get_modes returns the rates ascending); the node
 * charges q(t_n) at the n_t host times t[] (seconds, increasing, > 0), and
 * the rank-r time basis used by the FP32 path: the singular value
 * decomposition of the charge history [q(t_0) ... q(t_{n_t-1})] (one-sided
 * Jacobi, FP64), truncated at the smallest r <= 32 that leaves at most 1e-7
 * relative error in every time sample (wt_info.rank, wt_info.trunc_rel).
 * A history that still leaves more than 1e-6 at r = 32 relaxes normally,
 * but the FP32 field paths then return WT_ERR_ACCURACY.  Synchronous. */
wt_status wt_relax(wt_ctx* ctx, const double* t, int n_t);

/* Bulk extension (Abstract; Sec. 1 DFT; Sec. 3 |k|^2 spectral division):
 * writes H[t][c][x][y][z] for all n_t times.  WT_FP64: plain path, one
 * FP64 spectral transform per time sample, H as double (24 B per
 * point-sample).  WT_FP32: fast path, FP32 basis fields of the rank-r
 * time basis and a tensor-core expansion, H as float (12 B per
 * point-sample).  H may be device memory (written on cuda_stream, a
 * cudaStream_t or NULL; asynchronous) or host memory (the library computes
 * into an internal device buffer and copies out; returns after the copy).
 * H_bytes must be >= n_t * 3 * Nx*Ny*Nz * sizeof(element), else WT_ERR_ARG.
 * The first FP32 extension of a context (unless wt_batch_run came first)
 * runs the autotuner of wt_batch_run on it, writing trial results into H,
 * and returns only after that tuning; later calls reuse the choice.  The
 * environment variable WT_LAUNCH_SHAPES="nb,lb,nch,nepi,r_xy,r_z,x_direct[,two_pass[,store_vec[,table_rows[,table_flags]]]]"
 * (the values of wt_get_tuning) fixes the shapes without tuning.
 * WT_FP32 returns WT_ERR_ACCURACY when the time basis is truncated beyond
 * its limit (see wt_relax). */
wt_status wt_extend(wt_ctx* ctx, wt_precision prec, void* H, size_t H_bytes, void* cuda_stream);

/* Exact FP64 point evaluation of H (the band-limited spectral sum, no grid
 * interpolation) at n host points xyz[n][3] and n_t host times t[] (any
 * t >= 0, not only the relaxation samples).  out: host [n_t][n][3].
 * Synchronous. */
wt_status wt_sample_H(wt_ctx* ctx, const double* xyz, int n, const double* t, int n_t, double* out);

/* Eq. 1 (Ramo-Shockley-Riegler convolution) from an FP32 H produced by
 * wt_extend(WT_FP32): for each track and output time
 *   Q(tau_m) = sum_{m' <= m, m' < n_steps} H(x_m', (m - m' + 1/2) dt) . v_m' dt,
 *   i(tau_m) = -(q / V_w) (Q(tau_m) - Q(tau_{m-1})) / dt,
 * with trilinear interpolation in space (periodic x, y; z clamped to the
 * first/last grid plane) and linear interpolation in time (H = 0 at t = 0,
 * held after the last sample).  H must be device memory.  Track arrays and
 * i ([n_tracks][n_out] float32) may be device or host memory; the call
 * returns after the result is written. */
wt_status wt_eq1(wt_ctx* ctx, const void* H, const wt_tracks* tracks, float* i, void* cuda_stream);

/* Eq. 1 without any allocation.  Same result as wt_eq1, for callers that
 * cannot call cudaMalloc: code running where device allocation is not
 * allowed or not safe, for instance inside a memory-pool or arena manager
 * that owns all device memory, in a real-time loop that must not hit the
 * allocator's locks and synchronisation, or in a plugin host that hands out
 * only its own buffers.  The paper has no counterpart; this is a property of
 * the library only.
 *
 * The per-call scratch (the lag table, 12 bytes per output time) lives in a
 * fixed device array of WT_EQ1_NOALLOC_MAX_OUT entries, which every GPU that
 * loads the library holds (192 KB) until the process exits.  n_out above the
 * limit returns WT_ERR_ARG.  H, the track arrays and i must be device
 * memory (WT_ERR_ARG otherwise: host buffers would need staging).  Each buffer
 * must lie on the context's device and hold what the call touches: H
 * n_t x 3 x Nx x Ny x Nz floats (wt_extend's FP32 layout), i n_tracks x n_out
 * floats, each track array n_tracks x n_steps floats and q (if not NULL)
 * n_tracks floats; a buffer on another device, or one that ends before that
 * inside its allocation, returns WT_ERR_ARG.  The
 * call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) once; make that first call before any stream
 * capture.  All calls share the one array and each call overwrites the
 * entries it uses, so calls that overlap on the GPU (for example on two
 * streams at once) race on it: order them on one stream.  Asynchronous on
 * cuda_stream; the call reads the relaxation's time samples there, and a
 * later wt_relax on the context waits for it (through an event recorded on
 * cuda_stream) before it replaces them. */
#define WT_EQ1_NOALLOC_MAX_OUT 16384
wt_status wt_eq1_noalloc(wt_ctx* ctx, const float* H, const wt_tracks* tracks, float* i, void* cuda_stream);

/* Eq. 1 without writing H: the currents of wt_eq1 on wt_extend(WT_FP32)'s
 * field, computed from the rank-r form that the extension expands,
 * H[t][c][p] = sum_m W[t][m] E_m[c][p].  Interpolation is linear, so per
 * track step the r basis fields are interpolated once (r x 24 gathers
 * instead of n_t x 24 from H) and combined with the time coefficients;
 * lags, accumulation and currents as in wt_eq1.  Equal to wt_eq1 on the
 * FP32 H up to FP32 rounding.  The basis fields are computed when the
 * context does not hold them already (after wt_relax, or after another
 * call overwrote them).  Track arrays and i: host or device memory (as in
 * wt_eq1).  Ordered after the caller's work on cuda_stream; returns when i
 * is written.  Shares the FP32 work buffers of wt_extend and wt_batch_run:
 * do not run them concurrently on one context. */
wt_status wt_eq1_direct(wt_ctx* ctx, const wt_tracks* tracks, float* i, void* cuda_stream);

/* Loss of Eq. 1 currents, L = mean over tracks and output times of i(tau)^2
 * (Sec. 4's current of each track with its own charge, Eq. 1), computed in
 * one call: the field of the relaxed charges (WT_FP32: the fast path of
 * wt_extend; WT_FP64: the plain FP64 path) into an internal buffer, then
 * Eq. 1 on it.  Track arrays may be host or device memory (layout as in
 * wt_eq1).  Synchronous; *loss written on success.  Needs wt_relax. */
wt_status wt_eq1_loss(wt_ctx* ctx, wt_precision prec, const wt_tracks* tracks, double* loss);

/* Gradient of the loss of wt_eq1_loss (FP32 field) with respect to four
 * design parameters, by hand-written tangent-linear differentiation of the
 * whole chain: the constrained least-squares fit (Sec. 3), the capacitance
 * and resistive-line pencil and its modal solution (Sec. 5, derivative of
 * the matrix exponential in the modal basis), the field extension and Eq. 1.
 *   grad[0] = dL/ds_R   resistivity of the readout columns (terminal at the
 *                       top) scaled by s_R, at s_R = 1;
 *   grad[1] = dL/ds_B   the same for the bias columns (terminal at the bottom);
 *   grad[2] = dL/dr     every column radius moved by dr [per metre];
 *   grad[3] = dL/dlambda  lateral scale at lambda = 1: Lx, Ly, column centres
 *                       and the tracks' x, y, vx, vy scale together (z,
 *                       times and source counts fixed).
 * The source counts per column stay fixed under every perturbation.  The
 * fit must be unregularised (tikhonov = 0; WT_ERR_UNSUPPORTED otherwise).
 * *loss receives L (FP32 field), grad[4] the gradient.  Synchronous;
 * allocates device workspaces for the tangents and frees them on return. */
wt_status wt_eq1_loss_grad(wt_ctx* ctx, const wt_tracks* tracks, double* loss, double* grad);

/* Depth-dependent resistivity of one column (Sec. 5 names a depth-dependent
 * conductivity profile as a further improvement): rho[j] > 0 [Ohm*m] is
 * the resistivity of node j's cell, j = 0..n_sources-1 from z0 upward (n
 * must equal the column's n_sources).  Neighbouring nodes are joined
 * through two half cells, R = (rho_j + rho_j+1) dz / (2 pi r^2); the
 * terminal node reaches the electrode end through half a cell.  A uniform
 * profile gives the uniform column exactly.  rho = NULL returns to the
 * column's uniform resistivity.  Takes effect at the next wt_relax. */
wt_status wt_set_resistivity_profile(wt_ctx* ctx, int column, const double* rho, int n);

/* Directional derivative of the loss of wt_eq1_loss (FP32 field) along a
 * relative change of the node resistivities, rho_j -> rho_j (1 + eps
 * delta_j) (delta: host array of n_sources values in the order the columns
 * were added, each column's nodes from z0 upward), by the tangent-linear
 * chain of wt_eq1_loss_grad restricted to the resistive lines.  *loss
 * receives L, *dL = dL/deps at eps = 0.  Synchronous. */
wt_status wt_eq1_loss_grad_profile(wt_ctx* ctx, const wt_tracks* tracks, const double* delta, double* loss,
                                   double* dL);

/* Bulk extension of many sensors at once (FP32: the fast path of wt_extend
 * for every context, batched; the paper runs one geometry at a time, so
 * this is a property of the library).  ctxs[0..n-1]: relaxed contexts on
 * one device, each at most once; H[i]: device buffer of context i, layout
 * and size as wt_extend's.  FP32: the column transforms and spectral passes
 * of every context and one persistent tensor-core expansion launch over all
 * of them (one per 64 contexts) are captured once as a CUDA graph, kept on
 * ctxs[0] (the four most recently used batches) and replayed by later calls
 * with the same contexts, outputs and context states; a wt_relax on any of
 * them re-captures.  Before the first capture of a grid shape (Nx, Ny, Nz,
 * n_t) the autotuner times the candidate launch shapes on that context and
 * keeps the fastest for the process (see wt_get_tuning); tuning writes into
 * that context's H buffer.  The results equal wt_extend's bit for bit.
 * FP64: the plain path of each context in turn.  Asynchronous on
 * cuda_stream, ordered after the contexts' own pending work; the contexts'
 * FP32 work buffers are shared with wt_extend, so do not run either on the
 * same context concurrently. */
wt_status wt_batch_run(wt_ctx* const* ctxs, int n, wt_precision prec, void* const* H, void* cuda_stream);

/* Launch shapes the FP32 path of this context uses, set by the autotuner
 * (before the first extension: the defaults 1, 32, 256, 8, 0, 0, 0, 0, 4, 0, 0). */
typedef struct {
    int nb;         /* charge vectors per spectral launch: 1, 2, 4 */
    int lb;         /* (x, y) lines per z-pass block: 16, 32, 64 */
    int nch;        /* time samples per expansion accumulator chunk: 64, 128, 256 */
    int nepi;       /* expansion epilogue warps: 8, 12, 16 */
    int r_xy, r_z;  /* elements per lane of the lateral and z register FFTs */
    int x_direct;   /* 1: the x transforms store from registers (else staged) */
    int two_pass;   /* two-pass shared-memory FFTs in use, a bit mask: 1 the z pass (Nz of 64, 96,
                       128, 160, 192, 224, 256 or 384; r_z then unused), 2 the y transforms (Ny of 64 or 128; r_xy then
                       sets the x transforms only), 4 the x transforms too (with 2, Nx = Ny;
                       r_xy and x_direct then unused) */
    int store_vec;  /* floats per expansion store: 4 (4 x 4 lane-quad transposes), 2 (2 x 2
                       lane-pair transposes) or 1 (straight from the accumulator layout) */
    int table_rows; /* 0: basis fields by the per-basis spectral passes (deposit, lateral FFTs, z
                       pass); > 0: from the context's per-column lateral tables (Sec. 3's
                       translated fundamental-solution chunks in spectral form, built once per
                       context, 12 B x n_columns x Nx x Ny x Nz), combined per basis vector in y
                       slabs of table_rows rows and followed by the z pass */
    int table_flags; /* table path, a bit mask: 1 the combination of one slab overlaps the z pass
                       of the previous one on a second stream (two slab buffers); 2 the z pass
                       invalidates the L2 lines of the slab rows it has read, so that the slab
                       (scratch) is not written back to DRAM; 4 the combination takes one line per
                       thread (fewer registers, more resident warps) instead of vectors of lines */
} wt_tuning;
wt_status wt_get_tuning(wt_ctx* ctx, wt_tuning* out);

/* Static field of the electrodes held at fixed potentials (the paper's
 * static drift field, Fig. 2; the sigma -> infinity limit of the
 * relaxation): every node of column k at phi_cols[k] volts (host array of
 * n_columns values), node charges q = C_n phi, and their field
 * E[c][x][y][z] = -grad(potential) on the grid (V/m) by the extension's
 * spectral path (WT_FP32: float, WT_FP64: double).  E: device buffer of
 * at least 3 Nx Ny Nz elements.  Equal potentials on all electrodes give
 * no field.  Needs wt_fit; ordered after the caller's pending work on
 * cuda_stream, returns when E is written. */
wt_status wt_static_field(wt_ctx* ctx, const double* phi_cols, wt_precision prec, void* E, size_t E_bytes,
                          void* cuda_stream);

/* Carrier drift in a static field (the paper uses Garfield++ for the
 * transport; this is a constant-mobility drift that produces tracks for
 * wt_eq1): dx/dt = smu[a] E(x) (smu = signed mobility [m^2/(V s)], + for
 * holes, - for electrons), explicit midpoint steps of dt in FP64 on the
 * trilinear interpolation of E (FP32 [3][Nx][Ny][Nz], device; grid points
 * at (i hx, j hy, (k + 1/2) hz), x and y periodic, z clamped as in Eq. 1).
 * Step m of carrier a records its midpoint and velocity in
 * x..vz[a][m] (device FP32 arrays [n][n_steps], the wt_tracks layout); a
 * carrier stops after the step that ends inside a column or outside
 * 0 <= z <= Lz, and its later steps repeat its last position with zero
 * velocity.  x0: device [n][3] start positions (FP64).  Synchronous. */
wt_status wt_drift(wt_ctx* ctx, const float* E, const double* x0, const double* smu, int n, int n_steps, double dt,
                   float* x, float* y, float* z, float* vx, float* vy, float* vz, void* cuda_stream);

/* Front-end shaping of Eq. 1 currents.  The paper names the readout
 * electronics as the next step of the signal chain without giving a
 * transfer function; this is the common CR-(RC)^n shaper of unit area,
 *   h(t) = (t / tau)^n e^(-t / tau) / (n! tau),  peak at t = n tau,
 * applied on the output grid of wt_eq1 by the rectangle rule,
 *   v[tr][m] = gain * sum_k h(k dt) dt i[tr][m - k]  +  noise_rms * noise[tr][m],
 * with FP64 accumulation (taps beyond (n + 60) tau dropped).  i, noise (may
 * be NULL) and v: device arrays [n_tracks][n_out] (FP32); the noise samples
 * are drawn by the caller.  Asynchronous on cuda_stream.  n_out is limited
 * by one block's shared memory (12 bytes per sample, 200 KB). */
typedef struct {
    double tau;        /* shaping time constant [s] */
    int order;         /* n, 0..20 */
    double gain;       /* output per unit current */
    double noise_rms;  /* scale of the caller's noise samples */
} wt_shaper;
wt_status wt_shape(wt_ctx* ctx, const float* i, int n_tracks, int n_out, double dt, const wt_shaper* shaper,
                   const float* noise, float* v, void* cuda_stream);

/* Eq. 1 currents and their tangents along the four parameters of
 * wt_eq1_loss_grad (same chain, same parameters): i ([n_tracks][n_out]) and
 * di ([4][n_tracks][n_out], di/ds_R, di/ds_B, di/dr, di/dlambda), FP32
 * device buffers, either may be NULL; loss and grad (4 values) may be NULL.
 * Forward-mode derivatives of every current sample, for sensitivities of
 * signal features (wt_features).  Synchronous. */
wt_status wt_eq1_tangents(wt_ctx* ctx, const wt_tracks* tracks, float* i, float* di, double* loss, double* grad);

/* Signal-shape features of sampled waveforms, for the geometry scans of
 * Sec. 5 (sensor variants compared by the shape of their signals).  For
 * waveform r (x[r][m], m = 0..n-1, at tau_m = t0 + m dt):
 *   f[r][0] amplitude A = x_k, k the first index of the largest |x|;
 *   f[r][1] peak time tau_k + dt delta, delta the vertex of the parabola
 *           through samples k-1, k, k+1 (0 at the grid ends);
 *   f[r][2] charge dt sum_m x_m;
 *   f[r][3..5] leading-edge crossings of the levels lo A, hi A, cfd A:
 *           the last sample before k below the level (in s x, s = sign A)
 *           and linear interpolation to the next; t0 if there is none.
 * The indices are decided in FP32 (each level is one rounded FP32
 * product), the features evaluated in FP64.  With n_dir > 0 tangent
 * waveforms dx[d][r][m] (for example wt_eq1_tangents' di) give
 * df[d][r][0..5], the features' derivatives at fixed indices.  x, dx: FP32
 * device arrays; f, df: FP64 device arrays.  opts NULL: lo 0.1, hi 0.9,
 * cfd 0.5; each fraction in (0, 1].  n >= 1.  Asynchronous on
 * cuda_stream. */
#define WT_N_FEATURES 6
typedef struct {
    float lo, hi, cfd;
} wt_feature_opts;
wt_status wt_features(wt_ctx* ctx, const float* x, int n_tracks, int n, double t0, double dt,
                      const wt_feature_opts* opts, const float* dx, int n_dir, double* f, double* df,
                      void* cuda_stream);

/* Wait for the context's work and for cuda_stream, and report a device-side
 * failure of earlier asynchronous calls (wt_extend / wt_batch_run into
 * device buffers, wt_eq1): WT_ERR_TIMEOUT if a bounded wait in a kernel gave
 * up (the kernel unwound and freed its resources; the context stays
 * usable), WT_ERR_NAN for a non-finite result.  The error word is cleared.
 *
 * Failure injection for tests: the environment variable WT_FAULT, a comma
 * separated list of fit_singular (wt_fit reports WT_ERR_NOT_SPD),
 * alloc (every device allocation fails with WT_ERR_OOM), nan_q (wt_relax
 * meets a non-finite charge: WT_ERR_NAN) and queue_stall (the tensor-core
 * expansion withholds its accumulator signals, its bounded waits run out
 * after about 2 s and the call reports WT_ERR_TIMEOUT). */
wt_status wt_sync(wt_ctx* ctx, void* cuda_stream);

/* Copy intermediate results to host memory (for checks and diagnostics):
 * q: [n_t][n_sources] node charges (after wt_relax);
 * cn: [n_sources][n_sources] capacitance (after wt_fit);
 * mu: [n_sources - 1] relaxation rates (after wt_relax). */
wt_status wt_get_charges(wt_ctx* ctx, double* q);
wt_status wt_get_capacitance(wt_ctx* ctx, double* cn);
wt_status wt_get_modes(wt_ctx* ctx, double* mu);
wt_status wt_get_info(wt_ctx* ctx, wt_info* info);

/* Stage timing of wt_extend (instrumentation, off by default).  With
 * wt_set_timing(ctx, 1), each wt_extend records CUDA events on the stream it
 * launches on around its stages; wt_get_timing then waits for them and
 * returns ms[0] = column transforms, ms[1] = spectral passes, ms[2] =
 * expansion (FP32 path; 0 for FP64), and the number of kernels the call
 * launched. */
wt_status wt_set_timing(wt_ctx* ctx, int enable);
wt_status wt_get_timing(wt_ctx* ctx, double* ms3, int* n_launches);

/* Stage timing of the last wt_eq1_loss_grad / wt_eq1_loss_grad_profile /
 * wt_eq1_tangents call made with timing on (wt_set_timing), in ms of GPU
 * time between CUDA events on the context's stream, summed over the
 * parameters: ms6[0] base field, currents and loss; [1] the tables shared by
 * the tangents (fit residual, modal factors, potentials, cosine tables);
 * [2] fit tangents dC_n (derivative of the fit matrix, products, triangular
 * solves); [3] resistive-line and modal tangents and the charge tangent
 * dq(t); [4] time bases of the charge tangents; [5] tangent fields and
 * currents (extensions and Eq. 1).  All zero when timing was off. */
wt_status wt_get_grad_timing(wt_ctx* ctx, double* ms6);

/* Message of the last failed call on ctx (or of a failed wt_create when
 * ctx is NULL); valid until the next call on ctx. */
const char* wt_last_error(const wt_ctx* ctx);

/* Release the context and its device memory.  NULL is a no-op. */
void wt_destroy(wt_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* WT_H */
