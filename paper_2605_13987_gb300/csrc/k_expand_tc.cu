// Tensor-core expansion of the FP32 basis fields over time (the dense
// source/basis -> grid step of the bulk extension, Sec. 3's V_ext
// superposition of rescaled fundamental-solution chunks, here in its
// time-compressed form):
//
//   H[t][c][p] = sum_{m < 32} W[t][m] E[c][m][p]
//
// One CTA per SM, persistent over work units (128 grid points x one field
// component).  Per unit the 128 x 32 slice of E arrives by a 2D TMA load
// (double buffered) and is split into TF32 hi/lo parts in shared memory
// (128-byte swizzled, K-major); the time coefficients W (hi/lo) stay in
// shared memory for the whole kernel.  Three tcgen05.mma products
// (hi*hi + hi*lo + lo*hi, kind::tf32, FP32 accumulation in tensor memory)
// give FP32-level accuracy.  The accumulator D[p][t] lives in TMEM (lane =
// grid point, column = time sample), double buffered in two 256-column
// halves; eight, twelve or sixteen epilogue warps (two to four per TMEM lane
// quadrant, alternate 32-column slices) drain it with tcgen05.ld, transpose 4 x 4 blocks within
// lane quads by shuffles and write H with 16-byte stores: each warp store
// covers 4 time samples x 32 consecutive grid points (four full 128-byte
// lines), a quarter of the store instructions of one float per lane.  The
// 8-byte variant (2 x 2 transposes within lane pairs) halves the shuffles,
// which share the load/store data pipe with the stores, for twice the stores;
// the 4-byte variant stores straight from the TMEM layout (one 128-byte line
// per warp store, no shuffles).
//
// A launch may cover several expansions at once (one per sensor geometry of a
// batch, each with its own basis fields, coefficients, grid size and time
// count): the units of all jobs form one sequence that the persistent CTAs
// share round-robin.  When a CTA moves on to the next job, the producer waits
// until the MMAs of the previous job have completed and rewrites the
// coefficient tiles in shared memory.
//
// Warp roles: two producer warps (warp 0 and the last warp; each loads its
// half of the 128-point slice by TMA and splits it into hi/lo, with its own
// TMA barriers, so neither waits on the other), warp 1 TMEM owner + MMA
// issuer, warps 2 .. 1 + NEPI epilogue.  Every mbarrier wait gives up
// after ~2 s (globaltimer), sets the device error word and lets the CTA
// unwind: the producer waits (bounded) for the TMA loads it still has in
// flight and the MMA thread drains its own MMAs before tensor memory is
// freed.
#include "wt_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace wt {

namespace tc {

constexpr int BM = 128;            // grid points per unit (TMEM lanes)
// epilogue warps: a template parameter of the kernel (8 or 16, chosen by the autotuner)
constexpr int KR = 32;             // basis rank (TF32 elements per 128-byte row)
constexpr int NCH = 256;           // default time samples per accumulator chunk (a launch argument: 64, 128, 256)
constexpr int TMEM_COLS = 512;     // allocated accumulator columns: 512 / chunk buffers
constexpr int TILE_BYTES = BM * 128;  // one 128 x 32 TF32 tile
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;
constexpr int MAX_JOBS = 64;       // expansion jobs per launch

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false on timeout (and the abort flag is raised).
// Every caller is a whole warp: the lanes vote, so that a warp either proceeds or unwinds as
// one (a lane that saw the phase complete while another saw the abort flag takes the abort),
// and no warp-collective instruction after the wait sees a divided warp.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, volatile int* abort_flag,
                                          int* d_err) {
    bool ok = mbar_try(b, parity);
    if (!ok) {
        const unsigned long long t0 = globaltimer();
        while (true) {
            if (mbar_try(b, parity)) { ok = true; break; }
            if (*abort_flag) break;
            if (globaltimer() - t0 > TIMEOUT_NS) {
                *abort_flag = 1;
                atomicMax(d_err, (int)DERR_TIMEOUT);
                break;
            }
        }
    }
    return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// 2D tiled TMA load into shared memory, completion signalled on an mbarrier
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// Drain wait used while unwinding: ignores the abort flag, still bounded in time.
__device__ __forceinline__ bool mbar_wait_drain(unsigned long long* b, unsigned parity, int* d_err) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_try(b, parity)) {
        if (globaltimer() - t0 > TIMEOUT_NS) {
            atomicMax(d_err, (int)DERR_TIMEOUT);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ unsigned to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// byte offset of element (row, k) in a 128-byte-swizzled K-major tile
__device__ __forceinline__ unsigned sw128(int row, int k) {
    return (unsigned)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 2) ^ (row & 7))) << 4) + ((k & 3) << 2));
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ unsigned long long sdesc(unsigned addr) {
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) |
           (2ull << 61);
}
__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// Issue a 32-column TMEM load without waiting (tcgen05.wait::ld before the values are read).
__device__ __forceinline__ void tmem_ld32_nowait(unsigned taddr, unsigned (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float* v) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int RAW_BYTES = KR * BM * 4;   // one raw FP32 slice [32 basis][128 points], two halves
constexpr int HALF = BM / 2;             // points per producer warp

// 4 x 4 transposes within lane quads: on entry lane 4g + i holds v[4b + j] =
// D[point 4g + i][time 4b + j]; on return v[4b + j] = D[point 4g + j][time 4b + i],
// so that each lane can store 4 consecutive points of one time sample.
// Two butterfly exchanges per block (lanes i ^ 2, then i ^ 1).
__device__ __forceinline__ void quad_transpose(float (&v)[32], int lane) {
    const bool b1 = lane & 2, b0 = lane & 1;
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
        float* m = v + 4 * bb;
        const float s0 = b1 ? m[0] : m[2], s1 = b1 ? m[1] : m[3];
        const float r0 = __shfl_xor_sync(0xffffffffu, s0, 2), r1 = __shfl_xor_sync(0xffffffffu, s1, 2);
        if (b1) { m[0] = r0; m[1] = r1; } else { m[2] = r0; m[3] = r1; }
        const float u0 = b0 ? m[0] : m[1], u1 = b0 ? m[2] : m[3];
        const float w0 = __shfl_xor_sync(0xffffffffu, u0, 1), w1 = __shfl_xor_sync(0xffffffffu, u1, 1);
        if (b0) { m[0] = w0; m[2] = w1; } else { m[1] = w0; m[3] = w1; }
    }
}

struct Smem {
    // tiles first (1024-byte aligned base):
    // B_hi[nt_pad x 128 B], B_lo[...], A[2 stages][hi, lo], raw[2][32][128] FP32
    unsigned long long a_full[2], a_empty[2], acc_full[2], acc_empty[2], raw_full[2][2], drain, b_free;
    unsigned tmem_base;
    int abort_flag;
};

// Expansion jobs of one launch (kernel parameter; the tensor maps must live
// in parameter space).  Job j covers units [unit_end[j-1], unit_end[j]).
struct Jobs {
    CUtensorMap emap[MAX_JOBS];
    const float* W[MAX_JOBS];
    float* H[MAX_JOBS];
    unsigned long long npts[MAX_JOBS];
    int nt[MAX_JOBS];
    int r[MAX_JOBS];             // basis vectors in use (rows >= r of E are not read)
    int unit_end[MAX_JOBS];
    int n_jobs;
};

__device__ __forceinline__ int job_of(const Jobs& J, int u, int from) {
    int j = from;
    while (j + 1 < J.n_jobs && u >= J.unit_end[j]) ++j;
    return j;
}
__device__ __forceinline__ int unit0_of(const Jobs& J, int j) { return j ? J.unit_end[j - 1] : 0; }
__device__ __forceinline__ int pad32(int n) { return (n + 31) & ~31; }

// time coefficients of one job, split hi/lo, into the swizzled B tiles
// (rows = time samples); threads [t0, t0 + nthr) of the CTA take part
__device__ __forceinline__ void load_coeffs(const float* __restrict__ W, int nt, int nt_pad, unsigned char* b_hi,
                                            unsigned char* b_lo, int tid, int nthr) {
    for (int e = tid; e < nt_pad * KR; e += nthr) {
        const int t = e / KR, k = e % KR;
        const float v = t < nt ? W[(size_t)t * KR + k] : 0.f;
        const unsigned hi = to_tf32(v);
        const unsigned lo = to_tf32(v - __uint_as_float(hi));
        *reinterpret_cast<unsigned*>(b_hi + sw128(t, k)) = hi;
        *reinterpret_cast<unsigned*>(b_lo + sw128(t, k)) = lo;
    }
}

// 2 x 2 transposes within lane pairs: on entry lane 2g + i holds v[2b + j] =
// D[point 2g + i][time 2b + j]; on return v[2b + j] = D[point 2g + j][time 2b + i].
__device__ __forceinline__ void pair_transpose(float (&v)[32], int lane) {
    const bool b0 = lane & 1;
#pragma unroll
    for (int bb = 0; bb < 16; ++bb) {
        float* m = v + 2 * bb;
        const float r = __shfl_xor_sync(0xffffffffu, b0 ? m[0] : m[1], 1);
        if (b0) m[0] = r; else m[1] = r;
    }
}

template <int NEPI, int VEC>
__global__ void __launch_bounds__(96 + 32 * NEPI, 1)
    expand_tc_kernel(const __grid_constant__ Jobs J, int nt_pad_max, int n_units, int nch, int stall,
                     int* __restrict__ d_err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // align the tile region to 1024 bytes
    unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    unsigned char* b_hi = base;
    unsigned char* b_lo = b_hi + (size_t)nt_pad_max * 128;
    unsigned char* a_tiles = b_lo + (size_t)nt_pad_max * 128;      // [stage][hi|lo] x TILE_BYTES
    float* raw = reinterpret_cast<float*>(a_tiles + 4 * TILE_BYTES);  // [2 stages][2 halves][KR][HALF]
    Smem* S = reinterpret_cast<Smem*>(reinterpret_cast<unsigned char*>(raw) + 2 * RAW_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int job0 = job_of(J, blockIdx.x, 0);

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S->a_full[i], 64);            // both producer warps
            mbar_init(&S->a_empty[i], 1);
            mbar_init(&S->raw_full[i][0], 1);
            mbar_init(&S->raw_full[i][1], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S->acc_full[i], 1);
            mbar_init(&S->acc_empty[i], 32 * NEPI);
        }
        mbar_init(&S->drain, 1);
        mbar_init(&S->b_free, 1);
        S->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    load_coeffs(J.W[job0], J.nt[job0], pad32(J.nt[job0]), b_hi, b_lo, threadIdx.x, blockDim.x);
    fence_proxy_async();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)), "n"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = S->tmem_base;
    // two accumulator buffers of TMEM_COLS / 2 columns (one chunk each); deeper buffering (512 / chunk
    // buffers) measured 2-3 % slower on c2
    constexpr int nbuf = 2, bstride = TMEM_COLS / 2;
    volatile int* abort_flag = &S->abort_flag;

    if (warp == 0 || warp == 2 + NEPI) {
        // ---------------- producers: TMA loads of raw E half slices, hi/lo conversion into swizzled A tiles
        const int h = warp == 0 ? 0 : 1;             // points h HALF .. h HALF + HALF - 1 of each unit
        float* rawh = raw + h * KR * HALF;           // stage st at rawh + st * KR * BM
        int issued = 0;          // raw loads issued (unit k of this CTA goes to buffer k & 1)
        if (lane == 0)
            for (int jl = job0; issued < 2; ++issued) {
                const int u = blockIdx.x + issued * gridDim.x;
                if (u >= n_units) break;
                jl = job_of(J, u, jl);
                const int v = u - unit0_of(J, jl);
                mbar_expect_tx(&S->raw_full[issued][h], RAW_BYTES / 2);
                tma_load_2d(rawh + issued * KR * BM, &J.emap[jl], (v / 3) * BM + h * HALF, (v % 3) * KR,
                            &S->raw_full[issued][h]);
            }
        issued = __shfl_sync(0xffffffffu, issued, 0);
        int i = 0, cur = job0, jnext = job0, n_changes = 0;
        for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++i) {
            const int st = i & 1;
            const int j = job_of(J, u, cur);
            if (j != cur) {
                // new job: wait until the MMAs of the previous one are done, then its coefficients
                if (!mbar_wait(&S->b_free, n_changes & 1, abort_flag, d_err)) break;
                ++n_changes;
                load_coeffs(J.W[j], J.nt[j], pad32(J.nt[j]), b_hi, b_lo, h * 32 + lane, 64);
                cur = j;
            }
            if (!mbar_wait(&S->a_empty[st], ((i >> 1) & 1) ^ 1, abort_flag, d_err)) break;
            if (!mbar_wait(&S->raw_full[st][h], (i >> 1) & 1, abort_flag, d_err)) break;
            unsigned char* ah = a_tiles + (size_t)(2 * st) * TILE_BYTES;
            unsigned char* al = ah + TILE_BYTES;
            const float* rb = rawh + st * KR * BM;               // [KR][HALF]
            const int rk = J.r[cur];
#pragma unroll
            for (int rr = 0; rr < HALF / 32; ++rr) {
                const int hr = lane + 32 * rr;                    // lane = grid point of this half
                const int row = h * HALF + hr;
#pragma unroll
                for (int c = 0; c < KR / 4; ++c) {
                    unsigned hi[4], lo[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float x = (4 * c + j) < rk ? rb[(4 * c + j) * HALF + hr] : 0.f;
                        hi[j] = to_tf32(x);
                        lo[j] = to_tf32(x - __uint_as_float(hi[j]));
                    }
                    const unsigned off = sw128(row, 4 * c);
                    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(smem_u32(ah + off)), "r"(hi[0]),
                                 "r"(hi[1]), "r"(hi[2]), "r"(hi[3])
                                 : "memory");
                    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(smem_u32(al + off)), "r"(lo[0]),
                                 "r"(lo[1]), "r"(lo[2]), "r"(lo[3])
                                 : "memory");
                }
            }
            fence_proxy_async();     // A tiles for the tensor core; raw buffer reads before the TMA refill
            __syncwarp();
            const int u2 = u + 2 * gridDim.x;
            if (u2 < n_units) jnext = job_of(J, u2, max(jnext, cur));
            if (lane == 0 && u2 < n_units) {
                const int v2 = u2 - unit0_of(J, jnext);
                mbar_expect_tx(&S->raw_full[st][h], RAW_BYTES / 2);
                tma_load_2d(rawh + st * KR * BM, &J.emap[jnext], (v2 / 3) * BM + h * HALF, (v2 % 3) * KR,
                            &S->raw_full[st][h]);
            }
            if (u + 2 * gridDim.x < n_units) ++issued;
            mbar_arrive(&S->a_full[st]);
        }
        // loads still in flight after an abort: wait for them (bounded) before the CTA exits
        for (int k = i; k < issued; ++k) mbar_wait_drain(&S->raw_full[k & 1][h], (k >> 1) & 1, d_err);
    } else if (warp == 1) {
        // ---------------- MMA issuer (lane 0)
        int i = 0, g = 0, cur = job0;
        bool ok = true;
        for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++i) {
            const int st = i & 1;
            cur = job_of(J, u, cur);
            const int nt_pad = pad32(J.nt[cur]);
            const int n_chunks = (nt_pad + nch - 1) / nch;
            if (!mbar_wait(&S->a_full[st], (i >> 1) & 1, abort_flag, d_err)) { ok = false; break; }
            tc_fence_after();
            const unsigned a_hi = smem_u32(a_tiles + (size_t)(2 * st) * TILE_BYTES);
            const unsigned a_lo = a_hi + TILE_BYTES;
            for (int ch = 0; ch < n_chunks; ++ch, ++g) {
                const int b = g % nbuf;
                if (!mbar_wait(&S->acc_empty[b], ((g / nbuf) & 1) ^ 1, abort_flag, d_err)) { ok = false; break; }
                tc_fence_after();
                const int n = min(nch, nt_pad - ch * nch);
                const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) |
                                       ((unsigned)(BM >> 4) << 24);
                if (lane == 0) {
                    const unsigned bh = smem_u32(b_hi + (size_t)ch * nch * 128);
                    const unsigned bl = smem_u32(b_lo + (size_t)ch * nch * 128);
                    const unsigned d = tmem + (unsigned)(b * bstride);
#pragma unroll
                    for (int ks = 0; ks < KR / 8; ++ks) {
                        const unsigned off = ks * 32;   // 8 TF32 = 32 bytes along K
                        mma_tf32(d, sdesc(a_lo + off), sdesc(bh + off), idesc, ks > 0);
                        mma_tf32(d, sdesc(a_hi + off), sdesc(bl + off), idesc, 1);
                        mma_tf32(d, sdesc(a_hi + off), sdesc(bh + off), idesc, 1);
                    }
                    if (!stall) mma_commit(&S->acc_full[b]);     // stall: injected fault (WT_FAULT=queue_stall)
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) {
                mma_commit(&S->a_empty[st]);
                // last unit of this job for this CTA: its coefficient tiles may be replaced once these MMAs finish
                const int un = u + gridDim.x;
                if (un < n_units && job_of(J, un, cur) != cur) mma_commit(&S->b_free);
            }
            __syncwarp();
        }
        // drain: every MMA this thread issued has completed before TMEM is freed
        if (lane == 0) {
            mma_commit(&S->drain);
            mbar_wait_drain(&S->drain, 0, d_err);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM -> H; warps 2 .. 1 + NEPI, quadrant warp & 3, column slice (warp - 2) / 4
        const int q = warp & 3;
        const int slice = (warp - 2) >> 2;
        constexpr int NSL = NEPI / 4;
        int g = 0, cur = job0;
        bool ok = true;
        for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            cur = job_of(J, u, cur);
            const int v = u - unit0_of(J, cur);
            const int tile = v / 3, c = v % 3;
            const size_t npts = J.npts[cur];
            const int nt = J.nt[cur], nt_pad = pad32(nt);
            const int n_chunks = (nt_pad + nch - 1) / nch;
            // after the transposes lane VEC g + i stores points VEC g .. VEC g + VEC - 1 of time VEC b + i
            const size_t p4 = (size_t)tile * BM + q * 32 + VEC * (lane / VEC);
            const bool in = p4 < npts;                 // npts is a multiple of 4
            float* hp = J.H[cur] + (size_t)c * npts + p4;
            for (int ch = 0; ch < n_chunks; ++ch, ++g) {
                const int b = g % nbuf;
                if (!mbar_wait(&S->acc_full[b], (g / nbuf) & 1, abort_flag, d_err)) { ok = false; break; }
                tc_fence_after();
                const int n = min(nch, nt_pad - ch * nch);
                // two 32-column slices per round: both TMEM loads in flight before one wait
                for (int j = slice * 32; j < n; j += 64 * NSL) {
                    const int j2 = j + 32 * NSL;
                    const bool two = j2 < n;
                    unsigned ra[32], rb[32];
                    tmem_ld32_nowait(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(b * bstride + j), ra);
                    if (two) tmem_ld32_nowait(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(b * bstride + j2), rb);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h == 1 && !two) break;
                        float v[32];
#pragma unroll
                        for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(h ? rb[e] : ra[e]);
                        const int t0 = ch * nch + (h ? j2 : j) + (lane & (VEC - 1));
                        // rows t0 + VEC k (k < 32 / VEC) of this lane; all of them exist unless the
                        // slice reaches past nt (then each store is checked)
                        const bool full = t0 + 32 - VEC < nt;
                        const size_t rs = (size_t)VEC * 3 * npts;      // row step between stores
                        float* hr = hp + (size_t)t0 * 3 * npts;
                        if constexpr (VEC == 4) quad_transpose(v, lane);
                        else if constexpr (VEC == 2) pair_transpose(v, lane);
                        if (in) {
#pragma unroll
                            for (int k = 0; k < 32 / VEC; ++k) {
                                if (!full && t0 + VEC * k >= nt) break;
                                float* dst = hr + k * rs;
                                if constexpr (VEC == 4)
                                    *reinterpret_cast<float4*>(dst) =
                                        make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                                else if constexpr (VEC == 2)
                                    *reinterpret_cast<float2*>(dst) = make_float2(v[2 * k], v[2 * k + 1]);
                                else
                                    *dst = v[k];
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&S->acc_empty[b]);
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
    }
}

}  // namespace tc

bool expand_tc_available() { return true; }

size_t expand_tc_smem(int nt_pad) {
    return 1024 + (size_t)2 * nt_pad * 128 + 4 * (size_t)tc::TILE_BYTES + 2 * (size_t)tc::RAW_BYTES + sizeof(tc::Smem);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        WT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) fail(WT_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static void encode_basis_map(CUtensorMap* m, const float* E, size_t npts) {
    // E viewed as 96 rows (component x basis index) of npts points; one box = 32 rows x 64 points
    // (half a unit: each producer warp loads its own half)
    cuuint64_t dims[2] = {(cuuint64_t)npts, (cuuint64_t)3 * tc::KR};
    cuuint64_t strides[1] = {(cuuint64_t)npts * sizeof(float)};
    cuuint32_t box[2] = {tc::HALF, tc::KR};
    cuuint32_t es[2] = {1, 1};
    CUresult r = tensor_map_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(E), dims, strides, box,
                                      es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(WT_ERR_CUDA, "tensor map for the basis fields: error " + std::to_string((int)r));
}

int expand_tc_max_jobs() { return tc::MAX_JOBS; }

// jobs[j]: E [3][32][npts] FP32, W [nt][32] FP32, H [nt][3][npts] FP32; all
// expansions in one persistent launch of at most `max_ctas` CTAs (0: one per SM).
template <int VEC>
static void launch_expand(int nepi, int grid, size_t sh, cudaStream_t s, const tc::Jobs& J, int nt_pad_max, int units,
                          int nch, int stall, int* d_err) {
    if (nepi == 8) {
        allow_dyn_smem(tc::expand_tc_kernel<8, VEC>, sh);
        tc::expand_tc_kernel<8, VEC><<<grid, 96 + 32 * 8, sh, s>>>(J, nt_pad_max, units, nch, stall, d_err);
    } else if (nepi == 12) {
        allow_dyn_smem(tc::expand_tc_kernel<12, VEC>, sh);
        tc::expand_tc_kernel<12, VEC><<<grid, 96 + 32 * 12, sh, s>>>(J, nt_pad_max, units, nch, stall, d_err);
    } else {
        allow_dyn_smem(tc::expand_tc_kernel<16, VEC>, sh);
        tc::expand_tc_kernel<16, VEC><<<grid, 96 + 32 * 16, sh, s>>>(J, nt_pad_max, units, nch, stall, d_err);
    }
}

void expand_tc_jobs(cudaStream_t s, const ExpandJob* jobs, int n_jobs, int max_ctas, int nch, int* d_err, int nepi,
                    int vec) {
    if (n_jobs < 1) return;
    if (nch != 64 && nch != 128 && nch != 256) fail(WT_ERR_ARG, "expansion time chunk must be 64, 128 or 256");
    if (n_jobs > tc::MAX_JOBS) fail(WT_ERR_UNSUPPORTED, "too many expansion jobs for one launch");
    tc::Jobs J;             // kernel parameter block (about 10 KB)
    int nt_pad_max = 32, units = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const ExpandJob& jb = jobs[j];
        if (jb.r_pad != tc::KR) fail(WT_ERR_UNSUPPORTED, "tensor-core expansion needs rank padded to 32");
        if (jb.r < 0 || jb.r > tc::KR) fail(WT_ERR_ARG, "basis rank out of range");
        const int nt_pad = ((jb.nt + 31) / 32) * 32;
        if (jb.nt < 1 || nt_pad > 512) fail(WT_ERR_UNSUPPORTED, "tensor-core expansion handles 1 to 512 time samples");
        if (jb.npts % 4) fail(WT_ERR_UNSUPPORTED, "grid size must be a multiple of 4");
        if (reinterpret_cast<uintptr_t>(jb.E) % 16) fail(WT_ERR_ARG, "basis fields must be 16-byte aligned");
        if (reinterpret_cast<uintptr_t>(jb.H) % 16) fail(WT_ERR_ARG, "H must be 16-byte aligned");
        const size_t n_tiles = (jb.npts + tc::BM - 1) / tc::BM;
        if ((size_t)units + 3 * n_tiles > (size_t)INT32_MAX) fail(WT_ERR_UNSUPPORTED, "expansion batch too large");
        encode_basis_map(&J.emap[j], jb.E, jb.npts);
        J.W[j] = jb.W;
        J.H[j] = jb.H;
        J.npts[j] = jb.npts;
        J.nt[j] = jb.nt;
        J.r[j] = jb.r;
        units += (int)(3 * n_tiles);
        J.unit_end[j] = units;
        nt_pad_max = std::max(nt_pad_max, nt_pad);
    }
    J.n_jobs = n_jobs;
    const size_t sh = expand_tc_smem(nt_pad_max);
    int dev = 0, n_sm = 0, max_sh = 0;
    WT_CUDA(cudaGetDevice(&dev));
    WT_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    WT_CUDA(cudaDeviceGetAttribute(&max_sh, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (sh > (size_t)max_sh) fail(WT_ERR_UNSUPPORTED, "expansion tile does not fit shared memory");
    if (nepi != 8 && nepi != 12 && nepi != 16) fail(WT_ERR_ARG, "expansion epilogue warps must be 8, 12 or 16");
    if (vec != 1 && vec != 2 && vec != 4) fail(WT_ERR_ARG, "expansion store width must be 1, 2 or 4 floats");
    int grid = std::min(n_sm, units);
    if (max_ctas > 0) grid = std::min(grid, max_ctas);
    // WT_FAULT=queue_stall: the MMA warp withholds its accumulator-ready signals, so the epilogue's
    // bounded waits run out and the kernel unwinds with DERR_TIMEOUT (tests of the failure path)
    const int stall = fault_enabled("queue_stall") ? 1 : 0;
    if (vec == 4) launch_expand<4>(nepi, grid, sh, s, J, nt_pad_max, units, nch, stall, d_err);
    else if (vec == 2) launch_expand<2>(nepi, grid, sh, s, J, nt_pad_max, units, nch, stall, d_err);
    else launch_expand<1>(nepi, grid, sh, s, J, nt_pad_max, units, nch, stall, d_err);
    WT_LAUNCH("expand_tc");
}

// E: [3][32][npts] FP32 (rows >= r unused), W: [nt][32] FP32, H: [nt][3][npts] FP32.
void expand_tc(cudaStream_t s, const float* E, int r_pad, int r, const float* W, int nt, size_t npts, float* H,
               int* d_err) {
    ExpandJob jb{E, r_pad, r, W, nt, npts, H};
    expand_tc_jobs(s, &jb, 1, 0, tc::NCH, d_err, 8, 4);
}

}  // namespace wt
