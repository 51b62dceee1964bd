// Warp-level FFT held in registers (inverse sign exp(+i), unnormalised).
//
// A line of length N = W * R is owned by W lanes of a warp (W a power of two
// <= 32), R elements per lane: lane l (0 <= l < W) starts with
// v[j1] = x[j1 + R l].  Decomposition j = j1 + R j2, k = k2 + W k1:
//   X[k2 + W k1] = sum_j1 w_R^{j1 k1} w_N^{j1 k2} sum_j2 x[j1 + R j2] w_W^{j2 k2}
// (1) W-point DFTs across lanes (decimation in frequency with __shfl_xor,
//     output bit-reversed across lanes), (2) twiddles w_N^{j1 k2},
// (3) R-point DFTs in registers.  On return lane l holds
// v[k1] = X[bitrev_W(l) + W k1].  32/W lines share a warp (lane groups).
// tw: table of w_N^k = exp(+2 pi i k / N), k < N.
#pragma once
#include "fft_core.cuh"
#include <type_traits>

namespace wt {

// R-point DFT in registers (exp(+i)); w_R^m = tw[(m mod R) * U] with U = N / R
// the table's stride for this DFT length (no runtime division inside).
template <int R>
__device__ __forceinline__ void reg_dft(C2<float> (&v)[R], const C2<float>* __restrict__ tw, int U) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        const C2<float> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const C2<float> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const C2<float> s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
        const C2<float> id13 = {-d13.y, d13.x};
        v[0] = cadd(s02, s13);
        v[1] = cadd(d02, id13);
        v[2] = csub(s02, s13);
        v[3] = csub(d02, id13);
    } else if constexpr (R == 3 || R == 5 || R == 7) {
        C2<float> o[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            C2<float> acc = v[0];
#pragma unroll
            for (int j = 1; j < R; ++j) acc = cadd(acc, cmul(v[j], tw[((j * k) % R) * U]));
            o[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = o[k];
    } else {
        // R = A * B: B-point DFTs over x[j1 + A j2], twiddle w_R^{j1 k2}, A-point DFTs
        constexpr int A = (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : (R % 3 == 0) ? 3 : (R % 5 == 0) ? 5 : 7;
        constexpr int B = R / A;
        static_assert(A * B == R, "unsupported register DFT length");
        C2<float> y[A][B];
#pragma unroll
        for (int j1 = 0; j1 < A; ++j1) {
            C2<float> t[B];
#pragma unroll
            for (int j2 = 0; j2 < B; ++j2) t[j2] = v[j1 + A * j2];
            reg_dft<B>(t, tw, U * A);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) y[j1][k2] = (j1 && k2) ? cmul(t[k2], tw[((j1 * k2) % R) * U]) : t[k2];
        }
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            C2<float> t[A];
#pragma unroll
            for (int j1 = 0; j1 < A; ++j1) t[j1] = y[j1][k2];
            reg_dft<A>(t, tw, U * B);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) v[k2 + B * k1] = t[k1];
        }
    }
}

template <int R>
__device__ __forceinline__ void warp_fft(C2<float> (&v)[R], int gl, int W, const C2<float>* __restrict__ tw, int N) {
    (void)N;
    // (1) W-point DFTs across the lane group, one per j1; the stage twiddle
    // w_{2h}^{gl mod h} = tw[(gl mod h) * R * W / (2h)], stride doubling as h halves
    int step = R;
    for (int h = W >> 1; h >= 1; h >>= 1, step <<= 1) {
        const bool bottom = gl & h;
        const C2<float> w = tw[(gl & (h - 1)) * step];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const C2<float> a = v[j];
            const C2<float> b = {__shfl_xor_sync(0xffffffffu, a.x, h), __shfl_xor_sync(0xffffffffu, a.y, h)};
            v[j] = bottom ? cmul(csub(b, a), w) : cadd(a, b);
        }
    }
    // (2) twiddles w_N^{j1 k2}, k2 = bit-reversed lane
    const int lw = 31 - __clz(W);                 // log2 W
    const int k2 = lw ? (int)(__brev((unsigned)gl) >> (32 - lw)) : 0;
#pragma unroll
    for (int j = 1; j < R; ++j) v[j] = cmul(v[j], tw[j * k2]);          // j k2 < N
    // (3) R-point DFTs in registers: X[k2 + W k1] = sum_j1 w_R^{j1 k1} ...
    reg_dft<R>(v, tw, W);
}

// Decimation-in-time form: lane l starts with v[j1] = x[l + W j1] (consecutive
// lanes hold consecutive elements) and ends with v[k1] = X[k1 + R bitrev_W(l)]:
//   X[k1 + R k2] = sum_j2 w_W^{j2 k2} w_N^{j2 k1} sum_j1 x[j2 + W j1] w_R^{j1 k1}.
template <int R>
__device__ __forceinline__ void warp_fft_dit(C2<float> (&v)[R], int gl, int W, const C2<float>* __restrict__ tw,
                                             int N) {
    (void)N;
    reg_dft<R>(v, tw, W);
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[gl * k]);          // gl k < N
    int step = R;
    for (int h = W >> 1; h >= 1; h >>= 1, step <<= 1) {
        const bool bottom = gl & h;
        const C2<float> w = tw[(gl & (h - 1)) * step];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const C2<float> a = v[j];
            const C2<float> b = {__shfl_xor_sync(0xffffffffu, a.x, h), __shfl_xor_sync(0xffffffffu, a.y, h)};
            v[j] = bottom ? cmul(csub(b, a), w) : cadd(a, b);
        }
    }
}

// Per-lane twiddles of a W x R warp FFT, computed once per kernel: the
// cross-lane stage factors (stage s pairs lanes gl, gl ^ h with h = W >> (s+1);
// bottom lanes multiply b - a by w_{2h}^{gl mod h}, top lanes keep a + b, written
// as t = b + sg a, v = t st with st = 1 and sg = +1 on top lanes, sg = -1 below)
// and the twiddles between the register and cross-lane parts.
template <int R>
struct LaneTw {
    C2<float> st[5];
    C2<float> in[R];
};

// dit: inter twiddles w_N^{gl k} (decimation in time); else w_N^{j k2} (in frequency).
template <int R>
__device__ __forceinline__ void lane_twiddles(const C2<float>* __restrict__ tw, int gl, int W, bool dit,
                                              LaneTw<R>& t) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int h = W >> (s + 1);
        t.st[s] = {1.f, 0.f};
        if (h >= 1 && (gl & h)) t.st[s] = tw[(gl & (h - 1)) * R * (W / (2 * h))];
    }
    const int lw = 31 - __clz(W);
    const int k2 = lw ? (int)(__brev((unsigned)gl) >> (32 - lw)) : 0;
#pragma unroll
    for (int k = 0; k < R; ++k) t.in[k] = tw[(dit ? gl : k2) * k];
}

// Cross-lane stages with precomputed factors (h = W/2 .. 1).
template <int R>
__device__ __forceinline__ void lane_stages(C2<float> (&v)[R], int gl, int W, const LaneTw<R>& t) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int h = W >> (s + 1);
        if (h < 1) break;
        const C2<float> w = t.st[s];
        const float sg = (gl & h) ? -1.f : 1.f;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const C2<float> a = v[j];
            const C2<float> b = {__shfl_xor_sync(0xffffffffu, a.x, h), __shfl_xor_sync(0xffffffffu, a.y, h)};
            v[j] = cmul(C2<float>{fmaf(sg, a.x, b.x), fmaf(sg, a.y, b.y)}, w);
        }
    }
}

template <int R>
__device__ __forceinline__ void reg_dft_c(C2<float> (&v)[R]);

// R-point register DFT of the warp FFTs: compile-time twiddles where they exist
// (R = 8, 16: the same correctly rounded values as the table), else the table.
template <int R>
__device__ __forceinline__ void reg_dft_any(C2<float> (&v)[R], const C2<float>* __restrict__ tw, int W) {
    if constexpr (R == 8 || R == 16) reg_dft_c<R>(v);
    else reg_dft<R>(v, tw, W);
}

// warp_fft / warp_fft_dit with per-lane twiddles (same input and output orders).
template <int R>
__device__ __forceinline__ void warp_fft_t(C2<float> (&v)[R], int gl, int W, const LaneTw<R>& t,
                                           const C2<float>* __restrict__ tw) {
    lane_stages<R>(v, gl, W, t);
#pragma unroll
    for (int j = 1; j < R; ++j) v[j] = cmul(v[j], t.in[j]);
    reg_dft_any<R>(v, tw, W);
}
template <int R>
__device__ __forceinline__ void warp_fft_dit_t(C2<float> (&v)[R], int gl, int W, const LaneTw<R>& t,
                                               const C2<float>* __restrict__ tw) {
    reg_dft_any<R>(v, tw, W);
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], t.in[k]);
    lane_stages<R>(v, gl, W, t);
}

// cos(q pi / 8) for integer q (the sixteenth roots of unity, exp(+2 pi i m / 16) = cos + i sin
// with q = 2m): exact constants, folded at compile time.
__host__ __device__ constexpr float cos_pi8(int q) {
    q = ((q % 16) + 16) % 16;
    if (q > 8) q = 16 - q;
    return q == 0 ? 1.0f
         : q == 1 ? 0.92387953251128675613f
         : q == 2 ? 0.70710678118654752440f
         : q == 3 ? 0.38268343236508977173f
         : q == 4 ? 0.0f
         : q == 5 ? -0.38268343236508977173f
         : q == 6 ? -0.70710678118654752440f
         : q == 7 ? -0.92387953251128675613f
         : -1.0f;
}

// x w_R^M, w_R = exp(+2 pi i / R), R in {1, 2, 4, 8, 16}; the quarter turns are exact.
template <int R, int M>
__device__ __forceinline__ C2<float> twc(C2<float> x) {
    constexpr int q = (((M * (16 / R)) % 16) + 16) % 16;      // angle in units of pi / 8
    if constexpr (q == 0) return x;
    else if constexpr (q == 4) return {-x.y, x.x};
    else if constexpr (q == 8) return {-x.x, -x.y};
    else if constexpr (q == 12) return {x.y, -x.x};
    else {
        constexpr float c = cos_pi8(q), s = cos_pi8(q - 4);
        return {x.x * c - x.y * s, x.x * s + x.y * c};
    }
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// R-point DFT in registers with compile-time twiddles (exp(+i), natural order
// in and out), R in {1, 2, 4, 8, 16}: R = 4 B, B-point DFTs over x[j1 + 4 j2],
// twiddles w_R^{j1 k2}, 4-point DFTs.
template <int R>
__device__ __forceinline__ void reg_dft_c(C2<float> (&v)[R]) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2 || R == 4) {
        reg_dft<R>(v, nullptr, 0);
    } else {
        static_assert(R == 8 || R == 16, "compile-time twiddles cover R = 8, 16");
        constexpr int B = R / 4;
        C2<float> y[4][B];
        static_for<0, 4>([&](auto J1) {
            constexpr int j1 = decltype(J1)::value;
            C2<float> t[B];
#pragma unroll
            for (int j2 = 0; j2 < B; ++j2) t[j2] = v[j1 + 4 * j2];
            reg_dft_c<B>(t);
            static_for<0, B>([&](auto K2) {
                constexpr int k2 = decltype(K2)::value;
                y[j1][k2] = twc<R, j1 * k2>(t[k2]);
            });
        });
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            C2<float> t[4] = {y[0][k2], y[1][k2], y[2][k2], y[3][k2]};
            reg_dft<4>(t, nullptr, 0);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) v[k2 + B * k1] = t[k1];
        }
    }
}

// cos and sin of 2 pi q / R for the compile-time twiddles of the mixed-radix register DFTs:
// the angle reduced to [-pi, pi], then the Taylor series of cos and sin summed in double to far
// below float precision (terms up to x^40 / 40!), and rounded once to float.
__host__ __device__ constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 20; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k <= 20; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double turn_angle(int q, int R) {
    q = ((q % R) + R) % R;
    if (2 * q > R) q -= R;                      // q / R in (-1/2, 1/2]
    return 2.0 * 3.14159265358979323846 * (double)q / (double)R;
}

// x w_R^M with w_R = exp(+2 pi i / R) for any R; quarter and half turns exact.
template <int R, int M>
__device__ __forceinline__ C2<float> twr(C2<float> x) {
    constexpr int q = ((M % R) + R) % R;
    if constexpr (q == 0) return x;
    else if constexpr (4 * q == R) return {-x.y, x.x};
    else if constexpr (2 * q == R) return {-x.x, -x.y};
    else if constexpr (4 * q == 3 * R) return {x.y, -x.x};
    else {
        constexpr float c = (float)taylor_cos(turn_angle(q, R)), s = (float)taylor_sin(turn_angle(q, R));
        return {x.x * c - x.y * s, x.x * s + x.y * c};
    }
}

__host__ __device__ constexpr int smallest_factor(int R) {
    return R % 4 == 0 && R > 4 ? 4 : R % 2 == 0 ? 2 : R % 3 == 0 ? 3 : R % 5 == 0 ? 5 : R % 7 == 0 ? 7 : R;
}

// R-point DFT in registers (exp(+i), natural order in and out) for R built from the factors
// 2, 3, 4, 5, 7 (powers of two by reg_dft_c): R = P Q with P the first factor; Q-point DFTs over
// x[j1 + P j2], twiddles w_R^{j1 k2}, P-point DFTs into X[k2 + Q k1]; a prime R directly.
template <int R>
__device__ __forceinline__ void reg_dft_k(C2<float> (&v)[R]) {
    if constexpr (R == 1 || R == 2 || R == 4 || R == 8 || R == 16) {
        reg_dft_c<R>(v);
    } else if constexpr (smallest_factor(R) == R) {
        C2<float> out[R];
        static_for<0, R>([&](auto K) {
            constexpr int k = decltype(K)::value;
            C2<float> acc = v[0];
            static_for<1, R>([&](auto J) {
                constexpr int j = decltype(J)::value;
                acc = cadd(acc, twr<R, j * k>(v[j]));
            });
            out[k] = acc;
        });
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = out[k];
    } else {
        constexpr int P = smallest_factor(R), Q = R / P;
        C2<float> y[P][Q];
        static_for<0, P>([&](auto J1) {
            constexpr int j1 = decltype(J1)::value;
            C2<float> t[Q];
#pragma unroll
            for (int j2 = 0; j2 < Q; ++j2) t[j2] = v[j1 + P * j2];
            reg_dft_k<Q>(t);
            static_for<0, Q>([&](auto K2) {
                constexpr int k2 = decltype(K2)::value;
                y[j1][k2] = twr<R, j1 * k2>(t[k2]);
            });
        });
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
            C2<float> t[P];
#pragma unroll
            for (int j1 = 0; j1 < P; ++j1) t[j1] = y[j1][k2];
            reg_dft_k<P>(t);
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) v[k2 + Q * k1] = t[k1];
        }
    }
}

__device__ __forceinline__ int warp_fft_k2(int gl, int W) {
    const int lw = 31 - __clz(W);
    return lw ? (int)(__brev((unsigned)gl) >> (32 - lw)) : 0;
}

// Lanes per line (largest power of two <= 32 dividing N) and elements per lane.
inline void warp_fft_shape(int N, int* W, int* R) {
    int w = 32;
    while (N % w) w >>= 1;
    *W = w;
    *R = N / w;
}

}  // namespace wt
