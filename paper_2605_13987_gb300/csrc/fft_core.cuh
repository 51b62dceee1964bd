// Complex type and the mixed-radix Stockham FFT (shared-memory, inverse
// sign exp(+i), unnormalised) used by the spectral kernels.
#pragma once
#include "k_fft.cuh"

namespace wt {

template <class T>
struct C2 {
    T x, y;
};
template <class T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }

// One Stockham stage for element j of a line (N/R butterflies per line).
template <class T>
__device__ __forceinline__ void stage(const C2<T>* __restrict__ a, C2<T>* __restrict__ b, int N, int Ns, int R,
                                      int j, const C2<T>* __restrict__ tw) {
    const int stride = N / R;
    const int jm = j % Ns;
    const int idxD = (j / Ns) * Ns * R + jm;
    if (R == 4) {
        C2<T> v0 = a[j], v1 = a[j + stride], v2 = a[j + 2 * stride], v3 = a[j + 3 * stride];
        if (jm) {
            const int base = jm * (N / (Ns * 4));
            v1 = cmul(v1, tw[base]);
            v2 = cmul(v2, tw[2 * base]);
            v3 = cmul(v3, tw[3 * base]);
        }
        C2<T> s02 = cadd(v0, v2), d02 = csub(v0, v2), s13 = cadd(v1, v3), d13 = csub(v1, v3);
        C2<T> id13 = {-d13.y, d13.x};   // i * (v1 - v3)
        b[idxD] = cadd(s02, s13);
        b[idxD + Ns] = cadd(d02, id13);
        b[idxD + 2 * Ns] = csub(s02, s13);
        b[idxD + 3 * Ns] = csub(d02, id13);
    } else if (R == 2) {
        C2<T> v0 = a[j], v1 = a[j + stride];
        if (jm) v1 = cmul(v1, tw[jm * (N / (Ns * 2))]);
        b[idxD] = cadd(v0, v1);
        b[idxD + Ns] = csub(v0, v1);
    } else {
        C2<T> v[7];
        for (int r = 0; r < R; ++r) v[r] = a[j + r * stride];
        if (jm) {
            const int base = jm * (N / (Ns * R));
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r * base) % N]);
        }
        const int step = N / R;
        for (int k = 0; k < R; ++k) {
            C2<T> acc = v[0];
            for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], tw[((r * k) % R) * step]));
            b[idxD + k * Ns] = acc;
        }
    }
}

// Inverse (exp(+i)) unnormalised DFT of nl lines (line l at buf + l * ld) in
// shared memory.  Returns the buffer holding the result.
template <class T>
__device__ C2<T>* fft_lines(C2<T>* buf, C2<T>* scr, int ld, int nl, const FftPlan& pl,
                            const C2<T>* __restrict__ tw) {
    C2<T>* in = buf;
    C2<T>* out = scr;
    int Ns = 1;
    const int N = pl.N;
    for (int s = 0; s < pl.ns; ++s) {
        const int R = pl.r[s];
        const int nb = N / R;
        const int tot = nl * nb;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int l = e / nb, j = e - l * nb;
            stage<T>(in + l * ld, out + l * ld, N, Ns, R, j, tw);
        }
        __syncthreads();
        C2<T>* t = in;
        in = out;
        out = t;
        Ns *= R;
    }
    return in;
}


}  // namespace wt
