// Batched 2-D FFTs of square power-of-two tiles (T = 256, 512, 1024) in shared
// memory: Stockham auto-sort passes of radix 8 (then 4 or 2 to finish), a
// twiddle table of e^{-2 pi i m / T} built in double precision on the host,
// one kernel for the rows and one for the columns (the columns are loaded
// transposed into padded shared rows).  Forward transforms are unnormalised,
// inverse transforms are unscaled (the caller divides by T^2), as in numpy.
// The real type is float (image data) or double (PSF transforms).
#pragma once

#include <cuda_runtime.h>

// the butterflies and the pass are host-callable too, so that a CPU driver can
// run the same code thread by thread
#define FFT_HD __host__ __device__ __forceinline__

namespace fft {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename C> FFT_HD C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> FFT_HD C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> FFT_HD C cmul(C a, C b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> FFT_HD C cconj(C a) { return {a.x, -a.y}; }
// a * (s i), s = -1 (forward) or +1 (inverse)
template <int S, typename C> FFT_HD C cmul_i(C a) {
    return S < 0 ? C{a.y, -a.x} : C{-a.y, a.x};
}

template <int S, typename C> FFT_HD void dft2(C* v) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int S, typename C> FFT_HD void dft4(C& a0, C& a1, C& a2, C& a3) {
    const C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmul_i<S>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a1 = cadd(t1, t3);
    a2 = csub(t0, t2);
    a3 = csub(t1, t3);
}

template <int S, typename C> FFT_HD void dft8(C* v) {
    using R = decltype(v[0].x);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    const R r = (R)0.70710678118654752440;
    o1 = cmul(o1, C{r, (R)S * r});           // e^{S i pi / 4}
    o2 = cmul_i<S>(o2);                       // e^{S i pi / 2}
    o3 = cmul(o3, C{-r, (R)S * r});          // e^{S 3 i pi / 4}
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// One Stockham pass of radix RAD over a sequence of length T held in a
// (stride 1), writing b: butterfly j (0 <= j < T / RAD) reads a[j + r T/RAD],
// multiplies by e^{S 2 pi i r k / (Ns RAD)} (k = j mod Ns) and writes the
// RAD-point DFT to b[(j / Ns) Ns RAD + k + r Ns].  tw[m] = e^{-2 pi i m / T}.
template <int T, int RAD, int S, typename C>
FFT_HD void stockham_pass(const C* a, C* b, const C* tw, int Ns, int lane, int nlanes) {
    for (int j = lane; j < T / RAD; j += nlanes) {
        C v[RAD];
        const int k = j & (Ns - 1);
        const int step = T / (Ns * RAD);
#pragma unroll
        for (int r = 0; r < RAD; r++) {
            v[r] = a[j + r * (T / RAD)];
            if (r) {
                const C w = tw[(r * k * step) & (T - 1)];
                v[r] = cmul(v[r], S < 0 ? w : cconj(w));
            }
        }
        if (RAD == 8) dft8<S>(v);
        else if (RAD == 4) dft4<S>(v[0], v[1], v[2], v[3]);
        else dft2<S>(v);
        const int d = (j / Ns) * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; r++) b[d + r * Ns] = v[r];
    }
}

// All passes over one sequence: radix 8 while 8 Ns <= T, then 4 or 2.
// a and b are this sequence's two shared buffers; returns the one holding the
// result.  Every thread of the CTA calls it (barriers inside).
template <int T, int S, typename C>
__device__ __forceinline__ C* stockham(C* a, C* b, const C* tw, int lane, int nlanes) {
    int Ns = 1;
    while (Ns < T) {
        if (Ns * 8 <= T) {
            stockham_pass<T, 8, S>(a, b, tw, Ns, lane, nlanes);
            Ns *= 8;
        } else if (Ns * 4 <= T) {
            stockham_pass<T, 4, S>(a, b, tw, Ns, lane, nlanes);
            Ns *= 4;
        } else {
            stockham_pass<T, 2, S>(a, b, tw, Ns, lane, nlanes);
            Ns *= 2;
        }
        __syncthreads();
        C* t = a;
        a = b;
        b = t;
    }
    return a;
}

// Sequences per CTA and threads per sequence for a T-point transform.
template <int T, typename R> struct Shape {
    static constexpr int SEQ = (sizeof(R) == 4 ? 16 : 8) / (T > 512 ? 2 : 1);
    static constexpr int LANES = T / 8;                  // one radix-8 butterfly per thread
    static constexpr int THREADS = SEQ * LANES;
    static constexpr int PAD = T + 1;                    // padded shared row (transposed loads)
    static constexpr size_t SMEM = (2 * (size_t)SEQ * PAD + T) * sizeof(typename Cx<R>::T);
};

// FFT along the rows (COLS = false) or the columns (COLS = true) of n_tiles
// tiles [n][T][T] of complex values, in place.  S = -1 forward, +1 inverse.
template <int T, int S, bool COLS, typename R>
__global__ void __launch_bounds__(Shape<T, R>::THREADS) fft_pass_kernel(typename Cx<R>::T* data, int n_tiles,
                                                                      const typename Cx<R>::T* tw_global) {
    using C = typename Cx<R>::T;
    using Sh = Shape<T, R>;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    C* buf = reinterpret_cast<C*>(fft_smem);
    C* tw = buf + 2 * Sh::SEQ * Sh::PAD;
    for (int i = threadIdx.x; i < T; i += Sh::THREADS) tw[i] = tw_global[i];
    const long blocks_per_tile = T / Sh::SEQ;
    const long tile = blockIdx.x / blocks_per_tile;
    const int s0 = (int)(blockIdx.x % blocks_per_tile) * Sh::SEQ;   // first row or column
    if (tile >= n_tiles) return;                                    // uniform per CTA
    C* base = data + tile * (long)T * T;
    // load: sequence s of this CTA into buf[s * PAD ...]
    for (int e = threadIdx.x; e < Sh::SEQ * T; e += Sh::THREADS) {
        if (COLS) {
            const int y = e / Sh::SEQ, c = e - y * Sh::SEQ;           // SEQ consecutive columns per row
            buf[c * Sh::PAD + y] = base[(long)y * T + s0 + c];
        } else {
            const int s = e / T, x = e - s * T;
            buf[s * Sh::PAD + x] = base[(long)(s0 + s) * T + x];
        }
    }
    __syncthreads();
    const int seq = threadIdx.x / Sh::LANES, lane = threadIdx.x - seq * Sh::LANES;
    // the second buffer of sequence seq is SEQ rows further on
    C* res = stockham<T, S>(buf + seq * Sh::PAD, buf + (Sh::SEQ + seq) * Sh::PAD, tw, lane, Sh::LANES);
    const bool in_first = res == buf + seq * Sh::PAD;                // the same for every sequence
    C* out = in_first ? buf : buf + Sh::SEQ * Sh::PAD;
    for (int e = threadIdx.x; e < Sh::SEQ * T; e += Sh::THREADS) {
        if (COLS) {
            const int y = e / Sh::SEQ, c = e - y * Sh::SEQ;
            base[(long)y * T + s0 + c] = out[c * Sh::PAD + y];
        } else {
            const int s = e / T, x = e - s * T;
            base[(long)(s0 + s) * T + x] = out[s * Sh::PAD + x];
        }
    }
}

}  // namespace fft
