// Proper-image statistics on square tiles: ZOGY subtraction (below) and the
// proper coadd (after it) share one plan and the FFT kernels of fft.cuh.
//
// ZOGY proper image subtraction (paper Sec. 4.2: ZOGY at base cadence and in
// deep coadds; the statistic of Zackay, Ofek & Gal-Yam 2016).
//
// Per tile (T x T, periodic), with hats for DFTs:
//   1. pack:    z1 = N + i R (FP32), z2 = P_n + i P_r (FP64; the PSF stamps
//               placed with their centre at (0, 0), wrapping around);
//   2. forward: 2-D FFTs of z1 (FP32) and z2 (FP64) -- one complex transform
//               carries two real images, separated through the conjugate
//               symmetry X(k) = (Z(k) + conj Z(-k)) / 2, Y(k) = (Z(k) - conj Z(-k)) / 2i;
//   3. combine: per frequency pair (k, -k), one thread:
//                 den  = sqrt(sn^2 Fr^2 |Pr|^2 + sr^2 Fn^2 |Pn|^2)
//                 D    = (Fr Pr N - Fn Pn R) / den
//                 P_D  = Fr Fn Pr Pn / (F_D den),   F_D = Fr Fn / sqrt(sn^2 Fr^2 + sr^2 Fn^2)
//                 S    = F_D D conj(P_D)
//               all 0 where max(|Pn|, |Pr|) < eps (decided in FP64; below that
//               floor the PSF transforms are rounding); the result is written
//               as W = D + i S (both real images, so one inverse transform
//               returns D in the real part and S in the imaginary part), and
//               sum |P_D|^2 per tile (FP64) gives sigma_S = F_D ||P_D||_2;
//   4. inverse: 2-D FFT of W (and of P_D when asked for), divided by T^2.
// The PSF transforms are FP64 so that the floor decisions and the small
// transforms near it are those of an FP64 reference; the images and the
// combine are FP32.
#include "argus_internal.cuh"
#include "fft.cuh"

#include <cmath>
#include <cstdlib>

struct argus_proper_plan {
    int device;
    int tile;
    int max_tiles;
    int psf_tiles;    // ZOGY PSF transforms z2 holds: that many tiles', -1 one shared pair, 0 none
    float2* z1;       // [max_tiles][T][T]
    double2* z2;      // [max_tiles][T][T]
    float2* z3;       // [max_tiles][T][T] (ZOGY: P_D; coadd: the score accumulator, then P_R)
    double2* z4;      // [max_tiles][T][T] (coadd: sum F^2/s^2 |P|^2 and max |P|^2)
    double* psd;      // [max_tiles] sum |P_D(k)|^2
    float2* tw32;     // [T] e^{-2 pi i m / T}
    double2* tw64;
};

namespace {

struct ZArgs {
    const float* N;
    const float* R;
    long pitch;
    int w, h;
    const argus_zogy_tile* tiles;
    int n_tiles;
    const float* psf_n;
    const float* psf_r;
    int ps;
    int psf_tiles;            // tiles with their own PSF pair: n_tiles, or 1 when all share one
    double eps2;
    float2* z1;
    double2* z2;
    float2* z3;
    double* psd;
    float* D;
    float* S;
    float* PD;
    double* sigma_S;
};

template <int T>
__global__ void __launch_bounds__(256) zogy_pack_kernel(ZArgs a) {
    const long total = (long)a.n_tiles * T * T;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e / (T * T));
        const int q = (int)(e - (long)t * T * T);
        const int y = q / T, x = q - (q / T) * T;
        const int gx = a.tiles[t].x0 + x, gy = a.tiles[t].y0 + y;
        float n = 0.0f, r = 0.0f;
        if (gx >= 0 && gy >= 0 && gx < a.w && gy < a.h) {       // pixels off the frame are 0
            const long p = (long)gy * a.pitch + gx;
            n = a.N[p];
            r = a.R[p];
        }
        a.z1[e] = make_float2(n, r);
    }
}

template <int T>
__global__ void __launch_bounds__(256) zogy_psf_kernel(ZArgs a) {
    const int pp = a.ps * a.ps, hh = a.ps / 2;
    const long total = (long)a.psf_tiles * pp;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e / pp);
        const int i = (int)(e - (long)t * pp);
        const int v = i / a.ps, u = i - v * a.ps;
        const int yy = (v - hh + T) & (T - 1), xx = (u - hh + T) & (T - 1);
        a.z2[(long)t * T * T + yy * T + xx] = make_double2((double)a.psf_n[e], (double)a.psf_r[e]);
    }
}

__host__ __device__ __forceinline__ float2 f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// The pointwise step for one frequency pair: A = z1(k), B = z1(-k), C = z2(k),
// E = z2(-k).  Writes W(k) = D + i S and W(-k) = conj D + i conj S, P_D(k) and
// returns |P_D(k)|^2 (host-callable, so a CPU driver can run the same code).
__host__ __device__ __forceinline__ void zogy_pair(float2 A, float2 B, double2 C, double2 E, argus_zogy_tile tp,
                                                   double eps2, float2& Wq, float2& Wp, float2& PD, double& p2) {
    // N = (A + conj B) / 2, R = (A - conj B) / 2i
    const float2 Nh = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
    const float2 Rh = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
    const double2 Pn = make_double2(0.5 * (C.x + E.x), 0.5 * (C.y - E.y));
    const double2 Pr = make_double2(0.5 * (C.y + E.y), -0.5 * (C.x - E.x));
    const double mn = Pn.x * Pn.x + Pn.y * Pn.y, mr = Pr.x * Pr.x + Pr.y * Pr.y;
    const float Fn = tp.Fn, Fr = tp.Fr, sn = tp.sn, sr = tp.sr;
    const float FD = Fr * Fn / sqrtf(sn * sn * Fr * Fr + sr * sr * Fn * Fn);
    float2 Dh = make_float2(0.0f, 0.0f);
    PD = make_float2(0.0f, 0.0f);
    const float2 pn = f2(Pn), pr = f2(Pr);
    const float den = sqrtf(sn * sn * Fr * Fr * (pr.x * pr.x + pr.y * pr.y) +
                            sr * sr * Fn * Fn * (pn.x * pn.x + pn.y * pn.y));
    if ((mn >= eps2 || mr >= eps2) && den > 0.0f) {
        // Fr Pr N - Fn Pn R
        const float2 u = make_float2(Fr * (pr.x * Nh.x - pr.y * Nh.y) - Fn * (pn.x * Rh.x - pn.y * Rh.y),
                                     Fr * (pr.x * Nh.y + pr.y * Nh.x) - Fn * (pn.x * Rh.y + pn.y * Rh.x));
        Dh = make_float2(u.x / den, u.y / den);
        const float g = Fr * Fn / (FD * den);
        PD = make_float2(g * (pr.x * pn.x - pr.y * pn.y), g * (pr.x * pn.y + pr.y * pn.x));
    }
    // S = F_D D conj(P_D)
    const float2 Sh = make_float2(FD * (Dh.x * PD.x + Dh.y * PD.y), FD * (Dh.y * PD.x - Dh.x * PD.y));
    Wq = make_float2(Dh.x - Sh.y, Dh.y + Sh.x);
    Wp = make_float2(Dh.x + Sh.y, Sh.x - Dh.y);
    p2 = (double)PD.x * PD.x + (double)PD.y * PD.y;
}

template <int T>
__global__ void __launch_bounds__(256) zogy_combine_kernel(ZArgs a) {
    __shared__ double red[8];
    const long total = (long)a.n_tiles * T * T;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // one frequency per thread
    double psd = 0.0;
    int t = -1;
    if (e < total) {
        t = (int)(e / (T * T));
        const int q = (int)(e - (long)t * T * T);
        const int ky = q / T, kx = q - ky * T;
        const int pq = ((T - ky) & (T - 1)) * T + ((T - kx) & (T - 1));
        if (pq >= q) {                                   // the pair (q, pq) is this thread's
            const long base = (long)t * T * T;
            const long pbase = a.psf_tiles == 1 ? 0 : base;          // one shared PSF pair, or the tile's
            float2 Wq, Wp, PD;
            double p2;
            zogy_pair(a.z1[base + q], a.z1[base + pq], a.z2[pbase + q], a.z2[pbase + pq], a.tiles[t], a.eps2, Wq, Wp,
                      PD, p2);
            a.z1[base + q] = Wq;
            if (pq != q) a.z1[base + pq] = Wp;
            if (a.z3) {
                a.z3[base + q] = PD;
                if (pq != q) a.z3[base + pq] = make_float2(PD.x, -PD.y);
            }
            psd = p2 * (pq != q ? 2.0 : 1.0);
        }
    }
    // per-tile sum of |P_D|^2: a CTA of 256 frequencies lies in one tile (T^2 % 256 == 0)
    for (int o = 16; o > 0; o >>= 1) psd += __shfl_xor_sync(0xffffffffu, psd, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = psd;
    __syncthreads();
    if (threadIdx.x == 0 && t >= 0) {
        double s = 0.0;
        for (int i = 0; i < 8; i++) s += red[i];
        atomicAdd(a.psd + t, s);
    }
}

template <int T>
__global__ void __launch_bounds__(256) zogy_unpack_kernel(ZArgs a) {
    const long total = (long)a.n_tiles * T * T;
    const float inv = 1.0f / ((float)T * (float)T);                  // a power of two: exact
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const float2 w = a.z1[e];
        a.D[e] = w.x * inv;
        a.S[e] = w.y * inv;
        if (a.PD) a.PD[e] = a.z3[e].x * inv;
    }
}

template <int T>
__global__ void zogy_sigma_kernel(ZArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tiles) return;
    const argus_zogy_tile tp = a.tiles[t];
    const double Fn = tp.Fn, Fr = tp.Fr, sn = tp.sn, sr = tp.sr;
    const double FD = Fr * Fn / sqrt(sn * sn * Fr * Fr + sr * sr * Fn * Fn);
    a.sigma_S[t] = FD * sqrt(a.psd[t] / ((double)T * T));
}

template <int T, int S, typename R>
void fft2d(typename fft::Cx<R>::T* d, int n, const typename fft::Cx<R>::T* tw, cudaStream_t s) {
    using Sh = fft::Shape<T, R>;
    const unsigned blocks = (unsigned)n * (T / Sh::SEQ);
    fft::fft_pass_kernel<T, S, false, R><<<blocks, Sh::THREADS, Sh::SMEM, s>>>(d, n, tw);
    fft::fft_pass_kernel<T, S, true, R><<<blocks, Sh::THREADS, Sh::SMEM, s>>>(d, n, tw);
    argus_count_launch(2);
}

template <int T>
bool set_smem() {
    bool ok = true;
    ok &= cudaFuncSetAttribute(fft::fft_pass_kernel<T, -1, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fft::Shape<T, float>::SMEM) == cudaSuccess;
    ok &= cudaFuncSetAttribute(fft::fft_pass_kernel<T, -1, true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fft::Shape<T, float>::SMEM) == cudaSuccess;
    ok &= cudaFuncSetAttribute(fft::fft_pass_kernel<T, 1, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fft::Shape<T, float>::SMEM) == cudaSuccess;
    ok &= cudaFuncSetAttribute(fft::fft_pass_kernel<T, 1, true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fft::Shape<T, float>::SMEM) == cudaSuccess;
    ok &= cudaFuncSetAttribute(fft::fft_pass_kernel<T, -1, false, double>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft::Shape<T, double>::SMEM) == cudaSuccess;
    ok &= cudaFuncSetAttribute(fft::fft_pass_kernel<T, -1, true, double>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft::Shape<T, double>::SMEM) == cudaSuccess;
    return ok;
}

template <int T>
int run(argus_proper_plan* p, ZArgs& a, cudaStream_t s) {
    const long total = (long)a.n_tiles * T * T;
    const unsigned grid = (unsigned)((total + 255) / 256);
    unsigned g2 = grid > 152u * 16u ? 152u * 16u : grid;
    if (cudaMemsetAsync(p->psd, 0, (size_t)a.n_tiles * sizeof(double), s) != cudaSuccess) return ARGUS_ERR_CUDA;
    zogy_pack_kernel<T><<<g2, 256, 0, s>>>(a);
    argus_count_launch(1);
    fft2d<T, -1, float>(p->z1, a.n_tiles, p->tw32, s);
    if (a.psf_n) {                 // new PSFs: place and transform them (else z2 holds the last ones)
        const long ptotal = (long)a.psf_tiles * T * T;
        if (cudaMemsetAsync(p->z2, 0, (size_t)ptotal * sizeof(double2), s) != cudaSuccess) return ARGUS_ERR_CUDA;
        const long pp = (long)a.psf_tiles * a.ps * a.ps;
        zogy_psf_kernel<T><<<(unsigned)((pp + 255) / 256), 256, 0, s>>>(a);
        argus_count_launch(1);
        fft2d<T, -1, double>(p->z2, a.psf_tiles, p->tw64, s);
    }
    zogy_combine_kernel<T><<<grid, 256, 0, s>>>(a);
    argus_count_launch(1);
    fft2d<T, 1, float>(p->z1, a.n_tiles, p->tw32, s);
    if (a.PD) fft2d<T, 1, float>(p->z3, a.n_tiles, p->tw32, s);
    zogy_unpack_kernel<T><<<g2, 256, 0, s>>>(a);
    argus_count_launch(1);
    if (a.sigma_S) {
        zogy_sigma_kernel<T><<<(a.n_tiles + 127) / 128, 128, 0, s>>>(a);
        argus_count_launch(1);
    }
    return argus_launch_status();
}

// ---------------------------------------------------------------------------
// Proper coaddition (paper Sec. 4.1.3: a per-image matched filter; the
// statistic of Zackay & Ofek 2017).  Frames go through the transforms in
// pairs (M_j + i M_{j+1}, P_j + i P_{j+1}); per frequency the accumulators
// hold the score S = sum_j (F_j / s_j^2) conj(P_j) M_j (FP32) and, in FP64,
// den^2 = sum_j F_j^2 / s_j^2 |P_j|^2 and max_j |P_j|^2.  Then
//   R = S / den (0 below the frequency floor), W = S + i R -> one inverse
//   transform gives the score coadd (real part) and the proper coadd
//   (imaginary part);  P_R = IDFT[den / F_R],  F_R = sqrt(sum_j F_j^2 / s_j^2).

struct CArgs {
    const float* stack;     // [n_frames][h][pitch]
    long frame_stride;
    long pitch;
    int w, h;
    const int* origins;     // [n_tiles][2]
    int n_tiles;
    const float* F;         // [n_frames]
    const float* sig;       // [n_frames]
    int n_frames;
    const float* psfs;      // [psf_tiles][n_frames][ps][ps]
    int ps;
    int psf_tiles;          // n_tiles, or 1 when every tile shares a frame's PSF
    int j0;                 // first frame of the pair in flight
    double eps2;
    float2* z1;
    double2* z2;
    float2* acc;            // score accumulator, then the P_R spectrum
    double2* acc2;          // (den^2, max |P|^2)
    float* S;
    float* R;
    float* PR;
    double* F_R;
    double* sigma_S;
};

// Frame j's matched-filter weights: F / s^2 for the score, F^2 / s^2 for den^2
// (a frame with s <= 0, or past the last frame, has none).
__host__ __device__ __forceinline__ void frame_weights(const float* F, const float* sig, int n, int j, float& w,
                                                       double& a) {
    w = 0.0f;
    a = 0.0;
    if (j < n && sig[j] > 0.0f) {
        w = F[j] / (sig[j] * sig[j]);
        a = (double)F[j] * F[j] / ((double)sig[j] * sig[j]);
    }
}

// Accumulate one frame pair at frequency k: A = z1(k), B = z1(-k), C = z2(k),
// E = z2(-k) (host-callable, so a CPU driver can run the same code).
__host__ __device__ __forceinline__ void coadd_accum_point(float2 A, float2 B, double2 C, double2 E, float w0,
                                                           float w1, double a0, double a1, float2& acc,
                                                           double2& acc2) {
    const float2 M0 = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
    const float2 M1 = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
    const double2 P0 = make_double2(0.5 * (C.x + E.x), 0.5 * (C.y - E.y));
    const double2 P1 = make_double2(0.5 * (C.y + E.y), -0.5 * (C.x - E.x));
    const float2 p0 = f2(P0), p1 = f2(P1);
    // conj(P) M
    acc.x += w0 * (p0.x * M0.x + p0.y * M0.y) + w1 * (p1.x * M1.x + p1.y * M1.y);
    acc.y += w0 * (p0.x * M0.y - p0.y * M0.x) + w1 * (p1.x * M1.y - p1.y * M1.x);
    const double q0 = P0.x * P0.x + P0.y * P0.y, q1 = P1.x * P1.x + P1.y * P1.y;
    acc2.x += a0 * q0 + a1 * q1;
    double m = acc2.y;
    if (a0 > 0.0 && q0 > m) m = q0;
    if (a1 > 0.0 && q1 > m) m = q1;
    acc2.y = m;
}

// The last step at frequency k: W = S + i R and the P_R spectrum.
__host__ __device__ __forceinline__ void coadd_final_point(float2 Sh, double2 acc2, double FR, double eps2, float2& W,
                                                           float2& PRh) {
    const double den = sqrt(acc2.x);
    float2 Rh = make_float2(0.0f, 0.0f);
    PRh = make_float2(0.0f, 0.0f);
    if (acc2.y >= eps2 && den > 0.0) {
        const float d = (float)den;
        Rh = make_float2(Sh.x / d, Sh.y / d);
        PRh = make_float2((float)(den / FR), 0.0f);
    }
    W = make_float2(Sh.x - Rh.y, Sh.y + Rh.x);
}

template <int T>
__global__ void __launch_bounds__(256) coadd_pack_kernel(CArgs a) {
    const long total = (long)a.n_tiles * T * T;
    const bool two = a.j0 + 1 < a.n_frames;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e / (T * T));
        const int q = (int)(e - (long)t * T * T);
        const int gx = a.origins[2 * t] + (q % T), gy = a.origins[2 * t + 1] + q / T;
        float m0 = 0.0f, m1 = 0.0f;
        if (gx >= 0 && gy >= 0 && gx < a.w && gy < a.h) {       // pixels off the frame are 0
            const long p = (long)gy * a.pitch + gx;
            m0 = a.stack[a.j0 * a.frame_stride + p];
            if (two) m1 = a.stack[(a.j0 + 1) * a.frame_stride + p];
        }
        a.z1[e] = make_float2(m0, m1);
    }
}

template <int T>
__global__ void __launch_bounds__(256) coadd_psf_kernel(CArgs a) {
    const int pp = a.ps * a.ps, hh = a.ps / 2;
    const long total = (long)a.psf_tiles * pp;
    const bool two = a.j0 + 1 < a.n_frames;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e / pp);
        const int i = (int)(e - (long)t * pp);
        const int v = i / a.ps, u = i - v * a.ps;
        const int yy = (v - hh + T) & (T - 1), xx = (u - hh + T) & (T - 1);
        const float* pt = a.psfs + ((long)t * a.n_frames + a.j0) * pp;
        a.z2[(long)t * T * T + yy * T + xx] = make_double2((double)pt[i], two ? (double)pt[pp + i] : 0.0);
    }
}

template <int T>
__global__ void __launch_bounds__(256) coadd_accum_kernel(CArgs a) {
    const long total = (long)a.n_tiles * T * T;
    float w0, w1;
    double a0, a1;
    frame_weights(a.F, a.sig, a.n_frames, a.j0, w0, a0);
    frame_weights(a.F, a.sig, a.n_frames, a.j0 + 1, w1, a1);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e / (T * T));
        const int q = (int)(e - (long)t * T * T);
        const int ky = q / T, kx = q - ky * T;
        const long base = (long)t * T * T;
        const long pe = base + ((T - ky) & (T - 1)) * T + ((T - kx) & (T - 1));
        const long pb = a.psf_tiles == 1 ? base : 0;                 // shared PSFs live in tile 0
        float2 acc = a.acc[e];
        double2 acc2 = a.acc2[e];
        coadd_accum_point(a.z1[e], a.z1[pe], a.z2[e - pb], a.z2[pe - pb], w0, w1, a0, a1, acc, acc2);
        a.acc[e] = acc;
        a.acc2[e] = acc2;
    }
}

template <int T>
__global__ void __launch_bounds__(256) coadd_final_kernel(CArgs a) {
    const long total = (long)a.n_tiles * T * T;
    double fr2 = 0.0;
    for (int j = 0; j < a.n_frames; j++) {
        float w;
        double aj;
        frame_weights(a.F, a.sig, a.n_frames, j, w, aj);
        fr2 += aj;
    }
    const double FR = sqrt(fr2);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        float2 W, PRh;
        coadd_final_point(a.acc[e], a.acc2[e], FR, a.eps2, W, PRh);
        a.z1[e] = W;
        a.acc[e] = PRh;
    }
}

template <int T>
__global__ void __launch_bounds__(256) coadd_unpack_kernel(CArgs a) {
    const long total = (long)a.n_tiles * T * T;
    const float inv = 1.0f / ((float)T * (float)T);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const float2 w = a.z1[e];
        a.S[e] = w.x * inv;
        a.R[e] = w.y * inv;
        if (a.PR) a.PR[e] = a.acc[e].x * inv;
    }
}

// sigma_S per tile (sqrt(sum_j F_j^2 / s_j^2 sum P_tj^2)) and F_R, one thread per tile.
__global__ void coadd_norm_kernel(CArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tiles) return;
    const int pp = a.ps * a.ps;
    double v = 0.0, fr2 = 0.0;
    for (int j = 0; j < a.n_frames; j++) {
        float w;
        double aj;
        frame_weights(a.F, a.sig, a.n_frames, j, w, aj);
        const float* pt = a.psfs + ((long)(a.psf_tiles == 1 ? 0 : t) * a.n_frames + j) * pp;
        double s2 = 0.0;
        for (int i = 0; i < pp; i++) s2 += (double)pt[i] * pt[i];
        v += aj * s2;
        fr2 += aj;
    }
    if (a.sigma_S) a.sigma_S[t] = sqrt(v);
    if (a.F_R && t == 0) *a.F_R = sqrt(fr2);
}

template <int T>
int run_coadd(argus_proper_plan* p, CArgs& a, cudaStream_t s) {
    const long total = (long)a.n_tiles * T * T;
    long g = (total + 255) / 256;
    const unsigned grid = (unsigned)(g > 152L * 16 ? 152L * 16 : g);
    if (cudaMemsetAsync(a.acc, 0, (size_t)total * sizeof(float2), s) != cudaSuccess) return ARGUS_ERR_CUDA;
    if (cudaMemsetAsync(a.acc2, 0, (size_t)total * sizeof(double2), s) != cudaSuccess) return ARGUS_ERR_CUDA;
    const long pp = (long)a.psf_tiles * a.ps * a.ps;
    const long ptotal = (long)a.psf_tiles * T * T;
    for (int j0 = 0; j0 < a.n_frames; j0 += 2) {
        a.j0 = j0;
        if (cudaMemsetAsync(a.z2, 0, (size_t)ptotal * sizeof(double2), s) != cudaSuccess) return ARGUS_ERR_CUDA;
        coadd_pack_kernel<T><<<grid, 256, 0, s>>>(a);
        coadd_psf_kernel<T><<<(unsigned)((pp + 255) / 256), 256, 0, s>>>(a);
        argus_count_launch(2);
        fft2d<T, -1, float>(a.z1, a.n_tiles, p->tw32, s);
        fft2d<T, -1, double>(a.z2, a.psf_tiles, p->tw64, s);
        coadd_accum_kernel<T><<<grid, 256, 0, s>>>(a);
        argus_count_launch(1);
    }
    coadd_final_kernel<T><<<grid, 256, 0, s>>>(a);
    argus_count_launch(1);
    fft2d<T, 1, float>(a.z1, a.n_tiles, p->tw32, s);
    if (a.PR) fft2d<T, 1, float>(a.acc, a.n_tiles, p->tw32, s);
    coadd_unpack_kernel<T><<<grid, 256, 0, s>>>(a);
    coadd_norm_kernel<<<(a.n_tiles + 127) / 128, 128, 0, s>>>(a);
    argus_count_launch(2);
    return argus_launch_status();
}

}  // namespace

extern "C" int argus_proper_plan_create(int device, int tile, int max_tiles, argus_proper_plan** out) {
    if (!out || (tile != 256 && tile != 512 && tile != 1024) || max_tiles < 1 || max_tiles > 65536)
        return ARGUS_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return ARGUS_ERR_CUDA;
    const bool smem_ok = tile == 256 ? set_smem<256>() : tile == 512 ? set_smem<512>() : set_smem<1024>();
    if (!smem_ok) return ARGUS_ERR_CUDA;
    argus_proper_plan* p = (argus_proper_plan*)calloc(1, sizeof(argus_proper_plan));
    if (!p) return ARGUS_ERR_NOMEM;
    p->device = device;
    p->tile = tile;
    p->max_tiles = max_tiles;
    const size_t n = (size_t)max_tiles * tile * tile;
    bool ok = cudaMalloc((void**)&p->z1, n * sizeof(float2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&p->z2, n * sizeof(double2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&p->z3, n * sizeof(float2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&p->z4, n * sizeof(double2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&p->psd, (size_t)max_tiles * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&p->tw32, (size_t)tile * sizeof(float2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&p->tw64, (size_t)tile * sizeof(double2)) == cudaSuccess;
    if (ok) {
        // twiddles e^{-2 pi i m / T} in double on the host, rounded once to float
        double2* h64 = (double2*)malloc((size_t)tile * sizeof(double2));
        float2* h32 = (float2*)malloc((size_t)tile * sizeof(float2));
        ok = h64 && h32;
        if (ok) {
            const double two_pi = 6.283185307179586476925286766559;
            for (int m = 0; m < tile; m++) {
                const double ang = two_pi * (double)m / (double)tile;
                h64[m] = make_double2(std::cos(ang), -std::sin(ang));
                h32[m] = make_float2((float)h64[m].x, (float)h64[m].y);
            }
            ok = cudaMemcpy(p->tw64, h64, (size_t)tile * sizeof(double2), cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemcpy(p->tw32, h32, (size_t)tile * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
        }
        free(h64);
        free(h32);
    }
    if (!ok) {
        cudaFree(p->z1); cudaFree(p->z2); cudaFree(p->z3); cudaFree(p->z4); cudaFree(p->psd); cudaFree(p->tw32); cudaFree(p->tw64);
        free(p);
        return ARGUS_ERR_NOMEM;
    }
    *out = p;
    return ARGUS_OK;
}

extern "C" int argus_proper_plan_destroy(argus_proper_plan* p) {
    if (!p) return ARGUS_ERR_ARG;
    cudaSetDevice(p->device);
    cudaFree(p->z1); cudaFree(p->z2); cudaFree(p->z3); cudaFree(p->z4); cudaFree(p->psd); cudaFree(p->tw32); cudaFree(p->tw64);
    free(p);
    return ARGUS_OK;
}

// May a call without PSFs reuse the transforms a plan holds?  held: the plan's psf_tiles
// (> 0 that many tiles' own pairs, -1 one shared pair, 0 none).  A per-tile call needs at
// least n_tiles per-tile pairs; a shared call needs the shared pair.
__host__ __device__ inline bool zogy_psf_reuse_ok(int held, int psf_per_tile, int n_tiles) {
    return psf_per_tile ? (held >= 1 && n_tiles <= held) : held == -1;
}

extern "C" int argus_zogy(argus_proper_plan* plan, const float* N, const float* R, argus_shape shape,
                          const argus_zogy_tile* tiles, int n_tiles, const float* psf_n, const float* psf_r,
                          int psf_size, int psf_per_tile, float eps, float* D, float* S, float* P_D,
                          double* sigma_S, argus_stream stream) {
    if (!plan || !N || !R || !tiles || !D || !S || n_tiles < 1 || n_tiles > plan->max_tiles) return ARGUS_ERR_ARG;
    if (!psf_n != !psf_r || (psf_per_tile != 0 && psf_per_tile != 1)) return ARGUS_ERR_ARG;
    // what the plan holds: psf_tiles > 0 tiles of their own, -1 one shared pair, 0 nothing
    if (!psf_n && !zogy_psf_reuse_ok(plan->psf_tiles, psf_per_tile, n_tiles)) return ARGUS_ERR_ARG;
    if (psf_size < 1 || (psf_size & 1) == 0 || psf_size > 63 || !(eps >= 0.0f)) return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, (size_t)-1);
    if (st) return st;
    if (cudaSetDevice(plan->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    ZArgs a;
    a.N = N; a.R = R; a.pitch = shape.pitch; a.w = shape.w; a.h = shape.h;
    a.tiles = tiles; a.n_tiles = n_tiles; a.psf_n = psf_n; a.psf_r = psf_r; a.ps = psf_size;
    a.psf_tiles = psf_per_tile ? n_tiles : 1;
    a.eps2 = (double)eps * (double)eps;
    a.z1 = plan->z1; a.z2 = plan->z2; a.z3 = P_D ? plan->z3 : nullptr; a.psd = plan->psd;
    a.D = D; a.S = S; a.PD = P_D; a.sigma_S = sigma_S;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    switch (plan->tile) {
        case 256: rc = run<256>(plan, a, s); break;
        case 512: rc = run<512>(plan, a, s); break;
        default: rc = run<1024>(plan, a, s); break;
    }
    if (psf_n) plan->psf_tiles = rc != ARGUS_OK ? 0 : (psf_per_tile ? n_tiles : -1);
    return rc;
}

extern "C" int argus_proper_coadd(argus_proper_plan* plan, const float* stack, int n_frames, argus_shape shape,
                                  const int* origins, int n_tiles, const float* F, const float* sigma,
                                  const float* psfs, int psf_size, int psf_per_tile, float eps, float* S,
                                  float* R, float* P_R,
                                  double* F_R, double* sigma_S, argus_stream stream) {
    if (!plan || !stack || !origins || !F || !sigma || !psfs || !S || !R || n_tiles < 1 ||
        n_tiles > plan->max_tiles || n_frames < 1 || n_frames > ARGUS_MAX_FRAMES)
        return ARGUS_ERR_ARG;
    if (psf_size < 1 || (psf_size & 1) == 0 || psf_size > 63 || !(eps >= 0.0f)) return ARGUS_ERR_ARG;
    if (psf_per_tile != 0 && psf_per_tile != 1) return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, (size_t)-1);
    if (st) return st;
    if (cudaSetDevice(plan->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    CArgs a;
    a.psf_tiles = psf_per_tile ? n_tiles : 1;
    a.stack = stack; a.frame_stride = (long)shape.h * shape.pitch; a.pitch = shape.pitch;
    a.w = shape.w; a.h = shape.h; a.origins = origins; a.n_tiles = n_tiles; a.F = F; a.sig = sigma;
    a.n_frames = n_frames; a.psfs = psfs; a.ps = psf_size; a.j0 = 0; a.eps2 = (double)eps * (double)eps;
    a.z1 = plan->z1; a.z2 = plan->z2; a.acc = plan->z3; a.acc2 = plan->z4;
    plan->psf_tiles = 0;                                   // z2 is about to hold frame PSFs
    a.S = S; a.R = R; a.PR = P_R; a.F_R = F_R; a.sigma_S = sigma_S;
    cudaStream_t s = (cudaStream_t)stream;
    switch (plan->tile) {
        case 256: return run_coadd<256>(plan, a, s);
        case 512: return run_coadd<512>(plan, a, s);
        default: return run_coadd<1024>(plan, a, s);
    }
}
