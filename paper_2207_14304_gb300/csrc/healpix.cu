// Frame to HEALPix segment resampling (paper Sec. 3.3 "Image Segmentation";
// Table 2, GPU stage "Image segmentation and resampling to HEALPix grid").
//
// The segment's nested index gives its base face and face coordinates (X, Y);
// image pixel (column c, row r) is the HEALPix pixel (X 2^k + c, Y 2^k + r) at
// NSIDE_seg 2^k, whose centre (the ring / longitude formulas of the nested
// layout) is projected into the frame by the gnomonic WCS and the frame is
// interpolated there (bilinear, nested lerps, coverage as in the coadd).  The
// geometry is FP64 (a 9576-pixel frame needs positions to 1e-9 of the field);
// the output is FP32.  Exact path: one thread per pixel.  Row path (k >= 6):
// one warp per row, exact positions at four nodes per 64-pixel piece and a
// cubic between them in the equatorial belt (see healpix_rows_kernel).
#include "argus_internal.cuh"

#include <cmath>

namespace {

struct HpArgs {
    const float* frame;
    const uint8_t* flags;
    long pitch;
    int w, h;
    const long long* segs;
    int n_seg;
    long long nside_seg;
    int k;
    double n[3], e[3], u[3];   // tangent-plane basis at the WCS centre
    double cr, sr, inv_scale, cx, cy;
    float* out;
    uint8_t* cov;
};

__host__ __device__ __forceinline__ void hp_sincospi(double t, double* s, double* c) {
#ifdef __CUDA_ARCH__
    sincospi(t, s, c);
#else
    *s = std::sin(M_PI * t);
    *c = std::cos(M_PI * t);
#endif
}

// Frame position of the centre of segment-image pixel (c, r).  false when the
// direction is behind the tangent plane.
__host__ __device__ __forceinline__ bool hp_pixel_xy(const HpArgs& a, long long seg, int c, int r, double& x,
                                                     double& y) {
    const long long N = a.nside_seg;
    const long long face = seg / (N * N);
    if (seg < 0 || face >= 12) return false;            // not a pixel of this NSIDE
    const long long ipf = seg - face * N * N;
    long long X = 0, Y = 0;
    for (int b = 0; (1LL << b) < N; b++) {
        X |= ((ipf >> (2 * b)) & 1LL) << b;
        Y |= ((ipf >> (2 * b + 1)) & 1LL) << b;
    }
    const long long nside = N << a.k;
    const long long ix = (X << a.k) + c, iy = (Y << a.k) + r;
    const int jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
    const int jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};
    const long long jr = jrll[face] * nside - ix - iy - 1;
    long long nr, kshift = 0;
    double z, sin_t;
    if (jr < nside) {                                    // north polar cap
        nr = jr;
        const double cap = (double)nr * (double)nr / (3.0 * (double)nside * (double)nside);
        z = 1.0 - cap;
        sin_t = sqrt(cap * (2.0 - cap));
    } else if (jr > 3 * nside) {                         // south polar cap
        nr = 4 * nside - jr;
        const double cap = (double)nr * (double)nr / (3.0 * (double)nside * (double)nside);
        z = -1.0 + cap;
        sin_t = sqrt(cap * (2.0 - cap));
    } else {                                             // equatorial belt
        nr = nside;
        z = (double)(2 * nside - jr) * 2.0 / (3.0 * (double)nside);
        sin_t = sqrt((1.0 - z) * (1.0 + z));
        kshift = (jr - nside) & 1;
    }
    long long jp = (jpll[face] * nr + ix - iy + 1 + kshift) / 2;
    if (jp > 4 * nr) jp -= 4 * nr;
    if (jp < 1) jp += 4 * nr;
    // phi = (jp - (kshift + 1) / 2) (pi / 2) / nr
    double sp, cp;
    hp_sincospi(((double)jp - 0.5 * (double)(kshift + 1)) / (2.0 * (double)nr), &sp, &cp);
    const double v0 = sin_t * cp, v1 = sin_t * sp, v2 = z;
    const double d = v0 * a.n[0] + v1 * a.n[1] + v2 * a.n[2];
    if (!(d > 0.0)) return false;
    const double xi = (v0 * a.e[0] + v1 * a.e[1] + v2 * a.e[2]) / d;
    const double eta = (v0 * a.u[0] + v1 * a.u[1] + v2 * a.u[2]) / d;
    x = a.cx + (a.cr * xi + a.sr * eta) * a.inv_scale;
    y = a.cy + (-a.sr * xi + a.cr * eta) * a.inv_scale;
    return true;
}

// Nested-lerp bilinear value of the frame at (x, y); false when not covered
// (outside [0, w-1] x [0, h-1], or a neighbour with a nonzero weight flagged
// or not finite).
__host__ __device__ __forceinline__ bool hp_bilinear(const HpArgs& a, double x, double y, float& v) {
    if (!(x >= 0.0 && y >= 0.0 && x <= (double)(a.w - 1) && y <= (double)(a.h - 1))) return false;
    const int x0 = (int)floor(x), y0 = (int)floor(y);
    const double tx = x - x0, ty = y - y0;
    const bool ux = tx > 0.0, uy = ty > 0.0;
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    const bool used[4] = {true, ux, uy, ux && uy};
    for (int i = 0; i < 4; i++) {
        if (!used[i]) continue;
        const long p = (long)(y0 + (i >> 1)) * a.pitch + x0 + (i & 1);
        const float f = a.frame[p];
        if (!isfinite(f) || (a.flags && a.flags[p])) return false;
        q[i] = f;
    }
    const double top = q[0] + tx * (q[1] - q[0]);
    const double bot = q[2] + tx * (q[3] - q[2]);
    v = (float)(top + ty * (bot - top));
    return true;
}

// Row interpolation (the fast path).  Along a segment-image row in the
// equatorial belt the frame position is a smooth function of the column: on
// pieces of 64 pixels a cubic through the exact FP64 positions at columns
// 0, 21, 42, 63 of the piece reproduces it to a few 1e-8 pixel.  Newton form:
// d[0] = f0, d[1] = f[t0,t1], d[2] = f[t0,t1,t2], d[3] = f[t0..t3].
constexpr int HP_PIECE = 64;
__host__ __device__ __forceinline__ int hp_node(int j) { return j == 0 ? 0 : (j == 1 ? 21 : (j == 2 ? 42 : 63)); }

__host__ __device__ __forceinline__ void hp_cubic_coeffs(const double* f, double* d) {
    const double f01 = (f[1] - f[0]) / 21.0, f12 = (f[2] - f[1]) / 21.0, f23 = (f[3] - f[2]) / 21.0;
    const double f012 = (f12 - f01) / 42.0, f123 = (f23 - f12) / 42.0;
    d[0] = f[0];
    d[1] = f01;
    d[2] = f012;
    d[3] = (f123 - f012) / 63.0;
}

__host__ __device__ __forceinline__ double hp_cubic_eval(const double* d, double t) {
    return d[0] + t * (d[1] + (t - 21.0) * (d[2] + (t - 42.0) * d[3]));
}

// Whether a whole segment-image row lies in the equatorial belt (where the
// row interpolation is used): ring indices of its two end pixels in [N, 3N].
__host__ __device__ __forceinline__ bool hp_row_in_belt(const HpArgs& a, long long seg, int r) {
    const long long N = a.nside_seg;
    const long long face = seg / (N * N);
    if (seg < 0 || face >= 12) return false;
    const long long ipf = seg - face * N * N;
    long long X = 0, Y = 0;
    for (int b = 0; (1LL << b) < N; b++) {
        X |= ((ipf >> (2 * b)) & 1LL) << b;
        Y |= ((ipf >> (2 * b + 1)) & 1LL) << b;
    }
    const long long nside = N << a.k, m = 1LL << a.k;
    const long long jrll = face < 4 ? 2 : (face < 8 ? 3 : 4);
    const long long iy = (Y << a.k) + r;
    const long long jr0 = jrll * nside - (X << a.k) - iy - 1;         // column 0
    const long long jr1 = jr0 - (m - 1);                              // column m - 1
    return jr1 >= nside && jr0 <= 3 * nside;
}

// One warp per segment-image row (k >= 6): in the belt, lanes compute the
// exact positions of the four nodes of eight pieces at once and each lane
// evaluates 16 pixels of its piece from the cubic; elsewhere (and for pieces
// with a node behind the tangent plane) every pixel takes the exact path.
__global__ void __launch_bounds__(256) healpix_rows_kernel(HpArgs a) {
    const int lane = threadIdx.x & 31;
    const long m = 1L << a.k;
    const long rows = (long)a.n_seg * m;
    const int npieces = (int)(m / HP_PIECE);
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    for (long wr = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wr < rows; wr += warps) {
        const long s = wr / m;
        const int r = (int)(wr - s * m);
        const long long seg = a.segs[s];
        float* orow = a.out + wr * m;
        uint8_t* crow = a.cov ? a.cov + wr * m : nullptr;
        if (!hp_row_in_belt(a, seg, r)) {
            for (int c = lane; c < m; c += 32) {
                double x, y;
                float v = 0.0f;
                const bool ok = hp_pixel_xy(a, seg, c, r, x, y) && hp_bilinear(a, x, y, v);
                orow[c] = ok ? v : 0.0f;
                if (crow) crow[c] = ok ? 1 : 0;
            }
            continue;
        }
        for (int pg = 0; pg < npieces; pg += 8) {
            const int p = pg + (lane >> 2), j = lane & 3;
            double xn = 0.0, yn = 0.0;
            bool okn = false;
            if (p < npieces) okn = hp_pixel_xy(a, seg, p * HP_PIECE + hp_node(j), r, xn, yn);
            // the piece's four nodes from lanes 4 (lane / 4) + 0..3
            double fx[4], fy[4];
            bool all = true;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int src = (lane & ~3) + q;
                fx[q] = __shfl_sync(0xffffffffu, xn, src);
                fy[q] = __shfl_sync(0xffffffffu, yn, src);
                all = all && __shfl_sync(0xffffffffu, okn ? 1 : 0, src);
            }
            if (p >= npieces) continue;                 // no barrier or shuffle below
            double dx[4], dy[4];
            hp_cubic_coeffs(fx, dx);
            hp_cubic_coeffs(fy, dy);
            for (int i = 0; i < HP_PIECE / 4; i++) {
                const int t = 4 * i + j;
                const int c = p * HP_PIECE + t;
                double x, y;
                bool ok;
                if (all) {
                    x = hp_cubic_eval(dx, (double)t);
                    y = hp_cubic_eval(dy, (double)t);
                    ok = true;
                } else {
                    ok = hp_pixel_xy(a, seg, c, r, x, y);
                }
                float v = 0.0f;
                ok = ok && hp_bilinear(a, x, y, v);
                orow[c] = ok ? v : 0.0f;
                if (crow) crow[c] = ok ? 1 : 0;
            }
        }
    }
}

__global__ void __launch_bounds__(256) healpix_resample_kernel(HpArgs a) {
    const long m = 1L << a.k;
    const long total = (long)a.n_seg * m * m;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long s = e / (m * m);
        const long q = e - s * m * m;
        const int r = (int)(q >> a.k), c = (int)(q & (m - 1));
        double x, y;
        float v = 0.0f;
        const bool ok = hp_pixel_xy(a, a.segs[s], c, r, x, y) && hp_bilinear(a, x, y, v);
        a.out[e] = ok ? v : 0.0f;
        if (a.cov) a.cov[e] = ok ? 1 : 0;
    }
}

// Host side of the argument set: the tangent-plane basis from the WCS.
__host__ inline void hp_fill_wcs(HpArgs& a, const argus_wcs& w) {
    const double ca = std::cos(w.alpha0), sa = std::sin(w.alpha0), cd = std::cos(w.delta0), sd = std::sin(w.delta0);
    a.n[0] = cd * ca; a.n[1] = cd * sa; a.n[2] = sd;
    a.e[0] = -sa; a.e[1] = ca; a.e[2] = 0.0;
    a.u[0] = -sd * ca; a.u[1] = -sd * sa; a.u[2] = cd;
    a.cr = std::cos(w.rot);
    a.sr = std::sin(w.rot);
    a.inv_scale = 1.0 / w.scale;
    a.cx = w.cx;
    a.cy = w.cy;
}

}  // namespace

extern "C" int argus_healpix_resample(const float* frame, const uint8_t* flags, argus_shape shape, argus_wcs wcs,
                                      int nside_seg, int k, const long long* segs, int n_seg, float* out,
                                      uint8_t* coverage, argus_stream stream) {
    if (!frame || !segs || !out || n_seg < 1 || k < 0 || k > 12 || nside_seg < 1 || nside_seg > (1 << 17) ||
        (nside_seg & (nside_seg - 1)) || !(wcs.scale > 0.0))
        return ARGUS_ERR_ARG;
    if ((long long)nside_seg << k > (1LL << 29)) return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, (size_t)-1);
    if (st) return st;
    HpArgs a;
    a.frame = frame; a.flags = flags; a.pitch = shape.pitch; a.w = shape.w; a.h = shape.h;
    a.segs = segs; a.n_seg = n_seg; a.nside_seg = nside_seg; a.k = k; a.out = out; a.cov = coverage;
    hp_fill_wcs(a, wcs);
    if (k >= 6) {                                  // rows of whole 64-pixel pieces: row interpolation
        const long rows = (long)n_seg << k;
        long blocks = (rows + 7) / 8;                  // 8 warps (rows) per CTA
        if (blocks > 152L * 32) blocks = 152L * 32;
        healpix_rows_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a);
    } else {
        const long total = (long)n_seg << (2 * k);
        long blocks = (total + 255) / 256;
        if (blocks > 152L * 32) blocks = 152L * 32;
        healpix_resample_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a);
    }
    argus_count_launch(1);
    return argus_launch_status();
}
