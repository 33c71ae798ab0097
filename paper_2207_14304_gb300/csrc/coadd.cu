// K2: sigma-clipped mean coadd of a stack of raw frames with per-frame
// sub-pixel shifts (paper Sec. 4.1.3, deep coaddition of 30 x 30 s frames into
// a 15-minute coadd; the clipped mean stands in for the matched filter there),
// with calibration fused in.
//
// One thread per output pixel.  The frame loop is unrolled to the compile-time
// stack bound NMAX so every per-frame value lives in a register at a static
// index: invalid or absent frames hold +inf and sort to the end.  A bitonic
// network sorts the samples; because rejection |v - c| > kappa*s keeps a
// value-closed set, the survivors stay one contiguous range [lo, hi) of the
// sorted array, and every statistic is a predicated pass over static indices.
// Traffic: 2 bytes per frame plus 9 bytes of calibration per pixel in, 9 out.
#include "argus_internal.cuh"

namespace {

struct CoaddArgs {
    const uint16_t* raw;
    const float* shifts;
    const float* dark;
    const float* flat;
    const uint8_t* bpm;
    float* coadd;
    float* var;
    uint8_t* n_used;
    long pitch, frame_stride;
    int w, h, nf, bias, sat, max_iter;
    float gain, rn2, kappa;
};

__device__ __forceinline__ bool calib_px(const CoaddArgs& a, int f, int x, int y, float& v, float& vr) {
    if (x < 0 || y < 0 || x >= a.w || y >= a.h) return false;
    const long p = (long)y * a.pitch + x;
    const int raw = a.raw[(long)f * a.frame_stride + p];
    const float fl = a.flat ? __ldg(a.flat + p) : 1.0f;
    if ((a.bpm && __ldg(a.bpm + p)) || !(fl > 0.0f) || !(fl <= 3.402823466e38f) || raw >= a.sat) return false;
    const float ng = (float)(raw - a.bias) * a.gain;
    v = (ng - (a.dark ? __ldg(a.dark + p) : 0.0f)) / fl;
    vr = (fmaxf(ng, 0.0f) + a.rn2) / (fl * fl);
    return true;
}

template <int N>
__device__ __forceinline__ void bitonic_sort(float (&s)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const float a = s[i], b = s[l];
                    const bool up = (i & k) == 0;
                    s[i] = up ? fminf(a, b) : fmaxf(a, b);
                    s[l] = up ? fmaxf(a, b) : fminf(a, b);
                }
            }
}

template <int N>
__device__ __forceinline__ float pick(const float (&s)[N], int idx) {
    float r = 0.0f;
#pragma unroll
    for (int i = 0; i < N; i++) r = (i == idx) ? s[i] : r;
    return r;
}

template <int N>
__device__ __forceinline__ float median_range(const float (&s)[N], int lo, int hi) {
    const int n = hi - lo;
    const float a = pick(s, lo + (n - 1) / 2), b = pick(s, lo + n / 2);
    return (n & 1) ? b : 0.5f * (a + b);
}

template <int NMAX>
__global__ void __launch_bounds__(128) coadd_kernel(CoaddArgs a) {
    __shared__ int s_ix[NMAX], s_iy[NMAX];
    __shared__ float s_fx[NMAX], s_fy[NMAX];
    for (int f = threadIdx.x; f < NMAX; f += blockDim.x) {
        if (f < a.nf) {
            const double dx = a.shifts[2 * f], dy = a.shifts[2 * f + 1];
            const double fx = floor(dx), fy = floor(dy);
            s_ix[f] = (int)fx;
            s_iy[f] = (int)fy;
            s_fx[f] = (float)(dx - fx);
            s_fy[f] = (float)(dy - fy);
        } else {
            s_ix[f] = 0; s_iy[f] = 0; s_fx[f] = 0.0f; s_fy[f] = 0.0f;
        }
    }
    __syncthreads();
    const long np = (long)a.w * a.h;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < np; e += (long)gridDim.x * blockDim.x) {
        const int y = (int)(e / a.w), x = (int)(e - (long)y * a.w);
        float v[NMAX], vv[NMAX];
        int n = 0;
#pragma unroll
        for (int f = 0; f < NMAX; f++) {
            v[f] = __int_as_float(0x7f800000);   // +inf: absent
            vv[f] = 0.0f;
            if (f < a.nf) {
                const int ix = x + s_ix[f], iy = y + s_iy[f];
                const float fx = s_fx[f], fy = s_fy[f];
                const bool n1 = fx > 0.0f, n2 = fy > 0.0f;
                float v00, r00, v10 = 0.0f, r10 = 0.0f, v01 = 0.0f, r01 = 0.0f, v11 = 0.0f, r11 = 0.0f;
                bool ok = calib_px(a, f, ix, iy, v00, r00);
                if (ok && n1) ok = calib_px(a, f, ix + 1, iy, v10, r10);
                if (ok && n2) ok = calib_px(a, f, ix, iy + 1, v01, r01);
                if (ok && n1 && n2) ok = calib_px(a, f, ix + 1, iy + 1, v11, r11);
                if (ok) {
                    if (!n1) v10 = v00;
                    if (!n2) v01 = v00;
                    if (!(n1 && n2)) v11 = n1 ? v10 : v01;
                    const float top = v00 + fx * (v10 - v00);
                    const float bot = v01 + fx * (v11 - v01);
                    const float sv = top + fy * (bot - top);
                    ok = isfinite(sv);
                    v[f] = ok ? sv : __int_as_float(0x7f800000);
                    const float w0 = (1.0f - fx) * (1.0f - fy), w1 = fx * (1.0f - fy);
                    const float w2 = (1.0f - fx) * fy, w3 = fx * fy;
                    vv[f] = w0 * w0 * r00 + (n1 ? w1 * w1 * r10 : 0.0f) + (n2 ? w2 * w2 * r01 : 0.0f) +
                            (n1 && n2 ? w3 * w3 * r11 : 0.0f);
                    n += ok ? 1 : 0;
                }
            }
        }
        float s[NMAX];
#pragma unroll
        for (int f = 0; f < NMAX; f++) s[f] = v[f];
        bitonic_sort(s);
        int lo = 0, hi = n;
        for (int it = 0; it < a.max_iter && hi > lo; it++) {
            const int cnt = hi - lo;
            const float c = median_range(s, lo, hi);
            float sum = 0.0f;
#pragma unroll
            for (int i = 0; i < NMAX; i++) sum += (i >= lo && i < hi) ? s[i] : 0.0f;
            const float m = sum / (float)cnt;
            float s2 = 0.0f;
#pragma unroll
            for (int i = 0; i < NMAX; i++) {
                const float d = s[i] - m;
                s2 += (i >= lo && i < hi) ? d * d : 0.0f;
            }
            const float ks = a.kappa * sqrtf(s2 / (float)cnt);
            int nlo = 0, nhi = 0;
#pragma unroll
            for (int i = 0; i < NMAX; i++) {
                const bool in = i >= lo && i < hi;
                const bool rej = in && (fabsf(s[i] - c) > ks);
                nlo += (rej && s[i] < c) ? 1 : 0;
                nhi += (rej && s[i] >= c) ? 1 : 0;
            }
            if (nlo + nhi == 0 || nlo + nhi == cnt) break;
            lo += nlo;
            hi -= nhi;
        }
        const long p = (long)y * a.pitch + x;
        if (hi <= lo) {
            a.coadd[p] = 0.0f;
            a.var[p] = 0.0f;
            a.n_used[p] = 0;
            continue;
        }
        const int cnt = hi - lo;
        const float c = median_range(s, lo, hi);
        const float vlo = pick(s, lo), vhi = pick(s, hi - 1);
        float sd = 0.0f, sv = 0.0f;
#pragma unroll
        for (int i = 0; i < NMAX; i++) sd += (i >= lo && i < hi) ? s[i] - c : 0.0f;
#pragma unroll
        for (int f = 0; f < NMAX; f++) sv += (v[f] >= vlo && v[f] <= vhi) ? vv[f] : 0.0f;
        a.coadd[p] = c + sd / (float)cnt;
        a.var[p] = sv / ((float)cnt * (float)cnt);
        a.n_used[p] = (uint8_t)cnt;
    }
}

template <int NMAX>
int launch(const CoaddArgs& a, int sms, cudaStream_t st) {
    const long np = (long)a.w * a.h;
    long blocks = (np + 127) / 128;
    if (blocks > (long)sms * 16) blocks = (long)sms * 16;
    coadd_kernel<NMAX><<<(unsigned)blocks, 128, 0, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}

}  // namespace

extern "C" int argus_coadd(argus_ctx* ctx, const uint16_t* raw_stack, int n, argus_shape shape,
                           const float* shifts_xy, const argus_calib* calib, float kappa, int max_iter,
                           float* coadd, float* var, uint8_t* n_used, argus_stream stream) {
    if (!ctx || !raw_stack || !shifts_xy || !calib || !coadd || !var || !n_used) return ARGUS_ERR_ARG;
    if (n < 1 || n > ARGUS_MAX_FRAMES || max_iter < 0 || !(kappa > 0.0f)) return ARGUS_ERR_ARG;
    if (calib->bias_frame) return ARGUS_ERR_UNSUPPORTED;
    int rc = argus_check_shape(shape, ctx->max_pixels);
    if (rc) return rc;
    const void* ps[] = {raw_stack, coadd, var, n_used, calib->dark, calib->flat, calib->bpm};
    for (const void* p : ps)
        if (p && argus_check_ptr16(p)) return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    CoaddArgs a;
    a.raw = raw_stack; a.shifts = shifts_xy; a.dark = calib->dark; a.flat = calib->flat; a.bpm = calib->bpm;
    a.coadd = coadd; a.var = var; a.n_used = n_used; a.pitch = shape.pitch;
    a.frame_stride = shape.pitch * (long)shape.h; a.w = shape.w; a.h = shape.h; a.nf = n;
    a.bias = calib->bias_scalar; a.sat = calib->sat; a.max_iter = max_iter; a.gain = calib->gain;
    a.rn2 = calib->read_noise * calib->read_noise; a.kappa = kappa;
    cudaStream_t st = (cudaStream_t)stream;
    if (n <= 8) return launch<8>(a, ctx->num_sms, st);
    if (n <= 16) return launch<16>(a, ctx->num_sms, st);
    if (n <= 32) return launch<32>(a, ctx->num_sms, st);
    return launch<64>(a, ctx->num_sms, st);
}
