// K2: sigma-clipped mean coadd of a stack of raw frames with per-frame
// sub-pixel shifts (paper Sec. 4.1.3, deep coaddition of 30 x 30 s frames into
// a 15-minute coadd; the clipped mean stands in for the matched filter there),
// with calibration fused in.
//
// One thread per output pixel of a 32 x 8 tile.  Per frame, the raw window
// the tile needs is loaded once, coalesced, and calibrated into shared memory.
// The frame loop is unrolled to the compile-time stack bound NMAX so every
// per-frame value lives in a register at a static index: invalid or absent
// frames hold +inf and sort to the end.  A bitonic
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

// One CTA per 32 x 8 output tile.  Phase 1 loads, for every frame, the
// (33 x 9) window of raw pixels the tile's samples need -- placed at the
// frame's integer offset -- with coalesced reads (all frames' loads in flight
// together) and calibrates each pixel once into shared memory: value, or NaN
// where the pixel is unusable, and variance.  Phase 2: each thread
// interpolates its samples from four shared values per frame, sorts them in
// registers and clips; the survivors' variances are recomputed from shared
// memory in the last pass instead of being held in registers.
constexpr int CTX = 32, CTY = 8, CWX = CTX + 1, CWY = CTY + 1, CWN = CWX * CWY;

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fffffff); }

// Bilinear sample of one frame from its calibrated window (nested lerps with
// explicit fused multiply-adds, so that the two evaluations of a sample in the
// kernel round identically).  Non-finite when a needed pixel is unusable.
__device__ __forceinline__ float sample(const float* wv, int o, float fx, float fy) {
    const bool n1 = fx > 0.0f, n2 = fy > 0.0f;
    const float v00 = wv[o];
    const float v10 = n1 ? wv[o + 1] : v00;
    const float v01 = n2 ? wv[o + CWX] : v00;
    const float v11 = (n1 && n2) ? wv[o + CWX + 1] : (n1 ? v10 : v01);
    const float top = __fmaf_rn(fx, __fsub_rn(v10, v00), v00);
    const float bot = __fmaf_rn(fx, __fsub_rn(v11, v01), v01);
    return __fmaf_rn(fy, __fsub_rn(bot, top), top);
}

__device__ __forceinline__ float sample_var(const float* wr, int o, float fx, float fy) {
    const bool n1 = fx > 0.0f, n2 = fy > 0.0f;
    const float w0 = (1.0f - fx) * (1.0f - fy), w1 = fx * (1.0f - fy);
    const float w2 = (1.0f - fx) * fy, w3 = fx * fy;
    return w0 * w0 * wr[o] + (n1 ? w1 * w1 * wr[o + 1] : 0.0f) + (n2 ? w2 * w2 * wr[o + CWX] : 0.0f) +
           (n1 && n2 ? w3 * w3 * wr[o + CWX + 1] : 0.0f);
}

template <int NMAX>
__global__ void __launch_bounds__(CTX * CTY) coadd_kernel(CoaddArgs a) {
    extern __shared__ float4 coadd_smem[];
    float* wv = reinterpret_cast<float*>(coadd_smem);   // [nf][CWY][CWX] values
    float* wr = wv + a.nf * CWN;                         // [nf][CWY][CWX] variances
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
    const int ntx = (a.w + CTX - 1) / CTX, nty = (a.h + CTY - 1) / CTY;
    const int lx = threadIdx.x % CTX, ly = threadIdx.x / CTX;
    const int o = ly * CWX + lx;
    const int tot = a.nf * CWN;
    constexpr int U = 4;
    for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
        const int tx0 = (tile % ntx) * CTX, ty0 = (tile / ntx) * CTY;
        const int x = tx0 + lx, y = ty0 + ly;
        __syncthreads();   // shifts staged; previous tile's windows consumed
        for (int e0 = threadIdx.x; e0 < tot; e0 += U * CTX * CTY) {
            int raw[U];
            long p[U];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int e = e0 + u * CTX * CTY;
                const int f = e / CWN, j = e - f * CWN;
                const int jy = j / CWX, jx = j - jy * CWX;
                const int gx = tx0 + s_ix[f < a.nf ? f : 0] + jx, gy = ty0 + s_iy[f < a.nf ? f : 0] + jy;
                in[u] = e < tot && gx >= 0 && gy >= 0 && gx < a.w && gy < a.h;
                p[u] = in[u] ? (long)gy * a.pitch + gx : 0;
                raw[u] = in[u] ? (int)__ldg(a.raw + (long)f * a.frame_stride + p[u]) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int e = e0 + u * CTX * CTY;
                if (e >= tot) break;
                float cv = qnan(), cr = 0.0f;
                if (in[u]) {
                    const float fl = a.flat ? __ldg(a.flat + p[u]) : 1.0f;
                    const bool bad = (a.bpm && __ldg(a.bpm + p[u])) || !(fl > 0.0f) || !(fl <= 3.402823466e38f) ||
                                     raw[u] >= a.sat;
                    if (!bad) {
                        const float ng = (float)(raw[u] - a.bias) * a.gain;
                        cv = (ng - (a.dark ? __ldg(a.dark + p[u]) : 0.0f)) / fl;
                        cr = (fmaxf(ng, 0.0f) + a.rn2) / (fl * fl);
                        if (!(fabsf(cv) <= 3.402823466e38f)) cv = qnan();   // non-finite: unusable
                    }
                }
                wv[e] = cv;
                wr[e] = cr;
            }
        }
        __syncthreads();
        if (x >= a.w || y >= a.h) continue;
        float s[NMAX];
        int n = 0;
#pragma unroll
        for (int f = 0; f < NMAX; f++) {
            float sv = __int_as_float(0x7f800000);   // +inf: absent or invalid
            if (f < a.nf) {
                const float v = sample(wv + f * CWN, o, s_fx[f], s_fy[f]);
                const bool ok = fabsf(v) <= 3.402823466e38f;
                sv = ok ? v : sv;
                n += ok ? 1 : 0;
            }
            s[f] = sv;
        }
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
        float sd = 0.0f, svar = 0.0f;
#pragma unroll
        for (int i = 0; i < NMAX; i++) sd += (i >= lo && i < hi) ? s[i] - c : 0.0f;
        for (int f = 0; f < a.nf; f++) {
            const float fx = s_fx[f], fy = s_fy[f];
            const float v = sample(wv + f * CWN, o, fx, fy);
            if (v >= vlo && v <= vhi) svar += sample_var(wr + f * CWN, o, fx, fy);
        }
        a.coadd[p] = c + sd / (float)cnt;
        a.var[p] = svar / ((float)cnt * (float)cnt);
        a.n_used[p] = (uint8_t)cnt;
    }
}

template <int NMAX>
int launch(const CoaddArgs& a, int sms, cudaStream_t st) {
    const size_t smem = (size_t)a.nf * CWN * 2 * sizeof(float);
    if (cudaFuncSetAttribute(coadd_kernel<NMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return ARGUS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coadd_kernel<NMAX>, CTX * CTY, smem) != cudaSuccess ||
        per_sm < 1)
        return ARGUS_ERR_CUDA;
    const long tiles = (long)((a.w + CTX - 1) / CTX) * ((a.h + CTY - 1) / CTY);
    long blocks = tiles;
    if (blocks > (long)sms * per_sm) blocks = (long)sms * per_sm;
    coadd_kernel<NMAX><<<(unsigned)blocks, CTX * CTY, smem, st>>>(a); argus_count_launch(1);
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
