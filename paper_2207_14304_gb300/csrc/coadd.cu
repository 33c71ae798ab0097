// K2: sigma-clipped mean coadd of a stack of raw frames with per-frame
// sub-pixel shifts (paper Sec. 4.1.3, deep coaddition of 30 x 30 s frames into
// a 15-minute coadd; the clipped mean stands in for the matched filter there),
// with calibration fused in.
//
// One thread per output pixel of a 32 x 8 tile.  Per frame, the raw window
// the tile needs is loaded once, coalesced, and calibrated into shared memory.
// The frame loop is unrolled to the compile-time stack bound NMAX so every
// per-frame sample lives in a register at a static index: invalid or absent
// frames hold +inf and sort to the end.  A bitonic network sorts the samples;
// because rejection |v - c| > kappa*s keeps a value-closed set, the survivors
// stay one contiguous range [lo, hi) of the sorted array, so each clipping
// pass touches only that range of the sorted column in shared memory.
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

// One CTA per 32 x 8 output tile.  Per tile:
//
// Phase 0: the calibration constants (the reciprocal of the flat, or NaN where
// the pixel is unusable -- outside the frame, flagged bad, flat not positive
// and finite -- and the dark) of the union of the frames' windows into shared
// memory, once: frames share their pixels' calibration, and their windows
// differ only by the integer parts of the shifts.  When that union exceeds
// UCAP pixels (shifts spread by more than 4 px) each frame's window reads its
// constants from global memory instead.
//
// Phase 1: every frame's (33 x 9) window of raw pixels -- at the frame's
// integer offset -- calibrated into shared memory as (value, variance) pairs:
// value NaN where unusable.  The nf x 297 window pixels are spread evenly over
// the threads; per pixel one raw load and table lookups.  The flat enters
// through its correctly rounded reciprocal (within 1 ulp of the quotient).
//
// Phase 2: each thread interpolates its samples from four shared pairs per
// frame (the value by nested lerps, the variance by the squared weights) and
// sums the variances of the valid samples as it goes; it sorts the values in
// registers with a bitonic network and writes the sorted column to shared
// memory.  The survivors of a clipping pass stay one contiguous range [lo, hi)
// of the sorted samples, so each pass reads only that range: the median from
// two slots, the mean and the spread in two loops over the range, and the
// rejected samples by scanning inward from both ends (the rejected set is a
// prefix below the median and a suffix above it, because the rounded distance
// to the median is monotone in the sample).  The variance of the mean is the
// valid samples' sum minus the rejected samples' variances, summed with
// error-free transformations.
constexpr int CTX = 32, CTY = 8, CWX = CTX + 1, CWY = CTY + 1, CWN = CWX * CWY;
constexpr int CT = CTX * CTY;                  // threads (one per output pixel of the tile)
constexpr int UCAP = 512;                      // union window capacity (pixels): shift spreads up to 4 px
constexpr float FMAXF = 3.402823466e38f;

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fffffff); }

// Median of the sorted range [lo, hi) of one thread's column of samples
// (slot i at col[i * CT]); the mean of the two middle values for even counts.
__device__ __forceinline__ float median_col(const float* col, int lo, int hi) {
    const int n = hi - lo;
    const float a = col[(lo + (n - 1) / 2) * CT], b = col[(lo + n / 2) * CT];
    return (n & 1) ? b : 0.5f * (a + b);
}

// Calibration constants of frame pixel (gx, gy): (1 / flat, dark), with NaN
// in place of 1 / flat when the pixel is unusable.
__device__ __forceinline__ float2 calib_const(const CoaddArgs& a, int gx, int gy) {
    float2 c = make_float2(qnan(), 0.0f);
    if (gx >= 0 && gy >= 0 && gx < a.w && gy < a.h) {
        const long p = (long)gy * a.pitch + gx;
        const float fl = a.flat ? __ldg(a.flat + p) : 1.0f;
        const bool bad = a.bpm && __ldg(a.bpm + p);
        if (!bad && fl > 0.0f && fl <= FMAXF) c.x = __frcp_rn(fl);
        c.y = a.dark ? __ldg(a.dark + p) : 0.0f;
    }
    return c;
}

// Calibrated (value, variance) of one raw pixel given its constants.
__device__ __forceinline__ float2 calib_pair(const CoaddArgs& a, int raw, float2 c) {
    float2 r = make_float2(qnan(), 0.0f);
    if (c.x == c.x && raw < a.sat) {
        const float ng = (float)(raw - a.bias) * a.gain;
        const float cv = (ng - c.y) * c.x;
        if (fabsf(cv) <= FMAXF) {   // non-finite: unusable
            r.x = cv;
            r.y = (fmaxf(ng, 0.0f) + a.rn2) * (c.x * c.x);
        }
    }
    return r;
}

// s + e = a + b exactly (Knuth's two-sum; no reassociation: the library is not
// built with fast-math).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Bilinear sample of one frame from its calibrated window: the value by nested
// lerps with explicit fused multiply-adds (non-finite when a needed pixel is
// unusable), the variance as the sum of squared weights (q) times the four
// pixels' variances.
__device__ __forceinline__ float sample(const float2* w, int o, float fx, float fy, float4 q, float& var) {
    const bool n1 = fx > 0.0f, n2 = fy > 0.0f;
    const float2 p00 = w[o];
    const float2 p10 = n1 ? w[o + 1] : p00;
    const float2 p01 = n2 ? w[o + CWX] : p00;
    const float2 p11 = (n1 && n2) ? w[o + CWX + 1] : (n1 ? p10 : p01);
    var = q.x * p00.y + (n1 ? q.y * p10.y : 0.0f) + (n2 ? q.z * p01.y : 0.0f) + (n1 && n2 ? q.w * p11.y : 0.0f);
    const float top = __fmaf_rn(fx, __fsub_rn(p10.x, p00.x), p00.x);
    const float bot = __fmaf_rn(fx, __fsub_rn(p11.x, p01.x), p01.x);
    return __fmaf_rn(fy, __fsub_rn(bot, top), top);
}

template <int NMAX>
__global__ void __launch_bounds__(CT, NMAX <= 32 ? 2 : 1) coadd_kernel(CoaddArgs a) {
    extern __shared__ float4 coadd_smem[];
    float2* wvr = reinterpret_cast<float2*>(coadd_smem);         // [nf][CWN] (value, variance)
    float* ss = reinterpret_cast<float*>(wvr + a.nf * CWN);      // [NMAX][CT] sorted samples, a column per thread
    float2* ucal = reinterpret_cast<float2*>(ss + NMAX * CT);    // [UCAP] union calibration window
    __shared__ int2 s_j[CWN];              // window pixel j: (union offset jy * UW + jx, raw offset jy * pitch + jx)
    __shared__ short2 s_jxy[CWN];          // (jx, jy)
    __shared__ int s_ix[NMAX], s_iy[NMAX], s_fofs[NMAX];
    __shared__ long long s_rb[NMAX];       // per tile: raw element offset of frame f's window origin
    __shared__ float2 s_fxy[NMAX];
    __shared__ float4 s_q[NMAX];
    __shared__ int s_umin[2], s_uwh[2];
    const int tid = threadIdx.x;
    if (tid == 0) { s_umin[0] = s_umin[1] = 1 << 30; s_uwh[0] = s_uwh[1] = -(1 << 30); }
    __syncthreads();
    for (int f = tid; f < NMAX; f += blockDim.x) {
        float fxf = 0.0f, fyf = 0.0f;
        int ix = 0, iy = 0;
        if (f < a.nf) {
            const double dx = a.shifts[2 * f], dy = a.shifts[2 * f + 1];
            const double fx = floor(dx), fy = floor(dy);
            ix = (int)fx;
            iy = (int)fy;
            fxf = (float)(dx - fx);
            fyf = (float)(dy - fy);
            atomicMin(&s_umin[0], ix); atomicMin(&s_umin[1], iy);
            atomicMax(&s_uwh[0], ix); atomicMax(&s_uwh[1], iy);
        }
        s_ix[f] = ix;
        s_iy[f] = iy;
        s_fxy[f] = make_float2(fxf, fyf);
        const float w0 = (1.0f - fxf) * (1.0f - fyf), w1 = fxf * (1.0f - fyf);
        const float w2 = (1.0f - fxf) * fyf, w3 = fxf * fyf;
        s_q[f] = make_float4(w0 * w0, w1 * w1, w2 * w2, w3 * w3);
    }
    __syncthreads();
    const int ixmin = s_umin[0], iymin = s_umin[1];
    const int UW = CWX + (s_uwh[0] - ixmin), UH = CWY + (s_uwh[1] - iymin);
    const bool uni = UW * UH <= UCAP;      // the same for every CTA
    for (int j = tid; j < CWN; j += blockDim.x) {
        const int jy = j / CWX, jx = j - jy * CWX;
        s_j[j] = make_int2(jy * UW + jx, (int)(jy * a.pitch) + jx);
        s_jxy[j] = make_short2((short)jx, (short)jy);
    }
    for (int f = tid; f < a.nf; f += blockDim.x) s_fofs[f] = (s_iy[f] - iymin) * UW + (s_ix[f] - ixmin);
    const int ntx = (a.w + CTX - 1) / CTX, nty = (a.h + CTY - 1) / CTY;
    const int lx = tid % CTX, ly = tid / CTX;
    const int o = ly * CWX + lx;
    const int tot = a.nf * CWN;
    float* col = ss + tid;
    for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
        const int tx0 = (tile % ntx) * CTX, ty0 = (tile / ntx) * CTY;
        const int x = tx0 + lx, y = ty0 + ly;
        __syncthreads();   // tables staged; previous tile's windows consumed
        for (int f = tid; f < a.nf; f += blockDim.x)
            s_rb[f] = (long long)f * a.frame_stride + (long long)(ty0 + s_iy[f]) * a.pitch + (tx0 + s_ix[f]);
        if (uni)
            for (int e = tid; e < UW * UH; e += blockDim.x) {
                const int uy = e / UW, ux = e - uy * UW;
                ucal[e] = calib_const(a, tx0 + ixmin + ux, ty0 + iymin + uy);
            }
        __syncthreads();
        // window pixel e = f * CWN + j, e = tid + k * CT: j advances by CT < CWN, wrapping at most once
        int f = 0, j = tid;
        constexpr int U = 4;
        for (int e0 = tid; e0 < tot; e0 += U * CT) {
            int fu[U], ju[U], raw[U];
            float2 cu[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                fu[u] = f;
                ju[u] = j;
                j += CT;
                if (j >= CWN) { j -= CWN; f++; }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const bool live = e0 + u * CT < tot;
                const int fc = live ? fu[u] : 0;
                if (uni) {
                    cu[u] = ucal[s_fofs[fc] + s_j[ju[u]].x];
                } else {
                    const short2 jj = s_jxy[ju[u]];
                    cu[u] = calib_const(a, tx0 + s_ix[fc] + jj.x, ty0 + s_iy[fc] + jj.y);
                }
                raw[u] = (live && cu[u].x == cu[u].x) ? (int)__ldg(a.raw + s_rb[fc] + s_j[ju[u]].y) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; u++)
                if (e0 + u * CT < tot) wvr[fu[u] * CWN + ju[u]] = calib_pair(a, raw[u], cu[u]);
        }
        __syncthreads();
        if (x >= a.w || y >= a.h) continue;
        float u[NMAX], s[NMAX];
        int n = 0;
        float svh = 0.0f, svl = 0.0f;   // compensated sum of the valid samples' variances
#pragma unroll
        for (int fi = 0; fi < NMAX; fi++) {
            float sv = __int_as_float(0x7f800000);   // +inf: absent or invalid
            u[fi] = sv;
            if (fi < a.nf) {
                const float2 fxy = s_fxy[fi];
                float vr;
                const float v = sample(wvr + fi * CWN, o, fxy.x, fxy.y, s_q[fi], vr);
                const bool ok = fabsf(v) <= FMAXF;
                u[fi] = v;
                sv = ok ? v : sv;
                n += ok ? 1 : 0;
                float e;
                two_sum(svh, ok ? vr : 0.0f, svh, e);
                svl += e;
            }
            s[fi] = sv;
        }
        bitonic_sort(s);
#pragma unroll
        for (int i = 0; i < NMAX; i++) col[i * CT] = s[i];
        int lo = 0, hi = n;
        float last_s1 = 0.0f;   // sum of v - median over [lo, hi) when the last pass kept every sample
        bool have_s1 = false;
        for (int it = 0; it < a.max_iter && hi > lo; it++) {
            const int cnt = hi - lo;
            const float c = median_col(col, lo, hi);
            // mean and spread in one pass over the range, about the median (the sums of
            // v - c and (v - c)^2; the median lies inside the samples, so the difference
            // of the second sum and the squared first one does not cancel)
            float s1 = 0.0f, s2 = 0.0f;
            for (int i = lo; i < hi; i++) {
                const float d = col[i * CT] - c;
                s1 += d;
                s2 = fmaf(d, d, s2);
            }
            const float d1 = s1 / (float)cnt;
            const float ks = a.kappa * sqrtf(fmaxf(s2 / (float)cnt - d1 * d1, 0.0f));
            int nlo = 0, nhi = 0;
            while (lo + nlo < hi) {
                const float v = col[(lo + nlo) * CT];
                if (!(v < c && fabsf(v - c) > ks)) break;
                nlo++;
            }
            while (hi - 1 - nhi >= lo + nlo) {
                const float v = col[(hi - 1 - nhi) * CT];
                if (!(v >= c && fabsf(v - c) > ks)) break;
                nhi++;
            }
            if (nlo + nhi == 0) {
                last_s1 = s1;
                have_s1 = true;
                break;
            }
            if (nlo + nhi == cnt) break;
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
        const float c = median_col(col, lo, hi);
        const float vlo = col[lo * CT], vhi = col[(hi - 1) * CT];
        float sd = last_s1;   // the converged pass's sum over the same range about the same median
        if (!have_s1)
            for (int i = lo; i < hi; i++) sd += col[i * CT] - c;
        if (cnt < n) {   // the rejected samples' variances out (compensated: a rejected cosmic
                         // ray's variance can exceed the survivors' sum many times); the
                         // rejected frames as a bit mask first, then one sample per set bit,
                         // so a warp runs as many samples as its lane with the most rejections
            unsigned long long rej = 0ull;
#pragma unroll
            for (int fi = 0; fi < NMAX; fi++)
                if (fi < a.nf && fabsf(u[fi]) <= FMAXF && (u[fi] < vlo || u[fi] > vhi)) rej |= 1ull << fi;
            while (rej) {
                const int fi = __ffsll((long long)rej) - 1;
                rej &= rej - 1ull;
                const float2 fxy = s_fxy[fi];
                float vr;
                sample(wvr + fi * CWN, o, fxy.x, fxy.y, s_q[fi], vr);
                float e;
                two_sum(svh, -vr, svh, e);
                svl += e;
            }
        }
        const float svar = svh + svl;
        a.coadd[p] = c + sd / (float)cnt;
        a.var[p] = svar / ((float)cnt * (float)cnt);
        a.n_used[p] = (uint8_t)cnt;
    }
}

template <int NMAX>
int launch(const CoaddArgs& a, int sms, cudaStream_t st) {
    const size_t smem = ((size_t)a.nf * CWN * 2 + (size_t)NMAX * CT + (size_t)UCAP * 2) * sizeof(float);
    if (cudaFuncSetAttribute(coadd_kernel<NMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(coadd_kernel<NMAX>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coadd_kernel<NMAX>, CT, smem) != cudaSuccess ||
        per_sm < 1)
        return ARGUS_ERR_CUDA;
    const long tiles = (long)((a.w + CTX - 1) / CTX) * ((a.h + CTY - 1) / CTY);
    long blocks = tiles;
    if (blocks > (long)sms * per_sm) blocks = (long)sms * per_sm;
    coadd_kernel<NMAX><<<(unsigned)blocks, CT, smem, st>>>(a); argus_count_launch(1);
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
