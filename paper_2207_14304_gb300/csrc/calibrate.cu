// K1: CMOS calibration (paper Sec. 4.1: dark subtraction, flat fielding and
// bad-pixel masking; Table 2 "Calibration"; Table 1: 16-bit IMX455 data,
// 1.7 e- read noise).
//
// HBM-bound: each thread moves 8 pixels with 128-bit loads of raw (8 x u16),
// dark and flat (2 x float4 each) and a 64-bit load of the bad-pixel mask, and
// 128-bit stores of img and var.  Algorithmic traffic: 2 + 4 + 4 + 1 (+2 for
// a bias frame) bytes in, 4 + 4 + 1 bytes out per pixel.
#include "argus_internal.cuh"

namespace {

struct CalibArgs {
    const uint16_t* raw;
    const uint16_t* biasf;
    const float* dark;
    const float* flat;
    const uint8_t* bpm;
    float* img;
    float* var;
    uint8_t* flags;
    int bias, sat, w, h;
    long pitch;
    float gain, rn2;
};

__device__ __forceinline__ void calib_px(int raw, int bias, float d, float f, int bp, float gain,
                                         float rn2, int sat, float& I, float& V, uint8_t& fl) {
    const int n = raw - bias;
    const bool flat_ok = (f > 0.0f) && (f <= 3.402823466e38f);
    fl = (uint8_t)(((bp != 0) || !flat_ok ? ARGUS_FLAG_BAD : 0) | (raw >= sat ? ARGUS_FLAG_SAT : 0));
    const float ng = (float)n * gain;
    if (flat_ok) {
        I = (ng - d) / f;
        V = (fmaxf(ng, 0.0f) + rn2) / (f * f);
    } else {
        I = 0.0f;
        V = 0.0f;
    }
}

__global__ void __launch_bounds__(256) calibrate_kernel(CalibArgs a) {
    const long vpr = a.pitch >> 3;  // 8-pixel vectors per row
    const long nv = vpr * a.h;
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nv; v += (long)gridDim.x * blockDim.x) {
        const long y = v / vpr;
        const int x0 = (int)(v - y * vpr) << 3;
        if (x0 >= a.w) continue;
        const long base = y * a.pitch + x0;
        if (x0 + 8 <= a.w) {
            const uint4 rv = *reinterpret_cast<const uint4*>(a.raw + base);
            uint16_t r[8];
            *reinterpret_cast<uint4*>(r) = rv;
            uint16_t bf[8];
            if (a.biasf) *reinterpret_cast<uint4*>(bf) = *reinterpret_cast<const uint4*>(a.biasf + base);
            float dk[8], fl[8];
            if (a.dark) {
                *reinterpret_cast<float4*>(dk) = *reinterpret_cast<const float4*>(a.dark + base);
                *reinterpret_cast<float4*>(dk + 4) = *reinterpret_cast<const float4*>(a.dark + base + 4);
            } else {
#pragma unroll
                for (int i = 0; i < 8; i++) dk[i] = 0.0f;
            }
            if (a.flat) {
                *reinterpret_cast<float4*>(fl) = *reinterpret_cast<const float4*>(a.flat + base);
                *reinterpret_cast<float4*>(fl + 4) = *reinterpret_cast<const float4*>(a.flat + base + 4);
            } else {
#pragma unroll
                for (int i = 0; i < 8; i++) fl[i] = 1.0f;
            }
            uint8_t bp[8];
            if (a.bpm) *reinterpret_cast<uint2*>(bp) = *reinterpret_cast<const uint2*>(a.bpm + base);
            else *reinterpret_cast<uint2*>(bp) = make_uint2(0, 0);
            float I[8], V[8];
            uint8_t F[8];
#pragma unroll
            for (int i = 0; i < 8; i++)
                calib_px(r[i], a.biasf ? (int)bf[i] : a.bias, dk[i], fl[i], bp[i], a.gain, a.rn2, a.sat,
                         I[i], V[i], F[i]);
            *reinterpret_cast<float4*>(a.img + base) = *reinterpret_cast<float4*>(I);
            *reinterpret_cast<float4*>(a.img + base + 4) = *reinterpret_cast<float4*>(I + 4);
            *reinterpret_cast<float4*>(a.var + base) = *reinterpret_cast<float4*>(V);
            *reinterpret_cast<float4*>(a.var + base + 4) = *reinterpret_cast<float4*>(V + 4);
            *reinterpret_cast<uint2*>(a.flags + base) = *reinterpret_cast<uint2*>(F);
        } else {
            for (int i = 0; x0 + i < a.w; i++) {
                const long p = base + i;
                float I, V;
                uint8_t F;
                calib_px(a.raw[p], a.biasf ? (int)a.biasf[p] : a.bias, a.dark ? a.dark[p] : 0.0f,
                         a.flat ? a.flat[p] : 1.0f, a.bpm ? a.bpm[p] : 0, a.gain, a.rn2, a.sat, I, V, F);
                a.img[p] = I;
                a.var[p] = V;
                a.flags[p] = F;
            }
        }
    }
}

}  // namespace

extern "C" int argus_calibrate(argus_ctx* ctx, const uint16_t* raw, argus_shape shape,
                               const argus_calib* calib, float* img, float* var, uint8_t* flags,
                               argus_stream stream) {
    if (!ctx || !raw || !calib || !img || !var || !flags) return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, ctx->max_pixels);
    if (st) return st;
    const void* ps[] = {raw, img, var, flags, calib->bias_frame, calib->dark, calib->flat, calib->bpm};
    for (const void* p : ps)
        if (p && argus_check_ptr16(p)) return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    CalibArgs a;
    a.raw = raw; a.biasf = calib->bias_frame; a.dark = calib->dark; a.flat = calib->flat;
    a.bpm = calib->bpm; a.img = img; a.var = var; a.flags = flags;
    a.bias = calib->bias_scalar; a.sat = calib->sat; a.w = shape.w; a.h = shape.h;
    a.pitch = shape.pitch; a.gain = calib->gain; a.rn2 = calib->read_noise * calib->read_noise;
    const long nv = (shape.pitch / 8) * (long)shape.h;
    long blocks = (nv + 255) / 256;
    const long cap = (long)ctx->num_sms * 8;
    if (blocks > cap) blocks = cap;
    calibrate_kernel<<<(unsigned)blocks, 256, 0, stream>>>(a); argus_count_launch(1);
    return argus_launch_status();
}
