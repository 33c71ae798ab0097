// K9: learned PSF-matching kernel surrogate (the learned part of the system;
// the paper has no counterpart: it names the direct-subtraction and ZOGY
// methods, Sec. 4.2, whose kernels the least-squares fit supplies here).
//
// A small CNN maps a stamp pair (science, reference; 21x21 each, divided by
// the reference stamp sum) to a 21x21 kernel:
//   h1 = W1 x + b1 (1x1, 2 -> 32), h_{l+1} = relu(conv7(h_l) + b_l) for four
//   7x7 'same' 32 -> 32 layers, y = (W6 h5 + b6) / 441 (1x1, 32 -> 1; the fixed
//   1/441 keeps the last layer's values at order one).
// Parameters (200,961) follow the layout W1[32][2], b1, {W[7][7][32 in][32 out],
// b} x 4, W6[32], b6.  Weights are read as BF16 (or FP32) with FP32
// accumulation; activations are FP32, channels last with a padded channel
// stride of 33 in shared memory (conflict-free across pixels).  Training runs
// entirely in these kernels: forward, MSE, data and weight gradients, Adam on
// FP32 master weights with a BF16 working copy.  With ARGUS_PREC_BF16_SPLIT
// the forward and the data gradients of the 7x7 layers run instead on the
// tensor cores (cnn_tc.cu); the weight gradients stay on the CUDA cores.
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>

#include "argus_internal.cuh"

namespace {

constexpr int S = 21, NPX = S * S, C = 32, KS = 7, SP = S + KS - 1;   // padded side 27
constexpr int CS = 33;                                                 // padded channel stride
constexpr int PADSZ = (SP * SP * CS + 3) / 4 * 4;                      // keeps what follows 16-byte aligned
constexpr long NPARAM = 64 + 32 + 4L * (49 * 1024 + 32) + 32 + 1;
constexpr long OFF_W1 = 0, OFF_B1 = 64;
__host__ __device__ constexpr long off_w(int l) { return 96 + (long)l * (49 * 1024 + 32); }
__host__ __device__ constexpr long off_b(int l) { return off_w(l) + 49 * 1024; }
constexpr long OFF_W6 = 96 + 4L * (49 * 1024 + 32), OFF_B6 = OFF_W6 + 32;

__device__ __forceinline__ float ld(const float* p, long i) { return p[i]; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p, long i) { return __bfloat162float(p[i]); }

// h1 = W1 x + b1
template <typename WT>
__global__ void cnn_in_kernel(const float* x, const WT* w, float* h1, int n) {
    const long tot = (long)n * NPX * C;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const long q = e / C;
        const int o = (int)(e - q * C);
        h1[e] = ld(w, OFF_B1 + o) + ld(w, OFF_W1 + o * 2) * x[q * 2] + ld(w, OFF_W1 + o * 2 + 1) * x[q * 2 + 1];
    }
}

// Stage one image's [21][21][32] activations into a zero-padded [27][27][33] tile.
__device__ __forceinline__ void stage_padded(const float* src, float* pad, const float* relu_mask) {
    for (int e = threadIdx.x; e < SP * SP * CS; e += blockDim.x) pad[e] = 0.0f;
    __syncthreads();
    for (int e = threadIdx.x; e < NPX * C; e += blockDim.x) {
        const int p = e / C, c = e - p * C;
        const int y = p / S, x = p - y * S;
        float v = src[e];
        if (relu_mask && !(relu_mask[e] > 0.0f)) v = 0.0f;
        pad[((y + 3) * SP + (x + 3)) * CS + c] = v;
    }
}

// conv7 forward, one CTA per image (grid-stride): thread = 8 output channels x 7 pixels.
// out[y][x][o] = relu(b[o] + sum_{ky,kx,i} W[ky][kx][i][o] in[y+ky-3][x+kx-3][i])
template <typename WT>
__global__ void __launch_bounds__(256) cnn_conv7_fwd_kernel(const float* hin, const WT* w, const WT* b, float* hout,
                                                            int n) {
    extern __shared__ __align__(16) float sm[];
    float* pad = sm;                                 // [SP*SP*CS]
    float* ws = pad + PADSZ;                  // [7 kx][32 i][32 o] one kernel row
    const int oct = threadIdx.x & 3, pg = threadIdx.x >> 2;
    for (int img = blockIdx.x; img < n; img += gridDim.x) {
        __syncthreads();
        stage_padded(hin + (long)img * NPX * C, pad, nullptr);
        float acc[7][8];
#pragma unroll
        for (int j = 0; j < 7; j++)
#pragma unroll
            for (int o = 0; o < 8; o++) acc[j][o] = 0.0f;
        int py[7], px[7];
#pragma unroll
        for (int j = 0; j < 7; j++) {
            const int p = min(pg + 64 * j, NPX - 1);
            py[j] = p / S;
            px[j] = p - py[j] * S;
        }
        for (int ky = 0; ky < KS; ky++) {
            __syncthreads();
            for (int e = threadIdx.x; e < KS * C * C; e += blockDim.x) ws[e] = ld(w, (long)ky * KS * C * C + e);
            __syncthreads();
            for (int kx = 0; kx < KS; kx++) {
                int base[7];
#pragma unroll
                for (int j = 0; j < 7; j++) base[j] = ((py[j] + ky) * SP + (px[j] + kx)) * CS;
                const float* wk = ws + kx * C * C + oct * 8;
#pragma unroll 4
                for (int i = 0; i < C; i++) {
                    const float4 w0 = *reinterpret_cast<const float4*>(wk + i * C);
                    const float4 w1 = *reinterpret_cast<const float4*>(wk + i * C + 4);
                    const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                    for (int j = 0; j < 7; j++) {
                        const float v = pad[base[j] + i];
#pragma unroll
                        for (int o = 0; o < 8; o++) acc[j][o] = fmaf(wv[o], v, acc[j][o]);
                    }
                }
            }
        }
        float bo[8];
#pragma unroll
        for (int o = 0; o < 8; o++) bo[o] = ld(b, oct * 8 + o);
        float* dst = hout + (long)img * NPX * C;
#pragma unroll
        for (int j = 0; j < 7; j++) {
            const int p = pg + 64 * j;
            if (p >= NPX) break;
#pragma unroll
            for (int o = 0; o < 8; o++) dst[p * C + oct * 8 + o] = fmaxf(acc[j][o] + bo[o], 0.0f);
        }
    }
}

template <typename WT>
__global__ void cnn_out_kernel(const float* h5, const WT* w, float* y, int n) {
    const long tot = (long)n * NPX;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < tot; q += (long)gridDim.x * blockDim.x) {
        float s = ld(w, OFF_B6);
        const float* h = h5 + q * C;
#pragma unroll
        for (int i = 0; i < C; i++) s = fmaf(ld(w, OFF_W6 + i), h[i], s);
        y[q] = s * (1.0f / NPX);
    }
}

// loss = mean (y - t)^2 (accumulated in FP64), dy = 2 (y - t) / n_total; each block
// writes its partial sum to part[blockIdx.x] (reduced in a fixed order afterwards)
__global__ void __launch_bounds__(256) cnn_mse_kernel(const float* y, const float* t, long n, float* dy,
                                                      double* part) {
    __shared__ double red[8];
    double s = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        s += (double)d * d;
        if (dy) dy[i] = 2.0f * d / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w8 = 0; w8 < (int)(blockDim.x >> 5); w8++) v += red[w8];
        part[blockIdx.x] = v / (double)n;
    }
}

__global__ void cnn_sum_d_kernel(const double* part, int nb, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double v = 0.0;
        for (int b = 0; b < nb; b++) v += part[b];
        *out = v;
    }
}

// dst[e] = sum over b < nb of part[b * width + e], in the order of b (the per-CTA
// partial gradients reduced without atomics, so training is bit-reproducible)
__global__ void cnn_reduce_kernel(const float* part, int nb, long width, float* dst) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < width; e += (long)gridDim.x * blockDim.x) {
        float v = 0.0f;
        for (int b = 0; b < nb; b++) v += part[(long)b * width + e];
        dst[e] = v;
    }
}

// dh5 = W6 dy; grad W6 += sum dy h5; grad b6 += sum dy
template <typename WT>
__global__ void __launch_bounds__(256) cnn_out_bwd_kernel(const float* h5, const float* dy, const WT* w, float* dh5,
                                                          float* part, int n) {
    __shared__ float red[8][C + 1];
    float gw[C + 1];
#pragma unroll
    for (int c = 0; c <= C; c++) gw[c] = 0.0f;
    const long tot = (long)n * NPX;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < tot; q += (long)gridDim.x * blockDim.x) {
        const float d = dy[q] * (1.0f / NPX);
#pragma unroll
        for (int c = 0; c < C; c++) {
            gw[c] = fmaf(d, h5[q * C + c], gw[c]);
            dh5[q * C + c] = ld(w, OFF_W6 + c) * d;
        }
        gw[C] += d;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c <= C; c++) {
        float v = gw[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][c] = v;
    }
    __syncthreads();
    if (threadIdx.x <= C) {   // this block's (W6, b6) partial: part[blockIdx.x][C + 1]
        float v = 0.0f;
        for (int w8 = 0; w8 < (int)(blockDim.x >> 5); w8++) v += red[w8][threadIdx.x];
        part[(long)blockIdx.x * (C + 1) + threadIdx.x] = v;
    }
}

// data gradient of a conv7 layer: dz = dh_out * (h_out > 0);
// dh_in[y][x][i] = sum_{ky,kx,o} W[ky][kx][i][o] dz[y-ky+3][x-kx+3][o]
template <typename WT>
__global__ void __launch_bounds__(256) cnn_conv7_dgrad_kernel(const float* dh_out, const float* h_out, const WT* w,
                                                              float* dh_in, int n) {
    extern __shared__ __align__(16) float sm[];
    float* pad = sm;                                 // dz, zero padded
    float* ws = pad + PADSZ;                  // [7 kx][32 o][32 i] (transposed)
    const int oct = threadIdx.x & 3, pg = threadIdx.x >> 2;
    for (int img = blockIdx.x; img < n; img += gridDim.x) {
        __syncthreads();
        stage_padded(dh_out + (long)img * NPX * C, pad, h_out + (long)img * NPX * C);
        float acc[7][8];
#pragma unroll
        for (int j = 0; j < 7; j++)
#pragma unroll
            for (int o = 0; o < 8; o++) acc[j][o] = 0.0f;
        int py[7], px[7];
#pragma unroll
        for (int j = 0; j < 7; j++) {
            const int p = min(pg + 64 * j, NPX - 1);
            py[j] = p / S;
            px[j] = p - py[j] * S;
        }
        for (int ky = 0; ky < KS; ky++) {
            __syncthreads();
            for (int e = threadIdx.x; e < KS * C * C; e += blockDim.x) {
                const int kx = e / (C * C), r = e - kx * C * C, o = r / C, i = r - o * C;
                ws[e] = ld(w, ((long)(ky * KS + kx) * C + i) * C + o);
            }
            __syncthreads();
            for (int kx = 0; kx < KS; kx++) {
                int base[7];
#pragma unroll
                for (int j = 0; j < 7; j++) base[j] = ((py[j] - ky + 6) * SP + (px[j] - kx + 6)) * CS;
                const float* wk = ws + kx * C * C + oct * 8;
#pragma unroll 4
                for (int o = 0; o < C; o++) {
                    const float4 w0 = *reinterpret_cast<const float4*>(wk + o * C);
                    const float4 w1 = *reinterpret_cast<const float4*>(wk + o * C + 4);
                    const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                    for (int j = 0; j < 7; j++) {
                        const float v = pad[base[j] + o];
#pragma unroll
                        for (int q = 0; q < 8; q++) acc[j][q] = fmaf(wv[q], v, acc[j][q]);
                    }
                }
            }
        }
        float* dst = dh_in + (long)img * NPX * C;
#pragma unroll
        for (int j = 0; j < 7; j++) {
            const int p = pg + 64 * j;
            if (p >= NPX) break;
#pragma unroll
            for (int q = 0; q < 8; q++) dst[p * C + oct * 8 + q] = acc[j][q];
        }
    }
}

// weight gradient of a conv7 layer for one kernel row ky (blockIdx.y):
// dW[ky][kx][i][o] = sum_{img,y,x} in[y+ky-3][x+kx-3][i] dz[y][x][o], db[o] = sum dz[o].
// 448 threads: (kx, 4 input channels, 4 output channels) each; images in chunks per CTA.
// Each CTA (chunk bx of images, kernel row ky) writes its sums to its own partial slot
// part[bx][ky * KS * C * C .. + KS * C * C) (and the bias partial at [bx][49 C C ..] for
// ky = 0); the slots are reduced in a fixed order afterwards.
constexpr long WPART = 49L * 1024 + 32;   // one layer's weights and biases
__global__ void __launch_bounds__(448) cnn_conv7_wgrad_kernel(const float* hin, const float* dh_out,
                                                              const float* h_out, float* part, int n,
                                                              int per_cta) {
    extern __shared__ __align__(16) float sm[];
    float* pad = sm;                                 // input, zero padded
    float* dz = pad + PADSZ;                  // [441][CS]
    const int ky = blockIdx.y;
    const int t = threadIdx.x;
    const int kx = t / 64, r = t - kx * 64, i4 = r & 7, o4 = r >> 3;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[a][c] = 0.0f;
    float accb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int i0 = blockIdx.x * per_cta, i1 = min(n, i0 + per_cta);
    for (int img = i0; img < i1; img++) {
        __syncthreads();
        stage_padded(hin + (long)img * NPX * C, pad, nullptr);
        for (int e = threadIdx.x; e < NPX * C; e += blockDim.x) {
            const int p = e / C, c = e - p * C;
            const float hv = h_out[(long)img * NPX * C + e];
            dz[p * CS + c] = hv > 0.0f ? dh_out[(long)img * NPX * C + e] : 0.0f;
        }
        __syncthreads();
        if (kx < KS) {
            for (int p = 0; p < NPX; p++) {
                const int y = p / S, x = p - y * S;
                const float* hi = pad + ((y + ky) * SP + (x + kx)) * CS + i4 * 4;
                const float* dd = dz + p * CS + o4 * 4;
                float hv[4], dv[4];
#pragma unroll
                for (int a = 0; a < 4; a++) { hv[a] = hi[a]; dv[a] = dd[a]; }
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[a][c] = fmaf(hv[a], dv[c], acc[a][c]);
                if (ky == 0 && kx == 0 && i4 == 0)
#pragma unroll
                    for (int c = 0; c < 4; c++) accb[c] += dv[c];
            }
        }
    }
    if (kx < KS) {
        float* gW = part + (long)blockIdx.x * WPART;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 4; c++)
                gW[((long)(ky * KS + kx) * C + i4 * 4 + a) * C + o4 * 4 + c] = acc[a][c];
        if (ky == 0 && kx == 0 && i4 == 0)
#pragma unroll
            for (int c = 0; c < 4; c++) gW[49L * 1024 + o4 * 4 + c] = accb[c];
    }
}

// layer 1 (linear): grad W1[o][j] += sum x[q][j] dh1[q][o], grad b1[o] += sum dh1[q][o]
__global__ void __launch_bounds__(256) cnn_in_bwd_kernel(const float* x, const float* dh1, float* part, int n) {
    __shared__ float red[8][3 * C];
    float g[3 * C];
#pragma unroll
    for (int k = 0; k < 3 * C; k++) g[k] = 0.0f;
    const long tot = (long)n * NPX;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < tot; q += (long)gridDim.x * blockDim.x) {
        const float x0 = x[q * 2], x1 = x[q * 2 + 1];
#pragma unroll
        for (int o = 0; o < C; o++) {
            const float d = dh1[q * C + o];
            g[o * 2] = fmaf(x0, d, g[o * 2]);
            g[o * 2 + 1] = fmaf(x1, d, g[o * 2 + 1]);
            g[2 * C + o] += d;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3 * C; k++) {
        float v = g[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3 * C) {   // this block's (W1, b1) partial: part[blockIdx.x][3 C]
        float v = 0.0f;
        for (int w8 = 0; w8 < (int)(blockDim.x >> 5); w8++) v += red[w8][threadIdx.x];
        part[(long)blockIdx.x * 3 * C + threadIdx.x] = v;
    }
}

// Adam (Kingma & Ba 2015) on FP32 master weights; refreshes the BF16 working copy.
__global__ void cnn_adam_kernel(float* master, __nv_bfloat16* wbf, float* m, float* v, const float* g, long n,
                                float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float p = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        master[i] = p;
        wbf[i] = __float2bfloat16(p);
    }
}

__global__ void cnn_to_bf16_kernel(const float* src, __nv_bfloat16* dst, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16(src[i]);
}

// He-normal initialisation from a counter-based hash (SplitMix64 -> two uniforms -> Box-Muller).
__device__ __forceinline__ unsigned long long splitmix(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void cnn_init_kernel(float* p, long n, unsigned long long seed) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float fan_in = 1.0f;
        bool bias = false;
        if (i < OFF_B1) fan_in = 2.0f;
        else if (i < off_w(0)) bias = true;
        else if (i < OFF_W6) {
            const long r = (i - off_w(0)) % (49 * 1024 + 32);
            if (r >= 49 * 1024) bias = true;
            else fan_in = 49.0f * C;
        } else if (i < OFF_B6) fan_in = C;
        else bias = true;
        if (bias) {
            p[i] = 0.0f;
            continue;
        }
        const unsigned long long h1 = splitmix(seed * 0x100000001b3ull + 2 * (unsigned long long)i);
        const unsigned long long h2 = splitmix(seed * 0x100000001b3ull + 2 * (unsigned long long)i + 1);
        const double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
        const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        p[i] = (float)(z * sqrt(2.0 / fan_in));
    }
    // the output starts near the mean kernel (1/441 per pixel)
    if (blockIdx.x == 0 && threadIdx.x == 0) p[OFF_B6] = 1.0f;
}

// Network inputs from stamps: x[s][p][0] = I / sum(R), x[s][p][1] = R / sum(R) over the
// 21x21 window centred on centers[s] (one CTA per stamp).
// Block-wide sum (blockDim a multiple of 32, at most 256 threads); every thread gets the total.
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
    return t;
}

__global__ void __launch_bounds__(256) cnn_prepare_kernel(const float* sci, const float* ref, long pitch, int w,
                                                          int h, const int* centers, const int* n_stamps,
                                                          int max_stamps, float* x) {
    __shared__ float red[8];
    const int s = blockIdx.x;
    if (s >= min(*n_stamps, max_stamps)) return;
    const int xs = centers[2 * s], ys = centers[2 * s + 1];
    // sky of each stamp: mean of its border ring (the outermost pixels); the
    // inputs are the sky-subtracted stamps over the sky-subtracted reference flux
    __shared__ float sky[2];
    float ps = 0.0f, pr = 0.0f;
    for (int p = threadIdx.x; p < NPX; p += blockDim.x) {
        const int py = p / S, px = p % S;
        const int yy = ys - S / 2 + py, xx = xs - S / 2 + px;
        if ((px == 0 || px == S - 1 || py == 0 || py == S - 1) && xx >= 0 && yy >= 0 && xx < w && yy < h) {
            ps += sci[(long)yy * pitch + xx];
            pr += ref[(long)yy * pitch + xx];
        }
    }
    ps = block_sum(ps, red);
    pr = block_sum(pr, red);
    if (threadIdx.x == 0) {
        sky[0] = ps / (float)(4 * S - 4);
        sky[1] = pr / (float)(4 * S - 4);
    }
    __syncthreads();
    float part = 0.0f;
    for (int p = threadIdx.x; p < NPX; p += blockDim.x) {
        const int yy = ys - S / 2 + p / S, xx = xs - S / 2 + p % S;
        if (xx >= 0 && yy >= 0 && xx < w && yy < h) part += ref[(long)yy * pitch + xx] - sky[1];
    }
    const float tot = block_sum(part, red);
    const float inv = tot > 0.0f ? 1.0f / tot : 0.0f;
    for (int p = threadIdx.x; p < NPX; p += blockDim.x) {
        const int yy = ys - S / 2 + p / S, xx = xs - S / 2 + p % S;
        float a = 0.0f, b = 0.0f;
        if (xx >= 0 && yy >= 0 && xx < w && yy < h) {
            a = (sci[(long)yy * pitch + xx] - sky[0]) * inv;
            b = (ref[(long)yy * pitch + xx] - sky[1]) * inv;
        }
        x[((long)s * NPX + p) * 2] = a;
        x[((long)s * NPX + p) * 2 + 1] = b;
    }
}

// Spatial least squares across stamps (one CTA): the kernel at stamp s is
// y_s(u,v) = sum_k p_k(x_s, y_s) K_k(u,v); with A = sum_s p p^T (FP64) every
// kernel pixel solves A K(u,v) = sum_s p y_s(u,v).  The stamps' terms are
// computed once into shared memory; the right-hand sides (sums of at most a
// few thousand products of terms <= 1 with kernel values) accumulate in FP32,
// A, its Cholesky factor and the per-pixel solves are FP64.
__global__ void __launch_bounds__(512) learned_spatial_kernel(const float* y, const int* centers, const int* n_stamps,
                                                              int max_stamps, int W, int H, int sdeg, float* K,
                                                              int* status) {
    extern __shared__ float pk_s[];          // [max_stamps][6]
    __shared__ double A[6][6], Lc[6][6];
    __shared__ int bad;
    const int ns = min(*n_stamps, max_stamps);
    const int nk = (sdeg + 1) * (sdeg + 2) / 2;
    if (threadIdx.x == 0) bad = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const double xt = W > 1 ? (2.0 * centers[2 * s] - (W - 1)) / (double)(W - 1) : 0.0;
        const double yt = H > 1 ? (2.0 * centers[2 * s + 1] - (H - 1)) / (double)(H - 1) : 0.0;
        int k = 0;
        double xi = 1.0;
        for (int i = 0; i <= sdeg; i++) {
            double yj = 1.0;
            for (int j = 0; j <= sdeg - i; j++) {
                pk_s[s * 6 + k++] = (float)(xi * yj);
                yj *= yt;
            }
            xi *= xt;
        }
    }
    __syncthreads();
    if (threadIdx.x < nk * nk) {
        const int a = threadIdx.x / nk, b = threadIdx.x % nk;
        double acc = 0.0;
        for (int t = 0; t < ns; t++) acc += (double)pk_s[t * 6 + a] * (double)pk_s[t * 6 + b];
        A[a][b] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < nk; j++) {
            double d = A[j][j];
            for (int k = 0; k < j; k++) d -= Lc[j][k] * Lc[j][k];
            if (!(d > 0.0)) { bad = 1; break; }
            Lc[j][j] = sqrt(d);
            for (int i = j + 1; i < nk; i++) {
                double v = A[i][j];
                for (int k = 0; k < j; k++) v -= Lc[i][k] * Lc[j][k];
                Lc[i][j] = v / Lc[j][j];
            }
        }
        if (bad) argus_latch(status, ARGUS_ERR_SINGULAR);
    }
    __syncthreads();
    if (bad) return;
    for (int p = threadIdx.x; p < NPX; p += blockDim.x) {
        float rhs[6] = {0, 0, 0, 0, 0, 0};
        for (int s = 0; s < ns; s++) {
            const float v = y[(long)s * NPX + p];
#pragma unroll
            for (int k = 0; k < 6; k++) rhs[k] = fmaf(pk_s[s * 6 + k], v, rhs[k]);
        }
        double z[6], sol[6];
        for (int i = 0; i < nk; i++) {
            double v = rhs[i];
            for (int k = 0; k < i; k++) v -= Lc[i][k] * z[k];
            z[i] = v / Lc[i][i];
        }
        for (int i = nk - 1; i >= 0; i--) {
            double v = z[i];
            for (int k = i + 1; k < nk; k++) v -= Lc[k][i] * sol[k];
            sol[i] = v / Lc[i][i];
        }
        for (int k = 0; k < nk; k++) K[(long)k * NPX + p] = (float)sol[k];
    }
}

// p_k = xt^i yt^j, i + j <= deg, ordered i then j
__device__ __forceinline__ void terms_d(double xt, double yt, int deg, double* out) {
    int k = 0;
    double xi = 1.0;
    for (int i = 0; i <= deg; i++) {
        double yj = 1.0;
        for (int j = 0; j <= deg - i; j++) {
            out[k++] = xi * yj;
            yj *= yt;
        }
        xi *= xt;
    }
}

// Least squares on the stamp pixels given the kernel K_k, with c_k = R (x) K_k:
//   background only:     min sum w (I - sum_k p_k c_k - sum_j pb_j bg_j)^2 over bg;
//   scales + background: min sum w (I - sum_k alpha_k p_k c_k - sum_j pb_j bg_j)^2 over
//                        alpha and bg, and K_k <- alpha_k K_k.
// Pass 1 (grid over stamps): per-stamp partial normal equations, layout
// [A 12x12][rhs 12][t'Wt][n_pix]; the model convolution in FP32, the sums in FP64.
constexpr int BGN = 12, BGP = BGN * BGN + BGN + 2;

__global__ void __launch_bounds__(256) learned_bg_partial_kernel(const float* sci, const float* var, const float* ref,
                                                                 const uint8_t* flags, long pitch, int w, int h,
                                                                 const int* centers, const int* n_stamps,
                                                                 int max_stamps, int stamp, const float* K, int ksz,
                                                                 int sdeg, int bgdeg, int scale, double* part) {
    // shared: the nk kernels and the stamp's reference window (stamp + 2r)^2
    extern __shared__ float bsm[];
    __shared__ double red[8][BGP];
    const int s = blockIdx.x;
    const int nk = (sdeg + 1) * (sdeg + 2) / 2, nb = (bgdeg + 1) * (bgdeg + 2) / 2, kk = ksz * ksz, r = ksz / 2;
    const int n = scale ? nk + nb : nb;
    const int ww = stamp + 2 * r;
    float* Ks = bsm;
    float* Rw = bsm + nk * kk;
    double* out = part + (long)s * BGP;
    const bool live = s < min(*n_stamps, max_stamps);
    const int xs = live ? centers[2 * s] : 0, ys = live ? centers[2 * s + 1] : 0, hs = stamp / 2;
    const bool ok = live && xs - hs - r >= 0 && xs + hs + r <= w - 1 && ys - hs - r >= 0 && ys + hs + r <= h - 1;
    for (int e = threadIdx.x; e < nk * kk; e += blockDim.x) Ks[e] = K[e];
    for (int e = threadIdx.x; ok && e < ww * ww; e += blockDim.x) {
        const int jy = e / ww, jx = e - jy * ww;
        Rw[e] = ref[(long)(ys - hs - r + jy) * pitch + (xs - hs - r + jx)];
    }
    __syncthreads();
    double acc[BGP];
    for (int k = 0; k < BGP; k++) acc[k] = 0.0;
    for (int p = threadIdx.x; ok && p < stamp * stamp; p += blockDim.x) {
        const int px = p % stamp, py = p / stamp;
        const int x = xs - hs + px, y = ys - hs + py;
        const long q = (long)y * pitch + x;
        const float v = var[q], I = sci[q];
        if (flags[q] || !(v > 0.0f) || !isfinite(v) || !isfinite(I)) continue;
        const double wt = 1.0 / (double)v;
        const double xt = w > 1 ? (2.0 * x - (w - 1)) / (double)(w - 1) : 0.0;
        const double yt = h > 1 ? (2.0 * y - (h - 1)) / (double)(h - 1) : 0.0;
        double pk[6], pb[6], z[BGN];
        terms_d(xt, yt, sdeg, pk);
        terms_d(xt, yt, bgdeg, pb);
        double conv = 0.0;
        for (int k2 = 0; k2 < nk; k2++) {
            // R(x - (iu - r), y - (iv - r)) = Rw[py + 2r - iv][px + 2r - iu]
            float c = 0.0f;
            for (int iv = 0; iv < ksz; iv++) {
                const float* kr = Ks + k2 * kk + iv * ksz;
                const float* rr = Rw + (py + 2 * r - iv) * ww + px + 2 * r;
                for (int iu = 0; iu < ksz; iu++) c = fmaf(kr[iu], rr[-iu], c);
            }
            if (scale) z[k2] = pk[k2] * (double)c;
            conv += pk[k2] * (double)c;
        }
        for (int j = 0; j < nb; j++) z[(scale ? nk : 0) + j] = pb[j];
        const double t = scale ? (double)I : (double)I - conv;
        for (int a2 = 0; a2 < n; a2++) {
            const double wz = wt * z[a2];
            for (int b2 = 0; b2 < n; b2++) acc[a2 * BGN + b2] += wz * z[b2];
            acc[BGN * BGN + a2] += wz * t;
        }
        acc[BGN * BGN + BGN] += wt * t * t;
        acc[BGN * BGN + BGN + 1] += 1.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < BGP; k++) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < BGP; k += blockDim.x) {
        double v = 0.0;
        for (int w8 = 0; w8 < (int)(blockDim.x >> 5); w8++) v += red[w8][k];
        out[k] = v;
    }
}

// Pass 2 (one CTA): sum the partials, Cholesky solve of the n x n system
// (FP64), chi2 = t'Wt - 2 sol'rhs + sol'A sol, stats; with scale, K_k <- alpha_k K_k.
__global__ void __launch_bounds__(256) learned_bg_solve_kernel(const double* part, int max_stamps, int sdeg, int bgdeg,
                                                              int scale, float* K, int kk, double* bg,
                                                              argus_fit_stats* st, int* status) {
    __shared__ double T[BGP];
    __shared__ double alpha[6];
    __shared__ int bad_s;
    for (int k = threadIdx.x; k < BGP; k += blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < max_stamps; s++) v += part[(long)s * BGP + k];
        T[k] = v;
    }
    const int nk = (sdeg + 1) * (sdeg + 2) / 2, nb = (bgdeg + 1) * (bgdeg + 2) / 2;
    const int n = scale ? nk + nb : nb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double L[BGN][BGN], z[BGN], sol[BGN];
        bool bad = false;
        for (int j = 0; j < n && !bad; j++) {
            double d = T[j * BGN + j];
            for (int k = 0; k < j; k++) d -= L[j][k] * L[j][k];
            if (!(d > 0.0)) { bad = true; break; }
            L[j][j] = sqrt(d);
            for (int i = j + 1; i < n; i++) {
                double v = T[i * BGN + j];
                for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
                L[i][j] = v / L[j][j];
            }
        }
        argus_fit_stats o;
        o.chi2_a0 = 0.0; o.max_step = 0.0; o.refine_iters = 0; o.pad_ = 0; o.precision = -1; o.n_stamps_used = 0;
        o.n_coeffs = n;
        o.n_pix = (long long)T[BGN * BGN + BGN + 1];
        o.dof = o.n_pix - n;
        bad_s = bad ? 1 : 0;
        if (bad) {
            argus_latch(status, ARGUS_ERR_SINGULAR);
            o.status = ARGUS_ERR_SINGULAR;
            o.chi2 = 0.0;
            *st = o;
        } else {
            for (int i = 0; i < n; i++) {
                double v = T[BGN * BGN + i];
                for (int k = 0; k < i; k++) v -= L[i][k] * z[k];
                z[i] = v / L[i][i];
            }
            for (int i = n - 1; i >= 0; i--) {
                double v = z[i];
                for (int k = i + 1; k < n; k++) v -= L[k][i] * sol[k];
                sol[i] = v / L[i][i];
            }
            double chi2 = T[BGN * BGN + BGN];
            for (int i = 0; i < n; i++) {
                chi2 -= 2.0 * sol[i] * T[BGN * BGN + i];
                for (int j = 0; j < n; j++) chi2 += sol[i] * T[i * BGN + j] * sol[j];
            }
            for (int j = 0; j < nb; j++) bg[j] = sol[(scale ? nk : 0) + j];
            for (int k = 0; k < nk; k++) alpha[k] = scale ? sol[k] : 1.0;
            o.chi2 = chi2;
            o.status = ARGUS_OK;
            *st = o;
        }
    }
    __syncthreads();
    if (scale && !bad_s)
        for (int e = threadIdx.x; e < nk * kk; e += blockDim.x) K[e] = (float)(alpha[e / kk] * (double)K[e]);
}

}  // namespace

struct argus_cnn {
    int device, num_sms, max_batch, precision;
    float* master;          // [NPARAM] FP32
    __nv_bfloat16* wbf;     // [NPARAM] BF16 working copy
    float *m, *v, *grad;    // Adam moments and gradient
    float* acts;            // [5][max_batch][441][32] post-activation h1..h5
    float *dh0, *dh1;       // [max_batch][441][32] gradient ping-pong
    float* dy;              // [max_batch][441]
    float* y;               // [max_batch][441]
    double* loss;           // [1]
    float* part;            // per-CTA partial gradients: [num_sms][WPART] (a layer at a time)
    double* lpart;          // per-block partial losses [num_sms * 2]
    void* wpack;            // the 7x7 weights in the tensor-core operand layout
    int* d_status;          // latched device status word
    int step;
};

static size_t fwd_smem() { return sizeof(float) * ((size_t)PADSZ + (size_t)KS * C * C); }
static size_t wgrad_smem() { return sizeof(float) * ((size_t)PADSZ + (size_t)NPX * CS); }

extern "C" int argus_cnn_create(argus_cnn** out, int device, int max_batch, unsigned long long seed) {
    if (!out || max_batch < 1) return ARGUS_ERR_ARG;
    *out = NULL;
    if (cudaSetDevice(device) != cudaSuccess) return ARGUS_ERR_CUDA;
    argus_cnn* n = (argus_cnn*)calloc(1, sizeof(argus_cnn));
    if (!n) return ARGUS_ERR_NOMEM;
    n->device = device;
    n->max_batch = max_batch;
    n->precision = ARGUS_PREC_BF16;
    cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, device);
    const size_t L = (size_t)max_batch * NPX * C;
    bool ok = cudaMalloc(&n->master, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&n->wbf, sizeof(__nv_bfloat16) * NPARAM) == cudaSuccess &&
              cudaMalloc(&n->m, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&n->v, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&n->grad, sizeof(float) * NPARAM) == cudaSuccess &&
              cudaMalloc(&n->acts, sizeof(float) * 5 * L) == cudaSuccess &&
              cudaMalloc(&n->dh0, sizeof(float) * L) == cudaSuccess &&
              cudaMalloc(&n->dh1, sizeof(float) * L) == cudaSuccess &&
              cudaMalloc(&n->dy, sizeof(float) * (size_t)max_batch * NPX) == cudaSuccess &&
              cudaMalloc(&n->y, sizeof(float) * (size_t)max_batch * NPX) == cudaSuccess &&
              cudaMalloc(&n->loss, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&n->part, sizeof(float) * (size_t)n->num_sms * (size_t)WPART) == cudaSuccess &&
              cudaMalloc(&n->lpart, sizeof(double) * (size_t)n->num_sms * 2) == cudaSuccess &&
              cudaMalloc(&n->wpack, argus_cnn_tc_pack_bytes()) == cudaSuccess &&
              cudaMalloc(&n->d_status, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        argus_cnn_destroy(n);
        return ARGUS_ERR_NOMEM;
    }
    cudaMemset(n->d_status, 0, sizeof(int));
    cudaMemset(n->m, 0, sizeof(float) * NPARAM);
    cudaMemset(n->v, 0, sizeof(float) * NPARAM);
    cnn_init_kernel<<<n->num_sms * 4, 256>>>(n->master, NPARAM, seed); argus_count_launch(1);
    cnn_to_bf16_kernel<<<n->num_sms * 4, 256>>>(n->master, n->wbf, NPARAM); argus_count_launch(1);
    cudaFuncSetAttribute(cnn_conv7_fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    cudaFuncSetAttribute(cnn_conv7_fwd_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fwd_smem());
    cudaFuncSetAttribute(cnn_conv7_dgrad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem());
    cudaFuncSetAttribute(cnn_conv7_dgrad_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fwd_smem());
    cudaFuncSetAttribute(cnn_conv7_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem());
    if (cudaDeviceSynchronize() != cudaSuccess) {
        argus_cnn_destroy(n);
        return ARGUS_ERR_CUDA;
    }
    *out = n;
    return ARGUS_OK;
}

extern "C" int argus_cnn_destroy(argus_cnn* n) {
    if (!n) return ARGUS_ERR_ARG;
    cudaSetDevice(n->device);
    void* ps[] = {n->master, n->wbf, n->m, n->v, n->grad, n->acts, n->dh0, n->dh1, n->dy, n->y, n->loss, n->part,
                  n->lpart, n->wpack, n->d_status};
    for (void* p : ps)
        if (p) cudaFree(p);
    free(n);
    return ARGUS_OK;
}

extern "C" int argus_cnn_params(argus_cnn* n, float** master, float** adam_m, float** adam_v, long* count,
                                int* step) {
    if (!n) return ARGUS_ERR_ARG;
    if (master) *master = n->master;
    if (adam_m) *adam_m = n->m;
    if (adam_v) *adam_v = n->v;
    if (count) *count = NPARAM;
    if (step) *step = n->step;
    return ARGUS_OK;
}

extern "C" int argus_cnn_set_state(argus_cnn* n, int precision, int step, argus_stream stream) {
    if (!n || (precision != ARGUS_PREC_FP32 && precision != ARGUS_PREC_BF16 && precision != ARGUS_PREC_BF16_SPLIT) ||
        step < 0)
        return ARGUS_ERR_ARG;
    if (cudaSetDevice(n->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    n->precision = precision;
    n->step = step;
    cnn_to_bf16_kernel<<<n->num_sms * 4, 256, 0, (cudaStream_t)stream>>>(n->master, n->wbf, NPARAM); argus_count_launch(1);
    return argus_launch_status();
}

template <typename WT>
static void forward_impl(argus_cnn* nn, const WT* w, const float* x, int n, float* y, cudaStream_t st) {
    const size_t L = (size_t)nn->max_batch * NPX * C;
    const int g = nn->num_sms * 4;
    cnn_in_kernel<WT><<<g, 256, 0, st>>>(x, w, nn->acts, n); argus_count_launch(1);
    for (int l = 0; l < 4; l++) {
        cnn_conv7_fwd_kernel<WT><<<min(n, nn->num_sms * 2), 256, fwd_smem(), st>>>(
            nn->acts + l * L, w + off_w(l), w + off_b(l), nn->acts + (l + 1) * L, n); argus_count_launch(1);
    }
    cnn_out_kernel<WT><<<g, 256, 0, st>>>(nn->acts + 4 * L, w, y, n); argus_count_launch(1);
}

extern "C" int argus_cnn_forward(argus_cnn* nn, const float* x, int n, float* y, argus_stream stream) {
    if (!nn || !x || !y || n < 1 || n > nn->max_batch) return ARGUS_ERR_ARG;
    if (cudaSetDevice(nn->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (nn->precision == ARGUS_PREC_BF16_SPLIT)
        return argus_cnn_forward_tc(x, nn->wbf, nn->wpack, n, y, nn->acts, (long)nn->max_batch * NPX * C, nn->num_sms,
                                    nn->d_status, st);
    if (nn->precision == ARGUS_PREC_BF16) forward_impl<__nv_bfloat16>(nn, nn->wbf, x, n, y, st);
    else forward_impl<float>(nn, nn->master, x, n, y, st);
    return argus_launch_status();
}

extern "C" int argus_cnn_status(argus_cnn* nn, argus_stream stream) {
    if (!nn) return ARGUS_ERR_ARG;
    if (cudaSetDevice(nn->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, nn->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(nn->d_status, 0, sizeof(int), st);
    if (e != cudaSuccess) return argus_cuda_fail(e);
    return h;
}

// tc_dgrad: the data gradients of the 7x7 layers on the tensor cores (ARGUS_PREC_BF16_SPLIT:
// BF16 weights against BF16 hi + lo gradients, FP32-level); otherwise the CUDA-core kernel
template <typename WT>
static int backward_impl(argus_cnn* nn, const WT* w, const float* x, const float* dy, int n, bool tc_dgrad,
                         cudaStream_t st) {
    const size_t L = (size_t)nn->max_batch * NPX * C;
    // every gradient is a fixed-order sum of per-CTA partials (no float atomics): the
    // partial buffer holds num_sms slots of one layer, reused layer by layer in stream order
    const int gs = nn->num_sms;   // grid of the element-wise gradient kernels (<= num_sms slots)
    const int rg = nn->num_sms * 4;
    float* dh = nn->dh0;
    float* dn = nn->dh1;
    cnn_out_bwd_kernel<WT><<<gs, 256, 0, st>>>(nn->acts + 4 * L, dy, w, dh, nn->part, n); argus_count_launch(1);
    cnn_reduce_kernel<<<1, 64, 0, st>>>(nn->part, gs, C + 1, nn->grad + OFF_W6); argus_count_launch(1);
    for (int l = 3; l >= 0; l--) {
        const float* hin = nn->acts + l * L;
        const float* hout = nn->acts + (l + 1) * L;
        int per = (n + nn->num_sms - 1) / nn->num_sms;
        if (per < 1) per = 1;
        const int nbx = (n + per - 1) / per;
        cnn_conv7_wgrad_kernel<<<dim3(nbx, KS), 448, wgrad_smem(), st>>>(hin, dh, hout, nn->part, n, per); argus_count_launch(1);
        cnn_reduce_kernel<<<rg, 256, 0, st>>>(nn->part, nbx, WPART, nn->grad + off_w(l)); argus_count_launch(1);
        if (tc_dgrad) {
            const int rc = argus_cnn_dgrad_tc(dh, hout, nn->wbf, nn->wpack, l, n, dn, nn->num_sms, nn->d_status, st);
            if (rc) return rc;
        } else {
            cnn_conv7_dgrad_kernel<WT><<<min(n, nn->num_sms * 2), 256, fwd_smem(), st>>>(dh, hout, w + off_w(l), dn, n); argus_count_launch(1);
        }
        float* t = dh;
        dh = dn;
        dn = t;
    }
    cnn_in_bwd_kernel<<<gs, 256, 0, st>>>(x, dh, nn->part, n); argus_count_launch(1);
    cnn_reduce_kernel<<<1, 128, 0, st>>>(nn->part, gs, 3 * C, nn->grad + OFF_W1); argus_count_launch(1);
    return ARGUS_OK;
}

extern "C" int argus_cnn_backward(argus_cnn* nn, const float* x, const float* dy, int n, float* grad_out,
                                  argus_stream stream) {
    if (!nn || !x || !dy || n < 1 || n > nn->max_batch) return ARGUS_ERR_ARG;
    if (cudaSetDevice(nn->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int rc = nn->precision != ARGUS_PREC_FP32
                       ? backward_impl<__nv_bfloat16>(nn, nn->wbf, x, dy, n, nn->precision == ARGUS_PREC_BF16_SPLIT, st)
                       : backward_impl<float>(nn, nn->master, x, dy, n, false, st);
    if (rc) return rc;
    if (grad_out && cudaMemcpyAsync(grad_out, nn->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st) !=
                        cudaSuccess)
        return ARGUS_ERR_CUDA;
    return argus_launch_status();
}

extern "C" int argus_cnn_train_step(argus_cnn* nn, const float* x, const float* target, int n, float lr,
                                    double* loss_out, argus_stream stream) {
    if (!nn || !x || !target || n < 1 || n > nn->max_batch || !(lr > 0.0f)) return ARGUS_ERR_ARG;
    if (cudaSetDevice(nn->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = argus_cnn_forward(nn, x, n, nn->y, stream);
    if (rc) return rc;
    double* loss = loss_out ? loss_out : nn->loss;
    cnn_mse_kernel<<<nn->num_sms * 2, 256, 0, st>>>(nn->y, target, (long)n * NPX, nn->dy, nn->lpart); argus_count_launch(1);
    cnn_sum_d_kernel<<<1, 32, 0, st>>>(nn->lpart, nn->num_sms * 2, loss); argus_count_launch(1);
    rc = argus_cnn_backward(nn, x, nn->dy, n, NULL, stream);
    if (rc) return rc;
    nn->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)nn->step), c2 = 1.0f - powf(b2, (float)nn->step);
    cnn_adam_kernel<<<nn->num_sms * 4, 256, 0, st>>>(nn->master, nn->wbf, nn->m, nn->v, nn->grad, NPARAM, lr, b1,
                                                     b2, 1e-8f, c1, c2); argus_count_launch(1);
    return argus_launch_status();
}

extern "C" int argus_cnn_adam(argus_cnn* nn, const float* grad, float lr, argus_stream stream) {
    if (!nn || !grad || !(lr > 0.0f)) return ARGUS_ERR_ARG;
    if (cudaSetDevice(nn->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    nn->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)nn->step), c2 = 1.0f - powf(b2, (float)nn->step);
    cnn_adam_kernel<<<nn->num_sms * 4, 256, 0, (cudaStream_t)stream>>>(nn->master, nn->wbf, nn->m, nn->v, grad, NPARAM,
                                                                       lr, b1, b2, 1e-8f, c1, c2); argus_count_launch(1);
    return argus_launch_status();
}

extern "C" int argus_cnn_prepare(const float* sci, const float* ref, argus_shape shape, const int* centers,
                                 const int* n_stamps, int max_stamps, float* x, argus_stream stream) {
    if (!sci || !ref || !centers || !n_stamps || !x || max_stamps < 1) return ARGUS_ERR_ARG;
    if (shape.w <= 0 || shape.h <= 0 || shape.pitch < shape.w) return ARGUS_ERR_ARG;
    cnn_prepare_kernel<<<max_stamps, 256, 0, (cudaStream_t)stream>>>(sci, ref, shape.pitch, shape.w, shape.h, centers,
                                                                    n_stamps, max_stamps, x); argus_count_launch(1);
    return argus_launch_status();
}

extern "C" int argus_learned_kernel(argus_ctx* ctx, const float* y, const int* centers, const int* n_stamps,
                                    int max_stamps, int frame_w, int frame_h, int spatial_degree, float* K,
                                    argus_stream stream) {
    if (!ctx || !y || !centers || !n_stamps || !K || max_stamps < 1 || spatial_degree < 0 || spatial_degree > 2)
        return ARGUS_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    const size_t psm = sizeof(float) * 6 * (size_t)max_stamps;
    if (psm > 160 * 1024) return ARGUS_ERR_UNSUPPORTED;
    cudaFuncSetAttribute(learned_spatial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    learned_spatial_kernel<<<1, 512, psm, (cudaStream_t)stream>>>(y, centers, n_stamps, max_stamps, frame_w, frame_h,
                                                                  spatial_degree, K, ctx->d_status); argus_count_launch(1);
    return argus_launch_status();
}

static int fit_background_impl(argus_ctx* ctx, const float* sci, const float* sci_var, const float* ref,
                               const uint8_t* flags, argus_shape shape, const int* centers, const int* n_stamps,
                               int max_stamps, int stamp, float* K, int ksize, int spatial_degree, int bg_degree,
                               int scale, double* bg, argus_fit_stats* stats, cudaStream_t st) {
    if (!ctx || !sci || !sci_var || !ref || !flags || !centers || !n_stamps || !K || !bg || !stats) return ARGUS_ERR_ARG;
    if (max_stamps < 1 || (size_t)max_stamps * BGP > (size_t)ctx->resid_parts * (ctx->np_cols + 4) || ksize < 3 ||
        ksize > 31 || !(ksize & 1) || spatial_degree < 0 || spatial_degree > 2 || bg_degree < 0 || bg_degree > 2 ||
        stamp < 1)
        return ARGUS_ERR_ARG;
    int rc = argus_check_shape(shape, ctx->max_pixels);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    double* part = ctx->resid_part;
    const int nk = (spatial_degree + 1) * (spatial_degree + 2) / 2;
    const size_t bsm = sizeof(float) * ((size_t)nk * ksize * ksize + (size_t)(stamp + ksize - 1) * (stamp + ksize - 1));
    if (bsm > 200 * 1024) return ARGUS_ERR_UNSUPPORTED;
    cudaFuncSetAttribute(learned_bg_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
    learned_bg_partial_kernel<<<max_stamps, 256, bsm, st>>>(sci, sci_var, ref, flags, shape.pitch, shape.w, shape.h,
                                                            centers, n_stamps, max_stamps, stamp, K, ksize,
                                                            spatial_degree, bg_degree, scale, part); argus_count_launch(1);
    learned_bg_solve_kernel<<<1, 256, 0, st>>>(part, max_stamps, spatial_degree, bg_degree, scale, K, ksize * ksize,
                                               bg, stats, ctx->d_status); argus_count_launch(1);
    return argus_launch_status();
}

extern "C" int argus_fit_background(argus_ctx* ctx, const float* sci, const float* sci_var, const float* ref,
                                    const uint8_t* flags, argus_shape shape, const int* centers, const int* n_stamps,
                                    int max_stamps, int stamp, const float* K, int ksize, int spatial_degree,
                                    int bg_degree, double* bg, argus_fit_stats* stats, argus_stream stream) {
    return fit_background_impl(ctx, sci, sci_var, ref, flags, shape, centers, n_stamps, max_stamps, stamp,
                               const_cast<float*>(K), ksize, spatial_degree, bg_degree, 0, bg, stats,
                               (cudaStream_t)stream);
}

extern "C" int argus_fit_scale_background(argus_ctx* ctx, const float* sci, const float* sci_var, const float* ref,
                                          const uint8_t* flags, argus_shape shape, const int* centers,
                                          const int* n_stamps, int max_stamps, int stamp, float* K, int ksize,
                                          int spatial_degree, int bg_degree, double* bg, argus_fit_stats* stats,
                                          argus_stream stream) {
    return fit_background_impl(ctx, sci, sci_var, ref, flags, shape, centers, n_stamps, max_stamps, stamp, K, ksize,
                               spatial_degree, bg_degree, 1, bg, stats, (cudaStream_t)stream);
}
