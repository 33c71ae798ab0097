// K7: variance-weighted threshold detection on the difference image (paper
// Sec. 4.2 transient candidates; Table 2 "Source detection").
//
//  1. mask pass (HBM-bound, 16 pixels per thread, 128-bit loads of D, V_D and flags):
//     S = D / sqrt(V_D) in IEEE float, mask bits, and a compact list of the
//     above-threshold pixels (warp-aggregated append); label[p] = p.
//  2. union-find over the list only (8-connectivity, equal sign): lock-free
//     atomicMin linking, the root of a component is its smallest index.
//  3. flatten labels, number the roots, per-component peak key (|S| bits,
//     then lowest (y, x)) and pixel count by atomics.
//  4. deterministic output order (peak y, then peak x): row histogram,
//     exclusive scan, scatter, per-row insertion sort by x.
//  5. one warp per component: Gaussian-windowed centroid and optimal flux.
// Every loop that follows parent links is bounded; an overrun latches
// ARGUS_ERR_TIMEOUT instead of spinning.
#include "argus_internal.cuh"

namespace {

constexpr int MAX_FIND = 1 << 20;

struct DetArgs {
    const float* D;
    const float* V;
    const uint8_t* flags;
    uint8_t* mask;
    int* label;
    int* list;
    int* count;   // [0] listed pixels, [1] components
    unsigned long long* key;
    int* npix;
    int* order;   // [2][cap]
    int* rows;    // [h + 1] histogram / offsets, [h + 1 .. 2h + 2) cursors
    argus_source* out;
    int* n_found;
    int* status;
    long pitch;
    int w, h, cap, out_cap;
    float nsig, psf_sigma;
};

__device__ __forceinline__ uint8_t mask_of(float d, float v, uint8_t f, float nsig, float& s) {
    const bool valid = (f == 0) && (v > 0.0f) && isfinite(d) && isfinite(v);
    if (!valid) {
        s = 0.0f;
        return ARGUS_MASK_INVALID;
    }
    s = d / sqrtf(v);
    return (uint8_t)((s >= nsig ? ARGUS_MASK_POS : 0) | (s <= -nsig ? ARGUS_MASK_NEG : 0));
}

__global__ void __launch_bounds__(256) mask_kernel(DetArgs a) {
    // 16 pixels per thread and step: four 128-bit loads of D and of V_D, one of the flags,
    // one 128-bit store of the mask (rows start on 16-pixel boundaries: pitch % 16 == 0)
    const long vpr = a.pitch >> 4;
    const long nv = vpr * a.h;
    const int lane = threadIdx.x & 31;
    for (long v0 = blockIdx.x * (long)blockDim.x; v0 < nv; v0 += (long)gridDim.x * blockDim.x) {
        const long v = v0 + threadIdx.x;
        int nset = 0;
        long p0 = 0;
        uint8_t m[16];
#pragma unroll
        for (int i = 0; i < 16; i++) m[i] = 0;
        if (v < nv) {
            const long y = v / vpr;
            const int x0 = (int)(v - y * vpr) << 4;
            p0 = y * a.pitch + x0;
            if (x0 < a.w) {
                const uint4 f16 = *reinterpret_cast<const uint4*>(a.flags + p0);
                const uint32_t fw[4] = {f16.x, f16.y, f16.z, f16.w};
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float4 d4 = *reinterpret_cast<const float4*>(a.D + p0 + 4 * k);
                    const float4 v4 = *reinterpret_cast<const float4*>(a.V + p0 + 4 * k);
                    float s;
                    m[4 * k + 0] = mask_of(d4.x, v4.x, (uint8_t)(fw[k] & 0xffu), a.nsig, s);
                    m[4 * k + 1] = mask_of(d4.y, v4.y, (uint8_t)((fw[k] >> 8) & 0xffu), a.nsig, s);
                    m[4 * k + 2] = mask_of(d4.z, v4.z, (uint8_t)((fw[k] >> 16) & 0xffu), a.nsig, s);
                    m[4 * k + 3] = mask_of(d4.w, v4.w, (uint8_t)(fw[k] >> 24), a.nsig, s);
                }
                if (x0 + 16 <= a.w) {
                    uint32_t mw[4];
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        mw[k] = (uint32_t)m[4 * k] | ((uint32_t)m[4 * k + 1] << 8) | ((uint32_t)m[4 * k + 2] << 16) |
                                ((uint32_t)m[4 * k + 3] << 24);
                    *reinterpret_cast<uint4*>(a.mask + p0) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; i++)
                        if (x0 + i < a.w) a.mask[p0 + i] = m[i];
                }
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    if (x0 + i >= a.w) m[i] = 0;
                    nset += (m[i] & 3) ? 1 : 0;
                }
            }
        }
        // warp-aggregated append of the above-threshold pixels
        int incl = nset;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 31 && total) base = atomicAdd(a.count, total);
        base = __shfl_sync(0xffffffffu, base, 31);
        if (nset) {
            int pos = base + incl - nset;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                if (m[i] & 3) {
                    if (pos < a.cap) {
                        a.list[pos] = (int)(p0 + i);
                        a.label[p0 + i] = (int)(p0 + i);
                    } else {
                        argus_latch(a.status, ARGUS_ERR_CAPACITY);
                    }
                    pos++;
                }
            }
        }
    }
}

__device__ __forceinline__ int find_root(const int* label, int p, int* status) {
    for (int it = 0; it < MAX_FIND; it++) {
        const int q = *((volatile const int*)label + p);
        if (q == p) return p;
        p = q;
    }
    argus_latch(status, ARGUS_ERR_TIMEOUT);
    return p;
}

__device__ void unite(int* label, int a, int b, int* status) {
    for (int it = 0; it < MAX_FIND; it++) {
        a = find_root(label, a, status);
        b = find_root(label, b, status);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        const int old = atomicMin(label + a, b);
        if (old == a) return;
        a = old;
    }
    argus_latch(status, ARGUS_ERR_TIMEOUT);
}

__global__ void union_kernel(DetArgs a) {
    if (*a.count > a.cap) return;   // list overflowed: labels incomplete
    const int n = *a.count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = a.list[i];
        const int y = (int)(p / a.pitch), x = (int)(p - (long)y * a.pitch);
        const uint8_t bit = a.mask[p] & 3;
        if (x > 0 && (a.mask[p - 1] & bit)) unite(a.label, p, p - 1, a.status);
        if (y > 0) {
            const int q = (int)(p - a.pitch);
            if (x > 0 && (a.mask[q - 1] & bit)) unite(a.label, p, q - 1, a.status);
            if (a.mask[q] & bit) unite(a.label, p, q, a.status);
            if (x + 1 < a.w && (a.mask[q + 1] & bit)) unite(a.label, p, q + 1, a.status);
        }
    }
}

__global__ void flatten_kernel(DetArgs a) {
    if (*a.count > a.cap) return;   // list overflowed: labels incomplete
    const int n = *a.count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = a.list[i];
        a.label[p] = find_root(a.label, p, a.status);
    }
}

__global__ void roots_kernel(DetArgs a) {
    if (*a.count > a.cap) return;   // list overflowed: labels incomplete
    const int n = *a.count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = a.list[i];
        if (a.label[p] == p) {
            const int c = atomicAdd(a.count + 1, 1);
            a.key[c] = 0ull;
            a.npix[c] = 0;
            a.label[p] = -(c + 1);
        }
    }
}

__global__ void stats_kernel(DetArgs a) {
    if (*a.count > a.cap) return;   // list overflowed: labels incomplete
    const int n = *a.count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = a.list[i];
        int l = a.label[p];
        if (l >= 0) l = a.label[l];
        const int c = -l - 1;
        const float s = a.D[p] / sqrtf(a.V[p]);
        const int y = (int)(p / a.pitch), x = (int)(p - (long)y * a.pitch);
        const unsigned rm = (unsigned)y * (unsigned)a.w + (unsigned)x;   // row-major rank
        const unsigned long long k =
            ((unsigned long long)__float_as_uint(fabsf(s)) << 32) | (unsigned long long)(0xffffffffu - rm);
        atomicMax(a.key + c, k);
        atomicAdd(a.npix + c, 1);
    }
}

__device__ __forceinline__ int peak_rank(unsigned long long k) { return (int)(0xffffffffu - (unsigned)(k & 0xffffffffu)); }

__global__ void row_hist_kernel(DetArgs a) {
    const int nc = a.count[1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
        atomicAdd(a.rows + peak_rank(a.key[c]) / a.w, 1);
}

// exclusive scan of h row counts (single CTA of 1024 threads), cursors = offsets
__global__ void __launch_bounds__(1024) row_scan_kernel(DetArgs a) {
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b = 0; b < a.h; b += 1024) {
        const int i = b + threadIdx.x;
        const int v = i < a.h ? a.rows[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int ws = wsum[lane], wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - ws;
        }
        __syncthreads();
        const int excl = carry + wsum[wid] + incl - v;
        if (i < a.h) {
            a.rows[i] = excl;
            a.rows[a.h + 1 + i] = excl;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.rows[a.h] = carry;
}

__global__ void scatter_kernel(DetArgs a) {
    const int nc = a.count[1];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int y = peak_rank(a.key[c]) / a.w;
        const int pos = atomicAdd(a.rows + a.h + 1 + y, 1);
        a.order[pos] = c;
    }
}

__global__ void row_sort_kernel(DetArgs a) {
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < a.h; y += gridDim.x * blockDim.x) {
        const int b = a.rows[y], e = a.rows[y + 1];
        for (int i = b + 1; i < e; i++) {
            const int c = a.order[i];
            const int r = peak_rank(a.key[c]);
            int j = i - 1;
            while (j >= b && peak_rank(a.key[a.order[j]]) > r) {
                a.order[j + 1] = a.order[j];
                j--;
            }
            a.order[j + 1] = c;
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float pix_gauss(float a, float c, float inv_s2) {
    return 0.5f * (erff((a + 0.5f - c) * inv_s2) - erff((a - 0.5f - c) * inv_s2));
}

__global__ void measure_kernel(DetArgs a) {
    const int nc = a.count[1];
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int fw = (int)ceilf(3.0f * a.psf_sigma);
    const int side = 2 * fw + 1;
    const float inv2s2 = 1.0f / (2.0f * a.psf_sigma * a.psf_sigma);
    const float inv_s2 = 1.0f / (a.psf_sigma * 1.41421356237309505f);
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < min(nc, a.out_cap); i += nw) {
        const int c = a.order[i];
        const int r = peak_rank(a.key[c]);
        const int py = r / a.w, px = r - py * a.w;
        const long pp = (long)py * a.pitch + px;
        const float sg = (a.mask[pp] & ARGUS_MASK_POS) ? 1.0f : -1.0f;
        float xc = (float)px, yc = (float)py;
        for (int it = 0; it < 4; it++) {
            float sw = 0.0f, sx = 0.0f, sy = 0.0f;
            for (int e = lane; e < side * side; e += 32) {
                const int yy = py - fw + e / side, xx = px - fw + e % side;
                if (xx < 0 || yy < 0 || xx >= a.w || yy >= a.h) continue;
                const long q = (long)yy * a.pitch + xx;
                if (a.mask[q] & ARGUS_MASK_INVALID) continue;
                const float dx = (float)xx - xc, dy = (float)yy - yc;
                const float t = sg * a.D[q] * expf(-(dx * dx + dy * dy) * inv2s2);
                sw += t;
                sx += t * dx;
                sy += t * dy;
            }
            sw = warp_sum(sw);
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            if (!(sw > 0.0f)) break;
            xc += 2.0f * sx / sw;
            yc += 2.0f * sy / sw;
            xc = fminf(fmaxf(xc, px - 2.0f), px + 2.0f);
            yc = fminf(fmaxf(yc, py - 2.0f), py + 2.0f);
        }
        float num = 0.0f, den = 0.0f;
        for (int e = lane; e < side * side; e += 32) {
            const int yy = py - fw + e / side, xx = px - fw + e % side;
            if (xx < 0 || yy < 0 || xx >= a.w || yy >= a.h) continue;
            const long q = (long)yy * a.pitch + xx;
            if (a.mask[q] & ARGUS_MASK_INVALID) continue;
            const float P = pix_gauss((float)xx, xc, inv_s2) * pix_gauss((float)yy, yc, inv_s2);
            const float iv = 1.0f / a.V[q];
            num += P * a.D[q] * iv;
            den += P * P * iv;
        }
        num = warp_sum(num);
        den = warp_sum(den);
        if (lane == 0) {
            argus_source s;
            s.x = xc;
            s.y = yc;
            s.flux = den > 0.0f ? num / den : 0.0f;
            s.flux_err = den > 0.0f ? 1.0f / sqrtf(den) : 0.0f;
            s.peak_snr = a.D[pp] / sqrtf(a.V[pp]);
            s.npix = a.npix[c];
            s.sign = sg > 0 ? 1 : -1;
            s.px = px;
            s.py = py;
            a.out[i] = s;
        }
    }
}

__global__ void finish_kernel(DetArgs a) {
    const int nc = a.count[1];
    *a.n_found = nc;
    if (nc > a.out_cap) argus_latch(a.status, ARGUS_ERR_CAPACITY);
}

}  // namespace

extern "C" int argus_detect(argus_ctx* ctx, const float* diff, const float* diff_var, const uint8_t* flags,
                            argus_shape shape, float nsigma, float psf_sigma, uint8_t* mask,
                            argus_source* out, int cap, int* n_found, argus_stream stream) {
    if (!ctx || !diff || !diff_var || !flags || !mask || !n_found || (cap > 0 && !out) || cap < 0)
        return ARGUS_ERR_ARG;
    if (!(psf_sigma > 0.0f) || psf_sigma > 8.0f || !(nsigma > 0.0f)) return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, ctx->max_pixels);
    if (st) return st;
    if (shape.h > ctx->max_rows) return ARGUS_ERR_ARG;
    if ((long)shape.h * shape.pitch > 0x7fffffffL) return ARGUS_ERR_ARG;
    const void* ps[] = {diff, diff_var, flags, mask};
    for (const void* p : ps)
        if (argus_check_ptr16(p)) return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    DetArgs a;
    a.D = diff; a.V = diff_var; a.flags = flags; a.mask = mask; a.label = ctx->label;
    a.list = ctx->det_list; a.count = ctx->det_count; a.key = ctx->comp_key; a.npix = ctx->comp_npix;
    a.order = ctx->comp_order; a.rows = ctx->row_count; a.out = out; a.n_found = n_found;
    a.status = ctx->d_status; a.pitch = shape.pitch; a.w = shape.w; a.h = shape.h; a.cap = ctx->det_cap;
    a.out_cap = cap; a.nsig = nsigma; a.psf_sigma = psf_sigma;
    if (cudaMemsetAsync(ctx->det_count, 0, 2 * sizeof(int), s) != cudaSuccess) return ARGUS_ERR_CUDA;
    if (cudaMemsetAsync(ctx->row_count, 0, sizeof(int) * (2 * (size_t)shape.h + 2), s) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    const long nv = (shape.pitch / 16) * (long)shape.h;
    long blocks = (nv + 255) / 256;
    if (blocks > (long)ctx->num_sms * 8) blocks = (long)ctx->num_sms * 8;
    mask_kernel<<<(unsigned)blocks, 256, 0, s>>>(a); argus_count_launch(1);
    const int lb = ctx->num_sms * 2;
    union_kernel<<<lb, 256, 0, s>>>(a); argus_count_launch(1);
    flatten_kernel<<<lb, 256, 0, s>>>(a); argus_count_launch(1);
    roots_kernel<<<lb, 256, 0, s>>>(a); argus_count_launch(1);
    stats_kernel<<<lb, 256, 0, s>>>(a); argus_count_launch(1);
    row_hist_kernel<<<lb, 256, 0, s>>>(a); argus_count_launch(1);
    row_scan_kernel<<<1, 1024, 0, s>>>(a); argus_count_launch(1);
    scatter_kernel<<<lb, 256, 0, s>>>(a); argus_count_launch(1);
    row_sort_kernel<<<(shape.h + 255) / 256, 256, 0, s>>>(a); argus_count_launch(1);
    measure_kernel<<<lb, 256, 0, s>>>(a); argus_count_launch(1);
    finish_kernel<<<1, 1, 0, s>>>(a); argus_count_launch(1);
    return argus_launch_status();
}
