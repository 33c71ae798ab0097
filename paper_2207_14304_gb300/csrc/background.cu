// Median-filtered background map (paper Table 2, GPU timing "Median-filtered
// background map"; background maps held with the calibration frames, Sec. 3.2).
//
//   1. box_median_kernel: one CTA per box x box mesh box; the valid pixels
//      (flag 0, finite) stay in registers as order-preserving 32-bit keys and
//      an 8-bit radix select (4 passes over a 256-bin shared histogram) finds
//      the middle key(s); the box value is their mean in FP64 (exact), or NaN
//      when fewer than min_frac of the box's pixels are valid.
//   2. mesh_fill_kernel: one CTA; the median of all box values (the value of
//      boxes with nothing in reach), by the same radix select on 64-bit keys
//      of the doubles, reading the mesh from global memory.
//   3. mesh_filter_kernel: one thread per box; the median of the values that
//      exist in its filt x filt neighbourhood (clipped at the mesh edges).
//   4. interp_kernel: the map, bilinear between box centres (mean pixel
//      coordinate of each box), constant beyond the outermost ones, in FP32,
//      four pixels per thread.
#include "argus_internal.cuh"

#include <cstring>

namespace {

constexpr int BM_THREADS = 256;
constexpr int BM_MAX_PER = 16;          // box <= 64: at most 16 pixels per thread
constexpr int FILL_THREADS = 1024;

struct BgArgs {
    const float* img;
    const uint8_t* flags;
    double* raw;        // [ny][nx] box medians (NaN: no value)
    double* mesh;       // [ny][nx] filtered
    double* fill;       // [1] median of all box values
    float* map;
    long pitch;
    int w, h, box, filt, nx, ny;
    float min_frac;
};

// Bit patterns on host and device (the host side serves the CPU checks).
__host__ __device__ __forceinline__ unsigned f32_bits(float v) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(v);
#else
    unsigned u;
    memcpy(&u, &v, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float bits_f32(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float v;
    memcpy(&v, &u, 4);
    return v;
#endif
}
__host__ __device__ __forceinline__ unsigned long long f64_bits(double v) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long u;
    memcpy(&u, &v, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double bits_f64(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double v;
    memcpy(&v, &u, 8);
    return v;
#endif
}

// Order-preserving keys: a < b (as numbers, -0 before +0) iff key(a) < key(b).
__host__ __device__ __forceinline__ unsigned key32(float v) {
    const unsigned u = f32_bits(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float unkey32(unsigned k) {
    return bits_f32((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__host__ __device__ __forceinline__ unsigned long long key64(double v) {
    const unsigned long long u = f64_bits(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ double unkey64(unsigned long long k) {
    return bits_f64((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k);
}

// One thread's share of a box: pixels tid, tid + 256, ... of the box as keys
// (ok = valid); returns the count of valid pixels.
__host__ __device__ __forceinline__ int box_load(const BgArgs& a, int bx, int by, int tid, unsigned* key, bool* ok) {
    const int x0 = bx * a.box, y0 = by * a.box;
    const int bw = min(a.box, a.w - x0), bh = min(a.box, a.h - y0);
    const int npx = bw * bh;
    int nv = 0;
#pragma unroll
    for (int j = 0; j < BM_MAX_PER; j++) {
        const int i = tid + j * BM_THREADS;
        ok[j] = false;
        key[j] = 0;
        if (i < npx) {
            const int yy = i / bw, xx = i - yy * bw;
            const long p = (long)(y0 + yy) * a.pitch + x0 + xx;
            const float v = a.img[p];
            if (isfinite(v) && (!a.flags || a.flags[p] == 0)) {
                ok[j] = true;
                key[j] = key32(v);
                nv++;
            }
        }
    }
    return nv;
}

// One thread's histogram contribution of a radix pass: add(bin) for each of its
// keys that matches the prefix decided so far.
template <typename Add>
__host__ __device__ __forceinline__ void box_hist(const unsigned* key, const bool* ok, unsigned mask, unsigned prefix,
                                                  int shift, Add add) {
#pragma unroll
    for (int j = 0; j < BM_MAX_PER; j++)
        if (ok[j] && (key[j] & mask) == prefix) add((int)((key[j] >> shift) & 255u));
}

// One thread's count of keys <= k1 and its smallest key above k1.
__host__ __device__ __forceinline__ void box_le_min(const unsigned* key, const bool* ok, unsigned k1, int& le,
                                                    unsigned& m) {
    le = 0;
    m = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < BM_MAX_PER; j++) {
        if (!ok[j]) continue;
        if (key[j] <= k1) le++;
        else m = min(m, key[j]);
    }
}

// The median from the middle keys: n odd -> k1 == k2.
__host__ __device__ __forceinline__ double median_of_keys(unsigned k1, unsigned k2) {
    return 0.5 * ((double)unkey32(k1) + (double)unkey32(k2));
}

// Whether a box with n valid pixels of npx has a value.
__host__ __device__ __forceinline__ bool box_has_value(int n, int npx, float min_frac) {
    return n > 0 && (float)n >= min_frac * (float)npx;
}

// Block-wide sum of an int (every thread receives it); `red` holds 32 ints.
__device__ __forceinline__ int block_sum(int v, int* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int t = 0;
    for (int i = 0; i < nw; i++) t += red[i];
    return t;
}

// Bin of the 256-bin histogram holding the k-th element (0-based) in bin
// order; k is reduced to the rank inside that bin.  Called by every thread,
// result broadcast through shared memory.
__device__ __forceinline__ int pick_bin(const int* hist, int& k, int* sh) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int c[8], s = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            c[i] = hist[lane * 8 + i];
            s += c[i];
        }
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int run = incl - s;                      // elements in the bins before this lane's 8
        if (k >= run && k < incl) {              // exactly one lane
            int b = lane * 8;
            for (int i = 0; i < 8; i++, b++) {
                if (k < run + c[i]) break;
                run += c[i];
            }
            sh[0] = b;
            sh[1] = k - run;
        }
    }
    __syncthreads();
    const int b = sh[0];
    k = sh[1];
    __syncthreads();
    return b;
}

__global__ void __launch_bounds__(BM_THREADS) box_median_kernel(BgArgs a) {
    __shared__ int hist[256];
    __shared__ int red[32];
    __shared__ int sh[2];
    __shared__ unsigned umin[32];
    const int bx = blockIdx.x, by = blockIdx.y;
    const int npx = min(a.box, a.w - bx * a.box) * min(a.box, a.h - by * a.box);
    unsigned key[BM_MAX_PER];
    bool ok[BM_MAX_PER];
    const int n = block_sum(box_load(a, bx, by, threadIdx.x, key, ok), red);
    double out = __longlong_as_double(0x7ff8000000000000ll);     // NaN: no value
    if (box_has_value(n, npx, a.min_frac)) {
        // k-th smallest key for k1 = (n - 1) / 2
        int k = (n - 1) / 2;
        unsigned prefix = 0, mask = 0;
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = threadIdx.x; i < 256; i += BM_THREADS) hist[i] = 0;
            __syncthreads();
            box_hist(key, ok, mask, prefix, shift, [&](int b) { atomicAdd(&hist[b], 1); });
            __syncthreads();
            const int b = pick_bin(hist, k, sh);
            prefix |= (unsigned)b << shift;
            mask |= 255u << shift;
        }
        const unsigned k1 = prefix;
        unsigned k2 = k1;
        if ((n & 1) == 0) {
            // the next order statistic: k1 again if it repeats, else the smallest key above it
            int le;
            unsigned m;
            box_le_min(key, ok, k1, le, m);
            const int nle = block_sum(le, red);
            m = __reduce_min_sync(0xffffffffu, m);
            if ((threadIdx.x & 31) == 0) umin[threadIdx.x >> 5] = m;
            __syncthreads();
            unsigned mm = 0xffffffffu;
            for (int i = 0; i < BM_THREADS / 32; i++) mm = min(mm, umin[i]);
            k2 = nle >= n / 2 + 1 ? k1 : mm;
        }
        out = median_of_keys(k1, k2);
    }
    if (threadIdx.x == 0) a.raw[(long)by * a.nx + bx] = out;
}

// Median of the non-NaN doubles v[0..n) by radix select over global memory
// (one CTA); 0 if there are none.
__global__ void __launch_bounds__(FILL_THREADS) mesh_fill_kernel(BgArgs a) {
    __shared__ int hist[256];
    __shared__ int red[32];
    __shared__ int sh[2];
    __shared__ unsigned long long umin[32];
    const int ncell = a.nx * a.ny;
    int nv = 0;
    for (int i = threadIdx.x; i < ncell; i += FILL_THREADS) nv += isnan(a.raw[i]) ? 0 : 1;
    const int n = block_sum(nv, red);
    if (n == 0) {
        if (threadIdx.x == 0) *a.fill = 0.0;
        return;
    }
    int k = (n - 1) / 2;
    unsigned long long prefix = 0, mask = 0;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += FILL_THREADS) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < ncell; i += FILL_THREADS) {
            const double v = a.raw[i];
            if (isnan(v)) continue;
            const unsigned long long kk = key64(v);
            if ((kk & mask) == prefix) atomicAdd(&hist[(kk >> shift) & 255ull], 1);
        }
        __syncthreads();
        const int b = pick_bin(hist, k, sh);
        prefix |= (unsigned long long)b << shift;
        mask |= 255ull << shift;
    }
    const unsigned long long k1 = prefix;
    unsigned long long k2 = k1;
    if ((n & 1) == 0) {
        int le = 0;
        unsigned long long m = ~0ull;
        for (int i = threadIdx.x; i < ncell; i += FILL_THREADS) {
            const double v = a.raw[i];
            if (isnan(v)) continue;
            const unsigned long long kk = key64(v);
            if (kk <= k1) le++;
            else m = kk < m ? kk : m;
        }
        const int nle = block_sum(le, red);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
            m = t < m ? t : m;
        }
        if ((threadIdx.x & 31) == 0) umin[threadIdx.x >> 5] = m;
        __syncthreads();
        unsigned long long mm = ~0ull;
        for (int i = 0; i < FILL_THREADS / 32; i++) mm = umin[i] < mm ? umin[i] : mm;
        k2 = nle >= n / 2 + 1 ? k1 : mm;
    }
    if (threadIdx.x == 0) *a.fill = 0.5 * (unkey64(k1) + unkey64(k2));
}

// The filtered value of box (cx, cy): the median of the values that exist in its
// filt x filt neighbourhood, else `fill`.
__host__ __device__ __forceinline__ double filter_cell(const double* raw, int nx, int ny, int cx, int cy, int filt,
                                                       double fill) {
    const int r = filt / 2;
    double v[49];
    int n = 0;
    for (int y = max(0, cy - r); y <= min(ny - 1, cy + r); y++) {
        for (int x = max(0, cx - r); x <= min(nx - 1, cx + r); x++) {
            const double t = raw[(long)y * nx + x];
            if (isnan(t)) continue;
            int i = n++;                           // insertion into the sorted prefix
            while (i > 0 && v[i - 1] > t) {
                v[i] = v[i - 1];
                i--;
            }
            v[i] = t;
        }
    }
    return n ? 0.5 * (v[(n - 1) / 2] + v[n / 2]) : fill;
}

__global__ void __launch_bounds__(256) mesh_filter_kernel(BgArgs a) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.nx * a.ny) return;
    const int cy = c / a.nx, cx = c - cy * a.nx;
    a.mesh[c] = filter_cell(a.raw, a.nx, a.ny, cx, cy, a.filt, *a.fill);
}

// Interpolation coordinate along one axis: lower box index i (upper i + 1) and
// weight t of the upper one, clamped beyond the outermost centres.
__host__ __device__ __forceinline__ void axis_weight(int p, int n, int box, int nb, int& i, float& t) {
    if (nb == 1) {
        i = 0;
        t = 0.0f;
        return;
    }
    // box i's centre is i box + (box - 1) / 2 (a half-integer for even boxes):
    // i = floor((2 p - (box - 1)) / (2 box)), exact in integers
    const int num = 2 * p - (box - 1);
    i = num >= 0 ? num / (2 * box) : 0;
    i = min(i, nb - 2);
    const float c0 = i * box + 0.5f * (float)(box - 1);
    const int e1 = min((i + 2) * box, n);
    const float c1 = 0.5f * (float)((i + 1) * box + e1 - 1);
    t = fminf(fmaxf(((float)p - c0) / (c1 - c0), 0.0f), 1.0f);
}

// Bilinear value from the mesh row r0 (lower box ix, next box ix + jx, next row
// + jy) in FP32.
__host__ __device__ __forceinline__ float bilinear(const double* r0, int ix, int jx, int jy, float tx, float ty) {
    const float m00 = (float)r0[ix], m01 = (float)r0[ix + jx];
    const float m10 = (float)r0[jy + ix], m11 = (float)r0[jy + ix + jx];
    const float top = m00 + (m01 - m00) * tx;
    const float bot = m10 + (m11 - m10) * tx;
    return top + (bot - top) * ty;
}

__global__ void __launch_bounds__(256) interp_kernel(BgArgs a) {
    const int x0 = (blockIdx.x * 256 + threadIdx.x) * 4;
    if (x0 >= a.pitch) return;
    int ix[4];
    float tx[4];
#pragma unroll
    for (int k = 0; k < 4; k++) axis_weight(min(x0 + k, a.w - 1), a.w, a.box, a.nx, ix[k], tx[k]);
    const int jx = a.nx > 1 ? 1 : 0;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        int iy;
        float ty;
        axis_weight(y, a.h, a.box, a.ny, iy, ty);
        const int jy = a.ny > 1 ? a.nx : 0;
        const double* r0 = a.mesh + (long)iy * a.nx;
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; k++) o[k] = x0 + k < a.w ? bilinear(r0, ix[k], jx, jy, tx[k], ty) : 0.0f;
        *reinterpret_cast<float4*>(a.map + (long)y * a.pitch + x0) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

}  // namespace

extern "C" int argus_background(argus_ctx* ctx, const float* img, const uint8_t* flags, argus_shape shape,
                                int box, int filt, float min_frac, double* mesh, float* map, argus_stream stream) {
    if (!ctx || !img || !mesh || box < 8 || box > 64 || filt < 1 || filt > 7 || (filt & 1) == 0 ||
        !(min_frac >= 0.0f && min_frac <= 1.0f))
        return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, ctx->max_pixels);
    if (st) return st;
    if (argus_check_ptr16(img) || (flags && argus_check_ptr16(flags)) || (map && argus_check_ptr16(map)) ||
        ((uintptr_t)mesh & 7u))
        return ARGUS_ERR_ALIGN;
    const int nx = (shape.w + box - 1) / box, ny = (shape.h + box - 1) / box;
    if (ny > 65535 || ((size_t)nx * ny + 1) * sizeof(double) > ctx->max_pixels * sizeof(int)) return ARGUS_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    BgArgs a;
    a.img = img; a.flags = flags; a.mesh = mesh; a.map = map; a.pitch = shape.pitch;
    a.w = shape.w; a.h = shape.h; a.box = box; a.filt = filt; a.nx = nx; a.ny = ny; a.min_frac = min_frac;
    // scratch: the raw mesh and the fill value in the detection label buffer
    // (max_pixels ints >= 2 doubles per box + 1, as box >= 8)
    a.raw = reinterpret_cast<double*>(ctx->label);
    a.fill = a.raw + (long)nx * ny;
    box_median_kernel<<<dim3(nx, ny), BM_THREADS, 0, s>>>(a); argus_count_launch(1);
    mesh_fill_kernel<<<1, FILL_THREADS, 0, s>>>(a); argus_count_launch(1);
    mesh_filter_kernel<<<(nx * ny + 255) / 256, 256, 0, s>>>(a); argus_count_launch(1);
    if (map) {
        const int gx = (int)((shape.pitch / 4 + 255) / 256);
        int gy = ctx->num_sms * 16 / gx;
        gy = gy < 1 ? 1 : (gy > shape.h ? shape.h : gy);
        interp_kernel<<<dim3(gx, gy), 256, 0, s>>>(a); argus_count_launch(1);
    }
    return argus_launch_status();
}
