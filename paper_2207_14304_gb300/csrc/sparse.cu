// Sparse and low-resolution segment products (paper Sec. 3.3 "Sparse Image
// Segments"; Sec. 2, products 1c and 1d).
//
// Minipix stamping: a cell of cell x cell pixels is kept when a catalogue
// target or a detected source lies in it; the rest of the image is set to 0
// and the kept cells are compacted into a dense list.
//   1. mark:  one thread per target / source sets keep[cell] = 1 (keep is
//             cleared by a memset first; concurrent writers store the same 1).
//   2. count: per 1024-cell chunk, the number of kept cells.
//   3. scan:  one CTA: exclusive scan of the chunk counts, total -> *n_kept.
//   4. list:  per chunk, block-ranked kept cells -> cell_index[offset + rank],
//             so the list is in ascending cell order whatever the schedule.
//   5. pack:  each listed cell's pixels -> packed[k] (row-major, 0 off-image),
//             one thread per packed pixel.
//   6. zero:  out = kept ? img : 0, one float4 column per thread over a slice
//             of rows; img is read only where a kept cell covers the float4,
//             so the zeroed majority of a frame costs its 4-byte write alone.
// Low-resolution map: one CTA per (output row, strip of nx output columns):
// each thread sums a float4 column of `factor` rows (skipping flagged and
// non-finite pixels) into shared memory, then one thread per output pixel
// adds its `factor` column sums and divides by the valid count.
#include "argus_internal.cuh"

namespace {

constexpr int CHUNK = 1024;        // cells per count / list CTA (256 threads x 4)
constexpr int LR_THREADS = 256;    // low-resolution CTA: 1024 pixel columns at most

struct MiniArgs {
    const float* img;
    const int* targets;
    const argus_source* src;
    const int* n_src;
    uint8_t* keep;
    float* out;
    float* packed;
    int* cell_index;
    int* n_kept;
    int* chunk;       // [nchunks] counts, then exclusive offsets (in place)
    int* status;
    long pitch;
    int n_targets, src_cap, cap;
    int w, h, cell, ncx, ncy, nchunks;
};

__global__ void __launch_bounds__(256) mark_kernel(MiniArgs a) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y;
    if (i < a.n_targets) {
        x = a.targets[2 * i];
        y = a.targets[2 * i + 1];
    } else {
        const long j = i - a.n_targets;
        if (j >= a.src_cap || j >= *a.n_src) return;
        x = a.src[j].px;
        y = a.src[j].py;
    }
    if (x < 0 || y < 0 || x >= a.w || y >= a.h) return;
    a.keep[(long)(y / a.cell) * a.ncx + x / a.cell] = 1;
}

// Kept flags of this thread's 4 cells (cells past the end count as not kept).
__device__ __forceinline__ int chunk_flags(const MiniArgs& a, long c0, bool k[4]) {
    const long nc = (long)a.ncx * a.ncy;
    int n = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        k[i] = c0 + i < nc && a.keep[c0 + i] != 0;
        n += k[i] ? 1 : 0;
    }
    return n;
}

__global__ void __launch_bounds__(256) count_kernel(MiniArgs a) {
    __shared__ int ws[8];
    bool k[4];
    const int n = __reduce_add_sync(0xffffffffu, chunk_flags(a, (long)blockIdx.x * CHUNK + threadIdx.x * 4, k));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < 8; i++) t += ws[i];
        a.chunk[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) scan_kernel(MiniArgs a, int want_list) {
    __shared__ int ws[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < a.nchunks; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const int v = b < a.nchunks ? a.chunk[b] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int s = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            ws[lane] = s;
        }
        __syncthreads();
        const int excl = carry + (warp ? ws[warp - 1] : 0) + incl - v;
        if (b < a.nchunks) a.chunk[b] = excl;
        __syncthreads();                       // every thread has read carry and ws
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *a.n_kept = carry;
        if (want_list && carry > a.cap) argus_latch(a.status, ARGUS_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(256) list_kernel(MiniArgs a) {
    __shared__ int ws[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long c0 = (long)blockIdx.x * CHUNK + threadIdx.x * 4;
    bool k[4];
    const int n = chunk_flags(a, c0, k);
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    int pos = a.chunk[blockIdx.x] + incl - n;
    for (int i = 0; i < warp; i++) pos += ws[i];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (k[i]) {
            if (pos < a.cap) a.cell_index[pos] = (int)(c0 + i);
            pos++;
        }
    }
}

__global__ void __launch_bounds__(256) pack_kernel(MiniArgs a) {
    const long cc = (long)a.cell * a.cell;
    const long nk = min(*a.n_kept, a.cap);
    const long total = nk * cc;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long k = e / cc;
        const int r = (int)(e - k * cc);
        const int ci = a.cell_index[k];
        const int cy = ci / a.ncx, cx = ci - cy * a.ncx;
        const int yy = r / a.cell, xx = r - yy * a.cell;
        const int x = cx * a.cell + xx, y = cy * a.cell + yy;
        a.packed[e] = (x < a.w && y < a.h) ? a.img[(long)y * a.pitch + x] : 0.0f;
    }
}

// grid: x over 256-float4 column blocks, y over row slices (rows y, y + gridDim.y, ...)
__global__ void __launch_bounds__(256) zero_kernel(MiniArgs a) {
    const int x0 = (blockIdx.x * 256 + threadIdx.x) * 4;
    if (x0 >= a.pitch) return;                       // no barrier below
    // cell column of each of the 4 pixels, the same in every row; -1 past the image
    int c[4];
    {
        int cx = x0 / a.cell, next = (cx + 1) * a.cell;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            if (x0 + i >= next) {
                cx++;
                next += a.cell;
            }
            c[i] = x0 + i < a.w ? cx : -1;
        }
    }
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        const long p = (long)y * a.pitch + x0;
        float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (c[0] >= 0) {
            const uint8_t* krow = a.keep + (long)(y / a.cell) * a.ncx;
            bool k[4];
            bool any = false;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                k[i] = c[i] >= 0 && krow[c[i]] != 0;
                any |= k[i];
            }
            if (any) {
                const float4 v = *reinterpret_cast<const float4*>(a.img + p);
                o.x = k[0] ? v.x : 0.0f;
                o.y = k[1] ? v.y : 0.0f;
                o.z = k[2] ? v.z : 0.0f;
                o.w = k[3] ? v.w : 0.0f;
            }
        }
        *reinterpret_cast<float4*>(a.out + p) = o;
    }
}

struct LowArgs {
    const float* img;
    const uint8_t* flags;
    float* out;
    long pitch, opitch;
    int w, h, f, nx, ow;
};

__global__ void __launch_bounds__(LR_THREADS) lowres_kernel(LowArgs a) {
    __shared__ float cs[LR_THREADS * 4];
    __shared__ int cn[LR_THREADS * 4];
    const int Y = blockIdx.x;                          // rows on x: no 65535 limit
    const int X0 = blockIdx.y * a.nx;
    const int x = X0 * a.f + 4 * threadIdx.x;          // a multiple of 4, as nx * f is
    const int y0 = Y * a.f, y1 = min(y0 + a.f, a.h);
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int n[4] = {0, 0, 0, 0};
    if (4 * (int)threadIdx.x < a.nx * a.f && x < a.w) {   // x < w <= pitch, pitch % 4 == 0
#pragma unroll 5
        for (int y = y0; y < y1; y++) {
            const long p = (long)y * a.pitch + x;
            const float4 v4 = __ldg(reinterpret_cast<const float4*>(a.img + p));
            uchar4 f4 = make_uchar4(0, 0, 0, 0);
            if (a.flags) f4 = *reinterpret_cast<const uchar4*>(a.flags + p);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
            const uint8_t fl[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if (x + i < a.w && fl[i] == 0 && isfinite(v[i])) {
                    s[i] += v[i];
                    n[i]++;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        cs[4 * threadIdx.x + i] = s[i];
        cn[4 * threadIdx.x + i] = n[i];
    }
    __syncthreads();
    const int X = X0 + threadIdx.x;
    if ((int)threadIdx.x < a.nx && X < a.ow) {
        float t = 0.0f;
        int m = 0;
        for (int j = 0; j < a.f; j++) {
            t += cs[threadIdx.x * a.f + j];
            m += cn[threadIdx.x * a.f + j];
        }
        a.out[(long)Y * a.opitch + X] = m ? t / (float)m : 0.0f;
    }
}

}  // namespace

extern "C" int argus_minipix(argus_ctx* ctx, const float* img, argus_shape shape, int cell, const int* targets,
                             int n_targets, const argus_source* sources, const int* n_sources, int sources_cap,
                             uint8_t* keep, float* out, float* packed, int* cell_index, int cap, int* n_kept,
                             argus_stream stream) {
    if (!ctx || !img || !keep || !n_kept || cell < 1 || cell > 256 || n_targets < 0 || sources_cap < 0 || cap < 0)
        return ARGUS_ERR_ARG;
    if ((n_targets > 0 && !targets) || (sources_cap > 0 && (!sources || !n_sources))) return ARGUS_ERR_ARG;
    if ((packed && !cell_index) || (cell_index && cap == 0) || (out && (const float*)out == img))
        return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, ctx->max_pixels);
    if (st) return st;
    if (argus_check_ptr16(img) || (out && argus_check_ptr16(out))) return ARGUS_ERR_ALIGN;
    const int ncx = (shape.w + cell - 1) / cell, ncy = (shape.h + cell - 1) / cell;
    const long nc = (long)ncx * ncy;
    if (nc > 0x7fffffffL) return ARGUS_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    MiniArgs a;
    a.img = img; a.targets = targets; a.src = sources; a.n_src = n_sources; a.keep = keep; a.out = out;
    a.packed = packed; a.cell_index = cell_index; a.n_kept = n_kept; a.chunk = ctx->label;
    a.status = ctx->d_status; a.pitch = shape.pitch; a.n_targets = n_targets; a.src_cap = sources_cap;
    a.cap = cap; a.w = shape.w; a.h = shape.h; a.cell = cell; a.ncx = ncx; a.ncy = ncy;
    a.nchunks = (int)((nc + CHUNK - 1) / CHUNK);     // <= nc <= pixels <= max_pixels (label's length)
    if (cudaMemsetAsync(keep, 0, (size_t)nc, s) != cudaSuccess) return ARGUS_ERR_CUDA;
    const long nt = (long)n_targets + sources_cap;
    if (nt > 0) {
        mark_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(a); argus_count_launch(1);
    }
    count_kernel<<<a.nchunks, 256, 0, s>>>(a); argus_count_launch(1);
    scan_kernel<<<1, 1024, 0, s>>>(a, cell_index != nullptr); argus_count_launch(1);
    if (cell_index) {
        list_kernel<<<a.nchunks, 256, 0, s>>>(a); argus_count_launch(1);
    }
    if (packed) {
        const long work = (long)cap * cell * cell;
        long blocks = (work + 255) / 256;
        if (blocks > (long)ctx->num_sms * 8) blocks = (long)ctx->num_sms * 8;
        pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(a); argus_count_launch(1);
    }
    if (out) {
        const int gx = (int)((shape.pitch / 4 + 255) / 256);
        int gy = ctx->num_sms * 16 / gx;
        gy = gy < 1 ? 1 : (gy > shape.h ? shape.h : gy);
        zero_kernel<<<dim3(gx, gy), 256, 0, s>>>(a); argus_count_launch(1);
    }
    return argus_launch_status();
}

extern "C" int argus_lowres(argus_ctx* ctx, const float* img, const uint8_t* flags, argus_shape shape, int factor,
                            float* out, long out_pitch, argus_stream stream) {
    if (!ctx || !img || !out || factor < 1 || factor > 64) return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, ctx->max_pixels);
    if (st) return st;
    const int ow = (shape.w + factor - 1) / factor, oh = (shape.h + factor - 1) / factor;
    if (out_pitch < ow) return ARGUS_ERR_ARG;
    if (argus_check_ptr16(img) || argus_check_ptr16(out) || (flags && argus_check_ptr16(flags)))
        return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    // output columns per CTA: nx * factor <= 4 * LR_THREADS and a multiple of 4,
    // so every thread's first pixel column is a multiple of 4 (float4 loads)
    int nx = 4 * LR_THREADS / factor;
    while ((nx * factor) % 4) nx--;
    LowArgs a;
    a.img = img; a.flags = flags; a.out = out; a.pitch = shape.pitch; a.opitch = out_pitch;
    a.w = shape.w; a.h = shape.h; a.f = factor; a.nx = nx; a.ow = ow;
    const dim3 grid((unsigned)oh, (unsigned)((ow + nx - 1) / nx));
    lowres_kernel<<<grid, LR_THREADS, 0, (cudaStream_t)stream>>>(a); argus_count_launch(1);
    return argus_launch_status();
}
