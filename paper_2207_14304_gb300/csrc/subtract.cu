// K6: full-frame convolution of the reference with the spatially varying
// PSF-matching kernel, subtraction, and the difference variance (paper Sec. 4.2
// direct image subtraction, Table 2; noise maps, Sec. 3.2).
//
// The per-pixel work is NK * KS^2 + KS^2 multiply-adds (3087 at KS = 21,
// NK = 6), far above the 25 B/px of traffic: on the FP32 pipes the kernel is
// bound by instruction issue, not HBM.  For 11x11 and 21x21 kernels the
// difference image runs on the tensor cores (subtract_tc.cu), for other sizes
// on the SIMT tile body (subtract_tile.cuh, one CTA per 32x32 tile); the
// variance always comes from variance_kernel below.
#include "subtract_tile.cuh"

namespace {
using namespace argus_sub;

template <int KS, int NK, bool CONV>
__global__ void __launch_bounds__(THREADS) subtract_kernel(SubArgs a) {
    extern __shared__ __align__(16) float smem[];
    subtract_tile<KS, NK, CONV>(a, blockIdx.x * TILE, blockIdx.y * TILE, smem);
}

template <int KS, int NK, bool CONV = true>
int launch(const SubArgs& a, cudaStream_t st) {
    const size_t smem = tile_smem_bytes<KS, NK, CONV>();
    cudaFuncSetAttribute(subtract_kernel<KS, NK, CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((a.w + TILE - 1) / TILE, (a.h + TILE - 1) / TILE);
    subtract_kernel<KS, NK, CONV><<<grid, THREADS, smem, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}

// Difference variance alone, V_D = V_I + (Kc^2 (x) V_ref), Kc the kernel at the
// centre of the VAR_TILE tile (the same definition as the per-tile body).  One CTA
// of 64 threads per tile: thread (lx, half) owns column lx, rows 16*half ..
// +15.  V_ref is staged column-major (column stride 60 floats: a 16-byte load
// per lane is conflict-free within each quarter-warp), so a thread's 16 + KS - 1
// window rows of one column are (16 + KS - 1)/4 vector loads; the KS squared taps
// of that column sit in registers.  About 96 % of the issued instructions are FMAs.
constexpr int VCS = 60;   // column stride of the staged variance

template <int KS>
constexpr int var_smem_floats() {
    return (TILE + KS - 1) * VCS + KS * ((KS + 3) / 4 * 4);
}

template <int KS, int NK>
__global__ void __launch_bounds__(64) variance_kernel(SubArgs a) {
    constexpr int R = (KS - 1) / 2;
    constexpr int SW = TILE + 2 * R;               // staged tile side
    constexpr int NW = 16 + KS - 1;                // window rows per thread
    constexpr int NW4 = (NW + 3) / 4;
    constexpr int KP = (KS + 3) / 4 * 4;           // padded taps per column
    static_assert(SW + 3 <= VCS, "column stride");
    extern __shared__ __align__(16) float vsm[];
    float* Vc = vsm;                               // [SW][VCS]: Vc[ix * VCS + iy]
    float* K2 = vsm + SW * VCS;                    // [KS (iu)][KP (iv)]
    const int tx0 = blockIdx.x * TILE, ty0 = blockIdx.y * TILE;
    const int tid = threadIdx.x;
    for (int e = tid; e < SW * SW; e += blockDim.x) {
        const int iy = e / SW, ix = e - iy * SW;
        const int gy = ty0 - R + iy, gx = tx0 - R + ix;
        Vc[ix * VCS + iy] = (gy >= 0 && gy < a.h && gx >= 0 && gx < a.w) ? __ldg(a.ref_var + (long)gy * a.pitch + gx)
                                                                          : 0.0f;
    }
    {
        float pc[ARGUS_MAX_TERMS];
        const float xc = (float)(((tx0 + a.ox) / VAR_TILE) * VAR_TILE) + 0.5f * (VAR_TILE - 1);
        const float yc = (float)(((ty0 + a.oy) / VAR_TILE) * VAR_TILE) + 0.5f * (VAR_TILE - 1);
        const float xt = a.W > 1 ? (2.0f * xc - (float)(a.W - 1)) / (float)(a.W - 1) : 0.0f;
        const float yt = a.H > 1 ? (2.0f * yc - (float)(a.H - 1)) / (float)(a.H - 1) : 0.0f;
        spatial_terms(xt, yt, a.sdeg, pc);
        for (int e = tid; e < KS * KP; e += blockDim.x) {
            const int iu = e / KP, iv = e - iu * KP;
            float kc = 0.0f;
            if (iv < KS) {
#pragma unroll
                for (int k = 0; k < NK; k++) kc = fmaf(pc[k], __ldg(a.K + k * KS * KS + iv * KS + iu), kc);
            }
            K2[e] = kc * kc;
        }
    }
    __syncthreads();
    const int lx = tid & 31, ly0 = (tid >> 5) * 16;
    float acc[16];
#pragma unroll
    for (int j = 0; j < 16; j++) acc[j] = 0.0f;
    // output (lx, ly0 + j), tap (iu, iv): V_ref(x - iu + R, y - iv + R) = Vc[lx + 2R - iu][ly0 + j + 2R - iv]
#pragma unroll 1
    for (int iu = 0; iu < KS; iu++) {
        float kc[KP];
#pragma unroll
        for (int q = 0; q < KP; q += 4) *reinterpret_cast<float4*>(kc + q) = *reinterpret_cast<const float4*>(K2 + iu * KP + q);
        float win[NW4 * 4];
        const float* col = Vc + (lx + 2 * R - iu) * VCS + ly0;
#pragma unroll
        for (int q = 0; q < NW4; q++) *reinterpret_cast<float4*>(win + 4 * q) = *reinterpret_cast<const float4*>(col + 4 * q);
#pragma unroll
        for (int iv = 0; iv < KS; iv++)
#pragma unroll
            for (int j = 0; j < 16; j++) acc[j] = fmaf(kc[iv], win[j + 2 * R - iv], acc[j]);
    }
    const int x = tx0 + lx;
    if (x >= a.w) return;
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const int y = ty0 + ly0 + j;
        if (y >= a.h) break;
        const long p = (long)y * a.pitch + x;
        const bool inner = x >= R && y >= R && x <= a.w - 1 - R && y <= a.h - 1 - R;
        a.diff_var[p] = (inner && a.flags[p] == 0) ? a.sci_var[p] + acc[j] : 0.0f;
    }
}

template <int KS, int NK>
int launch_var(const SubArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(float) * var_smem_floats<KS>();
    cudaFuncSetAttribute(variance_kernel<KS, NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((a.w + TILE - 1) / TILE, (a.h + TILE - 1) / TILE);
    variance_kernel<KS, NK><<<grid, 64, smem, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}

// Kernel sizes with a tensor-core difference image: the SIMT body computes the
// variance only, then the tensor-core kernel writes D.
template <int KS>
int launch_split(const SubArgs& a, int nk, int* status, cudaStream_t st) {
    if (nk != 1 && nk != 3 && nk != 6) return ARGUS_ERR_UNSUPPORTED;
    if (a.diff_var) {
        // the variance on the tensor cores when the frame origin is on the variance-tile grid
        int rc = argus_subtract_var_tc(a, KS, status, st);
        if (rc == ARGUS_ERR_UNSUPPORTED) {
            switch (nk) {
                case 1: rc = launch_var<KS, 1>(a, st); break;
                case 3: rc = launch_var<KS, 3>(a, st); break;
                case 6: rc = launch_var<KS, 6>(a, st); break;
            }
        }
        if (rc) return rc;
    }
    return a.diff ? argus_subtract_tc(a, KS, nk, status, st) : ARGUS_OK;
}

// Other kernel sizes: the variance kernel, then the SIMT tile body for D alone.
template <int KS>
int launch_nk(const SubArgs& a, int nk, cudaStream_t st) {
    if (nk != 1 && nk != 3 && nk != 6) return ARGUS_ERR_UNSUPPORTED;
    if (a.diff_var) {
        const int rc = nk == 1 ? launch_var<KS, 1>(a, st) : (nk == 3 ? launch_var<KS, 3>(a, st) : launch_var<KS, 6>(a, st));
        if (rc || !a.diff) return rc;
    }
    SubArgs d = a;
    d.diff_var = nullptr;
    switch (nk) {
        case 1: return launch<KS, 1>(d, st);
        case 3: return launch<KS, 3>(d, st);
        default: return launch<KS, 6>(d, st);
    }
}

}  // namespace

extern "C" int argus_subtract(argus_ctx* ctx, const float* sci, const float* sci_var, const float* ref,
                              const float* ref_var, const uint8_t* flags, argus_shape shape, int frame_w,
                              int frame_h, int ox, int oy, int ksize, int spatial_degree, const float* K,
                              int bg_degree, const double* bg, float* diff, float* diff_var,
                              argus_stream stream) {
    if (!ctx || !sci_var || !ref_var || !flags || !K || (!diff && !diff_var)) return ARGUS_ERR_ARG;
    if (diff && (!sci || !ref)) return ARGUS_ERR_ARG;
    if (bg_degree >= 0 && !bg) return ARGUS_ERR_ARG;
    int st = argus_check_shape(shape, ctx->max_pixels);
    if (st) return st;
    const void* ps[] = {sci, sci_var, ref, ref_var, flags, diff, diff_var};
    for (const void* p : ps)
        if (p && argus_check_ptr16(p)) return ARGUS_ERR_ALIGN;
    if (spatial_degree < 0 || spatial_degree > 2 || bg_degree < -1 || bg_degree > 2) return ARGUS_ERR_ARG;
    if (frame_w < shape.w + ox || frame_h < shape.h + oy || ox < 0 || oy < 0) return ARGUS_ERR_ARG;
    if (spatial_degree > 0 && ((ox % TILE) || (oy % TILE))) return ARGUS_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    SubArgs a;
    a.sci = sci; a.sci_var = sci_var; a.ref = ref; a.ref_var = ref_var; a.flags = flags; a.K = K;
    a.bg = bg; a.diff = diff; a.diff_var = diff_var; a.pitch = shape.pitch; a.w = shape.w; a.h = shape.h;
    a.W = frame_w; a.H = frame_h; a.ox = ox; a.oy = oy; a.sdeg = spatial_degree;
    a.bg_deg = bg_degree < 0 ? 0 : bg_degree;
    a.nbg = bg_degree < 0 ? 0 : argus_nterms(bg_degree);
    const int nk = argus_nterms(spatial_degree);
    cudaStream_t s = (cudaStream_t)stream;
    switch (ksize) {
        case 7: return launch_nk<7>(a, nk, s);
        case 9: return launch_nk<9>(a, nk, s);
        case 11: return launch_split<11>(a, nk, ctx->d_status, s);
        case 15: return launch_nk<15>(a, nk, s);
        case 21: return launch_split<21>(a, nk, ctx->d_status, s);
    }
    return ARGUS_ERR_UNSUPPORTED;
}
