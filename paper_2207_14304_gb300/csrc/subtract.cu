// K6: full-frame convolution of the reference with the spatially varying
// PSF-matching kernel, subtraction, and the difference variance (paper Sec. 4.2
// direct image subtraction, Table 2; noise maps, Sec. 3.2).
//
// The per-pixel work is NK * KS^2 + KS^2 multiply-adds (3087 at KS = 21,
// NK = 6), far above the 25 B/px of traffic: on the FP32 pipes the kernel is
// bound by instruction issue, not HBM.  For 11x11 and 21x21 kernels the
// difference image runs on the tensor cores (subtract_tc.cu) and the SIMT
// tile body (subtract_tile.cuh, one CTA per 32x32 tile) computes only the
// variance; other sizes use the SIMT body for both.
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
    constexpr int R = (KS - 1) / 2;
    constexpr int SW = TILE + 2 * R;
    constexpr int NKP = NK == 1 ? 1 : (NK <= 4 ? 4 : 8);
    constexpr int KSP = (KS + 3) / 4 * 4;
    constexpr int KTSZ = (KS * KS * NKP + 3) / 4 * 4;
    const size_t smem = sizeof(float) * (2 * SW * SW + KTSZ + KS * KSP);
    cudaFuncSetAttribute(subtract_kernel<KS, NK, CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((a.w + TILE - 1) / TILE, (a.h + TILE - 1) / TILE);
    subtract_kernel<KS, NK, CONV><<<grid, THREADS, smem, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}

// Kernel sizes with a tensor-core difference image: the SIMT body computes the
// variance only, then the tensor-core kernel writes D.
template <int KS>
int launch_split(const SubArgs& a, int nk, int* status, cudaStream_t st) {
    if (a.diff_var) {
        int rc = ARGUS_ERR_UNSUPPORTED;
        switch (nk) {
            case 1: rc = launch<KS, 1, false>(a, st); break;
            case 3: rc = launch<KS, 3, false>(a, st); break;
            case 6: rc = launch<KS, 6, false>(a, st); break;
        }
        if (rc) return rc;
    }
    return a.diff ? argus_subtract_tc(a, KS, nk, status, st) : ARGUS_OK;
}

template <int KS>
int launch_nk(const SubArgs& a, int nk, cudaStream_t st) {
    if (!a.diff) {   // the variance only
        switch (nk) {
            case 1: return launch<KS, 1, false>(a, st);
            case 3: return launch<KS, 3, false>(a, st);
            case 6: return launch<KS, 6, false>(a, st);
        }
        return ARGUS_ERR_UNSUPPORTED;
    }
    switch (nk) {
        case 1: return launch<KS, 1>(a, st);
        case 3: return launch<KS, 3>(a, st);
        case 6: return launch<KS, 6>(a, st);
    }
    return ARGUS_ERR_UNSUPPORTED;
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
