// Context, status and argument checks of the libargusdia C ABI.
//
// The context owns every byte of scratch the path needs; it is allocated once
// in argus_create, mirroring the paper's pre-allocation of reference and
// calibration frames on the GPU at the start of each pointing (Sec. 4,
// "Pipeline Implementation").  No entry point allocates afterwards.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include <cstdio>

#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled

#include "argus_internal.cuh"

extern "C" const char* argus_status_string(int s) {
    switch (s) {
        case ARGUS_OK: return "ok";
        case ARGUS_ERR_ARG: return "invalid argument";
        case ARGUS_ERR_ALIGN: return "pointer or pitch not 16-byte aligned";
        case ARGUS_ERR_CUDA: return "CUDA runtime error";
        case ARGUS_ERR_NOMEM: return "out of device memory";
        case ARGUS_ERR_SINGULAR: return "normal matrix not positive definite";
        case ARGUS_ERR_CAPACITY: return "output or scratch capacity exceeded";
        case ARGUS_ERR_TIMEOUT: return "bounded device wait expired";
        case ARGUS_ERR_UNSUPPORTED: return "size outside the compiled kernel set";
        default: return "unknown status";
    }
}

int argus_check_shape(const argus_shape& s, size_t max_pixels) {
    if (s.w <= 0 || s.h <= 0 || s.pitch < s.w) return ARGUS_ERR_ARG;
    if (s.pitch % 16) return ARGUS_ERR_ALIGN;
    if ((size_t)s.h * (size_t)s.pitch > max_pixels) return ARGUS_ERR_ARG;
    return ARGUS_OK;
}

int argus_check_ptr16(const void* p) {
    return ((uintptr_t)p & 15u) ? ARGUS_ERR_ALIGN : ARGUS_OK;
}

static std::atomic<unsigned long long> g_launches{0};

void argus_count_launch(int n) { g_launches.fetch_add((unsigned long long)(long long)n, std::memory_order_relaxed); }

extern "C" unsigned long long argus_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

// The last CUDA error a call of this thread met, as "name: description".
static thread_local char g_last_cuda_error[256] = "";

int argus_cuda_fail(cudaError_t e) {
    snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return ARGUS_ERR_CUDA;
}

int argus_launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ARGUS_OK : argus_cuda_fail(e);
}

extern "C" const char* argus_last_cuda_error(void) { return g_last_cuda_error; }

// The driver's tensor-map encoder, looked up once through the runtime (no link
// against libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;
static std::once_flag g_encode_once;

int argus_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, int esize, const void* base, long w, long h, long pitch,
                  int bx, int by) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode_tiled = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    if (!g_encode_tiled) {
        snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "cuTensorMapEncodeTiled not available from the driver");
        return ARGUS_ERR_CUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * (cuuint64_t)esize};
    const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode_tiled(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "cuTensorMapEncodeTiled: CUresult %d", (int)r);
        return ARGUS_ERR_CUDA;
    }
    return ARGUS_OK;
}

template <typename T>
static bool dalloc(T** p, size_t n) {
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T)) == cudaSuccess;
}

extern "C" int argus_destroy(argus_ctx* c) {
    if (!c) return ARGUS_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    void* ps[] = {c->d_status, c->basis_img, c->basis_imgf, c->basis_h, c->basis_ab, c->basis_S, c->X, c->stamp_b,
                  c->rowmeta, c->design,
                  c->gram_part, c->M, c->L, c->Dinv, c->vec, c->resid_part, c->cell_key, c->label,
                  c->det_list, c->det_count, c->comp_key, c->comp_npix, c->comp_order,
                  c->row_count};
    for (void* p : ps)
        if (p) cudaFree(p);
    cudaSetDevice(prev);
    free(c);
    return ARGUS_OK;
}

extern "C" int argus_create(argus_ctx** out, int device, size_t max_pixels, int max_stamps,
                            int max_coeffs, int det_cap) {
    if (!out || max_pixels == 0 || max_stamps < 1 || max_coeffs < 2 || max_coeffs > 1008 ||
        det_cap < 1)
        return ARGUS_ERR_ARG;
    *out = NULL;
    if (cudaSetDevice(device) != cudaSuccess) return ARGUS_ERR_CUDA;
    argus_ctx* c = (argus_ctx*)calloc(1, sizeof(argus_ctx));
    if (!c) return ARGUS_ERR_NOMEM;
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->max_pixels = max_pixels;
    c->max_stamps = max_stamps;
    c->max_coeffs = max_coeffs;
    c->np_cols = argus_round_up(max_coeffs + 1, 16);
    c->det_cap = det_cap;
    c->gram_parts = 64;
    c->resid_parts = 512;
    c->max_cells = 4096;
    c->max_rows = (int)(max_pixels / 512 > 65536 ? (max_pixels / 512 > (1u << 26) ? (1u << 26) : max_pixels / 512) : 65536);
    const size_t np = (size_t)c->np_cols;
    bool ok = dalloc(&c->d_status, 4) &&
              dalloc(&c->basis_img, (size_t)ARGUS_MAX_NB * ARGUS_MAX_KS * ARGUS_MAX_KS) &&
              dalloc(&c->basis_imgf, (size_t)ARGUS_MAX_NB * ARGUS_MAX_KS * ARGUS_MAX_KS) &&
              dalloc(&c->basis_h, (size_t)ARGUS_MAX_NG * 16 * ARGUS_MAX_KS) &&
              dalloc(&c->basis_ab, (size_t)ARGUS_MAX_NB * 2) &&
              dalloc(&c->basis_S, (size_t)ARGUS_MAX_NB * ARGUS_MAX_NB) &&
              dalloc(&c->X, (size_t)max_stamps * ARGUS_MAX_STAMP * ARGUS_MAX_STAMP * ARGUS_MAX_NB) &&
              dalloc(&c->stamp_b, argus_stamp_conv_tc_bytes()) &&
              dalloc(&c->rowmeta, (size_t)max_stamps * ARGUS_MAX_STAMP * ARGUS_MAX_STAMP * 16) &&
              dalloc(&c->design, ((size_t)max_stamps * ARGUS_MAX_STAMP * ARGUS_MAX_STAMP + 32) * np) &&
              dalloc(&c->gram_part, (size_t)c->gram_parts * np * np) &&
              dalloc(&c->M, np * np) && dalloc(&c->L, np * np) &&
              dalloc(&c->Dinv, (np + 31) / 32 * 32 * 32) && dalloc(&c->vec, 8 * np) &&
              dalloc(&c->resid_part, (size_t)c->resid_parts * (np + 4)) &&
              dalloc(&c->cell_key, (size_t)c->max_cells) &&
              dalloc(&c->label, max_pixels) && dalloc(&c->det_list, (size_t)det_cap) &&
              dalloc(&c->det_count, 16) && dalloc(&c->comp_key, (size_t)det_cap) &&
              dalloc(&c->comp_npix, (size_t)det_cap) && dalloc(&c->comp_order, 2 * (size_t)det_cap) &&
              dalloc(&c->row_count, (size_t)c->max_rows * 2 + 2);
    if (!ok) {
        cudaGetLastError();
        argus_destroy(c);
        return ARGUS_ERR_NOMEM;
    }
    if (cudaMemset(c->d_status, 0, 4 * sizeof(int)) != cudaSuccess) {
        argus_destroy(c);
        return ARGUS_ERR_CUDA;
    }
    *out = c;
    return ARGUS_OK;
}

extern "C" int argus_sync_status(argus_ctx* c, argus_stream stream) {
    if (!c) return ARGUS_ERR_ARG;
    cudaSetDevice(c->device);
    int st = 0;
    if (cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return ARGUS_ERR_CUDA;
    if (st != 0 && cudaMemsetAsync(c->d_status, 0, sizeof(int), stream) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return ARGUS_ERR_CUDA;
    return st;
}
