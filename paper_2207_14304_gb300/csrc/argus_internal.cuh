// Internal declarations shared by the sm_103a translation units of libargusdia.
#pragma once

#include <cuda.h>   // CUtensorMap
#include <cuda_runtime.h>
#include <stdint.h>

#include "argus_dia.h"

// Limits of the compiled kernel set.
#define ARGUS_MAX_KS 31          // kernel side
#define ARGUS_MAX_NB 64          // basis functions
#define ARGUS_MAX_NG 4           // Gaussians
#define ARGUS_MAX_TERMS 6        // spatial terms (degree 2)
#define ARGUS_MAX_STAMP 31       // stamp side
#define ARGUS_MAX_FRAMES 64      // coadd stack depth
#define ARGUS_GRAM_KCHUNK 32     // design rows per Gram pipeline stage

struct argus_ctx {
    int device;
    int num_sms;
    size_t max_pixels;
    int max_stamps;
    int max_coeffs;   // Nc limit
    int np_cols;      // padded Gram width: round_up(max_coeffs + 1, 16)
    int det_cap;
    int* d_status;    // latched device status word

    // basis tables (rebuilt per call from the host basis spec)
    double* basis_img;   // [nb][ks*ks] FP64 normalised basis
    float* basis_imgf;   // [nb][ks*ks] FP32 orthonormalised images (B'_0 = B_0)
    double* basis_S;     // [nb][nb] B'_m = sum_n S[n][m] B_n (n, m >= 1), upper triangular
    float* basis_h;      // [ngauss*9][ks] 1-D factors u^p exp(-u^2/2s^2)
    float* basis_ab;     // [nb][2] alpha, beta: B_n = alpha (h_p x h_q) - beta B_0

    // fit scratch
    float* X;            // [max_stamps * 31*31][64] basis-convolved stamp pixels
    uint8_t* stamp_b;    // argus_stamp_conv_tc_bytes(): packed FP16 basis operands of the tensor-core stamp convolution
    float* rowmeta;      // [max_stamps * 31*31][16] per-row design weights of the fit
    float* design;       // [max_stamps * 31*31 rounded up to 32][np_cols] weighted design matrix (FP32)
    int gram_parts;      // number of partial Gram slots
    float* gram_part;    // [gram_parts][np_cols][np_cols]
    double* M;           // [np_cols][np_cols] reduced normal matrix (+ target column)
    double* L;           // [np_cols][np_cols] Cholesky factor
    double* Dinv;        // [np_cols / 32][32][32] inverses of the 32 x 32 diagonal blocks of L
    double* vec;         // [8][np_cols] b, a0, r, delta, a, work
    int resid_parts;
    double* resid_part;  // [resid_parts][np_cols + 2]

    // stamp selection scratch
    unsigned long long* cell_key;   // [max cells] best candidate key per cell
    int max_cells;

    // memo of the last basis tables built (host copy of the spec)
    argus_basis basis_memo;
    int basis_memo_valid;

    // detection scratch
    int* label;          // [max_pixels]
    int* det_list;       // [det_cap]
    int* det_count;      // [8] counters
    unsigned long long* comp_key;  // [det_cap]
    int* comp_npix;      // [det_cap]
    int* comp_order;     // [det_cap]
    int* row_count;      // [max_rows + 1]
    int max_rows;
};

// Device-side error latch: the first error wins.
__device__ __forceinline__ void argus_latch(int* st, int code) { atomicCAS(st, 0, code); }

// Host helpers (api.cu)
int argus_check_shape(const argus_shape& s, size_t max_pixels);
int argus_check_ptr16(const void* p);
int argus_launch_status();   // ARGUS_OK or ARGUS_ERR_CUDA after a launch
int argus_cuda_fail(cudaError_t e);   // records e for argus_last_cuda_error, returns ARGUS_ERR_CUDA
void argus_count_launch(int n);   // host-side tally of kernel launches
// Tensor map of a pitched 2-D image of w x h elements of esize bytes (row pitch
// in elements) for tiled TMA copies of bx x by boxes, zero fill outside the
// image; ARGUS_ERR_CUDA when the driver rejects it (the reason goes to
// argus_last_cuda_error).  Host only, no device work (legal during stream capture).
int argus_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, int esize, const void* base, long w, long h, long pitch,
                  int bx, int by);
extern "C" unsigned long long argus_launch_count(void);

// Inter-unit launchers
int argus_basis_prepare(argus_ctx* ctx, const argus_basis* b, cudaStream_t st);
int argus_cholesky_solve_prepare(argus_ctx* ctx, const double* M, int ld, int n, cudaStream_t st);
void argus_tri_solve(argus_ctx* ctx, int ld, int n, const double* rhs, int rs, double* x, cudaStream_t st);
int argus_basis_count(const argus_basis* b);
int argus_nterms(int deg);
// the learned kernel's forward on the tensor cores (cnn_tc.cu): wbf the BF16
// parameter vector, wpack argus_cnn_tc_pack_bytes() of scratch for the packed
// weights, acts (optional) the FP32 activations h1..h5 at acts + l * lstride
int argus_cnn_forward_tc(const float* x, const void* wbf, void* wpack, int n, float* y, float* acts, long lstride,
                         int num_sms, int* status, cudaStream_t st);
size_t argus_cnn_tc_pack_bytes();
// the data gradient of 7x7 layer `layer` on the tensor cores (cnn_tc.cu): dh_in =
// conv^T(dh_out (h_out > 0)); wpack receives the layer's packed transposed kernel
int argus_cnn_dgrad_tc(const float* dh_out, const float* h_out, const void* wbf, void* wpack, int layer, int n,
                       float* dh_in, int num_sms, int* status, cudaStream_t st);

// the basis convolution of 21 x 21 stamps with up to 64 images of 21 x 21 taps on
// the tensor cores (stamp_conv_tc.cu): X[(s nb + m) 441 + pix] = (ref (x) img_m) on
// stamp s < min(*n_stamps, max_stamps), zero where the stamp's window leaves the
// frame; bpack receives argus_stamp_conv_tc_bytes() of packed basis operands
int argus_stamp_conv_tc(const float* ref, long pitch, int w, int h, const int* centers, const int* n_stamps,
                        int max_stamps, const float* img, int nb, uint8_t* bpack, float* X, int num_sms, int* status,
                        cudaStream_t st);
size_t argus_stamp_conv_tc_bytes();

static inline int argus_round_up(int a, int m) { return (a + m - 1) / m * m; }
