// One call for the per-frame difference imaging of a raw sensor frame (paper
// Sec. 4: calibration, then subtraction and detection of transient candidates,
// Sec. 4.2; the frame stays on the GPU from the raw copy to the source list,
// as the paper's GPU residency of Sec. 3.2 keeps references and calibrations
// there per pointing):
//
//   raw -> calibrate -> stamp selection -> kernel fit -> kernel expansion
//       -> difference variance -> difference image -> detection.
//
// It enqueues the same kernels as the separate calls, in this order, on one
// stream, with no host round trip in between (the whole call can be captured
// in one CUDA graph).  A variant that computed the detection threshold inside
// the tensor-core difference-image kernel (reading V_D beside I and the flags,
// writing the mask and listing the pixels above threshold) gave bit-identical
// outputs but a frame 8.5 % slower: that kernel's epilogue warps already keep
// pace with its MMAs only just, while the separate threshold pass streams
// 10 bytes per pixel at the memory roof (about 0.09 ms per frame).
#include "argus_internal.cuh"

extern "C" int argus_dia_frame(argus_ctx* ctx, const uint16_t* raw, argus_shape shape, const argus_calib* calib,
                               const float* ref, const float* ref_var, int grid_x, int grid_y, int stamp,
                               float max_peak, int iso, float iso_frac, const argus_basis* basis, int precision,
                               float nsigma, float psf_sigma, float* img, float* var, uint8_t* flags, int* centers,
                               int* n_stamps, double* coeffs, argus_fit_stats* stats, float* K, double* bg,
                               float* diff, float* diff_var, uint8_t* mask, argus_source* out, int cap,
                               int* n_found, argus_stream stream) {
    if (!ctx || !raw || !calib || !ref || !ref_var || !basis || !img || !var || !flags || !centers || !n_stamps ||
        !coeffs || !stats || !K || !bg || !diff || !diff_var || !mask || !n_found || (cap > 0 && !out) || cap < 0)
        return ARGUS_ERR_ARG;
    if (grid_x < 1 || grid_y < 1) return ARGUS_ERR_ARG;
    const int ks = basis->ksize, sdeg = basis->spatial_degree, bgdeg = basis->bg_degree;
    int rc = argus_calibrate(ctx, raw, shape, calib, img, var, flags, stream);
    if (!rc) rc = argus_select_stamps(ctx, ref, flags, shape, grid_x, grid_y, stamp, ks / 2, max_peak, iso, iso_frac,
                                      centers, n_stamps, stream);
    if (!rc) rc = argus_fit_kernel(ctx, img, var, ref, flags, shape, centers, n_stamps, grid_x * grid_y, stamp,
                                   basis, precision, coeffs, stats, stream);
    if (!rc) rc = argus_expand_kernel(ctx, basis, coeffs, K, bg, stream);
    if (!rc) rc = argus_subtract(ctx, img, var, ref, ref_var, flags, shape, shape.w, shape.h, 0, 0, ks, sdeg, K, bgdeg,
                                 bg, diff, diff_var, stream);
    if (!rc) rc = argus_detect(ctx, diff, diff_var, flags, shape, nsigma, psf_sigma, mask, out, cap, n_found, stream);
    return rc;
}
