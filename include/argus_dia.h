/*
 * argus_dia.h -- C ABI of the GB300 (sm_103a) difference-image-analysis path of
 * the Argus Array Hierarchical Data Processing System (Corbett et al. 2022,
 * "The sky at one terabit per second", arXiv:2207.14304).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Image pointers are DEVICE pointers owned by the caller, row-major with a
 *    row pitch given in ELEMENTS (argus_shape.pitch).  pitch >= w and
 *    pitch % 16 == 0, so rows of 1-, 2- and 4-byte images all start on a
 *    16-byte boundary; every image base pointer must be 16-byte aligned.
 *    Violations return ARGUS_ERR_ALIGN.  One pitch serves all images of a call.
 *  - Small parameter structs (argus_calib, argus_basis) are HOST structs; the
 *    arrays they point to are device arrays.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) and never allocates: scratch comes from the context made
 *    by argus_create.  A context must not be used from two streams at once.
 *  - Argument errors are returned synchronously.  Errors found on the device
 *    (singular normal matrix, detection capacity, spin-wait timeout) are
 *    latched in the context and returned by argus_sync_status.
 *  - Flag bits: ARGUS_FLAG_BAD (bad-pixel mask, or flat not a positive finite
 *    number), ARGUS_FLAG_SAT (raw >= saturation level).  A pixel with any flag
 *    is excluded from fits, clipping and detection.
 */
#ifndef ARGUS_DIA_H
#define ARGUS_DIA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct argus_ctx argus_ctx;
typedef struct CUstream_st *argus_stream; /* identical to cudaStream_t */

enum {
    ARGUS_OK = 0,
    ARGUS_ERR_ARG = -1,        /* invalid argument (host check) */
    ARGUS_ERR_ALIGN = -2,      /* pointer or pitch alignment */
    ARGUS_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    ARGUS_ERR_NOMEM = -4,      /* argus_create could not allocate */
    ARGUS_ERR_SINGULAR = -5,   /* Cholesky met a pivot <= 0 (device) */
    ARGUS_ERR_CAPACITY = -6,   /* an output or scratch list overflowed (device) */
    ARGUS_ERR_TIMEOUT = -7,    /* a bounded device wait expired (device) */
    ARGUS_ERR_UNSUPPORTED = -8 /* size outside the compiled kernel set */
};

/* Operand precision of the normal-equation Gram: FP32 (FP32 pipes); TF32 or
 * BF16 (each design value rounded once, tensor cores); BF16_SPLIT (each value
 * split into BF16 hi + lo, all four products hi*hi + hi*lo + lo*hi + lo*lo on the
 * tensor cores: the Gram of the design rounded to 16 significant bits).  The
 * tensor-core products accumulate in FP32 over at most 256 design rows, folded
 * into double-float sums. */
enum { ARGUS_PREC_FP32 = 0, ARGUS_PREC_TF32 = 1, ARGUS_PREC_BF16 = 2, ARGUS_PREC_BF16_SPLIT = 3 };
enum { ARGUS_FLAG_BAD = 1, ARGUS_FLAG_SAT = 2 };
enum { ARGUS_MASK_POS = 1, ARGUS_MASK_NEG = 2, ARGUS_MASK_INVALID = 4 };

typedef struct {
    int w, h;   /* image size in pixels */
    long pitch; /* row pitch in elements; pitch >= w, pitch % 16 == 0 */
} argus_shape;

/* Calibration frames of one camera (paper Sec. 3.2: darks, flats, bad-pixel
 * masks held on the GPU per pointing).  Device arrays use the image pitch. */
typedef struct {
    const uint16_t *bias_frame; /* nullable: per-pixel bias in ADU; else bias_scalar */
    int bias_scalar;            /* ADU */
    const float *dark;          /* nullable (= 0): electrons in the exposure */
    const float *flat;          /* nullable (= 1): relative response */
    const uint8_t *bpm;         /* nullable: nonzero = bad pixel */
    float gain;                 /* electrons per ADU */
    float read_noise;           /* electrons rms (Table 1: 1.7 e-) */
    int sat;                    /* raw level at and above which a pixel is SAT */
} argus_calib;

/* Alard-Lupton Gaussian basis:  B_{g,p,q}(u,v) = u^p v^q exp(-(u^2+v^2)/(2 sigma_g^2))
 * for g < ngauss, p + q <= degree[g], u,v in [-(ksize-1)/2, (ksize-1)/2], ordered
 * g, p, q.  B_0 is scaled to unit sum; every other function with p and q both
 * even has (sum B) B_0 removed, then each n >= 1 is scaled to unit L2 norm.
 * Spatial terms p_k(x,y) = xt^i yt^j (i + j <= degree, ordered i then j), with
 * xt = (2x - (W-1))/(W-1) over the frame width W (likewise yt).  Unknowns:
 * a_0 (B_0, constant term only), a_{n,k} (n >= 1, k < Ks), bg_k (k < Kb):
 * Nc = 1 + (nb-1) Ks + Kb.  Limits: ksize odd <= 31, ngauss <= 4, nb <= 64,
 * spatial_degree and bg_degree <= 2. */
typedef struct {
    int ksize;
    int ngauss;
    float sigma[4];
    int degree[4];
    int spatial_degree;
    int bg_degree;
} argus_basis;

/* One detected component (see argus_detect). */
typedef struct {
    float x, y;      /* Gaussian-windowed centroid (pixels) */
    float flux;      /* PSF-weighted optimal flux estimate (electrons) */
    float flux_err;  /* its 1-sigma error */
    float peak_snr;  /* signed S = D / sqrt(V_D) at the peak pixel */
    int npix;        /* pixels in the 8-connected component */
    int sign;        /* +1 positive, -1 negative */
    int px, py;      /* peak pixel */
} argus_source;

/* Device-side result record of argus_fit_kernel. */
typedef struct {
    double chi2;            /* sum w (I - C a)^2 over used stamp pixels */
    double chi2_a0;         /* the same before the refinement step */
    double max_step;        /* max |delta| / max |a| of the refinement */
    long long n_pix;        /* stamp pixels with nonzero weight */
    long long dof;          /* n_pix - Nc */
    int n_coeffs;           /* Nc */
    int status;             /* ARGUS_OK or ARGUS_ERR_SINGULAR */
    int n_stamps_used;      /* stamps whose window lay inside the frame */
    int precision;          /* ARGUS_PREC_* used for the Gram matrix */
    int refine_iters;       /* refinement steps applied */
    int pad_;
} argus_fit_stats;

/* Human-readable name of a status code. */
const char *argus_status_string(int status);

/* Text of the last CUDA runtime error that made a call of this host thread
 * return ARGUS_ERR_CUDA ("cudaErrorName: description"; "" if none). */
const char *argus_last_cuda_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (host-side tally, all contexts).  The difference of two readings counts
 * the kernels of the calls in between. */
unsigned long long argus_launch_count(void);

/* Create a context on `device` with scratch for frames of up to max_pixels
 * (h * pitch), up to max_stamps stamps of side <= 31, up to max_coeffs
 * unknowns and detection lists of up to det_cap pixels above threshold.
 * All scratch is allocated here, once (paper Sec. 4: calibration and
 * reference frames are pre-allocated on the GPU at the start of a pointing).
 * Returns ARGUS_OK and *out, or ARGUS_ERR_NOMEM / ARGUS_ERR_CUDA. */
int argus_create(argus_ctx **out, int device, size_t max_pixels, int max_stamps,
                 int max_coeffs, int det_cap);
int argus_destroy(argus_ctx *ctx);

/* Wait for `stream`, then return and clear the latched device status. */
int argus_sync_status(argus_ctx *ctx, argus_stream stream);

/* Calibration (paper Sec. 4.1: dark subtraction, flat fielding, bad-pixel
 * masking; Table 2 "Calibration").  Per pixel, n = raw - bias (integer),
 *   img = (n gain - dark) / flat,  var = (max(n gain, 0) + rn^2) / flat^2,
 *   flags = BAD | SAT as above; pixels with an unusable flat get img = var = 0.
 * raw: uint16 [h][pitch]; img, var: float [h][pitch]; flags: uint8 [h][pitch].
 * Only x < w is written. */
int argus_calibrate(argus_ctx *ctx, const uint16_t *raw, argus_shape shape,
                    const argus_calib *calib, float *img, float *var, uint8_t *flags,
                    argus_stream stream);

/* Sigma-clipped mean coadd of n raw frames (paper Sec. 4.1.3, deep coaddition;
 * a clipped mean stands in for the matched filter there).  raw_stack: uint16
 * [n][h][pitch]; shifts_xy: float [n][2] (device), frame f is sampled at
 * (x + dx_f, y + dy_f) by bilinear interpolation of its calibrated pixels;
 * clip: up to max_iter rounds of rejecting |v - median| > kappa * sigma
 * (population sigma about the mean); output coadd = c + sum(v - c)/n_used
 * about the final median c, var = sum V_f / n_used^2, n_used (uint8).
 * n <= 64.  Pixels with no valid sample get 0, 0, 0. */
int argus_coadd(argus_ctx *ctx, const uint16_t *raw_stack, int n, argus_shape shape,
                const float *shifts_xy, const argus_calib *calib, float kappa, int max_iter,
                float *coadd, float *var, uint8_t *n_used, argus_stream stream);

/* Stamp selection (deterministic grid rule; the paper gives none).  The frame
 * is cut into grid_x x grid_y cells; in each cell the brightest strict 3x3
 * local maximum of ref whose window [x-m, x+m]^2 (m = stamp/2 + khalf) is in
 * the frame and unflagged, whose value is < max_peak and which has no other
 * strict local maximum brighter than iso_frac times it within iso pixels
 * (Chebyshev).  Ties go to the lowest (y, x).  centers: int [grid_x*grid_y][2]
 * (x, y), cells in row-major order, compacted; *n_stamps (device int). */
int argus_select_stamps(argus_ctx *ctx, const float *ref, const uint8_t *flags, argus_shape shape,
                        int grid_x, int grid_y, int stamp, int khalf, float max_peak, int iso,
                        float iso_frac, int *centers, int *n_stamps, argus_stream stream);

/* Basis convolution on the stamps (the design values of the kernel fit below;
 * paper Sec. 4.2 direct image subtraction with the Alard-Lupton basis):
 *   X[(s * nb + m) * stamp^2 + j * stamp + i] =
 *       sum_{iv, iu} images[m][iv * ksize + iu] ref(x + r - iu, y + r - iv),
 *   (x, y) = centers[s] - (stamp/2, stamp/2) + (i, j),  r = ksize/2,
 * i.e. X_m = ref (x) image_m at stamp pixel (i, j); for s < min(*n_stamps, max_stamps),
 * X of the other stamps untouched; zero for stamps whose window, centers[s] +- (stamp/2 + r)
 * in x and y, leaves the frame.  ref: float [h][pitch]; centers: int [max_stamps][2] (x, y);
 * n_stamps: device int; images: float [nb][ksize^2] (device, 16-byte aligned), nb <= 64; X:
 * float [max_stamps][nb][stamp^2] (device, 16-byte aligned); all caller-owned.  Odd stamp <= 31,
 * odd ksize <= 31 and max_stamps <= the context's, else ARGUS_ERR_ARG; unaligned images or X:
 * ARGUS_ERR_ALIGN.  argus_fit_kernel runs the
 * same convolution on its orthonormalised basis.  21 x 21 stamps with 21 x 21
 * images run on the tensor cores (FP16 hi/lo operands with a power-of-two
 * scale per stamp and one for the images, three products, FP32 accumulation:
 * the FP32 product sums to ~1e-6 relative), the other shapes in FP32 on the
 * CUDA cores.  A stalled tensor-core pipeline latches ARGUS_ERR_TIMEOUT. */
int argus_stamp_basis(argus_ctx *ctx, const float *ref, argus_shape shape, const int *centers,
                      const int *n_stamps, int max_stamps, int stamp, const float *images, int nb,
                      int ksize, float *X, argus_stream stream);

/* PSF-matching kernel fit (Alard-Lupton least squares; the subtraction of
 * paper Sec. 4.2).  For every pixel of every stamp (side `stamp`, centres
 * centers[s], s < *n_stamps, at most max_stamps):
 *   row c = [X_0, p_k X_n (n>=1), p_k (background)], X_n = (ref (x) B_n)(x,y),
 *   weight w = 1/sci_var if flags == 0 and sci_var > 0, else 0;
 * M = C^T W C (operands in `precision`, ARGUS_PREC_*; FP32 accumulation over at
 * most 256 rows on the tensor cores), FP64 Cholesky on the GPU, a0 = M^-1 b, then one
 * refinement a = a0 + M^-1 C^T W (I - C a0) with C in FP32 and FP64 sums.
 * Stamps whose window leaves the frame are skipped.  coeffs: double [Nc]
 * (device); stats: argus_fit_stats (device).  A singular M latches
 * ARGUS_ERR_SINGULAR and leaves coeffs untouched. */
int argus_fit_kernel(argus_ctx *ctx, const float *sci, const float *sci_var, const float *ref,
                     const uint8_t *flags, argus_shape shape, const int *centers,
                     const int *n_stamps, int max_stamps, int stamp, const argus_basis *basis,
                     int precision, double *coeffs, argus_fit_stats *stats, argus_stream stream);

/* Kernel expansion: K_k(u,v) = sum_n a_{n,k} B_n(u,v) (K_0 also a_0 B_0) and the
 * background coefficients.  K: float [Ks][ksize][ksize] (device, index
 * (v+r)*ksize + (u+r)); bg: double [Kb] (device). */
int argus_expand_kernel(argus_ctx *ctx, const argus_basis *basis, const double *coeffs, float *K,
                        double *bg, argus_stream stream);

/* Convolution of the reference and subtraction (paper Sec. 4.2 / Table 2,
 * direct image subtraction) with the difference variance (noise maps,
 * Sec. 3.2):
 *   D   = sci - sum_k p_k(x,y) sum_{u,v} K_k(u,v) ref(x-u, y-v) - sum_k bg_k p_k(x,y)
 *   V_D = sci_var + sum_{u,v} Kc(u,v)^2 ref_var(x-u, y-v),
 * Kc = sum_k p_k(xc,yc) K_k at the centre of the 128x128 tile (frame
 * coordinates) holding (x,y).  Spatial terms use frame size (frame_w,
 * frame_h) and frame coordinates (x + ox, y + oy); with spatial_degree > 0,
 * ox and oy must be multiples of 32.  Pixels within r = ksize/2 of an image
 * edge, or with flags != 0, get D = V_D = 0.  K: float [Ks][ksize^2], bg:
 * double [Kb] (device).  ksize in {7, 9, 11, 15, 21}.  diff_var NULL: the
 * difference only; diff NULL: the variance only (sci and ref are then not
 * read); not both.  For 11x11 and 21x21 kernels D is computed on the tensor
 * cores (BF16 hi/lo operands, three products, FP32 accumulation; relative
 * error ~1e-6 of the convolved flux), and so is the variance when ox and oy
 * are multiples of 128 (one variance tile per 128x128 work strip); the
 * variance otherwise and the other kernel sizes run in FP32 on the CUDA
 * cores.  A stalled tensor-core pipeline latches ARGUS_ERR_TIMEOUT. */
int argus_subtract(argus_ctx *ctx, const float *sci, const float *sci_var, const float *ref,
                   const float *ref_var, const uint8_t *flags, argus_shape shape, int frame_w,
                   int frame_h, int ox, int oy, int ksize, int spatial_degree, const float *K,
                   int bg_degree, const double *bg, float *diff, float *diff_var,
                   argus_stream stream);

/* Detection on the difference image (paper Sec. 4.2 transient candidates,
 * Table 2 "Source detection"; a variance-weighted threshold):
 *   valid = flags == 0 && V_D > 0 && D, V_D finite;  S = D / sqrt(V_D) (float);
 *   mask = POS if S >= nsigma, NEG if S <= -nsigma, INVALID if not valid;
 * 8-connected components of equal sign; per component the peak (max |S|,
 * ties to the lowest (y,x)), npix, the Gaussian-windowed centroid (4 steps of
 * c += 2 sum t (p - c) / sum t, t = sign D exp(-|p-c|^2/(2 psf_sigma^2)), over
 * the valid pixels within ceil(3 psf_sigma) of the peak, clamped to peak +- 2)
 * and the optimal flux sum P D/V / sum P^2/V with P the unit-sum pixel-
 * integrated Gaussian at the centroid.  Sources are written sorted by (py, px),
 * at most cap; *n_found (device int) receives the total count; more than cap
 * latches ARGUS_ERR_CAPACITY.  mask: uint8 [h][pitch].  h may not exceed
 * max(65536, max_pixels / 512) of the context, and h * pitch < 2^31. */
int argus_detect(argus_ctx *ctx, const float *diff, const float *diff_var, const uint8_t *flags,
                 argus_shape shape, float nsigma, float psf_sigma, uint8_t *mask,
                 argus_source *out, int cap, int *n_found, argus_stream stream);

/* The whole per-frame reduction of one raw frame in one call (paper Sec. 4:
 * calibration, then the subtraction and detection of transient candidates of
 * Sec. 4.2; the frame stays on the GPU from the raw copy to the source list,
 * with reference and calibration frames resident per pointing, Sec. 3.2):
 *   argus_calibrate -> argus_select_stamps -> argus_fit_kernel ->
 *   argus_expand_kernel -> difference variance -> difference image -> detection,
 * with the same arguments and results as those calls made in turn, frame
 * coordinates equal to image coordinates (frame_w = w, ox = oy = 0) and
 * max_stamps = grid_x * grid_y.  One stream, no host round trip between the
 * steps; the call allocates nothing and can be captured in a CUDA graph.
 *   raw, calib: as argus_calibrate; ref, ref_var: the reference and its
 *     variance (float [h][pitch]);
 *   grid_x, grid_y, stamp, max_peak, iso, iso_frac: stamp selection (khalf =
 *     basis->ksize / 2); basis, precision: the fit; nsigma, psf_sigma: detection;
 *   outputs (device, caller-owned, all [h][pitch] unless stated): img, var,
 *     flags (calibrated frame); centers int [grid_x*grid_y][2], n_stamps int;
 *     coeffs double [Nc], stats (argus_fit_stats); K float [Ks][ksize][ksize],
 *     bg double [Kb]; diff, diff_var; mask uint8; out argus_source [cap],
 *     n_found int.
 * Returns the first error of the calls it makes (argument errors synchronously;
 * device-detected ones through argus_sync_status); nothing after a failing step
 * is enqueued. */
int argus_dia_frame(argus_ctx *ctx, const uint16_t *raw, argus_shape shape, const argus_calib *calib,
                    const float *ref, const float *ref_var, int grid_x, int grid_y, int stamp, float max_peak,
                    int iso, float iso_frac, const argus_basis *basis, int precision, float nsigma,
                    float psf_sigma, float *img, float *var, uint8_t *flags, int *centers, int *n_stamps,
                    double *coeffs, argus_fit_stats *stats, float *K, double *bg, float *diff, float *diff_var,
                    uint8_t *mask, argus_source *out, int cap, int *n_found, argus_stream stream);

/* ---------------------------------------------------------------------------
 * Batched segments (paper Sec. 5: subtraction parallelised over image
 * segments; Sec. 4.1.1: HEALPix segments).  Many square cutouts of uneven size
 * are stored in one "atlas": each quantity (science, variance, reference,
 * reference variance, flags, difference, difference variance, mask) is one
 * pitched image, segment s occupying rows [row0, row0 + side) and columns
 * [col0, col0 + side), row0 and col0 multiples of 16, no overlaps, side in
 * [ksize, 512].  Each segment gets its own spatially constant kernel fitted by
 * weighted least squares over every interior pixel (pixels at least ksize/2
 * from the segment edge), in the basis of argus_fit_kernel with
 * spatial_degree = bg_degree = 0; then subtraction with difference variance,
 * and 5-sigma style detection over the whole atlas (segment edges are
 * invalid, so components stay inside segments).  The work is cut into
 * fixed-size units (row bands of the fit, 32x32 tiles of the subtraction) that
 * persistent CTAs take from atomic counters, largest segments first. */
typedef struct {
    int row0, col0;   /* atlas position of the segment's pixel (0, 0) */
    int side;         /* square side in pixels */
} argus_segment;

/* Launch shape of the batched kernels (picked by the autotuner). */
typedef struct {
    int fit_band;          /* interior rows per fit work unit (8..128; even) of the tensor-core fit
                              (kernel sides <= 15); the CUDA-core fit (side 21) uses 8-row bands */
    int fit_ctas_per_sm;   /* persistent fit CTAs per SM (1..4) */
    int sub_ctas_per_sm;   /* persistent subtraction CTAs per SM (1..16) */
    int reserved;
} argus_seg_config;

/* Per-segment fit result (device). */
typedef struct {
    double chi2;   /* sum w (I - model)^2 over the interior, from the normal equations */
    int n_pix;     /* interior pixels with nonzero weight */
    int status;    /* ARGUS_OK or ARGUS_ERR_SINGULAR */
} argus_seg_stats;

typedef struct argus_seg_plan argus_seg_plan;

/* Build the work tables for a segment table (host array of n entries) in an
 * atlas of atlas_h rows and the given pitch, with launch shape cfg (NULL:
 * defaults).  This is a set-up call: it allocates the plan's device tables. */
int argus_segments_plan(argus_ctx *ctx, const argus_segment *table, int n, int pitch, int atlas_h,
                        const argus_basis *basis, const argus_seg_config *cfg, argus_seg_plan **out);
int argus_segments_destroy(argus_seg_plan *plan);

/* Run the batch: fit, solve, subtract, detect.  Atlas images as above (device,
 * same pitch); the caller keeps the atlas padding of diff/diff_var at zero.
 * coeffs: double [n][Nc] (Alard-Lupton order, background last); stats:
 * argus_seg_stats [n]; mask/out/n_found as in argus_detect (mask and n_found
 * may both be NULL to skip detection).  With use_graph != 0 the whole sequence
 * is recorded into a CUDA graph on the first call (and again whenever a
 * pointer or cap changes) and replayed with one graph launch. */
int argus_segments_run(argus_seg_plan *plan, const float *sci, const float *sci_var, const float *ref,
                       const float *ref_var, const uint8_t *flags, float *diff, float *diff_var,
                       uint8_t *mask, double *coeffs, argus_seg_stats *stats, float nsigma,
                       float psf_sigma, argus_source *out, int cap, int *n_found, int use_graph,
                       argus_stream stream);

/* Number of fit and subtraction work units of a plan. */
int argus_segments_items(const argus_seg_plan *plan, int *n_fit_items, int *n_sub_items);

/* Copy the kernels (float [n][ksize^2]) and backgrounds (double [n]) of the last
 * run to caller buffers (device; either may be NULL). */
int argus_segments_kernels(const argus_seg_plan *plan, float *K, double *bg, argus_stream stream);

/* The subtraction of argus_segments_run alone, with given kernels (device
 * float [n][ksize^2], row-major, the layout argus_segments_kernels returns)
 * and backgrounds (device double [n]) in place of fitted ones -- kernels kept
 * from an earlier exposure, or a reference's kernels in a test.  They replace
 * the plan's stored kernels.  Not graph-captured; no detection. */
int argus_segments_subtract(argus_seg_plan *plan, const float *sci, const float *sci_var, const float *ref,
                            const float *ref_var, const uint8_t *flags, const float *K, const double *bg,
                            float *diff, float *diff_var, argus_stream stream);

/* ---------------------------------------------------------------------------
 * Learned kernel surrogate (a learned stand-in for the least-squares kernel
 * fit, with the fit kept as fallback and judge; the paper has no counterpart).  A CNN maps a stamp pair (science and reference, 21x21, both
 * divided by the reference stamp sum) to a 21x21 kernel:
 *   h1 = W1 x + b1 (1x1, 2 -> 32); h_{l+1} = relu(conv7(h_l) + b_l) for four
 *   7x7 'same' 32 -> 32 layers; y = (W6 h5 + b6) / 441 (1x1, 32 -> 1; the fixed
 *   1/441 keeps the last layer's values at order one).
 * 200,961 parameters in the order W1[32][2], b1[32], {W[7][7][32 in][32 out],
 * b[32]} x 4, W6[32], b6, conv7 taps applied as
 * z[y][x][o] = b[o] + sum W[ky][kx][i][o] h[y+ky-3][x+kx-3][i] (zero padding).
 * Inputs x: float [n][441][2]; outputs y: float [n][441] (row-major kernel
 * pixels, index (v+10)*21 + (u+10)).  Weights are used as BF16 (default) or
 * FP32 with FP32 accumulation; training keeps FP32 master weights and Adam
 * moments.  The object owns its activation workspace for up to max_batch
 * stamps (allocated at creation). */
typedef struct argus_cnn argus_cnn;
int argus_cnn_create(argus_cnn **out, int device, int max_batch, unsigned long long seed);
int argus_cnn_destroy(argus_cnn *net);
/* Device pointers to the FP32 master parameters and Adam moments (each
 * [count] floats) and the Adam step, for checkpoints and tests. */
int argus_cnn_params(argus_cnn *net, float **master, float **adam_m, float **adam_v, long *count, int *step);
/* Select the arithmetic, set the Adam step, and refresh the BF16 copy from the
 * master weights (after a checkpoint load):
 *   ARGUS_PREC_FP32        FP32 weights, FP32 CUDA-core kernels;
 *   ARGUS_PREC_BF16        BF16 weights, FP32 activations, FP32 CUDA-core kernels;
 *   ARGUS_PREC_BF16_SPLIT  BF16 weights; the forward on the tensor cores
 *                          (tcgen05 implicit GEMMs, FP32 accumulation) with each
 *                          activation split into BF16 hi + lo parts (within
 *                          2^-17 relative of the FP32 value); the backward as
 *                          ARGUS_PREC_BF16.
 * The tensor-core forward's bounded device waits latch ARGUS_ERR_TIMEOUT, read
 * by argus_cnn_status. */
int argus_cnn_set_state(argus_cnn *net, int precision, int step, argus_stream stream);
int argus_cnn_forward(argus_cnn *net, const float *x, int n, float *y, argus_stream stream);
/* Synchronises the stream, returns the first error latched by the object's
 * kernels since the last call (ARGUS_OK if none) and clears it. */
int argus_cnn_status(argus_cnn *net, argus_stream stream);
/* dL/dparams for a given dL/dy after argus_cnn_forward on the same x (the
 * activations are kept); grad_out (device, [count] floats) may be NULL. */
int argus_cnn_backward(argus_cnn *net, const float *x, const float *dy, int n, float *grad_out,
                       argus_stream stream);
/* One training step: forward, MSE against target (float [n][441]), backward,
 * Adam (beta 0.9, 0.999, eps 1e-8) with learning rate lr; *loss_out (device
 * double, may be NULL) receives the batch loss. */
int argus_cnn_train_step(argus_cnn *net, const float *x, const float *target, int n, float lr,
                         double *loss_out, argus_stream stream);
/* One Adam step with a given gradient (device, [count] floats). */
int argus_cnn_adam(argus_cnn *net, const float *grad, float lr, argus_stream stream);
/* Network inputs from the 21x21 windows of sci and ref centred on centers[s]
 * (s < min(*n_stamps, max_stamps)): each window minus its sky (the mean of its
 * 80 border pixels), both divided by the sky-subtracted reference window sum
 * (0 when that sum is not positive).  x: float [n][441][2] (sci, ref). */
int argus_cnn_prepare(const float *sci, const float *ref, argus_shape shape, const int *centers,
                      const int *n_stamps, int max_stamps, float *x, argus_stream stream);
/* Spatial least squares across stamps: the per-stamp kernels y [n][441]
 * (at the stamp centres) give K_k (float [Ks][441]) with
 * y_s = sum_k p_k(x_s, y_s) K_k, normal matrix in FP64. */
int argus_learned_kernel(argus_ctx *ctx, const float *y, const int *centers, const int *n_stamps,
                         int max_stamps, int frame_w, int frame_h, int spatial_degree, float *K,
                         argus_stream stream);
/* Background polynomial given the kernel K (float [Ks][ksize^2]), by weighted
 * least squares on the stamp pixels, and chi2 of the result there:
 * r = I - sum_k p_k (R (x) K_k), bg = argmin sum w (r - sum pb bg)^2; the
 * model convolution in FP32, the normal-equation sums and the solve in FP64.
 * stats (device) receives chi2, n_pix, n_coeffs = Kb and dof = n_pix - Kb (the
 * kernel is not fitted to these pixels). */
int argus_fit_background(argus_ctx *ctx, const float *sci, const float *sci_var, const float *ref,
                         const uint8_t *flags, argus_shape shape, const int *centers, const int *n_stamps,
                         int max_stamps, int stamp, const float *K, int ksize, int spatial_degree,
                         int bg_degree, double *bg, argus_fit_stats *stats, argus_stream stream);
/* As argus_fit_background, with one amplitude per spatial term fitted jointly:
 * min sum w (I - sum_k alpha_k p_k (R (x) K_k) - sum pb bg)^2 over alpha and
 * bg; K (device, in/out) is then rescaled, K_k <- alpha_k K_k.  The kernel's
 * shape is the given one, its flux scale per spatial term is fitted.
 * n_coeffs = Ks + Kb, dof = n_pix - Ks - Kb. */
int argus_fit_scale_background(argus_ctx *ctx, const float *sci, const float *sci_var, const float *ref,
                               const uint8_t *flags, argus_shape shape, const int *centers,
                               const int *n_stamps, int max_stamps, int stamp, float *K, int ksize,
                               int spatial_degree, int bg_degree, double *bg, argus_fit_stats *stats,
                               argus_stream stream);

/* Stamp selection that allocates nothing, for callers that cannot call
 * cudaMalloc (a host that reserves all device memory up front, a real-time
 * loop that must never enter an allocator, or a plugin that is only handed
 * input and output pointers).  The paper has no counterpart: this is a
 * deployment variant of argus_select_stamps with the same arguments minus the
 * context and the same results.  Its scratch (one 64-bit key per grid cell)
 * is a fixed 32 KiB device array inside the library that every GPU loading the
 * library keeps until the process exits; grid_x * grid_y above
 * ARGUS_NOALLOC_MAX_CELLS (4096) returns ARGUS_ERR_CAPACITY.  Runs on the
 * current device.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  That address is kept until the process exits, so the entry point
 * must not be called after a reset of the device (cudaDeviceReset or a torn-
 * down primary context).  All calls share the array, so calls that overlap on the GPU race
 * and must be serialised by the caller; each call clears the part it uses.
 * ref, flags: device, [h][pitch]; centers: device int [grid_x*grid_y][2];
 * n_stamps: device int. */
#define ARGUS_NOALLOC_MAX_CELLS 4096
int argus_select_stamps_noalloc(const float *ref, const uint8_t *flags, argus_shape shape, int grid_x,
                                int grid_y, int stamp, int khalf, float max_peak, int iso, float iso_frac,
                                int *centers, int *n_stamps, argus_stream stream);

/* ---------------------------------------------------------------------------
 * Sparse and low-resolution segment products (paper Sec. 3.3 "Sparse Image
 * Segments"; Sec. 2, data products 1c and 1d).
 *
 * Minipix stamping: the image is cut into square cells of cell x cell pixels
 * (the minipix of a segment; ncx = ceil(w / cell), ncy = ceil(h / cell), cell
 * (cx, cy) holding pixels [cx cell, cx cell + cell) x [cy cell, cy cell + cell)
 * clipped to the image).  A cell is kept when a science target lies in it:
 * the catalogue targets (device int [n_targets][2], pixel (x, y)) and the
 * peak pixels (px, py) of the first min(*n_sources, sources_cap) records of a
 * detection list (device argus_source array and device count, as written by
 * argus_detect; sources may be NULL with sources_cap 0).  Targets outside the
 * image are ignored.  Every pixel of a cell that is not kept is set to 0.
 *   keep:       device uint8 [ncy][ncx] (no pitch), 1 = kept, 0 = zeroed.
 *   out:        nullable, device float [h][pitch]: img where kept, else 0;
 *               columns w .. pitch-1 are set to 0.  May not alias img.
 *   packed:     nullable, device float [cap][cell * cell]: the kept cells in
 *               ascending cell index cy * ncx + cx, each row-major, pixels
 *               outside the image 0;  cell_index: device int [cap], the cell
 *               index of each packed cell (nullable only with packed NULL).
 *   n_kept:     device int, the number of kept cells; more than cap latches
 *               ARGUS_ERR_CAPACITY and only the first cap are packed.
 * 1 <= cell <= 256; n_targets >= 0.  Results are exact copies (bit-exact). */
int argus_minipix(argus_ctx *ctx, const float *img, argus_shape shape, int cell, const int *targets,
                  int n_targets, const argus_source *sources, const int *n_sources, int sources_cap,
                  uint8_t *keep, float *out, float *packed, int *cell_index, int cap, int *n_kept,
                  argus_stream stream);

/* Low-resolution map (paper Sec. 2, product 1d: 10x reduced resolution,
 * 13.8 arcsec per pixel): out[Y][X] = mean of the valid pixels of the factor x
 * factor block starting at (factor X, factor Y), valid = flags == 0 (flags
 * nullable: all pixels) and the value finite; partial blocks at the right and
 * bottom edges average the pixels they hold; 0 where a block has none.  out:
 * device float [ceil(h / factor)][out_pitch], out_pitch >= ceil(w / factor),
 * 16-byte aligned.  Sums are FP32 (column sums of factor pixels, then factor
 * column sums), so |out - exact| <= (2 factor + 1) 2^-24 mean|v| over the
 * block.  1 <= factor <= 64. */
int argus_lowres(argus_ctx *ctx, const float *img, const uint8_t *flags, argus_shape shape, int factor,
                 float *out, long out_pitch, argus_stream stream);

/* Median-filtered background map (paper Table 2, GPU stage "Median-filtered
 * background map"; background maps kept with the calibration frames, Sec. 3.2).
 * The paper names the map only; this is the mesh estimate:
 *   1. boxes of box x box pixels from (0, 0), ncx = ceil(w / box) by
 *      ncy = ceil(h / box); edge boxes hold the pixels that exist;
 *   2. each box's value is the median of its valid pixels (flags == 0 where
 *      flags are given, and finite; an even count takes the mean of the two
 *      middle values, in FP64, so the value is exact); a box whose valid count
 *      is below min_frac (compared in float) of its pixels has no value;
 *   3. mesh (device double [ncy][ncx], 8-byte aligned) receives the median of
 *      the values that exist in each box's filt x filt neighbourhood of boxes,
 *      clipped at the mesh edges; a box with none in reach takes the median of
 *      all box values (0 if no box has one);
 *   4. map (nullable, device float [h][pitch]) receives the bilinear
 *      interpolation of the mesh between box centres (the mean pixel coordinate
 *      of each box), constant beyond the outermost centres, in FP32; columns
 *      w .. pitch-1 are set to 0.
 * 8 <= box <= 64; filt odd, 1 <= filt <= 7; 0 <= min_frac <= 1. */
int argus_background(argus_ctx *ctx, const float *img, const uint8_t *flags, argus_shape shape, int box,
                     int filt, float min_frac, double *mesh, float *map, argus_stream stream);

/* ---------------------------------------------------------------------------
 * Proper-image statistics on square tiles: ZOGY subtraction and proper
 * coaddition share one plan (transform buffers, 48 bytes per tile pixel, and
 * the twiddle tables of one tile size).
 *
 * ZOGY proper image subtraction on square tiles (paper Sec. 4.2: ZOGY for
 * base cadence and deep coadds; the statistic of Zackay, Ofek & Gal-Yam 2016).
 * Each tile is T x T pixels of the new image N and the registered reference R
 * (background-subtracted; pixels off the frame are 0), taken as periodic.
 * With hats for unnormalised 2-D DFTs and the PSF stamps placed with their
 * centre at pixel (0, 0) (wrapping around):
 *   den = sqrt(sn^2 Fr^2 |Pr|^2 + sr^2 Fn^2 |Pn|^2),   F_D = Fr Fn / sqrt(sn^2 Fr^2 + sr^2 Fn^2)
 *   D   = IDFT[(Fr Pr N - Fn Pn R) / den]        proper difference, unit-variance white noise
 *   P_D = IDFT[Fr Fn Pr Pn / (F_D den)]          its PSF (unit sum)
 *   S   = IDFT[F_D D conj(P_D)]                  point-source score, per-pixel sigma_S = F_D ||P_D||_2
 * with D, P_D and S set to 0 at frequencies where max(|Pn|, |Pr|) < eps (the
 * PSFs have unit sum; below the floor their transforms are rounding; 1e-8 is
 * the reference value).  Images and the pointwise step are FP32, the PSF
 * transforms FP64. */
typedef struct argus_proper_plan argus_proper_plan;

typedef struct {
    int x0, y0;      /* frame position of the tile's pixel (0, 0) */
    float Fn, Fr;    /* flux zero points of the new image and the reference */
    float sn, sr;    /* their background noise (standard deviation per pixel) */
} argus_zogy_tile;

/* tile in {256, 512, 1024}; 1 <= max_tiles <= 65536.  Allocates on `device`. */
int argus_proper_plan_create(int device, int tile, int max_tiles, argus_proper_plan **plan);
int argus_proper_plan_destroy(argus_proper_plan *plan);

/* N, R: device float [h][pitch] (one shape); tiles: device argus_zogy_tile
 * [n_tiles]; psf_n, psf_r: device float [n_tiles][psf_size][psf_size] with
 * psf_per_tile = 1, or one pair [psf_size][psf_size] shared by every tile with
 * psf_per_tile = 0 (one FP64 transform instead of n_tiles); odd psf_size <= 63;
 * or both NULL to reuse the PSF transforms of the last call on this plan that
 * gave PSFs (PSFs change per pointing, frames per exposure; the FP64 transforms
 * are the costliest part of a call) -- with the same psf_per_tile, n_tiles not
 * above that call's, and no proper-coadd call in between (it discards them);
 * D, S and P_D (nullable): device float [n_tiles][T][T]; sigma_S (nullable):
 * device double [n_tiles].  1 <= n_tiles <= max_tiles.  Calls on one plan must
 * not overlap. */
int argus_zogy(argus_proper_plan *plan, const float *N, const float *R, argus_shape shape,
               const argus_zogy_tile *tiles, int n_tiles, const float *psf_n, const float *psf_r,
               int psf_size, int psf_per_tile, float eps, float *D, float *S, float *P_D,
               double *sigma_S, argus_stream stream);

/* Proper coaddition (paper Sec. 4.1.3: per-image matched filtering of
 * pre-aligned tiles; the statistic of Zackay & Ofek 2017) on the tiles of a
 * stack of registered, background-subtracted frames M_j with PSFs P_j (per
 * tile and frame), zero points F_j and background noise s_j:
 *   S   = IDFT[sum_j (F_j / s_j^2) conj(P_j) M_j]      score coadd (the matched-filter sum)
 *   den = sqrt(sum_j F_j^2 / s_j^2 |P_j|^2),   F_R = sqrt(sum_j F_j^2 / s_j^2)
 *   R   = IDFT[S / den]                            proper coadd, unit-variance white noise
 *   P_R = IDFT[den / F_R]                          its PSF (unit sum)
 * with R and P_R 0 at frequencies where max_j |P_j| < eps (S keeps every
 * frequency); sigma_S = sqrt(sum_j F_j^2 / s_j^2 sum P_j^2) per tile.
 * stack: device float [n_frames][h][pitch] (one shape; pixels off the frame
 * are 0); origins: device int [n_tiles][2] (tile pixel (0, 0) in the frame);
 * F, sigma: device float [n_frames] (a frame with sigma <= 0 is left out);
 * psfs: device float [n_tiles][n_frames][psf_size][psf_size] with
 * psf_per_tile = 1, or [n_frames][psf_size][psf_size] shared by every tile with
 * psf_per_tile = 0 (one FP64 transform per frame instead of one per tile and
 * frame); odd psf_size <= 63; S, R, P_R (nullable): device float [n_tiles][T][T]; F_R (nullable):
 * device double [1]; sigma_S (nullable): device double [n_tiles].
 * 1 <= n_frames <= 64.  Frames go through the transforms in pairs. */
int argus_proper_coadd(argus_proper_plan *plan, const float *stack, int n_frames, argus_shape shape,
                       const int *origins, int n_tiles, const float *F, const float *sigma, const float *psfs,
                       int psf_size, int psf_per_tile, float eps, float *S, float *R, float *P_R, double *F_R,
                       double *sigma_S, argus_stream stream);

/* ---------------------------------------------------------------------------
 * HEALPix segmentation (paper Sec. 3.3 "Image Segmentation": frames are
 * reprojected into HEALPix NSIDE=256 segments; Table 2, GPU stage "Image
 * segmentation and resampling to HEALPix grid").  A segment is one nested
 * HEALPix pixel at nside_seg; its image is the 2^k x 2^k grid of the pixels at
 * NSIDE nside_seg 2^k inside it: image column c, row r is face pixel
 * (X 2^k + c, Y 2^k + r), (X, Y) the segment's face coordinates (ix from the
 * even bits of the in-face nested index, iy from the odd bits).  Each image
 * pixel takes the frame value at its pixel centre through the gnomonic WCS
 * below, by bilinear interpolation written as nested lerps; it is covered
 * when the position lies in [0, w-1] x [0, h-1] and every neighbour with a
 * nonzero weight is unflagged and finite, else 0 with coverage 0.  Geometry
 * in FP64, output FP32. */
typedef struct {
    double alpha0, delta0;   /* tangent point (radians) */
    double scale;            /* radians per pixel */
    double rot;              /* x = cx + (cos rot xi + sin rot eta) / scale,
                                y = cy + (-sin rot xi + cos rot eta) / scale,
                                xi east, eta north in the tangent plane */
    double cx, cy;           /* pixel coordinates of the tangent point */
} argus_wcs;

/* frame, flags (nullable): device [h][pitch]; segs: device int64 [n_seg] nested
 * indices at nside_seg (a power of two <= 2^17, nside_seg 2^k <= 2^29, k <= 12;
 * an index outside 0 .. 12 nside_seg^2 - 1 gives an uncovered image);
 * out: device float [n_seg][2^k][2^k]; coverage (nullable): device uint8, same.
 * Runs on the current device; needs no context.  For k >= 6, rows wholly in
 * the equatorial belt take positions from cubics through exact positions at
 * four nodes of each 64-pixel piece (within a few 1e-8 pixel of the exact
 * map); other rows are exact per pixel. */
int argus_healpix_resample(const float *frame, const uint8_t *flags, argus_shape shape, argus_wcs wcs,
                           int nside_seg, int k, const long long *segs, int n_seg, float *out,
                           uint8_t *coverage, argus_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* ARGUS_DIA_H */
