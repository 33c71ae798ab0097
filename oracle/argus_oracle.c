/*
 * argus_oracle.c -- plain, slow, FP64 CPU oracle of the Argus-HDPS difference
 * imaging hot path (Corbett et al. 2022, "The sky at one terabit per second").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; it shares no code, header, table or constant generator with
 * the CUDA path.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline may load it.
 *
 * The paper names the steps (calibration: dark subtraction, flat fielding and
 * bad-pixel masking, Sec. 4.1 "Image Management"; GPU-resident calibration and
 * noise maps, Sec. 3.2 "Compute Nodes"; coaddition, Sec. 4.1.3; direct image
 * subtraction and transient detection, Sec. 4.2 "Transient Alerts" and Table 2;
 * minipix stamping and low-resolution maps, Sec. 3.3 "Sparse Image Segments")
 * but prints no formula for any of them.  Each function below states the
 * definition it computes.  Where the paper leaves the method open, the
 * Alard & Lupton (1998) / Alard (2000) Gaussian-basis least-squares kernel fit
 * defines subtraction and a per-pixel S/N threshold defines detection; these
 * readings are listed in the design notes.
 *
 * Everything is written as direct loops in index order: no FFT, no separable
 * factorisation, no blocking.  OpenMP parallelises over independent output
 * rows / stamps only; per-output arithmetic order is fixed, so results do not
 * depend on the thread count.
 *
 * Flag bits (interface values): 1 BAD, 2 SAT.  Detection mask bits: 1 = S >= +n,
 * 2 = S <= -n, 4 = invalid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_BAD 1
#define ORA_SAT 2
#define ORA_MPOS 1
#define ORA_MNEG 2
#define ORA_MINV 4

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Calibration (Sec. 4.1: dark subtraction, flat fielding, bad-pixel masks;  */
/* Sec. 3.2: per-camera calibration frames; Table 1: 1.7 e- read noise).    */
/*   n = raw - bias            (integer)                                     */
/*   I = (n*gain - dark) / flat                                              */
/*   V = (max(n*gain, 0) + rn^2) / flat^2                                    */
/*   flags: BAD if bpm != 0 or flat is not a positive finite number,         */
/*          SAT if raw >= sat.  Pixels with an unusable flat get I = V = 0.  */
/* ------------------------------------------------------------------------ */
void ora_calibrate(int w, int h, const uint16_t *raw, const uint16_t *bias_frame,
                   int bias_scalar, const float *dark, const float *flat,
                   const uint8_t *bpm, double gain, double rn, int sat,
                   double *img, double *var, uint8_t *flags, int32_t *n_out) {
    long np = (long)w * h;
    for (long i = 0; i < np; i++) {
        int32_t n = (int32_t)raw[i] - (bias_frame ? (int32_t)bias_frame[i] : bias_scalar);
        uint8_t f = 0;
        double fl = flat ? (double)flat[i] : 1.0;
        int flat_ok = (fl > 0.0) && isfinite(fl);
        if ((bpm && bpm[i]) || !flat_ok) f |= ORA_BAD;
        if ((int)raw[i] >= sat) f |= ORA_SAT;
        double d = dark ? (double)dark[i] : 0.0;
        double ng = (double)n * gain;
        if (flat_ok) {
            img[i] = (ng - d) / fl;
            var[i] = ((ng > 0.0 ? ng : 0.0) + rn * rn) / (fl * fl);
        } else {
            img[i] = 0.0;
            var[i] = 0.0;
        }
        flags[i] = f;
        if (n_out) n_out[i] = n;
    }
}

/* ------------------------------------------------------------------------ */
/* Alard-Lupton Gaussian basis (the fit the subtraction reading adopts).     */
/*   B_{g,p,q}(u,v) = u^p v^q exp(-(u^2+v^2) / (2 sigma_g^2)),  u,v in [-r,r] */
/* ordered g, then p = 0..deg_g, then q = 0..deg_g - p.                       */
/* B_0 (g=0,p=q=0) is scaled to unit sum and carries the photometric scale.  */
/* Every other function with both p and q even has (sum B) * B_0 removed so  */
/* that it sums to zero (Alard 2000); each n >= 1 is then scaled to unit L2.  */
/* Storage: B[n*ks*ks + (v+r)*ks + (u+r)].                                   */
/* ------------------------------------------------------------------------ */
int ora_basis_count(int ngauss, const int *degree) {
    int n = 0;
    for (int g = 0; g < ngauss; g++) n += (degree[g] + 1) * (degree[g] + 2) / 2;
    return n;
}

int ora_basis(int ks, int ngauss, const double *sigma, const int *degree, double *B,
              int *pq_out) {
    int r = (ks - 1) / 2, kk = ks * ks, n = 0;
    for (int g = 0; g < ngauss; g++) {
        double s2 = 2.0 * sigma[g] * sigma[g];
        for (int p = 0; p <= degree[g]; p++)
            for (int q = 0; q <= degree[g] - p; q++) {
                double *b = B + (long)n * kk;
                for (int v = -r; v <= r; v++)
                    for (int u = -r; u <= r; u++)
                        b[(v + r) * ks + (u + r)] =
                            pow((double)u, p) * pow((double)v, q) * exp(-(double)(u * u + v * v) / s2);
                if (pq_out) { pq_out[3 * n] = g; pq_out[3 * n + 1] = p; pq_out[3 * n + 2] = q; }
                n++;
            }
    }
    double s0 = 0.0;
    for (int i = 0; i < kk; i++) s0 += B[i];
    for (int i = 0; i < kk; i++) B[i] /= s0;
    n = 0;
    for (int g = 0; g < ngauss; g++)
        for (int p = 0; p <= degree[g]; p++)
            for (int q = 0; q <= degree[g] - p; q++) {
                if (n > 0) {
                    double *b = B + (long)n * kk;
                    if (p % 2 == 0 && q % 2 == 0) {
                        double s = 0.0;
                        for (int i = 0; i < kk; i++) s += b[i];
                        for (int i = 0; i < kk; i++) b[i] -= s * B[i];
                    }
                    double nn = 0.0;
                    for (int i = 0; i < kk; i++) nn += b[i] * b[i];
                    nn = sqrt(nn);
                    for (int i = 0; i < kk; i++) b[i] /= nn;
                }
                n++;
            }
    return n;
}

/* Spatial monomials p_k(x,y) = xt^i yt^j, i+j <= deg, ordered i then j,     */
/* with xt = (2x - (W-1)) / (W-1) in [-1, 1] (0 if W == 1), same for y.      */
int ora_nterms(int deg) { return deg < 0 ? 0 : (deg + 1) * (deg + 2) / 2; }

void ora_spatial_terms(double x, double y, int W, int H, int deg, double *out) {
    double xt = W > 1 ? (2.0 * x - (W - 1)) / (double)(W - 1) : 0.0;
    double yt = H > 1 ? (2.0 * y - (H - 1)) / (double)(H - 1) : 0.0;
    int k = 0;
    for (int i = 0; i <= deg; i++)
        for (int j = 0; j <= deg - i; j++) out[k++] = pow(xt, i) * pow(yt, j);
}

/* Number of unknowns: B_0 takes only the constant spatial term, every other */
/* basis function all Ks terms, then Kb background terms.                    */
int ora_ncoeffs(int nb, int sdeg, int bgdeg) {
    return 1 + (nb - 1) * ora_nterms(sdeg) + ora_nterms(bgdeg);
}

/* ------------------------------------------------------------------------ */
/* Stamp selection (deterministic reading; the paper gives no rule).         */
/* The frame is cut into gx x gy cells (cell cx spans x in                   */
/* [cx*W/gx, (cx+1)*W/gx), integer division).  In each cell the pixel with   */
/* the largest R is taken among pixels that                                  */
/*   - are strict maxima of their 3x3 neighbourhood,                         */
/*   - have the window [x-h-r, x+h+r]^2 inside the frame and unflagged,      */
/*   - have R < max_peak,                                                    */
/*   - have no other strict local maximum brighter than iso_frac * R within  */
/*     iso pixels (Chebyshev distance).                                      */
/* Ties go to the lowest (y, x).  Thresholds are evaluated in float.        */
/* ------------------------------------------------------------------------ */
static int is_lmax(const float *R, int w, int h, int x, int y) {
    if (x < 1 || y < 1 || x > w - 2 || y > h - 2) return 0;
    float c = R[(long)y * w + x];
    if (!isfinite(c)) return 0;
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            if (!dx && !dy) continue;
            if (!(c > R[(long)(y + dy) * w + x + dx])) return 0;
        }
    return 1;
}

int ora_select_stamps(int w, int h, const float *R, const uint8_t *flags, int gx, int gy,
                      int stamp, int khalf, float max_peak, int iso, float iso_frac,
                      int *centers) {
    int hs = stamp / 2, m = hs + khalf, n = 0;
    for (int cy = 0; cy < gy; cy++)
        for (int cx = 0; cx < gx; cx++) {
            int x0 = (int)((long)cx * w / gx), x1 = (int)((long)(cx + 1) * w / gx);
            int y0 = (int)((long)cy * h / gy), y1 = (int)((long)(cy + 1) * h / gy);
            int bx = -1, by = -1;
            float bv = 0.0f;
            for (int y = y0; y < y1; y++)
                for (int x = x0; x < x1; x++) {
                    if (x - m < 0 || x + m > w - 1 || y - m < 0 || y + m > h - 1) continue;
                    if (!is_lmax(R, w, h, x, y)) continue;
                    float c = R[(long)y * w + x];
                    if (!(c < max_peak)) continue;
                    int bad = 0;
                    for (int yy = y - m; yy <= y + m && !bad; yy++)
                        for (int xx = x - m; xx <= x + m; xx++)
                            if (flags[(long)yy * w + xx]) { bad = 1; break; }
                    if (bad) continue;
                    float thr = iso_frac * c;
                    for (int yy = y - iso; yy <= y + iso && !bad; yy++)
                        for (int xx = x - iso; xx <= x + iso; xx++) {
                            if (xx == x && yy == y) continue;
                            if (xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                            if (is_lmax(R, w, h, xx, yy) && R[(long)yy * w + xx] > thr) { bad = 1; break; }
                        }
                    if (bad) continue;
                    if (bx < 0 || c > bv) { bx = x; by = y; bv = c; }
                }
            if (bx >= 0) { centers[2 * n] = bx; centers[2 * n + 1] = by; n++; }
        }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Kernel fit (Alard & Lupton 1998; Alard 2000), weighted least squares.     */
/* For every pixel (x,y) of every stamp (|x-xs|<=hs, |y-ys|<=hs):            */
/*   X_n(x,y) = sum_{u,v} B_n(u,v) R(x-u, y-v)     (true convolution)         */
/*   columns  C_{0}      = X_0                                                */
/*            C_{n,k}    = p_k(x,y) X_n   (n >= 1, k < Ks)                    */
/*            C_{bg,k}   = p_k(x,y)       (k < Kb)                            */
/*   weight   w = 1/V_I if flags == 0, V_I > 0 and I finite, else 0           */
/*   M = sum w c c^T, b = sum w c I, a = M^{-1} b by Cholesky (FP64),         */
/*   chi2 = sum w (I - c.a)^2, dof = (#pixels with w > 0) - Nc.               */
/* A stamp whose window [xs-hs-r, xs+hs+r]^2 leaves the frame is skipped.    */
/* Returns 0, or -5 when the Cholesky meets a pivot <= 0.                    */
/* ------------------------------------------------------------------------ */
int ora_cholesky(int n, const double *M, double *L) {
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; j++) {
        double d = M[(long)j * n + j];
        for (int k = 0; k < j; k++) d -= L[(long)j * n + k] * L[(long)j * n + k];
        if (!(d > 0.0)) return -5;
        double ljj = sqrt(d);
        L[(long)j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double s = M[(long)i * n + j];
            for (int k = 0; k < j; k++) s -= L[(long)i * n + k] * L[(long)j * n + k];
            L[(long)i * n + j] = s / ljj;
        }
    }
    return 0;
}

void ora_cholesky_solve(int n, const double *L, const double *b, double *x) {
    double *y = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= L[(long)i * n + k] * y[k];
        y[i] = s / L[(long)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = y[i];
        for (int k = i + 1; k < n; k++) s -= L[(long)k * n + i] * x[k];
        x[i] = s / L[(long)i * n + i];
    }
    free(y);
}

static void design_row(const double *X, const double *pk, int nb, int Ks, const double *pb,
                       int Kb, double *c) {
    int j = 0;
    c[j++] = X[0];
    for (int n = 1; n < nb; n++)
        for (int k = 0; k < Ks; k++) c[j++] = pk[k] * X[n];
    for (int k = 0; k < Kb; k++) c[j++] = pb[k];
}

/* X_n at one pixel by direct 2-D convolution. */
static void basis_conv_at(const float *R, int w, int x, int y, const double *B, int nb, int ks,
                          double *X) {
    int r = (ks - 1) / 2, kk = ks * ks;
    for (int n = 0; n < nb; n++) {
        const double *b = B + (long)n * kk;
        double s = 0.0;
        for (int v = -r; v <= r; v++)
            for (int u = -r; u <= r; u++)
                s += b[(v + r) * ks + (u + r)] * (double)R[(long)(y - v) * w + (x - u)];
        X[n] = s;
    }
}

static int stamp_ok(int w, int h, int xs, int ys, int hs, int r) {
    return xs - hs - r >= 0 && xs + hs + r <= w - 1 && ys - hs - r >= 0 && ys + hs + r <= h - 1;
}

/* Basis images on every stamp pixel: X[(s*ss + pix)*nb + n], ss = stamp^2, */
/* pix = (y - ys + hs)*stamp + (x - xs + hs).  Skipped stamps are zero.      */
void ora_stamp_basis(int w, int h, const float *R, const int *centers, int n_stamps, int stamp,
                     const double *B, int nb, int ks, double *X) {
    int hs = stamp / 2, r = (ks - 1) / 2, ss = stamp * stamp;
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < n_stamps; s++) {
        int xs = centers[2 * s], ys = centers[2 * s + 1];
        double *Xs = X + (long)s * ss * nb;
        if (!stamp_ok(w, h, xs, ys, hs, r)) { memset(Xs, 0, sizeof(double) * ss * nb); continue; }
        for (int j = 0; j < stamp; j++)
            for (int i = 0; i < stamp; i++)
                basis_conv_at(R, w, xs - hs + i, ys - hs + j, B, nb, ks, Xs + (long)(j * stamp + i) * nb);
    }
}

int ora_fit(int w, int h, const float *sci, const float *sci_var, const float *R,
            const uint8_t *flags, const int *centers, int n_stamps, int stamp, int ks,
            int ngauss, const double *sigma, const int *degree, int sdeg, int bgdeg,
            double *coeffs, double *M_out, double *b_out, double *chi2_out, long *dof_out) {
    int nb = ora_basis_count(ngauss, degree);
    int Ks = ora_nterms(sdeg), Kb = ora_nterms(bgdeg), Nc = ora_ncoeffs(nb, sdeg, bgdeg);
    int hs = stamp / 2, r = (ks - 1) / 2, ss = stamp * stamp;
    double *B = (double *)malloc(sizeof(double) * nb * ks * ks);
    ora_basis(ks, ngauss, sigma, degree, B, NULL);
    double *X = (double *)malloc(sizeof(double) * (size_t)n_stamps * ss * nb);
    ora_stamp_basis(w, h, R, centers, n_stamps, stamp, B, nb, ks, X);
    /* per-stamp partial sums, added in stamp order afterwards */
    double *Mp = (double *)calloc((size_t)n_stamps * Nc * Nc, sizeof(double));
    double *bp = (double *)calloc((size_t)n_stamps * Nc, sizeof(double));
    long *np = (long *)calloc(n_stamps, sizeof(long));
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < n_stamps; s++) {
        int xs = centers[2 * s], ys = centers[2 * s + 1];
        if (!stamp_ok(w, h, xs, ys, hs, r)) continue;
        double pk[64], pb[64];
        double *c = (double *)malloc(sizeof(double) * Nc);
        double *Ms = Mp + (size_t)s * Nc * Nc, *bs = bp + (size_t)s * Nc;
        for (int j = 0; j < stamp; j++)
            for (int i = 0; i < stamp; i++) {
                int x = xs - hs + i, y = ys - hs + j;
                long p = (long)y * w + x;
                double v = sci_var[p], I = sci[p];
                if (flags[p] || !(v > 0.0) || !isfinite(I) || !isfinite(v)) continue;
                double wt = 1.0 / v;
                ora_spatial_terms(x, y, w, h, sdeg, pk);
                ora_spatial_terms(x, y, w, h, bgdeg, pb);
                design_row(X + ((size_t)s * ss + j * stamp + i) * nb, pk, nb, Ks, pb, Kb, c);
                for (int a = 0; a < Nc; a++) {
                    double wa = wt * c[a];
                    bs[a] += wa * I;
                    for (int b2 = 0; b2 < Nc; b2++) Ms[(size_t)a * Nc + b2] += wa * c[b2];
                }
                np[s]++;
            }
        free(c);
    }
    double *M = (double *)calloc((size_t)Nc * Nc, sizeof(double));
    double *bv = (double *)calloc(Nc, sizeof(double));
    long nvalid = 0;
    for (int s = 0; s < n_stamps; s++) {
        for (long i = 0; i < (long)Nc * Nc; i++) M[i] += Mp[(size_t)s * Nc * Nc + i];
        for (int i = 0; i < Nc; i++) bv[i] += bp[(size_t)s * Nc + i];
        nvalid += np[s];
    }
    free(Mp); free(bp); free(np);
    if (M_out) memcpy(M_out, M, sizeof(double) * Nc * Nc);
    if (b_out) memcpy(b_out, bv, sizeof(double) * Nc);
    double *L = (double *)malloc(sizeof(double) * Nc * Nc);
    int st = ora_cholesky(Nc, M, L);
    if (st == 0) {
        ora_cholesky_solve(Nc, L, bv, coeffs);
        double chi2 = 0.0, pk[64], pb[64];
        double *c = (double *)malloc(sizeof(double) * Nc);
        for (int s = 0; s < n_stamps; s++) {
            int xs = centers[2 * s], ys = centers[2 * s + 1];
            if (!stamp_ok(w, h, xs, ys, hs, r)) continue;
            for (int j = 0; j < stamp; j++)
                for (int i = 0; i < stamp; i++) {
                    int x = xs - hs + i, y = ys - hs + j;
                    long p = (long)y * w + x;
                    double v = sci_var[p], I = sci[p];
                    if (flags[p] || !(v > 0.0) || !isfinite(I) || !isfinite(v)) continue;
                    ora_spatial_terms(x, y, w, h, sdeg, pk);
                    ora_spatial_terms(x, y, w, h, bgdeg, pb);
                    design_row(X + ((size_t)s * ss + j * stamp + i) * nb, pk, nb, Ks, pb, Kb, c);
                    double m = 0.0;
                    for (int a = 0; a < Nc; a++) m += c[a] * coeffs[a];
                    chi2 += (I - m) * (I - m) / v;
                }
        }
        free(c);
        if (chi2_out) *chi2_out = chi2;
    }
    if (dof_out) *dof_out = nvalid - Nc;
    free(L); free(M); free(bv); free(X); free(B);
    return st;
}

/* ------------------------------------------------------------------------ */
/* The same least-squares fit over every pixel of a rectangle [x0,x1]x[y0,y1] */
/* (a whole segment interior) instead of stamps.  Pixels whose convolution   */
/* window leaves the image are skipped.  Spatial terms use the image size.   */
/* ------------------------------------------------------------------------ */
int ora_fit_rect(int w, int h, const float *sci, const float *sci_var, const float *R,
                 const uint8_t *flags, int x0, int y0, int x1, int y1, int ks, int ngauss,
                 const double *sigma, const int *degree, int sdeg, int bgdeg, double *coeffs,
                 double *M_out, double *b_out, double *chi2_out, long *dof_out) {
    int nb = ora_basis_count(ngauss, degree);
    int Ks = ora_nterms(sdeg), Kb = ora_nterms(bgdeg), Nc = ora_ncoeffs(nb, sdeg, bgdeg);
    int r = (ks - 1) / 2;
    double *B = (double *)malloc(sizeof(double) * nb * ks * ks);
    ora_basis(ks, ngauss, sigma, degree, B, NULL);
    int ny = y1 - y0 + 1;
    double *Mp = (double *)calloc((size_t)ny * Nc * Nc, sizeof(double));
    double *bp = (double *)calloc((size_t)ny * Nc, sizeof(double));
    long *np = (long *)calloc(ny, sizeof(long));
#pragma omp parallel for schedule(dynamic)
    for (int y = y0; y <= y1; y++) {
        double pk[64], pb[64];
        double *X = (double *)malloc(sizeof(double) * nb), *c = (double *)malloc(sizeof(double) * Nc);
        double *Ms = Mp + (size_t)(y - y0) * Nc * Nc, *bs = bp + (size_t)(y - y0) * Nc;
        for (int x = x0; x <= x1; x++) {
            if (x - r < 0 || x + r > w - 1 || y - r < 0 || y + r > h - 1) continue;
            long p = (long)y * w + x;
            double v = sci_var[p], I = sci[p];
            if (flags[p] || !(v > 0.0) || !isfinite(I) || !isfinite(v)) continue;
            double wt = 1.0 / v;
            basis_conv_at(R, w, x, y, B, nb, ks, X);
            ora_spatial_terms(x, y, w, h, sdeg, pk);
            ora_spatial_terms(x, y, w, h, bgdeg, pb);
            design_row(X, pk, nb, Ks, pb, Kb, c);
            for (int a = 0; a < Nc; a++) {
                double wa = wt * c[a];
                bs[a] += wa * I;
                for (int b2 = 0; b2 < Nc; b2++) Ms[(size_t)a * Nc + b2] += wa * c[b2];
            }
            np[y - y0]++;
        }
        free(X); free(c);
    }
    double *M = (double *)calloc((size_t)Nc * Nc, sizeof(double));
    double *bv = (double *)calloc(Nc, sizeof(double));
    long nvalid = 0;
    for (int t = 0; t < ny; t++) {
        for (long i = 0; i < (long)Nc * Nc; i++) M[i] += Mp[(size_t)t * Nc * Nc + i];
        for (int i = 0; i < Nc; i++) bv[i] += bp[(size_t)t * Nc + i];
        nvalid += np[t];
    }
    free(Mp); free(bp); free(np);
    if (M_out) memcpy(M_out, M, sizeof(double) * Nc * Nc);
    if (b_out) memcpy(b_out, bv, sizeof(double) * Nc);
    double *L = (double *)malloc(sizeof(double) * Nc * Nc);
    int st = ora_cholesky(Nc, M, L);
    if (st == 0) {
        ora_cholesky_solve(Nc, L, bv, coeffs);
        double chi2 = 0.0;
#pragma omp parallel for reduction(+ : chi2) schedule(dynamic)
        for (int y = y0; y <= y1; y++) {
            double pk[64], pb[64];
            double *X = (double *)malloc(sizeof(double) * nb), *c = (double *)malloc(sizeof(double) * Nc);
            for (int x = x0; x <= x1; x++) {
                if (x - r < 0 || x + r > w - 1 || y - r < 0 || y + r > h - 1) continue;
                long p = (long)y * w + x;
                double v = sci_var[p], I = sci[p];
                if (flags[p] || !(v > 0.0) || !isfinite(I) || !isfinite(v)) continue;
                basis_conv_at(R, w, x, y, B, nb, ks, X);
                ora_spatial_terms(x, y, w, h, sdeg, pk);
                ora_spatial_terms(x, y, w, h, bgdeg, pb);
                design_row(X, pk, nb, Ks, pb, Kb, c);
                double m = 0.0;
                for (int a = 0; a < Nc; a++) m += c[a] * coeffs[a];
                chi2 += (I - m) * (I - m) / v;
            }
            free(X); free(c);
        }
        if (chi2_out) *chi2_out = chi2;
    }
    if (dof_out) *dof_out = nvalid - Nc;
    free(L); free(M); free(bv); free(B);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Kernel expansion: K_k(u,v) = sum_n a_{n,k} B_n(u,v); K_0 also holds       */
/* a_0 B_0.  bg[k] = background coefficients.  K[k*ks*ks + (v+r)*ks+(u+r)].  */
/* ------------------------------------------------------------------------ */
void ora_expand(int ks, int ngauss, const double *sigma, const int *degree, int sdeg, int bgdeg,
                const double *a, double *K, double *bg) {
    int nb = ora_basis_count(ngauss, degree), Ks = ora_nterms(sdeg), Kb = ora_nterms(bgdeg);
    int kk = ks * ks;
    double *B = (double *)malloc(sizeof(double) * nb * kk);
    ora_basis(ks, ngauss, sigma, degree, B, NULL);
    memset(K, 0, sizeof(double) * Ks * kk);
    for (int i = 0; i < kk; i++) K[i] += a[0] * B[i];
    for (int n = 1; n < nb; n++)
        for (int k = 0; k < Ks; k++) {
            double c = a[1 + (n - 1) * Ks + k];
            for (int i = 0; i < kk; i++) K[(long)k * kk + i] += c * B[(long)n * kk + i];
        }
    for (int k = 0; k < Kb; k++) bg[k] = a[1 + (nb - 1) * Ks + k];
    free(B);
}

/* ------------------------------------------------------------------------ */
/* Subtraction (direct image subtraction, Sec. 4.2 / Table 2; formula from   */
/* the Alard-Lupton reading) and difference variance (noise maps, Sec. 3.2). */
/*   D(x,y)  = I - sum_k p_k(x,y) sum_{u,v} K_k(u,v) R(x-u,y-v) - B(x,y)     */
/*   B(x,y)  = sum_k bg_k p_k(x,y)                                           */
/*   V_D     = V_I + sum_{u,v} K_xy(u,v)^2 V_ref(x-u,y-v)                     */
/*   K_xy    = sum_k p_k(x,y) K_k, the kernel at the pixel itself: the        */
/*             variance of D for independent noise in I and R.               */
/* Pixels within r of an edge, or with flags != 0, get D = V_D = 0.          */
/* Spatial terms use the frame size (W,H) and frame coordinates x+ox, y+oy.  */
/* ------------------------------------------------------------------------ */
static void subtract_px(int w, int h, int W, int H, int ox, int oy, const float *sci,
                        const float *sci_var, const float *R, const float *Rv,
                        const uint8_t *flags, int ks, int sdeg, const double *K, int bgdeg,
                        const double *bg, int x, int y, double *Dp, double *Vp) {
    int r = (ks - 1) / 2, kk = ks * ks, Ks = ora_nterms(sdeg), Kb = ora_nterms(bgdeg);
    long p = (long)y * w + x;
    if (x < r || y < r || x > w - 1 - r || y > h - 1 - r || (flags && flags[p])) {
        *Dp = 0.0; if (Vp) *Vp = 0.0; return;
    }
    double pk[64], pb[64];
    ora_spatial_terms(x + ox, y + oy, W, H, sdeg, pk);
    ora_spatial_terms(x + ox, y + oy, W, H, bgdeg, pb);
    double conv = 0.0;
    for (int k = 0; k < Ks; k++) {
        double s = 0.0;
        const double *Kk = K + (long)k * kk;
        for (int v = -r; v <= r; v++)
            for (int u = -r; u <= r; u++)
                s += Kk[(v + r) * ks + (u + r)] * (double)R[(long)(y - v) * w + (x - u)];
        conv += pk[k] * s;
    }
    double bgv = 0.0;
    for (int k = 0; k < Kb; k++) bgv += bg[k] * pb[k];
    *Dp = (double)sci[p] - conv - bgv;
    if (Vp) {
        double vs = 0.0;
        for (int v = -r; v <= r; v++)
            for (int u = -r; u <= r; u++) {
                double kxy = 0.0;
                for (int k = 0; k < Ks; k++) kxy += pk[k] * K[(long)k * kk + (v + r) * ks + (u + r)];
                vs += kxy * kxy * (double)Rv[(long)(y - v) * w + (x - u)];
            }
        *Vp = (double)sci_var[p] + vs;
    }
}

void ora_subtract(int w, int h, int W, int H, int ox, int oy, const float *sci,
                  const float *sci_var, const float *R, const float *Rv, const uint8_t *flags,
                  int ks, int sdeg, const double *K, int bgdeg, const double *bg,
                  double *D, double *VD) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            long p = (long)y * w + x;
            subtract_px(w, h, W, H, ox, oy, sci, sci_var, R, Rv, flags, ks, sdeg, K, bgdeg, bg,
                        x, y, D + p, VD ? VD + p : NULL);
        }
}

/* The same definition evaluated at n listed pixels xy[2i], xy[2i+1]. */
void ora_subtract_at(int w, int h, int W, int H, int ox, int oy, const float *sci,
                     const float *sci_var, const float *R, const float *Rv, const uint8_t *flags,
                     int ks, int sdeg, const double *K, int bgdeg, const double *bg,
                     int n, const int *xy, double *D, double *VD) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++)
        subtract_px(w, h, W, H, ox, oy, sci, sci_var, R, Rv, flags, ks, sdeg, K, bgdeg, bg,
                    xy[2 * i], xy[2 * i + 1], D + i, VD ? VD + i : NULL);
}

/* ------------------------------------------------------------------------ */
/* Detection on the difference image (Sec. 4.2 transient candidates; the    */
/* variance-weighted threshold reading):                                    */
/*   valid = flags == 0 && V_D > 0 && D, V_D finite                          */
/*   S = D / sqrt(V_D) in float (the decision precision of the kernel)       */
/*   mask: 1 if S >= n, 2 if S <= -n, 4 if invalid                           */
/*   8-connected components of equal-sign pixels; per component:            */
/*     peak = max |S| (ties to lowest (y,x)), npix, sign                     */
/*     window = valid pixels within fw = ceil(3 sigma) of the peak pixel     */
/*     centroid: start at the peak pixel, then 4 windowed steps              */
/*       g_i = exp(-|p_i - c|^2 / (2 sigma^2)), t_i = sign * D_i * g_i,       */
/*       c += 2 sum t_i (p_i - c) / sum t_i   (stop when sum t_i <= 0),       */
/*       c clamped to the peak pixel +- 2 (the Gaussian-windowed centroid,   */
/*       exact in one step for a Gaussian of width sigma);                   */
/*     flux = sum P D/V / sum P^2/V over the window,                         */
/*       P the unit-sum pixel-integrated Gaussian at the centroid;          */
/*     flux_err = (sum P^2/V)^-1/2                                           */
/*   sources sorted by (peak y, peak x).                                     */
/* Record: x, y, flux, flux_err, peak_snr (float), npix, sign, px, py (int). */
/* Returns the number of components (may exceed cap; only cap written).     */
/* ------------------------------------------------------------------------ */
typedef struct { float x, y, flux, flux_err, peak_snr; int npix, sign, px, py; } ora_source;

static int cmp_src(const void *a, const void *b) {
    const ora_source *s = (const ora_source *)a, *t = (const ora_source *)b;
    if (s->py != t->py) return s->py < t->py ? -1 : 1;
    if (s->px != t->px) return s->px < t->px ? -1 : 1;
    return 0;
}

static double pix_gauss(double a, double c, double sig) {
    double s2 = sig * sqrt(2.0);
    return 0.5 * (erf((a + 0.5 - c) / s2) - erf((a - 0.5 - c) / s2));
}

int ora_detect(int w, int h, const float *D, const float *VD, const uint8_t *flags, float nsig,
               double psf_sigma, uint8_t *mask, ora_source *out, int cap) {
    long np = (long)w * h;
    float *S = (float *)malloc(sizeof(float) * np);
    for (long p = 0; p < np; p++) {
        float d = D[p], v = VD[p];
        int valid = (!flags || flags[p] == 0) && v > 0.0f && isfinite(d) && isfinite(v);
        if (!valid) { mask[p] = ORA_MINV; S[p] = 0.0f; continue; }
        float s = d / sqrtf(v);
        S[p] = s;
        mask[p] = (s >= nsig ? ORA_MPOS : 0) | (s <= -nsig ? ORA_MNEG : 0);
    }
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * np);
    for (long p = 0; p < np; p++) lab[p] = -1;
    long *stack = (long *)malloc(sizeof(long) * np);
    int ncomp = 0, fw = (int)ceil(3.0 * psf_sigma);
    ora_source *all = NULL;
    int allcap = 0;
    for (long p0 = 0; p0 < np; p0++) {
        int bit = mask[p0] & (ORA_MPOS | ORA_MNEG);
        if (!bit || lab[p0] >= 0) continue;
        long top = 0, npix = 0, pk = p0;
        float pkv = fabsf(S[p0]);
        stack[top++] = p0;
        lab[p0] = ncomp;
        while (top) {
            long q = stack[--top];
            npix++;
            float a = fabsf(S[q]);
            if (a > pkv || (a == pkv && q < pk)) { pkv = a; pk = q; }
            int qx = (int)(q % w), qy = (int)(q / w);
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int nx = qx + dx, ny = qy + dy;
                    if ((!dx && !dy) || nx < 0 || ny < 0 || nx >= w || ny >= h) continue;
                    long nq = (long)ny * w + nx;
                    if ((mask[nq] & bit) && lab[nq] < 0) { lab[nq] = ncomp; stack[top++] = nq; }
                }
        }
        ora_source s;
        int px = (int)(pk % w), py = (int)(pk / w);
        double xc = px, yc = py;
        double sg = bit == ORA_MPOS ? 1.0 : -1.0;
        for (int it = 0; it < 4; it++) {
            double sw = 0, sx = 0, sy = 0;
            for (int y = py - fw; y <= py + fw; y++)
                for (int x = px - fw; x <= px + fw; x++) {
                    if (x < 0 || y < 0 || x >= w || y >= h) continue;
                    long q = (long)y * w + x;
                    if (mask[q] & ORA_MINV) continue;
                    double ddx = x - xc, ddy = y - yc;
                    double t = sg * (double)D[q] * exp(-(ddx * ddx + ddy * ddy) / (2.0 * psf_sigma * psf_sigma));
                    sw += t; sx += t * ddx; sy += t * ddy;
                }
            if (!(sw > 0)) break;
            xc += 2.0 * sx / sw; yc += 2.0 * sy / sw;
            if (xc < px - 2.0) xc = px - 2.0;
            if (xc > px + 2.0) xc = px + 2.0;
            if (yc < py - 2.0) yc = py - 2.0;
            if (yc > py + 2.0) yc = py + 2.0;
        }
        double num = 0, den = 0;
        for (int y = py - fw; y <= py + fw; y++)
            for (int x = px - fw; x <= px + fw; x++) {
                if (x < 0 || y < 0 || x >= w || y >= h) continue;
                long q = (long)y * w + x;
                if (mask[q] & ORA_MINV) continue;
                double P = pix_gauss(x, xc, psf_sigma) * pix_gauss(y, yc, psf_sigma);
                num += P * (double)D[q] / (double)VD[q];
                den += P * P / (double)VD[q];
            }
        s.x = (float)xc; s.y = (float)yc;
        s.flux = den > 0 ? (float)(num / den) : 0.0f;
        s.flux_err = den > 0 ? (float)(1.0 / sqrt(den)) : 0.0f;
        s.peak_snr = S[pk];
        s.npix = (int)npix;
        s.sign = bit == ORA_MPOS ? 1 : -1;
        s.px = px; s.py = py;
        if (ncomp >= allcap) {
            allcap = allcap ? 2 * allcap : 1024;
            all = (ora_source *)realloc(all, sizeof(ora_source) * allcap);
        }
        all[ncomp++] = s;
    }
    if (ncomp) qsort(all, ncomp, sizeof(ora_source), cmp_src);
    for (int i = 0; i < ncomp && i < cap; i++) out[i] = all[i];
    free(all); free(stack); free(lab); free(S);
    return ncomp;
}

/* ------------------------------------------------------------------------ */
/* Sigma-clipped mean coadd of n raw frames (coaddition, Sec. 4.1.3; the    */
/* clipped mean replaces the matched filter there).  Per output pixel:      */
/*  1. frame f is sampled at (x+dx_f, y+dy_f): ix = x + floor(dx_f),         */
/*     fx = dx_f - floor(dx_f) (same for y); neighbours (ix,iy), (ix+1,iy)    */
/*     if fx > 0, (ix,iy+1) if fy > 0, (ix+1,iy+1) if both; each neighbour is */
/*     calibrated as above; the sample is invalid if a used neighbour is     */
/*     outside the frame or flagged, or if its value is not finite.  Value   */
/*     by nested lerps                                                        */
/*       top = v00 + fx (v10 - v00), bot = v01 + fx (v11 - v01),             */
/*       v = top + fy (bot - top);   V_f = sum w_i^2 V_i (bilinear w_i).     */
/*  2. S = valid samples.  Repeat at most max_iter times: c = median(S)      */
/*     (mean of the two middle values for even |S|), m = mean(S),            */
/*     s = sqrt(mean((v-m)^2)); reject v with |v - c| > kappa s; stop when  */
/*     nothing is rejected (or when everything would be).                    */
/*  3. c = median(S); coadd = c + sum_S (v - c) / |S|; var = sum_S V_f / |S|^2;*/
/*     n_used = |S|; an empty S gives 0, 0, 0.                               */
/* margin (optional) = min over decisions of ||v-c| - kappa s| / s.          */
/* ------------------------------------------------------------------------ */
static int cmp_dbl(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static double median_of(const double *v, int n, double *tmp) {
    memcpy(tmp, v, sizeof(double) * n);
    qsort(tmp, n, sizeof(double), cmp_dbl);
    return (n & 1) ? tmp[n / 2] : 0.5 * (tmp[n / 2 - 1] + tmp[n / 2]);
}

void ora_coadd(int nf, int w, int h, const uint16_t *raw, const float *shifts, int bias_scalar,
               const float *dark, const float *flat, const uint8_t *bpm, double gain, double rn,
               int sat, double kappa, int max_iter, double *coadd, double *var, uint8_t *n_used,
               double *margin) {
#pragma omp parallel
    {
        double *v = (double *)malloc(sizeof(double) * nf), *vv = (double *)malloc(sizeof(double) * nf);
        double *tmp = (double *)malloc(sizeof(double) * nf), *nv = (double *)malloc(sizeof(double) * nf);
        double *nvv = (double *)malloc(sizeof(double) * nf);
#pragma omp for schedule(static)
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                int n = 0;
                for (int f = 0; f < nf; f++) {
                    double dx = shifts[2 * f], dy = shifts[2 * f + 1];
                    double flx = floor(dx), fly = floor(dy);
                    int ix = x + (int)flx, iy = y + (int)fly;
                    double fx = dx - flx, fy = dy - fly;
                    int need[4] = {1, fx > 0, fy > 0, fx > 0 && fy > 0};
                    int nx[4] = {ix, ix + 1, ix, ix + 1}, ny[4] = {iy, iy, iy + 1, iy + 1};
                    double val[4] = {0, 0, 0, 0}, vr[4] = {0, 0, 0, 0};
                    int ok = 1;
                    for (int k = 0; k < 4 && ok; k++) {
                        if (!need[k]) continue;
                        if (nx[k] < 0 || ny[k] < 0 || nx[k] >= w || ny[k] >= h) { ok = 0; break; }
                        long p = (long)ny[k] * w + nx[k];
                        const uint16_t rv = raw[(long)f * w * h + p];
                        double fl = flat ? flat[p] : 1.0;
                        if ((bpm && bpm[p]) || !(fl > 0.0) || !isfinite(fl) || (int)rv >= sat) { ok = 0; break; }
                        double ng = ((int)rv - bias_scalar) * gain;
                        val[k] = (ng - (dark ? dark[p] : 0.0)) / fl;
                        vr[k] = ((ng > 0 ? ng : 0) + rn * rn) / (fl * fl);
                    }
                    if (!ok) continue;
                    if (!need[1]) val[1] = val[0];
                    if (!need[2]) val[2] = val[0];
                    if (!need[3]) val[3] = need[1] ? val[1] : val[2];
                    double top = val[0] + fx * (val[1] - val[0]);
                    double bot = val[2] + fx * (val[3] - val[2]);
                    double sv = top + fy * (bot - top);
                    if (!isfinite(sv)) continue;
                    v[n] = sv;
                    double w0 = (1 - fx) * (1 - fy), w1 = fx * (1 - fy), w2 = (1 - fx) * fy, w3 = fx * fy;
                    vv[n] = w0 * w0 * vr[0] + (need[1] ? w1 * w1 * vr[1] : 0) +
                            (need[2] ? w2 * w2 * vr[2] : 0) + (need[3] ? w3 * w3 * vr[3] : 0);
                    n++;
                }
                long p = (long)y * w + x;
                double mg = INFINITY;
                for (int it = 0; it < max_iter && n > 0; it++) {
                    double c = median_of(v, n, tmp), m = 0, s2 = 0;
                    for (int i = 0; i < n; i++) m += v[i];
                    m /= n;
                    for (int i = 0; i < n; i++) s2 += (v[i] - m) * (v[i] - m);
                    double s = sqrt(s2 / n);
                    int k = 0;
                    for (int i = 0; i < n; i++) {
                        double d = fabs(v[i] - c);
                        if (s > 0) { double g = fabs(d - kappa * s) / s; if (g < mg) mg = g; }
                        if (!(d > kappa * s)) { nv[k] = v[i]; nvv[k] = vv[i]; k++; }
                    }
                    if (k == n || k == 0) break;
                    memcpy(v, nv, sizeof(double) * k);
                    memcpy(vv, nvv, sizeof(double) * k);
                    n = k;
                }
                if (n == 0) { coadd[p] = 0; var[p] = 0; n_used[p] = 0; }
                else {
                    double c = median_of(v, n, tmp), sd = 0, sv = 0;
                    for (int i = 0; i < n; i++) { sd += v[i] - c; sv += vv[i]; }
                    coadd[p] = c + sd / n;
                    var[p] = sv / ((double)n * n);
                    n_used[p] = (uint8_t)n;
                }
                if (margin) margin[p] = mg;
            }
        free(v); free(vv); free(tmp); free(nv); free(nvv);
    }
}

/* ------------------------------------------------------------------------ */
/* Learned kernel surrogate (a learned stand-in for the least-squares fit;  */
/* no counterpart in the paper).  A CNN maps a stamp pair (science and      */
/* reference, each 21x21 and divided by the reference stamp sum) to a 21x21 */
/* kernel:                                                                    */
/*   h1 = W1 x + b1                       (1x1 conv, 2 -> 32, linear)         */
/*   h_{l+1} = relu(conv7(h_l; W_l) + b_l), l = 2..5  (7x7, 32 -> 32, 'same' */
/*                                           zero padding)                    */
/*   y = (W6 h5 + b6) / 441               (1x1 conv, 32 -> 1, linear; the    */
/*                                          fixed 1/441 puts the last layer's */
/*                                          values at order one)              */
/* Parameter vector (FP64 here), in this order:                              */
/*   W1[32][2], b1[32], {W_l[7][7][32 in][32 out], b_l[32]} x 4, W6[32], b6   */
/* conv7: z[y][x][o] = b[o] + sum_{ky,kx,i} W[ky][kx][i][o] h[y+ky-3][x+kx-3][i]*/
/* Activations are [B][21][21][C] (channels last).                           */
/* ------------------------------------------------------------------------ */
#define CNN_S 21
#define CNN_P (CNN_S * CNN_S)
#define CNN_C 32
#define CNN_K 7

long ora_cnn_nparams(void) { return 64 + 32 + 4L * (49 * 1024 + 32) + 32 + 1; }

static void cnn_offsets(long *oW1, long *ob1, long oW[4], long ob[4], long *oW6, long *ob6) {
    long o = 0;
    *oW1 = o; o += 64;
    *ob1 = o; o += 32;
    for (int l = 0; l < 4; l++) { oW[l] = o; o += 49 * 1024; ob[l] = o; o += 32; }
    *oW6 = o; o += 32;
    *ob6 = o;
}

/* acts: h1..h5 [5][B][P][C] (post-activation); y [B][P]. */
void ora_cnn_forward(int B, const double *prm, const double *x /*[B][P][2]*/, double *acts, double *y) {
    long oW1, ob1, oW[4], ob[4], oW6, ob6;
    cnn_offsets(&oW1, &ob1, oW, ob, &oW6, &ob6);
    long L = (long)B * CNN_P * CNN_C;
    double *h1 = acts;
#pragma omp parallel for
    for (long q = 0; q < (long)B * CNN_P; q++)
        for (int o = 0; o < CNN_C; o++)
            h1[q * CNN_C + o] = prm[ob1 + o] + prm[oW1 + o * 2] * x[q * 2] + prm[oW1 + o * 2 + 1] * x[q * 2 + 1];
    for (int l = 0; l < 4; l++) {
        const double *hin = acts + l * L;
        double *hout = acts + (l + 1) * L;
        const double *W = prm + oW[l], *bb = prm + ob[l];
#pragma omp parallel for
        for (long q = 0; q < (long)B * CNN_P; q++) {
            int b = (int)(q / CNN_P), p = (int)(q % CNN_P), yy = p / CNN_S, xx = p % CNN_S;
            for (int o = 0; o < CNN_C; o++) {
                double z = bb[o];
                for (int ky = 0; ky < CNN_K; ky++)
                    for (int kx = 0; kx < CNN_K; kx++) {
                        int sy = yy + ky - 3, sx = xx + kx - 3;
                        if (sy < 0 || sx < 0 || sy >= CNN_S || sx >= CNN_S) continue;
                        const double *hi = hin + ((long)b * CNN_P + sy * CNN_S + sx) * CNN_C;
                        const double *w = W + ((ky * CNN_K + kx) * CNN_C) * CNN_C + o;
                        for (int i = 0; i < CNN_C; i++) z += w[i * CNN_C] * hi[i];
                    }
                hout[q * CNN_C + o] = z > 0.0 ? z : 0.0;
            }
        }
    }
    const double *h5 = acts + 4 * L;
    for (long q = 0; q < (long)B * CNN_P; q++) {
        double s = prm[ob6];
        for (int i = 0; i < CNN_C; i++) s += prm[oW6 + i] * h5[q * CNN_C + i];
        y[q] = s / (double)CNN_P;
    }
}

/* Gradient of loss with respect to the parameters given dL/dy (grad zeroed here). */
void ora_cnn_backward(int B, const double *prm, const double *x, const double *acts, const double *dy,
                      double *grad) {
    long oW1, ob1, oW[4], ob[4], oW6, ob6;
    cnn_offsets(&oW1, &ob1, oW, ob, &oW6, &ob6);
    long NP = ora_cnn_nparams(), L = (long)B * CNN_P * CNN_C;
    memset(grad, 0, sizeof(double) * NP);
    double *dh = (double *)calloc(L, sizeof(double)), *dz = (double *)calloc(L, sizeof(double));
    const double *h5 = acts + 4 * L;
    for (long q = 0; q < (long)B * CNN_P; q++) {
        double d = dy[q] / (double)CNN_P;
        grad[ob6] += d;
        for (int i = 0; i < CNN_C; i++) {
            grad[oW6 + i] += d * h5[q * CNN_C + i];
            dh[q * CNN_C + i] = prm[oW6 + i] * d;
        }
    }
    for (int l = 3; l >= 0; l--) {
        const double *hin = acts + l * L, *hout = acts + (l + 1) * L;
        const double *W = prm + oW[l];
        for (long e = 0; e < L; e++) dz[e] = hout[e] > 0.0 ? dh[e] : 0.0;
        for (long q = 0; q < (long)B * CNN_P; q++)
            for (int o = 0; o < CNN_C; o++) grad[ob[l] + o] += dz[q * CNN_C + o];
        /* dW[ky][kx][i][o] = sum_q hin[q + tap][i] dz[q][o] */
#pragma omp parallel for
        for (int t = 0; t < 49; t++) {
            int ky = t / CNN_K, kx = t % CNN_K;
            for (int i = 0; i < CNN_C; i++)
                for (int o = 0; o < CNN_C; o++) {
                    double s = 0.0;
                    for (int b = 0; b < B; b++)
                        for (int p = 0; p < CNN_P; p++) {
                            int yy = p / CNN_S, xx = p % CNN_S, sy = yy + ky - 3, sx = xx + kx - 3;
                            if (sy < 0 || sx < 0 || sy >= CNN_S || sx >= CNN_S) continue;
                            s += hin[((long)b * CNN_P + sy * CNN_S + sx) * CNN_C + i] *
                                 dz[((long)b * CNN_P + p) * CNN_C + o];
                        }
                    grad[oW[l] + (t * CNN_C + i) * CNN_C + o] += s;
                }
        }
        /* dh_in[q'][i] = sum over outputs q with q' = q + tap: W[tap][i][o] dz[q][o] */
        memset(dh, 0, sizeof(double) * L);
#pragma omp parallel for
        for (long qs = 0; qs < (long)B * CNN_P; qs++) {
            int b = (int)(qs / CNN_P), ps = (int)(qs % CNN_P), sy = ps / CNN_S, sx = ps % CNN_S;
            for (int i = 0; i < CNN_C; i++) {
                double s = 0.0;
                for (int ky = 0; ky < CNN_K; ky++)
                    for (int kx = 0; kx < CNN_K; kx++) {
                        int yy = sy - ky + 3, xx = sx - kx + 3;
                        if (yy < 0 || xx < 0 || yy >= CNN_S || xx >= CNN_S) continue;
                        const double *d = dz + ((long)b * CNN_P + yy * CNN_S + xx) * CNN_C;
                        const double *w = W + ((ky * CNN_K + kx) * CNN_C + i) * CNN_C;
                        for (int o = 0; o < CNN_C; o++) s += w[o] * d[o];
                    }
                dh[qs * CNN_C + i] = s;
            }
        }
    }
    /* layer 1 (linear): dW1[o][j] = sum_q x[q][j] dh1[q][o] */
    for (long q = 0; q < (long)B * CNN_P; q++)
        for (int o = 0; o < CNN_C; o++) {
            grad[ob1 + o] += dh[q * CNN_C + o];
            grad[oW1 + o * 2] += x[q * 2] * dh[q * CNN_C + o];
            grad[oW1 + o * 2 + 1] += x[q * 2 + 1] * dh[q * CNN_C + o];
        }
    free(dh); free(dz);
}

/* Mean squared error over B*P outputs and its gradient dL/dy. */
double ora_cnn_mse(long n, const double *y, const double *t, double *dy) {
    double s = 0.0;
    for (long i = 0; i < n; i++) {
        double d = y[i] - t[i];
        s += d * d;
        if (dy) dy[i] = 2.0 * d / (double)n;
    }
    return s / (double)n;
}

/* One Adam step (Kingma & Ba 2015), bias-corrected, step >= 1. */
void ora_adam(long n, double *p, double *m, double *v, const double *g, double lr, double b1, double b2,
              double eps, int step) {
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (long i = 0; i < n; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Sparse "minipix" stamping (Sec. 3.3, Sparse Image Segments): within an   */
/* image, square cells of cell x cell pixels stand for the NSIDE=16384      */
/* minipix of a segment; a cell is kept when a science target (x, y) lies   */
/* in it, and every pixel of the other cells is set to zero.  keep[cy * ncx */
/* + cx] = 1 for kept cells (ncx = ceil(w / cell)); partial cells at the    */
/* right and bottom edges hold the pixels that exist.  Targets outside the  */
/* image are ignored.  Returns the number of kept cells.                    */
/* ------------------------------------------------------------------------ */
int ora_minipix(int w, int h, const float *img, int cell, const int *targets, int n, float *out,
                uint8_t *keep) {
    int ncx = (w + cell - 1) / cell, ncy = (h + cell - 1) / cell;
    memset(keep, 0, (size_t)ncx * ncy);
    for (int t = 0; t < n; t++) {
        int x = targets[2 * t], y = targets[2 * t + 1];
        if (x < 0 || y < 0 || x >= w || y >= h) continue;
        keep[(y / cell) * ncx + x / cell] = 1;
    }
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++)
            out[(long)y * w + x] = keep[(y / cell) * ncx + x / cell] ? img[(long)y * w + x] : 0.0f;
    int kept = 0;
    for (int c = 0; c < ncx * ncy; c++) kept += keep[c];
    return kept;
}

/* Low-resolution map (Sec. 2, segments at 10x reduced resolution): out[Y][X] */
/* is the mean of the valid pixels (flags == 0 where flags are given, finite */
/* values) of the f x f block at (f X, f Y); partial blocks at the right and */
/* bottom edges average the pixels they hold; 0 where a block has none.      */
/* out is [ceil(h / f)][ceil(w / f)], sums in FP64.                           */
void ora_lowres(int w, int h, const float *img, const uint8_t *flags, int f, double *out) {
    int ow = (w + f - 1) / f, oh = (h + f - 1) / f;
    for (int Y = 0; Y < oh; Y++)
        for (int X = 0; X < ow; X++) {
            double s = 0.0;
            long n = 0;
            for (int y = Y * f; y < Y * f + f && y < h; y++)
                for (int x = X * f; x < X * f + f && x < w; x++) {
                    float v = img[(long)y * w + x];
                    if ((flags && flags[(long)y * w + x]) || !isfinite(v)) continue;
                    s += v;
                    n++;
                }
            out[(long)Y * ow + X] = n ? s / (double)n : 0.0;
        }
}
