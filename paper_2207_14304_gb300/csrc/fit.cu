// K3-K5 and a3/a7: stamp selection, basis convolution on stamps, the
// normal-equation Gram matrix (SIMT FP32 with double-float block accumulation,
// or tcgen05 tensor cores in TF32 / BF16 with FP32 accumulation in TMEM), FP64
// Cholesky with iterative refinement, and kernel expansion.  The fit is the
// Alard & Lupton (1998) / Alard (2000) Gaussian-basis least-squares kernel
// adopted for the direct image subtraction of paper Sec. 4.2 (Table 2).
//
// Conditioning.  The 49-function basis is nearly degenerate: for the full
// frame workload the Jacobi-scaled normal matrix has condition ~4e9, far
// beyond what an FP32-accumulated Gram can keep positive definite.  The fit is
// therefore carried out in an equivalent basis: the functions n >= 1 are
// orthonormalised in pixel space (B' = B S, S upper triangular from the
// Cholesky factor of their Gram), which spans the same space, so the least-
// squares solution is the same; the condition drops to ~1e6.  The solution c
// in that basis is mapped back to Alard-Lupton coefficients a = S c in FP64.
//
// Design rows are stamp pixels; the columns are [X_0, p_k X_m (m >= 1),
// p_k (background)] scaled by sqrt(w), plus the target sqrt(w) I as one extra
// column, so the Gram of the augmented design holds M = C^T W C, b = C^T W I
// and I^T W I at once.  X_m = R (x) B'_m by direct 2-D convolution: on the
// tensor cores for 21 x 21 stamps and kernels (stamp_conv_tc.cu), on the CUDA
// cores otherwise (below).
#include <cuda_bf16.h>
#include <string.h>

#include <mutex>

#include "argus_internal.cuh"
#include "basis.cuh"
#include "tc_ptx.cuh"

namespace {

__device__ __forceinline__ double ipow(double x, int p) {
    double r = 1.0;
    for (int i = 0; i < p; i++) r *= x;
    return r;
}

__device__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
    return t;
}

// One block per basis function: normalised image (FP64 and FP32), its
// separable coefficients alpha/beta, and the 1-D factor rows.
__global__ void __launch_bounds__(256) basis_prepare_kernel(BasisDev b, double* img, float* imgf, float* hrow,
                                                            float* ab) {
    __shared__ double red[8];
    __shared__ double vals[ARGUS_MAX_KS * ARGUS_MAX_KS];
    const int n = blockIdx.x, g = b.g[n], p = b.p[n], q = b.q[n];
    const int ks = b.ks, r = b.r, kk = ks * ks;
    const double s0d = 2.0 * (double)b.sigma[0] * (double)b.sigma[0];
    const double sgd = 2.0 * (double)b.sigma[g] * (double)b.sigma[g];
    double part = 0.0;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
        const int u = e % ks - r, v = e / ks - r;
        part += exp(-(double)(u * u + v * v) / s0d);
        vals[e] = ipow(u, p) * ipow(v, q) * exp(-(double)(u * u + v * v) / sgd);
    }
    const double S0 = block_sum_d(part, red);
    double alpha, beta = 0.0, s = 0.0;
    if (n == 0) {
        alpha = 1.0 / S0;
    } else {
        if (p % 2 == 0 && q % 2 == 0) {
            double ps = 0.0;
            for (int e = threadIdx.x; e < kk; e += blockDim.x) ps += vals[e];
            s = block_sum_d(ps, red);
        }
        double pn = 0.0;
        for (int e = threadIdx.x; e < kk; e += blockDim.x) {
            const int u = e % ks - r, v = e / ks - r;
            const double bp = vals[e] - s * exp(-(double)(u * u + v * v) / s0d) / S0;
            pn += bp * bp;
        }
        const double nrm = sqrt(block_sum_d(pn, red));
        alpha = 1.0 / nrm;
        beta = s / nrm;
    }
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
        double Bv;
        if (n == 0) {
            Bv = vals[e] * alpha;
        } else {
            const int u = e % ks - r, v = e / ks - r;
            Bv = (vals[e] - s * exp(-(double)(u * u + v * v) / s0d) / S0) * alpha;
        }
        img[(long)n * kk + e] = Bv;
        imgf[(long)n * kk + e] = (float)Bv;
    }
    if (threadIdx.x == 0) {
        ab[2 * n] = (float)alpha;
        ab[2 * n + 1] = (float)beta;
    }
    if (q == 0)
        for (int iu = threadIdx.x; iu < ks; iu += blockDim.x) {
            const int u = iu - r;
            hrow[(b.hoff[g] + p) * ks + iu] = (float)(ipow(u, p) * exp(-(double)(u * u) / sgd));
        }
}

// Orthonormalise basis functions 1..nb-1 in pixel space (one CTA, FP64):
// G = B^T B, G = L L^T, S = L^-T (upper triangular), B'_m = sum_n S[n][m] B_n.
// imgf receives the FP32 images of B'_0 = B_0 and B'_m; S is stored [nb][nb]
// with S[0][0] = 1.  work holds G / L ((nb-1)^2 doubles).
__global__ void __launch_bounds__(1024) basis_ortho_kernel(BasisDev b, const double* img, float* imgf, double* S,
                                                           double* work) {
    const int nb = b.nb, m1 = nb - 1, kk = b.ks * b.ks, tid = threadIdx.x;
    double* G = work;                       // [m1][m1], lower triangle becomes L
    for (int e = tid; e < m1 * m1; e += blockDim.x) {
        const int i = e / m1, j = e - i * m1;
        if (j > i) continue;
        const double* bi = img + (long)(i + 1) * kk;
        const double* bj = img + (long)(j + 1) * kk;
        double acc = 0.0;
        for (int t = 0; t < kk; t++) acc += bi[t] * bj[t];
        G[i * m1 + j] = acc;
    }
    __syncthreads();
    // Cholesky (column by column, the column's rows in parallel)
    for (int j = 0; j < m1; j++) {
        if (tid == 0) {
            double d = G[j * m1 + j];
            for (int k = 0; k < j; k++) d -= G[j * m1 + k] * G[j * m1 + k];
            G[j * m1 + j] = sqrt(d > 0.0 ? d : 1e-300);
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < m1; i += blockDim.x) {
            double v = G[i * m1 + j];
            for (int k = 0; k < j; k++) v -= G[i * m1 + k] * G[j * m1 + k];
            G[i * m1 + j] = v / G[j * m1 + j];
        }
        __syncthreads();
    }
    // S = L^-T: column m of S solves L^T s = e_m (back substitution)
    for (int e = tid; e < nb * nb; e += blockDim.x) S[e] = 0.0;
    __syncthreads();
    if (tid == 0) S[0] = 1.0;
    for (int m = tid; m < m1; m += blockDim.x) {
        for (int i = m; i >= 0; i--) {
            double v = (i == m) ? 1.0 : 0.0;
            for (int k = i + 1; k <= m; k++) v -= G[k * m1 + i] * S[(k + 1) * nb + (m + 1)];
            S[(i + 1) * nb + (m + 1)] = v / G[i * m1 + i];
        }
    }
    __syncthreads();
    for (int e = tid; e < nb * kk; e += blockDim.x) {
        const int m = e / kk, t = e - m * kk;
        double v;
        if (m == 0) {
            v = img[t];
        } else {
            v = 0.0;
            for (int n = 1; n <= m; n++) v += S[n * nb + m] * img[(long)n * kk + t];
        }
        imgf[e] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// K3: X_m = R (x) B'_m on every stamp pixel by direct 2-D convolution, one CTA
// per stamp.  The reference window and a group of basis images sit in shared
// memory; each work item is 4 basis functions x 4 stamp pixels (16 FP32
// accumulators).  X layout: X[(s * nb + m) * ss + pix], pix = j * stamp + i.
__global__ void __launch_bounds__(256) stamp_conv_kernel(BasisDev b, const float* ref, long pitch, int w, int h,
                                                         const int* centers, const int* n_stamps, int stamp,
                                                         const float* imgf, int group, float* X) {
    extern __shared__ __align__(16) float sm[];
    const int s = blockIdx.x;
    if (s >= *n_stamps) return;
    const int ks = b.ks, r = b.r, kk = ks * ks, hs = stamp / 2, WW = stamp + 2 * r, ss = stamp * stamp;
    const int nb = b.nb;
    const int xs = centers[2 * s], ys = centers[2 * s + 1];
    float* Xs = X + (long)s * nb * ss;
    const bool valid = xs - hs - r >= 0 && xs + hs + r <= w - 1 && ys - hs - r >= 0 && ys + hs + r <= h - 1;
    if (!valid) {
        for (int e = threadIdx.x; e < nb * ss; e += blockDim.x) Xs[e] = 0.0f;
        return;
    }
    float* Rw = sm;                  // [WW][WW]
    float* Bs = Rw + WW * WW;        // [group][kk]
    const int wx0 = xs - hs - r, wy0 = ys - hs - r;
    for (int e = threadIdx.x; e < WW * WW; e += blockDim.x) {
        const int wj = e / WW, wi = e - wj * WW;
        Rw[e] = __ldg(ref + (long)(wy0 + wj) * pitch + wx0 + wi);
    }
    const int npq = (ss + 3) / 4;
    for (int g0 = 0; g0 < nb; g0 += group) {
        const int gn = min(group, nb - g0);
        __syncthreads();
        for (int e = threadIdx.x; e < gn * kk; e += blockDim.x) Bs[e] = __ldg(imgf + (long)g0 * kk + e);
        __syncthreads();
        const int nfq = (gn + 3) / 4;
        for (int item = threadIdx.x; item < nfq * npq; item += blockDim.x) {
            const int fq = item / npq, pq = item - fq * npq;
            int off[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int pix = min(pq * 4 + t, ss - 1);
                const int j = pix / stamp, i = pix - j * stamp;
                off[t] = (j + 2 * r) * WW + (i + 2 * r);   // window index of R(x, y) + (2r, 2r) shift
            }
            const float* bf[4];
#pragma unroll
            for (int q = 0; q < 4; q++) bf[q] = Bs + (long)min(fq * 4 + q, gn - 1) * kk;
            float acc[4][4];
#pragma unroll
            for (int q = 0; q < 4; q++)
#pragma unroll
                for (int t = 0; t < 4; t++) acc[q][t] = 0.0f;
            // tap (du, dv) = (iu - r, iv - r): R(x - du, y - dv) = Rw[(j + 2r - iv) * WW + (i + 2r - iu)]
            for (int iv = 0; iv < ks; iv++) {
                for (int iu = 0; iu < ks; iu++) {
                    const int tap = iv * ks + iu, sh = iv * WW + iu;
                    float rv[4], bv[4];
#pragma unroll
                    for (int t = 0; t < 4; t++) rv[t] = Rw[off[t] - sh];
#pragma unroll
                    for (int q = 0; q < 4; q++) bv[q] = bf[q][tap];
#pragma unroll
                    for (int q = 0; q < 4; q++)
#pragma unroll
                        for (int t = 0; t < 4; t++) acc[q][t] = fmaf(bv[q], rv[t], acc[q][t]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int m = g0 + fq * 4 + q;
                if (fq * 4 + q >= gn) break;
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const int pix = pq * 4 + t;
                    if (pix < ss) Xs[(long)m * ss + pix] = acc[q][t];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Design rows
struct GramArgs {
    const float* X;
    const float* sci;
    const float* var;
    const uint8_t* flags;
    const int* centers;
    const int* n_stamps;
    long pitch;
    int w, h, W, H;
    int stamp, ss, r, max_stamps;
    int nb, Ks, Kb, Nc, NP, sdeg, bgdeg;
    float* part;
    int nslots;
    int* status;
};

constexpr int META = 16;   // per-row metadata: sqw, sqw*I, w, valid, s, pix, p_k[6] at 6.., pb[6] at 12..? (see row_meta)

__device__ __forceinline__ void terms_f(float xt, float yt, int deg, float* out) {
    int k = 0;
    float xi = 1.0f;
    for (int i = 0; i <= deg; i++) {
        float yj = 1.0f;
        for (int j = 0; j <= deg - i; j++) {
            out[k++] = xi * yj;
            yj *= yt;
        }
        xi *= xt;
    }
}

// meta layout: [0] sqrt(w) (0 if unused), [1] sqrt(w) * I, [2] w, [3] I, [4..10) p_k, [10..16) pb_k.
// Row index and stamp are recomputed by callers from rho.
__device__ void row_meta(const GramArgs& g, long rho, long nrows, float* m) {
    for (int i = 0; i < META; i++) m[i] = 0.0f;
    if (rho >= nrows) return;
    const int s = (int)(rho / g.ss), pix = (int)(rho - (long)s * g.ss);
    const int hs = g.stamp / 2;
    const int xs = g.centers[2 * s], ys = g.centers[2 * s + 1];
    if (!(xs - hs - g.r >= 0 && xs + hs + g.r <= g.w - 1 && ys - hs - g.r >= 0 && ys + hs + g.r <= g.h - 1))
        return;
    const int x = xs - hs + pix % g.stamp, y = ys - hs + pix / g.stamp;
    const long p = (long)y * g.pitch + x;
    const float v = g.var[p], I = g.sci[p];
    const float xt = g.W > 1 ? (float)(2 * x - (g.W - 1)) / (float)(g.W - 1) : 0.0f;
    const float yt = g.H > 1 ? (float)(2 * y - (g.H - 1)) / (float)(g.H - 1) : 0.0f;
    terms_f(xt, yt, g.sdeg, m + 4);
    terms_f(xt, yt, g.bgdeg, m + 10);
    if (g.flags[p] == 0 && v > 0.0f && isfinite(v) && isfinite(I)) {
        const float wt = 1.0f / v;
        m[0] = sqrtf(wt);
        m[1] = m[0] * I;
        m[2] = wt;
        m[3] = I;
    }
}

// column descriptor: code = n (>= 0) with spatial term k, or -1 - kb for a
// background term, or -100 for the target, or -200 for padding.
__device__ __forceinline__ void col_code(const GramArgs& g, int j, int& n, int& k) {
    if (j == 0) { n = 0; k = 0; return; }
    const int nx = 1 + (g.nb - 1) * g.Ks;
    if (j < nx) { n = 1 + (j - 1) / g.Ks; k = (j - 1) % g.Ks; return; }
    if (j < g.Nc) { n = -1 - (j - nx); k = 0; return; }
    if (j == g.Nc) { n = -100; k = 0; return; }
    n = -200; k = 0;
}


// K3, register-blocked form for 21x21 stamps (used for 11 x 11 kernels; 21 x 21
// kernels run on the tensor cores): three stamps side by side per
// CTA (63 columns over two lane-halves), warp g owns basis functions
// 4g .. 4g+3 (warp-uniform basis loads are broadcasts), a thread owns one
// column and all 21 rows of its four functions (84 accumulators).  Per tap
// column the 41 window values of the thread's column are loaded once, then
// KS taps x 21 rows x 4 functions of FMAs: ~93 % of the issued instructions.
constexpr int SC_ST = 21, SC_NS = 3;

template <int KS>
__global__ void __launch_bounds__(416, 1) stamp_conv_fast_kernel(BasisDev b, const float* ref, long pitch, int w,
                                                                 int h, const int* centers, const int* n_stamps,
                                                                 const float* imgf, float* X) {
    constexpr int R = KS / 2, WW = SC_ST + 2 * R, SS = SC_ST * SC_ST, KK = KS * KS;
    extern __shared__ __align__(16) float scs[];
    float* Rw = scs;                               // [SC_NS][WW][WW]
    float* Bs = Rw + SC_NS * WW * WW;              // [nb][KK]
    __shared__ int valid_s[SC_NS];
    const int nb = b.nb;
    const int ns = *n_stamps;
    const int s0 = blockIdx.x * SC_NS;
    if (s0 >= ns) return;
    if (threadIdx.x < SC_NS) {
        const int s = s0 + threadIdx.x, hs = SC_ST / 2;
        int v = 0;
        if (s < ns) {
            const int xs = centers[2 * s], ys = centers[2 * s + 1];
            v = xs - hs - R >= 0 && xs + hs + R <= w - 1 && ys - hs - R >= 0 && ys + hs + R <= h - 1;
        }
        valid_s[threadIdx.x] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < SC_NS * WW * WW; e += blockDim.x) {
        const int t = e / (WW * WW), rem = e - t * WW * WW;
        const int wj = rem / WW, wi = rem - wj * WW;
        float v = 0.0f;
        if (valid_s[t]) {
            const int s = s0 + t;
            const int wx0 = centers[2 * s] - SC_ST / 2 - R, wy0 = centers[2 * s + 1] - SC_ST / 2 - R;
            v = __ldg(ref + (long)(wy0 + wj) * pitch + wx0 + wi);
        }
        Rw[e] = v;
    }
    for (int e = threadIdx.x; e < nb * KK; e += blockDim.x) Bs[e] = __ldg(imgf + e);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = warp;                           // function group
    if (4 * g >= nb) return;
    for (int half = 0; half < 2; half++) {
        const int c = half * 32 + lane;           // column of the 63-wide strip
        const bool live = c < SC_NS * SC_ST;
        const int t = live ? c / SC_ST : 0, i = live ? c - t * SC_ST : 0;
        const float* rw = Rw + t * WW * WW;
        float acc[SC_ST][4];
#pragma unroll
        for (int j = 0; j < SC_ST; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[j][q] = 0.0f;
        const float* bf[4];
#pragma unroll
        for (int q = 0; q < 4; q++) bf[q] = Bs + min(4 * g + q, nb - 1) * KK;
        // tap (iu, iv): R(x - iu + R, y - iv + R) = Rw[j + 2R - iv][i + 2R - iu]
#pragma unroll 1
        for (int iu = 0; iu < KS; iu++) {
            float win[WW];
#pragma unroll
            for (int m = 0; m < WW; m++) win[m] = rw[m * WW + i + 2 * R - iu];
#pragma unroll
            for (int iv = 0; iv < KS; iv++) {
                float bv[4];
#pragma unroll
                for (int q = 0; q < 4; q++) bv[q] = bf[q][iv * KS + iu];
#pragma unroll
                for (int j = 0; j < SC_ST; j++)
#pragma unroll
                    for (int q = 0; q < 4; q++) acc[j][q] = fmaf(bv[q], win[j + 2 * R - iv], acc[j][q]);
            }
        }
        if (live && s0 + t < ns) {
            float* Xs = X + (long)(s0 + t) * nb * SS;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int m = 4 * g + q;
                if (m < nb)
#pragma unroll
                    for (int j = 0; j < SC_ST; j++) Xs[(long)m * SS + j * SC_ST + i] = valid_s[t] ? acc[j][q] : 0.0f;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Per-row design weights, computed once per fit for every design row:
// [0, 6) sqrt(w) p_k, [6, 12) sqrt(w) pb_k, [12] sqrt(w) I, the rest 0; all 0
// for unweighted rows, rows of skipped stamps and rows past the stamp count.
constexpr int RMETA = 16;

__global__ void __launch_bounds__(256) row_weights_kernel(GramArgs g, float* rw) {
    const long nrows = (long)min(*g.n_stamps, g.max_stamps) * g.ss;
    const long rows_alloc = (long)g.max_stamps * g.ss;
    for (long rho = blockIdx.x * (long)blockDim.x + threadIdx.x; rho < rows_alloc;
         rho += (long)gridDim.x * blockDim.x) {
        float m[META];
        row_meta(g, rho, nrows, m);
        float o[RMETA];
#pragma unroll
        for (int k = 0; k < 6; k++) {
            o[k] = m[0] * m[4 + k];
            o[6 + k] = m[0] * m[10 + k];
        }
        o[12] = m[1];
        o[13] = o[14] = o[15] = 0.0f;
        float4* dst = reinterpret_cast<float4*>(rw + rho * RMETA);
#pragma unroll
        for (int q = 0; q < 4; q++) dst[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
}

// The weighted design matrix C [rows][NP] (FP32, row-major), materialised once
// per fit: C[rho][j] = sqrt(w) p_k X_n (n >= 0), sqrt(w) pb_k (background),
// sqrt(w) I (target), 0 (padding); rows past the stamp count are zero up to the
// next multiple of 32.  One CTA per 32 rows stages the rows' weights and basis
// values in shared memory and writes whole rows (coalesced).
constexpr int GT = 64;
constexpr int GK = 32;

__global__ void __launch_bounds__(256) design_kernel(GramArgs g, const float* rw, float* C) {
    extern __shared__ int dsm[];
    int* cn = dsm;                                   // [NP] basis index, or -1
    int* cs = dsm + g.NP;                            // [NP] weight slot, or -1 (padding)
    __shared__ float w[GK][RMETA];
    __shared__ float xv[GK][ARGUS_MAX_NB + 1];
    for (int j = threadIdx.x; j < g.NP; j += blockDim.x) {
        int n, k;
        col_code(g, j, n, k);
        cn[j] = n >= 0 ? n : -1;
        cs[j] = n >= 0 ? k : (n == -100 ? 12 : (n == -200 ? -1 : 6 + (-1 - n)));
    }
    const long nrows = (long)min(*g.n_stamps, g.max_stamps) * g.ss;
    const long nchunks = (nrows + GK - 1) / GK;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long rho0 = ch * GK;
        __syncthreads();
        // weights: two rows per warp per step (row warp * 2 + (lane >> 4), slot lane & 15)
        for (int k = warp * 2 + (lane >> 4); k < GK; k += 16) {
            const long rho = rho0 + k;
            w[k][lane & 15] = rho < nrows ? rw[rho * RMETA + (lane & 15)] : 0.0f;
        }
        // basis values: lane = row within the chunk (coalesced over pixels), warp strides over n
        {
            const long rho = rho0 + lane;
            const bool in = rho < nrows;
            const int s = in ? (int)(rho / g.ss) : 0;
            const int pix = in ? (int)(rho - (long)s * g.ss) : 0;
            const float* xs = g.X + (long)s * g.nb * g.ss + pix;
            for (int n = warp; n < g.nb; n += 8) xv[lane][n] = in ? __ldg(xs + (long)n * g.ss) : 0.0f;
        }
        __syncthreads();
        // one warp per row, lanes along the columns (coalesced writes)
        for (int k = warp; k < GK; k += 8) {
            float* crow = C + (rho0 + k) * g.NP;
            for (int j = lane; j < g.NP; j += 32) {
                const int n = cn[j], sl = cs[j];
                const float wt = sl >= 0 ? w[k][sl] : 0.0f;
                // X of skipped stamps holds no defined values: a zero weight gives 0
                crow[j] = (n >= 0 && wt != 0.0f) ? wt * xv[k][n] : wt;
            }
        }
    }
}

// K4 (FP32): C^T C on 64x64 tiles of the upper triangle, 4x4 outputs per
// thread.  Grid (tile pair, slot): the pairs that read one row chunk are
// launched side by side, so a chunk comes from DRAM about once and from L2 for
// the other pairs.  The 32-row chunks of A and B stream in by 16-byte cp.async,
// double-buffered; per chunk the FP32 products are summed and folded into a
// double-float accumulator (error-free two-sum).
__global__ void __launch_bounds__(256, 3) gram_cp_kernel(GramArgs g, const float* C, int ntile) {
    __shared__ __align__(16) float As[2][GK][GT + 4];
    __shared__ __align__(16) float Bs[2][GK][GT + 4];
    int pr = blockIdx.x, ti = 0;
    while (pr >= ntile - ti) { pr -= ntile - ti; ti++; }
    const int tj = ti + pr;
    const bool diag = ti == tj;
    const int tid = threadIdx.x;
    const int slot = blockIdx.y, nslots = gridDim.y;
    const long nrows = (long)min(*g.n_stamps, g.max_stamps) * g.ss;
    const long nchunks = (nrows + GK - 1) / GK;
    auto load = [&](int buf, long ch) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int idx = tid + h * 256;       // 32 rows x 16 float4 per operand
            const int row = idx >> 4, c4 = idx & 15;
            const long rbase = (ch * GK + row) * g.NP;
            const int ca = ti * GT + 4 * c4, cb = tj * GT + 4 * c4;
            tc::cp_async16(&As[buf][row][4 * c4], C + rbase + (ca < g.NP ? ca : 0), ca < g.NP ? 16 : 0);
            if (!diag) tc::cp_async16(&Bs[buf][row][4 * c4], C + rbase + (cb < g.NP ? cb : 0), cb < g.NP ? 16 : 0);
        }
    };
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) hi[i][j] = lo[i][j] = 0.0f;
    const int ty = tid / 16, tx = tid % 16;
    long ch = slot;
    if (ch < nchunks) load(0, ch);
    tc::cp_async_commit();
    for (int it = 0; ch < nchunks; ch += nslots, it++) {
        const int cur = it & 1;
        if (ch + nslots < nchunks) load(cur ^ 1, ch + nslots);
        tc::cp_async_commit();
        tc::cp_async_wait<1>();                  // chunk ch has landed (own copies)
        __syncthreads();
        const float(*Ab)[GT + 4] = As[cur];
        const float(*Bb)[GT + 4] = diag ? As[cur] : Bs[cur];
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = 0.0f;
#pragma unroll 8
        for (int k = 0; k < GK; k++) {
            const float4 a4 = *reinterpret_cast<const float4*>(&Ab[k][ty * 4]);
            const float4 b4 = *reinterpret_cast<const float4*>(&Bb[k][tx * 4]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float a = hi[i][j], b = acc[i][j];
                const float sum = a + b;
                const float bp = sum - a;
                lo[i][j] += (a - (sum - bp)) + (b - bp);
                hi[i][j] = sum;
            }
        __syncthreads();                         // buffer cur is free for the load two chunks on
    }
    tc::cp_async_wait<0>();
    float* out = g.part + (long)slot * g.NP * g.NP;
    float* outl = g.part + (long)(slot + nslots) * g.NP * g.NP;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int row = ti * GT + ty * 4 + i;
        if (row >= g.NP) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int col = tj * GT + tx * 4 + j;
            if (col < g.NP) {
                out[(long)row * g.NP + col] = hi[i][j];
                outl[(long)row * g.NP + col] = lo[i][j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K4 on the tensor cores (TF32, BF16, or BF16 split into hi + lo).
//
// The weighted design matrix is written once per fit as tiles of 32 rows that
// are already in the MMA's no-swizzle K-major operand layout: for chunk ch,
// element (row r of the chunk, column j) sits at
//   ch * CH_BYTES + part * TILE_BYTES + (j / 8) * SBO + (r / E) * 128 + (j % 8) * 16 + (r % E) * ESZ,
// E = elements per 16-byte core-matrix row (8 BF16 or 4 TF32), SBO = (32 / E) * 128,
// part 0 = the value rounded to the format (hi), part 1 = the rounded remainder
// (lo, BF16 split only).  A column range of 8 g .. 8 g + 8 n - 1 of a chunk is then
// n * SBO contiguous bytes, so a block's operands are single bulk copies.
constexpr int TC_KC = 32;                              // design rows per chunk (pipeline stage)
constexpr long long TC_WAIT_LIMIT = 4000000000LL;      // ~2 s of SM clock

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t to_tf32(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return r;
}

// FMT 1 = BF16, 2 = TF32; P = 1 (rounded operand) or 4 (BF16 hi + lo split, all four
// products hi*hi + hi*lo + lo*hi + lo*lo).  Either way the result is the exact Gram
// (up to FP32 accumulation) of a design perturbed by its rounding: positive
// semi-definite and consistent.  Dropping lo*lo would subtract the PSD matrix
// sum lo lo^T instead, which moves near-degenerate directions of the normal
// matrix towards singularity (measured: worse than one rounded operand).
template <int FMT, int P>
struct TcGram {
    static constexpr int ESZ = FMT == 1 ? 2 : 4;
    static constexpr int E = 16 / ESZ;
    static constexpr int NQ = TC_KC / E;                       // core matrices along K per chunk
    static constexpr uint32_t SBO = NQ * 128;                  // bytes per 8-column group of a chunk
    static constexpr int KMMA = FMT == 1 ? 16 : 8;             // K per MMA
    static constexpr int NPART = P == 4 ? 2 : 1;
    static_assert(P == 1 || (P == 4 && FMT == 1), "hi/lo split of BF16 only");
    __host__ __device__ static constexpr uint32_t tile_bytes(int NP) { return (uint32_t)(NP / 8) * SBO; }
    __host__ __device__ static constexpr uint32_t chunk_bytes(int NP) { return NPART * tile_bytes(NP); }
};

// Design tiles: one CTA per chunk of 32 rows at a time stages the rows'
// weights and basis values (as design_kernel does), then each thread writes
// one 16-byte core-matrix row (E rows of one column) of each part; consecutive
// threads write consecutive 16-byte rows of one core-matrix column group.
template <int FMT, int P>
__global__ void __launch_bounds__(256) design_tiles_kernel(GramArgs g, const float* rw, uint8_t* tiles) {
    using T = TcGram<FMT, P>;
    extern __shared__ int dsm[];
    int* cn = dsm;                                   // [NP] basis index, or -1
    int* cs = dsm + g.NP;                            // [NP] weight slot, or -1 (padding)
    __shared__ float w[TC_KC][RMETA];
    __shared__ float xv[TC_KC][ARGUS_MAX_NB + 1];
    for (int j = threadIdx.x; j < g.NP; j += blockDim.x) {
        int n, k;
        col_code(g, j, n, k);
        cn[j] = n >= 0 ? n : -1;
        cs[j] = n >= 0 ? k : (n == -100 ? 12 : (n == -200 ? -1 : 6 + (-1 - n)));
    }
    const long nrows = (long)min(*g.n_stamps, g.max_stamps) * g.ss;
    const long nchunks = (nrows + TC_KC - 1) / TC_KC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int units = g.NP * T::NQ;                  // 16-byte rows per part of a chunk
    const uint32_t tb = T::tile_bytes(g.NP);
    for (long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long rho0 = ch * TC_KC;
        __syncthreads();
        for (int k = warp * 2 + (lane >> 4); k < TC_KC; k += 16) {
            const long rho = rho0 + k;
            w[k][lane & 15] = rho < nrows ? rw[rho * RMETA + (lane & 15)] : 0.0f;
        }
        {
            const long rho = rho0 + lane;
            const bool in = rho < nrows;
            const int s = in ? (int)(rho / g.ss) : 0;
            const int pix = in ? (int)(rho - (long)s * g.ss) : 0;
            const float* xs = g.X + (long)s * g.nb * g.ss + pix;
            for (int n = warp; n < g.nb; n += 8) xv[lane][n] = in ? __ldg(xs + (long)n * g.ss) : 0.0f;
        }
        __syncthreads();
        uint8_t* base = tiles + (size_t)ch * T::chunk_bytes(g.NP);
        for (int u = threadIdx.x; u < units; u += blockDim.x) {
            const int jg = u / (8 * T::NQ), q = (u >> 3) % T::NQ, j = jg * 8 + (u & 7);
            const int n = cn[j], sl = cs[j];
            float v[T::E];
#pragma unroll
            for (int t = 0; t < T::E; t++) {
                const int r = q * T::E + t;
                const float wt = sl >= 0 ? w[r][sl] : 0.0f;
                // X of skipped stamps holds no defined values: a zero weight gives 0
                v[t] = (n >= 0 && wt != 0.0f) ? wt * xv[r][n] : wt;
            }
            uint4 hi, lo;
            if constexpr (FMT == 1) {
                hi = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                                pack_bf16x2(v[6], v[7]));
                if constexpr (P == 4) {
                    float l[8];
                    const uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        l[2 * t] = v[2 * t] - __uint_as_float(hw[t] << 16);
                        l[2 * t + 1] = v[2 * t + 1] - __uint_as_float(hw[t] & 0xffff0000u);
                    }
                    lo = make_uint4(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]), pack_bf16x2(l[4], l[5]),
                                    pack_bf16x2(l[6], l[7]));
                }
            } else {
                hi = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
            }
            const uint32_t off = (uint32_t)jg * T::SBO + (uint32_t)q * 128 + (uint32_t)(u & 7) * 16;
            *reinterpret_cast<uint4*>(base + off) = hi;
            if constexpr (P == 4) *reinterpret_cast<uint4*>(base + tb + off) = lo;
        }
    }
}

// One block of the augmented Gram: rows 128 rb .. +127 (the MMA's M; rows past
// NP are zero) and columns c0 .. c0 + n - 1 (the MMA's N, n <= GRAM_CW).
struct GramBlock {
    int rb, c0, n;
};
constexpr int GRAM_MAX_BLOCKS = 64;
struct GramBlocks {
    GramBlock b[GRAM_MAX_BLOCKS];
};
// 128 columns per block: an epilogue thread then holds 2 x 64 accumulators; ten
// warps put three on some SM partitions, which caps a thread at 168 registers
constexpr int GRAM_CW = 128;                           // columns per block
constexpr int GRAM_GROUP = 8;                          // chunks (256 rows) per FP32 accumulation
constexpr int GRAM_STAGES = 3;
constexpr int GRAM_EPI_WARPS = 8;                      // two per TMEM lane quadrant
constexpr int GRAM_THREADS = (2 + GRAM_EPI_WARPS) * 32;
constexpr int GRAM_EPI_COLS = GRAM_CW / 2;             // columns per epilogue warp

template <int FMT, int P>
struct GramShared {
    using T = TcGram<FMT, P>;
    // per stage: A (16 column groups) then B (GRAM_CW / 8 column groups), part after part
    uint8_t stage[GRAM_STAGES][T::NPART][16 + GRAM_CW / 8][T::SBO];
    uint64_t full[GRAM_STAGES], empty[GRAM_STAGES], tfull[2], tempty[2];
    uint32_t tmem;
    int abort;
};

template <class SH>
__device__ __forceinline__ bool gram_wait(SH& S, uint64_t* bar, uint32_t parity, int* status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (S.abort) return false;
    if (!tc::mbar_wait_bounded(bar, parity, TC_WAIT_LIMIT)) {
        S.abort = 1;
        argus_latch(status, ARGUS_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// CTA (split, block): the block's partial sum over the chunks ch = split,
// split + nsplit, ...  Warp 0 (one thread) moves each chunk's A and B column
// ranges into a stage by bulk copies; warp 1 (one thread) issues the MMAs of a
// chunk into one of two TMEM accumulators, switching every GRAM_GROUP chunks;
// warps 2-9 drain a finished accumulator (256 rows of FP32 sums) into
// double-float (hi, lo) registers with an error-free two-sum, so the FP32
// accumulation never runs over more than 256 rows.  The block's hi and lo halves
// go to partial slots split and split + nsplit.
template <int FMT, int P>
__global__ void __launch_bounds__(GRAM_THREADS, 1) gram_tc_kernel(GramArgs g, const uint8_t* tiles, GramBlocks blocks) {
    using T = TcGram<FMT, P>;
    using Sh = GramShared<FMT, P>;
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    Sh& S = *reinterpret_cast<Sh*>(gsm_raw + ((1024 - (tc::smem_u32(gsm_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GramBlock blk = blocks.b[blockIdx.y];
    const int split = blockIdx.x, nsplit = gridDim.x;
    const int NP = g.NP, ngrp = NP / 8;
    const int ag0 = 16 * blk.rb, nag = min(16, ngrp - ag0);   // A column groups (rows of the block)
    const int bg0 = blk.c0 / 8, nbg = blk.n / 8;               // B column groups
    const uint32_t tb = T::tile_bytes(NP), cb = T::chunk_bytes(NP);
    const long nrows = (long)min(*g.n_stamps, g.max_stamps) * g.ss;
    const long nchunks = (nrows + TC_KC - 1) / TC_KC;
    const int nit = nchunks > split ? (int)((nchunks - 1 - split) / nsplit + 1) : 0;   // this CTA's chunks
    const int ngroups = (nit + GRAM_GROUP - 1) / GRAM_GROUP;

    // A rows past NP are never copied: zero them once in every stage and part
    for (int e = tid; e < GRAM_STAGES * T::NPART * (16 - nag) * (int)(T::SBO / 16); e += blockDim.x) {
        const int per = (16 - nag) * (T::SBO / 16);
        const int sp = e / per, rem = e - sp * per;
        const int st = sp / T::NPART, pt = sp - st * T::NPART;
        *reinterpret_cast<uint4*>(&S.stage[st][pt][nag][0] + 16 * rem) = make_uint4(0, 0, 0, 0);
    }
    if (tid == 0) {
        for (int s = 0; s < GRAM_STAGES; s++) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&S.tfull[b], 1);
            tc::mbar_init(&S.tempty[b], GRAM_EPI_WARPS);
        }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, 2 * GRAM_CW);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;

    if (warp == 0) {
        // ---------------- producer
        if (lane == 0) {
            const uint32_t abytes = (uint32_t)nag * T::SBO, bbytes = (uint32_t)nbg * T::SBO;
            for (int it = 0; it < nit; it++) {
                const int s = it % GRAM_STAGES;
                if (it >= GRAM_STAGES && !gram_wait(S, &S.empty[s], (it / GRAM_STAGES - 1) & 1, g.status)) break;
                const uint8_t* src = tiles + (size_t)(split + (long)it * nsplit) * cb;
                tc::mbar_arrive_expect_tx(&S.full[s], T::NPART * (abytes + bbytes));
#pragma unroll
                for (int pt = 0; pt < T::NPART; pt++) {
                    tc::bulk_g2s(&S.stage[s][pt][0][0], src + pt * tb + (size_t)ag0 * T::SBO, abytes, &S.full[s]);
                    tc::bulk_g2s(&S.stage[s][pt][16][0], src + pt * tb + (size_t)bg0 * T::SBO, bbytes, &S.full[s]);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(FMT, 128, blk.n);
            int last = -1;
            for (int it = 0; it < nit; it++) {
                const int s = it % GRAM_STAGES, gi = it / GRAM_GROUP, ab = gi & 1;
                const bool first = it % GRAM_GROUP == 0;
                if (first && gi >= 2 && !gram_wait(S, &S.tempty[ab], (gi / 2 - 1) & 1, g.status)) break;
                if (!gram_wait(S, &S.full[s], (it / GRAM_STAGES) & 1, g.status)) break;
                tc::fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * GRAM_CW);
#pragma unroll
                for (int k = 0; k < TC_KC / T::KMMA; k++) {
                    const uint32_t koff = (uint32_t)k * 2 * 128;
#pragma unroll
                    for (int pr = 0; pr < P; pr++) {
                        // products hi*hi, hi*lo, lo*hi, lo*lo
                        const int pa = pr >> 1, pb = pr & 1;
                        const uint64_t ad = tc::smem_desc(tc::smem_u32(&S.stage[s][pa][0][0]) + koff, 128, T::SBO);
                        const uint64_t bd = tc::smem_desc(tc::smem_u32(&S.stage[s][pb][16][0]) + koff, 128, T::SBO);
                        const uint32_t acc = (first && k == 0 && pr == 0) ? 0u : 1u;
                        if constexpr (FMT == 1) tc::mma_bf16(d, ad, bd, idesc, acc);
                        else tc::mma_tf32(d, ad, bd, idesc, acc);
                    }
                }
                tc::commit(&S.empty[s]);
                if (it % GRAM_GROUP == GRAM_GROUP - 1 || it == nit - 1) tc::commit(&S.tfull[ab]);
                last = it;
            }
            // every MMA lands before TMEM is released: the last commit covers all
            if (last >= 0) {
                const int gi = last / GRAM_GROUP;
                if (!tc::mbar_wait_bounded(&S.tfull[gi & 1], (gi / 2) & 1, TC_WAIT_LIMIT)) {
                    S.abort = 1;
                    argus_latch(g.status, ARGUS_ERR_TIMEOUT);
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM lane quadrant q = warp % 4, column half h
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = blk.rb * 128 + q * 32 + lane;
        const int cl0 = h * GRAM_EPI_COLS;                         // first local column of this warp
        float hi[GRAM_EPI_COLS], lo[GRAM_EPI_COLS];
#pragma unroll
        for (int c = 0; c < GRAM_EPI_COLS; c++) hi[c] = lo[c] = 0.0f;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        for (int gi = 0; gi < ngroups; gi++) {
            const int ab = gi & 1;
            bool ok = true;
            if (lane == 0) ok = gram_wait(S, &S.tfull[ab], (gi / 2) & 1, g.status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc::fence_after();
#pragma unroll
            for (int c16 = 0; c16 < GRAM_EPI_COLS / 16; c16++) {
                if (cl0 + c16 * 16 < blk.n) {                      // warp-uniform
                    uint32_t r[16];
                    tc::tmem_ld16_nowait(tl + (uint32_t)(ab * GRAM_CW + cl0 + c16 * 16), r);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 16; t++) {
                        const int c = c16 * 16 + t;
                        const float v = __uint_as_float(r[t]);
                        const float a = hi[c], sum = a + v, bp = sum - a;
                        lo[c] += (a - (sum - bp)) + (v - bp);
                        hi[c] = sum;
                    }
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.tempty[ab]);
        }
        if (row < NP) {
            float* oh = g.part + (long)split * NP * NP + (long)row * NP + blk.c0 + cl0;
            float* ol = g.part + (long)(split + nsplit) * NP * NP + (long)row * NP + blk.c0 + cl0;
#pragma unroll
            for (int c = 0; c < GRAM_EPI_COLS; c++) {
                if (cl0 + c < blk.n) {
                    oh[c] = hi[c];
                    ol[c] = lo[c];
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * GRAM_CW);
}

// M[i][j] = M[j][i] = sum over slots of part[slot][i][j] (i <= j), FP64, fixed order.
__global__ void gram_reduce_kernel(const float* part, int nslots, int NP, double* M) {
    const long tot = (long)NP * NP;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / NP), j = (int)(e - (long)i * NP);
        if (i > j) continue;
        double s = 0.0;
        for (int sl = 0; sl < nslots; sl++) s += (double)part[(long)sl * tot + e];
        M[(long)i * NP + j] = s;
        M[(long)j * NP + i] = s;
    }
}

// ---------------------------------------------------------------------------
// K5: FP64 linear algebra of the normal equations.
//
// Blocked right-looking Cholesky with 32-column panels, three launches per
// panel (no grid-wide waits).  FP64 issues at a small fraction of the FP32
// rate on this part, so the kernels keep FP64 dependency chains short and
// spread the FP64 work over many SMs: four warps factor the diagonal block
// (columns interleaved over the warps, reciprocal square roots from an FP32
// estimate and two FP64 Newton steps); the panel below, L_ip = A_ip L_pp^-T,
// is one row-parallel triangular solve per warp over the whole GPU, and the
// same launch solves 32 identity rows, which gives the inverse of the
// diagonal block; the trailing lower triangle is updated in 16x16 tiles
// spread over all SMs.  The diagonal-block inverses are kept, and every solve
// is one blocked forward and backward substitution that multiplies by them.
// flag[0] != 0 marks a failed factorisation for all kernels that follow.
constexpr int CB = 32;

__global__ void chol_init_kernel(const double* M, int ld, int n, double* L, double* flag) {
    const long tot = (long)n * ld;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ld), j = (int)(e - (long)i * ld);
        L[e] = (j <= i && j < n) ? M[(long)i * ld + j] : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) flag[0] = 0.0;
}

// 1/sqrt(d) for d > 0: FP32 estimate, then two Newton-Raphson steps
// r <- r (3 - d r^2) / 2 in FP64 (each squares the relative error, 2^-22 ->
// 2^-44 -> FP64 rounding).  Outside the FP32 range the FP64 library path.
__device__ __forceinline__ double rsqrt_newton(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double r = (double)rsqrtf((float)d);
    const double hd = 0.5 * d;
    r = r * fma(-hd, r * r, 1.5);
    r = r * fma(-hd, r * r, 1.5);
    return r;
}

// Factor the pb x pb diagonal block at (p, p) in place; rdiag[j] = 1 / L_jj.
// Four warps; warp w holds columns k = 4 q + w of row `lane`.
__global__ void __launch_bounds__(128) chol_diag_kernel(double* L, int ld, int p, int pb, double* rdiag, double* flag,
                                                        int* status) {
    __shared__ double col[CB];
    __shared__ int bad;
    if (flag[0] != 0.0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a[CB / 4];
#pragma unroll
    for (int q = 0; q < CB / 4; q++) {
        const int k = 4 * q + warp;
        a[q] = (lane < pb && k <= lane) ? L[(long)(p + lane) * ld + p + k] : 0.0;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CB; j++) {
        if (j < pb) {
            if (warp == (j & 3)) {
                const double d = __shfl_sync(0xffffffffu, a[j >> 2], j);
                const bool ok = d > 0.0;
                const double r = rsqrt_newton(ok ? d : 1.0);
                const double lij = lane == j ? d * r : (lane > j ? a[j >> 2] * r : 0.0);
                a[j >> 2] = lij;
                col[lane] = lij;
                if (lane == 0) {
                    rdiag[p + j] = r;
                    if (!ok) bad = 1;
                }
            }
            __syncthreads();
            const double lij = col[lane];
#pragma unroll
            for (int q = 0; q < CB / 4; q++) {
                const int k = 4 * q + warp;
                if (k > j && k <= lane) a[q] -= lij * col[k];
            }
            __syncthreads();
        }
    }
    if (bad) {
        if (threadIdx.x == 0) {
            flag[0] = 1.0;
            argus_latch(status, ARGUS_ERR_SINGULAR);
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < CB / 4; q++) {
        const int k = 4 * q + warp;
        if (lane < pb && k <= lane) L[(long)(p + lane) * ld + p + k] = a[q];
    }
}

// Row solves x L_pp^T = a, one warp per row (lane j holds x_j and row j of
// L_pp): rows p+pb .. n-1 of the panel (x replaces a in L), then identity
// rows e_r, r < pb, whose solutions are the columns of L_pp^-1 (stored to
// Dinv, row-major CB x CB).
__global__ void __launch_bounds__(256) chol_panel_kernel(double* L, int ld, int n, int p, int pb,
                                                         const double* rdiag, double* Dinv, const double* flag) {
    if (flag[0] != 0.0) return;
    const int lane = threadIdx.x & 31;
    const int rest = n - p - pb;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rest + pb) return;
    double lrow[CB];   // row `lane` of the diagonal block
#pragma unroll
    for (int k = 0; k < CB; k++) lrow[k] = (lane < pb && k <= lane) ? L[(long)(p + lane) * ld + p + k] : 0.0;
    const double rd = lane < pb ? rdiag[p + lane] : 0.0;
    const bool ident = row >= rest;
    double* Li = L + (long)(p + pb + row) * ld + p;
    double s = ident ? (lane == row - rest ? 1.0 : 0.0) : (lane < pb ? Li[lane] : 0.0);
    double x = 0.0;
#pragma unroll
    for (int j = 0; j < CB; j++) {
        if (j < pb) {
            const double xj = __shfl_sync(0xffffffffu, s, j) * __shfl_sync(0xffffffffu, rd, j);
            if (lane == j) x = xj;
            if (lane > j) s -= xj * lrow[j];
        }
    }
    if (lane < pb) {
        if (ident) {
            Dinv[lane * CB + (row - rest)] = x;
        } else {
            Li[lane] = x;
            L[(long)(p + lane) * ld + (p + pb + row)] = x;   // mirrored into the upper triangle for the backward solve
        }
    }
    if (ident && lane >= pb) Dinv[lane * CB + (row - rest)] = 0.0;
    if (ident && row - rest == pb - 1) {
        // rows/columns past pb of the block inverse are zero
        for (int r = pb; r < CB; r++) Dinv[lane * CB + r] = 0.0;
    }
}

// Trailing update A[i][k] -= sum_t L[i][p+t] L[k][p+t], p+pb <= k <= i < n, 16x16 tiles.
__global__ void __launch_bounds__(256) chol_update_kernel(double* L, int ld, int n, int p, int pb, const double* flag) {
    __shared__ double Pi[16][CB + 1], Pk[16][CB + 1];
    if (flag[0] != 0.0) return;
    const int q0 = p + pb, m = n - q0;
    const int T = (m + 15) / 16;
    int t = blockIdx.x, ti = 0;
    while (t >= ti + 1) { t -= ti + 1; ti++; }   // lower-triangle tile (ti, tk), tk <= ti
    if (ti >= T) return;
    const int tk = t;
    const int i0 = q0 + ti * 16, k0 = q0 + tk * 16;
    for (int e = threadIdx.x; e < 16 * CB; e += blockDim.x) {
        const int r = e / CB, c = e % CB;
        Pi[r][c] = (i0 + r < n && c < pb) ? L[(long)(i0 + r) * ld + p + c] : 0.0;
        Pk[r][c] = (k0 + r < n && c < pb) ? L[(long)(k0 + r) * ld + p + c] : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x / 16, c = threadIdx.x % 16;
    const int i = i0 + r, k = k0 + c;
    if (i < n && k <= i) {
        double acc = 0.0;
#pragma unroll 8
        for (int u = 0; u < CB; u++) acc += Pi[r][u] * Pk[c][u];
        L[(long)i * ld + k] -= acc;
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// x = (L L^T)^-1 rhs (rhs read with stride rs) by blocked substitution in one
// CTA of 32 warps: per 32-row block, warp w forms row w's remainder
// (rhs minus the already solved blocks) and then the block's solution is the
// product with the stored inverse of its diagonal block.  Forward with L,
// backward with L^T, read by rows from the upper triangle where the panel
// kernel mirrors L's off-diagonal blocks.  Skips when flag[0] or flag[1] is set.
__global__ void __launch_bounds__(1024) tri_solve_kernel(const double* L, int ld, int n, const double* Dinv,
                                                         const double* rhs, int rs, double* x, const double* flag) {
    extern __shared__ double ts[];   // y [n], then x [n]
    __shared__ double tt[CB];
    if (flag[0] != 0.0 || flag[1] != 0.0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = (n + CB - 1) / CB;
    double* y = ts;
    double* xs = ts + n;
    for (int p = 0; p < nb; p++) {
        const int i = p * CB + warp;
        double t = 0.0;
        if (i < n) {
            const double* Li = L + (long)i * ld;
            for (int k = lane; k < p * CB; k += 32) t += Li[k] * y[k];
            t = warp_sum_d(t);
        }
        if (lane == 0) tt[warp] = i < n ? rhs[(long)i * rs] - t : 0.0;
        __syncthreads();
        if (i < n) {
            const double v = warp_sum_d(Dinv[(long)p * CB * CB + warp * CB + lane] * tt[lane]);
            if (lane == 0) y[i] = v;
        }
        __syncthreads();
    }
    for (int p = nb - 1; p >= 0; p--) {
        const int i = p * CB + warp;
        double t = 0.0;
        if (i < n) {
            const double* Ui = L + (long)i * ld;   // row i of L^T (the mirrored upper triangle)
            for (int k = (p + 1) * CB + lane; k < n; k += 32) t += Ui[k] * xs[k];
            t = warp_sum_d(t);
        }
        if (lane == 0) tt[warp] = i < n ? y[i] - t : 0.0;
        __syncthreads();
        if (i < n) {
            const double v = warp_sum_d(Dinv[(long)p * CB * CB + lane * CB + warp] * tt[lane]);
            if (lane == 0) xs[i] = v;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xs[i];
}

// Residual pass over all design rows with coefficients a (FP64 in, FP32 model).
// A CTA takes 256 rows at a time (one per thread): each thread forms its
// row's model and residual e, stages its X_m in shared memory (row stride odd:
// no bank conflicts either way) and g_k = w e p_k, gb_k = w e pb_k beside them.
// Then the outputs r_(m,k) = sum_rows X_m g_k are owned by basis function:
// groups of nb threads split the 256 rows into contiguous chunks, thread
// (q, m) sums X_m g_k for every k over chunk q (the g_k are one broadcast
// read per row), and thread (q, 0) also the gb_k.  Sums are FP32 per
// chunk (at most 52 rows), FP64 across chunks, tiles and (in a fixed order)
// groups.  Also chi2 = sum w e^2 and the count of weighted rows.  Per-CTA
// partials [NP + 4] are reduced in a fixed order.
constexpr int RT = 256;
constexpr int RG = 16;   // staged g_k (0..5) and gb_k (8..13) per row

__host__ __device__ inline int resid_xst(int nb) { return nb | 1; }

__global__ void __launch_bounds__(RT) resid_kernel(GramArgs g, const float* rw, const double* a, const double* flag,
                                                   int want_r, double* part) {
    extern __shared__ __align__(16) float rsm[];   // Gs[RT][RG], Xs[RT][xst]; after the rows: red (FP64)
    __shared__ float af[1024];
    __shared__ double wchi[RT / 32], wn[RT / 32];
    if (flag[0] != 0.0 || (want_r && flag[1] != 0.0)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = g.nb, Ks = g.Ks, Kb = g.Kb, xst = resid_xst(nb);
    float* Gs = rsm;
    float* Xs = rsm + RT * RG;
    for (int j = tid; j < g.Nc; j += RT) af[j] = (float)a[j];
    const long nrows = (long)min(*g.n_stamps, g.max_stamps) * g.ss;
    const int nx = 1 + (nb - 1) * Ks;
    // output ownership: thread (q, m), q < ng groups of nb threads, rows [q ch, q ch + ch) of a tile
    const int ng = RT / nb, ch = (RT + ng - 1) / ng;
    const int q = tid / nb, m = tid - q * nb;
    const bool owner = q < ng;
    const int t0 = owner ? q * ch : 0, t1 = owner ? min(RT, t0 + ch) : 0;
    double racc[6], rbg[6];   // Ks, Kb <= 6
#pragma unroll
    for (int k = 0; k < 6; k++) racc[k] = rbg[k] = 0.0;
    double chi = 0.0, cnt = 0.0;
    __syncthreads();
    for (long base = (long)blockIdx.x * RT; base < nrows; base += (long)gridDim.x * RT) {
        const long rho = base + tid;
        // the row's weights from the per-fit table: sqrt(w) p_k, sqrt(w) pb_k, sqrt(w) I
        // (all zero for unweighted rows; p_0 = 1, so o[0] = sqrt(w))
        float o[RMETA];
        if (rho < nrows) {
            const float4* src = reinterpret_cast<const float4*>(rw + rho * RMETA);
#pragma unroll
            for (int u = 0; u < 4; u++) *reinterpret_cast<float4*>(o + 4 * u) = __ldg(src + u);
        } else {
#pragma unroll
            for (int u = 0; u < RMETA; u++) o[u] = 0.0f;
        }
        const bool use = o[0] > 0.0f;
        const int s = (int)(rho / g.ss), pix = (int)(rho - (long)s * g.ss);
        float model = 0.0f;   // sqrt(w) times the model
        // the row's nb design values are independent loads: unrolled so that several are in flight
#pragma unroll 8
        for (int n = 0; n < nb; n++) {
            const float xv = use ? __ldg(g.X + ((long)s * nb + n) * g.ss + pix) : 0.0f;
            Xs[tid * xst + n] = xv;
            float qn;
            if (n == 0) {
                qn = af[0] * o[0];
            } else {
                qn = 0.0f;
#pragma unroll
                for (int k = 0; k < 6; k++)
                    if (k < Ks) qn = fmaf(o[k], af[1 + (n - 1) * Ks + k], qn);
            }
            model = fmaf(xv, qn, model);
        }
#pragma unroll
        for (int k = 0; k < 6; k++)
            if (k < Kb) model = fmaf(o[6 + k], af[nx + k], model);
        const float ew = use ? o[12] - model : 0.0f;   // sqrt(w) (I - model)
        chi += (double)ew * (double)ew;
        cnt += use ? 1.0 : 0.0;
        {
            float gr[RG];
#pragma unroll
            for (int k = 0; k < 6; k++) {
                gr[k] = k < Ks ? ew * o[k] : 0.0f;
                gr[8 + k] = k < Kb ? ew * o[6 + k] : 0.0f;
            }
            gr[6] = gr[7] = gr[14] = gr[15] = 0.0f;
            float4* gd = reinterpret_cast<float4*>(Gs + tid * RG);
#pragma unroll
            for (int u = 0; u < 4; u++) gd[u] = make_float4(gr[4 * u], gr[4 * u + 1], gr[4 * u + 2], gr[4 * u + 3]);
        }
        __syncthreads();
        if (want_r && owner) {
            float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            float abg[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            const bool bgt = m == 0;
            for (int t = t0; t < t1; t++) {
                const float xv = Xs[t * xst + m];
                const float4 g0 = *reinterpret_cast<const float4*>(Gs + t * RG);
                const float4 g1 = *reinterpret_cast<const float4*>(Gs + t * RG + 4);
                acc[0] = fmaf(xv, g0.x, acc[0]);
                acc[1] = fmaf(xv, g0.y, acc[1]);
                acc[2] = fmaf(xv, g0.z, acc[2]);
                acc[3] = fmaf(xv, g0.w, acc[3]);
                acc[4] = fmaf(xv, g1.x, acc[4]);
                acc[5] = fmaf(xv, g1.y, acc[5]);
                if (bgt) {
                    const float4 b0 = *reinterpret_cast<const float4*>(Gs + t * RG + 8);
                    const float4 b1 = *reinterpret_cast<const float4*>(Gs + t * RG + 12);
                    abg[0] += b0.x; abg[1] += b0.y; abg[2] += b0.z; abg[3] += b0.w; abg[4] += b1.x; abg[5] += b1.y;
                }
            }
#pragma unroll
            for (int k = 0; k < 6; k++) {
                racc[k] += (double)acc[k];
                rbg[k] += (double)abg[k];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        chi += __shfl_xor_sync(0xffffffffu, chi, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) { wchi[warp] = chi; wn[warp] = cnt; }
    // the groups' sums, added in group order: red[q][m][k] (k < 6), then redbg[q][k]
    double* red = reinterpret_cast<double*>(rsm);
    double* redbg = red + ng * nb * 8;
    if (want_r && owner) {
#pragma unroll
        for (int k = 0; k < 6; k++) red[(q * nb + m) * 8 + k] = racc[k];
        if (m == 0)
#pragma unroll
            for (int k = 0; k < 6; k++) redbg[q * 8 + k] = rbg[k];
    }
    __syncthreads();
    double* out = part + (long)blockIdx.x * (g.NP + 4);
    for (int j = tid; j < g.Nc; j += RT) {
        int mm, kk;
        if (j == 0) { mm = 0; kk = 0; }
        else if (j < nx) { mm = 1 + (j - 1) / Ks; kk = (j - 1) % Ks; }
        else { mm = -1; kk = j - nx; }
        double v = 0.0;
        if (want_r)
            for (int qq = 0; qq < ng; qq++) v += mm >= 0 ? red[(qq * nb + mm) * 8 + kk] : redbg[qq * 8 + kk];
        out[j] = v;
    }
    if (tid == 0) {
        double c = 0.0, n = 0.0;
        for (int w = 0; w < RT / 32; w++) { c += wchi[w]; n += wn[w]; }
        out[g.NP] = c;
        out[g.NP + 1] = n;
    }
}

// Column j of the partials summed over parts in a fixed order: one warp per column.
__global__ void resid_reduce_kernel(const double* part, int nparts, int NP, int Nc, double* r, double* chi_n,
                                    const double* flag, int skip_if_done) {
    if (flag[0] != 0.0 || (skip_if_done && flag[1] != 0.0)) return;
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= Nc + 2) return;
    const int col = j < Nc ? j : NP + (j - Nc);
    double s = 0.0;
    for (int p = lane; p < nparts; p += 32) s += part[(long)p * (NP + 4) + col];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        if (j < Nc) r[j] = s;
        else chi_n[j - Nc] = s;
    }
}

// Refinement state, flag[]: [0] singular, [1] done, [2] previous step, [3] steps
// applied, [4] last applied step.  A step delta (relative max-norm) is applied
// unless it is larger than the previous one (the iteration diverges: keep the
// current iterate and stop); the loop also stops once a step is below 1e-4,
// an order under the kernel-coefficient tolerance: with an FP32 model the
// residual carries FP32 rounding noise, and steps of 1e-5 and below are that
// noise (measured: FP32 and TF32 settle at 1e-5..1e-6 relative).
__global__ void __launch_bounds__(256) refine_update_kernel(double* a, const double* delta, int Nc, double* flag) {
    __shared__ double red[2][8];
    __shared__ double mx[2];
    if (flag[0] != 0.0 || flag[1] != 0.0) return;
    double ms = 0.0, ma = 0.0;
    for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
        ms = fmax(ms, fabs(delta[j]));
        ma = fmax(ma, fabs(a[j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ms = fmax(ms, __shfl_xor_sync(0xffffffffu, ms, o));
        ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ms; red[1][threadIdx.x >> 5] = ma; }
    __syncthreads();
    if (threadIdx.x == 0) {
        ms = 0.0; ma = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { ms = fmax(ms, red[0][w]); ma = fmax(ma, red[1][w]); }
        const double step = ma > 0.0 ? ms / ma : ms;
        mx[0] = step;
        mx[1] = (flag[3] > 0.0 && !(step <= flag[2])) ? 1.0 : 0.0;   // diverging (or NaN)
    }
    __syncthreads();
    if (mx[1] != 0.0) {
        if (threadIdx.x == 0) flag[1] = 1.0;
        return;
    }
    for (int j = threadIdx.x; j < Nc; j += blockDim.x) a[j] += delta[j];
    if (threadIdx.x == 0) {
        flag[2] = mx[0];
        flag[3] += 1.0;
        flag[4] = mx[0];
        if (mx[0] < 1e-4) flag[1] = 1.0;
    }
}

// chi^2 of the refined solution c + delta from the first residual pass, without a
// second pass over the design rows: with r = C^T W (I - C c),
//   chi^2(c + delta) = chi^2(c) - 2 delta.r + delta^T M delta
// (M the Gram the solves used; delta is small, so its rounding enters only at
// second order).  chi_n[0..1] = (chi^2, n) of c; out[0..1] the same for c + delta
// (unchanged when no step was applied).  One CTA of 32 warps, a warp per row of M,
// FP64 sums in a fixed order.
__global__ void __launch_bounds__(1024) chi2_update_kernel(const double* M, int ld, int Nc, const double* r,
                                                           const double* delta, const double* chi_n,
                                                           const double* flag, double* out) {
    __shared__ double red[32];
    if (flag[0] != 0.0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool applied = flag[3] > 0.0;
    double acc = 0.0;   // lane 0 of each warp: its rows' delta_i (M delta - 2 r)_i
    if (applied) {
        for (int i = warp; i < Nc; i += 32) {   // one warp per row, lanes along the row
            const double* Mi = M + (long)i * ld;
            double q = 0.0;
            for (int j = lane; j < Nc; j += 32) q = fma(Mi[j], delta[j], q);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
            acc += delta[i] * (q - 2.0 * r[i]);
        }
    }
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 32; w++) t += red[w];
        out[0] = chi_n[0] + t;
        out[1] = chi_n[1];
    }
}

// Map the solution c of the orthonormalised basis back to Alard-Lupton
// coefficients (a_{n,k} = sum_m S[n][m] c_{m,k}, FP64) and write the stats.
__global__ void finalize_kernel(BasisDev b, const double* c, const double* S, const double* flag,
                                const double* chi_a0, const double* chi_a, int n_stamps_max, const int* n_stamps,
                                const int* centers, int stamp, int w, int h, int prec, double* coeffs,
                                argus_fit_stats* st) {
    const bool bad = flag[0] != 0.0;
    const int nb = b.nb, Ks = b.Ks, Nc = b.Nc;
    if (threadIdx.x == 0) {
        argus_fit_stats s;
        s.chi2 = bad ? 0.0 : chi_a[0];
        s.chi2_a0 = bad ? 0.0 : chi_a0[0];
        s.max_step = bad ? 0.0 : flag[4];
        s.n_pix = bad ? 0 : (long long)chi_a[1];
        s.dof = s.n_pix - Nc;
        s.n_coeffs = Nc;
        s.status = bad ? ARGUS_ERR_SINGULAR : ARGUS_OK;
        int used = 0;
        const int hs = stamp / 2, r = b.r, ns = min(*n_stamps, n_stamps_max);
        for (int i = 0; i < ns; i++) {
            const int xs = centers[2 * i], ys = centers[2 * i + 1];
            used += (xs - hs - r >= 0 && xs + hs + r <= w - 1 && ys - hs - r >= 0 && ys + hs + r <= h - 1);
        }
        s.n_stamps_used = used;
        s.precision = prec;
        s.refine_iters = bad ? 0 : (int)flag[3];
        s.pad_ = 0;
        *st = s;
    }
    if (bad) return;
    for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
        double v;
        if (j == 0 || j >= 1 + (nb - 1) * Ks) {
            v = c[j];
        } else {
            const int n = 1 + (j - 1) / Ks, k = (j - 1) % Ks;
            v = 0.0;
            for (int m = n; m < nb; m++) v += S[n * nb + m] * c[1 + (m - 1) * Ks + k];
        }
        coeffs[j] = v;
    }
}

// a7: K_k(u,v) = sum_n a_{n,k} B_n(u,v) (K_0 also a_0 B_0); bg_k.
__global__ void expand_kernel(BasisDev b, const double* img, const double* a, float* K, double* bg) {
    const int k = blockIdx.x, kk = b.ks * b.ks;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
        double s = (k == 0) ? a[0] * img[e] : 0.0;
        for (int n = 1; n < b.nb; n++) s += a[1 + (n - 1) * b.Ks + k] * img[(long)n * kk + e];
        K[(long)k * kk + e] = (float)s;
    }
    if (k == 0)
        for (int t = threadIdx.x; t < b.Kb; t += blockDim.x) bg[t] = a[1 + (b.nb - 1) * b.Ks + t];
}

// ---------------------------------------------------------------------------
// a3: stamp selection.  One thread per pixel: cheap tests first, isolation and
// window-flag scans with early exit, then a 64-bit atomicMax per cell of
// (order-preserving bits of R, inverted row-major rank).
__device__ __forceinline__ bool is_lmax(const float* R, long pitch, int w, int h, int x, int y) {
    if (x < 1 || y < 1 || x > w - 2 || y > h - 2) return false;
    const float c = R[(long)y * pitch + x];
    if (!isfinite(c)) return false;
#pragma unroll
    for (int dy = -1; dy <= 1; dy++)
#pragma unroll
        for (int dx = -1; dx <= 1; dx++) {
            if (!dx && !dy) continue;
            if (!(c > R[(long)(y + dy) * pitch + x + dx])) return false;
        }
    return true;
}

__global__ void select_kernel(const float* R, const uint8_t* flags, long pitch, int w, int h, int gx, int gy,
                              int m, float max_peak, int iso, float iso_frac, unsigned long long* cell_key) {
    const long np = (long)w * h;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < np; e += (long)gridDim.x * blockDim.x) {
        const int y = (int)(e / w), x = (int)(e - (long)y * w);
        if (x - m < 0 || x + m > w - 1 || y - m < 0 || y + m > h - 1) continue;
        if (!is_lmax(R, pitch, w, h, x, y)) continue;
        const float c = R[(long)y * pitch + x];
        if (!(c < max_peak)) continue;
        const float thr = iso_frac * c;
        bool bad = false;
        for (int yy = y - iso; yy <= y + iso && !bad; yy++)
            for (int xx = x - iso; xx <= x + iso; xx++) {
                if ((xx == x && yy == y) || xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                if (R[(long)yy * pitch + xx] > thr && is_lmax(R, pitch, w, h, xx, yy)) { bad = true; break; }
            }
        if (bad) continue;
        for (int yy = y - m; yy <= y + m && !bad; yy++)
            for (int xx = x - m; xx <= x + m; xx++)
                if (flags[(long)yy * pitch + xx]) { bad = true; break; }
        if (bad) continue;
        const int cx = (int)(((long)(x + 1) * gx - 1) / w), cy = (int)(((long)(y + 1) * gy - 1) / h);
        const unsigned bits = __float_as_uint(c);
        const unsigned ord = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
        const unsigned rank = (unsigned)y * (unsigned)w + (unsigned)x;
        const unsigned long long key = ((unsigned long long)ord << 32) | (unsigned long long)(0xffffffffu - rank);
        atomicMax(cell_key + cy * gx + cx, key);
    }
}

// Faster form of the same rule for the context path: a byte map of strict
// local maxima first, then per candidate the isolation window is scanned in
// Chebyshev rings of growing radius (noise peaks meet a brighter neighbour
// within a ring or two), reading R only where the map is set.
__global__ void select_lmax_kernel(const float* R, long pitch, int w, int h, uint8_t* lmax) {
    const long np = (long)w * h;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < np; e += (long)gridDim.x * blockDim.x) {
        const int y = (int)(e / w), x = (int)(e - (long)y * w);
        lmax[e] = is_lmax(R, pitch, w, h, x, y) ? 1 : 0;
    }
}

__global__ void select_ring_kernel(const float* R, const uint8_t* flags, const uint8_t* lmax, long pitch, int w, int h,
                                   int gx, int gy, int m, float max_peak, int iso, float iso_frac,
                                   unsigned long long* cell_key) {
    const long np = (long)w * h;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < np; e += (long)gridDim.x * blockDim.x) {
        if (!lmax[e]) continue;
        const int y = (int)(e / w), x = (int)(e - (long)y * w);
        if (x - m < 0 || x + m > w - 1 || y - m < 0 || y + m > h - 1) continue;
        const float c = R[(long)y * pitch + x];
        if (!(c < max_peak)) continue;
        const float thr = iso_frac * c;
        bool bad = false;
        for (int rad = 1; rad <= iso && !bad; rad++) {
            for (int t = 0; t < 8 * rad && !bad; t++) {
                // walk the ring of Chebyshev radius rad
                int dx, dy;
                const int side = 2 * rad;
                if (t < side) { dx = -rad + t; dy = -rad; }
                else if (t < 2 * side) { dx = rad; dy = -rad + (t - side); }
                else if (t < 3 * side) { dx = rad - (t - 2 * side); dy = rad; }
                else { dx = -rad; dy = rad - (t - 3 * side); }
                const int xx = x + dx, yy = y + dy;
                if (xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                if (lmax[(long)yy * w + xx] && R[(long)yy * pitch + xx] > thr) bad = true;
            }
        }
        if (bad) continue;
        for (int yy = y - m; yy <= y + m && !bad; yy++)
            for (int xx = x - m; xx <= x + m; xx++)
                if (flags[(long)yy * pitch + xx]) { bad = true; break; }
        if (bad) continue;
        const int cx = (int)(((long)(x + 1) * gx - 1) / w), cy = (int)(((long)(y + 1) * gy - 1) / h);
        const unsigned bits = __float_as_uint(c);
        const unsigned ord = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
        const unsigned rank = (unsigned)y * (unsigned)w + (unsigned)x;
        const unsigned long long key = ((unsigned long long)ord << 32) | (unsigned long long)(0xffffffffu - rank);
        atomicMax(cell_key + cy * gx + cx, key);
    }
}

// Tiled form for the context path (isolation radius <= 32), same decisions as
// the per-pixel rule above.  One CTA per 128 x 64 tile:
//  1. R over the tile plus a halo of iso + 1 is copied to shared memory with
//     16-byte cp.async (rows start on a 4-float boundary; outside the frame 0).
//  2. Strict local maxima over the tile plus a QR-pixel halo (QR = min(3, iso))
//     become a masked copy mv (R there, -inf elsewhere), four rows per thread
//     from separable 3-wide maxima; NaN neighbours propagate through max.NaN,
//     so a pixel next to a NaN is never a maximum.  Candidates (maxima of the
//     tile with their stamp window in the frame, below max_peak) are listed in
//     the same pass; a tile holds at most one strict maximum per 2 x 2 block.
//  3. Each candidate is tested against the other maxima within QR (the
//     (2 QR + 1)^2 - 1 taps of mv): in a star field most fail here.
//  4. One warp per remaining candidate scans the rest of the isolation window
//     in R, testing the local-maximum rule only where R exceeds iso_frac * c,
//     then the flag window (32-bit loads), then the cell atomicMax.
constexpr int SEL_TX = 128, SEL_TY = 64, SEL_QR = 3, SEL_MAX_ISO = 32, SEL_THREADS = 512;
constexpr int SEL_LIST = SEL_TX * SEL_TY / 4;

struct SelGeom {
    int qr, ox, rw, rh, mw, mh;
};

__host__ __device__ inline SelGeom sel_geom(int iso) {
    SelGeom g;
    g.qr = iso < SEL_QR ? iso : SEL_QR;
    g.ox = (4 - ((iso + 1) & 3)) & 3;                     // r column 0 is frame x0 - iso - 1 - ox
    g.rw = (SEL_TX + 2 * iso + 2 + g.ox + 3) & ~3;
    g.rh = SEL_TY + 2 * iso + 2;
    // mv rows are padded so that 4-column groups aligned with r start on 16-byte boundaries
    // (mv element (jy, jx) at jy * mw + jx + moff, moff = (4 - qr % 4) % 4)
    g.mw = (SEL_TX + 2 * g.qr + (4 - g.qr % 4) % 4 + 3) & ~3;
    g.mh = SEL_TY + 2 * g.qr;
    return g;
}

// r is followed by SEL_RPAD spare rows: the last strip of step 2 reads past the
// staged rows (into values it discards) without a bounds test.
constexpr int SEL_RPAD = 4;

__host__ __device__ inline size_t select_tile_smem(int iso) {
    const SelGeom g = sel_geom(iso);
    return sizeof(float) * ((size_t)g.rw * (g.rh + SEL_RPAD) + (size_t)g.mw * g.mh) +
           2 * SEL_LIST * sizeof(unsigned short);
}

// Taps of the Chebyshev rings of radius 1 .. SEL_MAX_ISO around a pixel, ring by
// ring: ring rho holds entries (2 rho - 1)^2 - 1 .. (2 rho + 1)^2 - 2 as (dx, dy).
struct SelRing {
    alignas(16) signed char d[2 * ((2 * SEL_MAX_ISO + 1) * (2 * SEL_MAX_ISO + 1) - 1)];
};
constexpr SelRing make_sel_ring() {
    SelRing t{};
    int k = 0;
    for (int rho = 1; rho <= SEL_MAX_ISO; rho++)
        for (int s = 0; s < 8 * rho; s++) {
            const int side = 2 * rho;
            int dx = -rho, dy = rho - (s - 3 * side);
            if (s < side) { dx = -rho + s; dy = -rho; }
            else if (s < 2 * side) { dx = rho; dy = -rho + (s - side); }
            else if (s < 3 * side) { dx = rho - (s - 2 * side); dy = rho; }
            t.d[2 * k] = (signed char)dx;
            t.d[2 * k + 1] = (signed char)dy;
            k++;
        }
    return t;
}
__device__ const SelRing g_sel_ring = make_sel_ring();

__device__ __forceinline__ float fmax_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

template <int QR>
__global__ void __launch_bounds__(SEL_THREADS, 2) select_tile_kernel(const float* R, const uint8_t* flags, long pitch,
                                                                    int w, int h, int gx, int gy, int m,
                                                                    float max_peak, int iso, float iso_frac,
                                                                    unsigned long long* cell_key) {
    constexpr int MW = SEL_TX + 2 * QR, MH = SEL_TY + 2 * QR;
    constexpr int MOFF = (4 - QR % 4) % 4;                       // r column of mv column 0 is cx = -QR mod 4
    constexpr int MWP = (MW + MOFF + 3) & ~3;                    // padded mv row
    extern __shared__ float4 sel_smem[];
    const SelGeom g = sel_geom(iso);
    float* r = reinterpret_cast<float*>(sel_smem);              // [rh][rw]
    float* mvr = r + g.rw * (g.rh + SEL_RPAD);                   // [MH][MWP]
    float* mv = mvr + MOFF;                                      // mv[jy * MWP + jx]
    unsigned short* cand = reinterpret_cast<unsigned short*>(mvr + MWP * MH);
    unsigned short* surv = cand + SEL_LIST;
    __shared__ int n_cand, n_surv, n_fin;
    const int ntx = (w + SEL_TX - 1) / SEL_TX;
    const int x0 = (int)(blockIdx.x % ntx) * SEL_TX, y0 = (int)(blockIdx.x / ntx) * SEL_TY;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = SEL_THREADS / 32;
    const int XS = x0 - iso - 1 - g.ox, YS = y0 - iso - 1;      // frame position of r[0][0]
    if (tid == 0) { n_cand = 0; n_surv = 0; n_fin = 0; }
    // 1. stage R in 16-byte chunks; XS is a multiple of 4, so a chunk is inside or
    //    outside the frame but for the one that holds column w (partly zero-filled)
    {
        const int cpr = g.rw >> 2, n = cpr * g.rh;
        const int sy = SEL_THREADS / cpr, sc = SEL_THREADS - sy * cpr;
        int jy = tid / cpr, jc = tid - jy * cpr;
        for (int e = tid; e < n; e += SEL_THREADS) {
            const int Y = YS + jy, X = XS + 4 * jc;
            int nb = 0;
            if (Y >= 0 && Y < h && X >= 0 && X < w) nb = 4 * min(4, w - X);
            tc::cp_async16(r + jy * g.rw + 4 * jc, nb ? R + (long)Y * pitch + X : R, nb);
            jc += sc;
            jy += sy;
            if (jc >= cpr) { jc -= cpr; jy++; }
        }
        tc::cp_async_commit();
        tc::cp_async_wait<0>();
    }
    __syncthreads();
    // 2. masked strict local maxima over the tile + QR, four rows x four columns per item
    //    (each row of the item is one aligned 16-byte load of r and its two neighbours),
    //    and the candidate list
    const float NEG = __int_as_float(0xff800000), INF = __int_as_float(0x7f800000);
    {
        const int cx = iso + 1 + g.ox - QR, cy = iso + 1 - QR;     // r position of mv[0][0]; cx % 4 == MOFF
        constexpr int NSTRIP = (MH + 3) / 4, NCG = MWP / 4, N = NCG * NSTRIP;
        for (int e = tid; e < N; e += SEL_THREADS) {
            const int js = e / NCG, jg = e - js * NCG;
            const int jy0 = 4 * js, jx0 = 4 * jg - MOFF;          // columns jx0 .. jx0 + 3 (cx + jx0: 16-byte aligned)
            const float* q = r + (cy + jy0 - 1) * g.rw + (cx + jx0);
            // v[t][k]: r at row jy0 - 1 + t, column jx0 - 1 + k
            float v[6][6], h3[6][4];
#pragma unroll
            for (int t = 0; t < 6; t++) {
                const float* qt = q + t * g.rw;
                const float4 c4 = *reinterpret_cast<const float4*>(qt);
                v[t][0] = cx + jx0 > 0 ? qt[-1] : NEG;   // r column -1 only feeds a column jx < 0 (discarded)
                v[t][1] = c4.x; v[t][2] = c4.y; v[t][3] = c4.z; v[t][4] = c4.w;
                v[t][5] = qt[4];
#pragma unroll
                for (int c = 0; c < 4; c++) h3[t][c] = fmax_nan(fmax_nan(v[t][c], v[t][c + 1]), v[t][c + 2]);
            }
            int nc = 0, ev0 = 0, ev1 = 0, ev2 = 0, ev3 = 0;
#pragma unroll
            for (int t = 1; t <= 4; t++) {
                const int jy = jy0 + t - 1, y = jy - QR;
                const int Y = y0 + y;
                float o[4];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int jx = jx0 + c, x = jx - QR, X = x0 - QR + jx;
                    const bool xin = X >= 1 && X <= w - 2;
                    const bool xc = x >= 0 && x < SEL_TX && X - m >= 0 && X + m <= w - 1;
                    const float cv = v[t][c + 1];
                    const float nb = fmax_nan(fmax_nan(h3[t - 1][c], h3[t + 1][c]), fmax_nan(v[t][c], v[t][c + 2]));
                    const bool l = jy < MH && jx >= 0 && jx < MW && xin && Y >= 1 && Y <= h - 2 && cv > nb && cv < INF;
                    o[c] = l ? cv : NEG;
                    // at most one strict maximum per 2 x 2 block: at most four per item
                    if (l && xc && y >= 0 && y < SEL_TY && Y - m >= 0 && Y + m <= h - 1 && cv < max_peak) {
                        const int ev = y * SEL_TX + x;
                        ev3 = nc == 3 ? ev : ev3;
                        ev2 = nc == 2 ? ev : ev2;
                        ev1 = nc == 1 ? ev : ev1;
                        ev0 = nc == 0 ? ev : ev0;
                        nc++;
                    }
                }
                if (jy < MH) *reinterpret_cast<float4*>(mv + jy * MWP + jx0) = make_float4(o[0], o[1], o[2], o[3]);
            }
            if (nc) {
                const int base = atomicAdd(&n_cand, nc);
                cand[base] = (unsigned short)ev0;
                if (nc > 1) cand[base + 1] = (unsigned short)ev1;
                if (nc > 2) cand[base + 2] = (unsigned short)ev2;
                if (nc > 3) cand[base + 3] = (unsigned short)ev3;
            }
        }
    }
    __syncthreads();
    // 3. the other maxima within QR: radius 1 holds none (the neighbours of a strict
    //    maximum are below it, so none of them is one); radius 2 for every candidate,
    //    radius 3 only for the survivors of radius 2 (most noise peaks meet another
    //    maximum at radius 2), listed in between so that warps stay full
    for (int i = tid; i < n_cand; i += SEL_THREADS) {
        const int e = cand[i];
        const int y = e / SEL_TX, x = e - y * SEL_TX;
        const float* q = mv + y * MWP + x;                         // window corner (y - QR, x - QR)
        const float c = q[QR * MWP + QR];
        float other = NEG;
        if (QR >= 2) {
#pragma unroll
            for (int dy = QR - 2; dy <= QR + 2; dy++)
#pragma unroll
                for (int dx = QR - 2; dx <= QR + 2; dx++)
                    if (dy == QR - 2 || dy == QR + 2 || dx == QR - 2 || dx == QR + 2) other = fmaxf(other, q[dy * MWP + dx]);
        }
        if (!(other > iso_frac * c)) surv[atomicAdd(&n_surv, 1)] = (unsigned short)e;
    }
    __syncthreads();
    for (int i = tid; i < n_surv; i += SEL_THREADS) {
        const int e = surv[i];
        const int y = e / SEL_TX, x = e - y * SEL_TX;
        const float* q = mv + y * MWP + x;
        const float c = q[QR * MWP + QR];
        float other = NEG;
        if (QR >= 3) {
#pragma unroll
            for (int dy = 0; dy <= 2 * QR; dy++)
#pragma unroll
                for (int dx = 0; dx <= 2 * QR; dx++)
                    if (dy == 0 || dy == 2 * QR || dx == 0 || dx == 2 * QR) other = fmaxf(other, q[dy * MWP + dx]);
        }
        if (!(other > iso_frac * c)) cand[atomicAdd(&n_fin, 1)] = (unsigned short)e;
    }
    __syncthreads();
    // 4. one warp per survivor: rest of the isolation window, flag window, cell key
    const int side = 2 * iso + 1, fside = 2 * m + 1;
    for (int i = wid; i < n_fin; i += nw) {
        const int e = cand[i];
        const int y = e / SEL_TX, x = e - y * SEL_TX;
        const int X = x0 + x, Y = y0 + y;
        const float c = mv[(y + QR) * MWP + x + QR];
        const float thr = iso_frac * c;
        bool bad = false;
        if (iso > QR) {
            // rings QR + 1 .. iso, 32 taps per step, nearest first: a noise peak meets
            // a brighter maximum within a step or two
            const float* qc = r + (y + iso + 1) * g.rw + (x + iso + 1 + g.ox);   // the candidate
            const char2* ring = reinterpret_cast<const char2*>(g_sel_ring.d);
            const int p1 = side * side - 1;
            for (int pb = (2 * QR + 1) * (2 * QR + 1) - 1; pb < p1; pb += 32) {
                const int p = pb + lane;
                bool b = false;
                if (p < p1) {
                    const char2 d = __ldg(ring + p);
                    const float* q = qc + d.y * g.rw + d.x;
                    const float v = *q;
                    const int XX = X + d.x, YY = Y + d.y;
                    if (v > thr && v < INF && XX >= 1 && XX <= w - 2 && YY >= 1 && YY <= h - 2) {
                        const float nb = fmax_nan(fmax_nan(fmax_nan(q[-g.rw - 1], q[-g.rw]), fmax_nan(q[-g.rw + 1], q[-1])),
                                                  fmax_nan(fmax_nan(q[1], q[g.rw - 1]), fmax_nan(q[g.rw], q[g.rw + 1])));
                        b = v > nb;
                    }
                }
                if (__any_sync(0xffffffffu, b)) { bad = true; break; }
            }
        }
        if (bad) continue;
        // flag window rows Y - m .. Y + m, bytes X - m .. X + m, as aligned 32-bit words
        // (rows are 16-byte aligned and the words end inside the row's pitch)
        const int wa = (X - m) & ~3, nwr = (((X + m) & ~3) - wa) / 4 + 1;
        const int sr = 32 / nwr, sc = 32 - sr * nwr;
        int ry = lane / nwr, rc = lane - ry * nwr;
        unsigned f = 0;
#pragma unroll 4
        for (int t = lane; t < nwr * fside; t += 32) {
            const int xa = wa + 4 * rc;
            unsigned v = __ldg(reinterpret_cast<const unsigned*>(flags + (long)(Y - m + ry) * pitch + xa));
            const int lo = X - m - xa, hi = X + m - xa;                      // byte range inside this word
            if (lo > 0) v &= 0xffffffffu << (8 * lo);
            if (hi < 3) v &= 0xffffffffu >> (8 * (3 - hi));
            f |= v;
            rc += sc;
            ry += sr;
            if (rc >= nwr) { rc -= nwr; ry++; }
        }
        if (__any_sync(0xffffffffu, f != 0) || lane != 0) continue;
        const int cx = (int)(((long)(X + 1) * gx - 1) / w), cy = (int)(((long)(Y + 1) * gy - 1) / h);
        const unsigned bits = __float_as_uint(c);
        const unsigned ord = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
        const unsigned rank = (unsigned)Y * (unsigned)w + (unsigned)X;
        const unsigned long long key = ((unsigned long long)ord << 32) | (unsigned long long)(0xffffffffu - rank);
        atomicMax(cell_key + cy * gx + cx, key);
    }
}

template <int QR>
int launch_select_tile(const float* ref, const uint8_t* flags, const argus_shape& shape, int grid_x, int grid_y,
                       int m, float max_peak, int iso, float iso_frac, unsigned long long* keys, cudaStream_t st) {
    const size_t smem = select_tile_smem(iso);
    if (cudaFuncSetAttribute(select_tile_kernel<QR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return ARGUS_ERR_CUDA;
    const long tiles = (long)((shape.w + SEL_TX - 1) / SEL_TX) * ((shape.h + SEL_TY - 1) / SEL_TY);
    select_tile_kernel<QR><<<(unsigned)tiles, SEL_THREADS, smem, st>>>(ref, flags, shape.pitch, shape.w, shape.h,
                                                                       grid_x, grid_y, m, max_peak, iso, iso_frac,
                                                                       keys);
    argus_count_launch(1);
    return ARGUS_OK;
}

__global__ void __launch_bounds__(1024) select_compact_kernel(const unsigned long long* cell_key, int ncell, int w,
                                                              int* centers, int* n_out) {
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b0 = 0; b0 < ncell; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const unsigned long long k = i < ncell ? cell_key[i] : 0ull;
        const int v = k != 0ull;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int ws = wsum[lane];
            int wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - ws;
        }
        __syncthreads();
        const int pos = carry + wsum[wid] + incl - v;
        if (v) {
            const unsigned rank = 0xffffffffu - (unsigned)(k & 0xffffffffu);
            centers[2 * pos] = (int)(rank % (unsigned)w);
            centers[2 * pos + 1] = (int)(rank / (unsigned)w);
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = pos + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = carry;
}

}  // namespace

int argus_nterms(int deg) { return nterms(deg); }

int argus_basis_count(const argus_basis* b) {
    BasisDev d;
    if (make_basis_dev(b, &d)) return -1;
    return d.nb;
}

static bool same_basis(const argus_basis& a, const argus_basis& b) {
    return memcmp(&a, &b, sizeof(argus_basis)) == 0;
}

int argus_basis_prepare(argus_ctx* ctx, const argus_basis* b, cudaStream_t st) {
    BasisDev d;
    int rc = make_basis_dev(b, &d);
    if (rc) return rc;
    argus_basis key;
    memset(&key, 0, sizeof(key));
    key.ksize = b->ksize; key.ngauss = b->ngauss;
    for (int g = 0; g < b->ngauss; g++) { key.sigma[g] = b->sigma[g]; key.degree[g] = b->degree[g]; }
    key.spatial_degree = b->spatial_degree; key.bg_degree = b->bg_degree;
    if (ctx->basis_memo_valid && same_basis(ctx->basis_memo, key)) return ARGUS_OK;
    basis_prepare_kernel<<<d.nb, 256, 0, st>>>(d, ctx->basis_img, ctx->basis_imgf, ctx->basis_h, ctx->basis_ab); argus_count_launch(1);
    basis_ortho_kernel<<<1, 1024, 0, st>>>(d, ctx->basis_img, ctx->basis_imgf, ctx->basis_S, ctx->L); argus_count_launch(1);
    rc = argus_launch_status();
    if (rc == ARGUS_OK) {
        ctx->basis_memo = key;
        ctx->basis_memo_valid = 1;
    }
    return rc;
}

// Factor M[0:n,0:n] (ld) into ctx->L (lower triangle; the off-diagonal blocks also mirrored
// into the upper triangle), keeping the inverses of its diagonal blocks in ctx->Dinv; flag = vec row 7.
int argus_cholesky_solve_prepare(argus_ctx* ctx, const double* M, int ld, int n, cudaStream_t st) {
    double* flag = ctx->vec + 7 * (size_t)ctx->np_cols;
    double* rdiag = ctx->vec + 6 * (size_t)ctx->np_cols;
    chol_init_kernel<<<ctx->num_sms, 256, 0, st>>>(M, ld, n, ctx->L, flag); argus_count_launch(1);
    for (int p = 0; p < n; p += CB) {
        const int pb = min(CB, n - p);
        double* Dp = ctx->Dinv + (size_t)(p / CB) * CB * CB;
        chol_diag_kernel<<<1, 128, 0, st>>>(ctx->L, ld, p, pb, rdiag, flag, ctx->d_status); argus_count_launch(1);
        const int rest = n - p - pb;
        chol_panel_kernel<<<(rest + pb + 7) / 8, 256, 0, st>>>(ctx->L, ld, n, p, pb, rdiag, Dp, flag); argus_count_launch(1);
        if (rest <= 0) break;
        const int T = (rest + 15) / 16;
        chol_update_kernel<<<T * (T + 1) / 2, 256, 0, st>>>(ctx->L, ld, n, p, pb, flag); argus_count_launch(1);
    }
    return argus_launch_status();
}

// x = (L L^T)^-1 rhs: one blocked forward and backward substitution.
void argus_tri_solve(argus_ctx* ctx, int ld, int n, const double* rhs, int rs, double* x, cudaStream_t st) {
    double* flag = ctx->vec + 7 * (size_t)ctx->np_cols;
    const size_t sm = sizeof(double) * 2 * (size_t)n;
    cudaFuncSetAttribute(tri_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    tri_solve_kernel<<<1, 1024, sm, st>>>(ctx->L, ld, n, ctx->Dinv, rhs, rs, x, flag); argus_count_launch(1);
}

// a4: X[(s nb + m) ss + pix] = (ref (x) img_m) at every pixel of every stamp s <
// *n_stamps (zero for stamps whose window leaves the frame).  21 x 21 stamps
// and kernels with at most 64 images run on the tensor cores
// (stamp_conv_tc.cu), 21 x 21 stamps with 11 x 11 kernels in the register-
// blocked CUDA-core kernel, everything else in the general one.
static int stamp_basis_conv(argus_ctx* ctx, const float* ref, const argus_shape& shape, const int* centers,
                     const int* n_stamps, int max_stamps, int stamp, const float* img, int nb, int ks, float* X,
                     cudaStream_t st) {
    if (stamp == SC_ST && ks == 21 && nb <= 64)
        return argus_stamp_conv_tc(ref, shape.pitch, shape.w, shape.h, centers, n_stamps, max_stamps, img, nb,
                                   ctx->stamp_b, X, ctx->num_sms, ctx->d_status, st);
    BasisDev d;
    memset(&d, 0, sizeof(d));
    d.ks = ks;
    d.r = (ks - 1) / 2;
    d.nb = nb;
    const int WW = stamp + 2 * d.r, kk = ks * ks;
    if (stamp == SC_ST && ks == 11 && nb <= 52) {
        // 13 warps x 4 functions cover up to 52 basis functions
        const size_t fsm = sizeof(float) * ((size_t)SC_NS * WW * WW + (size_t)nb * kk);
        const int nblk = (max_stamps + SC_NS - 1) / SC_NS;
        cudaFuncSetAttribute(stamp_conv_fast_kernel<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
        stamp_conv_fast_kernel<11><<<nblk, 416, fsm, st>>>(d, ref, shape.pitch, shape.w, shape.h, centers,
                                                           n_stamps, img, X); argus_count_launch(1);
        return argus_launch_status();
    }
    int group = (int)((200 * 1024 / sizeof(float) - (size_t)WW * WW) / kk);
    if (group > nb) group = nb;
    if (group < 4 && group < nb) return ARGUS_ERR_UNSUPPORTED;
    const size_t conv_smem = sizeof(float) * ((size_t)WW * WW + (size_t)group * kk);
    cudaFuncSetAttribute(stamp_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem);
    stamp_conv_kernel<<<max_stamps, 256, conv_smem, st>>>(d, ref, shape.pitch, shape.w, shape.h, centers, n_stamps,
                                                          stamp, img, group, X); argus_count_launch(1);
    return argus_launch_status();
}

extern "C" int argus_stamp_basis(argus_ctx* ctx, const float* ref, argus_shape shape, const int* centers,
                                 const int* n_stamps, int max_stamps, int stamp, const float* images, int nb,
                                 int ksize, float* X, argus_stream stream) {
    if (!ctx || !ref || !centers || !n_stamps || !images || !X) return ARGUS_ERR_ARG;
    if (max_stamps < 1 || max_stamps > ctx->max_stamps || stamp < 1 || stamp > ARGUS_MAX_STAMP || !(stamp & 1))
        return ARGUS_ERR_ARG;
    if (nb < 1 || nb > ARGUS_MAX_NB || ksize < 3 || ksize > ARGUS_MAX_KS || !(ksize & 1)) return ARGUS_ERR_ARG;
    int rc = argus_check_shape(shape, ctx->max_pixels);
    if (rc) return rc;
    if (argus_check_ptr16(X) || argus_check_ptr16(images)) return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    return stamp_basis_conv(ctx, ref, shape, centers, n_stamps, max_stamps, stamp, images, nb, ksize, X,
                            (cudaStream_t)stream);
}

// Steps of iterative refinement after the first solve: one, with the residual
// C^T W (I - C c) from the FP32 design and FP64 sums; its relative size is
// reported as max_step.
constexpr int REFINE_MAX = 1;
static_assert(REFINE_MAX == 1, "chi2_update_kernel takes r and delta of the first iterate");

extern "C" int argus_fit_kernel(argus_ctx* ctx, const float* sci, const float* sci_var, const float* ref,
                                const uint8_t* flags, argus_shape shape, const int* centers,
                                const int* n_stamps, int max_stamps, int stamp, const argus_basis* basis,
                                int precision, double* coeffs, argus_fit_stats* stats, argus_stream stream) {
    if (!ctx || !sci || !sci_var || !ref || !flags || !centers || !n_stamps || !coeffs || !stats || !basis)
        return ARGUS_ERR_ARG;
    if (max_stamps < 1 || max_stamps > ctx->max_stamps || stamp < 1 || stamp > ARGUS_MAX_STAMP || !(stamp & 1))
        return ARGUS_ERR_ARG;
    if (precision < ARGUS_PREC_FP32 || precision > ARGUS_PREC_BF16_SPLIT) return ARGUS_ERR_ARG;
    int rc = argus_check_shape(shape, ctx->max_pixels);
    if (rc) return rc;
    BasisDev d;
    rc = make_basis_dev(basis, &d);
    if (rc) return rc;
    if (d.Nc > ctx->max_coeffs) return ARGUS_ERR_ARG;
    if (d.Nc > 2 * RT) return ARGUS_ERR_UNSUPPORTED;   // the residual pass gives each thread two outputs
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    rc = argus_basis_prepare(ctx, basis, st);
    if (rc) return rc;

    const int ss = stamp * stamp;
    rc = stamp_basis_conv(ctx, ref, shape, centers, n_stamps, max_stamps, stamp, ctx->basis_imgf, d.nb, d.ks, ctx->X,
                          st);
    if (rc) return rc;

    GramArgs g;
    g.X = ctx->X; g.sci = sci; g.var = sci_var; g.flags = flags; g.centers = centers; g.n_stamps = n_stamps;
    g.pitch = shape.pitch; g.w = shape.w; g.h = shape.h; g.W = shape.w; g.H = shape.h;
    g.stamp = stamp; g.ss = ss; g.r = d.r; g.max_stamps = max_stamps; g.nb = d.nb; g.Ks = d.Ks; g.Kb = d.Kb;
    g.Nc = d.Nc;
    g.NP = argus_round_up(d.Nc + 1, 16);
    g.sdeg = d.sdeg; g.bgdeg = d.bgdeg; g.part = ctx->gram_part; g.status = ctx->d_status;

    const long max_rows = (long)max_stamps * ss;
    int part_slots;
    // per-row weights for every precision; the weighted design matrix is written as FP32
    // rows (FP32 Gram) or as operand tiles (tensor-core Gram)
    {
        long rwb = (max_rows + 255) / 256;
        if (rwb > (long)ctx->num_sms * 8) rwb = (long)ctx->num_sms * 8;
        row_weights_kernel<<<(unsigned)rwb, 256, 0, st>>>(g, ctx->rowmeta); argus_count_launch(1);
    }
    if (precision == ARGUS_PREC_FP32) {
        design_kernel<<<ctx->num_sms * 4, 256, sizeof(int) * 2 * g.NP, st>>>(g, ctx->rowmeta, ctx->design); argus_count_launch(1);
        const int ntile = (g.NP + GT - 1) / GT;
        const int npair = ntile * (ntile + 1) / 2;
        int nslots = ctx->num_sms * 3 / npair;   // three CTAs per SM
        if (nslots < 1) nslots = 1;
        if (nslots > ctx->gram_parts / 2) nslots = ctx->gram_parts / 2;
        const long nch = (max_rows + GK - 1) / GK;
        if (nslots > nch) nslots = (int)nch;
        g.nslots = nslots;
        part_slots = 2 * nslots;   // hi and lo halves of the double-float partials
        gram_cp_kernel<<<dim3(npair, nslots), 256, 0, st>>>(g, ctx->design, ntile); argus_count_launch(1);
    } else {
        // blocks of 128 rows x up to GRAM_CW columns that hold part of the upper triangle
        GramBlocks blocks;
        int nblk = 0;
        for (int rb = 0; rb * 128 < g.NP; rb++)
            for (int c0 = 0; c0 < g.NP; c0 += GRAM_CW) {
                const int n = g.NP - c0 < GRAM_CW ? g.NP - c0 : GRAM_CW;
                if (128 * rb > c0 + n - 1) continue;
                if (nblk == GRAM_MAX_BLOCKS) return ARGUS_ERR_UNSUPPORTED;
                blocks.b[nblk++] = GramBlock{rb, c0, n};
            }
        int nsplit = ctx->num_sms / nblk;
        if (nsplit < 1) nsplit = 1;
        if (nsplit > ctx->gram_parts / 2) nsplit = ctx->gram_parts / 2;
        const long nch = (max_rows + TC_KC - 1) / TC_KC;
        if (nsplit > nch) nsplit = (int)nch;
        g.nslots = nsplit;
        part_slots = 2 * nsplit;   // hi and lo halves of the double-float partials
        uint8_t* tiles = reinterpret_cast<uint8_t*>(ctx->design);
        const size_t dsm = sizeof(int) * 2 * g.NP;
        const int dgrid = ctx->num_sms * 4;
        auto launch = [&](auto kern, auto dkern, size_t shsz) -> int {
            size_t smem = shsz + 1024;
            if (smem > 227 * 1024) return ARGUS_ERR_UNSUPPORTED;
            dkern<<<dgrid, 256, dsm, st>>>(g, ctx->rowmeta, tiles); argus_count_launch(1);
            const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return argus_cuda_fail(e);
            kern<<<dim3(nsplit, nblk), GRAM_THREADS, smem, st>>>(g, tiles, blocks); argus_count_launch(1);
            return ARGUS_OK;
        };
        if (precision == ARGUS_PREC_TF32)
            rc = launch(gram_tc_kernel<2, 1>, design_tiles_kernel<2, 1>, sizeof(GramShared<2, 1>));
        else if (precision == ARGUS_PREC_BF16)
            rc = launch(gram_tc_kernel<1, 1>, design_tiles_kernel<1, 1>, sizeof(GramShared<1, 1>));
        else
            rc = launch(gram_tc_kernel<1, 4>, design_tiles_kernel<1, 4>, sizeof(GramShared<1, 4>));
        if (rc) return rc;
    }
    if ((rc = argus_launch_status())) return rc;
    const int NP = g.NP;
    gram_reduce_kernel<<<ctx->num_sms, 256, 0, st>>>(ctx->gram_part, part_slots, NP, ctx->M); argus_count_launch(1);

    const size_t ld = (size_t)ctx->np_cols;
    double* c = ctx->vec + 1 * ld;      // current solution (orthonormal basis)
    double* rv = ctx->vec + 2 * ld;     // residual C^T W (I - C c)
    double* dl = ctx->vec + 3 * ld;     // correction
    double* chi0 = ctx->vec + 5 * ld;   // chi2, n of the first iterate
    double* chiw = ctx->vec + 5 * ld + 2;
    double* chif = ctx->vec + 5 * ld + 4;
    double* flag = ctx->vec + 7 * ld;   // refinement state
    if (cudaMemsetAsync(flag, 0, 8 * sizeof(double), st) != cudaSuccess) return ARGUS_ERR_CUDA;
    const int n = d.Nc;
    rc = argus_cholesky_solve_prepare(ctx, ctx->M, NP, n, st);
    if (rc) return rc;
    // first solve: c = M^-1 b, b = column N_c of the augmented Gram
    argus_tri_solve(ctx, NP, n, ctx->M + n, NP, c, st);
    int nparts = ctx->num_sms * 2;
    if (nparts > ctx->resid_parts) nparts = ctx->resid_parts;
    // rows staged as Gs [RT][RG] and Xs [RT][xst] floats; the group sums reuse the
    // space as [RT / nb][nb][8] + [RT / nb][8] doubles (at most 2 * 256 * 8 doubles)
    size_t rsmem = sizeof(float) * (size_t)(RG + resid_xst(d.nb)) * RT;
    if (rsmem < sizeof(double) * RT * 16) rsmem = sizeof(double) * RT * 16;
    cudaFuncSetAttribute(resid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
    const int rr_blocks = (n + 2 + 7) / 8;
    for (int it = 0; it < REFINE_MAX; it++) {
        resid_kernel<<<nparts, RT, rsmem, st>>>(g, ctx->rowmeta, c, flag, 1, ctx->resid_part); argus_count_launch(1);
        resid_reduce_kernel<<<rr_blocks, 256, 0, st>>>(ctx->resid_part, nparts, NP, n, rv, it == 0 ? chi0 : chiw, flag, 1); argus_count_launch(1);
        argus_tri_solve(ctx, NP, n, rv, 1, dl, st);
        refine_update_kernel<<<1, 256, 0, st>>>(c, dl, n, flag); argus_count_launch(1);
    }
    // chi^2 of the refined solution from the first residual pass (rv = r of c, dl = delta)
    chi2_update_kernel<<<1, 1024, 0, st>>>(ctx->M, NP, n, rv, dl, chi0, flag, chif); argus_count_launch(1);
    finalize_kernel<<<1, 256, 0, st>>>(d, c, ctx->basis_S, flag, chi0, chif, max_stamps, n_stamps, centers, stamp,
                                       shape.w, shape.h, precision, coeffs, stats); argus_count_launch(1);
    return argus_launch_status();
}

extern "C" int argus_expand_kernel(argus_ctx* ctx, const argus_basis* basis, const double* coeffs, float* K,
                                   double* bg, argus_stream stream) {
    if (!ctx || !basis || !coeffs || !K || !bg) return ARGUS_ERR_ARG;
    BasisDev d;
    int rc = make_basis_dev(basis, &d);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = argus_basis_prepare(ctx, basis, st))) return rc;
    expand_kernel<<<d.Ks, 256, 0, st>>>(d, ctx->basis_img, coeffs, K, bg); argus_count_launch(1);
    return argus_launch_status();
}

extern "C" int argus_select_stamps(argus_ctx* ctx, const float* ref, const uint8_t* flags, argus_shape shape,
                                   int grid_x, int grid_y, int stamp, int khalf, float max_peak, int iso,
                                   float iso_frac, int* centers, int* n_stamps, argus_stream stream) {
    if (!ctx || !ref || !flags || !centers || !n_stamps) return ARGUS_ERR_ARG;
    if (grid_x < 1 || grid_y < 1 || grid_x * grid_y > ctx->max_cells || stamp < 1 || khalf < 0 || iso < 0 ||
        iso > 64)
        return ARGUS_ERR_ARG;
    int rc = argus_check_shape(shape, ctx->max_pixels);
    if (rc) return rc;
    if (argus_check_ptr16(ref) || argus_check_ptr16(flags)) return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int ncell = grid_x * grid_y;
    if (cudaMemsetAsync(ctx->cell_key, 0, sizeof(unsigned long long) * ncell, st) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    const long np = (long)shape.w * shape.h;
    long blocks = (np + 255) / 256;
    if (blocks > (long)ctx->num_sms * 16) blocks = (long)ctx->num_sms * 16;
    if (iso <= SEL_MAX_ISO) {
        const int m = stamp / 2 + khalf;
        rc = iso == 0   ? launch_select_tile<0>(ref, flags, shape, grid_x, grid_y, m, max_peak, iso, iso_frac, ctx->cell_key, st)
             : iso == 1 ? launch_select_tile<1>(ref, flags, shape, grid_x, grid_y, m, max_peak, iso, iso_frac, ctx->cell_key, st)
             : iso == 2 ? launch_select_tile<2>(ref, flags, shape, grid_x, grid_y, m, max_peak, iso, iso_frac, ctx->cell_key, st)
                        : launch_select_tile<3>(ref, flags, shape, grid_x, grid_y, m, max_peak, iso, iso_frac, ctx->cell_key, st);
        if (rc) return rc;
    } else {
        uint8_t* lmax = reinterpret_cast<uint8_t*>(ctx->label);   // the label scratch, one byte per pixel
        const long rblocks = (np + 255) / 256;                      // one pixel per thread: latency-bound scans
        select_lmax_kernel<<<(unsigned)blocks, 256, 0, st>>>(ref, shape.pitch, shape.w, shape.h, lmax); argus_count_launch(1);
        select_ring_kernel<<<(unsigned)rblocks, 256, 0, st>>>(ref, flags, lmax, shape.pitch, shape.w, shape.h,
                                                             grid_x, grid_y, stamp / 2 + khalf, max_peak, iso,
                                                             iso_frac, ctx->cell_key); argus_count_launch(1);
    }
    select_compact_kernel<<<1, 1024, 0, st>>>(ctx->cell_key, ncell, shape.w, centers, n_stamps); argus_count_launch(1);
    return argus_launch_status();
}

// ---------------------------------------------------------------------------
// Stamp selection without a context, for callers that cannot allocate device
// memory: code running where cudaMalloc is not allowed or not wanted (a host
// that pre-reserves all GPU memory up front, a real-time loop that must never
// enter the allocator, or a plugin handed only input and output pointers by
// its host application).  It runs the per-pixel selection kernel (the same
// rule as argus_select_stamps' tiled kernels) and the same compaction kernel;
// their scratch -- one 64-bit key per grid cell -- lives in the file-scope
// device array below instead of a context.
//
// The array is part of the library image: every GPU that loads the library
// holds these 32 KiB until the process exits.  Host code cannot use the
// symbol's name as a device address, so the address is looked up once per
// device with cudaGetSymbolAddress, under a lock, with that device current.
// That lookup happens on the first call on a device; make that first call
// before any stream capture.  The address is then kept until the process
// exits: after a device reset (cudaDeviceReset, or the primary context torn
// down) it is stale, so do not call this entry point after one.  All calls share the array and it keeps the last
// call's contents, so each call clears the keys it uses first; calls that
// overlap on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.
static __device__ __align__(256) unsigned long long g_select_scratch[ARGUS_NOALLOC_MAX_CELLS];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];
int g_noalloc_sms[64];
}  // namespace

extern "C" int argus_select_stamps_noalloc(const float* ref, const uint8_t* flags, argus_shape shape,
                                           int grid_x, int grid_y, int stamp, int khalf, float max_peak,
                                           int iso, float iso_frac, int* centers, int* n_stamps,
                                           argus_stream stream) {
    if (!ref || !flags || !centers || !n_stamps) return ARGUS_ERR_ARG;
    if (grid_x < 1 || grid_y < 1 || stamp < 1 || khalf < 0 || iso < 0 || iso > 64) return ARGUS_ERR_ARG;
    if ((long)grid_x * grid_y > ARGUS_NOALLOC_MAX_CELLS) return ARGUS_ERR_CAPACITY;
    if (shape.w <= 0 || shape.h <= 0 || shape.pitch < shape.w) return ARGUS_ERR_ARG;
    if (shape.pitch % 16) return ARGUS_ERR_ALIGN;
    if (argus_check_ptr16(ref) || argus_check_ptr16(flags)) return ARGUS_ERR_ALIGN;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ARGUS_ERR_CUDA;
    void* scratch = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess || !p) return ARGUS_ERR_CUDA;
            int n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ARGUS_ERR_CUDA;
            g_noalloc_sms[dev] = n;
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
        sms = g_noalloc_sms[dev];
    }
    unsigned long long* keys = static_cast<unsigned long long*>(scratch);
    cudaStream_t st = (cudaStream_t)stream;
    const int ncell = grid_x * grid_y;
    if (cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * ncell, st) != cudaSuccess) return ARGUS_ERR_CUDA;
    const long np = (long)shape.w * shape.h;
    long blocks = (np + 255) / 256;
    if (blocks > (long)sms * 16) blocks = (long)sms * 16;
    select_kernel<<<(unsigned)blocks, 256, 0, st>>>(ref, flags, shape.pitch, shape.w, shape.h, grid_x, grid_y,
                                                    stamp / 2 + khalf, max_peak, iso, iso_frac, keys); argus_count_launch(1);
    select_compact_kernel<<<1, 1024, 0, st>>>(keys, ncell, shape.w, centers, n_stamps); argus_count_launch(1);
    return argus_launch_status();
}
