// K8: thousands of uneven target segments through one CUDA-graph launch of
// persistent kernels (paper Sec. 5: subtraction parallelised at the segment
// level; Sec. 4.1.1 HEALPix segments).  Each segment has its own spatially
// constant PSF-matching kernel fitted over its whole interior.
//
// Segments live in an "atlas": one pitched image per quantity with segment s
// at rows [row0_s, row0_s + side_s) and columns [0, side_s).  The work is cut
// into fixed-size units, not segments, so that 64-px and 512-px segments
// balance:
//   1. fit: persistent CTAs take (segment, row band) items from an atomic
//      counter (largest segments first); per band, X_m = R (x) B'_m (the
//      orthonormalised basis) for every interior pixel, 64-pixel chunks of the
//      weighted design [X_m, 1, I] in shared memory, the Gram's upper triangle
//      summed per chunk in FP32 and folded into double-float, then added to the
//      segment's FP64 normal matrix with one atomicAdd per entry per item;
//   2. solve: one CTA per segment, FP64 Cholesky in shared memory, mapping to
//      Alard-Lupton coefficients, kernel expansion, chi2 from the Gram;
//   3. subtract: persistent CTAs take 32x32 tiles (the same tile body as the
//      full-frame kernel) with the segment's kernel;
//   4. detection on the atlas (edge pixels of every segment are invalid, so
//      components never cross segments).
// The plan records the sequence in a CUDA graph on first run and replays it.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "basis.cuh"
#include "segments_fit.cuh"
#include "subtract_tile.cuh"

struct argus_seg_plan {
    argus_ctx* ctx;
    int n;                 // segments
    int pitch, atlas_h, max_side;
    argus_basis basis;
    BasisDev bd;
    int NPC;               // Gram columns: nb + 2 (basis, background, target)
    argus_seg_config cfg;
    int4* d_seg;           // (row0, side, col0, -)
    int2* d_fit_items;     // (segment, band y0): CUDA-core fit
    int n_fit_items;
    int fit_tc;            // the fit runs on the tensor cores (kernel sides <= 15)
    int4* d_fit_tc_items;  // (segment, x0, y0, -): tensor-core fit, 128 columns x band rows
    int n_fit_tc_items;
    int* d_fit_tc_start;   // [fit_tc_ctas + 1] item range of each CTA, equal row pairs
    float* d_rscale;       // [n] per-segment scale of R for the FP16 operands
    int fit_tc_ctas;
    int2* d_sub_items;     // (segment, tile index)
    int n_sub_items;
    int* d_counters;       // [4]
    double* d_gram;        // [n][NPC][NPC]
    float* d_K;            // [n][ks*ks]
    double* d_bg;          // [n]
    cudaGraphExec_t exec;
    cudaGraph_t graph;
    cudaStream_t cap_stream;   // recording stream (capture is not allowed on the legacy stream)
    const void* key[12];   // pointers the graph was recorded with
    int key_cap;
    int graph_kernels;     // kernels recorded in the graph
};

namespace {

using argus_sub::SubArgs;

// Fit work unit: a band of FIT_ROWS interior rows of one segment, processed
// in chunks of FIT_ROWS x 32 pixels.  One warp per group of FG basis
// functions: each lane owns one pixel column of the chunk and accumulates
// FIT_ROWS x FG outputs while streaming a window of reference values and
// broadcast basis taps (stored [tap][function] so FG taps are one vector load).
constexpr int FIT_ROWS = 8;
constexpr int FIT_COLS = 32;
constexpr int FIT_CH = FIT_ROWS * FIT_COLS;   // design pixels per Gram chunk
constexpr int FG = 8;                         // functions per warp group
constexpr int GRAM_FOLD = 8;                  // pixels per FP32 partial sum of the Gram

struct SegFitArgs {
    const float* sci;
    const float* var;
    const float* ref;
    const uint8_t* flags;
    long pitch;
    const int4* seg;
    const int2* items;
    int n_items;
    int* counter;
    const float* bimg;     // orthonormal basis images [nb][kk] (B'_0 = B_0)
    int nb, ks, r, NPC, ngroups;
    double* gram;
    int* n_pix;            // per segment count of weighted pixels
};

template <int KS>
__global__ void __launch_bounds__(256) seg_fit_kernel(SegFitArgs a) {
    constexpr int R = (KS - 1) / 2, KK = KS * KS;
    constexpr int WR = FIT_ROWS + KS - 1;             // window rows per column
    extern __shared__ __align__(16) float sm[];
    const int nb = a.nb, NPC = a.NPC, ng = a.ngroups;
    const int ZS = NPC + 1;                           // Z row stride
    float* Bt = sm;                                   // [ng][KK][FG] transposed taps
    float* Z = Bt + ng * KK * FG;                     // [FIT_CH][ZS]
    float* Rw = Z + FIT_CH * ZS;                      // [WR][512 + 2R]
    constexpr int WST = 512 + 2 * R;
    __shared__ int s_item;
    __shared__ int s_npix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < ng * KK * FG; e += blockDim.x) {
        const int f = e % FG, t = (e / FG) % KK, gi = e / (FG * KK);
        const int m = gi * FG + f;
        Bt[e] = m < nb ? a.bimg[(long)m * KK + t] : 0.0f;
    }
    // Gram blocks: 4x4 entry blocks of the upper triangle of NPC x NPC
    const int nbk = (NPC + 3) / 4;
    const int nblk = nbk * (nbk + 1) / 2;
    int bi = 0, bj = 0;
    {
        int rem = tid;
        while (bi < nbk && rem >= nbk - bi) { rem -= nbk - bi; bi++; }
        bj = bi + rem;
    }
    const bool gram_thread = tid < nblk;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) break;
        const int2 it = a.items[item];
        const int4 sg = a.seg[it.x];
        const int side = sg.y;
        const long base = (long)sg.x * a.pitch + sg.z;
        const int ylo = max(it.y, R), yhi = min(it.y + FIT_ROWS, side - R);
        const int xw = side - 2 * R;
        if (yhi <= ylo || xw <= 0) continue;
        // reference window: rows ylo - R .. ylo + FIT_ROWS - 1 + R, all columns
        for (int e = tid; e < WR * side; e += blockDim.x) {
            const int j = e / side, i = e - j * side;
            const int yy = ylo - R + j;
            Rw[j * WST + i] = yy < side ? __ldg(a.ref + base + (long)yy * a.pitch + i) : 0.0f;
        }
        if (tid == 0) s_npix = 0;
        float hi[16], lo[16];
#pragma unroll
        for (int q = 0; q < 16; q++) hi[q] = lo[q] = 0.0f;
        for (int c0 = 0; c0 < xw; c0 += FIT_COLS) {
            __syncthreads();
            // convolution: warp = function group, lane = column
            if (warp < ng) {
                const int xi = min(c0 + lane, xw - 1);   // interior column (clamped; extra lanes discarded)
                float acc[FIT_ROWS][FG];
#pragma unroll
                for (int j = 0; j < FIT_ROWS; j++)
#pragma unroll
                    for (int f = 0; f < FG; f++) acc[j][f] = 0.0f;
                const float* bt = Bt + warp * KK * FG;
#pragma unroll 1
                for (int iu = 0; iu < KS; iu++) {
                    // column x - du = (xi + R) - (iu - R) = xi + 2R - iu
                    float col[WR];
#pragma unroll
                    for (int m = 0; m < WR; m++) col[m] = Rw[m * WST + xi + 2 * R - iu];
#pragma unroll
                    for (int iv = 0; iv < KS; iv++) {
                        float kv[FG];
                        *reinterpret_cast<float4*>(kv) = *reinterpret_cast<const float4*>(bt + (iv * KS + iu) * FG);
                        *reinterpret_cast<float4*>(kv + 4) =
                            *reinterpret_cast<const float4*>(bt + (iv * KS + iu) * FG + 4);
#pragma unroll
                        for (int j = 0; j < FIT_ROWS; j++) {
                            // row y - dv = (ylo + j) - (iv - R) -> window row j + 2R - iv
                            const float rv = col[j + 2 * R - iv];
#pragma unroll
                            for (int f = 0; f < FG; f++) acc[j][f] = fmaf(kv[f], rv, acc[j][f]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < FIT_ROWS; j++)
#pragma unroll
                    for (int f = 0; f < FG; f++) {
                        const int m = warp * FG + f;
                        if (m < nb) Z[(j * FIT_COLS + lane) * ZS + m] = acc[j][f];
                    }
            }
            __syncthreads();
            // weights, background and target columns; pixels outside the band are zero
            {
                const int j = tid / FIT_COLS, l = tid % FIT_COLS;
                const int y = ylo + j, xi = c0 + l;
                float sqw = 0.0f, Iv = 0.0f;
                if (y < yhi && xi < xw) {
                    const long p = base + (long)y * a.pitch + (xi + R);
                    const float v = a.var[p], iv = a.sci[p];
                    if (a.flags[p] == 0 && v > 0.0f && isfinite(v) && isfinite(iv)) {
                        sqw = sqrtf(1.0f / v);
                        Iv = iv;
                        atomicAdd(&s_npix, 1);
                    }
                }
                float* zr = Z + tid * ZS;
                for (int m = 0; m < nb; m++) zr[m] *= sqw;
                zr[nb] = sqw;
                zr[nb + 1] = sqw * Iv;
                for (int m = nb + 2; m < ZS; m++) zr[m] = 0.0f;
            }
            __syncthreads();
            // Gram 4x4 block per thread: FP32 over GRAM_FOLD pixels at a time, each
            // partial folded into a double-float accumulator (error-free two-sum).
            // The FP32 partial sums are the only rounding left: with the
            // conditioning of single-segment normal matrices (~1e4 to 1e5 in the
            // orthonormal basis) sums over 256 pixels put ~1e-3 on the kernel,
            // sums over 8 pixels ~1e-4.
            if (gram_thread) {
                for (int p0 = 0; p0 < FIT_CH; p0 += GRAM_FOLD) {
                    float acc[16];
#pragma unroll
                    for (int q = 0; q < 16; q++) acc[q] = 0.0f;
#pragma unroll
                    for (int p = p0; p < p0 + GRAM_FOLD; p++) {
                        const float* zp = Z + p * ZS;
                        float zi[4], zj[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            zi[u] = (bi * 4 + u < NPC) ? zp[bi * 4 + u] : 0.0f;
                            zj[u] = (bj * 4 + u < NPC) ? zp[bj * 4 + u] : 0.0f;
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++)
#pragma unroll
                            for (int v = 0; v < 4; v++) acc[u * 4 + v] = fmaf(zi[u], zj[v], acc[u * 4 + v]);
                    }
#pragma unroll
                    for (int q = 0; q < 16; q++) {
                        const float sum = hi[q] + acc[q], bp = sum - hi[q];
                        lo[q] += (hi[q] - (sum - bp)) + (acc[q] - bp);
                        hi[q] = sum;
                    }
                }
            }
        }
        // one FP64 atomic per entry per item into the segment's normal matrix (upper triangle)
        if (gram_thread) {
            double* G = a.gram + (long)it.x * NPC * NPC;
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const int i = bi * 4 + u, j = bj * 4 + v;
                    if (i < NPC && j < NPC && i <= j) atomicAdd(G + i * NPC + j, (double)hi[u * 4 + v] + (double)lo[u * 4 + v]);
                }
        }
        __syncthreads();
        if (tid == 0 && s_npix) atomicAdd(a.n_pix + it.x, s_npix);
    }
}

template <int KS>
size_t seg_fit_smem(int nb, int NPC) {
    const int ng = (nb + FG - 1) / FG;
    return sizeof(float) * ((size_t)ng * KS * KS * FG + (size_t)FIT_CH * (NPC + 1) +
                            (size_t)(FIT_ROWS + KS - 1) * (512 + KS - 1));
}

template <int KS>
int launch_seg_fit(const SegFitArgs& a, int grid, cudaStream_t st) {
    const size_t smem = seg_fit_smem<KS>(a.nb, a.NPC);
    cudaFuncSetAttribute(seg_fit_kernel<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    seg_fit_kernel<KS><<<grid, 256, smem, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}

struct SegSolveArgs {
    const double* gram;
    const int* n_pix;
    int NPC, nb;
    const double* S;       // [nb][nb] orthonormalisation (B' = B S)
    const double* img;     // FP64 Alard-Lupton basis images [nb][kk]
    int kk;
    double* coeffs;        // [n][Nc] (Alard-Lupton order: a_0..a_48, bg)
    argus_seg_stats* stats;
    float* K;              // [n][kk]
    double* bg;            // [n]
    int* status;
};

// One CTA per segment: FP64 Cholesky of the 50 x 50 normal matrix (in shared
// memory), solution c in the orthonormal basis, a = S c, kernel, background,
// chi2 = t'Wt - 2 c'b + c'Mc from the augmented Gram.
__global__ void __launch_bounds__(128) seg_solve_kernel(SegSolveArgs a) {
    extern __shared__ double ds[];
    const int n = a.NPC - 1;          // unknowns: nb basis + background
    const int ld = a.NPC + 1;
    double* L = ds;                   // [NPC][ld]
    double* y = L + a.NPC * ld;       // [NPC]
    double* c = y + a.NPC;            // [NPC]
    __shared__ int bad;
    const int s = blockIdx.x, tid = threadIdx.x;
    const double* G = a.gram + (long)s * a.NPC * a.NPC;
    for (int e = tid; e < a.NPC * a.NPC; e += blockDim.x) {
        const int i = e / a.NPC, j = e - i * a.NPC;
        L[i * ld + j] = i <= j ? G[i * a.NPC + j] : G[j * a.NPC + i];   // full symmetric copy
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        if (tid == 0) {
            const double d = L[j * ld + j];
            if (!(d > 0.0)) bad = 1;
            L[j * ld + j] = sqrt(d > 0.0 ? d : 1.0);
        }
        __syncthreads();
        if (bad) break;
        for (int i = j + 1 + tid; i < n; i += blockDim.x) L[i * ld + j] /= L[j * ld + j];
        __syncthreads();
        for (int e = tid; e < (n - j - 1) * (n - j - 1); e += blockDim.x) {
            const int i = j + 1 + e / (n - j - 1), k = j + 1 + e % (n - j - 1);
            if (k <= i) L[i * ld + k] -= L[i * ld + j] * L[k * ld + j];
        }
        __syncthreads();
    }
    argus_seg_stats st;
    if (bad) {
        if (tid == 0) {
            argus_latch(a.status, ARGUS_ERR_SINGULAR);
            st.chi2 = 0.0; st.n_pix = a.n_pix[s]; st.status = ARGUS_ERR_SINGULAR;
            a.stats[s] = st;
        }
        for (int e = tid; e < a.kk; e += blockDim.x) a.K[(long)s * a.kk + e] = 0.0f;
        if (tid == 0) a.bg[s] = 0.0;
        return;
    }
    if (tid == 0) {
        // forward / back substitution with b = G[:, n] (the target column)
        for (int i = 0; i < n; i++) {
            double v = G[i * a.NPC + n];
            for (int k = 0; k < i; k++) v -= L[i * ld + k] * y[k];
            y[i] = v / L[i * ld + i];
        }
        for (int i = n - 1; i >= 0; i--) {
            double v = y[i];
            for (int k = i + 1; k < n; k++) v -= L[k * ld + i] * c[k];
            c[i] = v / L[i * ld + i];
        }
        // chi2 = t'Wt - 2 c'b + c'Mc
        double tt = G[n * a.NPC + n], cb = 0.0, cmc = 0.0;
        for (int i = 0; i < n; i++) {
            cb += c[i] * G[i * a.NPC + n];
            double mi = 0.0;
            for (int k = 0; k < n; k++) mi += (i <= k ? G[i * a.NPC + k] : G[k * a.NPC + i]) * c[k];
            cmc += c[i] * mi;
        }
        st.chi2 = tt - 2.0 * cb + cmc;
        st.n_pix = a.n_pix[s];
        st.status = ARGUS_OK;
        a.stats[s] = st;
    }
    __syncthreads();
    // a_0 = c_0; a_n = sum_{m >= n} S[n][m] c_m; background last
    double* co = a.coeffs + (long)s * (n);
    for (int j = tid; j < n; j += blockDim.x) {
        double v;
        if (j == 0 || j >= a.nb) {
            v = c[j];
        } else {
            v = 0.0;
            for (int m = j; m < a.nb; m++) v += a.S[j * a.nb + m] * c[m];
        }
        co[j] = v;
        y[j] = v;
    }
    __syncthreads();
    for (int e = tid; e < a.kk; e += blockDim.x) {
        double v = 0.0;
        for (int m = 0; m < a.nb; m++) v += y[m] * a.img[(long)m * a.kk + e];
        a.K[(long)s * a.kk + e] = (float)v;
    }
    if (tid == 0) a.bg[s] = c[a.nb];
}

struct SegSubArgs {
    const float* sci;
    const float* var;
    const float* ref;
    const float* ref_var;
    const uint8_t* flags;
    float* diff;
    float* diff_var;
    long pitch;
    const int4* seg;
    const int2* items;     // (segment, tile index)
    int n_items;
    int* counter;
    const float* K;
    const double* bg;
    int kk;
};

template <int KS>
__global__ void __launch_bounds__(argus_sub::THREADS) seg_sub_kernel(SegSubArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) break;
        const int2 it = a.items[item];
        const int4 sg = a.seg[it.x];
        const int side = sg.y, nt = (side + argus_sub::TILE - 1) / argus_sub::TILE;
        const int ty = it.y / nt, tx = it.y - ty * nt;
        SubArgs s;
        const long off = (long)sg.x * a.pitch + sg.z;
        s.sci = a.sci + off; s.sci_var = a.var + off; s.ref = a.ref + off; s.ref_var = a.ref_var + off;
        s.flags = a.flags + off; s.K = a.K + (long)it.x * a.kk; s.bg = a.bg + it.x;
        s.diff = a.diff + off; s.diff_var = a.diff_var + off;
        s.pitch = a.pitch; s.w = side; s.h = side; s.W = side; s.H = side; s.ox = 0; s.oy = 0;
        s.nbg = 1; s.bg_deg = 0; s.sdeg = 0;
        argus_sub::subtract_tile<KS, 1>(s, tx * argus_sub::TILE, ty * argus_sub::TILE, smem);
    }
}

template <int KS>
int launch_seg_sub(const SegSubArgs& a, int grid, cudaStream_t st) {
    const size_t smem = argus_sub::tile_smem_bytes<KS, 1>();
    cudaFuncSetAttribute(seg_sub_kernel<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    seg_sub_kernel<KS><<<grid, argus_sub::THREADS, smem, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}

}  // namespace

extern "C" int argus_segments_plan(argus_ctx* ctx, const argus_segment* table, int n, int pitch, int atlas_h,
                                   const argus_basis* basis, const argus_seg_config* cfg, argus_seg_plan** out) {
    if (!ctx || !table || n < 1 || !basis || !out || pitch < 16 || pitch % 16 || atlas_h < 1) return ARGUS_ERR_ARG;
    *out = NULL;
    BasisDev bd;
    int rc = make_basis_dev(basis, &bd);
    if (rc) return rc;
    if (bd.sdeg != 0 || bd.bgdeg != 0) return ARGUS_ERR_UNSUPPORTED;   // one constant kernel per segment
    if (bd.ks != 7 && bd.ks != 9 && bd.ks != 11 && bd.ks != 15 && bd.ks != 21) return ARGUS_ERR_UNSUPPORTED;
    if ((size_t)atlas_h * pitch > ctx->max_pixels) return ARGUS_ERR_ARG;
    argus_seg_config c = cfg ? *cfg : argus_seg_config{32, 1, 4, 0};
    if (c.fit_band < 8 || c.fit_band > 128 || c.fit_ctas_per_sm < 1 || c.fit_ctas_per_sm > 4 ||
        c.sub_ctas_per_sm < 1 || c.sub_ctas_per_sm > 16)
        return ARGUS_ERR_ARG;
    std::vector<int4> seg(n);
    int max_side = 0;
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) {
        const argus_segment& t = table[i];
        if (t.side < bd.ks || t.side > pitch || t.side > 512 || t.row0 < 0 || t.row0 + t.side > atlas_h)
            return ARGUS_ERR_ARG;
        if (t.col0 < 0 || t.col0 + t.side > pitch) return ARGUS_ERR_ARG;
        seg[i] = make_int4(t.row0, t.side, t.col0, 0);
        max_side = std::max(max_side, t.side);
        order[i] = i;
    }
    // segments must not overlap in the atlas (checked on a coarse occupancy grid of 16 x 16 cells)
    {
        const int cw = (pitch + 15) / 16, ch = (atlas_h + 15) / 16;
        std::vector<int> owner((size_t)cw * ch, -1);
        for (int i = 0; i < n; i++) {
            const argus_segment& t = table[i];
            if (t.row0 % 16 || t.col0 % 16) return ARGUS_ERR_ALIGN;
            for (int cy = t.row0 / 16; cy < (t.row0 + t.side + 15) / 16; cy++)
                for (int cx = t.col0 / 16; cx < (t.col0 + t.side + 15) / 16; cx++) {
                    int& o = owner[(size_t)cy * cw + cx];
                    if (o >= 0) return ARGUS_ERR_ARG;
                    o = i;
                }
        }
    }
    // work items, largest segments first
    std::sort(order.begin(), order.end(), [&](int a, int b) { return table[a].side > table[b].side; });
    std::vector<int2> fit_items, sub_items;
    std::vector<int4> fit_tc_items;
    const int NPC0 = bd.nb + 2;
    const bool fit_tc = argus_seg_fit_tc_smem(bd.ks, NPC0) != 0 && argus_seg_fit_tc_smem(bd.ks, NPC0) <= 227 * 1024 &&
                        bd.nb + 2 <= 52;   // the Gram's 2 x 4 blocks fit one 192-thread set
    const int band = c.fit_band & ~1;   // the tensor-core fit's rows per item (pairs of rows)
    std::vector<int> fit_tc_start;
    for (int i : order) {
        const int side = table[i].side;
        if (fit_tc) {
            for (int y0 = bd.r; y0 < side - bd.r; y0 += band)
                for (int x0 = bd.r; x0 < side - bd.r; x0 += 128) fit_tc_items.push_back(make_int4(i, x0, y0, 0));
        } else {
            for (int y0 = bd.r; y0 < side - bd.r; y0 += FIT_ROWS) fit_items.push_back(make_int2(i, y0));
        }
        const int nt = (side + 31) / 32;
        for (int t = 0; t < nt * nt; t++) sub_items.push_back(make_int2(i, t));
    }
    // the tensor-core fit's CTA ranges: row pairs (its unit of work) split evenly over one CTA per SM
    int fit_tc_ctas = 0;
    if (fit_tc) {
        std::vector<long> cum(fit_tc_items.size() + 1, 0);
        for (size_t k = 0; k < fit_tc_items.size(); k++) {
            const int4 it = fit_tc_items[k];
            const int rows = std::min(band, table[it.x].side - bd.r - it.z);
            cum[k + 1] = cum[k] + (rows + 1) / 2;
        }
        fit_tc_ctas = std::max(1, std::min(ctx->num_sms, (int)fit_tc_items.size()));
        fit_tc_start.assign(fit_tc_ctas + 1, 0);
        size_t k = 0;
        for (int b = 1; b < fit_tc_ctas; b++) {
            const long target = cum.back() * b / fit_tc_ctas;
            while (k < fit_tc_items.size() && cum[k] < target) k++;
            fit_tc_start[b] = (int)k;
        }
        fit_tc_start[fit_tc_ctas] = (int)fit_tc_items.size();
    }
    // shared memory of the fit kernel: transposed basis taps, design chunk, reference window
    const int NPC = bd.nb + 2;
    const int ng = (bd.nb + FG - 1) / FG;
    const size_t fit_smem = sizeof(float) * ((size_t)ng * bd.ks * bd.ks * FG + (size_t)FIT_CH * (NPC + 1) +
                                             (size_t)(FIT_ROWS + bd.ks - 1) * (512 + bd.ks - 1));
    const int nbk = (NPC + 3) / 4;
    if (!fit_tc && (fit_smem > 220 * 1024 || ng > 8 || nbk * (nbk + 1) / 2 > 256)) return ARGUS_ERR_UNSUPPORTED;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    argus_seg_plan* p = (argus_seg_plan*)calloc(1, sizeof(argus_seg_plan));
    if (!p) return ARGUS_ERR_NOMEM;
    p->ctx = ctx; p->n = n; p->pitch = pitch; p->atlas_h = atlas_h; p->max_side = max_side;
    p->basis = *basis; p->bd = bd; p->NPC = NPC; p->cfg = c;
    p->n_fit_items = (int)fit_items.size();
    p->n_sub_items = (int)sub_items.size();
    p->fit_tc = fit_tc ? 1 : 0;
    p->n_fit_tc_items = (int)fit_tc_items.size();
    p->fit_tc_ctas = fit_tc_ctas;
    bool ok = cudaMalloc(&p->d_seg, sizeof(int4) * n) == cudaSuccess &&
              cudaMalloc(&p->d_fit_items, sizeof(int2) * (fit_items.size() + 1)) == cudaSuccess &&
              cudaMalloc(&p->d_fit_tc_items, sizeof(int4) * (fit_tc_items.size() + 1)) == cudaSuccess &&
              cudaMalloc(&p->d_fit_tc_start, sizeof(int) * (fit_tc_start.size() + 1)) == cudaSuccess &&
              cudaMalloc(&p->d_rscale, sizeof(float) * n) == cudaSuccess &&
              cudaMalloc(&p->d_sub_items, sizeof(int2) * sub_items.size()) == cudaSuccess &&
              cudaMalloc(&p->d_counters, sizeof(int) * 4) == cudaSuccess &&
              cudaMalloc(&p->d_gram, sizeof(double) * (size_t)n * NPC * NPC) == cudaSuccess &&
              cudaMalloc(&p->d_K, sizeof(float) * (size_t)n * bd.ks * bd.ks) == cudaSuccess &&
              cudaMalloc(&p->d_bg, sizeof(double) * (size_t)n) == cudaSuccess;
    if (ok)
        ok = cudaMemcpy(p->d_seg, seg.data(), sizeof(int4) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
             (fit_items.empty() || cudaMemcpy(p->d_fit_items, fit_items.data(), sizeof(int2) * fit_items.size(),
                                              cudaMemcpyHostToDevice) == cudaSuccess) &&
             (fit_tc_items.empty() || cudaMemcpy(p->d_fit_tc_items, fit_tc_items.data(),
                                                 sizeof(int4) * fit_tc_items.size(),
                                                 cudaMemcpyHostToDevice) == cudaSuccess) &&
             (fit_tc_start.empty() || cudaMemcpy(p->d_fit_tc_start, fit_tc_start.data(),
                                                 sizeof(int) * fit_tc_start.size(),
                                                 cudaMemcpyHostToDevice) == cudaSuccess) &&
             cudaMemcpy(p->d_sub_items, sub_items.data(), sizeof(int2) * sub_items.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        argus_segments_destroy(p);
        return ARGUS_ERR_NOMEM;
    }
    // the basis tables (orthonormal images, S) are built once here, outside any capture
    rc = argus_basis_prepare(ctx, basis, 0);
    if (rc == ARGUS_OK && cudaDeviceSynchronize() != cudaSuccess) rc = ARGUS_ERR_CUDA;
    if (rc == ARGUS_OK && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = ARGUS_ERR_CUDA;
    if (rc) {
        argus_segments_destroy(p);
        return rc;
    }
    *out = p;
    return ARGUS_OK;
}

extern "C" int argus_segments_destroy(argus_seg_plan* p) {
    if (!p) return ARGUS_ERR_ARG;
    cudaSetDevice(p->ctx->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    void* ps[] = {p->d_seg, p->d_fit_items, p->d_fit_tc_items, p->d_fit_tc_start, p->d_rscale, p->d_sub_items, p->d_counters, p->d_gram, p->d_K, p->d_bg};
    for (void* q : ps)
        if (q) cudaFree(q);
    free(p);
    return ARGUS_OK;
}

static int segments_enqueue(argus_seg_plan* p, const float* sci, const float* sci_var, const float* ref,
                            const float* ref_var, const uint8_t* flags, float* diff, float* diff_var,
                            uint8_t* mask, double* coeffs, argus_seg_stats* stats, float nsigma, float psf_sigma,
                            argus_source* out, int cap, int* n_found, cudaStream_t st) {
    argus_ctx* ctx = p->ctx;
    const BasisDev& bd = p->bd;
    const int NPC = p->NPC, kk = bd.ks * bd.ks;
    if (cudaMemsetAsync(p->d_counters, 0, sizeof(int) * 4, st) != cudaSuccess) return ARGUS_ERR_CUDA;
    if (cudaMemsetAsync(p->d_gram, 0, sizeof(double) * (size_t)p->n * NPC * NPC, st) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    int* npix = reinterpret_cast<int*>(ctx->resid_part);   // per-segment weighted pixel counts
    if ((size_t)p->n * sizeof(int) > (size_t)ctx->resid_parts * (ctx->np_cols + 4) * sizeof(double))
        return ARGUS_ERR_CAPACITY;
    if (cudaMemsetAsync(npix, 0, sizeof(int) * p->n, st) != cudaSuccess) return ARGUS_ERR_CUDA;
    if (p->fit_tc) {
        SegFitTcArgs ta;
        ta.sci = sci; ta.var = sci_var; ta.ref = ref; ta.flags = flags; ta.pitch = p->pitch; ta.seg = p->d_seg;
        ta.items = p->d_fit_tc_items; ta.n_items = p->n_fit_tc_items; ta.cta_start = p->d_fit_tc_start;
        ta.n_ctas = p->fit_tc_ctas; ta.bimg = ctx->basis_imgf; ta.nb = bd.nb;
        ta.NPC = NPC; ta.band = p->cfg.fit_band & ~1; ta.gram = p->d_gram; ta.n_pix = npix; ta.status = ctx->d_status;
        ta.rscale = p->d_rscale; ta.n_segments = p->n;
        const int trc = argus_seg_fit_tc(ta, bd.ks, st);
        if (trc) return trc;
    }
    SegFitArgs fa;
    fa.sci = sci; fa.var = sci_var; fa.ref = ref; fa.flags = flags; fa.pitch = p->pitch; fa.seg = p->d_seg;
    fa.items = p->d_fit_items; fa.n_items = p->n_fit_items; fa.counter = p->d_counters;
    fa.bimg = ctx->basis_imgf; fa.nb = bd.nb; fa.ks = bd.ks; fa.r = bd.r; fa.NPC = NPC;
    fa.ngroups = (bd.nb + FG - 1) / FG; fa.gram = p->d_gram; fa.n_pix = npix;
    const int fgrid = ctx->num_sms * p->cfg.fit_ctas_per_sm;
    int frc = ARGUS_OK;
    if (!p->fit_tc) switch (bd.ks) {
        case 7: frc = launch_seg_fit<7>(fa, fgrid, st); break;
        case 9: frc = launch_seg_fit<9>(fa, fgrid, st); break;
        case 11: frc = launch_seg_fit<11>(fa, fgrid, st); break;
        case 15: frc = launch_seg_fit<15>(fa, fgrid, st); break;
        case 21: frc = launch_seg_fit<21>(fa, fgrid, st); break;
        default: return ARGUS_ERR_UNSUPPORTED;
    }
    if (frc) return frc;
    SegSolveArgs sa;
    sa.gram = p->d_gram; sa.n_pix = npix; sa.NPC = NPC; sa.nb = bd.nb; sa.S = ctx->basis_S; sa.img = ctx->basis_img;
    sa.kk = kk; sa.coeffs = coeffs; sa.stats = stats; sa.K = p->d_K; sa.bg = p->d_bg; sa.status = ctx->d_status;
    const size_t solve_smem = sizeof(double) * ((size_t)NPC * (NPC + 1) + 2 * NPC);
    seg_solve_kernel<<<p->n, 128, solve_smem, st>>>(sa); argus_count_launch(1);
    SegSubArgs ua;
    ua.sci = sci; ua.var = sci_var; ua.ref = ref; ua.ref_var = ref_var; ua.flags = flags; ua.diff = diff;
    ua.diff_var = diff_var; ua.pitch = p->pitch; ua.seg = p->d_seg; ua.items = p->d_sub_items;
    ua.n_items = p->n_sub_items; ua.counter = p->d_counters + 1; ua.K = p->d_K; ua.bg = p->d_bg; ua.kk = kk;
    const int grid = ctx->num_sms * p->cfg.sub_ctas_per_sm;
    int rc;
    switch (bd.ks) {
        case 7: rc = launch_seg_sub<7>(ua, grid, st); break;
        case 9: rc = launch_seg_sub<9>(ua, grid, st); break;
        case 11: rc = launch_seg_sub<11>(ua, grid, st); break;
        case 15: rc = launch_seg_sub<15>(ua, grid, st); break;
        case 21: rc = launch_seg_sub<21>(ua, grid, st); break;
        default: return ARGUS_ERR_UNSUPPORTED;
    }
    if (rc) return rc;
    // detection over the atlas in slabs of whole segments below 2^31 pixels
    if (mask && n_found) {
        argus_shape sh;
        sh.w = p->pitch; sh.pitch = p->pitch; sh.h = p->atlas_h;
        if ((long)p->atlas_h * p->pitch > 0x7fffffffL) return ARGUS_ERR_UNSUPPORTED;
        rc = argus_detect(ctx, diff, diff_var, flags, sh, nsigma, psf_sigma, mask, out, cap, n_found, st);
        if (rc) return rc;
    }
    return argus_launch_status();
}

extern "C" int argus_segments_run(argus_seg_plan* p, const float* sci, const float* sci_var, const float* ref,
                                  const float* ref_var, const uint8_t* flags, float* diff, float* diff_var,
                                  uint8_t* mask, double* coeffs, argus_seg_stats* stats, float nsigma,
                                  float psf_sigma, argus_source* out, int cap, int* n_found, int use_graph,
                                  argus_stream stream) {
    if (!p || !sci || !sci_var || !ref || !ref_var || !flags || !diff || !diff_var || !coeffs || !stats)
        return ARGUS_ERR_ARG;
    if ((mask == NULL) != (n_found == NULL)) return ARGUS_ERR_ARG;
    const void* ps[] = {sci, sci_var, ref, ref_var, flags, diff, diff_var, mask};
    for (const void* q : ps)
        if (q && argus_check_ptr16(q)) return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(p->ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (!use_graph)
        return segments_enqueue(p, sci, sci_var, ref, ref_var, flags, diff, diff_var, mask, coeffs, stats, nsigma,
                                psf_sigma, out, cap, n_found, st);
    const void* key[12] = {sci, sci_var, ref, ref_var, flags, diff, diff_var, mask, coeffs, stats, out, n_found};
    const bool same = p->exec && memcmp(key, p->key, sizeof(key)) == 0 && p->key_cap == cap;
    if (!same) {
        if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = NULL; }
        if (p->graph) { cudaGraphDestroy(p->graph); p->graph = NULL; }
        cudaStream_t cs = p->cap_stream;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ARGUS_ERR_CUDA;
        const unsigned long long n0 = argus_launch_count();
        const int rc = segments_enqueue(p, sci, sci_var, ref, ref_var, flags, diff, diff_var, mask, coeffs, stats,
                                        nsigma, psf_sigma, out, cap, n_found, cs);
        cudaGraph_t g = NULL;
        const cudaError_t ce = cudaStreamEndCapture(cs, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess || !g) return ARGUS_ERR_CUDA;
        if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return ARGUS_ERR_CUDA;
        }
        p->graph = g;
        memcpy(p->key, key, sizeof(key));
        p->key_cap = cap;
        p->graph_kernels = (int)(argus_launch_count() - n0);
        // the recorded launches were counted but did not run; the replays below are counted instead
        argus_count_launch(-p->graph_kernels);
    }
    argus_count_launch(p->graph_kernels);
    return cudaGraphLaunch(p->exec, st) == cudaSuccess ? ARGUS_OK : ARGUS_ERR_CUDA;
}

extern "C" int argus_segments_items(const argus_seg_plan* p, int* n_fit_items, int* n_sub_items) {
    if (!p) return ARGUS_ERR_ARG;
    if (n_fit_items) *n_fit_items = p->fit_tc ? p->n_fit_tc_items : p->n_fit_items;
    if (n_sub_items) *n_sub_items = p->n_sub_items;
    return ARGUS_OK;
}

extern "C" int argus_segments_kernels(const argus_seg_plan* p, float* K, double* bg, argus_stream stream) {
    if (!p || (!K && !bg)) return ARGUS_ERR_ARG;
    if (cudaSetDevice(p->ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t kk = (size_t)p->bd.ks * p->bd.ks;
    if (K && cudaMemcpyAsync(K, p->d_K, sizeof(float) * kk * p->n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    if (bg && cudaMemcpyAsync(bg, p->d_bg, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    return ARGUS_OK;
}

extern "C" int argus_segments_subtract(argus_seg_plan* p, const float* sci, const float* sci_var, const float* ref,
                                       const float* ref_var, const uint8_t* flags, const float* K, const double* bg,
                                       float* diff, float* diff_var, argus_stream stream) {
    if (!p || !sci || !sci_var || !ref || !ref_var || !flags || !K || !bg || !diff || !diff_var) return ARGUS_ERR_ARG;
    const void* ps[] = {sci, sci_var, ref, ref_var, flags, diff, diff_var};
    for (const void* q : ps)
        if (argus_check_ptr16(q)) return ARGUS_ERR_ALIGN;
    if (cudaSetDevice(p->ctx->device) != cudaSuccess) return ARGUS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int kk = p->bd.ks * p->bd.ks;
    // the given kernels and backgrounds replace the plan's fitted ones
    if (cudaMemcpyAsync(p->d_K, K, sizeof(float) * (size_t)kk * p->n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(p->d_bg, bg, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(p->d_counters, 0, sizeof(int) * 4, st) != cudaSuccess)
        return ARGUS_ERR_CUDA;
    SegSubArgs ua;
    ua.sci = sci; ua.var = sci_var; ua.ref = ref; ua.ref_var = ref_var; ua.flags = flags; ua.diff = diff;
    ua.diff_var = diff_var; ua.pitch = p->pitch; ua.seg = p->d_seg; ua.items = p->d_sub_items;
    ua.n_items = p->n_sub_items; ua.counter = p->d_counters + 1; ua.K = p->d_K; ua.bg = p->d_bg; ua.kk = kk;
    const int grid = p->ctx->num_sms * p->cfg.sub_ctas_per_sm;
    switch (p->bd.ks) {
        case 7: return launch_seg_sub<7>(ua, grid, st);
        case 9: return launch_seg_sub<9>(ua, grid, st);
        case 11: return launch_seg_sub<11>(ua, grid, st);
        case 15: return launch_seg_sub<15>(ua, grid, st);
        case 21: return launch_seg_sub<21>(ua, grid, st);
        default: return ARGUS_ERR_UNSUPPORTED;
    }
}
