// Per-tile body of the reference convolution, subtraction and difference
// variance (paper Sec. 4.2 direct image subtraction; noise maps, Sec. 3.2),
// shared by the full-frame kernel (subtract.cu) and the persistent batched
// segment kernel (segments.cu).
//
//   D   = I - sum_k p_k(x,y) (R (x) K_k)(x,y) - sum_k bg_k p_k(x,y)
//   V_D = V_I + (Kc^2 (x) V_ref)(x,y),  Kc the kernel at the centre of the VAR_TILE tile
//
// One CTA owns one 32x32 output tile, which lies inside one variance tile, so
// the squared tile-centre kernel is built once per CTA.  The reference and its
// variance are staged with their halo in shared memory; each of the 128
// threads computes a column strip of 8 outputs for all NK spatial terms.
#pragma once
#include "argus_internal.cuh"

namespace argus_sub {

constexpr int TILE = 32;
// The difference variance uses the kernel at the centre of the VAR_TILE x
// VAR_TILE frame tile holding the pixel (a multiple of TILE, so the 32x32
// output tiles nest in it).
constexpr int VAR_TILE = 128;
constexpr int ROWS_PER_THREAD = 8;
constexpr int THREADS = 128;

struct SubArgs {
    const float* sci;
    const float* sci_var;
    const float* ref;
    const float* ref_var;
    const uint8_t* flags;
    const float* K;     // [NK][KS*KS]
    const double* bg;   // [Kb]
    float* diff;
    float* diff_var;
    long pitch;
    int w, h, W, H, ox, oy, nbg, bg_deg, sdeg;
};

__device__ __forceinline__ void spatial_terms(float xt, float yt, int deg, float* out) {
    // p_k = xt^i yt^j, i + j <= deg, ordered i then j
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

// CONV = false computes only the difference variance (the difference image
// then comes from the tensor-core kernel).
template <int KS, int NK, bool CONV = true>
__device__ __forceinline__ void subtract_tile(const SubArgs& a, const int tx0, const int ty0, float* smem) {
    constexpr int R = (KS - 1) / 2;
    constexpr int SW = TILE + 2 * R;             // staged tile side
    constexpr int NKP = NK == 1 ? 1 : (NK <= 4 ? 4 : 8);
    constexpr int KSP = (KS + 3) / 4 * 4;
    constexpr int KTSZ = (KS * KS * NKP + 3) / 4 * 4;   // keeps Kc2 16-byte aligned

    // CONV: Rs [SW][SW], Vs [SW][SW], Kt [KS][KS][NKP], Kc2 [KS][KSP];
    // variance only: Vs [SW][SW], Kc2 [KS][KSP]  (SW even, Kc2 16-byte aligned)
    float* Rs = smem;
    float* Vs = CONV ? Rs + SW * SW : smem;
    float* Kt = Vs + SW * SW;
    float* Kc2 = CONV ? Kt + KTSZ : Vs + SW * SW;

    const int tid = threadIdx.x;
    __syncthreads();   // the previous tile's readers are done with shared memory

    // stage reference and reference variance with halo (zero outside the image)
    for (int e = tid; e < SW * SW; e += THREADS) {
        const int iy = e / SW, ix = e - iy * SW;
        const int gy = ty0 - R + iy, gx = tx0 - R + ix;
        float rv = 0.0f, vv = 0.0f;
        if (gy >= 0 && gy < a.h && gx >= 0 && gx < a.w) {
            const long p = (long)gy * a.pitch + gx;
            if (CONV) rv = __ldg(a.ref + p);
            vv = __ldg(a.ref_var + p);
        }
        if (CONV) Rs[e] = rv;
        Vs[e] = vv;
    }
    // kernel taps, transposed to [iu][iv][k]
    for (int e = tid; e < (CONV ? KS * KS * NKP : 0); e += THREADS) {
        const int k = e % NKP, t = e / NKP;
        const int iu = t / KS, iv = t - iu * KS;
        Kt[e] = k < NK ? __ldg(a.K + k * KS * KS + iv * KS + iu) : 0.0f;
    }
    // squared kernel at the tile centre (frame coordinates)
    {
        float pc[ARGUS_MAX_TERMS];
        const float xc = (float)(((tx0 + a.ox) / VAR_TILE) * VAR_TILE) + 0.5f * (VAR_TILE - 1);
        const float yc = (float)(((ty0 + a.oy) / VAR_TILE) * VAR_TILE) + 0.5f * (VAR_TILE - 1);
        const float xt = a.W > 1 ? (2.0f * xc - (float)(a.W - 1)) / (float)(a.W - 1) : 0.0f;
        const float yt = a.H > 1 ? (2.0f * yc - (float)(a.H - 1)) / (float)(a.H - 1) : 0.0f;
        spatial_terms(xt, yt, a.sdeg, pc);
        for (int e = tid; e < KS * KSP; e += THREADS) {
            const int iu = e / KSP, iv = e - iu * KSP;
            float kc = 0.0f;
            if (iv < KS) {
#pragma unroll
                for (int k = 0; k < NK; k++) kc = fmaf(pc[k], __ldg(a.K + k * KS * KS + iv * KS + iu), kc);
            }
            Kc2[e] = kc * kc;
        }
    }
    __syncthreads();

    const int lx = tid & 31;
    const int ly0 = (tid >> 5) * ROWS_PER_THREAD;

    float acc[NK][ROWS_PER_THREAD];
#pragma unroll
    for (int k = 0; k < NK; k++)
#pragma unroll
        for (int j = 0; j < ROWS_PER_THREAD; j++) acc[k][j] = 0.0f;

    // output (lx, ly0 + j), tap (du, dv) = (iu - R, iv - R):
    //   R(x - du, y - dv) = Rs[ly0 + j + 2R - iv][lx + 2R - iu]
    // The iv taps run in blocks of IVB: each block loads its own window of
    // ROWS_PER_THREAD + IVB - 1 reference values, which keeps the unrolled body
    // small enough for the instruction cache.
    constexpr int IVB = (KS % 7 == 0) ? 7 : ((KS % 5 == 0) ? 5 : KS);
    constexpr int NW = ROWS_PER_THREAD + IVB - 1;
#pragma unroll 1
    for (int iu = 0; iu < (CONV ? KS : 0); iu++) {
        const float* kt = Kt + iu * KS * NKP;
        const float* rcol = Rs + ly0 * SW + lx + 2 * R - iu;
#pragma unroll 1
        for (int b = 0; b < KS / IVB; b++) {
            // window row m holds Rs[ly0 + m + 2R - b*IVB - (IVB-1)]
            const int base = 2 * R - b * IVB - (IVB - 1);
            float win[NW];
#pragma unroll
            for (int m = 0; m < NW; m++) win[m] = rcol[(m + base) * SW];
#pragma unroll
            for (int i = 0; i < IVB; i++) {
                const int iv = b * IVB + i;
                float kk[NKP];
                if constexpr (NKP == 1) {
                    kk[0] = kt[iv];
                } else {
#pragma unroll
                    for (int q = 0; q < NKP; q += 4)
                        *reinterpret_cast<float4*>(kk + q) = *reinterpret_cast<const float4*>(kt + iv * NKP + q);
                }
#pragma unroll
                for (int j = 0; j < ROWS_PER_THREAD; j++) {
                    // row ly0 + j + 2R - iv  ->  window index j + (IVB - 1) - i
                    const float rv = win[j + (IVB - 1) - i];
#pragma unroll
                    for (int k = 0; k < NK; k++) acc[k][j] = fmaf(kk[k], rv, acc[k][j]);
                }
            }
        }
    }

    float accv[ROWS_PER_THREAD];
#pragma unroll
    for (int j = 0; j < ROWS_PER_THREAD; j++) accv[j] = 0.0f;
#pragma unroll 1
    for (int iu = 0; iu < (a.diff_var ? KS : 0); iu++) {   // no variance output: skipped
        const float* vcol = Vs + ly0 * SW + lx + 2 * R - iu;
#pragma unroll 1
        for (int b = 0; b < KS / IVB; b++) {
            const int base = 2 * R - b * IVB - (IVB - 1);
            float win[NW];
#pragma unroll
            for (int m = 0; m < NW; m++) win[m] = vcol[(m + base) * SW];
#pragma unroll
            for (int i = 0; i < IVB; i++) {
                const float kc = Kc2[iu * KSP + b * IVB + i];
#pragma unroll
                for (int j = 0; j < ROWS_PER_THREAD; j++) accv[j] = fmaf(kc, win[j + (IVB - 1) - i], accv[j]);
            }
        }
    }

    // epilogue: spatial combination, background, edge and flag handling
    const int x = tx0 + lx;
    if (x >= a.w) return;
    const float xt = a.W > 1 ? (float)(2 * (x + a.ox) - (a.W - 1)) / (float)(a.W - 1) : 0.0f;
    float bgc[ARGUS_MAX_TERMS];
    for (int k = 0; k < a.nbg; k++) bgc[k] = (float)a.bg[k];
#pragma unroll
    for (int j = 0; j < ROWS_PER_THREAD; j++) {
        const int y = ty0 + ly0 + j;
        if (y >= a.h) break;
        const long p = (long)y * a.pitch + x;
        float D = 0.0f, VD = 0.0f;
        const bool inner = x >= R && y >= R && x <= a.w - 1 - R && y <= a.h - 1 - R;
        if (!CONV) {
            if (inner && a.flags[p] == 0) VD = a.sci_var[p] + accv[j];
            a.diff_var[p] = VD;
            continue;
        }
        if (inner && a.flags[p] == 0) {
            const float yt = a.H > 1 ? (float)(2 * (y + a.oy) - (a.H - 1)) / (float)(a.H - 1) : 0.0f;
            float pk[ARGUS_MAX_TERMS];
            spatial_terms(xt, yt, a.sdeg, pk);
            float conv = 0.0f;
#pragma unroll
            for (int k = 0; k < NK; k++) conv = fmaf(pk[k], acc[k][j], conv);
            float pb[ARGUS_MAX_TERMS];
            spatial_terms(xt, yt, a.bg_deg, pb);
            float b = 0.0f;
            for (int k = 0; k < a.nbg; k++) b = fmaf(bgc[k], pb[k], b);
            D = a.sci[p] - conv - b;
            VD = a.sci_var[p] + accv[j];
        }
        a.diff[p] = D;
        if (a.diff_var) a.diff_var[p] = VD;
    }
}


template <int KS, int NK, bool CONV = true>
constexpr size_t tile_smem_bytes() {
    constexpr int R = (KS - 1) / 2;
    constexpr int SW = TILE + 2 * R;
    constexpr int NKP = NK == 1 ? 1 : (NK <= 4 ? 4 : 8);
    constexpr int KSP = (KS + 3) / 4 * 4;
    constexpr int KTSZ = (KS * KS * NKP + 3) / 4 * 4;
    return CONV ? sizeof(float) * (2 * SW * SW + KTSZ + KS * KSP) : sizeof(float) * (SW * SW + KS * KSP);
}

}  // namespace argus_sub

// Difference image on the tensor cores (subtract_tc.cu) for the kernel sizes it
// is built for; ARGUS_ERR_UNSUPPORTED for the others.
int argus_subtract_tc(const argus_sub::SubArgs& a, int ksize, int nk, int* status, cudaStream_t st);
// Difference variance on the tensor cores for the kernel sizes and frame origins it
// is built for; ARGUS_ERR_UNSUPPORTED for the others.
int argus_subtract_var_tc(const argus_sub::SubArgs& a, int ksize, int* status, cudaStream_t st);
