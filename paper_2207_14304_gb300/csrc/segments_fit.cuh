// The batched segments' fit on the tensor cores (segments_tc.cu), called by the
// segment plan (segments.cu).
#pragma once
#include "argus_internal.cuh"

struct SegFitTcArgs {
    const float* sci;
    const float* var;
    const float* ref;
    const uint8_t* flags;
    long pitch;
    const int4* seg;       // (row0, side, col0, -)
    const int4* items;     // (segment, x0, y0, -): interior strip origin, segment pixels
    int n_items;
    const int* cta_start;  // [n_ctas + 1]: CTA b takes items cta_start[b] .. cta_start[b + 1] - 1
    int n_ctas;
    const float* bimg;     // orthonormal basis images [nb][ks * ks]
    int nb, NPC;           // basis functions, Gram columns (nb + 2)
    int band;              // interior rows per item (even)
    double* gram;          // [segments][NPC][NPC], upper triangle accumulated
    float* rscale;         // [segments] scratch: the power of two applied to each segment's R
    int n_segments;
    int* n_pix;            // per segment count of weighted pixels
    int* status;
};

// Shared memory of the kernel for kernel side ks and NPC Gram columns (0: no
// tensor-core kernel for this side).
size_t argus_seg_fit_tc_smem(int ks, int NPC);
// Enqueue the fit over a.items on a.n_ctas persistent CTAs.
int argus_seg_fit_tc(const SegFitTcArgs& a, int ks, cudaStream_t st);
