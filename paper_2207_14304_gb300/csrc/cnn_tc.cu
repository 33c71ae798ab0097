// K9 forward on the tensor cores: the learned kernel surrogate's whole forward
// pass (1x1 conv 2 -> 32, four 7x7 'same' 32 -> 32 convolutions with ReLU,
// 1x1 conv 32 -> 1, output / 441) in one persistent kernel, the four 7x7
// convolutions as implicit GEMMs on tcgen05 (kind::f16: BF16 operands, FP32
// accumulation in TMEM).  The paper has no learned kernel; this is the learned
// alternative to its least-squares PSF-matching kernel (Sec. 4.2).
//
// Implicit GEMM.  A stamp's activations sit in shared memory zero padded to
// 27 columns (21 + 6) and flattened: plane pixel P = row * 27 + col.  Output q
// = y * 27 + x (y < 21, every x < 27; x >= 21 are computed and discarded)
// reads tap (ky, kx) at plane pixel q + ky * 27 + kx, so the A operand of one
// tap for 128 consecutive outputs is 128 consecutive plane pixels: a plain
// descriptor offset, no gather.  Per tap: D[q][o] += sum_i A[q + off][i]
// W[ky][kx][i][o], M = 128 outputs, N = 32 output channels, K = 32 input
// channels (two K = 16 MMAs).  Five M tiles cover q < 567 (the last one starts
// at 439 and owns q >= 512), 160 TMEM columns.
//
// Precision.  Activations are split into BF16 hi + lo (v = hi + lo + e, |e| <=
// 2^-17 |v|) and each tap runs both against the BF16 weights, so the layer is
// the FP32 layer to within FP32-level rounding: the same weights as the SIMT
// BF16 path, activations to ~16 significant bits instead of BF16's 8.
//
// Layouts.  Operand planes [hi|lo][chunk of 8 channels][756 plane pixels][8]
// (BF16, 16 bytes per pixel and chunk): a K-major core matrix is 8 consecutive
// pixels of one chunk (128 contiguous bytes), LBO = one plane (the next 8
// channels), SBO = 128 bytes.  Weights are packed once per call into
// [layer][tap][chunk][o][8] (2 KB per tap, LBO 512, SBO 128) and streamed
// through a ring of 7 tap slots by bulk copies.
//
// Roles (192 threads): warp 0 allocates TMEM and one lane issues the MMAs;
// warp 1 lane 0 streams the weights; warps 2-5 (128 threads, one TMEM lane
// each) compute layer 1 into the planes, and after each convolution read the
// accumulators, add the bias, apply ReLU and write the next layer's planes in
// place (the MMAs of the layer have completed), optionally the FP32
// activations for the backward pass, and after the last one the 1x1 output.
// Two CTAs per SM overlap one another's epilogues and weight waits.  Every
// wait is bounded; a timeout latches ARGUS_ERR_TIMEOUT and all roles stop.
//
// The data gradient of each 7x7 layer is the same implicit GEMM with the
// layer's kernel transposed and flipped (cnn_dgrad_tc_kernel): the gradient
// planes dz (BF16 hi + lo) against W'[ky][kx][o][i] = W[6 - ky][6 - kx][i][o].
#include <cuda_bf16.h>

#include "argus_internal.cuh"
#include "split16.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int S = 21, NPX = S * S, C = 32, KS = 7, NTAP = KS * KS;
constexpr int WP = S + KS - 1;            // 27: padded row length
constexpr int HPR = 28;                   // plane rows: q + 6 * 27 + 6 < 756 for q < 567
constexpr int NPP = WP * HPR;             // 756 plane pixels
constexpr int PLANE = NPP * 16;           // one 8-channel chunk plane (BF16): 12,096 bytes
constexpr int SETB = (C / 8) * PLANE;     // one operand set (hi or lo): 48,384 bytes
constexpr int NQ = S * WP;                // 567 flattened outputs
constexpr int MT = 5;                     // M tiles
constexpr int TAPB = (C / 8) * C * 16;    // one tap's B operand: 2,048 bytes
constexpr int NSLOT = 7;                  // weight ring depth (taps)
constexpr int NTHR = 192;
constexpr int NEPI = 128;                 // epilogue threads
constexpr uint32_t TMEM_COLS = 256;       // 160 used
constexpr long long WAIT_LIMIT = 2000000000LL;   // ~1 s of SM clock
static_assert(MT * 128 >= NQ && 4 * 128 < NQ, "five M tiles, the last one overlapping the fourth");
static_assert(NQ - 1 + (KS - 1) * WP + (KS - 1) < NPP, "the last tile's reads stay inside the planes");
static_assert(MT * C <= (int)TMEM_COLS, "accumulators fit the allocation");

// parameter offsets (the layout of the library's parameter vector)
constexpr long OFF_W1 = 0, OFF_B1 = 64;
__host__ __device__ constexpr long off_w(int l) { return 96 + (long)l * (49 * 1024 + 32); }
__host__ __device__ constexpr long off_b(int l) { return off_w(l) + 49 * 1024; }
constexpr long OFF_W6 = 96 + 4L * (49 * 1024 + 32), OFF_B6 = OFF_W6 + 32;

__device__ __forceinline__ int tile_q0(int t) { return t < MT - 1 ? 128 * t : NQ - 128; }

struct CnnTcShared {
    alignas(128) uint8_t act[2][SETB];    // operand planes: [hi | lo][chunk][pixel][8 channels]
    alignas(128) uint8_t wb[NSLOT][TAPB];   // ring of per-tap B operands
    float w1[2 * C], b1[C], bc[4][C], w6[C], b6;
    uint64_t wfull[NSLOT], wempty[NSLOT], ready, accfull, drain;
    uint32_t tmem;
    int abort;
};
static_assert(sizeof(CnnTcShared) + 1024 <= 228 * 1024 / 2, "two CTAs per SM");

// One try first (the common case), then a bounded wait that also gives up once
// another role has aborted.
__device__ __forceinline__ bool wait_or_abort(CnnTcShared& sh, uint64_t* bar, uint32_t parity, int* status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (*(volatile int*)&sh.abort) return false;
    if (!tc::mbar_wait_bounded(bar, parity, WAIT_LIMIT)) {
        sh.abort = 1;
        argus_latch(status, ARGUS_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// The 32 channels of plane pixel P as BF16 hi and lo parts into both operand sets.
__device__ __forceinline__ void store_planes(CnnTcShared& sh, int P, const float (&h)[C]) {
#pragma unroll
    for (int ic = 0; ic < C / 8; ic++) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float v0 = h[ic * 8 + 2 * k], v1 = h[ic * 8 + 2 * k + 1];
            hi[k] = bf16x2_rn(v0, v1);
            lo[k] = bf16x2_rn(v0 - __uint_as_float(hi[k] << 16), v1 - __uint_as_float(hi[k] & 0xffff0000u));
        }
        *reinterpret_cast<uint4*>(sh.act[0] + ic * PLANE + P * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(sh.act[1] + ic * PLANE + P * 16) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

__device__ __forceinline__ void store_acts(float* dst, const float (&h)[C]) {
#pragma unroll
    for (int k = 0; k < C / 4; k++)
        reinterpret_cast<float4*>(dst)[k] = make_float4(h[4 * k], h[4 * k + 1], h[4 * k + 2], h[4 * k + 3]);
}

// Packs the BF16 weights W[l][ky][kx][i][o] of the four 7x7 layers into the
// B-operand layout [l][tap][i / 8][o][i % 8].
__global__ void cnn_pack_tc_kernel(const __nv_bfloat16* w, __nv_bfloat16* wp) {
    const long tot = 4L * NTAP * C * C;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e & 7), o = (int)((e >> 3) & 31), ic = (int)((e >> 8) & 3);
        const long lt = e >> 10;
        const int l = (int)(lt / NTAP), tap = (int)(lt % NTAP);
        wp[e] = w[off_w(l) + ((long)tap * C + ic * 8 + j) * C + o];
    }
}

// x [n][441][2]; y [n][441]; acts (optional) [5][lstride] with layer l at
// acts + l * lstride, [n][441][32] FP32 (h1 .. h5, post-activation).
__global__ void __launch_bounds__(NTHR, 2) cnn_fwd_tc_kernel(const float* __restrict__ x,
                                                             const __nv_bfloat16* __restrict__ w,
                                                             const uint8_t* __restrict__ wpack, float* __restrict__ y,
                                                             float* __restrict__ acts, long lstride, int n,
                                                             int* status) {
    extern __shared__ __align__(1024) uint8_t cnn_tc_smem[];
    CnnTcShared& sh = *reinterpret_cast<CnnTcShared*>(cnn_tc_smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < 2 * C; e += NTHR) sh.w1[e] = __bfloat162float(w[OFF_W1 + e]);
    for (int e = tid; e < C; e += NTHR) {
        sh.b1[e] = __bfloat162float(w[OFF_B1 + e]);
        sh.w6[e] = __bfloat162float(w[OFF_W6 + e]);
    }
    for (int e = tid; e < 4 * C; e += NTHR) sh.bc[e / C][e % C] = __bfloat162float(w[off_b(e / C) + e % C]);
    // both operand sets zeroed once: the padding stays zero, interiors are rewritten per layer
    for (int e = tid; e < 2 * SETB / 16; e += NTHR) reinterpret_cast<uint4*>(sh.act[0])[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        sh.b6 = __bfloat162float(w[OFF_B6]);
        for (int s = 0; s < NSLOT; s++) {
            tc::mbar_init(&sh.wfull[s], 1);
            tc::mbar_init(&sh.wempty[s], 1);
        }
        tc::mbar_init(&sh.ready, NEPI);
        tc::mbar_init(&sh.accfull, 1);
        tc::mbar_init(&sh.drain, 1);
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&sh.tmem, TMEM_COLS);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sh.tmem;

    if (warp == 0) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(1, 128, C);
            const uint32_t abase = tc::smem_u32(sh.act[0]), bbase = tc::smem_u32(sh.wb[0]);
            int cnt = 0, rk = 0;
            bool run = true, any = false;
            for (int img = blockIdx.x; img < n && run; img += gridDim.x) {
                for (int l = 0; l < 4 && run; l++) {
                    if (!wait_or_abort(sh, &sh.ready, rk & 1, status)) { run = false; break; }
                    rk++;
                    tc::fence_after();
                    for (int tap = 0; tap < NTAP; tap++, cnt++) {
                        const int s = cnt % NSLOT;
                        if (!wait_or_abort(sh, &sh.wfull[s], (cnt / NSLOT) & 1, status)) { run = false; break; }
                        tc::fence_after();
                        const int ky = tap / KS, kx = tap - KS * ky;
                        const uint32_t bs = bbase + (uint32_t)(s * TAPB);
#pragma unroll
                        for (int t = 0; t < MT; t++) {
                            const uint32_t arow = abase + (uint32_t)((tile_q0(t) + ky * WP + kx) * 16);
#pragma unroll
                            for (int kc = 0; kc < 2; kc++) {
                                const uint64_t bd = tc::smem_desc(bs + (uint32_t)(kc * 2 * 512), 512, 128);
#pragma unroll
                                for (int hl = 0; hl < 2; hl++) {
                                    const uint64_t ad =
                                        tc::smem_desc(arow + (uint32_t)(hl * SETB + 2 * kc * PLANE), PLANE, 128);
                                    tc::mma_bf16(tmem + (uint32_t)(t * C), ad, bd, idesc, (tap | kc | hl) ? 1u : 0u);
                                }
                            }
                        }
                        tc::commit(&sh.wempty[s]);
                        any = true;
                    }
                    if (run) tc::commit(&sh.accfull);
                }
            }
            // every issued MMA lands before TMEM is released
            if (any) {
                tc::commit(&sh.drain);
                if (!tc::mbar_wait_bounded(&sh.drain, 0, WAIT_LIMIT)) {
                    sh.abort = 1;
                    argus_latch(status, ARGUS_ERR_TIMEOUT);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- weight producer: one bulk copy per tap, in the MMA order
        if (lane == 0) {
            int cnt = 0;
            bool run = true;
            for (int img = blockIdx.x; img < n && run; img += gridDim.x)
                for (int l = 0; l < 4 && run; l++)
                    for (int tap = 0; tap < NTAP; tap++, cnt++) {
                        const int s = cnt % NSLOT;
                        if (cnt >= NSLOT && !wait_or_abort(sh, &sh.wempty[s], (cnt / NSLOT - 1) & 1, status)) {
                            run = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&sh.wfull[s], TAPB);
                        tc::bulk_g2s(sh.wb[s], wpack + ((long)l * NTAP + tap) * TAPB, TAPB, &sh.wfull[s]);
                    }
            // copies in flight land before the CTA exits (the latest phase of each slot)
            for (int j = cnt > NSLOT ? cnt - NSLOT : 0; j < cnt; j++)
                if (!tc::mbar_wait_bounded(&sh.wfull[j % NSLOT], (j / NSLOT) & 1, WAIT_LIMIT)) {
                    sh.abort = 1;
                    argus_latch(status, ARGUS_ERR_TIMEOUT);
                    break;
                }
        }
        __syncwarp();
    } else {
        // ---------------- layer 1, epilogues, output
        const int et = tid - 64;                     // 0 .. 127
        const int lq = warp & 3;                     // the TMEM lane quarter this warp may read
        const int r = lq * 32 + lane;                // accumulator row (TMEM lane) of this thread
        const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16);
        int ak = 0;
        bool run = true;
        for (int img = blockIdx.x; img < n && run; img += gridDim.x) {
            const float* xi = x + (long)img * NPX * 2;
            for (int p = et; p < NPX; p += NEPI) {
                const float x0 = xi[2 * p], x1 = xi[2 * p + 1];
                float h[C];
#pragma unroll
                for (int o = 0; o < C; o++) h[o] = sh.b1[o] + sh.w1[2 * o] * x0 + sh.w1[2 * o + 1] * x1;
                const int py = p / S, px = p - py * S;
                store_planes(sh, (py + 3) * WP + px + 3, h);
                if (acts) store_acts(acts + ((long)img * NPX + p) * C, h);
            }
            tc::fence_proxy_async();   // plane writes visible to the tensor cores
            tc::fence_before();
            tc::mbar_arrive(&sh.ready);
            for (int l = 0; l < 4; l++) {
                bool ok = true;
                if (lane == 0) ok = wait_or_abort(sh, &sh.accfull, ak & 1, status);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                ak++;
                if (!ok) { run = false; break; }
                tc::fence_after();
#pragma unroll 1
                for (int t = 0; t < MT; t++) {
                    uint32_t v[32];
                    tc::tmem_ld32_nowait(tl + (uint32_t)(t * C), v);
                    tc::tmem_wait_ld32(v);
                    const int q = tile_q0(t) + r;
                    const int qy = q / WP, qx = q - qy * WP;
                    if ((t == MT - 1 && q < 128 * (MT - 1)) || qx >= S) continue;   // not owned, or padding
                    float h[C];
#pragma unroll
                    for (int o = 0; o < C; o++) h[o] = fmaxf(__uint_as_float(v[o]) + sh.bc[l][o], 0.0f);
                    const int p = qy * S + qx;
                    if (acts) store_acts(acts + (long)(l + 1) * lstride + ((long)img * NPX + p) * C, h);
                    if (l < 3) {
                        store_planes(sh, q + 3 * WP + 3, h);
                    } else {
                        float s = sh.b6;
#pragma unroll
                        for (int o = 0; o < C; o++) s = fmaf(sh.w6[o], h[o], s);
                        y[(long)img * NPX + p] = s * (1.0f / NPX);
                    }
                }
                if (l < 3) {
                    tc::fence_proxy_async();
                    tc::fence_before();
                    tc::mbar_arrive(&sh.ready);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

// Packs the BF16 weights of 7x7 layer l for its data gradient: the transposed, flipped
// kernel W'[ky][kx][o][i] = W[6 - ky][6 - kx][i][o] in the B-operand layout
// [tap][o / 8][i][o % 8] (N = the layer's input channels, K = its output channels).
__global__ void cnn_pack_dgrad_tc_kernel(const __nv_bfloat16* w, __nv_bfloat16* wp, int l) {
    const long tot = (long)NTAP * C * C;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e & 7), i = (int)((e >> 3) & 31), oc = (int)((e >> 8) & 3), tap = (int)(e >> 10);
        const int ky = tap / KS, kx = tap - KS * ky;
        const int ft = (KS - 1 - ky) * KS + (KS - 1 - kx);
        wp[e] = w[off_w(l) + ((long)ft * C + i) * C + oc * 8 + j];
    }
}

// Data gradient of one 7x7 layer on the tensor cores: dz = dh_out (h_out > 0) and
//   dh_in[y][x][i] = sum_{ky,kx,o} W[ky][kx][i][o] dz[y - ky + 3][x - kx + 3][o]
//                  = sum_{ky,kx,o} W'[ky][kx][o][i] dz[y + ky - 3][x + kx - 3][o],
// the forward's implicit GEMM with the packed W' (cnn_pack_dgrad_tc_kernel) and dz in
// the operand planes (BF16 hi + lo).  dh_out, h_out, dh_in: [n][441][32] FP32.  Roles as
// in the forward: warp 0 issues the MMAs of the 49 taps per image, warp 1 streams the
// weights, warps 2-5 write dz into the planes and read the accumulators into dh_in.
__global__ void __launch_bounds__(NTHR, 2) cnn_dgrad_tc_kernel(const float* __restrict__ dh_out,
                                                               const float* __restrict__ h_out,
                                                               const uint8_t* __restrict__ wpack,
                                                               float* __restrict__ dh_in, int n, int* status) {
    extern __shared__ __align__(1024) uint8_t cnn_tc_smem[];
    CnnTcShared& sh = *reinterpret_cast<CnnTcShared*>(cnn_tc_smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // both operand sets zeroed once: the padding stays zero, interiors are rewritten per image
    for (int e = tid; e < 2 * SETB / 16; e += NTHR) reinterpret_cast<uint4*>(sh.act[0])[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int s = 0; s < NSLOT; s++) {
            tc::mbar_init(&sh.wfull[s], 1);
            tc::mbar_init(&sh.wempty[s], 1);
        }
        tc::mbar_init(&sh.ready, NEPI);
        tc::mbar_init(&sh.accfull, 1);
        tc::mbar_init(&sh.drain, 1);
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&sh.tmem, TMEM_COLS);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sh.tmem;

    if (warp == 0) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(1, 128, C);
            const uint32_t abase = tc::smem_u32(sh.act[0]), bbase = tc::smem_u32(sh.wb[0]);
            int cnt = 0, rk = 0;
            bool run = true, any = false;
            for (int img = blockIdx.x; img < n && run; img += gridDim.x) {
                if (!wait_or_abort(sh, &sh.ready, rk & 1, status)) { run = false; break; }
                rk++;
                tc::fence_after();
                for (int tap = 0; tap < NTAP; tap++, cnt++) {
                    const int s = cnt % NSLOT;
                    if (!wait_or_abort(sh, &sh.wfull[s], (cnt / NSLOT) & 1, status)) { run = false; break; }
                    tc::fence_after();
                    const int ky = tap / KS, kx = tap - KS * ky;
                    const uint32_t bs = bbase + (uint32_t)(s * TAPB);
#pragma unroll
                    for (int t = 0; t < MT; t++) {
                        const uint32_t arow = abase + (uint32_t)((tile_q0(t) + ky * WP + kx) * 16);
#pragma unroll
                        for (int kc = 0; kc < 2; kc++) {
                            const uint64_t bd = tc::smem_desc(bs + (uint32_t)(kc * 2 * 512), 512, 128);
#pragma unroll
                            for (int hl = 0; hl < 2; hl++) {
                                const uint64_t ad = tc::smem_desc(arow + (uint32_t)(hl * SETB + 2 * kc * PLANE), PLANE, 128);
                                tc::mma_bf16(tmem + (uint32_t)(t * C), ad, bd, idesc, (tap | kc | hl) ? 1u : 0u);
                            }
                        }
                    }
                    tc::commit(&sh.wempty[s]);
                    any = true;
                }
                if (run) tc::commit(&sh.accfull);
            }
            if (any) {
                tc::commit(&sh.drain);
                if (!tc::mbar_wait_bounded(&sh.drain, 0, WAIT_LIMIT)) {
                    sh.abort = 1;
                    argus_latch(status, ARGUS_ERR_TIMEOUT);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- weight producer: one bulk copy per tap, in the MMA order
        if (lane == 0) {
            int cnt = 0;
            bool run = true;
            for (int img = blockIdx.x; img < n && run; img += gridDim.x)
                for (int tap = 0; tap < NTAP; tap++, cnt++) {
                    const int s = cnt % NSLOT;
                    if (cnt >= NSLOT && !wait_or_abort(sh, &sh.wempty[s], (cnt / NSLOT - 1) & 1, status)) {
                        run = false;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&sh.wfull[s], TAPB);
                    tc::bulk_g2s(sh.wb[s], wpack + (long)tap * TAPB, TAPB, &sh.wfull[s]);
                }
            for (int j = cnt > NSLOT ? cnt - NSLOT : 0; j < cnt; j++)
                if (!tc::mbar_wait_bounded(&sh.wfull[j % NSLOT], (j / NSLOT) & 1, WAIT_LIMIT)) {
                    sh.abort = 1;
                    argus_latch(status, ARGUS_ERR_TIMEOUT);
                    break;
                }
        }
        __syncwarp();
    } else {
        // ---------------- dz into the planes, accumulators into dh_in
        const int et = tid - 64;
        const int lq = warp & 3;
        const int r = lq * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16);
        int ak = 0;
        for (int img = blockIdx.x; img < n; img += gridDim.x) {
            const float* go = dh_out + (long)img * NPX * C;
            const float* ho = h_out + (long)img * NPX * C;
            for (int p = et; p < NPX; p += NEPI) {
                float g[C];
#pragma unroll
                for (int k = 0; k < C / 4; k++) {
                    const float4 gv = reinterpret_cast<const float4*>(go + (long)p * C)[k];
                    const float4 hv = reinterpret_cast<const float4*>(ho + (long)p * C)[k];
                    g[4 * k] = hv.x > 0.0f ? gv.x : 0.0f;
                    g[4 * k + 1] = hv.y > 0.0f ? gv.y : 0.0f;
                    g[4 * k + 2] = hv.z > 0.0f ? gv.z : 0.0f;
                    g[4 * k + 3] = hv.w > 0.0f ? gv.w : 0.0f;
                }
                const int py = p / S, px = p - py * S;
                store_planes(sh, (py + 3) * WP + px + 3, g);
            }
            tc::fence_proxy_async();   // plane writes visible to the tensor cores
            tc::fence_before();
            tc::mbar_arrive(&sh.ready);
            bool ok = true;
            if (lane == 0) ok = wait_or_abort(sh, &sh.accfull, ak & 1, status);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            ak++;
            if (!ok) break;
            tc::fence_after();
            float* dst = dh_in + (long)img * NPX * C;
#pragma unroll 1
            for (int t = 0; t < MT; t++) {
                uint32_t v[32];
                tc::tmem_ld32_nowait(tl + (uint32_t)(t * C), v);
                tc::tmem_wait_ld32(v);
                const int q = tile_q0(t) + r;
                const int qy = q / WP, qx = q - qy * WP;
                if ((t == MT - 1 && q < 128 * (MT - 1)) || qx >= S) continue;   // not owned, or padding
                float h[C];
#pragma unroll
                for (int o = 0; o < C; o++) h[o] = __uint_as_float(v[o]);
                store_acts(dst + (long)(qy * S + qx) * C, h);
            }
            tc::fence_before();   // the accumulators are read before the next image's MMAs
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

int argus_cnn_dgrad_tc(const float* dh_out, const float* h_out, const void* wbf, void* wpack, int layer, int n,
                       float* dh_in, int num_sms, int* status, cudaStream_t st) {
    cnn_pack_dgrad_tc_kernel<<<num_sms, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(wbf),
                                                       static_cast<__nv_bfloat16*>(wpack), layer); argus_count_launch(1);
    const int smem = (int)sizeof(CnnTcShared);
    cudaError_t e = cudaFuncSetAttribute(cnn_dgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cnn_dgrad_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return argus_cuda_fail(e);
    const int grid = n < 2 * num_sms ? n : 2 * num_sms;
    cnn_dgrad_tc_kernel<<<grid, NTHR, smem, st>>>(dh_out, h_out, static_cast<const uint8_t*>(wpack), dh_in, n, status); argus_count_launch(1);
    return argus_launch_status();
}

int argus_cnn_forward_tc(const float* x, const void* wbf, void* wpack, int n, float* y, float* acts, long lstride,
                         int num_sms, int* status, cudaStream_t st) {
    static_assert(sizeof(__nv_bfloat16) == 2, "BF16 storage");
    cnn_pack_tc_kernel<<<num_sms, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(wbf),
                                                 static_cast<__nv_bfloat16*>(wpack)); argus_count_launch(1);
    const int smem = (int)sizeof(CnnTcShared);
    cudaError_t e = cudaFuncSetAttribute(cnn_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)   // all of the unified L1 / shared storage as shared memory: two CTAs per SM
        e = cudaFuncSetAttribute(cnn_fwd_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return argus_cuda_fail(e);
    const int grid = n < 2 * num_sms ? n : 2 * num_sms;
    cnn_fwd_tc_kernel<<<grid, NTHR, smem, st>>>(x, static_cast<const __nv_bfloat16*>(wbf),
                                                static_cast<const uint8_t*>(wpack), y, acts, lstride, n, status); argus_count_launch(1);
    return argus_launch_status();
}

size_t argus_cnn_tc_pack_bytes() { return (size_t)4 * NTAP * TAPB; }
