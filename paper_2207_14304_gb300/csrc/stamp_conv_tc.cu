// a4 on the tensor cores: the basis convolution of the fit's stamps (the design
// values of the least-squares kernel fit, Sec. 4 difference imaging with the
// Alard-Lupton Gaussian basis),
//
//   X_m(i, j) = sum_{iv, iu} B_m[iv][iu] R(x0 + i + 2r - iu, y0 + j + 2r - iv)
//
// for the 21 x 21 pixels of every stamp and the 21 x 21 taps of each of up to
// 64 basis images, as one implicit GEMM per stamp on tcgen05 (kind::f16: FP16
// hi/lo operands, FP32 accumulation in TMEM).
//
// Implicit GEMM.  The stamp's 41 x 41 window W, flattened row by row
// (W[P] = window(P / 41, P % 41), zero past its 1681 values), is stored as an
// operand plane: plane pixel P, chunk c holds W[P + 8c .. P + 8c + 7] (FP16,
// 16 bytes).  Output q = 41 y + x (y < 21 and every x < 41; x >= 21 is computed
// and discarded) at plane row offset v and tap u reads W[q + 41 v + u] =
// window(y + v, x + u), i.e. basis tap (iv, iu) = (20 - v, 20 - u); the A
// operand of plane row v for 128 consecutive outputs is therefore 128
// consecutive plane pixels, a plain descriptor offset.  K-major core matrices
// are 8 consecutive pixels of one chunk (128 contiguous bytes, SBO = 128); the
// K-group step (LBO) is one chunk plane for taps 0..15 of row v (chunks 0 and
// 1), or 41 pixels for taps 16..23 of rows v and v + 1 in one MMA (chunk 2 of
// pixels q + 41 v and q + 41 (v + 1)), so 21 taps cost 24 and 21 rows 32 K
// steps.  Per stamp: 7 M tiles (q < 896) x 32 K steps x 3 products (hi hi,
// hi lo, lo hi) of M = 128, N = 64 (the basis functions), K = 16.
//
// Precision.  Window values are scaled by a power of two per stamp (largest
// |value| in [2^13, 2^14)) and the basis by one for all images, then split into
// FP16 hi + lo (v = hi + lo + e, |e| <= 2^-22 |v|); the three products leave
// out lo lo only, so each product is the FP32 product to ~2^-21, and the
// accumulators are scaled back exactly.
//
// Roles (480 threads, one CTA per SM, persistent over stamps): warps 0-3 read
// the accumulators (thread = TMEM lane = output row of a tile) and write X;
// warps 4-11 load each stamp's window, find its scale and write the plane (the
// window of the next stamp is loaded while the MMAs of the current one run);
// warp 12 allocates TMEM; one lane each of warps 12 and 14 issues the MMAs of
// tiles 0-3 and 4-6; warp 13 lane 0 streams the packed basis (12 KB per pair of
// plane rows, bulk copies into a ring of four).
// Every wait is bounded; a timeout latches ARGUS_ERR_TIMEOUT and all roles stop.
#include <cuda_fp16.h>

#include "argus_internal.cuh"
#include "split16.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int SCT_ST = 21;                   // stamp side
constexpr int SCT_KS = 21;                   // kernel side
constexpr int SCT_W = SCT_ST + SCT_KS - 1;   // 41: window side
constexpr int SCT_WN = SCT_W * SCT_W;        // 1681 window values
constexpr int SCT_NQ = SCT_ST * SCT_W;       // 861 flattened outputs
constexpr int SCT_MT = 7;                    // M tiles of 128 outputs
constexpr int SCT_NPP = 1760;                // plane pixels: tile rows + 41 (v + 1) < 1760 for v <= 20
constexpr uint32_t SCT_CH = SCT_NPP * 16;    // one chunk plane (bytes)
constexpr uint32_t SCT_PART = 3 * SCT_CH;    // one operand part (hi or lo): 3 chunks
constexpr int SCT_NPAIR = 11;                // pairs of plane rows (row 21 of the last pair is zero)
constexpr uint32_t SCT_KSTEP_B = 2048;       // B of one K step and part: 64 functions x 16 taps
constexpr uint32_t SCT_BSLOT = 3 * 2 * SCT_KSTEP_B;   // B of a pair: 3 K steps x 2 parts
constexpr int SCT_WINF = 1784;               // staged window floats (reads reach W[1759 + 16 + 7])
constexpr int SCT_NPW = 8;                   // producer warps
constexpr int SCT_NPT = SCT_NPW * 32;        // producer threads
constexpr int SCT_NBS = 4;                   // basis ring slots
constexpr int SCT_MMA_WARP = 4 + SCT_NPW, SCT_LOAD_WARP = SCT_MMA_WARP + 1, SCT_MMA_WARP2 = SCT_LOAD_WARP + 1;
constexpr int SCT_THREADS = (SCT_MMA_WARP2 + 1) * 32;
constexpr int SCT_T1 = 4;                    // tiles 0..3 on the first MMA issuer, 4..6 on the second
constexpr uint32_t SCT_TMEM_COLS = 512;      // 7 tiles x 64 columns used
constexpr long long SCT_WAIT = 2000000000LL;   // ~1 s of SM clock
static_assert(SCT_MT * 128 >= SCT_NQ, "the tiles cover every output row");
static_assert((SCT_MT * 128 - 1) + SCT_W * (SCT_KS - 1) + SCT_W < SCT_NPP, "MMA reads stay inside the plane");
static_assert(SCT_NPP - 1 + 16 + 7 < SCT_WINF, "plane writes read inside the staged window");
static_assert(SCT_MT * 64 <= (int)SCT_TMEM_COLS, "accumulators fit the allocation");

struct SctcShared {
    alignas(128) uint8_t plane[2][SCT_PART];        // [hi | lo][chunk][pixel][8 values]
    alignas(128) uint8_t bring[SCT_NBS][SCT_BSLOT];   // [slot][K step][hi | lo][2 KB]
    alignas(16) float win[SCT_WINF];                // the stamp's window, FP32, flattened
    uint64_t pfull, pempty, tfull, tempty, bfull[SCT_NBS], bempty[SCT_NBS], sfull[4];
    float sinv[4];                                  // 1 / (window scale) per stamp slot
    float wmax[SCT_NPW];
    uint32_t tmem;
    int pok;
    int abort;
};

static_assert(sizeof(SctcShared) + 128 <= 227 * 1024, "one CTA's shared memory");

__device__ __forceinline__ bool sct_wait(SctcShared& S, uint64_t* bar, uint32_t parity, int* status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (*(volatile int*)&S.abort) return false;
    if (!tc::mbar_wait_bounded(bar, parity, SCT_WAIT)) {
        S.abort = 1;
        argus_latch(status, ARGUS_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// lane 0 waits, the warp follows (and then observes the phase itself)
__device__ __forceinline__ bool sct_warp_wait(SctcShared& S, uint64_t* bar, uint32_t parity, int* status, int lane) {
    bool ok = true;
    if (lane == 0) ok = sct_wait(S, bar, parity, status);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok)
        while (!tc::mbar_try_wait(bar, parity)) {
        }
    return ok;
}

// Packs the basis images img [nb][21 * 21] (FP32) into the B operands of the 11
// plane-row pairs: pair p, K step ks (0: taps 0..15 of row 2p, 1: of row 2p + 1,
// 2: taps 16..23 of rows 2p and 2p + 1), part (hi, lo), function f, tap index kk
// at p SCT_BSLOT + ks 4096 + part 2048 + (f / 8) 128 + (kk / 8) 1024 + (f % 8) 16 +
// (kk % 8) 2; plane row v, tap u is basis tap (20 - v, 20 - u), zero past the
// image.  One CTA: the scale (a power of two for the largest |value|) first;
// its inverse is stored as a float after the packed operands.
__global__ void __launch_bounds__(1024) stamp_pack_b_kernel(const float* img, int nb, uint8_t* bpack) {
    __shared__ float wmax[32];
    __shared__ float s_scale;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kk2 = SCT_KS * SCT_KS;
    float mx = 0.0f;
    for (int e = tid; e < nb * kk2; e += blockDim.x) {
        const float v = __ldg(img + e);
        if (isfinite(v)) mx = fmaxf(mx, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        float m = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, wmax[w]);
        s_scale = f16_range_scale(m);
        *reinterpret_cast<float*>(bpack + SCT_NPAIR * SCT_BSLOT) = 1.0f / s_scale;
    }
    __syncthreads();
    const float sc = s_scale;
    const int tot = SCT_NPAIR * 3 * 64 * 16;
    for (int e = tid; e < tot; e += blockDim.x) {
        const int kk = e & 15, f = (e >> 4) & 63, ks = (e >> 10) % 3, p = (e >> 10) / 3;
        const int v = ks < 2 ? 2 * p + ks : 2 * p + (kk >> 3);
        const int u = ks < 2 ? kk : 16 + (kk & 7);
        float val = 0.0f;
        if (f < nb && v < SCT_KS && u < SCT_KS) val = __ldg(img + f * kk2 + (SCT_KS - 1 - v) * SCT_KS + (SCT_KS - 1 - u)) * sc;
        const __half hi = __float2half_rn(val);
        const __half lo = __float2half_rn(val - __half2float(hi));
        const uint32_t off = (uint32_t)p * SCT_BSLOT + (uint32_t)ks * 2 * SCT_KSTEP_B + (uint32_t)(f >> 3) * 128 +
                             (uint32_t)(kk >> 3) * 1024 + (uint32_t)(f & 7) * 16 + (uint32_t)(kk & 7) * 2;
        *reinterpret_cast<__half*>(bpack + off) = hi;
        *reinterpret_cast<__half*>(bpack + off + SCT_KSTEP_B) = lo;
    }
}

struct SctcArgs {
    const float* ref;
    long pitch;
    int w, h;
    const int* centers;
    const int* n_stamps;
    int max_stamps;         // capacity of centers and X
    int nb;
    const uint8_t* bpack;   // packed B operands, then the basis scale's inverse
    float* X;               // [stamp][nb][441]
    int* status;
};

__global__ void __launch_bounds__(SCT_THREADS, 1) stamp_conv_tc_kernel(SctcArgs a) {
    extern __shared__ __align__(128) uint8_t sct_smem_raw[];
    SctcShared& S = *reinterpret_cast<SctcShared*>(sct_smem_raw + ((128 - (tc::smem_u32(sct_smem_raw) & 127)) & 127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int* status = a.status;
    const int ns = min(*a.n_stamps, a.max_stamps);
    const int nk = (int)blockIdx.x < ns ? (ns - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    for (int e = tid; e < SCT_WINF; e += SCT_THREADS) S.win[e] = 0.0f;
    if (tid == 0) {
        tc::mbar_init(&S.pfull, SCT_NPW);   // the producer warps' lane 0
        tc::mbar_init(&S.pempty, 2);    // both MMA issuers' commits
        tc::mbar_init(&S.tfull, 2);     // both MMA issuers' commits
        tc::mbar_init(&S.tempty, 4);    // the four accumulator-reading warps
        for (int i = 0; i < SCT_NBS; i++) {
            tc::mbar_init(&S.bfull[i], 1);    // the loader's expect_tx arrival (+ the copy's bytes)
            tc::mbar_init(&S.bempty[i], 2);   // both MMA issuers' commits
        }
        for (int i = 0; i < 4; i++) tc::mbar_init(&S.sfull[i], 1);
        S.abort = 0;
        S.pok = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == SCT_MMA_WARP) tc::tmem_alloc(&S.tmem, SCT_TMEM_COLS);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;

    if (warp >= 4 && warp < 4 + SCT_NPW) {
        // ---------------- producers: window, scale, plane
        const int ptid = tid - 128, pw = warp - 4;   // 0 .. SCT_NPT - 1, 0 .. SCT_NPW - 1
        for (int k = 0; k < nk; k++) {
            const int s = (int)blockIdx.x + k * (int)gridDim.x;
            tc::named_sync(1, SCT_NPT);   // every producer is done reading the previous window
            const int xs = __ldg(a.centers + 2 * s), ys = __ldg(a.centers + 2 * s + 1);
            const int x0 = xs - SCT_ST / 2 - (SCT_KS - 1) / 2, y0 = ys - SCT_ST / 2 - (SCT_KS - 1) / 2;
            const bool valid = x0 >= 0 && y0 >= 0 && x0 + SCT_W - 1 <= a.w - 1 && y0 + SCT_W - 1 <= a.h - 1;
            float mx = 0.0f;
            for (int e = ptid; e < SCT_WN; e += SCT_NPT) {
                const int wy = e / SCT_W, wx = e - wy * SCT_W;
                const float v = valid ? __ldg(a.ref + (long)(y0 + wy) * a.pitch + (x0 + wx)) : 0.0f;
                S.win[e] = v;
                if (isfinite(v)) mx = fmaxf(mx, fabsf(v));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) S.wmax[pw] = mx;
            tc::named_sync(1, SCT_NPT);
            float wm = S.wmax[0];
#pragma unroll
            for (int i = 1; i < SCT_NPW; i++) wm = fmaxf(wm, S.wmax[i]);
            const float sc = f16_range_scale(wm);
            if (ptid == 0) {
                // the epilogue of stamp k - 4 read this slot before the MMAs of stamp k - 2
                // began, and those finished before the plane of stamp k - 1 was written
                S.sinv[k & 3] = 1.0f / sc;
                tc::mbar_arrive(&S.sfull[k & 3]);
                // the MMAs of the previous stamp are done with the plane
                S.pok = k == 0 || sct_wait(S, &S.pempty, (uint32_t)(k - 1) & 1u, status);
            }
            tc::named_sync(1, SCT_NPT);
            if (!S.pok) break;
            if (k > 0)
                while (!tc::mbar_try_wait(&S.pempty, (uint32_t)(k - 1) & 1u)) {
                }
            // plane pixel P, chunk c: W[P + 8c .. P + 8c + 7] scaled, as FP16 hi and lo
            for (int e = ptid; e < 3 * SCT_NPP; e += SCT_NPT) {
                const int c = e / SCT_NPP, P = e - c * SCT_NPP;
                const float* src = S.win + P + 8 * c;
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const float v0 = src[2 * t] * sc, v1 = src[2 * t + 1] * sc;
                    hi[t] = f16x2_rn(v0, v1);
                    lo[t] = f16x2_rn(v0 - f16_lo(hi[t]), v1 - f16_hi(hi[t]));
                }
                const uint32_t off = (uint32_t)c * SCT_CH + (uint32_t)P * 16;
                *reinterpret_cast<uint4*>(S.plane[0] + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4*>(S.plane[1] + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.pfull);
        }
    } else if (warp == SCT_MMA_WARP || warp == SCT_MMA_WARP2) {
        // ---------------- MMA issuers: one lane of each issues the MMAs of its tiles
        // (a thread that issues an MMA waits for it to be accepted; two issuers keep the
        // narrow MMAs of the two tile sets in flight together)
        const int t0 = warp == SCT_MMA_WARP ? 0 : SCT_T1, t1 = warp == SCT_MMA_WARP ? SCT_T1 : SCT_MT;
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(0, 128, 64);   // FP16 operands, FP32 accumulate
            const uint32_t phi = tc::smem_u32(S.plane[0]), plo = tc::smem_u32(S.plane[1]);
            const uint32_t b0 = tc::smem_u32(S.bring[0]);
            // descriptors at the operands' origins; an operand at a byte offset o is the
            // origin's descriptor plus o / 16 (the start-address field, which the offsets
            // keep below 2^14)
            const uint64_t a01h = tc::smem_desc(phi, SCT_CH, 128), a01l = tc::smem_desc(plo, SCT_CH, 128);
            const uint64_t a2h = tc::smem_desc(phi + 2 * SCT_CH, SCT_W * 16, 128);
            const uint64_t a2l = tc::smem_desc(plo + 2 * SCT_CH, SCT_W * 16, 128);
            const uint64_t bh0 = tc::smem_desc(b0, 1024, 128), bl0 = tc::smem_desc(b0 + SCT_KSTEP_B, 1024, 128);
            int ncommit = 0;        // tfull commits
            bool pending = false;   // MMAs issued since the last tfull commit
            bool run = true;
            for (int k = 0; k < nk && run; k++) {
                if (k > 0 && !sct_wait(S, &S.tempty, (uint32_t)(k - 1) & 1u, status)) break;
                if (!sct_wait(S, &S.pfull, (uint32_t)k & 1u, status)) break;
                tc::fence_after();
                for (int p = 0; p < SCT_NPAIR; p++) {
                    const int g = k * SCT_NPAIR + p;
                    if (!sct_wait(S, &S.bfull[g % SCT_NBS], (uint32_t)(g / SCT_NBS) & 1u, status)) { run = false; break; }
                    tc::fence_after();
                    const uint64_t bso = (uint64_t)((g % SCT_NBS) * (SCT_BSLOT / 16));
                    const uint64_t row = (uint64_t)(SCT_W * 2 * p);          // plane pixel of row 2p (16-byte units)
                    const bool last = p == SCT_NPAIR - 1;                    // plane row 21 is zero
                    for (int t = t0; t < t1; t++) {
                        const uint32_t d = tmem + (uint32_t)(t * 64);
                        const uint64_t q0 = 128u * (uint64_t)t + row;
                        // taps 0..15 of row 2p, of row 2p + 1, then taps 16..23 of both
                        tc::mma_bf16(d, a01h + q0, bh0 + bso, idesc, p == 0 ? 0u : 1u);
                        tc::mma_bf16(d, a01h + q0, bl0 + bso, idesc, 1u);
                        tc::mma_bf16(d, a01l + q0, bh0 + bso, idesc, 1u);
                        if (!last) {
                            tc::mma_bf16(d, a01h + q0 + SCT_W, bh0 + bso + 256, idesc, 1u);
                            tc::mma_bf16(d, a01h + q0 + SCT_W, bl0 + bso + 256, idesc, 1u);
                            tc::mma_bf16(d, a01l + q0 + SCT_W, bh0 + bso + 256, idesc, 1u);
                        }
                        tc::mma_bf16(d, a2h + q0, bh0 + bso + 512, idesc, 1u);
                        tc::mma_bf16(d, a2h + q0, bl0 + bso + 512, idesc, 1u);
                        tc::mma_bf16(d, a2l + q0, bh0 + bso + 512, idesc, 1u);
                    }
                    pending = true;
                    tc::commit(&S.bempty[g % SCT_NBS]);
                }
                if (!run) break;
                tc::commit(&S.pempty);
                tc::commit(&S.tfull);
                ncommit++;
                pending = false;
            }
            // every issued MMA lands before TMEM is released (after an abort the
            // partial stamp's MMAs are committed too; its results are not used)
            if (pending) {
                tc::commit(&S.tfull);
                ncommit++;
            }
            if (ncommit > 0 && !tc::mbar_wait_bounded(&S.tfull, (uint32_t)(ncommit - 1) & 1u, SCT_WAIT)) {
                S.abort = 1;
                argus_latch(status, ARGUS_ERR_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp == SCT_LOAD_WARP) {
        // ---------------- basis loader: the same 11 pair slices for every stamp
        if (lane == 0) {
            const int G = nk * SCT_NPAIR;
            int g = 0;
            for (; g < G; g++) {
                const int sl = g % SCT_NBS;
                if (g >= SCT_NBS && !sct_wait(S, &S.bempty[sl], (uint32_t)(g / SCT_NBS - 1) & 1u, status)) break;
                tc::mbar_arrive_expect_tx(&S.bfull[sl], SCT_BSLOT);
                tc::bulk_g2s(S.bring[sl], a.bpack + (size_t)(g % SCT_NPAIR) * SCT_BSLOT, SCT_BSLOT, &S.bfull[sl]);
            }
            // copies in flight land before the CTA exits
            for (int q = g - SCT_NBS < 0 ? 0 : g - SCT_NBS; q < g; q++)
                if (!tc::mbar_wait_bounded(&S.bfull[q % SCT_NBS], (uint32_t)(q / SCT_NBS) & 1u, SCT_WAIT)) {
                    S.abort = 1;
                    argus_latch(status, ARGUS_ERR_TIMEOUT);
                }
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------- accumulator readers: thread = output row r of every tile
        const float binv = *reinterpret_cast<const float*>(a.bpack + SCT_NPAIR * SCT_BSLOT);
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        const int r = tid;
        const int nb = a.nb;
        for (int k = 0; k < nk; k++) {
            const int s = (int)blockIdx.x + k * (int)gridDim.x;
            if (!sct_warp_wait(S, &S.sfull[k & 3], (uint32_t)(k >> 2) & 1u, status, lane)) break;
            const float inv = S.sinv[k & 3] * binv;
            bool ok = true;
            if (lane == 0) ok = sct_wait(S, &S.tfull, (uint32_t)k & 1u, status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc::fence_after();
            float* Xs = a.X + (size_t)s * nb * (SCT_ST * SCT_ST);
            for (int t = 0; t < SCT_MT; t++) {
                uint32_t v0[32], v1[32];
                tc::tmem_ld32_nowait(tl + (uint32_t)(t * 64), v0);
                tc::tmem_ld32_nowait(tl + (uint32_t)(t * 64 + 32), v1);
                tc::tmem_wait_ld32(v0);
                tc::tmem_wait_ld32(v1);
                const int q = 128 * t + r, y = q / SCT_W, x = q - y * SCT_W;
                if (y < SCT_ST && x < SCT_ST) {
                    float* xp = Xs + y * SCT_ST + x;
#pragma unroll
                    for (int m = 0; m < 32; m++)
                        if (m < nb) xp[(size_t)m * (SCT_ST * SCT_ST)] = __uint_as_float(v0[m]) * inv;
#pragma unroll
                    for (int m = 0; m < 32; m++)
                        if (m + 32 < nb) xp[(size_t)(m + 32) * (SCT_ST * SCT_ST)] = __uint_as_float(v1[m]) * inv;
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.tempty);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == SCT_MMA_WARP) tc::tmem_dealloc(tmem, SCT_TMEM_COLS);
}

}  // namespace

size_t argus_stamp_conv_tc_bytes() { return (size_t)SCT_NPAIR * SCT_BSLOT + 16; }

int argus_stamp_conv_tc(const float* ref, long pitch, int w, int h, const int* centers, const int* n_stamps,
                        int max_stamps, const float* img, int nb, uint8_t* bpack, float* X, int num_sms, int* status,
                        cudaStream_t st) {
    if (nb < 1 || nb > 64 || max_stamps < 1) return ARGUS_ERR_ARG;
    stamp_pack_b_kernel<<<1, 1024, 0, st>>>(img, nb, bpack); argus_count_launch(1);
    const size_t smem = sizeof(SctcShared) + 128;
    const cudaError_t e = cudaFuncSetAttribute(stamp_conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return argus_cuda_fail(e);
    SctcArgs a;
    a.ref = ref; a.pitch = pitch; a.w = w; a.h = h; a.centers = centers; a.n_stamps = n_stamps; a.max_stamps = max_stamps; a.nb = nb;
    a.bpack = bpack; a.X = X; a.status = status;
    const int grid = max_stamps < num_sms ? max_stamps : num_sms;
    stamp_conv_tc_kernel<<<grid, SCT_THREADS, smem, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}
