// K8 fit on the tensor cores: the per-segment least-squares fit of the batched
// segments (paper Sec. 5, subtraction parallelised at the segment level; Sec.
// 4.1.1 HEALPix segments), for kernels of side KS <= 15 (one K = 16 MMA per
// source row).  For every interior pixel the design row is
//   Z = sqrt(w) [X_0 .. X_{nb-1}, 1, I],  X_m(x, y) = sum_{iu,iv} B'_m[iv][iu] R(x - iu + r, y - iv + r)
// (B'_m the orthonormalised basis images, w = 1 / V_I where the pixel is
// valid), and the segment's normal matrix is sum Z^T Z over its interior.
//
// Work item: a strip of 128 interior columns x a band of `band` interior rows
// of one segment; persistent CTAs (one per SM) take contiguous ranges of the
// item list of equal numbers of row pairs; a segment's items are consecutive,
// so a CTA adds its Gram blocks to the segment's normal matrix only when the
// segment changes.  The
// convolutions are tcgen05 MMAs of M = 128 pixels, N = 128, K = 16 taps: for
// output rows y, y + 1 (a pair) and source row rho = y - r .. y + 1 + r,
//   T[m][(h, f)] += sum_u A_rho[m][u] Bz[iv0 + 1 + h][f][u],  iv0 = y + r - rho,
// A_rho[m][u] = R(x0 + m - r + u, rho) (a Hankel matrix: 17 distinct core
// matrices, written once per source row into a ring the pairs share; each row
// feeds eight pairs), Bz[s][f][u] = B'_f[s - 1][KS - 1 - u] for 1 <= s <= KS
// and zero for s = 0, KS + 1: columns f of the accumulator are row y (h = 0)
// and columns 64 + f row y + 1 (h = 1), and every (pair, source row) is one
// descriptor offset of 2048 bytes into the one stored Bz.  R and Bz are split
// into FP16 hi + lo with three products (hi hi + hi lo + lo hi, FP32 in TMEM):
// 11-bit parts keep the convolution within about 2^-22 of its terms, FP32
// level.  (BF16 parts, 2^-16, moved the fitted kernels of ill-conditioned
// segments by up to 7e-4 of max |K|; the normal matrices of single segments
// amplify design errors.)  FP16 needs range: each segment's R is scaled by a
// power of two that puts its largest |R| at 2^14 (a pass before the fit), the
// basis by one that puts max |B'| at 2^14, and the accumulators are scaled back
// exactly.
//
// The normal matrix stays on the CUDA cores in the fold the precision needs:
// FP32 sums over 8 pixels, each folded into a double-float accumulator
// (error-free two-sum; sums over 16 and 32 pixels measured 1.8x and 2.1x the
// kernel error).  The design rows of a pair are stored pixel-pair interleaved
// and the arithmetic is on packed FP32 pairs (fma/add/sub.rn.f32x2): the two
// lanes of a register hold an even and an odd pixel, so each lane still sums
// 8 pixels per fold while one instruction does two of the operations.  Each
// thread owns a 2 x 4 block of the upper triangle of the (nb + 2)^2 Gram; when
// the CTA's next item belongs to another segment the blocks go to the
// segment's FP64 normal matrix by atomics.
//
// Roles (16 warps): warps 0-3 read the accumulators (thread = pixel, the TMEM
// lane), weight them and write the design rows of the pair (256 pixels) to
// shared memory; warps 4-6 stage the source rows (16-byte cp.async, zero past
// the segment) and write the A operands; warp 7 issues the MMAs; warps 8-15
// and, once the rows are written, warps 0-3 sum the Gram: two sets of 192
// threads (the 182 blocks of a 51-column Gram), one per row of the pair.  Two
// TMEM accumulators let the MMAs of one pair run while the previous one is read.
// Every wait is bounded; a timeout latches ARGUS_ERR_TIMEOUT and all roles stop.
#include <cuda_fp16.h>

#include "segments_fit.cuh"
#include "split16.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int FT_WARPS = 16;
constexpr int FT_THREADS = FT_WARPS * 32;
constexpr int FT_NPROD = 3;                       // producer warps (4..6)
constexpr int FT_MMA_WARP = 7;
constexpr int FT_GRAM_WARP = 8;                   // warps 8..15
constexpr int FT_NA = 20;                         // A ring slots (source rows; a pair holds 16)
constexpr int FT_NCM = 17;                        // distinct core matrices of a Hankel operand (M 128, K 16)
constexpr uint32_t FT_A_BYTES = FT_NCM * 128;     // one part (hi or lo) of one source row
constexpr int FT_WIN = FT_NCM * 8 + 8;            // staged values of a source row (x0 - r .. + 143)
constexpr int FT_LA = 3;                          // rows a producer warp stages ahead
constexpr int FT_NWIN = 4;                        // its staging slots (> FT_LA)
constexpr uint32_t FT_BZ_SLOT = 64 * 16 * 2;      // one kernel-row slot of Bz: 64 functions x 16 taps, FP16
constexpr uint32_t FT_SBO_B = 256, FT_LBO = 128, FT_SBO_A = 128;
constexpr long long FT_WAIT = 2000000000LL;       // ~1 s of SM clock
static_assert(FT_WIN % 4 == 0 && FT_WIN / 4 <= 64, "two 16-byte chunks per lane at most");

struct FtBar {
    uint64_t afull[FT_NA], aempty[FT_NA], tfull[2], tempty[2], zfull, zempty;
    uint32_t tmem;
    int abort;
    float bscale;   // power of two: max |B'| bscale = 2^14
};

// Shared memory: Bz (hi, lo) | A ring | staged windows | row buffers | Z | barriers.
struct FtLayout {
    uint32_t bz, a, win, rowb, z, bar, total;
};

__host__ __device__ inline FtLayout ft_layout(int ks, int zs) {
    FtLayout L;
    uint32_t o = 0;
    L.bz = o; o += 2 * (uint32_t)(ks + 2) * FT_BZ_SLOT;
    L.a = o; o += FT_NA * 2 * FT_A_BYTES;
    L.win = o; o += FT_NPROD * FT_NWIN * FT_WIN * 4;
    L.rowb = o; o += FT_NPROD * 2 * (FT_NCM + 1) * 4 * 4;
    L.z = o; o += 256 * (uint32_t)zs * 4;
    o = (o + 15) & ~15u;
    L.bar = o; o += (uint32_t)sizeof(FtBar);
    L.total = o;
    return L;
}

// Packed FP32 pairs (two lanes of one 64-bit register), round to nearest.
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float f2_x(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_y(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

__device__ __forceinline__ bool ft_wait(FtBar& S, uint64_t* bar, uint32_t parity, int* status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (S.abort) return false;
    if (!tc::mbar_wait_bounded(bar, parity, FT_WAIT)) {
        S.abort = 1;
        argus_latch(status, ARGUS_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// lane 0 waits, the warp follows (and then observes the phase itself)
__device__ __forceinline__ bool ft_warp_wait(FtBar& S, uint64_t* bar, uint32_t parity, int* status, int lane) {
    bool ok = true;
    if (lane == 0) ok = ft_wait(S, bar, parity, status);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok)
        while (!tc::mbar_try_wait(bar, parity)) {
        }
    return ok;
}

struct FtItem {
    int s, x0, y0, cols, rows, pairs, nsrc, side;
    long base;   // atlas offset of the segment's pixel (0, 0)
};

template <int KS>
__device__ __forceinline__ FtItem ft_item(const SegFitTcArgs& a, int item) {
    constexpr int R = (KS - 1) / 2;
    FtItem t;
    const int4 it = a.items[item];
    t.s = it.x;
    t.x0 = it.y;
    t.y0 = it.z;
    const int4 sg = a.seg[t.s];
    t.side = sg.y;
    t.base = (long)sg.x * a.pitch + sg.z;
    t.cols = min(128, t.side - R - t.x0);
    t.rows = min(a.band, t.side - R - t.y0);
    t.pairs = (t.rows + 1) / 2;
    t.nsrc = 2 * t.pairs + 2 * R;
    return t;
}

// One thread's share of the Gram of a pair's 256 design rows, stored pixel-pair
// interleaved (Z [128 pixel pairs][zs][2]): the 2 x 4 block bidx (rows 2 bi, 2 bi + 1,
// columns 4 bj .. 4 bj + 3) of the upper triangle of the NPC x NPC matrix, over the
// pixel pairs of one half of the pair (two sets of 192 threads).  Arithmetic on packed
// FP32 pairs: the two lanes of every accumulator sum the even and the odd pixel of the
// pixel pairs, 8 pixels each per fold group (8 pixel pairs), each group folded into
// (hi, lo) by an error-free two-sum.
struct GramShare {
    int bi, bj, half;
    bool active;
    uint64_t hi[8], lo[8];
    __device__ __forceinline__ void init(int bidx, int half_, int NPC) {
        const int nbi = (NPC + 1) / 2, nbj = (NPC + 3) / 4;
        half = half_;
        active = false;
        bi = bj = 0;
        int rem = bidx;
        for (int c = 0; c < nbj; c++) {   // column block c holds row blocks 0 .. min(nbi - 1, (4c + 3) / 2)
            const int nr = min(nbi - 1, (4 * c + 3) / 2) + 1;
            if (rem < nr) { bi = rem; bj = c; active = true; break; }
            rem -= nr;
        }
#pragma unroll
        for (int q = 0; q < 8; q++) hi[q] = lo[q] = 0ull;
    }
    __device__ __forceinline__ void add(const float* Z, int zs) {
        if (!active) return;
        for (int g = 0; g < 8; g++) {
            uint64_t acc[8];
#pragma unroll
            for (int q = 0; q < 8; q++) acc[q] = 0ull;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const float* zp = Z + (size_t)(half * 64 + g * 8 + k) * zs * 2;
                const ulonglong2 i01 = *reinterpret_cast<const ulonglong2*>(zp + 4 * bi);
                const ulonglong2 j01 = *reinterpret_cast<const ulonglong2*>(zp + 8 * bj);
                const ulonglong2 j23 = *reinterpret_cast<const ulonglong2*>(zp + 8 * bj + 4);
                const uint64_t ai[2] = {i01.x, i01.y}, aj[4] = {j01.x, j01.y, j23.x, j23.y};
#pragma unroll
                for (int u = 0; u < 2; u++)
#pragma unroll
                    for (int v = 0; v < 4; v++) acc[u * 4 + v] = f2_fma(ai[u], aj[v], acc[u * 4 + v]);
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint64_t sum = f2_add(hi[q], acc[q]), bp = f2_sub(sum, hi[q]);
                lo[q] = f2_add(lo[q], f2_add(f2_sub(hi[q], f2_sub(sum, bp)), f2_sub(acc[q], bp)));
                hi[q] = sum;
            }
        }
    }
    // add the block to the segment's FP64 normal matrix (upper triangle) and restart
    __device__ __forceinline__ void flush(double* G, int NPC) {
        if (!active) return;
#pragma unroll
        for (int u = 0; u < 2; u++)
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int i = bi * 2 + u, j = bj * 4 + v, q = u * 4 + v;
                if (i < NPC && j < NPC && i <= j)
                    atomicAdd(G + i * NPC + j, ((double)f2_x(hi[q]) + (double)f2_x(lo[q])) +
                                                   ((double)f2_y(hi[q]) + (double)f2_y(lo[q])));
            }
#pragma unroll
        for (int q = 0; q < 8; q++) hi[q] = lo[q] = 0ull;
    }
};

template <int KS>
__global__ void __launch_bounds__(FT_THREADS, 1) seg_fit_tc_kernel(SegFitTcArgs a) {
    constexpr int R = (KS - 1) / 2;
    static_assert(KS <= 16, "one K = 16 MMA per source row");
    extern __shared__ __align__(1024) uint8_t ft_smem_raw[];
    uint8_t* sm = ft_smem_raw + ((1024 - (tc::smem_u32(ft_smem_raw) & 1023)) & 1023);
    const int nb = a.nb, NPC = a.NPC, zs = (NPC + 3) & ~3;
    const FtLayout L = ft_layout(KS, zs);
    uint8_t* bz = sm + L.bz;                        // [2 parts][KS + 2 slots][64 f][16 u], canonical K-major
    uint8_t* aring = sm + L.a;                      // [FT_NA][2 parts][FT_A_BYTES]
    float* win = reinterpret_cast<float*>(sm + L.win);          // [FT_NPROD][FT_NWIN][FT_WIN]
    uint32_t* rowb = reinterpret_cast<uint32_t*>(sm + L.rowb);  // [FT_NPROD][2][(FT_NCM + 1) * 4]
    float* Z = reinterpret_cast<float*>(sm + L.z);               // [128 pixel pairs][zs][2]
    FtBar& S = *reinterpret_cast<FtBar*>(sm + L.bar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int* status = a.status;
    // this CTA's items: [ilo, ihi), cut by row pairs (the unit of cost)
    const int ilo = a.cta_start[blockIdx.x], ihi = a.cta_start[blockIdx.x + 1];

    // ---- the basis scale (a CTA-wide max of |B'|), then Bz: slot s (kernel row s - 1),
    // N-row n = s 64 + f, tap u: B'_f[s - 1][KS - 1 - u] bscale
    constexpr int NSLOT = KS + 2;
    {
        __shared__ float wmax[FT_WARPS];
        float mx = 0.0f;
        for (int e = tid; e < nb * KS * KS; e += FT_THREADS) mx = fmaxf(mx, fabsf(__ldg(a.bimg + e)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) wmax[warp] = mx;
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < FT_WARPS; w++) mx = fmaxf(mx, wmax[w]);
            S.bscale = f16_range_scale(wmax[0] > mx ? wmax[0] : mx);
        }
        __syncthreads();
    }
    const float bscale = S.bscale;
    for (int e = tid; e < NSLOT * 64 * 16; e += FT_THREADS) {
        const int sl = e / 1024, r = e - sl * 1024, f = r >> 4, u = r & 15;
        const int iv = sl - 1;
        float v = 0.0f;
        if (iv >= 0 && iv < KS && f < nb && u < KS)
            v = __ldg(a.bimg + (long)f * KS * KS + iv * KS + (KS - 1 - u)) * bscale;
        const __half hi = __float2half_rn(v);
        const __half lo = __float2half_rn(v - __half2float(hi));
        const int n = sl * 64 + f;
        const uint32_t off = (uint32_t)(n >> 3) * FT_SBO_B + (uint32_t)(u >> 3) * FT_LBO + (uint32_t)(n & 7) * 16 +
                             (uint32_t)(u & 7) * 2;
        *reinterpret_cast<__half*>(bz + off) = hi;
        *reinterpret_cast<__half*>(bz + NSLOT * FT_BZ_SLOT + off) = lo;
    }
    if (tid == 0) {
        for (int i = 0; i < FT_NA; i++) {
            tc::mbar_init(&S.afull[i], 1);    // the producing warp's lane 0
            tc::mbar_init(&S.aempty[i], 1);   // an MMA commit
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&S.tfull[b], 1);
            tc::mbar_init(&S.tempty[b], 4);   // the four accumulator-reading warps
        }
        tc::mbar_init(&S.zfull, 4);
        tc::mbar_init(&S.zempty, FT_WARPS - FT_GRAM_WARP + 4);   // the Gram warps and the readers
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, 256);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;

    if (warp >= 4 && warp < 4 + FT_NPROD) {
        // ---------------- producers: source row g (global over this CTA's items) belongs to
        // warp 4 + g mod 3; the warp stages its rows FT_LA ahead of the one it writes
        const int pw = warp - 4;
        float* wbase = win + pw * FT_NWIN * FT_WIN;
        uint32_t* rb = rowb + pw * 2 * (FT_NCM + 1) * 4;
        // cursor over this warp's rows: item, row within the item, global row index
        struct Cur { int item, j, g; FtItem t; };
        auto first = [&](Cur& c) {
            c.item = ilo; c.j = 0; c.g = 0;
            if (c.item < ihi) c.t = ft_item<KS>(a, c.item);
            // advance to the warp's first row
            while (c.item < ihi && (c.g % FT_NPROD) != pw) {
                c.g++;
                if (++c.j == c.t.nsrc) { c.j = 0; c.item++; if (c.item < ihi) c.t = ft_item<KS>(a, c.item); }
            }
        };
        auto next = [&](Cur& c) {
            for (int k = 0; k < FT_NPROD && c.item < ihi; k++) {
                c.g++;
                if (++c.j == c.t.nsrc) { c.j = 0; c.item++; if (c.item < ihi) c.t = ft_item<KS>(a, c.item); }
            }
        };
        // stage row c (one cp.async group, empty past the last row) into window slot q
        auto stage = [&](const Cur& c, int q) {
            if (c.item < ihi) {
                const int rho = c.t.y0 - R + c.j;                 // segment row
                const int XS = c.t.x0 - R;                        // segment column of window value 0 (a multiple of 4)
                float* dst = wbase + (q % FT_NWIN) * FT_WIN;
                for (int ch = lane; ch < FT_WIN / 4; ch += 32) {
                    const int X = XS + 4 * ch;
                    const int nbytes = (rho < c.t.side && X < c.t.side) ? 4 * min(4, c.t.side - X) : 0;
                    tc::cp_async16(dst + 4 * ch, nbytes ? a.ref + c.t.base + (long)rho * a.pitch + X : a.ref, nbytes);
                }
            }
            tc::cp_async_commit();
        };
        Cur cw, ci;
        first(cw);
        ci = cw;
        for (int k = 0; k < FT_LA; k++) {
            stage(ci, k);
            next(ci);
        }
        bool run = true;
        for (int q = 0; cw.item < ihi && run; q++) {
            stage(ci, q + FT_LA);
            next(ci);
            const int g = cw.g, sl = g % FT_NA;
            bool ok = true;
            if (lane == 0 && g >= FT_NA) ok = ft_wait(S, &S.aempty[sl], (uint32_t)(g / FT_NA - 1) & 1u, status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) { run = false; break; }
            tc::cp_async_wait<FT_LA>();
            __syncwarp();
            // round the row once (value pairs by consecutive lanes, scaled by the segment's
            // power of two), then the operand rows: row t holds values t .. t + 7
            const float* src = wbase + (q % FT_NWIN) * FT_WIN;
            const float rs = __ldg(a.rscale + cw.t.s);
#pragma unroll
            for (int p = lane; p < 4 * (FT_NCM + 1); p += 32) {
                const float v0 = src[2 * p] * rs, v1 = src[2 * p + 1] * rs;
                const uint32_t h = f16x2_rn(v0, v1);
                rb[p] = h;
                rb[4 * (FT_NCM + 1) + p] = f16x2_rn(v0 - f16_lo(h), v1 - f16_hi(h));
            }
            __syncwarp();
            uint8_t* dst = aring + (uint32_t)sl * 2 * FT_A_BYTES;
            const int A = lane & 7;
            const uint32_t sel = (A & 1) ? 0x5432u : 0x3210u;
#pragma unroll
            for (int rr = 0; rr * 32 < FT_NCM * 8; rr++) {
                const int t = lane + 32 * rr;
                if (t < FT_NCM * 8) {
                    const int wb = 4 * (t >> 3) + (A >> 1);
#pragma unroll
                    for (int pt = 0; pt < 2; pt++) {
                        const uint32_t* w = rb + pt * 4 * (FT_NCM + 1);
                        uint32_t wv[5];
#pragma unroll
                        for (int k = 0; k < 5; k++) wv[k] = w[wb + k];
                        *reinterpret_cast<uint4*>(dst + pt * FT_A_BYTES + 16 * t) =
                            make_uint4(__byte_perm(wv[0], wv[1], sel), __byte_perm(wv[1], wv[2], sel),
                                       __byte_perm(wv[2], wv[3], sel), __byte_perm(wv[3], wv[4], sel));
                    }
                }
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.afull[sl]);
            next(cw);
        }
        tc::cp_async_wait<0>();
        __syncwarp();
    } else if (warp == FT_MMA_WARP) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(0, 128, 128);   // FP16 operands, FP32 accumulate
            const uint32_t bz_hi = tc::smem_u32(bz), bz_lo = bz_hi + NSLOT * FT_BZ_SLOT;
            const uint32_t a0 = tc::smem_u32(aring);
            int g0 = 0, tp = 0, issued = -1;
            int seen = -1;   // source rows up to this one are known to be written (a row stays
                             // written until its last pair's MMAs release it)
            bool run = true;
            for (int item = ilo; item < ihi && run; item++) {
                const FtItem t = ft_item<KS>(a, item);
                for (int p = 0; p < t.pairs && run; p++, tp++) {
                    const int acc = tp & 1;
                    if (tp >= 2 && !ft_wait(S, &S.tempty[acc], (uint32_t)(tp / 2 - 1) & 1u, status)) { run = false; break; }
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * 128);
                    for (int i = 0; i < 2 * R + 2; i++) {
                        const int g = g0 + 2 * p + i, sl = g % FT_NA;
                        if (g > seen) {
                            if (!ft_wait(S, &S.afull[sl], (uint32_t)(g / FT_NA) & 1u, status)) { run = false; break; }
                            seen = g;
                            tc::fence_after();
                        }
                        const uint32_t boff = (uint32_t)(2 * R - i + 1) * (64 / 8) * FT_SBO_B;   // slot iv0 + 1
                        const uint32_t ahi = a0 + (uint32_t)sl * 2 * FT_A_BYTES, alo = ahi + FT_A_BYTES;
                        const uint64_t dah = tc::smem_desc(ahi, FT_LBO, FT_SBO_A), dal = tc::smem_desc(alo, FT_LBO, FT_SBO_A);
                        const uint64_t dbh = tc::smem_desc(bz_hi + boff, FT_LBO, FT_SBO_B);
                        const uint64_t dbl = tc::smem_desc(bz_lo + boff, FT_LBO, FT_SBO_B);
                        tc::mma_bf16(d, dah, dbh, idesc, i ? 1u : 0u);
                        tc::mma_bf16(d, dah, dbl, idesc, 1u);
                        tc::mma_bf16(d, dal, dbh, idesc, 1u);
                    }
                    if (!run) break;
                    tc::commit(&S.tfull[acc]);
                    issued = tp;
                    // source rows no later pair of the item reads
                    const int nrel = p + 1 < t.pairs ? 2 : 2 * R + 2;
                    for (int i = 0; i < nrel; i++) tc::commit(&S.aempty[(g0 + 2 * p + i) % FT_NA]);
                }
                g0 += t.nsrc;
            }
            if (issued >= 0 && !tc::mbar_wait_bounded(&S.tfull[issued & 1], (uint32_t)(issued / 2) & 1u, FT_WAIT)) {
                S.abort = 1;
                argus_latch(status, ARGUS_ERR_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------- accumulator readers: thread = pixel column x0 + tid of the strip
        const int m = tid;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        GramShare gs;   // Gram threads 0 .. 127 of 384: set 0 (with Gram warps 8 and 9)
        gs.init(tid, 0, NPC);
        int tp = 0;
        bool run = true;
        for (int item = ilo; item < ihi && run; item++) {
            const FtItem t = ft_item<KS>(a, item);
            int nvalid = 0;
            // the pixel's variance, value and flag in the pair's two rows (read one pair ahead,
            // before this set's Gram share, so that the loads overlap it)
            float pv[2], pi[2];
            uint32_t pf[2];
            auto fetch = [&](int p) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    pv[h] = 0.0f; pi[h] = 0.0f; pf[h] = 1u;
                    if (m < t.cols && 2 * p + h < t.rows) {
                        const long q = t.base + (long)(t.y0 + 2 * p + h) * a.pitch + (t.x0 + m);
                        pv[h] = __ldg(a.var + q);
                        pi[h] = __ldg(a.sci + q);
                        pf[h] = __ldg(a.flags + q);
                    }
                }
            };
            fetch(0);
            for (int p = 0; p < t.pairs; p++, tp++) {
                float sqw[2], Iv[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    sqw[h] = 0.0f;
                    Iv[h] = 0.0f;
                    if (pf[h] == 0 && pv[h] > 0.0f && isfinite(pv[h]) && isfinite(pi[h])) {
                        sqw[h] = sqrtf(1.0f / pv[h]);
                        Iv[h] = pi[h];
                        nvalid++;
                    }
                }
                // the accumulators hold X rscale bscale (powers of two): scaled back exactly
                // with the weight
                const float unscale = 1.0f / (__ldg(a.rscale + t.s) * bscale);
                const float wx[2] = {sqw[0] * unscale, sqw[1] * unscale};
                const int acc = tp & 1;
                bool ok = true;
                if (lane == 0) ok = ft_wait(S, &S.tfull[acc], (uint32_t)(tp / 2) & 1u, status);
                if (ok && lane == 0 && tp >= 1) ok = ft_wait(S, &S.zempty, (uint32_t)(tp - 1) & 1u, status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) { run = false; break; }
                tc::fence_after();
                // design rows, two pixels interleaved: value f of pixel px at
                // Z[((px / 2) zs + f) 2 + px % 2]; lanes m, m + 1 (pixels 2k, 2k + 1) swap
                // half of their values so that each writes whole 16-byte groups
                const bool odd = m & 1;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    float* zp = Z + (size_t)((h * 128 + m) >> 1) * zs * 2;
                    // two 16-column chunks per TMEM wait
                    for (int c2 = 0; c2 < nb; c2 += 32) {
                        uint32_t rv[2][16];
                        tc::tmem_ld16_nowait(tl + (uint32_t)(acc * 128 + h * 64 + c2), rv[0]);
                        if (c2 + 16 < nb) {
                            tc::tmem_ld16_nowait(tl + (uint32_t)(acc * 128 + h * 64 + c2 + 16), rv[1]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; j++) rv[1][j] = 0u;
                        }
                        tc::tmem_wait_ld(rv[0], rv[1]);
#pragma unroll
                        for (int hc = 0; hc < 2; hc++) {
                            const int c = c2 + 16 * hc;
#pragma unroll
                            for (int g = 0; g < 4; g++) {
                                const float x0 = __uint_as_float(rv[hc][4 * g]) * wx[h];
                                const float x1 = __uint_as_float(rv[hc][4 * g + 1]) * wx[h];
                                const float x2 = __uint_as_float(rv[hc][4 * g + 2]) * wx[h];
                                const float x3 = __uint_as_float(rv[hc][4 * g + 3]) * wx[h];
                                const float r0 = __shfl_xor_sync(0xffffffffu, odd ? x0 : x2, 1);
                                const float r1 = __shfl_xor_sync(0xffffffffu, odd ? x1 : x3, 1);
                                const int f = c + 4 * g + (odd ? 2 : 0);
                                if (c < nb && c + 4 * g + 3 < zs)
                                    *reinterpret_cast<float4*>(zp + 2 * f) =
                                        odd ? make_float4(r0, x2, r1, x3) : make_float4(x0, r0, x1, r1);
                            }
                        }
                    }
                }
                __syncwarp();   // the swapped groups are written before the last columns
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    float* zp = Z + (size_t)((h * 128 + m) >> 1) * zs * 2 + (odd ? 1 : 0);
                    zp[2 * nb] = sqw[h];
                    zp[2 * (nb + 1)] = sqw[h] * Iv[h];
                    for (int c = nb + 2; c < zs; c++) zp[2 * c] = 0.0f;
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(&S.tempty[acc]);
                    tc::mbar_arrive(&S.zfull);
                }
                if (p + 1 < t.pairs) fetch(p + 1);
                // this set's share of the pair's Gram, once all four readers have written
                if (!ft_warp_wait(S, &S.zfull, (uint32_t)tp & 1u, status, lane)) { run = false; break; }
                gs.add(Z, zs);
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.zempty);
            }
            if (!run) break;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
            if (lane == 0 && nvalid) atomicAdd(a.n_pix + t.s, nvalid);
            if (item + 1 == ihi || a.items[item + 1].x != t.s) gs.flush(a.gram + (long)t.s * NPC * NPC, NPC);
        }
    } else if (warp >= FT_GRAM_WARP) {
        // ---------------- Gram warps: Gram threads 128 .. 383 (the readers are 0 .. 127); set
        // s = gt / 192 takes the pixel pairs of half s of the pair's rows
        const int gt = 128 + tid - FT_GRAM_WARP * 32;
        GramShare gs;
        gs.init(gt % 192, gt / 192, NPC);
        int tp = 0;
        bool run = true;
        for (int item = ilo; item < ihi && run; item++) {
            const FtItem t = ft_item<KS>(a, item);
            for (int p = 0; p < t.pairs; p++, tp++) {
                if (!ft_warp_wait(S, &S.zfull, (uint32_t)tp & 1u, status, lane)) { run = false; break; }
                gs.add(Z, zs);
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.zempty);
            }
            if (!run) break;
            // the segment's blocks are complete in this CTA when its next item is another segment's
            if (item + 1 == ihi || a.items[item + 1].x != t.s) gs.flush(a.gram + (long)t.s * NPC * NPC, NPC);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// The power of two that puts each segment's largest |R| at 2^14: one CTA per segment.
__global__ void __launch_bounds__(256) seg_rscale_kernel(const float* ref, long pitch, const int4* seg, float* rscale) {
    __shared__ float wmax[8];
    const int4 sg = seg[blockIdx.x];
    const int side = sg.y;
    const float* base = ref + (long)sg.x * pitch + sg.z;
    float mx = 0.0f;
    for (int y = threadIdx.x >> 5; y < side; y += 8)
        for (int x = threadIdx.x & 31; x < side; x += 32) mx = fmaxf(mx, fabsf(__ldg(base + (long)y * pitch + x)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) mx = fmaxf(mx, wmax[w]);
        rscale[blockIdx.x] = f16_range_scale(fmaxf(mx, wmax[0]));
    }
}

template <int KS>
int launch_fit_tc(const SegFitTcArgs& a, cudaStream_t st) {
    seg_rscale_kernel<<<a.n_segments, 256, 0, st>>>(a.ref, a.pitch, a.seg, a.rscale); argus_count_launch(1);
    const int zs = (a.NPC + 3) & ~3;
    const size_t smem = ft_layout(KS, zs).total + 1024;
    if (smem > 227 * 1024) return ARGUS_ERR_UNSUPPORTED;
    const cudaError_t e = cudaFuncSetAttribute(seg_fit_tc_kernel<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return argus_cuda_fail(e);
    seg_fit_tc_kernel<KS><<<a.n_ctas, FT_THREADS, smem, st>>>(a); argus_count_launch(1);
    return argus_launch_status();
}

}  // namespace

size_t argus_seg_fit_tc_smem(int ks, int NPC) {
    if (ks > 15) return 0;
    return ft_layout(ks, (NPC + 3) & ~3).total + 1024;
}

int argus_seg_fit_tc(const SegFitTcArgs& a, int ks, cudaStream_t st) {
    if (a.band < 2 || (a.band & 1) || a.nb > 64 || a.n_ctas < 1) return ARGUS_ERR_ARG;
    if (a.NPC > 52) return ARGUS_ERR_UNSUPPORTED;   // more 2 x 4 Gram blocks than a 192-thread set
    switch (ks) {
        case 7: return launch_fit_tc<7>(a, st);
        case 9: return launch_fit_tc<9>(a, st);
        case 11: return launch_fit_tc<11>(a, st);
        case 15: return launch_fit_tc<15>(a, st);
        default: return ARGUS_ERR_UNSUPPORTED;
    }
}
