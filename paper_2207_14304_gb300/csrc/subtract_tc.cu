// K6 on the tensor cores: the reference convolution of the full-frame
// subtraction (paper Sec. 4.2 direct image subtraction, Table 2), with the
// same definition as the per-tile SIMT body:
//
//   D = I - sum_k p_k(x,y) sum_{iu,iv} K_k[iv][iu] R(x - iu + r, y - iv + r) - sum_k bg_k p_k(x,y)
//
// For a strip of 128 output columns x0 .. x0+127 and a block of G
// consecutive source rows rho0 .. rho0+G-1, one TMEM accumulator collects
//   T[m][(j, k)] = sum_g sum_{u'} A_g[m][u'] B_g[u'][(j, k)],
//   A_g[m][u'] = R(x0 + m - r + u', rho0 + g)          (a Hankel matrix, u' < 32),
//   B_g[u'][(j, k)] = K_k[j - g][KS - 1 - u']          (zero unless 0 <= j - g < KS),
// tcgen05 MMAs of M = 128, N = (KS - 1 + G) * NK (144 for a 21 x 21 kernel of
// degree 2 and G = 4): K = 16 per row for taps 0..15, and one K = 16 MMA per
// row pair for taps 16..23, whose K groups are taken from the two rows'
// operands.  Column (j, k) is the contribution of the block to output row
// rho0 - 2r + j for term k: shifting B by g rows of taps makes the G source
// rows land on the columns of the output rows they feed, so the MMAs do part
// of the sum over iv and the epilogue reads (KS - 1 + G) * NK instead of
// KS * NK * G columns per block.
//
// The difference image stores the G matrices B_g (hi and lo) in the canonical
// layout.  In the variance every B_g is one stored operand Z read at a
// descriptor offset: Z row z holds the taps of column n = z - NK (G - 1) of
// B_0, and B_g[u'][n] = B_0[u'][n - NK g] is Z from row NK (G - 1 - g) on.
// With the 8-row groups of the canonical no-swizzle K-major layout 128 bytes
// apart, Z's rows are consecutive 16-byte lines, so a shift by NK g rows is an
// offset of 16 NK g bytes.  K group 3 of Z (taps 24..31, always zero in B)
// holds taps 16..23 of row z - NK instead: the row-pair MMA then reads B_g's
// taps 16..23 as its K group 0 and B_{g+1}'s as its K group 1 from one
// descriptor whose K-group stride is that of Z.  (The offsets put B's core
// matrices off 128-byte boundaries, which costs shared-memory bandwidth: the
// difference image's dense MMAs ran at 1.34 instead of 0.85 ms on Z; the
// variance's narrow MMAs leave that bandwidth idle.)
//
// Precision.  The difference image splits R and K into BF16 hi + lo (each
// rounded to nearest) and sums hi*hi + hi*lo + lo*hi in FP32 in TMEM: the
// dropped lo*lo term is below 2^-16 relative, FP32-level agreement.  The
// difference variance (VAR) computes sum Kc^2 (x) V_ref with Kc the kernel at
// the centre of the strip's 128 x 128 variance tile from one BF16 product
// (V_ref and Kc^2 each rounded once): its error is at most 2^-8 of that
// convolved-reference term, which for a deep reference is a small part of
// V_D (about 1 %), far inside the detection margin.
//
// A is stored once per source row as its 19 distinct core matrices: in the
// canonical no-swizzle K-major layout the core matrix of row group i and K
// group j holds A[8i + a][8j + b] = R(x0 - r + 8(i + j) + a + b, rs), a
// function of i + j, so the descriptor's row-group stride equals its K-group
// stride (both 128 bytes) and 16-byte row t of the stored operand is
// R(x0 - r + t + b), b = 0..7.  A producer warp rounds its source row to BF16
// once (lane l: value pairs l, l + 32, ...) into a small row buffer; lane l then
// writes operand rows t = l, l + 32, ... (consecutive lanes, consecutive 16-byte
// rows: no bank conflicts), each from five aligned 32-bit words of the buffer
// and a byte permutation (rows starting at an odd element straddle words).
//
// Staging.  The variance stages by the tensor-memory accelerator: every input
// tile is one tiled 2-D TMA copy (cp.async.bulk.tensor) from a tensor map of the
// pitched image, the image's edges and the halo past them read as zero by the
// copy itself, each slot's landing signalled on an mbarrier.  The difference
// image stages by 16-byte cp.async with zero fill: with TMA its per-block
// mbarrier rounds lengthened a critical path the epilogue only just keeps
// (measured 1.02-1.11 against 0.85 ms per full frame, whatever the waits and
// fences were).  Persistent CTAs walk the strips of 128 columns x a band of TCY
// output rows (256 for the difference image, 128 for the variance), streaming
// each band's TCY + 2r source rows in blocks of G (the difference image: G = 4,
// one CTA of 320 threads per SM; the variance: G = 8, two CTAs per SM).
// Warps 0-3: epilogue, one output column per thread and TMEM lane; warp w
// stages the observed values and flag bytes of its 32 columns for the G output
// rows a block completes, LA blocks ahead (variance: lane 0, two boxes of
// 32 x G).  Warps 4-7: producers, warp 4 + p for source rows p G/4 .. of each
// block (their windows staged LA blocks ahead: variance, one box of PWIN x 2
// by lane 0); it writes those rows' A operands.  Warps 8-9: one thread each
// issues the MMAs of alternate blocks.  TMEM holds NTB accumulators.  Every
// wait is bounded; a timeout latches ARGUS_ERR_TIMEOUT, all roles stop, and
// each warp waits (bounded) for the copies it still has in flight before the
// CTA exits.
#include <cuda_bf16.h>
#include <string.h>

#include "subtract_tile.cuh"
#include "tc_ptx.cuh"

namespace {
using namespace argus_sub;

constexpr int TCX = 128;                     // output columns per CTA (MMA M)
// output rows per band: the variance's strip is one 128 x 128 variance tile; the
// difference image takes 256-row bands (half the halo rows of 128-row bands)
template <bool VAR>
__host__ __device__ constexpr int tcy() { return VAR ? VAR_TILE : 256; }
// source rows per block: the variance's narrow MMAs leave the tensor pipe idle, so its
// blocks are larger (fewer barrier rounds per row); the difference image's MMA width
// grows with G (N = (KS - 1 + G) NK), so it keeps four
template <bool VAR>
__host__ __device__ constexpr int gsz() { return VAR ? 8 : 4; }
// blocks staged ahead (24 source rows either way) and staging slots per warp (> LA)
template <bool VAR>
__host__ __device__ constexpr int lahead() { return VAR ? 3 : 6; }
template <bool VAR>
__host__ __device__ constexpr int nslot() { return VAR ? 4 : 8; }
constexpr int TKC = 32;                      // MMA K: taps u', padded
constexpr int NCM = TCX / 8 + TKC / 8 - 1;   // distinct core matrices of one Hankel tile
constexpr uint32_t A_BYTES = NCM * 128;      // one operand part (hi or lo) of one source row
// block stages of A: three for both kernels (the variance's fit in two CTAs per SM)
constexpr int NSB = 3;
constexpr int NPW = 4;                       // producer warps
constexpr int PWIN = 176;                    // staged window of a source row (160 values + offset)
constexpr int MMA_WARP = 4 + NPW;            // warps 8 and 9 issue the MMAs of even and odd blocks
constexpr int TC_THREADS = (MMA_WARP + 2) * 32;
constexpr uint32_t LBO = 128, SBO_A = 128, SBO_Z = 128, SBO_B = 512;
constexpr long long WAIT_LIMIT = 2000000000LL;   // ~1 s of SM clock
constexpr int NTB = 3;                       // TMEM accumulators
static_assert(MMA_WARP == 8 && TC_THREADS == 320, "warp roles");
static_assert(NCM * 8 == TCX + TKC - 8 && NCM + 1 <= 32, "one lane per 8 operand rows, plus one");

template <int KS, int NK, int G>
struct TcCfg {
    static constexpr int NJB = KS - 1 + G;                  // output rows a block feeds
    static constexpr int NCOL = NJB * NK;                   // used MMA columns
    static constexpr int N = (NCOL + 15) / 16 * 16;         // MMA N
    static constexpr int TSTRIDE = (N + 31) / 32 * 32;      // TMEM columns per accumulator
    static constexpr int Z0 = NK * (G - 1);                 // Z row of column 0 of B_0
    static constexpr int ZROWS = Z0 + N;                    // rows of Z read by some B_g
    static constexpr uint32_t ZLBO = (uint32_t)ZROWS * 16;  // K-group stride of Z
    static constexpr uint32_t Z_BYTES = 4 * ZLBO;           // one part of Z (four K groups)
    static constexpr uint32_t B_BYTES = (uint32_t)N / 8 * SBO_B;   // one part of one B_g
    static constexpr int RLP = (NJB + G - 1) / G * G;       // ring of pending output rows
    // one term: the ring rotates (RLP / G unrolled blocks per turn, no register moves);
    // more terms: a compact loop that shifts the ring by G after each block
    static constexpr bool ROT = NK == 1;
    static constexpr int UNR = ROT ? RLP / G : 1;
    static_assert(N <= 256 && NTB * TSTRIDE <= 512, "MMA shape");
    static_assert(KS <= 24 && G % 2 == 0 && G % NPW == 0, "taps 16..23 of row pairs share one MMA");
    static_assert(ZROWS * 16 < (1 << 18), "descriptor offsets");
};

template <int KS, int NK, bool VAR>
struct TcShared {
    static constexpr int G = gsz<VAR>();
    static constexpr int NP = VAR ? 1 : 2;   // operand parts: hi (and lo)
    static constexpr int RPW = G / NPW;      // source rows per producer warp and block
    static constexpr int NSL = nslot<VAR>();
    static constexpr int WSLOT = (RPW * PWIN + 31) / 32 * 32;   // floats per staging slot (128-byte multiple)
    using C = TcCfg<KS, NK, G>;
    // The MMA operands come first (measured: with the staging buffers ahead of them the
    // difference image took 0.94 instead of 0.84 ms per full frame).
    // The variance: Z, one set per strip parity; the difference image: the G row-shifted
    // copies B_g (their MMAs run at the dense rate, and Z's row offsets of 16 NK g bytes
    // would put B's core matrices off 128-byte boundaries)
    alignas(128) uint8_t z[VAR ? 2 : 1][NP][VAR ? C::Z_BYTES : 16];
    alignas(128) uint8_t b[VAR ? 1 : G][NP][VAR ? 16 : C::B_BYTES];
    alignas(128) uint8_t a[NSB][NP][G][A_BYTES];   // A operands of a block: [stage][part][row]
    alignas(128) float wsrc[NPW][NSL][WSLOT];   // staged windows of each producer warp's source rows
    alignas(128) float qI[4][NSL][G][32];       // staged observed values of each epilogue warp's columns
    alignas(128) uint8_t qF[4][NSL][G][32];     // their flag bytes
    alignas(16) uint32_t rowb[NPW][NP][(NCM + 1) * 4];   // a source row rounded to BF16 (hi, lo), 2 per word
    uint64_t filled[NSB], empty[NSB], tfull[NTB], tempty[NTB];
    uint64_t bready[2], bfree[2];               // VAR: Z set written / no longer read by the MMAs
    uint64_t sfull[NPW][NSL];                   // a producer warp's staging slot landed
    uint64_t qfull[4][NSL];                     // an epilogue warp's staging slot landed
    uint32_t tmem;
    int abort;       // set by any role that timed out
};

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Two floats rounded to BF16 and packed, v0 in the low half.
__device__ __forceinline__ uint32_t bf16x2_rn(float v0, float v1) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
    return d;
}

// One try first (the common case: the phase is already complete), then a
// bounded wait that also gives up once another role has aborted.
template <class SH>
__device__ __forceinline__ bool wait_or_abort(SH& S, uint64_t* bar, uint32_t parity, int* status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (S.abort) return false;
    if (!tc::mbar_wait_bounded(bar, parity, WAIT_LIMIT)) {
        S.abort = 1;
        argus_latch(status, ARGUS_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// A staging slot's copy has landed: lane 0 waits (bounded), the warp follows, and
// every lane then observes the completed phase itself (so the copied bytes are
// visible to it).  The phase cannot move on meanwhile: only this warp re-arms the slot.
template <class SH>
__device__ __forceinline__ bool warp_wait_copy(SH& S, uint64_t* bar, uint32_t parity, int* status, int lane) {
    bool ok = true;
    if (lane == 0) ok = wait_or_abort(S, bar, parity, status);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok)
        while (!tc::mbar_try_wait(bar, parity)) {
        }
    return ok;
}

// After an abort at block blk of an item whose block 0 is slot use q0 (nblk blocks,
// copies issued la blocks ahead): wait (bounded) for the copies of blocks blk ..
// min(nblk, blk + la + 1) - 1, those the warp issued and did not consume.
__device__ __noinline__ void drain_copies(uint64_t* bars, int nsl, int q0, int blk, int nblk, int la) {
    for (int b = blk; b < min(nblk, blk + la + 1); b++)
        tc::mbar_wait_bounded(&bars[(q0 + b) % nsl], (uint32_t)((q0 + b) / nsl) & 1u, WAIT_LIMIT);
}

// VAR = false: the difference image (NK spatial terms, background, D = I - model).
// VAR = true: the convolution of the difference variance, sum Kc^2 V_ref with Kc the
// kernel at the centre of the CTA's VAR_TILE x VAR_TILE variance tile (one term),
// V_D = V_I + that sum; the CTA's strip then has to lie in one variance tile.
// tm_src: the convolved image (R or V_ref), boxes of PWIN x G/4; tm_obs: the observed
// image (I or V_I), boxes of 32 x G; tm_flg: the flags, boxes of 32 x G.
template <int KS, int NK, bool VAR>
__global__ void __launch_bounds__(TC_THREADS, VAR ? 2 : 1)
    subtract_tc_kernel(SubArgs a, const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_obs,
                       const __grid_constant__ CUtensorMap tm_flg, int* status) {
    using Sh = TcShared<KS, NK, VAR>;
    constexpr int G = Sh::G;
    using C = TcCfg<KS, NK, G>;
    constexpr int NP = Sh::NP;                   // operand parts
    constexpr int RPW = Sh::RPW, NSL = Sh::NSL;
    constexpr int LA = lahead<VAR>();
    static_assert(NSL > LA, "a slot is re-armed only after its last reads");
    constexpr int P = VAR ? 1 : 3;               // products per K slice: hi*hi (+ hi*lo + lo*hi)
    static_assert(!VAR || NK == 1, "the variance convolution has one term");
    constexpr int TCY = tcy<VAR>();
    static_assert(!VAR || (TCX == VAR_TILE && TCY == VAR_TILE), "one variance tile per strip");
    float* outp = VAR ? a.diff_var : a.diff;
    constexpr int R = (KS - 1) / 2;
    constexpr int SOFF = (4 - R % 4) % 4;        // wsrc[.][SOFF + c] = R(x0 - R + c); x0 - R - SOFF is a multiple of 4
    static_assert(KS <= TKC && SOFF + 8 * NCM + 16 <= PWIN, "tile shape");
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    Sh& S = *reinterpret_cast<Sh*>(tc_smem_raw + ((1024 - (tc::smem_u32(tc_smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // work items: strips of TCX columns x TCY rows, item = by * gx + bx, taken by the
    // CTAs round robin; Z is built once (difference image) or per strip by the
    // producers into one of two sets (variance: it depends on the strip's variance tile)
    const int gx = (a.w + TCX - 1) / TCX, nitems = gx * ((a.h + TCY - 1) / TCY);
    auto geom = [&](int item, int& x0, int& y0, int& nout, int& nblk) {
        const int by = item / gx;
        x0 = (item - by * gx) * TCX;
        y0 = by * TCY;
        nout = min(TCY, a.h - y0);
        nblk = (nout + 2 * R + G - 1) / G;       // source rows y0 - R .. y0 + nout - 1 + R; rows past them are zero
    };

    // ---- Z from the kernel taps: row z, tap slot u < 24 holds column n = z - Z0 of B_0,
    // K_k[j][KS - 1 - u] for n = j NK + k (VAR: Kc^2, Kc the kernel at the centre of the
    // strip's variance tile); slot u >= 24 holds tap u - 8 of row z - NK.  Threads
    // first .. first + count - 1 write set bs.
    auto build_z = [&](int item, int bs, int first, int count) {
        float pc[ARGUS_MAX_TERMS];
        int nkt = NK;
        if (VAR) {
            int x0, y0, nout, nblk;
            geom(item, x0, y0, nout, nblk);
            const float xc = (float)(((x0 + a.ox) / VAR_TILE) * VAR_TILE) + 0.5f * (VAR_TILE - 1);
            const float yc = (float)(((y0 + a.oy) / VAR_TILE) * VAR_TILE) + 0.5f * (VAR_TILE - 1);
            const float xt = a.W > 1 ? (2.0f * xc - (float)(a.W - 1)) / (float)(a.W - 1) : 0.0f;
            const float yt = a.H > 1 ? (2.0f * yc - (float)(a.H - 1)) / (float)(a.H - 1) : 0.0f;
            spatial_terms(xt, yt, a.sdeg, pc);
            nkt = (a.sdeg + 1) * (a.sdeg + 2) / 2;
        }
        for (int e = tid - first; e < C::ZROWS * TKC; e += count) {
            const int zr = e / TKC, u = e - zr * TKC;
            const int zz = u < 24 ? zr : zr - NK, uu = u < 24 ? u : u - 8;
            const int n = zz - C::Z0;
            float v = 0.0f;
            if (n >= 0 && n < C::NCOL && uu < KS) {
                const int j = n / NK, k = n - j * NK;
                if (j < KS) {
                    if (VAR) {
                        float kc = 0.0f;
                        for (int q = 0; q < nkt; q++) kc = fmaf(pc[q], __ldg(a.K + q * KS * KS + j * KS + (KS - 1 - uu)), kc);
                        v = kc * kc;
                    } else {
                        v = __ldg(a.K + k * KS * KS + j * KS + (KS - 1 - uu));
                    }
                }
            }
            __nv_bfloat16 hi, lo;
            split_bf16(v, hi, lo);
            const uint32_t off = (uint32_t)(u >> 3) * C::ZLBO + (uint32_t)zr * 16 + (uint32_t)(u & 7) * 2;
            *reinterpret_cast<__nv_bfloat16*>(S.z[bs][0] + off) = hi;
            if constexpr (NP == 2) *reinterpret_cast<__nv_bfloat16*>(S.z[bs][NP - 1] + off) = lo;
        }
    };
    // ---- the difference image's B_g: column n = j NK + k holds K_k[j - g][KS - 1 - u'] in the
    // canonical layout (8-row groups SBO_B apart, K groups 128 bytes apart)
    auto build_b = [&]() {
        for (int e = tid; e < G * C::N * TKC; e += TC_THREADS) {
            const int g = e / (C::N * TKC), r = e - g * (C::N * TKC);
            const int n = r / TKC, u = r - n * TKC;
            const int j = n / NK, k = n - j * NK, iv = j - g;
            float v = 0.0f;
            if (n < C::NCOL && u < KS && iv >= 0 && iv < KS) v = __ldg(a.K + k * KS * KS + iv * KS + (KS - 1 - u));
            __nv_bfloat16 hi, lo;
            split_bf16(v, hi, lo);
            const uint32_t off = (uint32_t)(n >> 3) * SBO_B + (uint32_t)(u >> 3) * LBO + (uint32_t)(n & 7) * 16 +
                                 (uint32_t)(u & 7) * 2;
            *reinterpret_cast<__nv_bfloat16*>(S.b[g][0] + off) = hi;
            if constexpr (NP == 2) *reinterpret_cast<__nv_bfloat16*>(S.b[g][NP - 1] + off) = lo;
        }
    };
    if constexpr (!VAR) build_b();
    if (tid == 0) {
        if (VAR) {
            tc::tma_prefetch_map(&tm_src);
            tc::tma_prefetch_map(&tm_obs);
            tc::tma_prefetch_map(&tm_flg);
        }
        for (int s = 0; s < NSB; s++) {
            tc::mbar_init(&S.filled[s], NPW);   // one arrival per producer warp
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < NTB; b++) {
            tc::mbar_init(&S.tfull[b], 1);
            tc::mbar_init(&S.tempty[b], 4);   // one arrival per epilogue warp
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&S.bready[b], NPW);  // one arrival per producer warp
            tc::mbar_init(&S.bfree[b], 2);     // one commit per MMA issuer
        }
        for (int w = 0; w < 4; w++)
            for (int q = 0; q < NSL; q++) {
                tc::mbar_init(&S.sfull[w][q], 1);   // the issuing lane's arrival + the copy's bytes
                tc::mbar_init(&S.qfull[w][q], 1);
            }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    constexpr uint32_t TMEM_COLS = NTB * C::TSTRIDE <= 128 ? 128 : (NTB * C::TSTRIDE <= 256 ? 256 : 512);
    if (warp == 0) tc::tmem_alloc(&S.tmem, TMEM_COLS);
    tc::fence_proxy_async();   // Z written through the generic proxy
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;
    // every role walks the same items and blocks; gb counts blocks over the items and
    // drives the stage and TMEM rings and their barrier phases

    if (warp >= 4 && warp < MMA_WARP) {
        // ---------------- producers: warp 4 + pw writes the A operands of source rows
        // pw RPW .. pw RPW + RPW - 1 of every block, with no barrier between producer
        // warps.  The warp stages those rows' windows (PWIN values from frame column XS, a
        // multiple of 4; variance: lane 0, one box of RPW rows) LA blocks ahead into its
        // slot ring; the lanes round each row to BF16 once and write its operand rows;
        // after the writes and a proxy fence lane 0 arrives on the stage's filled barrier
        // (one arrival per producer warp).
        const int pw = warp - 4;
        bool run = true;
        int gb = 0, li = 0, gs = 0;   // gs: this warp's blocks over the items
        for (int item = blockIdx.x; item < nitems && run; item += gridDim.x, li++) {
            int x0, y0, nout, nblk;
            geom(item, x0, y0, nout, nblk);
            const int nsrc = nout + 2 * R;
            if constexpr (VAR) {   // this strip's Z set, once the MMAs of the strip two back are done with it
                bool ok = true;
                if (lane == 0 && li >= 2) ok = wait_or_abort(S, &S.bfree[li & 1], ((li - 2) >> 1) & 1, status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) { run = false; break; }
                build_z(item, li & 1, 4 * 32, NPW * 32);
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.bready[li & 1]);
            }
            const int XS = x0 - R - SOFF;        // frame column of a window's element 0, a multiple of 4
            const int gs0 = gs;
            auto issue = [&](int blk) {          // VAR, lane 0: the window box of block blk
                const int q = gs0 + blk, sl = q % NSL;
                tc::mbar_arrive_expect_tx(&S.sfull[pw][sl], RPW * PWIN * 4);
                tc::tma_load_2d(S.wsrc[pw][sl], &tm_src, XS, y0 - R + blk * G + pw * RPW, &S.sfull[pw][sl]);
            };
            // the difference image: 16-byte cp.async by the whole warp, one group per block
            // (past the band: an empty group), zero-filled outside the frame
            auto issue_cp = [&](int blk) {
                if (blk < nblk) {
                    const int rr = blk * G + pw, gy = y0 - R + rr;
                    const bool rin = rr < nsrc && gy >= 0 && gy < a.h;
                    float* dst = S.wsrc[pw][(gs0 + blk) % NSL];
                    for (int q = lane; q < PWIN / 4; q += 32) {
                        const int X = XS + 4 * q;
                        const int nb = (rin && X >= 0 && X < a.w) ? 4 * min(4, a.w - X) : 0;
                        tc::cp_async16(dst + 4 * q, nb ? a.ref + (long)gy * a.pitch + X : a.ref, nb);
                    }
                }
                tc::cp_async_commit();
            };
            const int npre = min(LA, nblk);
            if constexpr (VAR) {
                if (lane == 0)
                    for (int b = 0; b < npre; b++) issue(b);
            } else {
                for (int b = 0; b < LA; b++) issue_cp(b);
            }
            uint32_t (*rb)[(NCM + 1) * 4] = S.rowb[pw];
            for (int blk = 0; blk < nblk; blk++, gb++) {
                const int s = gb % NSB, fill = gb / NSB;
                if constexpr (VAR) {
                    if (lane == 0 && blk + LA < nblk) issue(blk + LA);
                } else {
                    issue_cp(blk + LA);
                }
                bool ok = true;
                if (lane == 0 && fill >= 1) ok = wait_or_abort(S, &S.empty[s], (fill - 1) & 1, status);
                const int q = gs0 + blk, sl = q % NSL;
                if (!__shfl_sync(0xffffffffu, ok, 0) ||
                    (VAR && !warp_wait_copy(S, &S.sfull[pw][sl], (uint32_t)(q / NSL) & 1u, status, lane))) {
                    if (VAR && lane == 0) drain_copies(S.sfull[pw], NSL, gs0, blk, nblk, LA);
                    run = false;
                    break;
                }
                if constexpr (!VAR) {
                    tc::cp_async_wait<LA>();     // block blk (own copies) ...
                    __syncwarp();                // ... and the other lanes' copies are visible
                }
#pragma unroll
                for (int rq = 0; rq < RPW; rq++) {
                    const int g = pw * RPW + rq;
                    // rows past the band's source rows are zero (the difference image's copies
                    // zero-fill them already)
                    const bool rin = !VAR || blk * G + g < nsrc;
                    // round the row once: lane l takes value pairs l, l + 32, ... (values 2p, 2p + 1:
                    // consecutive lanes read and write consecutive words, no bank conflicts)
                    {
                        const float* src = S.wsrc[pw][sl] + rq * PWIN + SOFF;
#pragma unroll
                        for (int p = lane; p < 4 * (NCM + 1); p += 32) {
                            const float v0 = rin ? src[2 * p] : 0.0f, v1 = rin ? src[2 * p + 1] : 0.0f;
                            const uint32_t h = bf16x2_rn(v0, v1);
                            rb[0][p] = h;
                            if constexpr (NP == 2)
                                rb[NP - 1][p] = bf16x2_rn(v0 - __uint_as_float(h << 16), v1 - __uint_as_float(h & 0xffff0000u));
                        }
                    }
                    __syncwarp();
                    // operand row t = lane + 32 rho holds elements t .. t + 7 of the rounded row
                    const int A = lane & 7;
                    const uint32_t sel = (A & 1) ? 0x5432u : 0x3210u;
#pragma unroll
                    for (int rho = 0; rho * 32 < NCM * 8; rho++) {
                        const int t = lane + 32 * rho;
                        if (t < NCM * 8) {
                            const int wb = 4 * (t >> 3) + (A >> 1);
#pragma unroll
                            for (int pt = 0; pt < NP; pt++) {
                                uint32_t wv[5];
#pragma unroll
                                for (int k = 0; k < 5; k++) wv[k] = rb[pt][wb + k];
                                *reinterpret_cast<uint4*>(S.a[s][pt][g] + 16 * t) =
                                    make_uint4(__byte_perm(wv[0], wv[1], sel), __byte_perm(wv[1], wv[2], sel),
                                               __byte_perm(wv[2], wv[3], sel), __byte_perm(wv[3], wv[4], sel));
                            }
                        }
                    }
                    __syncwarp();                // the row buffer is free for the next row
                }
                tc::fence_proxy_async();
                __syncwarp();                    // writes and fences of all lanes done
                if (lane == 0) tc::mbar_arrive(&S.filled[s]);
            }
            if constexpr (!VAR) {
                tc::cp_async_wait<0>();          // every copy of the strip landed before the next
                __syncwarp();                    // strip's copies reuse the slots
            }
            gs = gs0 + nblk;
        }
        if constexpr (!VAR) tc::cp_async_wait<0>();
        __syncwarp();
    } else if (warp >= MMA_WARP) {
        // ---------------- MMA issuers: warp MMA_WARP + q takes the blocks gb = q mod 2
        // (the issuing thread is held for about the MMAs' execution time, so two
        // issuers keep the tensor pipe fed while each waits on its barriers)
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(1, 128, C::N);
            int issued = -1, gb = 0, li = 0;
            bool run = true;
            for (int item = blockIdx.x; item < nitems && run; item += gridDim.x, li++) {
                int x0, y0, nout, nblk;
                geom(item, x0, y0, nout, nblk);
                const int bs = VAR ? (li & 1) : 0;
                if (VAR && !wait_or_abort(S, &S.bready[bs], (li >> 1) & 1, status)) { run = false; break; }
                for (int blk = 0; blk < nblk; blk++, gb++) {
                    if ((gb & 1) != warp - MMA_WARP) continue;
                    const int s = gb % NSB, tb = gb % NTB;
                    if (!wait_or_abort(S, &S.filled[s], (gb / NSB) & 1, status)) { run = false; break; }
                    if (gb >= NTB && !wait_or_abort(S, &S.tempty[tb], (gb / NTB - 1) & 1, status)) { run = false; break; }
                    tc::fence_after();
                    const uint32_t d = tmem + (uint32_t)(tb * C::TSTRIDE);
                    // taps u' = 0..15 of each source row: one K = 16 MMA per row and product
                    // (VAR: B_g is Z from row Z0 - NK g on)
#pragma unroll
                    for (int g = 0; g < G; g++) {
#pragma unroll
                        for (int pr = 0; pr < P; pr++) {
                            const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;   // hi*hi, hi*lo, lo*hi
                            const uint64_t ad = tc::smem_desc(tc::smem_u32(S.a[s][pa][g]), LBO, SBO_A);
                            const uint64_t bd =
                                VAR ? tc::smem_desc(tc::smem_u32(S.z[bs][pb]) + (uint32_t)(C::Z0 - NK * g) * 16,
                                                    C::ZLBO, SBO_Z)
                                    : tc::smem_desc(tc::smem_u32(S.b[g][pb]), LBO, SBO_B);
                            tc::mma_bf16(d, ad, bd, idesc, (g | pr) ? 1u : 0u);
                        }
                    }
                    // taps 16..23 of two source rows in one K = 16 MMA: K group 0 is group 2
                    // of row g, K group 1 group 2 of row g + 1 (the K-group stride is the
                    // distance between the two rows' operands, of A and of B_g; Z: group 3
                    // holds group 2 of the row NK lower, i.e. B_{g+1}'s taps 16..23)
#pragma unroll
                    for (int g = 0; g < (KS > 16 ? G : 0); g += 2) {
#pragma unroll
                        for (int pr = 0; pr < P; pr++) {
                            const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
                            const uint64_t ad = tc::smem_desc(tc::smem_u32(S.a[s][pa][g]) + 2 * 128, A_BYTES, SBO_A);
                            const uint64_t bd =
                                VAR ? tc::smem_desc(tc::smem_u32(S.z[bs][pb]) + 2 * C::ZLBO +
                                                        (uint32_t)(C::Z0 - NK * g) * 16,
                                                    C::ZLBO, SBO_Z)
                                    : tc::smem_desc(tc::smem_u32(S.b[g][pb]) + 2 * 128, NP * C::B_BYTES, SBO_B);
                            tc::mma_bf16(d, ad, bd, idesc, 1u);
                        }
                    }
                    tc::commit(&S.empty[s]);
                    tc::commit(&S.tfull[tb]);
                    issued = gb;
                }
                // this issuer's MMAs of the strip done: its Z set may be rewritten (both
                // issuers have blocks in every strip: a strip has at least 3)
                if (VAR && run) tc::commit(&S.bfree[bs]);
            }
            // every issued MMA must land before TMEM is released (a commit
            // tracks all earlier MMAs of this thread, so its last one suffices)
            if (issued >= 0) {
                if (!tc::mbar_wait_bounded(&S.tfull[issued % NTB], (issued / NTB) & 1, WAIT_LIMIT)) {
                    S.abort = 1;
                    argus_latch(status, ARGUS_ERR_TIMEOUT);
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warp w owns output columns x0 + 32 w .. + 31 (TMEM lanes
        // 32 w ..), one per thread; its lane 0 copies their observed values and flag bytes.
        const int m = tid, w = warp;
        const float ysc = a.H > 1 ? 2.0f / (float)(a.H - 1) : 0.0f;   // yt = 2 (y + oy) / (H - 1) - 1
        const float yof = a.H > 1 ? -1.0f : 0.0f;
        const uint32_t tl = tmem + ((uint32_t)(w * 32) << 16);
        // p_k = xt^i yt^j: the xt^i factor is fixed for a column, so each T column
        // enters the ring already multiplied by it and the ring keeps one sum per
        // power of yt (NJ = degree + 1) instead of one per term
        constexpr int NJ = NK == 1 ? 1 : (NK == 3 ? 2 : 3);
        constexpr int RLP = C::RLP, UNR = C::UNR;
        bool run = true;
        int gb = 0, gq = 0;   // gq: this warp's blocks over the items
        for (int item = blockIdx.x; item < nitems && run; item += gridDim.x) {
            int x0, y0, nout, nblk;
            geom(item, x0, y0, nout, nblk);
            const int x = x0 + m;
            const float xt = a.W > 1 ? (float)(2 * (x + a.ox) - (a.W - 1)) / (float)(a.W - 1) : 0.0f;
            // the background as B0 + B1 yt + B2 yt^2 with the x terms of this column
            // folded into B0 and B1
            float B0 = 0.0f, B1 = 0.0f, B2 = 0.0f;
            if (VAR) {
            } else if (a.nbg == 6) {
                B0 = fmaf((float)a.bg[5], xt * xt, fmaf((float)a.bg[3], xt, (float)a.bg[0]));
                B1 = fmaf((float)a.bg[4], xt, (float)a.bg[1]);
                B2 = (float)a.bg[2];
            } else if (a.nbg == 3) {
                B0 = fmaf((float)a.bg[2], xt, (float)a.bg[0]);
                B1 = (float)a.bg[1];
            } else if (a.nbg == 1) {
                B0 = (float)a.bg[0];
            }
            const bool xin = x >= R && x <= a.w - 1 - R;
            const float xp[3] = {1.0f, VAR ? 1.0f : xt, VAR ? 1.0f : xt * xt};
            float acc[RLP][NJ];
#pragma unroll
            for (int i = 0; i < RLP; i++)
#pragma unroll
                for (int j = 0; j < NJ; j++) acc[i][j] = 0.0f;
            // observed values and flag bytes of this warp's columns in the output rows the
            // block blk completes (rows blk G - 2R + i, i < G: one box of each, zero outside
            // the frame) into slot (gq0 + blk) mod NSL
            const int gq0 = gq;
            // the difference image: 16-byte cp.async by the whole warp, one group per block
            // (past the band: an empty group), zero-filled outside the band
            auto fetch_cp = [&](int blk) {
                const int q = gq0 + blk, sl = q % NSL;
                if (blk < nblk) {
                    for (int e = lane; e < G * 8; e += 32) {
                        const int i = e >> 3, c = e & 7;
                        const int eta = blk * G - 2 * R + i, X = x0 + 32 * w + 4 * c;
                        const bool in = eta >= 0 && eta < nout && X < a.w;
                        const int nb = in ? 4 * min(4, a.w - X) : 0;
                        tc::cp_async16(&S.qI[w][sl][i][4 * c], nb ? a.sci + (long)(y0 + eta) * a.pitch + X : a.sci, nb);
                    }
                    for (int e = lane; e < G * 2; e += 32) {
                        const int i = e >> 1, c = e & 1;
                        const int eta = blk * G - 2 * R + i, X = x0 + 32 * w + 16 * c;
                        const bool in = eta >= 0 && eta < nout && X < a.w;
                        const int nb = in ? min(16, a.w - X) : 0;
                        tc::cp_async16(&S.qF[w][sl][i][16 * c], nb ? a.flags + (long)(y0 + eta) * a.pitch + X : a.flags, nb);
                    }
                }
                tc::cp_async_commit();
            };
            auto fetch = [&](int blk) {          // VAR, lane 0: one box of values, one of flags
                const int q = gq0 + blk, sl = q % NSL;
                tc::mbar_arrive_expect_tx(&S.qfull[w][sl], G * 32 * 5);
                tc::tma_load_2d(S.qI[w][sl], &tm_obs, x0 + 32 * w, y0 + blk * G - 2 * R, &S.qfull[w][sl]);
                tc::tma_load_2d(S.qF[w][sl], &tm_flg, x0 + 32 * w, y0 + blk * G - 2 * R, &S.qfull[w][sl]);
            };
            const int npre = min(LA, nblk);
            if constexpr (VAR) {
                if (lane == 0)
                    for (int b = 0; b < npre; b++) fetch(b);
            } else {
                for (int b = 0; b < LA; b++) fetch_cp(b);
            }
            // ring: output row blk G - 2R + j of block blk sits in slot (U G + j) mod RLP, U = blk
            // mod UNR; a block completes the rows in slots U G .. U G + G - 1, which are then
            // written out and cleared for the rows RLP further down (ROT), or written out
            // before the ring shifts by G (U = 0)
#pragma unroll 1
            for (int blk0 = 0; blk0 < nblk && run; blk0 += UNR) {
#pragma unroll
                for (int U = 0; U < UNR; U++) {
                    const int blk = blk0 + U;
                    if (blk >= nblk) break;
                    if constexpr (VAR) {
                        if (lane == 0 && blk + LA < nblk) fetch(blk + LA);
                    } else {
                        fetch_cp(blk + LA);
                    }
                    const int tb = gb % NTB;
                    // lane 0 waits (fewer pollers on the barrier), the warp follows
                    bool ok = true;
                    if (lane == 0) ok = wait_or_abort(S, &S.tfull[tb], (gb / NTB) & 1, status);
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) {
                        if (VAR && lane == 0) drain_copies(S.qfull[w], NSL, gq0, blk, nblk, LA);
                        run = false;
                        break;
                    }
                    tc::fence_after();
                    constexpr int NCH = (C::NCOL + 15) / 16;   // 16-column chunks
                    constexpr int LG = C::ROT ? 3 : 2;          // chunks per TMEM wait (registers)
#pragma unroll
                    for (int c3 = 0; c3 < NCH; c3 += LG) {
                        uint32_t r[3][16];
#pragma unroll
                        for (int q = 0; q < 3; q++) {
                            if (q < LG && c3 + q < NCH) {
                                tc::tmem_ld16_nowait(tl + (uint32_t)(tb * C::TSTRIDE + (c3 + q) * 16), r[q]);
                            } else {
#pragma unroll
                                for (int j = 0; j < 16; j++) r[q][j] = 0u;
                            }
                        }
                        tc::tmem_wait_ld(r[0], r[1], r[2]);
#pragma unroll
                        for (int q = 0; q < LG; q++)
#pragma unroll
                            for (int j = 0; j < 16; j++) {
                                const int n = (c3 + q) * 16 + j;
                                if (n < C::NCOL) {
                                    const int jj = n / NK, k = n - jj * NK;
                                    // term k of 1, y, y^2, x, x y, x^2 (or 1, y, x) as (i, j)
                                    const int ti = NK == 6 ? (k < 3 ? 0 : (k < 5 ? 1 : 2)) : (NK == 3 ? (k == 2) : 0);
                                    const int tj = NK == 6 ? (k < 3 ? k : (k == 4 ? 1 : 0)) : (NK == 3 ? (k == 1) : 0);
                                    float& dst = acc[(U * G + jj) % RLP][tj];
                                    dst = VAR ? dst + __uint_as_float(r[q][j]) : fmaf(xp[ti], __uint_as_float(r[q][j]), dst);
                                }
                            }
                    }
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&S.tempty[tb]);
                    const int q = gq0 + blk, sl = q % NSL;
                    if constexpr (VAR) {
                        if (!warp_wait_copy(S, &S.qfull[w][sl], (uint32_t)(q / NSL) & 1u, status, lane)) {
                            if (lane == 0) drain_copies(S.qfull[w], NSL, gq0, blk, nblk, LA);
                            run = false;
                            break;
                        }
                    } else {
                        tc::cp_async_wait<LA>();     // this block's rows have landed (own copies)
                        __syncwarp();                // ... and the other lanes' copies are visible
                    }
#pragma unroll
                    for (int i = 0; i < G; i++) {
                        const int eta = blk * G - 2 * R + i;
                        if (eta >= 0 && eta < nout && x < a.w) {
                            const float I = S.qI[w][sl][i][lane];
                            const uint32_t fl = S.qF[w][sl][i][lane];
                            const int y = y0 + eta;
                            const float yt = fmaf((float)(y + a.oy), ysc, yof);
                            // model = (acc0 + B0) + (acc1 + B1) yt + (acc2 + B2) yt^2
                            float c2 = B2, c1 = B1;
                            if constexpr (NJ > 2) c2 += acc[(U * G + i) % RLP][NJ > 2 ? 2 : 0];
                            if constexpr (NJ > 1) c1 += acc[(U * G + i) % RLP][NJ > 1 ? 1 : 0];
                            const float a0 = acc[(U * G + i) % RLP][0];
                            const float model = fmaf(fmaf(c2, yt, c1), yt, a0 + B0);
                            const bool inner = xin && y >= R && y <= a.h - 1 - R && fl == 0;
                            if (VAR) outp[(long)y * a.pitch + x] = inner ? I + a0 : 0.0f;
                            else outp[(long)y * a.pitch + x] = inner ? I - model : 0.0f;
                        }
                        if constexpr (C::ROT) {
#pragma unroll
                            for (int j = 0; j < NJ; j++) acc[(U * G + i) % RLP][j] = 0.0f;
                        }
                    }
                    __syncwarp();                    // the slot's reads before lane 0 re-arms it
                    if constexpr (!C::ROT) {
#pragma unroll
                        for (int i = 0; i + G < RLP; i++)
#pragma unroll
                            for (int j = 0; j < NJ; j++) acc[i][j] = acc[i + G][j];
#pragma unroll
                        for (int i = RLP - G; i < RLP; i++)
#pragma unroll
                            for (int j = 0; j < NJ; j++) acc[i][j] = 0.0f;
                    }
                    gb++;
                }
            }
            if constexpr (!VAR) {
                tc::cp_async_wait<0>();          // every copy of the strip landed before the next
                __syncwarp();                    // strip's copies reuse the slots
            }
            gq = gq0 + nblk;
        }
        if constexpr (!VAR) tc::cp_async_wait<0>();
        __syncwarp();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

template <int KS, int NK, bool VAR>
int launch_tc(const SubArgs& a, int* status, cudaStream_t st) {
    using Sh = TcShared<KS, NK, VAR>;
    // the difference image: more than half the shared memory, so one CTA per SM; the
    // variance: two CTAs per SM
    size_t smem = sizeof(Sh) + 1024;
    if (!VAR && smem < 116 * 1024) smem = 116 * 1024;
    if (VAR && smem > 113 * 1024) return ARGUS_ERR_UNSUPPORTED;
    cudaError_t e = cudaFuncSetAttribute(subtract_tc_kernel<KS, NK, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return argus_cuda_fail(e);
    // the variance: tensor maps of the three images it stages (pointers 16-byte aligned
    // and the pitch a multiple of 16 elements, as every entry point checks); the
    // difference image stages by cp.async and takes none
    CUtensorMap tsrc, tobs, tflg;
    memset(&tsrc, 0, sizeof tsrc);
    memset(&tobs, 0, sizeof tobs);
    memset(&tflg, 0, sizeof tflg);
    if (VAR) {
        int rc = argus_tmap_2d(&tsrc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.ref_var, a.w, a.h, a.pitch, PWIN, Sh::RPW);
        if (!rc) rc = argus_tmap_2d(&tobs, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.sci_var, a.w, a.h, a.pitch, 32, Sh::G);
        if (!rc) rc = argus_tmap_2d(&tflg, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, a.flags, a.w, a.h, a.pitch, 32, Sh::G);
        if (rc) return rc;
    }
    const int nitems = ((a.w + TCX - 1) / TCX) * ((a.h + tcy<VAR>() - 1) / tcy<VAR>());
    // persistent: the CTAs walk the strips (the set-up once per CTA)
    int grid = nitems, dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return argus_cuda_fail(e);
    if (grid > (VAR ? 2 : 1) * sms) grid = (VAR ? 2 : 1) * sms;
    subtract_tc_kernel<KS, NK, VAR><<<grid, TC_THREADS, smem, st>>>(a, tsrc, tobs, tflg, status); argus_count_launch(1);
    return argus_launch_status();
}

}  // namespace

// Difference image on the tensor cores for the kernel sizes it is built for;
// returns ARGUS_ERR_UNSUPPORTED for the others (the caller uses the SIMT body).
int argus_subtract_tc(const SubArgs& a, int ksize, int nk, int* status, cudaStream_t st) {
    if (ksize == 21) {
        if (nk == 1) return launch_tc<21, 1, false>(a, status, st);
        if (nk == 3) return launch_tc<21, 3, false>(a, status, st);
        if (nk == 6) return launch_tc<21, 6, false>(a, status, st);
    }
    if (ksize == 11) {
        if (nk == 1) return launch_tc<11, 1, false>(a, status, st);
        if (nk == 3) return launch_tc<11, 3, false>(a, status, st);
        if (nk == 6) return launch_tc<11, 6, false>(a, status, st);
    }
    return ARGUS_ERR_UNSUPPORTED;
}

// Difference variance on the tensor cores (the sum Kc^2 (x) V_ref, one variance tile
// per CTA): for the kernel sizes it is built for and frame origins on the
// VAR_TILE grid; ARGUS_ERR_UNSUPPORTED otherwise (the caller uses the SIMT kernel).
int argus_subtract_var_tc(const SubArgs& a, int ksize, int* status, cudaStream_t st) {
    if (a.ox % VAR_TILE || a.oy % VAR_TILE) return ARGUS_ERR_UNSUPPORTED;
    if (ksize == 21) return launch_tc<21, 1, true>(a, status, st);
    if (ksize == 11) return launch_tc<11, 1, true>(a, status, st);
    return ARGUS_ERR_UNSUPPORTED;
}
