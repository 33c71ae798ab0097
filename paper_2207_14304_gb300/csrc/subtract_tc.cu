// K6 on the tensor cores: the reference convolution of the full-frame
// subtraction (paper Sec. 4.2 direct image subtraction, Table 2), with the
// same definition as the per-tile SIMT body:
//
//   D = I - sum_k p_k(x,y) sum_{iu,iv} K_k[iv][iu] R(x - iu + r, y - iv + r) - sum_k bg_k p_k(x,y)
//
// For one source row R(., rs) and a strip of 128 output columns x0 .. x0+127,
//   T[m][(iv, k)] = sum_{u'} A[m][u'] B[u'][(iv, k)],
//   A[m][u'] = R(x0 + m - r + u', rs)  (a Hankel matrix, u' < 32),
//   B[u'][(iv, k)] = K_k[iv][KS - 1 - u']  (zero for u' >= KS),
// is one tcgen05 MMA of M = 128, N = 128 (KS * NK <= 128 columns used),
// K = 32.  T holds every contribution of that source row to the output rows
// rs - r .. rs + r: column (iv, k) belongs to output row rs + iv - r.  The
// epilogue warps add T into a ring of pending output rows (one register set
// per row) and finish a row once its last source row is in.  Operands are
// BF16 hi/lo pairs (v = hi + lo, each rounded to nearest) and every product
// is hi*hi + hi*lo + lo*hi, accumulated in FP32 in TMEM: the dropped lo*lo
// term is below 2^-16 relative, well inside FP32-level agreement.
//
// A is stored once per source row as its 19 distinct core matrices: in the
// canonical no-swizzle K-major layout the core matrix of row group i and K
// group j holds A[8i + a][8j + b] = R(x0 - r + 8(i + j) + a + b, rs), a
// function of i + j, so the descriptor's row-group stride equals its K-group
// stride (both 128 bytes) and group (i, j) reads the matrix stored at i + j.
//
// CTA: 128 columns x a band of TCY output rows, streaming the band's
// TCY + 2r source rows.  Warps 0-3: epilogue, one output column per thread
// and TMEM lane, holding the ring of pending rows in registers (one sum per
// power of y: the x powers are folded in as each T column is added).  The
// row loop is unrolled U = 3 times with a ring of KS + U - 1 entries that
// shifts by U, so the ring moves once per U rows.  Science values and flag
// words reach shared memory by cp.async LQ rows ahead, each thread fetching
// its own column.  Warps 4-9: producers (source rows arrive by 16-byte
// cp.async DP rows ahead; each value is split into BF16 hi/lo once, one row
// ahead of its use; 152 threads then write the 19 core matrices with 32-bit
// loads and byte permutes, NSTAGE stages; one named barrier per row).  Warp
// 10: one thread issues the MMAs.  TMEM holds four 128-column accumulators, so
// the MMAs run up to three rows ahead of the epilogue.  Every wait is
// bounded; a timeout latches ARGUS_ERR_TIMEOUT and all roles stop.
#include <cuda_bf16.h>

#include "subtract_tile.cuh"
#include "tc_ptx.cuh"

namespace {
using namespace argus_sub;

constexpr int TCX = 128;                     // output columns per CTA (MMA M)
constexpr int TCY = 128;                     // output rows per CTA band
constexpr int TKC = 32;                      // MMA K: taps u', padded
constexpr int NCM = TCX / 8 + TKC / 8 - 1;   // distinct core matrices of one Hankel tile
constexpr uint32_t A_BYTES = NCM * 128;      // one operand (hi or lo) of one source row
constexpr uint32_t B_BYTES = 128 * TKC * 2;
constexpr int NSTAGE = 8;                    // Hankel stages
constexpr int SRCW = TCX + TKC;              // source values per row
constexpr int SRCC = SRCW / 4 + 1;           // 16-byte chunks staged per row (one spare for the offset)
constexpr int NSRC = 8;                      // fp32 source-row ring
constexpr int DP = 6;                        // source rows in flight ahead of the one being tiled
constexpr int NBUILD = NCM * 8;              // one builder thread per core-matrix row
constexpr int NPROD = (NBUILD + 31) / 32 * 32;   // producer threads (warps 4-8)
constexpr int MMA_WARP = 4 + NPROD / 32;     // warps 9 and 10 issue the MMAs of even and odd rows
constexpr int TC_THREADS = (MMA_WARP + 2) * 32;   // warps 0-3 epilogue, 4-8 producers, 9-10 MMA issuers
constexpr uint32_t LBO = 128, SBO_A = 128, SBO_B = 512;
constexpr long long WAIT_LIMIT = 2000000000LL;   // ~1 s of SM clock
constexpr int NTB = 4;                       // TMEM accumulator buffers of 128 columns
constexpr int LQ = 4, NQ = 8;                // science/flag rows fetched LQ ahead into an NQ-slot ring
constexpr int U = 3;                         // epilogue rows per ring shift
static_assert(MMA_WARP == 9 && TC_THREADS == 352 && SRCC <= NPROD, "warp roles");

struct TcShared {
    uint8_t bhi[B_BYTES];
    uint8_t blo[B_BYTES];
    uint8_t ahi[NSTAGE][A_BYTES];
    uint8_t alo[NSTAGE][A_BYTES];
    alignas(16) float srcf[NSRC][SRCC * 4];
    alignas(16) float qI[NQ][TCX];                // science values of output rows, by row & (NQ - 1)
    alignas(16) uint32_t qF[NQ][TCX];             // the 32-bit word holding each output pixel's flag byte
    uint64_t filled[NSTAGE];
    uint64_t empty[NSTAGE], tfull[NTB], tempty[NTB];
    uint32_t tmem;
    int abort;       // set by any role that timed out
    int pstop;       // producers' common decision, written by producer 0 between barriers
};

__device__ __forceinline__ uint32_t canon_off(int row, int kk) {
    return (uint32_t)(row >> 3) * SBO_B + (uint32_t)(kk >> 3) * LBO + (uint32_t)(row & 7) * 16 + (uint32_t)(kk & 7) * 2;
}

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

// hi/lo split of a pair (hi = rn(v), lo = rn(v - hi)), each packed two per word.
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    hi = bf16x2_rn(v0, v1);
    lo = bf16x2_rn(v0 - __uint_as_float(hi << 16), v1 - __uint_as_float(hi & 0xffff0000u));
}

// One try first (the common case: the phase is already complete), then a
// bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_or_abort(TcShared& S, uint64_t* bar, uint32_t parity, int* status) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (S.abort) return false;
    if (!tc::mbar_wait_bounded(bar, parity, WAIT_LIMIT)) {
        S.abort = 1;
        argus_latch(status, ARGUS_ERR_TIMEOUT);
        return false;
    }
    return true;
}

template <int KS, int NK>
__global__ void __launch_bounds__(TC_THREADS, 1) subtract_tc_kernel(SubArgs a, int* status) {
    constexpr int R = (KS - 1) / 2;
    constexpr int NCOL = KS * NK;                // used MMA columns, <= 128
    constexpr int SOFF = (4 - R % 4) % 4;        // srcf[.][SOFF + c] = R(x0 - R + c)
    static_assert(NCOL <= 128 && KS <= TKC, "tile shape");
    static_assert(SOFF + SRCW <= SRCC * 4, "staged row");
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>(
        tc_smem_raw + ((1024 - (tc::smem_u32(tc_smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * TCX, y0 = blockIdx.y * TCY;
    const int nout = min(TCY, a.h - y0);
    const int nsrc = nout + 2 * R;   // source rows y0 - R .. y0 + nout - 1 + R

    // ---- set-up: B (hi/lo) from the kernel taps, barriers, TMEM
    // B column n = iv * NK + k
    for (int e = tid; e < 128 * TKC; e += TC_THREADS) {
        const int n = e / TKC, u = e - n * TKC;
        float v = 0.0f;
        if (n < NCOL && u < KS) {
            const int iv = n / NK, k = n - iv * NK;
            v = __ldg(a.K + k * KS * KS + iv * KS + (KS - 1 - u));
        }
        __nv_bfloat16 hi, lo;
        split_bf16(v, hi, lo);
        *reinterpret_cast<__nv_bfloat16*>(S.bhi + canon_off(n, u)) = hi;
        *reinterpret_cast<__nv_bfloat16*>(S.blo + canon_off(n, u)) = lo;
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; s++) {
            tc::mbar_init(&S.filled[s], 1);
            tc::mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < NTB; b++) {
            tc::mbar_init(&S.tfull[b], 1);
            tc::mbar_init(&S.tempty[b], 4);   // one arrival per epilogue warp
        }
        S.abort = 0;
        S.pstop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, 128 * NTB);
    tc::fence_proxy_async();   // B tiles written through the generic proxy
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = S.tmem;

    if (warp >= 4 && warp < MMA_WARP) {
        // ---------------- producers.  Row t of the stored A operand (16 bytes) holds
        // the 8 values R(x0 - R + t + b), b = 0..7: core matrix t >> 3, its row t & 7.
        // Producer t < NBUILD writes row t of the current source row from the staged
        // floats (each value is split into hi/lo where it is used); producers
        // c < SRCC fetch chunk c of source row rho + DP.
        const int pt = tid - 128;
        const int XS = x0 - R - SOFF;            // frame column of srcf[.][0], a multiple of 4
        // chunk pt of source row rr into its ring slot (zero outside the image; the
        // chunk holding column w is partly zero-filled)
        auto issue = [&](int rr) {
            if (pt < SRCC) {
                const int gy = y0 - R + rr, X = XS + 4 * pt;
                const int nb = (rr < nsrc && gy >= 0 && gy < a.h && X >= 0 && X < a.w) ? 4 * min(4, a.w - X) : 0;
                tc::cp_async16(&S.srcf[rr & (NSRC - 1)][4 * pt], nb ? a.ref + (long)gy * a.pitch + X : a.ref, nb);
            }
            tc::cp_async_commit();
        };
        for (int d = 0; d < DP; d++) issue(d);
        tc::cp_async_wait<DP - 2>();             // rows 0 and 1
        // One barrier per row.  Before barrier rho: every producer holds its chunk
        // of row rho + 1 landed and has written and fenced its part of row
        // rho - 1's tile; producer 0 has found stage s(rho) free.  After it,
        // producer 0 marks stage s(rho - 1) filled, the producers fetch row
        // rho + DP and build row rho.
        for (int rho = 0; rho < nsrc; rho++) {
            const int s = rho % NSTAGE, fill = rho / NSTAGE;
            if (pt == 0) {
                bool ok = !S.abort;
                if (ok && fill >= 1) ok = wait_or_abort(S, &S.empty[s], (fill - 1) & 1, status);
                S.pstop = ok ? 0 : 1;
            }
            tc::named_sync(1, NPROD);
            if (pt == 0 && rho >= 1) tc::mbar_arrive(&S.filled[(rho - 1) % NSTAGE]);
            if (S.pstop) break;
            issue(rho + DP);                     // may be past the band: zero-filled, never used
            if (pt < NBUILD) {
                const float* src = S.srcf[rho & (NSRC - 1)] + SOFF + pt;
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; k++) v[k] = src[k];
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int k = 0; k < 4; k++) split_pair(v[2 * k], v[2 * k + 1], hw[k], lw[k]);
                *reinterpret_cast<uint4*>(S.ahi[s] + 16 * pt) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(S.alo[s] + 16 * pt) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                tc::fence_proxy_async();
            }
            tc::cp_async_wait<DP - 2>();         // own chunk of row rho + 2 has landed
            if (rho == nsrc - 1) {               // the last tile: one more barrier to publish it
                tc::named_sync(1, NPROD);
                if (pt == 0) tc::mbar_arrive(&S.filled[s]);
            }
        }
        tc::cp_async_wait<0>();
    } else if (warp >= MMA_WARP) {
        // ---------------- MMA issuers: warp MMA_WARP + q takes the rows rho = q mod 2
        // (its own stages and TMEM buffers; the issuing thread is held for about
        // the MMAs' execution time, so two issuers keep the tensor pipe fed while
        // each waits on its barriers)
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(1, 128, 128);
            const uint32_t bh = tc::smem_u32(S.bhi), bl = tc::smem_u32(S.blo);
            int issued = 0;
            for (int rho = warp - MMA_WARP; rho < nsrc; rho += 2) {
                const int s = rho % NSTAGE, b = rho % NTB;
                if (!wait_or_abort(S, &S.filled[s], (rho / NSTAGE) & 1, status)) break;
                if (rho >= NTB && !wait_or_abort(S, &S.tempty[b], (rho / NTB - 1) & 1, status)) break;
                tc::fence_after();
                const uint32_t ahs = tc::smem_u32(S.ahi[s]), als = tc::smem_u32(S.alo[s]);
                const uint32_t d = tmem + (uint32_t)(b * 128);
#pragma unroll
                for (int kh = 0; kh < 2; kh++) {   // two K = 16 halves: K groups 2 kh, 2 kh + 1
                    const uint32_t ko = kh * 2 * LBO;
                    const uint64_t ad_h = tc::smem_desc(ahs + ko, LBO, SBO_A), ad_l = tc::smem_desc(als + ko, LBO, SBO_A);
                    const uint64_t bd_h = tc::smem_desc(bh + ko, LBO, SBO_B), bd_l = tc::smem_desc(bl + ko, LBO, SBO_B);
                    tc::mma_bf16(d, ad_h, bd_h, idesc, kh > 0 ? 1u : 0u);
                    tc::mma_bf16(d, ad_h, bd_l, idesc, 1u);
                    tc::mma_bf16(d, ad_l, bd_h, idesc, 1u);
                }
                tc::commit(&S.empty[s]);
                tc::commit(&S.tfull[b]);
                issued = rho + 1;
            }
            // every issued MMA must land before TMEM is released (a commit
            // tracks all earlier MMAs of this thread, so its last one suffices)
            if (issued > 0) {
                const int last = issued - 1;
                if (!tc::mbar_wait_bounded(&S.tfull[last % NTB], (last / NTB) & 1, WAIT_LIMIT)) {
                    S.abort = 1;
                    argus_latch(status, ARGUS_ERR_TIMEOUT);
                }
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------- epilogue: output column x0 + tid
        const int m = tid, x = x0 + m;
        const float xt = a.W > 1 ? (float)(2 * (x + a.ox) - (a.W - 1)) / (float)(a.W - 1) : 0.0f;
        // yt = 2 (y + oy) / (H - 1) - 1; the background as B0 + B1 yt + B2 yt^2 with the
        // x terms of this column folded into B0 and B1
        const float ysc = a.H > 1 ? 2.0f / (float)(a.H - 1) : 0.0f;
        const float yof = a.H > 1 ? -1.0f : 0.0f;
        float B0 = 0.0f, B1 = 0.0f, B2 = 0.0f;
        if (a.nbg == 6) {
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
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        // p_k = xt^i yt^j: the xt^i factor is fixed for this column, so each T
        // column enters the ring already multiplied by it and the ring keeps
        // one sum per power of yt (NJ = degree + 1) instead of one per term
        constexpr int NJ = NK == 1 ? 1 : (NK == 3 ? 2 : 3);
        constexpr int RL = KS + U - 1;
        const float xp[3] = {1.0f, xt, xt * xt};
        float acc[RL][NJ];
#pragma unroll
        for (int i = 0; i < RL; i++)
#pragma unroll
            for (int j = 0; j < NJ; j++) acc[i][j] = 0.0f;
        // science value and flag word of output row eta into slot eta & (NQ - 1),
        // one cp.async group per row (the pitch is a multiple of 16, so the flag
        // byte sits at byte x & 3 of its word)
        auto fetch = [&](int eta) {
            const bool in = eta >= 0 && eta < nout && x < a.w;
            const long p = in ? (long)(y0 + eta) * a.pitch + x : 0;
            const int slot = eta & (NQ - 1);
            tc::cp_async4(&S.qI[slot][m], a.sci + p, in ? 4 : 0);
            tc::cp_async4(&S.qF[slot][m], a.flags + (p & ~3L), in ? 4 : 0);
            tc::cp_async_commit();
        };
        const int fsh = 8 * (x & 3);
#pragma unroll 1
        for (int i = 0; i < LQ; i++) fetch(i - 2 * R);
        // ring index i holds output row rb - 2r + i for the current block start rb;
        // source row rb + u adds its column (iv, k) at index u + iv, and output row
        // rb + u - 2r is then complete at index u
        bool run = true;
#pragma unroll 1
        for (int rb = 0; rb < nsrc && run; rb += U) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int rho = rb + u;
                if (rho < nsrc && run) {
                    const int eta = rho - 2 * R;
                    fetch(eta + LQ);
                    const int b = rho % NTB;
                    // lane 0 waits (fewer pollers on the barrier), the warp follows
                    bool ok = true;
                    if (lane == 0) ok = wait_or_abort(S, &S.tfull[b], (rho / NTB) & 1, status);
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) {
                        run = false;
                    } else {
                        tc::fence_after();
#pragma unroll
                        for (int c2 = 0; c2 < 4; c2++) {
                            if (c2 * 32 < NCOL) {
                                uint32_t r0[16], r1[16];
                                tc::tmem_ld16_nowait(tl + (uint32_t)(b * 128 + c2 * 32), r0);
                                if (c2 * 32 + 16 < NCOL) {
                                    tc::tmem_ld16_nowait(tl + (uint32_t)(b * 128 + c2 * 32 + 16), r1);
                                } else {
#pragma unroll
                                    for (int j = 0; j < 16; j++) r1[j] = 0u;
                                }
                                tc::tmem_wait_ld(r0, r1);
#pragma unroll
                                for (int j = 0; j < 32; j++) {
                                    const int n = c2 * 32 + j;
                                    if (n < NCOL) {
                                        const int iv = n / NK, k = n - iv * NK;
                                        // term k of 1, y, y^2, x, x y, x^2 (or 1, y, x) as (i, j)
                                        const int ti = NK == 6 ? (k < 3 ? 0 : (k < 5 ? 1 : 2)) : (NK == 3 ? (k == 2) : 0);
                                        const int tj = NK == 6 ? (k < 3 ? k : (k == 4 ? 1 : 0)) : (NK == 3 ? (k == 1) : 0);
                                        const float v = __uint_as_float(j < 16 ? r0[j] : r1[j - 16]);
                                        acc[u + iv][tj] = fmaf(xp[ti], v, acc[u + iv][tj]);
                                    }
                                }
                            }
                        }
                        tc::fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&S.tempty[b]);
                        tc::cp_async_wait<LQ>();         // row eta's group has landed
                        if (eta >= 0 && eta < nout && x < a.w) {
                            const int slot = eta & (NQ - 1);
                            const float I = S.qI[slot][m];
                            const uint32_t fl = (S.qF[slot][m] >> fsh) & 0xffu;
                            const int y = y0 + eta;
                            const float yt = fmaf((float)(y + a.oy), ysc, yof);
                            // model = (acc0 + B0) + (acc1 + B1) yt + (acc2 + B2) yt^2
                            float c2 = B2, c1 = B1;
                            if constexpr (NJ > 2) c2 += acc[u][2];
                            if constexpr (NJ > 1) c1 += acc[u][1];
                            const float model = fmaf(fmaf(c2, yt, c1), yt, acc[u][0] + B0);
                            const bool inner = xin && y >= R && y <= a.h - 1 - R && fl == 0;
                            a.diff[(long)y * a.pitch + x] = inner ? I - model : 0.0f;
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i + U < RL; i++)
#pragma unroll
                for (int j = 0; j < NJ; j++) acc[i][j] = acc[i + U][j];
#pragma unroll
            for (int i = RL - U; i < RL; i++)
#pragma unroll
                for (int j = 0; j < NJ; j++) acc[i][j] = 0.0f;
        }
        tc::cp_async_wait<0>();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 128 * NTB);
}

template <int KS, int NK>
int launch_tc(const SubArgs& a, int* status, cudaStream_t st) {
    // more than half the shared memory: one CTA per SM, which holds all 512 TMEM columns
    size_t smem = sizeof(TcShared) + 1024;
    if (smem < 116 * 1024) smem = 116 * 1024;
    if (cudaFuncSetAttribute(subtract_tc_kernel<KS, NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return ARGUS_ERR_CUDA;
    dim3 grid((a.w + TCX - 1) / TCX, (a.h + TCY - 1) / TCY);
    subtract_tc_kernel<KS, NK><<<grid, TC_THREADS, smem, st>>>(a, status); argus_count_launch(1);
    return argus_launch_status();
}

}  // namespace

// Difference image on the tensor cores for the kernel sizes it is built for;
// returns ARGUS_ERR_UNSUPPORTED for the others (the caller uses the SIMT body).
int argus_subtract_tc(const SubArgs& a, int ksize, int nk, int* status, cudaStream_t st) {
    if (ksize == 21) {
        if (nk == 1) return launch_tc<21, 1>(a, status, st);
        if (nk == 3) return launch_tc<21, 3>(a, status, st);
        if (nk == 6) return launch_tc<21, 6>(a, status, st);
    }
    if (ksize == 11) {
        if (nk == 1) return launch_tc<11, 1>(a, status, st);
        if (nk == 3) return launch_tc<11, 3>(a, status, st);
        if (nk == 6) return launch_tc<11, 6>(a, status, st);
    }
    return ARGUS_ERR_UNSUPPORTED;
}
