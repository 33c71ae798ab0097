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
// epilogue warps add T into a ring of KS pending output rows (one register
// set per row) and finish a row once its last source row is in.  Operands are BF16
// hi/lo pairs (v = hi + lo, each rounded to nearest) and every product is
// hi*hi + hi*lo + lo*hi, accumulated in FP32 in TMEM: the dropped lo*lo
// term is below 2^-16 relative, well inside FP32-level agreement.
//
// CTA: 128 columns x a band of TCY output rows, streaming the band's
// TCY + 2r source rows.  Warps 0-3: epilogue, one output column per thread
// and TMEM lane, holding the ring of pending rows in registers (one sum per
// power of y: the x powers are folded in as each T column is added; the ring
// shifts by register moves, so the row loop has a single body).  Warps 4-10:
// producers (source rows arrive by cp.async DP rows ahead; each value is
// split into BF16 hi/lo once, one row ahead of its use, and the Hankel rows
// are copied out of the split row with 32-bit loads and byte permutes into
// the canonical no-swizzle K-major layout, NSTAGE stages; one named barrier
// per row).  Warp 11: one thread issues the MMAs.  TMEM holds four
// 128-column accumulators, so the MMAs run up to three rows ahead of the
// epilogue, which loads its science and flag values four rows ahead into a
// register queue.  Every wait is bounded; a timeout latches ARGUS_ERR_TIMEOUT
// and all roles stop.
#include <cuda_bf16.h>

#include "subtract_tile.cuh"
#include "tc_ptx.cuh"

namespace {
using namespace argus_sub;

constexpr int TCX = 128;                  // output columns per CTA (MMA M)
constexpr int TCY = 128;                  // output rows per CTA band
constexpr int TKC = 32;                   // MMA K: taps u', padded
constexpr int NSTAGE = 4;                 // Hankel stages
constexpr int SRCW = TCX + TKC;           // source columns per row
constexpr int NSRC = 8;                   // fp32 source-row ring
constexpr int DP = 6;                     // source rows in flight ahead of the one being tiled
constexpr int NPROD = 224;                // producer threads (warps 4-10)
constexpr int TC_THREADS = 384;           // warps 0-3 epilogue, 4-10 producers, 11 MMA issuer
constexpr uint32_t LBO = 128, SBO = 512;  // K-major canonical layout, 32 K per row
constexpr uint32_t TILE_BYTES = 128 * TKC * 2;
constexpr long long WAIT_LIMIT = 2000000000LL;   // ~1 s of SM clock
constexpr int NTB = 4;                    // TMEM accumulator buffers of 128 columns

struct TcShared {
    uint8_t bhi[TILE_BYTES];
    uint8_t blo[TILE_BYTES];
    uint8_t ahi[NSTAGE][TILE_BYTES];
    uint8_t alo[NSTAGE][TILE_BYTES];
    float srcf[NSRC][SRCW];
    alignas(16) uint32_t srch[2][SRCW / 2 + 4];   // BF16 hi of a source row, two per word (double-buffered)
    alignas(16) uint32_t srcl[2][SRCW / 2 + 4];   // BF16 lo
    uint64_t filled[NSTAGE];
    uint64_t empty[NSTAGE], tfull[NTB], tempty[NTB];
    uint32_t tmem;
    int abort;       // set by any role that timed out
    int pstop;       // producers' common decision, written by producer 0 between barriers
};

__device__ __forceinline__ uint32_t canon_off(int row, int kk) {
    return (uint32_t)(row >> 3) * SBO + (uint32_t)(kk >> 3) * LBO + (uint32_t)(row & 7) * 16 + (uint32_t)(kk & 7) * 2;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__device__ __forceinline__ bool wait_or_abort(TcShared& S, uint64_t* bar, uint32_t parity, int* status) {
    if (S.abort) return false;
    if (!tc::mbar_wait_bounded(bar, parity, WAIT_LIMIT)) {
        S.abort = 1;
        argus_latch(status, ARGUS_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// Background polynomial sum_k c_k p_k (p_k = x^i y^j, i + j <= deg, ordered i then
// j: 1, y, y^2, x, x y, x^2), written out so nothing is indexed at run time.
__device__ __forceinline__ float background(const float (&c)[6], int nbg, float xt, float yt) {
    if (nbg == 6) return fmaf(c[5], xt * xt, fmaf(c[4], xt * yt, fmaf(c[3], xt, fmaf(c[2], yt * yt, fmaf(c[1], yt, c[0])))));
    if (nbg == 3) return fmaf(c[2], xt, fmaf(c[1], yt, c[0]));
    if (nbg == 1) return c[0];
    return 0.0f;
}

template <int KS, int NK>
__global__ void __launch_bounds__(TC_THREADS, 1) subtract_tc_kernel(SubArgs a, int* status) {
    constexpr int R = (KS - 1) / 2;
    constexpr int NCOL = KS * NK;   // used MMA columns, <= 128
    static_assert(NCOL <= 128 && KS <= TKC, "tile shape");
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    TcShared& S = *reinterpret_cast<TcShared*>(
        tc_smem_raw + ((1024 - (tc::smem_u32(tc_smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * TCX, y0 = blockIdx.y * TCY;
    const int nout = min(TCY, a.h - y0);
    const int nsrc = nout + 2 * R;   // source rows y0 - R .. y0 + nout - 1 + R

    // ---- set-up: B (hi/lo) from the kernel taps, barriers, TMEM, first source rows
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

    if (warp >= 4 && warp < 11) {
        // ---------------- producers: warps 8-10 fetch and split source rows one row
        // ahead, warps 4-7 build the Hankel tile of the current row (one row m each)
        const int pt = tid - 128;
        const bool splitter = pt >= TCX;
        const int ps = pt - TCX;                 // splitter index, 0 .. 95
        constexpr int NSPLIT = NPROD - TCX;
        // source row rr into its ring slot with cp.async (zero outside the image)
        auto issue_row = [&](int rr) {
            for (int c = ps; c < SRCW; c += NSPLIT) {
                const int gy = y0 - R + rr, gx = x0 - R + c;
                const bool in = rr < nsrc && gy >= 0 && gy < a.h && gx >= 0 && gx < a.w;
                tc::cp_async4(&S.srcf[rr & (NSRC - 1)][c], in ? a.ref + (long)gy * a.pitch + gx : a.ref, in ? 4 : 0);
            }
        };
        // BF16 split of source row rr into buffer rr & 1, two values per word
        auto split_row = [&](int rr) {
            const float2* src = reinterpret_cast<const float2*>(S.srcf[rr & (NSRC - 1)]);
            uint32_t* dh = S.srch[rr & 1];
            uint32_t* dl = S.srcl[rr & 1];
            for (int i = ps; i < SRCW / 2; i += NSPLIT) {
                const float2 v = src[i];
                __nv_bfloat16 h0, l0, h1, l1;
                split_bf16(v.x, h0, l0);
                split_bf16(v.y, h1, l1);
                dh[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                dl[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
        };
        if (splitter) {
            for (int d = 0; d < DP; d++) {
                issue_row(d);
                tc::cp_async_commit();
            }
            tc::cp_async_wait<DP - 2>();         // rows 0 and 1
        }
        tc::named_sync(1, NPROD);
        if (splitter) split_row(0);
        // One barrier per row.  Before barrier rho: the splitters have split row rho
        // and hold row rho + 1 landed; the builders have built and fenced row
        // rho - 1's tile; producer 0 has found stage s(rho) free.  After it,
        // producer 0 marks stage s(rho - 1) filled, the splitters split row
        // rho + 1 and fetch row rho + DP + 1, the builders build row rho.
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
            if (splitter) {
                if (rho + 1 < nsrc) split_row(rho + 1);
                issue_row(rho + DP);             // may be past the band: zero-filled, never used
                tc::cp_async_commit();
                tc::cp_async_wait<DP - 2>();     // row rho + 2 has landed
            } else {
                // Hankel row m: A[m][u'] = src[m + u'], chunk q = taps 8q .. 8q+7 as four
                // words taken from src words (m >> 1) + 4q .. + 4 (shifted by one value
                // when m is odd)
                const int m = pt;
                uint8_t* ah = S.ahi[s];
                uint8_t* al = S.alo[s];
                const uint32_t* sh = S.srch[rho & 1];
                const uint32_t* sl = S.srcl[rho & 1];
                const int w0 = m >> 1;
                const uint32_t sel = (m & 1) ? 0x5432u : 0x3210u;
                uint32_t hw[17], lw[17];
#pragma unroll
                for (int k = 0; k < 17; k++) {
                    hw[k] = sh[w0 + k];
                    lw[k] = sl[w0 + k];
                }
#pragma unroll
                for (int q = 0; q < TKC / 8; q++) {
                    const uint32_t off = canon_off(m, 8 * q);
                    *reinterpret_cast<uint4*>(ah + off) =
                        make_uint4(__byte_perm(hw[4 * q], hw[4 * q + 1], sel), __byte_perm(hw[4 * q + 1], hw[4 * q + 2], sel),
                                   __byte_perm(hw[4 * q + 2], hw[4 * q + 3], sel), __byte_perm(hw[4 * q + 3], hw[4 * q + 4], sel));
                    *reinterpret_cast<uint4*>(al + off) =
                        make_uint4(__byte_perm(lw[4 * q], lw[4 * q + 1], sel), __byte_perm(lw[4 * q + 1], lw[4 * q + 2], sel),
                                   __byte_perm(lw[4 * q + 2], lw[4 * q + 3], sel), __byte_perm(lw[4 * q + 3], lw[4 * q + 4], sel));
                }
                tc::fence_proxy_async();
            }
            if (rho == nsrc - 1) {               // the last tile: one more barrier to publish it
                tc::named_sync(1, NPROD);
                if (pt == 0) tc::mbar_arrive(&S.filled[s]);
            }
        }
        if (splitter) tc::cp_async_wait<0>();
    } else if (warp == 11) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(1, 128, 128);
            const uint32_t bh = tc::smem_u32(S.bhi), bl = tc::smem_u32(S.blo);
            int issued = 0;
            for (int rho = 0; rho < nsrc; rho++) {
                const int s = rho % NSTAGE, b = rho % NTB;
                if (!wait_or_abort(S, &S.filled[s], (rho / NSTAGE) & 1, status)) break;
                if (rho >= NTB && !wait_or_abort(S, &S.tempty[b], (rho / NTB - 1) & 1, status)) break;
                tc::fence_after();
                const uint32_t ahs = tc::smem_u32(S.ahi[s]), als = tc::smem_u32(S.alo[s]);
                const uint32_t d = tmem + (uint32_t)(b * 128);
#pragma unroll
                for (int kh = 0; kh < 2; kh++) {   // two K = 16 halves
                    const uint32_t ko = kh * 2 * LBO;
                    tc::mma_bf16(d, tc::smem_desc(ahs + ko, LBO, SBO), tc::smem_desc(bh + ko, LBO, SBO), idesc,
                                 kh > 0 ? 1u : 0u);
                    tc::mma_bf16(d, tc::smem_desc(ahs + ko, LBO, SBO), tc::smem_desc(bl + ko, LBO, SBO), idesc, 1u);
                    tc::mma_bf16(d, tc::smem_desc(als + ko, LBO, SBO), tc::smem_desc(bh + ko, LBO, SBO), idesc, 1u);
                }
                tc::commit(&S.empty[s]);
                tc::commit(&S.tfull[b]);
                issued = rho + 1;
            }
            // every issued MMA must land before TMEM is released (a commit
            // tracks all earlier MMAs of this thread, so the last one suffices)
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
        float bgc[6];
#pragma unroll
        for (int k = 0; k < 6; k++) bgc[k] = k < a.nbg ? (float)a.bg[k] : 0.0f;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        // p_k = xt^i yt^j: the xt^i factor is fixed for this column, so each T
        // column enters the ring already multiplied by it and the ring keeps
        // one sum per power of yt (NJ = degree + 1) instead of one per term
        constexpr int NJ = NK == 1 ? 1 : (NK == 3 ? 2 : 3);
        const float xp[3] = {1.0f, xt, xt * xt};
        float acc[KS][NJ];
#pragma unroll
        for (int i = 0; i < KS; i++)
#pragma unroll
            for (int j = 0; j < NJ; j++) acc[i][j] = 0.0f;
        // science value and flags of output rows eta .. eta + LQ - 1 in a register FIFO,
        // loaded LQ rows before use
        constexpr int LQ = 4;
        float qI[LQ];
        int qF[LQ];
        auto load_out = [&](int rr, float& Iv, int& Fv) {
            const bool in = rr >= 0 && rr < nout && x < a.w;
            const long pp = in ? (long)(y0 + rr) * a.pitch + x : 0;
            Iv = in ? __ldg(a.sci + pp) : 0.0f;
            Fv = in ? (int)__ldg(a.flags + pp) : 1;
        };
#pragma unroll
        for (int i = 0; i < LQ; i++) load_out(i - 2 * R, qI[i], qF[i]);
        // ring index i holds output row rho - 2r + i; source row rho adds its
        // column (iv, k) at index iv, row rho - 2r is then complete at index 0
        // and the ring shifts down by one (register moves, one loop body)
        for (int rho = 0; rho < nsrc; rho++) {
            const int eta = rho - 2 * R;
            const int y = y0 + eta;
            const bool out = eta >= 0 && x < a.w && y < a.h;
            const long p = out ? (long)y * a.pitch + x : 0;
            const float I = qI[0];
            const int fl = qF[0];
#pragma unroll
            for (int i = 0; i + 1 < LQ; i++) {
                qI[i] = qI[i + 1];
                qF[i] = qF[i + 1];
            }
            load_out(eta + LQ, qI[LQ - 1], qF[LQ - 1]);
            const int b = rho % NTB;
            bool run = wait_or_abort(S, &S.tfull[b], (rho / NTB) & 1, status);
            run = __all_sync(0xffffffffu, run);
            if (!run) break;
            tc::fence_after();
#pragma unroll
            for (int c = 0; c < 8; c++) {
                if (c * 16 < NCOL) {
                    float v[16];
                    tc::tmem_ld16(tl + (uint32_t)(b * 128 + c * 16), v);
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const int n = c * 16 + j;
                        if (n < NCOL) {
                            const int iv = n / NK, k = n - iv * NK;
                            // term k of 1, y, y^2, x, x y, x^2 (or 1, y, x) as (i, j)
                            const int ti = NK == 6 ? (k < 3 ? 0 : (k < 5 ? 1 : 2)) : (NK == 3 ? (k == 2) : 0);
                            const int tj = NK == 6 ? (k < 3 ? k : (k == 4 ? 1 : 0)) : (NK == 3 ? (k == 1) : 0);
                            acc[iv][tj] = fmaf(xp[ti], v[j], acc[iv][tj]);
                        }
                    }
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.tempty[b]);
            if (out) {
                float D = 0.0f;
                const bool inner = x >= R && y >= R && x <= a.w - 1 - R && y <= a.h - 1 - R;
                if (inner && fl == 0) {
                    const float yt = a.H > 1 ? (float)(2 * (y + a.oy) - (a.H - 1)) / (float)(a.H - 1) : 0.0f;
                    float conv = acc[0][0];
                    if constexpr (NJ > 1) conv = fmaf(acc[0][1], yt, conv);
                    if constexpr (NJ > 2) conv = fmaf(acc[0][2], yt * yt, conv);
                    D = I - conv - background(bgc, a.nbg, xt, yt);
                }
                a.diff[p] = D;
            }
#pragma unroll
            for (int i = 0; i + 1 < KS; i++)
#pragma unroll
                for (int j = 0; j < NJ; j++) acc[i][j] = acc[i + 1][j];
#pragma unroll
            for (int j = 0; j < NJ; j++) acc[KS - 1][j] = 0.0f;
        }
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
