// Runs the FFT row/column kernels' work on the CPU, thread by thread: the
// same butterflies and Stockham pass (fft.cuh, host-callable) with the
// kernels' load/store mapping.  Within a pass the threads write disjoint
// outputs and read only the previous pass, so running them in sequence with
// the pass boundary as the barrier gives the kernels' results.
#pragma once
#include <vector>
#include <utility>
#include "fft.cuh"
using namespace fft;

template <int T, int S, bool COLS, typename R>
void host_pass(typename Cx<R>::T* data, int n_tiles, const typename Cx<R>::T* twg) {
    using C = typename Cx<R>::T;
    using Sh = Shape<T, R>;
    std::vector<C> smem(2 * Sh::SEQ * Sh::PAD + T);
    C* buf = smem.data();
    C* tw = buf + 2 * Sh::SEQ * Sh::PAD;
    const long blocks_per_tile = T / Sh::SEQ;
    for (long blk = 0; blk < n_tiles * blocks_per_tile; blk++) {
        for (int i = 0; i < T; i++) tw[i] = twg[i];
        const long tile = blk / blocks_per_tile;
        const int s0 = (int)(blk % blocks_per_tile) * Sh::SEQ;
        C* base = data + tile * (long)T * T;
        for (int e = 0; e < Sh::SEQ * T; e++) {
            if (COLS) { const int y = e / Sh::SEQ, c = e - y * Sh::SEQ; buf[c * Sh::PAD + y] = base[(long)y * T + s0 + c]; }
            else { const int s = e / T, x = e - s * T; buf[s * Sh::PAD + x] = base[(long)(s0 + s) * T + x]; }
        }
        // stockham(): passes with a barrier between them
        std::vector<C*> A(Sh::SEQ), B(Sh::SEQ);
        for (int q = 0; q < Sh::SEQ; q++) { A[q] = buf + q * Sh::PAD; B[q] = buf + (Sh::SEQ + q) * Sh::PAD; }
        int Ns = 1;
        while (Ns < T) {
            int rad = Ns * 8 <= T ? 8 : (Ns * 4 <= T ? 4 : 2);
            for (int tid = 0; tid < Sh::THREADS; tid++) {
                const int seq = tid / Sh::LANES, lane = tid - seq * Sh::LANES;
                if (rad == 8) stockham_pass<T, 8, S>(A[seq], B[seq], tw, Ns, lane, Sh::LANES);
                else if (rad == 4) stockham_pass<T, 4, S>(A[seq], B[seq], tw, Ns, lane, Sh::LANES);
                else stockham_pass<T, 2, S>(A[seq], B[seq], tw, Ns, lane, Sh::LANES);
            }
            Ns *= rad;
            for (int q = 0; q < Sh::SEQ; q++) std::swap(A[q], B[q]);
        }
        const bool in_first = A[0] == buf;
        C* out = in_first ? buf : buf + Sh::SEQ * Sh::PAD;
        for (int e = 0; e < Sh::SEQ * T; e++) {
            if (COLS) { const int y = e / Sh::SEQ, c = e - y * Sh::SEQ; base[(long)y * T + s0 + c] = out[c * Sh::PAD + y]; }
            else { const int s = e / T, x = e - s * T; base[(long)(s0 + s) * T + x] = out[s * Sh::PAD + x]; }
        }
    }
}

