// qld_block.cuh -- block-mode push: a push of at least N frames into a small
// frame, where the window is rebuilt from the pushed frames alone.
//
// The single-stream push gives each thread one pixel vector and walks every
// pushed frame in turn: right for wide frames, but a 128 x 128 frame has only
// 1024 such vectors, and a thread then waits out the latency of N / 4 load
// groups one after the other. Here a thread owns one 8-pixel vector and one
// of TS time slices (the frames f with f mod TS = its slice): each thread
// issues its few loads at once, writes each frame into its ring slot, and
// keeps exact int32 partial sums; the partial sums of the slices are added in
// shared memory (integer adds: the order cannot change the result), and the
// sums and the image are written as by push_vector<T, RESET = true, EPI>.
// The paper's QLD image from a stack of N frames (Methods, R(j,k)).

#pragma once

#include "qld_kernels.cuh"

namespace qldk {

// 32 vectors (one warp per time slice, so a warp's frames share their index
// residue mod 4 and the sign pattern of accumulate does not diverge) times 16
// time slices.
constexpr int kBlockPV = 32;
constexpr int kBlockTS = 16;
constexpr int kBlockThreads = kBlockPV * kBlockTS;

// a.nvec counts Fmt<T> vectors of 8 pixels (T = uint16_t, u8h_t or p12h_t);
// a.nf frames of the window, frame f of absolute index a.s_first + f.
template <typename T, bool EPI>
__global__ void __launch_bounds__(kBlockThreads) block_push_kernel(const PushArgs a) {
    using F = Fmt<T>;
    constexpr int VP = F::VP;
    static_assert(VP == 8, "8-pixel vectors");
    // partial sums [slice][S | C][vector][pixel], the pixel row padded to 9
    // words so that neither the writes nor the reads collide on a bank
    __shared__ int32_t part[kBlockTS][2][kBlockPV][VP + 1];
    const int pv = threadIdx.x % kBlockPV, ts = threadIdx.x / kBlockPV;
    const long long v = (long long)blockIdx.x * kBlockPV + pv;
    int32_t sacc[VP], cacc[VP];
#pragma unroll
    for (int q = 0; q < VP; ++q) sacc[q] = cacc[q] = 0;
    if (v < a.nvec) {
        const uint8_t* src = a.frames + v * F::VB;
        uint8_t* ring = a.ring + v * F::VB;
        int f = ts;
        // four frames at a time, all loads issued before the stores
        for (; f + 3 * kBlockTS < a.nf; f += 4 * kBlockTS) {
            typename F::Vec x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = F::load(src + (long long)(f + u * kBlockTS) * a.frame_stride);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long s = a.s_first + f + u * kBlockTS;
                F::store(ring + (s % a.N) * a.slot_stride, x[u]);
                accumulate<T, false>(sacc, cacc, x[u], x[u], (int)(s & 3));
            }
        }
        for (; f < a.nf; f += kBlockTS) {
            const typename F::Vec x = F::load(src + (long long)f * a.frame_stride);
            const long long s = a.s_first + f;
            F::store(ring + (s % a.N) * a.slot_stride, x);
            accumulate<T, false>(sacc, cacc, x, x, (int)(s & 3));
        }
    }
#pragma unroll
    for (int q = 0; q < VP; ++q) {
        part[ts][0][pv][q] = sacc[q];
        part[ts][1][pv][q] = cacc[q];
    }
    __syncthreads();
    // one pixel per thread: pixel j of the CTA's kBlockPV * VP = 256
    if (threadIdx.x < kBlockPV * VP) {
        const int j = threadIdx.x, jv = j / VP, jq = j % VP;
        const long long p = (long long)blockIdx.x * kBlockPV * VP + j;
        if ((long long)blockIdx.x * kBlockPV + jv < a.nvec) {
            int32_t S = 0, C = 0;
#pragma unroll
            for (int t = 0; t < kBlockTS; ++t) {
                S += part[t][0][jv][jq];
                C += part[t][1][jv][jq];
            }
            a.S[p] = S;
            a.C[p] = C;
            if (EPI) {
                if (a.amp) a.amp[p] = amplitude(S, C);
                if (a.phase) a.phase[p] = phase_of(S, C);
            }
        }
    }
}

}  // namespace qldk
