// qld_batch.cuh -- one persistent launch that pushes frames into many
// streams of different sizes, windows and pixel formats.
//
// The paper's real-time loop acquires and processes frames of one camera as
// they arrive (SI, "Timing sequence for hybrid parallelisation"). Serving
// several cameras at once, each stream's push (ring update, exact int32 sums,
// amplitude/phase image) is the per-vector work of push_vec_kernel; here the
// vectors of every stream with pending frames form one list of tiles that a
// persistent grid walks, so uneven streams share one launch.

#pragma once

#include "qld_kernels.cuh"

namespace qldk {

// One stream's share of a batch.
struct BatchItem {
    PushArgs a;       // nvec counts batch_vec_bytes(fmt)-byte vectors (8 pixels each)
    int fmt;          // 1 = uint8, 2 = uint16, 3 = packed 12-bit
    int reset;        // the push holds at least N frames: rebuild the window
    int epi;          // write the amplitude / phase image after the push
    long long tile0;  // first tile of this item in the batch
};

struct BatchHeader {
    int nitems;
    int gated;         // 1: run only if the doorbell gate before it left *gate == 0
    long long ntiles;  // sum over items of ceil(nvec / tile vectors)
};

// Most items one launch carries.
constexpr int kMaxBatchItems = 64;

// A tick's descriptors, passed by value as the kernel's parameter: they reach
// every CTA through the constant cache with the launch itself, so a tick
// needs no host-to-device copy before its kernel and a CTA's search for its
// tile's item reads no global memory. ~9.5 KB, inside the 32 KB a kernel's
// parameters may take.
struct BatchParams {
    BatchHeader hdr;
    BatchItem items[kMaxBatchItems];
};
static_assert(sizeof(BatchParams) + 64 <= 32000, "batch descriptors exceed the kernel parameter space");

template <typename T>
__device__ __forceinline__ void push_vector_mode(const PushArgs& a, int reset, int epi, long long v) {
    if (reset) {
        if (epi) push_vector<T, true, true, false>(a, v);
        else push_vector<T, true, false, false>(a, v);
    } else {
        if (epi) push_vector<T, false, true, false>(a, v);
        else push_vector<T, false, false, false>(a, v);
    }
}

// Tile = NT * VPT consecutive vectors of one item; CTA b takes tiles b,
// b + gridDim.x, ... The item of a tile is found by binary search over the
// items' tile0 (the same for every thread of the CTA, so no divergence).
template <int NT, int VPT>
__global__ void __launch_bounds__(NT) batch_push_kernel(const __grid_constant__ BatchParams p, const int* gate) {
    if (p.hdr.gated && *(volatile const int*)gate != 0) return;  // the doorbell wait ran out: no work
    const int n = p.hdr.nitems;
    const long long ntiles = p.hdr.ntiles;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.items[mid].tile0 <= tile) lo = mid;
            else hi = mid - 1;
        }
        const BatchItem& it = p.items[lo];
        const PushArgs a = it.a;
        const int fmt = it.fmt, reset = it.reset, epi = it.epi;
        const long long vbase = (tile - it.tile0) * (long long)(NT * VPT);
#pragma unroll 1
        for (int k = 0; k < VPT; ++k) {
            const long long v = vbase + (long long)k * NT + threadIdx.x;
            if (v >= a.nvec) break;
            if (fmt == 2) push_vector_mode<uint16_t>(a, reset, epi, v);
            else if (fmt == 1) push_vector_mode<u8h_t>(a, reset, epi, v);
            else push_vector_mode<p12h_t>(a, reset, epi, v);
        }
    }
}

// Bytes of the 8-pixel vectors the batch kernel reads a pixel format in.
inline int batch_vec_bytes(int pixfmt) { return pixfmt == 2 ? 16 : (pixfmt == 1 ? 8 : 12); }

// Launch shapes the autotuner chooses from: threads per CTA, vectors per
// thread per tile, resident CTAs per SM of the persistent grid.
struct BatchShape {
    int threads, vpt, ctas_per_sm;
};

// ctas_per_sm = 0: one CTA per tile instead of a persistent grid (the grid
// is the number of tiles to cover; CTAs past the tick's tile count return at
// once), so the hardware overlaps consecutive tiles the way it overlaps the
// CTAs of the single-stream push.
constexpr BatchShape kBatchShapes[] = {{128, 1, 4}, {128, 2, 4}, {128, 4, 4}, {256, 1, 2}, {256, 2, 2}, {256, 1, 4},
                                       {128, 1, 8}, {64, 2, 8},  {128, 2, 8}, {256, 2, 4}, {128, 4, 8}, {128, 1, 0},
                                       {256, 1, 0}, {128, 2, 0}};
constexpr int kNumBatchShapes = (int)(sizeof(kBatchShapes) / sizeof(kBatchShapes[0]));

inline long long batch_tile_vectors(const BatchShape& s) { return (long long)s.threads * s.vpt; }

// `tiles`: the tiles a one-CTA-per-tile grid covers (unused by persistent
// shapes).
inline void launch_batch(const BatchShape& s, int num_sms, long long tiles, const BatchParams& p, const int* gate,
                         cudaStream_t st) {
    const unsigned grid = s.ctas_per_sm > 0 ? (unsigned)(num_sms * s.ctas_per_sm)
                                            : (unsigned)(tiles < 1 ? 1 : (tiles > 0x7FFFFFFF ? 0x7FFFFFFF : tiles));
    if (s.threads == 128 && s.vpt == 1) batch_push_kernel<128, 1><<<grid, 128, 0, st>>>(p, gate);
    else if (s.threads == 128 && s.vpt == 2) batch_push_kernel<128, 2><<<grid, 128, 0, st>>>(p, gate);
    else if (s.threads == 128 && s.vpt == 4) batch_push_kernel<128, 4><<<grid, 128, 0, st>>>(p, gate);
    else if (s.threads == 256 && s.vpt == 1) batch_push_kernel<256, 1><<<grid, 256, 0, st>>>(p, gate);
    else if (s.threads == 256 && s.vpt == 2) batch_push_kernel<256, 2><<<grid, 256, 0, st>>>(p, gate);
    else batch_push_kernel<64, 2><<<grid, 64, 0, st>>>(p, gate);
}

// Bounded device wait on a doorbell before a gated tick: one thread polls
// *doorbell with volatile loads (re-read every time, so a word in mapped
// host memory or one a copy engine writes is seen) until it reaches
// `target`, backing off with __nanosleep, for at most timeout_ns of
// %globaltimer time. *gate = 0 when the doorbell rang in time, 1 when the
// wait ran out; the tick launched after it on the same stream then does no
// work. Nothing else waits on this kernel's threads.
__global__ void doorbell_gate_kernel(const int* doorbell, int target, long long timeout_ns, int* gate) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (*(volatile const int*)doorbell >= target) {
            *gate = 0;
            return;
        }
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if ((long long)(t - t0) > timeout_ns) {
            *gate = 1;
            return;
        }
        __nanosleep(500);
    }
}

}  // namespace qldk
