// qld_internal.h -- definitions shared by the library's translation units
// (not part of the C ABI).

#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

struct qld_ctx {
    int H, W, N, pixfmt;
    long long frame_bytes;  // bytes of one frame (of the band) in the input format
    // Row band of a larger frame (qld_create_band): the caller's frames are
    // H_total x W, this context owns rows row0 .. row0 + H - 1. Frame f of a
    // device push starts band_offset + f * frame_pitch bytes into the
    // caller's buffer. A whole-frame context has H_total = H, row0 = 0,
    // band_offset = 0 and frame_pitch = frame_bytes.
    int H_total, row0;
    long long band_offset, frame_pitch;
    long long npix;
    long long npad;         // padded pixel count of S and C
    long long slot_stride;  // bytes
    int device;
    uint8_t* ring;
    int32_t* S;
    int32_t* C;
    float2* tw;
    int tw_k;               // bin whose twiddles are in tw, -1 if none
    long long pushed;
    cudaStream_t stream;
    long long footprint;
    // host-buffer variants (created on first use)
    struct HostPipe* pipe;
};

// Device staging for the host-buffer calls. Frames go host -> stage[i] on
// the copy-in stream, the push reads stage[i] on the context's stream;
// images go to out[o] on the context's stream and out[o] -> host on the
// copy-out stream. Two input stages and four output buffers, each guarded by
// a ready / free event pair, let the copies of one step overlap the kernels
// of the next and previous steps.
struct HostPipe {
    static constexpr int kIn = 2, kOut = 4;
    cudaStream_t cin, cout;
    uint8_t* stage[kIn];
    long long stage_bytes;
    cudaEvent_t in_ready[kIn], in_free[kIn];
    float* out[kOut];
    long long out_elems;
    cudaEvent_t out_ready[kOut], out_free[kOut];
    int in_idx, out_idx;
};

namespace qldi {
// Records a non-OK status as the calling thread's last error; returns it.
int set_err(int status);
// Adds n to the library's kernel launch counter (qld_launch_count).
void count_launches(int n);
// Bytes of one frame / of one kernel vector, and the vector path's pointer
// alignment, per pixel format.
long long frame_bytes_of(long long npix, int pixfmt);
int vec_bytes_of(int pixfmt);
unsigned vec_align_of(int pixfmt);
}  // namespace qldi
