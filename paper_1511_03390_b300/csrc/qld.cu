// qld.cu -- context management and the C ABI declared in include/qld.h.
//
// A context owns, in device memory:
//   ring   N slots of one frame each (slot stride padded to 256 bytes): the
//          sliding buffer of N frames (SI, closing paragraph);
//   S, C   int32 quadrature sums, padded to a multiple of 64 pixels
//          (SI "Timing sequence" item 3: the two 2-D accumulators);
//   tw     float2 twiddles of the last DFT bin requested (SI item 1: the
//          pre-calculated sine / cosine tables).
// Frame s (absolute, 1-based) lives in slot s mod N.

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <cuda_runtime.h>

#include "qld.h"
#include "qld_block.cuh"
#include "qld_kernels.cuh"

#include "qld_internal.h"

namespace qldi {

thread_local int g_last_error = QLD_OK;
std::atomic<long long> g_launches{0};

int set_err(int st) {
    if (st != QLD_OK) g_last_error = st;
    return st;
}

void count_launches(int n) { g_launches.fetch_add(n); }

}  // namespace qldi

using qldi::g_launches;
using qldi::set_err;

namespace {

std::atomic<long long> g_budget{0};
std::atomic<long long> g_in_use{0};

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

bool valid_dims(int H, int W, int N, int pixfmt) {
    if (H < 1 || W < 1 || N < 4 || N > QLD_MAX_N || (N % 4) != 0) return false;
    if (pixfmt != QLD_U8 && pixfmt != QLD_U16 && pixfmt != QLD_P12) return false;
    const long long npix = (long long)H * W;
    if (pixfmt == QLD_P12 && (npix % 2) != 0) return false;  // pixel pairs must not straddle frames
    return npix <= (1ll << 31) - 1;
}

}  // namespace

namespace qldi {
long long frame_bytes_of(long long npix, int pixfmt) { return pixfmt == QLD_P12 ? npix / 2 * 3 : npix * pixfmt; }
int vec_bytes_of(int pixfmt) { return pixfmt == QLD_P12 ? qldk::Fmt<qldk::p12_t>::VB : qldk::kVecBytes; }
unsigned vec_align_of(int pixfmt) { return pixfmt == QLD_P12 ? qldk::Fmt<qldk::p12_t>::ALIGN : 16u; }
}  // namespace qldi

using qldi::frame_bytes_of;
using qldi::vec_align_of;
using qldi::vec_bytes_of;

namespace {

struct Layout {
    long long npix, npad, slot_stride, ring_bytes, sums_bytes, tw_bytes, total;
};

Layout layout_of(int H, int W, int N, int pixfmt) {
    Layout L;
    L.npix = (long long)H * W;
    L.npad = round_up(L.npix, 64);
    // a whole number of kernel vectors, and 256-byte aligned slots
    L.slot_stride = round_up(round_up(frame_bytes_of(L.npix, pixfmt), vec_bytes_of(pixfmt)), 256);
    L.ring_bytes = L.slot_stride * N;
    L.sums_bytes = L.npad * (long long)sizeof(int32_t);
    L.tw_bytes = round_up((long long)N * (long long)sizeof(float2), 256);
    L.total = L.ring_bytes + 2 * L.sums_bytes + L.tw_bytes;
    return L;
}

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Any CUDA error raised since the last call (launch or asynchronous).
int pending_error() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QLD_OK : QLD_E_CUDA;
}

bool aligned(const void* p, unsigned a) { return ((uintptr_t)p % a) == 0; }

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <bool RESET, bool EPI>
void launch_push_t(const qld_ctx* c, const qldk::PushArgs& a, bool vec) {
    if (c->pixfmt == QLD_P12) {
        if (vec)
            qldk::push_vec_kernel<qldk::p12_t, RESET, EPI><<<blocks_for(a.nvec, 128), 128, 0, c->stream>>>(a);
        else
            qldk::push_scalar_p12_kernel<RESET, EPI><<<blocks_for(a.npix / 2, 256), 256, 0, c->stream>>>(a);
        return;
    }
    if (vec) {
        if (c->pixfmt == QLD_U16)
            qldk::push_vec_kernel<uint16_t, RESET, EPI><<<blocks_for(a.nvec, 128), 128, 0, c->stream>>>(a);
        else
            qldk::push_vec_kernel<uint8_t, RESET, EPI><<<blocks_for(a.nvec, 128), 128, 0, c->stream>>>(a);
    } else {
        if (c->pixfmt == QLD_U16)
            qldk::push_scalar_kernel<uint16_t, RESET, EPI><<<blocks_for(a.npix, 256), 256, 0, c->stream>>>(a);
        else
            qldk::push_scalar_kernel<uint8_t, RESET, EPI><<<blocks_for(a.npix, 256), 256, 0, c->stream>>>(a);
    }
}

// Enqueues the push of `count` device frames (and, if epi, the image) on
// c->stream. The band of frame f starts at frames + f * pitch (the caller's
// buffer with the band offset applied, or a contiguous stage). Arguments are
// already validated.
int enqueue_push(qld_ctx* c, const uint8_t* frames, long long pitch, int count, bool epi, float* amp, float* phase) {
    if (count == 0) return QLD_OK;
    const long long frame_bytes = c->frame_bytes;
    const bool reset = count >= c->N;
    const int first = reset ? count - c->N : 0;
    qldk::PushArgs a;
    a.frames = frames + (long long)first * pitch;
    a.frame_stride = pitch;
    a.nf = reset ? c->N : count;
    a.s_first = c->pushed + first + 1;
    a.ring = c->ring;
    a.slot_stride = c->slot_stride;
    a.N = c->N;
    a.S = c->S;
    a.C = c->C;
    a.npix = c->npix;
    a.amp = amp;
    a.phase = phase;
    a.out_aligned = (aligned(amp, 16) && aligned(phase, 16)) ? 1 : 0;
    const int vb = vec_bytes_of(c->pixfmt);
    const bool vec = aligned(a.frames, vec_align_of(c->pixfmt)) && (frame_bytes % vb) == 0 &&
                     (pitch % vec_align_of(c->pixfmt)) == 0;
    // A window rebuilt from the pushed frames alone in a frame of at most
    // 2^20 pixels: the block-mode kernel, whose threads split the frames into
    // time slices (the vector kernel would have too few threads, each walking
    // every frame).
    const int hb = c->pixfmt == QLD_U16 ? 16 : (c->pixfmt == QLD_U8 ? 8 : 12);  // 8-pixel vector bytes
    if (reset && c->npix <= (1ll << 20) && aligned(a.frames, 16) && (pitch % 16) == 0 && (frame_bytes % hb) == 0) {
        a.nvec = frame_bytes / hb;
        const unsigned grid = (unsigned)((a.nvec + qldk::kBlockPV - 1) / qldk::kBlockPV);
        g_launches.fetch_add(1);
        if (c->pixfmt == QLD_U16) {
            if (epi) qldk::block_push_kernel<uint16_t, true><<<grid, qldk::kBlockThreads, 0, c->stream>>>(a);
            else qldk::block_push_kernel<uint16_t, false><<<grid, qldk::kBlockThreads, 0, c->stream>>>(a);
        } else if (c->pixfmt == QLD_U8) {
            if (epi) qldk::block_push_kernel<qldk::u8h_t, true><<<grid, qldk::kBlockThreads, 0, c->stream>>>(a);
            else qldk::block_push_kernel<qldk::u8h_t, false><<<grid, qldk::kBlockThreads, 0, c->stream>>>(a);
        } else {
            if (epi) qldk::block_push_kernel<qldk::p12h_t, true><<<grid, qldk::kBlockThreads, 0, c->stream>>>(a);
            else qldk::block_push_kernel<qldk::p12h_t, false><<<grid, qldk::kBlockThreads, 0, c->stream>>>(a);
        }
        if (cudaGetLastError() != cudaSuccess) return QLD_E_CUDA;
        c->pushed += count;
        return QLD_OK;
    }
    a.nvec = vec ? frame_bytes / vb : c->npix;
    g_launches.fetch_add(1);
    if (reset) {
        if (epi) launch_push_t<true, true>(c, a, vec);
        else launch_push_t<true, false>(c, a, vec);
    } else {
        if (epi) launch_push_t<false, true>(c, a, vec);
        else launch_push_t<false, false>(c, a, vec);
    }
    if (cudaGetLastError() != cudaSuccess) return QLD_E_CUDA;
    c->pushed += count;
    return QLD_OK;
}

int enqueue_image(qld_ctx* c, float* amp, float* phase) {
    if (!amp && !phase) return QLD_OK;
    const long long nthr = (c->npix + 3) / 4;
    const int oa = (aligned(amp, 16) && aligned(phase, 16)) ? 1 : 0;
    g_launches.fetch_add(1);
    qldk::image_kernel<<<blocks_for(nthr, 256), 256, 0, c->stream>>>(c->S, c->C, c->npix, amp, phase, oa);
    return cudaGetLastError() == cudaSuccess ? QLD_OK : QLD_E_CUDA;
}

// Twiddles of bin k in c->tw (recomputed only when k changes).
int ensure_twiddles(qld_ctx* c, int k) {
    if (c->tw_k != k) {
        g_launches.fetch_add(1);
        qldk::twiddle_kernel<<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->tw, c->N, k);
        if (cudaGetLastError() != cudaSuccess) return QLD_E_CUDA;
        c->tw_k = k;
    }
    return QLD_OK;
}

int enqueue_fft_bin(qld_ctx* c, int k, float* out) {
    if (ensure_twiddles(c, k) != QLD_OK) return QLD_E_CUDA;
    g_launches.fetch_add(1);
    if (c->pixfmt == QLD_P12)
        qldk::launch_bin<qldk::p12_t, qldk::kBinPower>(c->ring, c->slot_stride, c->N, c->tw, c->frame_bytes, c->npix,
                                                       out, nullptr, c->stream);
    else if (c->pixfmt == QLD_U16)
        qldk::launch_bin<uint16_t, qldk::kBinPower>(c->ring, c->slot_stride, c->N, c->tw, c->frame_bytes, c->npix,
                                                   out, nullptr, c->stream);
    else
        qldk::launch_bin<uint8_t, qldk::kBinPower>(c->ring, c->slot_stride, c->N, c->tw, c->frame_bytes, c->npix,
                                                  out, nullptr, c->stream);
    return cudaGetLastError() == cudaSuccess ? QLD_OK : QLD_E_CUDA;
}

template <typename B>
void launch_step_t(const qld_ctx* c, const qldk::PushArgs& a, float* out) {
    using qldk::bin_kernel;
    constexpr int P = qldk::kBinPower;
    const int pv_log = qldk::fftbin_pv_log(a.nvec);
    const unsigned grid = (unsigned)((a.nvec + (1ll << pv_log) - 1) >> pv_log);
    const uint8_t* r = c->ring;
    const long long ss = c->slot_stride;
    cudaStream_t st = c->stream;
    switch (pv_log) {
        case 5: bin_kernel<B, 5, 128, P, true><<<grid, 128, 0, st>>>(r, ss, c->N, c->tw, a.nvec, a.npix, out, nullptr, a);
            break;
        case 4: bin_kernel<B, 4, 256, P, true><<<grid, 256, 0, st>>>(r, ss, c->N, c->tw, a.nvec, a.npix, out, nullptr, a);
            break;
        case 3: bin_kernel<B, 3, 256, P, true><<<grid, 256, 0, st>>>(r, ss, c->N, c->tw, a.nvec, a.npix, out, nullptr, a);
            break;
        default: bin_kernel<B, 2, 256, P, true><<<grid, 256, 0, st>>>(r, ss, c->N, c->tw, a.nvec, a.npix, out, nullptr, a);
            break;
    }
}

// Enqueues push + image + DFT bin of one step (arguments validated, window
// full afterwards): one bin_kernel with the push folded in (PUSH) for uint16
// frames with 1 <= count <= N in whole 16-byte vectors, else the push kernel
// and the bin kernel.
int enqueue_step(qld_ctx* c, const uint8_t* frames, long long pitch, int count, float* amp, float* phase, int k,
                 float* out) {
    const long long frame_bytes = c->frame_bytes;
    // uint16 only: the uint8 and packed 12-bit DFT bins are near their
    // instruction-issue limit, and the push riding in the same kernel made
    // the step slower than the two launches (1024^2, N = 1024, 4 frames:
    // uint8 210.6 against 206.6 us, packed 12-bit 284.7 against 281.0 us).
    const bool one = c->pixfmt == QLD_U16 && count >= 1 && count <= c->N && aligned(frames, 16) &&
                     (frame_bytes % 16) == 0 && (pitch % 16) == 0 && aligned(amp, 4) && aligned(phase, 4);
    if (!one) {
        const int rc = enqueue_push(c, frames, pitch, count, amp || phase, amp, phase);
        return rc != QLD_OK ? rc : enqueue_fft_bin(c, k, out);
    }
    if (ensure_twiddles(c, k) != QLD_OK) return QLD_E_CUDA;
    qldk::PushArgs a;
    a.frames = frames;
    a.frame_stride = pitch;
    a.nf = count;
    a.s_first = c->pushed + 1;
    a.ring = c->ring;
    a.slot_stride = c->slot_stride;
    a.N = c->N;
    a.S = c->S;
    a.C = c->C;
    a.nvec = frame_bytes / 16;
    a.npix = c->npix;
    a.amp = amp;
    a.phase = phase;
    a.out_aligned = 0;
    g_launches.fetch_add(1);
    launch_step_t<uint16_t>(c, a, out);
    if (cudaGetLastError() != cudaSuccess) return QLD_E_CUDA;
    c->pushed += count;
    return QLD_OK;
}

void free_pipe(HostPipe* hp) {
    if (!hp) return;
    if (hp->cin) cudaStreamSynchronize(hp->cin);
    if (hp->cout) cudaStreamSynchronize(hp->cout);
    for (int i = 0; i < HostPipe::kIn; ++i) {
        if (hp->stage[i]) cudaFree(hp->stage[i]);
        if (hp->in_ready[i]) cudaEventDestroy(hp->in_ready[i]);
        if (hp->in_free[i]) cudaEventDestroy(hp->in_free[i]);
    }
    for (int o = 0; o < HostPipe::kOut; ++o) {
        if (hp->out[o]) cudaFree(hp->out[o]);
        if (hp->out_ready[o]) cudaEventDestroy(hp->out_ready[o]);
        if (hp->out_free[o]) cudaEventDestroy(hp->out_free[o]);
    }
    if (hp->cin) cudaStreamDestroy(hp->cin);
    if (hp->cout) cudaStreamDestroy(hp->cout);
    delete hp;
}

void free_ctx_memory(qld_ctx* c) {
    if (c->ring) cudaFree(c->ring);
    if (c->S) cudaFree(c->S);
    if (c->C) cudaFree(c->C);
    if (c->tw) cudaFree(c->tw);
    free_pipe(c->pipe);
    c->ring = nullptr;
    c->S = c->C = nullptr;
    c->tw = nullptr;
    c->pipe = nullptr;
}

// Creates the host pipeline with input stages of at least `stage_bytes`
// (staging up to 64 MiB per chunk) and output buffers of two images.
int ensure_pipe(qld_ctx* c, long long stage_bytes) {
    if (c->pipe && c->pipe->stage_bytes >= stage_bytes) return QLD_OK;
    if (c->pipe) {  // grow: wait for everything in flight, then rebuild
        cudaStreamSynchronize(c->stream);
        free_pipe(c->pipe);
        c->pipe = nullptr;
    }
    HostPipe* hp = new HostPipe();
    std::memset(hp, 0, sizeof(*hp));
    bool ok = cudaStreamCreateWithFlags(&hp->cin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&hp->cout, cudaStreamNonBlocking) == cudaSuccess;
    hp->stage_bytes = stage_bytes;
    hp->out_elems = 2 * c->npad;
    for (int i = 0; ok && i < HostPipe::kIn; ++i)
        ok = cudaMalloc(&hp->stage[i], (size_t)stage_bytes) == cudaSuccess &&
             cudaEventCreateWithFlags(&hp->in_ready[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&hp->in_free[i], cudaEventDisableTiming) == cudaSuccess;
    for (int o = 0; ok && o < HostPipe::kOut; ++o)
        ok = cudaMalloc(&hp->out[o], (size_t)hp->out_elems * sizeof(float)) == cudaSuccess &&
             cudaEventCreateWithFlags(&hp->out_ready[o], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&hp->out_free[o], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_pipe(hp);
        return QLD_E_NOMEM;
    }
    c->pipe = hp;
    return QLD_OK;
}

// Next output buffer: the context's stream waits until its previous
// device-to-host copy has finished.
float* acquire_out(qld_ctx* c, int* slot) {
    HostPipe* hp = c->pipe;
    const int o = hp->out_idx;
    hp->out_idx = (o + 1) % HostPipe::kOut;
    cudaStreamWaitEvent(c->stream, hp->out_free[o], 0);
    *slot = o;
    return hp->out[o];
}

// Copies n floats of buffer `slot` (after its producer on the context's
// stream) to each non-NULL host pointer, on the copy-out stream.
int release_out(qld_ctx* c, int slot, const float* d0, float* h0, const float* d1, float* h1) {
    HostPipe* hp = c->pipe;
    const size_t bytes = (size_t)c->npix * sizeof(float);
    if (cudaEventRecord(hp->out_ready[slot], c->stream) != cudaSuccess ||
        cudaStreamWaitEvent(hp->cout, hp->out_ready[slot], 0) != cudaSuccess)
        return QLD_E_CUDA;
    if (h0 && cudaMemcpyAsync(h0, d0, bytes, cudaMemcpyDeviceToHost, hp->cout) != cudaSuccess) return QLD_E_CUDA;
    if (h1 && cudaMemcpyAsync(h1, d1, bytes, cudaMemcpyDeviceToHost, hp->cout) != cudaSuccess) return QLD_E_CUDA;
    return cudaEventRecord(hp->out_free[slot], hp->cout) == cudaSuccess ? QLD_OK : QLD_E_CUDA;
}

// Copies the band of host frames first .. first + n - 1 into a contiguous
// device stage on `st`: one copy for a whole-frame context, a strided copy of
// the band's rows for a row band (only the band's bytes cross the bus).
cudaError_t copy_frames_in(const qld_ctx* c, uint8_t* dst, const uint8_t* src, long long first, long long n,
                           cudaStream_t st) {
    if (c->band_offset == 0 && c->frame_pitch == c->frame_bytes)
        return cudaMemcpyAsync(dst, src + first * c->frame_bytes, (size_t)(n * c->frame_bytes), cudaMemcpyHostToDevice,
                               st);
    return cudaMemcpy2DAsync(dst, (size_t)c->frame_bytes, src + c->band_offset + first * c->frame_pitch,
                             (size_t)c->frame_pitch, (size_t)c->frame_bytes, (size_t)n, cudaMemcpyHostToDevice, st);
}

// Creates a context for rows row0 .. row0 + rows - 1 of H_total x W frames
// (validated by the caller).
qld_ctx* create_ctx(int H_total, int W, int N, int pixfmt, int row0, int rows) {
    const int H = rows;
    const Layout L = layout_of(H, W, N, pixfmt);
    // Reserve against the budget before touching the device.
    const long long budget = g_budget.load();
    long long prev = g_in_use.fetch_add(L.total);
    if (budget > 0 && prev + L.total > budget) {
        g_in_use.fetch_sub(L.total);
        set_err(QLD_E_NOMEM);
        return nullptr;
    }
    qld_ctx* c = new qld_ctx();
    std::memset(c, 0, sizeof(*c));
    c->H = H;
    c->W = W;
    c->N = N;
    c->pixfmt = pixfmt;
    c->frame_bytes = frame_bytes_of(L.npix, pixfmt);
    c->H_total = H_total;
    c->row0 = row0;
    c->band_offset = frame_bytes_of((long long)row0 * W, pixfmt);
    c->frame_pitch = frame_bytes_of((long long)H_total * W, pixfmt);
    c->npix = L.npix;
    c->npad = L.npad;
    c->slot_stride = L.slot_stride;
    c->tw_k = -1;
    c->footprint = L.total;
    c->stream = nullptr;
    int st = QLD_OK;
    if (cudaGetDevice(&c->device) != cudaSuccess) st = QLD_E_CUDA;
    if (st == QLD_OK && (cudaMalloc(&c->ring, (size_t)L.ring_bytes) != cudaSuccess ||
                         cudaMalloc(&c->S, (size_t)L.sums_bytes) != cudaSuccess ||
                         cudaMalloc(&c->C, (size_t)L.sums_bytes) != cudaSuccess ||
                         cudaMalloc(&c->tw, (size_t)L.tw_bytes) != cudaSuccess)) {
        st = QLD_E_NOMEM;
    }
    if (st == QLD_OK && (cudaMemset(c->ring, 0, (size_t)L.ring_bytes) != cudaSuccess ||
                         cudaMemset(c->S, 0, (size_t)L.sums_bytes) != cudaSuccess ||
                         cudaMemset(c->C, 0, (size_t)L.sums_bytes) != cudaSuccess ||
                         cudaDeviceSynchronize() != cudaSuccess)) {
        st = QLD_E_CUDA;
    }
    if (st != QLD_OK) {
        cudaGetLastError();
        free_ctx_memory(c);
        delete c;
        g_in_use.fetch_sub(L.total);
        set_err(st);
        return nullptr;
    }
    return c;
}

}  // namespace

extern "C" {

const char* qld_version(void) { return "qld 0.1 (sm_103a)"; }

const char* qld_strerror(int st) {
    switch (st) {
        case QLD_OK: return "ok";
        case QLD_E_INVAL: return "invalid argument";
        case QLD_E_NOMEM: return "out of device memory or over the memory budget";
        case QLD_E_NOT_READY: return "window not full: fewer than N frames pushed";
        case QLD_E_CUDA: return "CUDA runtime error";
        case QLD_E_TIMEOUT: return "bounded wait timed out";
        default: return "unknown status";
    }
}

int qld_last_error(void) { return qldi::g_last_error; }

long long qld_footprint_bytes(int H, int W, int N, int pixfmt) {
    if (!valid_dims(H, W, N, pixfmt)) return QLD_E_INVAL;
    return layout_of(H, W, N, pixfmt).total;
}

void qld_set_mem_budget(long long bytes) { g_budget.store(bytes < 0 ? 0 : bytes); }

long long qld_mem_in_use(void) { return g_in_use.load(); }

long long qld_launch_count(void) { return g_launches.load(); }

qld_ctx* qld_create(int H, int W, int N, int pixfmt) {
    if (!valid_dims(H, W, N, pixfmt)) {
        set_err(QLD_E_INVAL);
        return nullptr;
    }
    return create_ctx(H, W, N, pixfmt, 0, H);
}

qld_ctx* qld_create_band(int H_total, int W, int N, int pixfmt, int row0, int rows) {
    // the band is a valid frame of its own, lies inside the full frame, and
    // (packed 12-bit) starts on a whole pixel pair
    if (row0 < 0 || rows < 1 || H_total < 1 || (long long)row0 + rows > H_total || !valid_dims(rows, W, N, pixfmt) ||
        !valid_dims(H_total, W, N, pixfmt) || (pixfmt == QLD_P12 && ((long long)row0 * W) % 2 != 0)) {
        set_err(QLD_E_INVAL);
        return nullptr;
    }
    return create_ctx(H_total, W, N, pixfmt, row0, rows);
}

void qld_destroy(qld_ctx* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->stream);
        free_ctx_memory(c);
    }
    g_in_use.fetch_sub(c->footprint);
    delete c;
}

int qld_push_frames(qld_ctx* c, const void* frames, int count, void* stream) {
    if (!c || count < 0 || (count > 0 && !frames)) return set_err(QLD_E_INVAL);
    if (c->pixfmt == QLD_U16 && !aligned(frames, 2)) return set_err(QLD_E_INVAL);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    c->stream = (cudaStream_t)stream;
    return set_err(enqueue_push(c, (const uint8_t*)frames + c->band_offset, c->frame_pitch, count, false, nullptr,
                                nullptr));
}

int qld_push_image(qld_ctx* c, const void* frames, int count, void* stream, float* amp, float* phase) {
    if (!c || count < 0 || (count > 0 && !frames)) return set_err(QLD_E_INVAL);
    if (c->pixfmt == QLD_U16 && !aligned(frames, 2)) return set_err(QLD_E_INVAL);
    if (!aligned(amp, 4) || !aligned(phase, 4)) return set_err(QLD_E_INVAL);
    if (c->pushed + count < c->N) return set_err(QLD_E_NOT_READY);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    c->stream = (cudaStream_t)stream;
    if (count == 0) return set_err(enqueue_image(c, amp, phase));
    return set_err(enqueue_push(c, (const uint8_t*)frames + c->band_offset, c->frame_pitch, count, amp || phase, amp,
                                phase));
}

int qld_image(qld_ctx* c, float* amp, float* phase) {
    if (!c || !aligned(amp, 4) || !aligned(phase, 4)) return set_err(QLD_E_INVAL);
    if (c->pushed < c->N) return set_err(QLD_E_NOT_READY);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    return set_err(enqueue_image(c, amp, phase));
}

int qld_step(qld_ctx* c, const void* frames, int count, void* stream, float* amp, float* phase, int k, float* power) {
    if (!c || count < 1 || !frames || !power || !aligned(power, 4) || k < 0 || k >= c->N) return set_err(QLD_E_INVAL);
    if (c->pixfmt == QLD_U16 && !aligned(frames, 2)) return set_err(QLD_E_INVAL);
    if (!aligned(amp, 4) || !aligned(phase, 4)) return set_err(QLD_E_INVAL);
    if (c->pushed + count < c->N) return set_err(QLD_E_NOT_READY);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    c->stream = (cudaStream_t)stream;
    return set_err(enqueue_step(c, (const uint8_t*)frames + c->band_offset, c->frame_pitch, count, amp, phase, k,
                                power));
}

int qld_fft_bin(qld_ctx* c, int k, float* out) {
    if (!c || !out || !aligned(out, 4) || k < 0 || k >= (c ? c->N : 0)) return set_err(QLD_E_INVAL);
    if (c->pushed < c->N) return set_err(QLD_E_NOT_READY);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    return set_err(enqueue_fft_bin(c, k, out));
}

int qld_push_frames_host(qld_ctx* c, const void* host_frames, int count, void* stream) {
    if (!c || count < 0 || (count > 0 && !host_frames)) return set_err(QLD_E_INVAL);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    c->stream = (cudaStream_t)stream;
    if (count == 0) return QLD_OK;
    const long long frame_bytes = c->frame_bytes;
    // Chunks of at most 64 MiB (and at least one frame); consecutive chunks
    // are the same as one push.
    long long chunk = (64ll << 20) / frame_bytes;
    if (chunk < 1) chunk = 1;
    if (chunk > count) chunk = count;
    int st = ensure_pipe(c, round_up(chunk * frame_bytes, 256));
    if (st != QLD_OK) return set_err(st);
    HostPipe* hp = c->pipe;
    const uint8_t* src = (const uint8_t*)host_frames;
    for (long long done = 0; done < count; done += chunk) {
        const long long n = (count - done < chunk) ? count - done : chunk;
        const int i = hp->in_idx;
        hp->in_idx = (i + 1) % HostPipe::kIn;
        if (cudaStreamWaitEvent(hp->cin, hp->in_free[i], 0) != cudaSuccess ||
            copy_frames_in(c, hp->stage[i], src, done, n, hp->cin) != cudaSuccess ||
            cudaEventRecord(hp->in_ready[i], hp->cin) != cudaSuccess ||
            cudaStreamWaitEvent(c->stream, hp->in_ready[i], 0) != cudaSuccess)
            return set_err(QLD_E_CUDA);
        st = enqueue_push(c, hp->stage[i], frame_bytes, (int)n, false, nullptr, nullptr);
        if (st != QLD_OK) return set_err(st);
        if (cudaEventRecord(hp->in_free[i], c->stream) != cudaSuccess) return set_err(QLD_E_CUDA);
    }
    return QLD_OK;
}

int qld_image_host(qld_ctx* c, float* amp_host, float* phase_host) {
    if (!c) return set_err(QLD_E_INVAL);
    if (c->pushed < c->N) return set_err(QLD_E_NOT_READY);
    if (!amp_host && !phase_host) return QLD_OK;
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    int st = ensure_pipe(c, c->pipe ? c->pipe->stage_bytes : round_up(c->frame_bytes, 256));
    if (st != QLD_OK) return set_err(st);
    int slot = 0;
    float* buf = acquire_out(c, &slot);
    float* da = amp_host ? buf : nullptr;
    float* dp = phase_host ? buf + c->npad : nullptr;
    st = enqueue_image(c, da, dp);
    if (st != QLD_OK) return set_err(st);
    return set_err(release_out(c, slot, da, amp_host, dp, phase_host));
}

int qld_fft_bin_host(qld_ctx* c, int k, float* out_host) {
    if (!c || !out_host || k < 0 || k >= c->N) return set_err(QLD_E_INVAL);
    if (c->pushed < c->N) return set_err(QLD_E_NOT_READY);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    int st = ensure_pipe(c, c->pipe ? c->pipe->stage_bytes : round_up(c->frame_bytes, 256));
    if (st != QLD_OK) return set_err(st);
    int slot = 0;
    float* buf = acquire_out(c, &slot);
    st = enqueue_fft_bin(c, k, buf);
    if (st != QLD_OK) return set_err(st);
    return set_err(release_out(c, slot, buf, out_host, nullptr, nullptr));
}

int qld_step_host(qld_ctx* c, const void* host_frames, int count, void* stream, float* amp_host, float* phase_host,
                  int k, float* power_host) {
    if (!c || count < 1 || !host_frames || !power_host || k < 0 || k >= c->N) return set_err(QLD_E_INVAL);
    if (c->pushed + count < c->N) return set_err(QLD_E_NOT_READY);
    const long long bytes = (long long)count * c->frame_bytes;
    if (bytes > (64ll << 20)) {  // more than one input stage: the three host calls
        int st = qld_push_frames_host(c, host_frames, count, stream);
        if (st == QLD_OK) st = qld_image_host(c, amp_host, phase_host);
        return st != QLD_OK ? st : qld_fft_bin_host(c, k, power_host);
    }
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    c->stream = (cudaStream_t)stream;
    int st = ensure_pipe(c, c->pipe ? c->pipe->stage_bytes : round_up(bytes, 256));
    if (st == QLD_OK && c->pipe->stage_bytes < bytes) st = ensure_pipe(c, round_up(bytes, 256));
    if (st != QLD_OK) return set_err(st);
    HostPipe* hp = c->pipe;
    const int i = hp->in_idx;
    hp->in_idx = (i + 1) % HostPipe::kIn;
    if (cudaStreamWaitEvent(hp->cin, hp->in_free[i], 0) != cudaSuccess ||
        copy_frames_in(c, hp->stage[i], (const uint8_t*)host_frames, 0, count, hp->cin) != cudaSuccess ||
        cudaEventRecord(hp->in_ready[i], hp->cin) != cudaSuccess ||
        cudaStreamWaitEvent(c->stream, hp->in_ready[i], 0) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    int s_img = 0, s_pow = 0;
    float* img = acquire_out(c, &s_img);
    float* pw = acquire_out(c, &s_pow);
    float* da = amp_host ? img : nullptr;
    float* dp = phase_host ? img + c->npad : nullptr;
    st = enqueue_step(c, hp->stage[i], c->frame_bytes, count, da, dp, k, pw);
    if (st != QLD_OK) return set_err(st);
    if (cudaEventRecord(hp->in_free[i], c->stream) != cudaSuccess) return set_err(QLD_E_CUDA);
    st = release_out(c, s_img, da, amp_host, dp, phase_host);
    return set_err(st != QLD_OK ? st : release_out(c, s_pow, pw, power_host, nullptr, nullptr));
}

int qld_get_iq(qld_ctx* c, int32_t* S, int32_t* C) {
    if (!c || !aligned(S, 4) || !aligned(C, 4)) return set_err(QLD_E_INVAL);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    const size_t bytes = (size_t)c->npix * sizeof(int32_t);
    if (S && cudaMemcpyAsync(S, c->S, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    if (C && cudaMemcpyAsync(C, c->C, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    return QLD_OK;
}

int qld_iq_pointers(qld_ctx* c, const int32_t** S, const int32_t** C) {
    if (!c) return set_err(QLD_E_INVAL);
    if (S) *S = c->S;
    if (C) *C = c->C;
    return QLD_OK;
}

int qld_reset(qld_ctx* c) {
    if (!c) return set_err(QLD_E_INVAL);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    if (cudaMemsetAsync(c->ring, 0, (size_t)(c->slot_stride * c->N), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->S, 0, (size_t)c->npad * sizeof(int32_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->C, 0, (size_t)c->npad * sizeof(int32_t), c->stream) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    c->pushed = 0;
    return QLD_OK;
}

long long qld_frames_pushed(const qld_ctx* c) { return c ? c->pushed : -1; }

int qld_sync(qld_ctx* c) {
    if (!c) return set_err(QLD_E_INVAL);
    DeviceGuard g(c->device);
    if (!g.ok) return set_err(QLD_E_CUDA);
    bool ok = cudaStreamSynchronize(c->stream) == cudaSuccess;
    if (c->pipe) {
        ok = cudaStreamSynchronize(c->pipe->cin) == cudaSuccess && ok;
        ok = cudaStreamSynchronize(c->pipe->cout) == cudaSuccess && ok;
    }
    if (!ok) {
        cudaGetLastError();
        return set_err(QLD_E_CUDA);
    }
    return set_err(pending_error());
}

void* qld_stream(const qld_ctx* c) { return c ? (void*)c->stream : nullptr; }

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free DFT bin over caller frames.
//
// For callers that must not allocate device memory while they run: the
// twiddle table this computation needs lives in a fixed file-scope device
// array instead of a context. Host code cannot use the array's name as a
// device address (on the host it names a stand-in object), so the device
// address is looked up once per device with cudaGetSymbolAddress and cached.
// The cache lives as long as the process: a device reset (cudaDeviceReset)
// after the first call would leave it pointing into a destroyed context, so
// that is not supported.

namespace {

constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) float2 g_noalloc_twiddles[QLD_NOALLOC_MAX_N];
float2* g_noalloc_twiddles_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of g_noalloc_twiddles on the current device (looked up on
// the first call on that device), or nullptr on error.
float2* noalloc_twiddles(int dev) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_twiddles_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_twiddles) != cudaSuccess || !p) {
            cudaGetLastError();
            return nullptr;
        }
        g_noalloc_twiddles_addr[dev] = (float2*)p;
    }
    return g_noalloc_twiddles_addr[dev];
}

}  // namespace

extern "C" int qld_fft_bin_frames_noalloc(const void* frames, int H, int W, int N, int pixfmt, int k, float* out,
                                          void* stream) {
    if (!frames || !out || H < 1 || W < 1 || (pixfmt != QLD_U8 && pixfmt != QLD_U16)) return set_err(QLD_E_INVAL);
    if (N < 4 || (N % 4) != 0 || N > QLD_NOALLOC_MAX_N || k < 0 || k >= N) return set_err(QLD_E_INVAL);
    const long long npix = (long long)H * W;
    const long long frame_bytes = npix * pixfmt;
    if (npix > (1ll << 31) - 1 || (frame_bytes % qldk::kVecBytes) != 0 || !aligned(frames, 16) || !aligned(out, 4))
        return set_err(QLD_E_INVAL);
    // A sticky error from earlier asynchronous work: report it before
    // queueing anything, so a failure here never hides work of this call.
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_err(QLD_E_CUDA);
    float2* tw = noalloc_twiddles(dev);
    if (!tw) return set_err(QLD_E_CUDA);
    cudaStream_t st = (cudaStream_t)stream;
    // Frame i of the block plays the part of ring slot i. Its absolute index
    // in a fresh stream would be i + 1; that shifts every X_k by the same
    // unit-modulus factor, so |X_k|^2 is unchanged.
    g_launches.fetch_add(1);
    qldk::twiddle_kernel<<<blocks_for(N, 256), 256, 0, st>>>(tw, N, k);
    const uint8_t* base = (const uint8_t*)frames;
    g_launches.fetch_add(1);
    if (pixfmt == QLD_U16)
        qldk::launch_bin<uint16_t, qldk::kBinPower>(base, frame_bytes, N, tw, frame_bytes, npix, out, nullptr, st);
    else
        qldk::launch_bin<uint8_t, qldk::kBinPower>(base, frame_bytes, N, tw, frame_bytes, npix, out, nullptr, st);
    return set_err(cudaGetLastError() == cudaSuccess ? QLD_OK : QLD_E_CUDA);
}

// ------------------------------------------------------------------------
// Lock-in at an arbitrary frequency over caller frames (block mode).

extern "C" int qld_lockin_table(double omega_dt, long long s0, int N, float* table, void* stream) {
    if (!table || !aligned(table, 8) || N < 1 || N > (1 << 30)) return set_err(QLD_E_INVAL);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    g_launches.fetch_add(1);
    qldk::lockin_table_kernel<<<blocks_for(N, 256), 256, 0, (cudaStream_t)stream>>>((float2*)table, N, omega_dt, s0);
    return set_err(cudaGetLastError() == cudaSuccess ? QLD_OK : QLD_E_CUDA);
}

extern "C" int qld_lockin_frames(const void* frames, int H, int W, int N, int pixfmt, const float* table, float* amp,
                                 float* phase, void* stream) {
    if (!frames || !table || (!amp && !phase) || H < 1 || W < 1 || N < 1 || (pixfmt != QLD_U8 && pixfmt != QLD_U16))
        return set_err(QLD_E_INVAL);
    const long long npix = (long long)H * W;
    const long long frame_bytes = npix * pixfmt;
    if (npix > (1ll << 31) - 1 || (frame_bytes % qldk::kVecBytes) != 0 || !aligned(frames, 16) ||
        !aligned(table, 8) || !aligned(amp, 4) || !aligned(phase, 4))
        return set_err(QLD_E_INVAL);
    if (pending_error() != QLD_OK) return set_err(QLD_E_CUDA);
    const uint8_t* base = (const uint8_t*)frames;
    cudaStream_t st = (cudaStream_t)stream;
    g_launches.fetch_add(1);
    if (pixfmt == QLD_U16)
        qldk::launch_bin<uint16_t, qldk::kBinAmpPhase>(base, frame_bytes, N, (const float2*)table, frame_bytes, npix,
                                                       amp, phase, st);
    else
        qldk::launch_bin<uint8_t, qldk::kBinAmpPhase>(base, frame_bytes, N, (const float2*)table, frame_bytes, npix,
                                                      amp, phase, st);
    return set_err(cudaGetLastError() == cudaSuccess ? QLD_OK : QLD_E_CUDA);
}
