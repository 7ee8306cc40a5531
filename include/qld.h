/* qld.h -- C ABI of the B300 quadrature lock-in discrimination (QLD) library.
 *
 * The library computes, for every pixel of a stream of camera frames sampled
 * at four times the source modulation frequency, the quadrature lock-in sums
 * of the paper (Methods, "Numerical simulations": the equation for R(j,k))
 *
 *     S = sum_{s in window} x_s * sin(pi s / 2),
 *     C = sum_{s in window} x_s * cos(pi s / 2),
 *
 * exactly in int32 over a sliding window of the last N frames, the amplitude
 * R = sqrt(S^2 + C^2) and phase atan2(-S, C) images, and the single-bin DFT
 * power |X_k|^2 with X_k = sum_s x_s exp(-2 pi i k s / N) (Methods, the FFT
 * map the paper compares QLD against).
 *
 * Frame index convention: s is the absolute 1-based index of a frame in the
 * stream (the first frame ever pushed has s = 1; Methods: t_s = s dt,
 * s = 1, 2, ...). After T frames have been pushed the window is
 * s = T-N+1 .. T. At four samples per period sin(pi s/2) and cos(pi s/2)
 * take only the values 0, +1, -1, so S and C are signed sums of frame
 * values and need no multiplications.
 *
 * Memory: all frame, image and sum pointers are DEVICE pointers unless the
 * function name ends in _host. Frames are laid out [count][H][W], row-major,
 * contiguous, uint8 (QLD_U8), uint16 (QLD_U16, 12- or 16-bit data in the
 * low bits) or packed 12-bit (QLD_P12). Images are float32 [H][W]; sums are int32 [H][W]. Any H and W
 * are accepted. Pointers must be aligned to their element size (uint16
 * frames to 2 bytes, float and int32 buffers to 4), else QLD_E_INVAL; frame
 * buffers that are not 16-byte aligned (8 for QLD_P12), or frames whose size
 * is not a multiple of 16 bytes (24 for QLD_P12), take a slower scalar path. The context owns its ring
 * buffer, sums and scratch; the caller owns every pointer it passes.
 *
 * Streams: qld_push_frames and its variants enqueue on the stream they are
 * given and make it the context's current stream; every other call enqueues
 * on the context's current stream. All calls are asynchronous with respect
 * to the host except qld_create, qld_destroy and qld_sync. A frame buffer may
 * be reused once its push has completed on that stream.
 *
 * Errors: functions returning int return QLD_OK (0) or a negative status.
 * Argument errors are detected synchronously and change no state. A CUDA
 * error from a launch or copy is returned as QLD_E_CUDA; an error raised
 * later by the device is reported by the next call or by qld_sync.
 * qld_last_error() returns the last non-OK status set on the calling thread.
 *
 * Threads: there is no internal locking; a context must not be used by two
 * host threads at once. Distinct contexts are independent.
 */
#ifndef QLD_H
#define QLD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qld_ctx qld_ctx;

/* QLD_P12: 12-bit pixels packed two in three bytes, least significant bits
 * first (GenICam Mono12p: pixel 2i = b0 | (b1 & 0xF) << 8, pixel 2i+1 =
 * (b1 >> 4) | b2 << 4); H*W must be even. The window ring stores frames in
 * the input format, so packed data moves 25 % fewer bytes than uint16. */
enum qld_pixfmt { QLD_U8 = 1, QLD_U16 = 2, QLD_P12 = 3 };

enum qld_status {
    QLD_OK = 0,
    QLD_E_INVAL = -1,     /* bad argument */
    QLD_E_NOMEM = -2,     /* device allocation failed or over the memory budget */
    QLD_E_NOT_READY = -3, /* fewer than N frames pushed since creation/reset */
    QLD_E_CUDA = -4,      /* a CUDA runtime error */
    QLD_E_TIMEOUT = -5    /* a bounded wait ran out */
};

/* Largest window. S adds N/4 frames and subtracts N/4 others (likewise C),
 * so with |x| <= 65535, |S|, |C| <= (N/4) * 65535 < 2^31 for N <= 65536 and
 * the int32 sums are exact. */
#define QLD_MAX_N 65536

/* Creates a context for H x W frames of the given pixel format and a window
 * of N frames (SI, "Timing sequence", item 1: the set-up thread allocates
 * memory and builds the reference tables; SI closing paragraph: a sliding
 * window needs a buffer of N frames). N must be a positive multiple of 4 and
 * at most QLD_MAX_N so the window holds whole modulation periods. Allocates
 * on the current CUDA device a zeroed ring of N frames, the int32 sums and a
 * twiddle table: see qld_footprint_bytes. Returns NULL on error
 * (qld_last_error() gives QLD_E_INVAL or QLD_E_NOMEM). Synchronous. */
qld_ctx* qld_create(int H, int W, int N, int pixfmt);

/* A context for the row band row0 .. row0 + rows - 1 of a stream of
 * H_total x W frames. Pixels are independent (Methods, "Numerical
 * simulations": every pixel's time series gives its own R(j,k)), so a frame
 * split into row bands, each with its own ring and sums (on its own GPU, or
 * several on one), gives exactly the whole frame's sums, images and DFT bins
 * row for row, with no exchange between bands.
 *
 * The context behaves as qld_create(rows, W, N, pixfmt) -- its images, sums
 * and bins are rows x W and its footprint is qld_footprint_bytes(rows, W, N,
 * pixfmt) -- except that pushes take WHOLE frames ([count][H_total][W]; the
 * host variants too) and read only the band: frame f's band starts
 * row0 * W * b + f * H_total * W * b bytes into the buffer (b = bytes per
 * pixel; 3/2 for QLD_P12). A host push copies only the band's rows. The
 * single-kernel qld_step needs the band's start 16-byte aligned and the
 * frame pitch a multiple of 16 bytes, as for whole frames. Returns NULL with
 * QLD_E_INVAL unless 0 <= row0, rows >= 1, row0 + rows <= H_total, both the
 * band and the whole frame are valid for qld_create, and (QLD_P12) the band
 * starts on a whole pixel pair; QLD_E_NOMEM as qld_create. */
qld_ctx* qld_create_band(int H_total, int W, int N, int pixfmt, int row0, int rows);

/* Device bytes qld_create(H, W, N, pixfmt) would allocate, or a negative
 * status for invalid arguments. */
long long qld_footprint_bytes(int H, int W, int N, int pixfmt);

/* Caps the device bytes that contexts created afterwards in this process may
 * hold in total (0 = no cap). qld_create fails with QLD_E_NOMEM when the cap
 * would be exceeded. Used for admission by memory footprint and to test
 * allocation failure without exhausting the device. */
void qld_set_mem_budget(long long bytes);
long long qld_mem_in_use(void);

/* Frees the context and everything it owns. Waits for its pending work. */
void qld_destroy(qld_ctx* ctx);

/* Pushes `count` frames (device, [count][H][W]) into the window on `stream`
 * (a cudaStream_t; NULL = the legacy default stream), frame i getting the
 * absolute index frames_pushed + 1 + i (SI, "Timing sequence", item 3:
 * every frame updates the two quadrature accumulators as it arrives). For
 * each frame s the ring slot s mod N is read (frame s - N, or zero while the
 * window fills), overwritten with x_s, and the difference x_s - x_{s-N} is
 * added to S with sign sin(pi s/2) or to C with sign cos(pi s/2). count = 0
 * is a no-op; count > N behaves as count sequential pushes (only the last N
 * frames remain). Returns QLD_E_INVAL for a NULL frame pointer with
 * count > 0 or count < 0. */
int qld_push_frames(qld_ctx* ctx, const void* frames, int count, void* stream);

/* Writes the amplitude R = sqrt(S^2 + C^2) and phase atan2(-S, C) images
 * (device float32 [H][W]; either may be NULL) of the current window (Methods,
 * R(j,k); SI item 3: the components are squared and added after the required
 * number of frames). Phase is in (-pi, pi], 0 where S = C = 0. Returns
 * QLD_E_NOT_READY until N frames have been pushed. */
int qld_image(qld_ctx* ctx, float* amp, float* phase);

/* qld_push_frames followed by qld_image in one kernel: the image is written
 * while S and C are still in registers. Requires that the window is full
 * after the push (else QLD_E_NOT_READY and nothing is done). */
int qld_push_image(qld_ctx* ctx, const void* frames, int count, void* stream, float* amp, float* phase);

/* Writes |X_k|^2 for every pixel (device float32 [H][W]), X_k the DFT bin k
 * of the pixel's time series over the current window with absolute frame
 * indices (Methods, the map |F(j,k,omega_q)|^2). 0 <= k < N. Accumulates in
 * float32 with twiddles rounded from FP64. For k = N/4, X_k = C - iS.
 * Returns QLD_E_NOT_READY until N frames have been pushed. */
int qld_fft_bin(qld_ctx* ctx, int k, float* out);

/* One step of the hot path: qld_push_image(ctx, frames, count, stream, amp,
 * phase) followed by qld_fft_bin(ctx, k, power), bit for bit the same
 * results, in ONE kernel for uint16 frames when 1 <= count <= N, the frames
 * are 16-byte aligned and a frame is a whole number of 16-byte vectors;
 * otherwise (and for uint8 and packed 12-bit frames, whose DFT bin is bound
 * by instruction issue, so the push in the same kernel measured slower) as
 * the two calls. In the single kernel the bin's time slice that later reads
 * a ring slot is the thread that writes the new frame into it, so the slot is
 * read back by its writer, and the DFT bin streams the window once per step
 * with the push riding along. amp and phase may be NULL; power is device float32
 * [H][W]. Returns QLD_E_INVAL for count < 1, k outside [0, N), a NULL or
 * misaligned power, or the arguments qld_push_image rejects, and
 * QLD_E_NOT_READY (nothing done) when the window would not be full. */
int qld_step(qld_ctx* ctx, const void* frames, int count, void* stream, float* amp, float* phase, int k,
             float* power);

/* Host-buffer variants: frames are read from, and images written to, HOST
 * memory (SI "Timing sequence" item 3: frames cross the PCI express bus to
 * the GPU). The context keeps device staging (two input stages of up to
 * 64 MiB, four output images; created on first use, not counted in
 * qld_footprint_bytes) and two private copy streams: host-to-device copies,
 * kernels on the context's stream and device-to-host copies are ordered by
 * events, so copies of one call overlap the kernels of neighbouring calls.
 * Pinned host memory makes the copies asynchronous (pageable memory works,
 * with synchronous copies). Host results are valid after qld_sync, which
 * also waits for the copy streams; a host frame buffer may be reused after
 * qld_sync. */
int qld_push_frames_host(qld_ctx* ctx, const void* host_frames, int count, void* stream);
int qld_image_host(qld_ctx* ctx, float* amp_host, float* phase_host);
int qld_fft_bin_host(qld_ctx* ctx, int k, float* out_host);
/* qld_step with host buffers: the frames are copied from host memory into
 * an input stage, the step runs as in qld_step, and the amplitude, phase
 * (either may be NULL) and power images are copied back to host memory
 * through the output ring (valid after qld_sync). Steps of more than 64 MiB
 * of frames run as qld_push_frames_host, qld_image_host, qld_fft_bin_host.
 * Errors as qld_step. */
int qld_step_host(qld_ctx* ctx, const void* host_frames, int count, void* stream, float* amp_host, float* phase_host,
                  int k, float* power_host);

/* Copies the exact int32 sums S and C (device [H][W]; either may be NULL).
 * Valid at any time (partial sums while the window fills). */
int qld_get_iq(qld_ctx* ctx, int32_t* S, int32_t* C);

/* The device addresses of the context's own sums S and C (int32 [H][W],
 * owned by the context, valid until qld_destroy), for kernels that read them
 * in place instead of a copy (the paper has no counterpart: a zero-copy
 * accessor). Their contents change with every push: read them in the
 * context's stream order. Either output may be NULL. QLD_E_INVAL for a NULL
 * context. */
int qld_iq_pointers(qld_ctx* ctx, const int32_t** S, const int32_t** C);

/* Empties the window: zeroes the ring and the sums, frames_pushed = 0. */
int qld_reset(qld_ctx* ctx);

/* Frames pushed since creation or the last reset. -1 for NULL. */
long long qld_frames_pushed(const qld_ctx* ctx);

/* Waits for the context's stream; returns any pending CUDA error. */
int qld_sync(qld_ctx* ctx);

/* The context's current stream (a cudaStream_t). */
void* qld_stream(const qld_ctx* ctx);

/* General-frequency lock-in (Methods, "Numerical simulations": the sums of
 * I(t_s) sin(omega_i t_s) and I(t_s) cos(omega_i t_s) with the sine and
 * cosine read from pre-calculated arrays; Fig. 1 uses 20-29 Hz sources and
 * N = 82 or 41 frames, not four samples per period).
 *
 * qld_lockin_table fills table (device float32 [N][2], caller-owned, 8-byte
 * aligned) with (cos, -sin) of omega_dt * s for s = s0 .. s0+N-1, omega_dt =
 * omega * dt in radians per frame, evaluated in FP64 and rounded to float
 * (SI item 1: the set-up thread builds the tables). With omega_dt = 2 pi k / N
 * the table holds the DFT twiddles of bin k.
 *
 * qld_lockin_frames computes, for every pixel of a block of N frames (device
 * [N][H][W], 16-byte aligned, H*W*pixfmt a multiple of 16 bytes; N >= 1, not
 * restricted to multiples of 4), X = sum_j x_j * table[j] accumulated in
 * float32, and writes the amplitude R = |X| = sqrt(S^2 + C^2) into amp and the
 * phase atan2(-S, C) into phase (device float32 [H][W]; either may be NULL).
 * Frame j of the block is the frame of index s0 + j the table was built for.
 * Both enqueue on `stream` and return QLD_E_INVAL for bad arguments. */
int qld_lockin_table(double omega_dt, long long s0, int N, float* table, void* stream);
int qld_lockin_frames(const void* frames, int H, int W, int N, int pixfmt, const float* table, float* amp,
                      float* phase, void* stream);

/* Largest N accepted by qld_fft_bin_frames_noalloc. */
#define QLD_NOALLOC_MAX_N 16384

/* |X_k|^2 of every pixel over a block of N caller frames (device,
 * [N][H][W]) on `stream`, without allocating any memory. The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc while
 * they run -- for example a fixed-memory real-time camera loop, or code that
 * must not trigger the device-wide synchronisation cudaMalloc / cudaFree can
 * cause. The result equals qld_fft_bin on a fresh context into which the
 * same N frames were pushed.
 *
 * Limits and sharing: N must be a multiple of 4 between 4 and
 * QLD_NOALLOC_MAX_N (QLD_E_INVAL otherwise, as for any bad argument); frames
 * must be 16-byte aligned and a frame (H*W*pixfmt bytes) a multiple of 16
 * bytes; out is device float32 [H][W]. The twiddle table lives in one fixed
 * 128 KiB device array that every GPU loading this library holds until the
 * process exits. Each call rewrites the part it uses before reading it, so
 * nothing needs clearing, but all calls share that array: calls that may
 * overlap on the GPU (different streams, no ordering between them) race and
 * can return wrong values.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for the life of the process, so a
 * device reset (cudaDeviceReset) after that first call is not supported.
 * With lazy module loading (the CUDA default) that first call, and the first
 * call with each pixel format, may also load the library's code onto the
 * device, which can allocate device memory and synchronise. Make one call per
 * device and pixel format as a warm-up before the allocation-free region and
 * before any stream capture (or set CUDA_MODULE_LOADING=EAGER, which loads
 * everything when the context is created). Later calls allocate nothing.
 * An error left by earlier asynchronous work is returned (QLD_E_CUDA) before
 * anything is queued. */
int qld_fft_bin_frames_noalloc(const void* frames, int H, int W, int N, int pixfmt, int k, float* out,
                               void* stream);

/* ---- Serving several camera streams (continuous batching) ---------------
 *
 * The paper runs one camera through a real-time loop in which acquisition,
 * transfer and processing overlap and each new frame yields an image (SI,
 * "Timing sequence for hybrid parallelisation"). A server runs that loop for
 * up to QLD_SERVER_MAX_STREAMS streams of different sizes, windows and pixel
 * formats on the current device:
 *  - qld_server_request asks for a stream (H, W, N, pixfmt as for
 *    qld_create; H*W*pixel bytes must be a whole number of 16-byte vectors,
 *    24 for QLD_P12) and returns its ticket. It is admitted at once if its
 *    footprint (qld_footprint_bytes + two float images) fits the server's
 *    HBM budget and a slot is free; otherwise it waits, and waiting requests
 *    are admitted in arrival order whenever a close frees room. A request
 *    larger than the whole budget fails with QLD_E_NOMEM.
 *  - qld_server_submit hands over the next frames of an admitted stream
 *    (device memory, aligned to 16 bytes, 8 for QLD_P12; at most one submission
 *    per stream per tick; QLD_E_NOT_READY while the request waits). The frames
 *    must stay valid until the tick that consumes them has completed.
 *  - qld_server_tick runs every submitted push, with its amplitude/phase image
 *    once the stream's window is full, in ONE kernel launch replayed
 *    from a CUDA graph, on `stream`; it returns the number of streams served.
 *    Streams admitted while earlier ticks are still running join the next tick
 *    (with a one-CTA-per-tile shape, the first tick whose tiles exceed the
 *    graphs' grid waits for the ticks in flight and rebuilds the graphs).
 *  - qld_server_image gives the device pointers of a stream's latest images
 *    (owned by the server; read them after the tick, in stream order).
 *  - qld_server_autotune times the batched kernel's candidate launch shapes
 *    on small-window replicas of the active streams (same bytes per pushed
 *    frame; temporary memory outside the budget), each as the best of three
 *    runs of eight launches back to back (as ticks run), keeps the fastest
 *    and returns its index (best time per tick in *best_us).
 * One host thread must drive a server at a time. */
#define QLD_SERVER_MAX_STREAMS 64
typedef struct qld_server qld_server;
qld_server* qld_server_create(long long hbm_budget_bytes, int max_streams);
void qld_server_destroy(qld_server* srv);
int qld_server_request(qld_server* srv, int H, int W, int N, int pixfmt);
/* 1 = waiting, 0 = admitted, -1 = closed or failed, QLD_E_INVAL = no such ticket */
int qld_server_state(qld_server* srv, int ticket);
int qld_server_close(qld_server* srv, int ticket);
int qld_server_submit(qld_server* srv, int ticket, const void* frames, int count);
/* n submissions in one call (host arrays: tickets[i], frames[i], counts[i],
 * each as for qld_server_submit, distinct tickets). All are checked first;
 * on an error none is taken. */
int qld_server_submit_many(qld_server* srv, int n, const int* tickets, const void* const* frames, const int* counts);
int qld_server_tick(qld_server* srv, void* stream);
/* qld_server_tick behind a bounded device wait on a doorbell: first waits
 * for earlier ticks, then launches, on `stream`, a one-thread kernel that
 * polls *doorbell (a 4-byte-aligned int the device can read: device memory,
 * or the device pointer of mapped pinned host memory; written by a copy
 * engine, e.g. a cudaMemcpyAsync on another non-blocking stream, or by the
 * host -- never by a kernel that could be queued behind this tick, and not
 * through a stream that synchronises with `stream`) until it is >= target,
 * then the tick's
 * kernel, which starts the moment the doorbell rings with no
 * host round trip. The wait gives up after timeout_ns (0 < timeout_ns <=
 * 10 s) of GPU time; the tick then does no work, the submissions stay
 * pending for a later tick, and the call returns QLD_E_TIMEOUT. Otherwise
 * it returns, once the tick has completed, the number of streams served (0,
 * with no wait, when nothing was submitted). QLD_E_INVAL for a NULL or
 * misaligned doorbell or a timeout out of range. */
int qld_server_tick_gated(qld_server* srv, void* stream, const int* doorbell, int target, long long timeout_ns);
/* GPU time of the last gated tick that ran, from the end of its doorbell wait
 * (the doorbell seen) to the tick's images complete, in microseconds (CUDA
 * events on the tick's stream). QLD_E_NOT_READY before the first one. */
int qld_server_last_gated_us(const qld_server* srv, float* us);
int qld_server_image(qld_server* srv, int ticket, float** amp, float** phase);
int qld_server_iq(qld_server* srv, int ticket, int32_t* S, int32_t* C);
long long qld_server_frames_pushed(qld_server* srv, int ticket);
long long qld_server_mem_in_use(const qld_server* srv);
int qld_server_sync(qld_server* srv);
int qld_server_autotune(qld_server* srv, void* stream, float* best_us);
/* The current launch shape; *ctas_per_sm = 0 means one CTA per tile of
 * threads x vectors_per_thread vectors (a grid covering every admitted
 * stream) instead of a persistent grid of SMs x ctas_per_sm CTAs. */
int qld_server_shape(const qld_server* srv, int* threads, int* vectors_per_thread, int* ctas_per_sm);
/* Number of candidate launch shapes, and a fixed choice of one (0 <= index <
 * qld_server_num_shapes(), else QLD_E_INVAL) in place of the autotuner's:
 * waits for the ticks in flight; the next tick runs with it. */
int qld_server_num_shapes(void);
int qld_server_set_shape(qld_server* srv, int index);

/* ---- Learned short-window QLD: network kernels --------------------------
 *
 * No counterpart in the paper (which motivates shorter time series for lower
 * latency, SI "Timing sequence" and the tree/cow experiment): a small U-Net
 * maps the I/Q maps of a short window to the amplitude plain QLD reaches with
 * a long window. Its building blocks, all on `stream`, all device pointers:
 *  - qldnn_conv3x3_fwd: out = relu?(conv3x3(in, w) + bias), zero padding 1,
 *    BF16 tensor-core implicit GEMM with FP32 accumulation. in [B][H][W][Cin]
 *    bf16 (Cin % 16 == 0, 16-byte aligned), w [9][Cin][Cout] bf16 (tap =
 *    3 ky + kx; Cout % 32 == 0), bias [Cout] f32 or NULL; out_bf16 and/or
 *    out_f32 [B][H][W][Cout].
 *  - qldnn_conv3x3_dgrad: din = data gradient of that convolution for the
 *    output gradient g [B][H][W][Cout] bf16 (Cin % 32 == 0); wt_scratch holds
 *    9 Cin Cout bf16 (the flipped, transposed weights).
 *  - qldnn_conv3x3_wgrad: dw [9][Cin][Cout] f32 += weight gradient (the
 *    caller zeroes dw); tensor-core GEMM over pixels, split across CTAs.
 *  - qldnn_bias_grad (db [C] += sum of g; C <= 256), qldnn_relu_bwd
 *    (out = bf16(g * (act > 0))), qldnn_avgpool2 / _bwd, qldnn_upsample2
 *    (nearest) / _bwd, qldnn_concat / qldnn_split (channels), qldnn_head /
 *    _bwd (1x1 convolution to one f32 channel), qldnn_mse (loss += mean
 *    square error, grad = its gradient), qldnn_adam (Adam on f32 master
 *    weights, refreshing an optional bf16 copy), qldnn_cast_bf16, qldnn_add,
 *    qldnn_pack_input (network input: S, C, sqrt(S^2 + C^2) times `scale`,
 *    zero-padded to 16 channels; optionally the scaled amplitude in f32 as
 *    `baseline`; out 16-byte aligned), qldnn_zero (clears a device buffer).
 * Pooling, upsampling, concatenation and the head move 8 channels (16 bytes)
 * per thread when the channel counts are multiples of 8 and the pointers
 * 16-byte aligned, else one element per thread.
 * All return QLD_OK or QLD_E_INVAL / QLD_E_CUDA. */
int qldnn_conv3x3_fwd(const void* in, const void* w, const float* bias, int B, int H, int W, int Cin, int Cout,
                      int relu, void* out_bf16, float* out_f32, void* stream);
int qldnn_conv3x3_dgrad(const void* g, const void* w, int B, int H, int W, int Cin, int Cout, void* wt_scratch,
                        void* din_bf16, float* din_f32, void* stream);
int qldnn_conv3x3_wgrad(const void* in, const void* g, int B, int H, int W, int Cin, int Cout, float* dw,
                        void* stream);
int qldnn_bias_grad(const void* g, long long P, int C, float* db, void* stream);
int qldnn_relu_bwd(const float* g, const void* act, long long n, void* out_bf16, void* stream);
/* qldnn_relu_bwd and qldnn_bias_grad in one pass over [P][C] (C % 8 == 0,
 * C <= 256, pointers 16-byte aligned): out = bf16(g * (act > 0)), db [C] +=
 * the per-channel sums of those bf16 values. */
int qldnn_relu_bwd_bias(const float* g, const void* act, long long P, int C, void* out_bf16, float* db,
                        void* stream);
int qldnn_avgpool2(const void* in, int B, int H, int W, int C, void* out, void* stream);
int qldnn_avgpool2_bwd(const float* g, int B, int H, int W, int C, float* out, int accumulate, void* stream);
int qldnn_upsample2(const void* in, int B, int h, int w, int C, void* out, void* stream);
int qldnn_upsample2_bwd(const float* g, int B, int h, int w, int C, float* out, void* stream);
int qldnn_concat(const void* a, int Ca, const void* b, int Cb, long long P, void* out, void* stream);
/* Decoder skip input in one pass: out [B][2h][2w][Cu + Ce] bf16 = the
 * nearest 2x upsampling of u [B][h][w][Cu] followed by e [B][2h][2w][Ce]
 * along channels (Cu, Ce multiples of 8; pointers 16-byte aligned). */
int qldnn_upsample_concat(const void* u, int Cu, const void* e, int Ce, int B, int h, int w, void* out,
                          void* stream);
int qldnn_split(const float* g, long long P, int Ca, int Cb, float* ga, float* gb, int accumulate_b, void* stream);
int qldnn_head(const void* in, const float* w, const float* b, long long P, int C, float* out, void* stream);
int qldnn_head_bwd(const void* in, const float* g, const float* w, long long P, int C, float* din, float* dw,
                   float* db, void* stream);
int qldnn_mse(const float* pred, const float* target, long long n, float* grad, float* loss, void* stream);
int qldnn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
               int t, void* p_bf16, void* stream);
int qldnn_cast_bf16(const float* x, long long n, void* y, void* stream);
int qldnn_add(float* y, const float* x, long long n, void* stream);
int qldnn_pack_input(const int32_t* S, const int32_t* C, long long npix, float scale, void* out, float* baseline,
                     void* stream);
int qldnn_zero(void* p, long long bytes, void* stream);
/* The same forward convolution on the 5th-generation tensor cores
 * (tcgen05.mma, accumulator in tensor memory, operands staged by cp.async in
 * the canonical K-major layout). wk holds the weights K-major, as written by
 * qldnn_kmajor_weights(w, Cin, Cout, 0, wk): wk[tap][co][ci]. With
 * qldnn_kmajor_weights(w, Cin, Cout, 1, wk) (wk[tap][ci][co] = w[8-tap][ci][co])
 * the call qldnn_conv3x3_fwd_tc(g, wk, NULL, B, H, W, Cout, Cin, 0, ...) is the
 * data gradient. out_bf16 / out_f32 must be 16-byte aligned. status (device
 * int, may be NULL) becomes 1 if a bounded wait inside the kernel ran out. */
int qldnn_kmajor_weights(const void* w, int Cin, int Cout, int flip, void* wk, void* stream);
/* The learned network's first layer fused with its input packing: out =
 * act(conv3x3(pack(S, C)) + bias) where pack is qldnn_pack_input's tensor
 * (channels s, c, sqrt(s^2 + c^2) times `scale` in bf16, zeros after them);
 * only the weights of input channels 0..2 of w [9][Cin][Cout] bf16 enter.
 * Computed on the FP32 cores (27 x Cout per pixel). S, C int32 [B][H][W];
 * out [B][H][W] rows of ldo >= Cout channels (a multiple of 8, 16-byte
 * aligned), Cout 32 or 64; baseline [B][H][W] f32 (or NULL) = the scaled
 * amplitude, as qldnn_pack_input writes it. */
int qldnn_input_conv3x3(const int32_t* S, const int32_t* C, int B, int H, int W, float scale, const void* w,
                        int Cin, int Cout, const float* bias, int relu, void* out_bf16, long long ldo, float* baseline,
                        void* stream);
/* Warp-specialised version of qldnn_conv3x3_fwd_tc (same arguments and
 * results; Cout must be 32, 64, 128 or 256, one tile of all output channels):
 * producer warps keep a 4-stage shared-memory ring of gathered K steps ahead
 * of a single MMA-issuing warp, synchronised by mbarriers. */
int qldnn_conv3x3_fwd_tc2(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout,
                          int relu, void* out_bf16, float* out_f32, int* status, void* stream);
/* Persistent TMA-fed version (same arguments and results; Cout 32, 64, 128
 * or 256; Cin a multiple of 16): output tiles of 8 x 16 pixels, the input
 * halo staged once per channel chunk by the tensor-memory accelerator (zero
 * fill at the image border), two TMEM accumulators so one tile's read-out
 * overlaps the next tile's MMAs. Launches one CTA per SM. */
int qldnn_conv3x3_fwd_tma(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout,
                          int relu, void* out_bf16, float* out_f32, int* status, void* stream);
/* The same with the kernel variant chosen by the caller. qldnn_conv3x3_fwd_tma
 * keeps the weights resident in shared memory when 9 Cin (Cout / splits) bf16
 * fit beside two halo stages (loaded once per CTA, only the halos streamed)
 * and streams them per tile otherwise; when a layer has at most half as many
 * output tiles as there are SMs it splits each tile's output channels over 2
 * or 4 CTAs (at least 32 channels each, weights resident), and 128-channel
 * layers of at most 128 input channels and 64-channel layers of 128+ input
 * channels with at most one tile per SM always split; 32-channel layers (any input width) whose weights and two halo
 * stages fit in half the shared memory run two CTAs per SM when each gets at
 * least two tiles (one
 * CTA's MMAs fill the other's pauses for barriers); 32-channel slices of 64+
 * input channels with at least 8 tiles per SM or of 128+ input channels, and
 * 64-channel slices of 128+ input channels with at least 2 tiles per SM,
 * stack the column taps (bit 16 below);
 * weight-streaming slices of 64+ columns read out with eight epilogue warps
 * (bit 18 below). The choice depends on the shape (and a fused head) only, so
 * a layer gives the same result with fused and with separate outputs. mode bit
 * 0 set: always stream the weights;
 * mode >> 4 (0 = automatic, else 1, 2 or 4): the CTAs per tile; bit 12 /
 * bit 13: force / forbid 16 x 16-pixel tiles where they fit; bit 14 / bit 15:
 * forbid / force two CTAs per SM where they fit; bit 16 / bit 17: ask for /
 * forbid the column-stacked form for 32- and 64-channel slices with resident
 * weights (the three column taps kx of a tap row as one MMA of 3 x the
 * slice's columns against an unshifted halo, tiles 14 columns wide, the
 * three column groups added in the epilogue: (D_0 + D_1) + D_2, FP32); bit
 * 18 / bit 19: ask for / forbid eight epilogue warps in the weight-streaming
 * variant for slices of 64+ columns (two warps per accumulator lane quarter,
 * each reading half the columns; not with a fused head; the default there). Other bits:
 * QLD_E_INVAL. For tests and measurements of every variant. */
int qldnn_conv3x3_fwd_tma_mode(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin,
                               int Cout, int relu, void* out_bf16, float* out_f32, int* status, int mode,
                               void* stream);
/* Self-test of the failure path shared by the tcgen05 kernels' bounded waits
 * (the paper has no counterpart): one role waits on an mbarrier nothing ever
 * arrives on for limit_ns (1 us .. 2 s) and must time out and raise the
 * failure flag; a second role, waiting with a one-minute limit, must then give
 * up at once. out (device, 3 x int64): [0] = 1 if the first wait timed out,
 * [1] = 1 if the second left because of the flag, [2] = the kernel's device
 * time in ns. Nothing faults; the context stays usable. */
int qldnn_wait_selftest(long long limit_ns, long long* out, void* stream);
/* flags bit QLDNN_EARLY_LAUNCH of qldnn_conv3x3_fwd_tma_epi: launch with
 * programmatic stream serialisation. The kernel may then start while the
 * kernel before it on the stream is still running: it allocates TMEM, sets
 * up its barriers and loads resident weights, and waits for that kernel to
 * complete (griddepcontrol.wait) before it reads its input or writes any
 * output. The caller guarantees that the preceding kernel does not write
 * this layer's weights or bias (inference); the layer-to-layer gaps of a
 * network then overlap. Other flag bits: QLD_E_INVAL. */
#define QLDNN_EARLY_LAUNCH 1
/* The persistent TMA convolution with the layer's neighbours fused into its
 * epilogue (inference of the learned network). Any of:
 *   out_bf16  the activation, rows of ldo >= Cout channels (a multiple of 8):
 *             with ldo > Cout it fills a channel slice of a concatenated tensor
 *   pool_bf16 [B][H/2][W/2][Cout], the 2x2 average of the bf16 activation
 *             (H and W even)
 *   up_bf16   [B][2H][2W], rows of ldu channels: the nearest 2x upsampling,
 *             e.g. into the first channels of the next level's skip concat
 *   head      pred [B][H][W] f32 = head_b[0] + sum_c act[c] head_w[c] +
 *             baseline[p] (head_w [Cout], head_b, baseline, pred all given)
 * The pooled, upsampled and head outputs equal qldnn_avgpool2,
 * qldnn_upsample_concat and qldnn_head + qldnn_add on the bf16 activation bit
 * for bit. Pointers 16-byte aligned. */
int qldnn_conv3x3_fwd_tma_epi(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin,
                              int Cout, int relu, void* out_bf16, long long ldo, void* pool_bf16, void* up_bf16,
                              long long ldu, const float* head_w, const float* head_b, const float* baseline,
                              float* pred, int* status, int flags, void* stream);
/* The same with the kernel variant chosen by the caller: mode bits 0, 4-7
 * and 12-19 as in qldnn_conv3x3_fwd_tma_mode (4-7, the CTAs per tile, only
 * without a head; other bits: QLD_E_INVAL). For tests and measurements of
 * every variant with fused outputs. */
int qldnn_conv3x3_fwd_tma_epi_mode(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin,
                                   int Cout, int relu, void* out_bf16, long long ldo, void* pool_bf16, void* up_bf16,
                                   long long ldu, const float* head_w, const float* head_b, const float* baseline,
                                   float* pred, int* status, int flags, int mode, void* stream);
/* Weight gradient of the 3x3 convolution on the tensor cores: dw [9][Cin][Cout]
 * f32 += sum over pixels of in (shifted by the tap) x g, in [B][H][W][Cin]
 * and g [B][H][W][Cout] bf16 (the caller zeroes dw; 16-byte aligned). Cin is
 * 16, 32, 64 or a multiple of 128; Cout is 32, 64 or 128. TMA-fed, operands
 * read MN-major from the NHWC tiles, FP32 accumulation in TMEM per work item
 * (column shift kx, 128-channel block, range of 8 x 16-pixel tiles), then
 * 16-byte float atomics into dw (the summation order across items is not
 * fixed). *status = 1 if a pipeline wait timed out. */
int qldnn_conv3x3_wgrad_tma(const void* in, const void* g, int B, int H, int W, int Cin, int Cout, float* dw,
                            int* status, void* stream);
int qldnn_conv3x3_fwd_tc(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout,
                         int relu, void* out_bf16, float* out_f32, int* status, void* stream);

/* Kernels this library has launched in this process (all contexts). */
long long qld_launch_count(void);

/* Status text; last status set on this thread; version string. */
const char* qld_strerror(int status);
int qld_last_error(void);
const char* qld_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QLD_H */
