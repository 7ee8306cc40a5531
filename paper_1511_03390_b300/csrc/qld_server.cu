// qld_server.cu -- serving several camera streams with continuous batching.
//
// The paper runs one camera through a real-time loop in which acquisition,
// transfer and QLD processing overlap and every new frame yields an image
// (SI, "Timing sequence for hybrid parallelisation"; its closing paragraph on
// the sliding sequence). The server keeps that loop for many streams of
// different resolutions, windows and pixel formats on one GPU:
//   * each admitted stream owns a context (ring, sums, twiddles) and two
//     image buffers; requests are admitted in arrival order while their
//     footprint fits the server's HBM budget and a slot is free, and a
//     request that does not fit waits until closes free enough memory;
//   * a tick takes the frames submitted since the previous tick and runs all
//     of their pushes and images in ONE launch (batch_push_kernel)
//     replayed from a CUDA graph; streams admitted while earlier ticks are
//     still on the GPU simply join the next tick's batch;
//   * the launch shape is chosen by timing the candidate shapes on small
//     replicas of the current stream mix (qld_server_autotune).
// One host thread drives a server at a time (no internal locking).

#include <algorithm>
#include <cstring>
#include <deque>
#include <vector>

#include "qld.h"
#include "qld_batch.cuh"
#include "qld_internal.h"

using qldi::set_err;

namespace {

struct SrvStream {
    int state;  // 1 waiting, 0 active, -1 closed
    int H, W, N, pixfmt;
    long long footprint;  // context + amplitude and phase images
    qld_ctx* ctx;
    float* amp;
    float* phase;
    const void* pending;
    int pending_count;
};

long long stream_footprint(int H, int W, int N, int pixfmt) {
    const long long f = qld_footprint_bytes(H, W, N, pixfmt);
    return f < 0 ? f : f + 2ll * H * W * (long long)sizeof(float);
}

}  // namespace

struct qld_server {
    int device;
    int num_sms;
    long long budget;
    long long in_use;
    int max_streams;
    std::vector<SrvStream> streams;  // index = ticket
    std::deque<int> waiting;         // tickets in arrival order
    // a tick's descriptors (alternating ticks), handed to the batch kernel as
    // its parameter by updating the graph's kernel node: no copy to the device
    qldk::BatchParams* prm[2];
    int* gate_dev;                   // outcome of a gated tick's doorbell wait
    cudaEvent_t gate_ev[2];          // after the doorbell wait, after the gated tick (timing)
    float last_gated_us;             // the last gated tick: doorbell seen -> images complete
    cudaEvent_t used[2];
    bool used_valid[2];
    cudaGraphExec_t graph[2];
    cudaGraph_t graph_def[2];         // kept for their kernel nodes
    cudaGraphNode_t node[2];          // the batch kernel of graph b
    cudaKernelNodeParams node_prm[2]; // its function and launch shape
    bool graph_valid;
    long long graph_tiles;           // tiles the graphs' grid covers (one-CTA-per-tile shapes)
    cudaStream_t cap;
    int shape;
    int flip;
};

namespace {

// Longest doorbell wait a gated tick accepts (10 s).
constexpr long long kMaxGateNs = 10000000000ll;

static_assert(QLD_SERVER_MAX_STREAMS <= qldk::kMaxBatchItems, "a tick's descriptors must fit its kernel parameter");

int active_count(const qld_server* s) {
    int n = 0;
    for (const SrvStream& t : s->streams) n += t.state == 0;
    return n;
}

// Waits for every tick that may still use stream memory or the pinned
// descriptors.
void wait_ticks(qld_server* s) {
    for (int b = 0; b < 2; ++b)
        if (s->used_valid[b]) cudaEventSynchronize(s->used[b]);
}

void release_stream(qld_server* s, SrvStream& t) {
    if (t.ctx) qld_destroy(t.ctx);
    if (t.amp) cudaFree(t.amp);
    if (t.phase) cudaFree(t.phase);
    t.ctx = nullptr;
    t.amp = t.phase = nullptr;
}

// Admits waiting requests in arrival order while the first one fits.
void admit_waiting(qld_server* s) {
    while (!s->waiting.empty()) {
        SrvStream& t = s->streams[s->waiting.front()];
        if (s->in_use + t.footprint > s->budget || active_count(s) >= s->max_streams) return;
        s->waiting.pop_front();
        const long long npix = (long long)t.H * t.W;
        t.ctx = qld_create(t.H, t.W, t.N, t.pixfmt);
        if (!t.ctx || cudaMalloc(&t.amp, npix * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&t.phase, npix * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            release_stream(s, t);
            t.state = -1;  // the device itself is out of memory: the request fails
            continue;
        }
        t.state = 0;
        s->in_use += t.footprint;
    }
}

// Fills the descriptors of one push per pending stream (for the given
// contexts / counts); returns the number of items and the number of tiles.
int build_items(qld_server* s, qldk::BatchItem* items, qldk::BatchHeader* hdr, std::vector<int>* which) {
    const long long tv = qldk::batch_tile_vectors(qldk::kBatchShapes[s->shape]);
    int n = 0;
    long long tiles = 0;
    for (int id = 0; id < (int)s->streams.size(); ++id) {
        SrvStream& t = s->streams[id];
        if (t.state != 0 || t.pending_count == 0) continue;
        qld_ctx* c = t.ctx;
        const int count = t.pending_count;
        const bool reset = count >= c->N;
        const int first = reset ? count - c->N : 0;
        qldk::BatchItem& it = items[n];
        std::memset(&it, 0, sizeof(it));
        qldk::PushArgs& a = it.a;
        a.frames = (const uint8_t*)t.pending + (long long)first * c->frame_bytes;
        a.frame_stride = c->frame_bytes;
        a.nf = reset ? c->N : count;
        a.s_first = c->pushed + first + 1;
        a.ring = c->ring;
        a.slot_stride = c->slot_stride;
        a.N = c->N;
        a.S = c->S;
        a.C = c->C;
        a.npix = c->npix;
        a.nvec = c->frame_bytes / qldk::batch_vec_bytes(c->pixfmt);
        a.amp = t.amp;
        a.phase = t.phase;
        a.out_aligned = 1;
        it.fmt = c->pixfmt;
        it.reset = reset ? 1 : 0;
        it.epi = (c->pushed + count >= c->N) ? 1 : 0;
        it.tile0 = tiles;
        tiles += (a.nvec + tv - 1) / tv;
        if (which) which->push_back(id);
        ++n;
    }
    hdr->nitems = n;
    hdr->gated = 0;
    hdr->ntiles = tiles;
    return n;
}

// Tiles of one push of every admitted stream with the current shape: the
// most a tick can launch.
long long admitted_tiles(const qld_server* s) {
    const long long tv = qldk::batch_tile_vectors(qldk::kBatchShapes[s->shape]);
    long long tiles = 0;
    for (const SrvStream& t : s->streams)
        if (t.state == 0 && t.ctx) tiles += (t.ctx->frame_bytes / qldk::batch_vec_bytes(t.ctx->pixfmt) + tv - 1) / tv;
    return tiles;
}

// One-CTA-per-tile graphs are rebuilt when a tick has more tiles than their
// grid covers (streams admitted since they were captured).
void check_graph_grid(qld_server* s, long long tick_tiles) {
    if (qldk::kBatchShapes[s->shape].ctas_per_sm == 0 && s->graph_valid && tick_tiles > s->graph_tiles) {
        wait_ticks(s);
        s->graph_valid = false;
    }
}

void free_graphs(qld_server* s) {
    for (int b = 0; b < 2; ++b) {
        if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
        if (s->graph_def[b]) cudaGraphDestroy(s->graph_def[b]);
        s->graph[b] = nullptr;
        s->graph_def[b] = nullptr;
        s->node[b] = nullptr;
    }
}

// Captures the two tick graphs (one batch kernel node each) for the current
// launch shape; a tick then only sets that node's parameter.
int ensure_graphs(qld_server* s) {
    if (s->graph_valid) return QLD_OK;
    free_graphs(s);
    s->graph_tiles = admitted_tiles(s);
    for (int b = 0; b < 2; ++b) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return QLD_E_CUDA;
        qldk::launch_batch(qldk::kBatchShapes[s->shape], s->num_sms, s->graph_tiles, *s->prm[b], s->gate_dev, s->cap);
        if (cudaStreamEndCapture(s->cap, &g) != cudaSuccess || !g) {
            cudaGetLastError();
            return QLD_E_CUDA;
        }
        s->graph_def[b] = g;
        size_t nn = 1;
        cudaGraphNode_t nd = nullptr;
        if (cudaGraphGetNodes(g, &nd, &nn) != cudaSuccess || nn != 1 || !nd ||
            cudaGraphKernelNodeGetParams(nd, &s->node_prm[b]) != cudaSuccess ||
            cudaGraphInstantiate(&s->graph[b], g, 0) != cudaSuccess) {
            cudaGetLastError();
            free_graphs(s);
            return QLD_E_CUDA;
        }
        s->node[b] = nd;
    }
    s->graph_valid = true;
    return QLD_OK;
}

// Hands the descriptors in s->prm[b] to graph b's kernel (copied by the call).
int set_tick_params(qld_server* s, int b) {
    void* args[2] = {s->prm[b], &s->gate_dev};
    cudaKernelNodeParams kp = s->node_prm[b];
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphExecKernelNodeSetParams(s->graph[b], s->node[b], &kp) == cudaSuccess ? QLD_OK : QLD_E_CUDA;
}

SrvStream* get_stream(qld_server* s, int ticket) {
    if (!s || ticket < 0 || ticket >= (int)s->streams.size()) return nullptr;
    return &s->streams[ticket];
}

}  // namespace

extern "C" {

qld_server* qld_server_create(long long hbm_budget_bytes, int max_streams) {
    if (hbm_budget_bytes <= 0 || max_streams < 1 || max_streams > QLD_SERVER_MAX_STREAMS) {
        set_err(QLD_E_INVAL);
        return nullptr;
    }
    qld_server* s = new qld_server();
    s->budget = hbm_budget_bytes;
    s->in_use = 0;
    s->max_streams = max_streams;
    s->prm[0] = s->prm[1] = nullptr;
    s->gate_dev = nullptr;
    s->gate_ev[0] = s->gate_ev[1] = nullptr;
    s->last_gated_us = -1.f;
    s->used_valid[0] = s->used_valid[1] = false;
    s->graph[0] = s->graph[1] = nullptr;
    s->graph_def[0] = s->graph_def[1] = nullptr;
    s->node[0] = s->node[1] = nullptr;
    s->graph_valid = false;
    s->graph_tiles = 0;
    s->cap = nullptr;
    s->shape = 0;
    s->flip = 0;
    bool ok = cudaGetDevice(&s->device) == cudaSuccess &&
              cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess &&
              cudaMalloc(&s->gate_dev, 16) == cudaSuccess && cudaMemset(s->gate_dev, 0, 16) == cudaSuccess &&
              cudaEventCreate(&s->gate_ev[0]) == cudaSuccess && cudaEventCreate(&s->gate_ev[1]) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b < 2; ++b) {
        s->prm[b] = new qldk::BatchParams();
        std::memset(s->prm[b], 0, sizeof(qldk::BatchParams));
        ok = cudaEventCreateWithFlags(&s->used[b], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        qld_server_destroy(s);
        set_err(QLD_E_NOMEM);
        return nullptr;
    }
    return s;
}

void qld_server_destroy(qld_server* s) {
    if (!s) return;
    wait_ticks(s);
    for (SrvStream& t : s->streams) release_stream(s, t);
    free_graphs(s);
    for (int b = 0; b < 2; ++b) {
        delete s->prm[b];
        if (s->used[b]) cudaEventDestroy(s->used[b]);
    }
    if (s->gate_dev) cudaFree(s->gate_dev);
    for (int e = 0; e < 2; ++e)
        if (s->gate_ev[e]) cudaEventDestroy(s->gate_ev[e]);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

int qld_server_request(qld_server* s, int H, int W, int N, int pixfmt) {
    if (!s) return set_err(QLD_E_INVAL);
    const long long fp = stream_footprint(H, W, N, pixfmt);
    if (fp < 0) return set_err(QLD_E_INVAL);
    // batched pushes use the vector path: whole vectors per frame
    if (qldi::frame_bytes_of((long long)H * W, pixfmt) % qldi::vec_bytes_of(pixfmt) != 0) return set_err(QLD_E_INVAL);
    if (fp > s->budget) return set_err(QLD_E_NOMEM);
    SrvStream t;
    std::memset(&t, 0, sizeof(t));
    t.state = 1;
    t.H = H;
    t.W = W;
    t.N = N;
    t.pixfmt = pixfmt;
    t.footprint = fp;
    s->streams.push_back(t);
    const int ticket = (int)s->streams.size() - 1;
    s->waiting.push_back(ticket);
    admit_waiting(s);
    return ticket;
}

int qld_server_state(qld_server* s, int ticket) {
    SrvStream* t = get_stream(s, ticket);
    if (!t) return set_err(QLD_E_INVAL);
    return t->state;
}

int qld_server_close(qld_server* s, int ticket) {
    SrvStream* t = get_stream(s, ticket);
    if (!t || t->state < 0) return set_err(QLD_E_INVAL);
    if (t->state == 1) {
        s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), ticket));
    } else {
        wait_ticks(s);
        release_stream(s, *t);
        s->in_use -= t->footprint;
    }
    t->state = -1;
    admit_waiting(s);
    return QLD_OK;
}

int qld_server_submit(qld_server* s, int ticket, const void* frames, int count) {
    SrvStream* t = get_stream(s, ticket);
    if (!t || count < 0 || (count > 0 && !frames)) return set_err(QLD_E_INVAL);
    if (t->state == 1) return set_err(QLD_E_NOT_READY);
    if (t->state != 0 || t->pending_count > 0) return set_err(QLD_E_INVAL);
    if (count > 0 && ((uintptr_t)frames % qldi::vec_align_of(t->pixfmt)) != 0) return set_err(QLD_E_INVAL);
    t->pending = frames;
    t->pending_count = count;
    return QLD_OK;
}

int qld_server_submit_many(qld_server* s, int n, const int* tickets, const void* const* frames, const int* counts) {
    if (!s || n < 0 || (n > 0 && (!tickets || !frames || !counts))) return set_err(QLD_E_INVAL);
    // validate everything first: either every submission is taken or none
    for (int i = 0; i < n; ++i) {
        const SrvStream* t = get_stream(s, tickets[i]);
        const int count = counts[i];
        if (!t || count < 0 || (count > 0 && !frames[i])) return set_err(QLD_E_INVAL);
        if (t->state == 1) return set_err(QLD_E_NOT_READY);
        if (t->state != 0 || t->pending_count > 0) return set_err(QLD_E_INVAL);
        if (count > 0 && ((uintptr_t)frames[i] % qldi::vec_align_of(t->pixfmt)) != 0) return set_err(QLD_E_INVAL);
        for (int j = 0; j < i; ++j)
            if (tickets[j] == tickets[i]) return set_err(QLD_E_INVAL);  // one submission per stream per tick
    }
    for (int i = 0; i < n; ++i) {
        SrvStream* t = get_stream(s, tickets[i]);
        t->pending = frames[i];
        t->pending_count = counts[i];
    }
    return QLD_OK;
}

int qld_server_tick(qld_server* s, void* stream) {
    if (!s) return set_err(QLD_E_INVAL);
    const cudaStream_t st = (cudaStream_t)stream;
    const int b = s->flip;
    if (s->used_valid[b] && cudaEventSynchronize(s->used[b]) != cudaSuccess) return set_err(QLD_E_CUDA);
    std::vector<int> which;
    const int n = build_items(s, s->prm[b]->items, &s->prm[b]->hdr, &which);
    if (n == 0) return 0;
    check_graph_grid(s, s->prm[b]->hdr.ntiles);
    int rc = ensure_graphs(s);
    if (rc == QLD_OK) rc = set_tick_params(s, b);
    if (rc != QLD_OK) return set_err(rc);
    if (cudaGraphLaunch(s->graph[b], st) != cudaSuccess || cudaEventRecord(s->used[b], st) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    s->used_valid[b] = true;
    qldi::count_launches(1);
    for (int id : which) {
        SrvStream& t = s->streams[id];
        t.ctx->pushed += t.pending_count;
        t.ctx->stream = st;
        t.pending = nullptr;
        t.pending_count = 0;
    }
    s->flip ^= 1;
    return n;
}

int qld_server_tick_gated(qld_server* s, void* stream, const int* doorbell, int target, long long timeout_ns) {
    if (!s || !doorbell || ((uintptr_t)doorbell & 3) != 0 || timeout_ns <= 0 || timeout_ns > kMaxGateNs)
        return set_err(QLD_E_INVAL);
    const cudaStream_t st = (cudaStream_t)stream;
    // no earlier tick in flight, so a timed-out tick is undone on the host alone
    wait_ticks(s);
    const int b = s->flip;
    std::vector<int> which;
    const int n = build_items(s, s->prm[b]->items, &s->prm[b]->hdr, &which);
    if (n == 0) return 0;
    s->prm[b]->hdr.gated = 1;
    check_graph_grid(s, s->prm[b]->hdr.ntiles);
    int rc = ensure_graphs(s);
    if (rc == QLD_OK) rc = set_tick_params(s, b);
    if (rc != QLD_OK) return set_err(rc);
    qldk::doorbell_gate_kernel<<<1, 32, 0, st>>>(doorbell, target, timeout_ns, s->gate_dev);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(s->gate_ev[0], st) != cudaSuccess ||
        cudaGraphLaunch(s->graph[b], st) != cudaSuccess || cudaEventRecord(s->gate_ev[1], st) != cudaSuccess ||
        cudaEventRecord(s->used[b], st) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    s->used_valid[b] = true;
    qldi::count_launches(2);
    s->flip ^= 1;
    // the device wait is bounded, so this returns within about timeout_ns
    int gate = 1;
    if (cudaEventSynchronize(s->used[b]) != cudaSuccess ||
        cudaMemcpy(&gate, s->gate_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    if (gate != 0) return set_err(QLD_E_TIMEOUT);  // nothing ran; the submissions stay pending
    float ms = -1.f;
    s->last_gated_us = cudaEventElapsedTime(&ms, s->gate_ev[0], s->gate_ev[1]) == cudaSuccess ? ms * 1e3f : -1.f;
    for (int id : which) {
        SrvStream& t = s->streams[id];
        t.ctx->pushed += t.pending_count;
        t.ctx->stream = st;
        t.pending = nullptr;
        t.pending_count = 0;
    }
    return n;
}

int qld_server_last_gated_us(const qld_server* s, float* us) {
    if (!s || !us) return set_err(QLD_E_INVAL);
    if (s->last_gated_us < 0.f) return set_err(QLD_E_NOT_READY);
    *us = s->last_gated_us;
    return QLD_OK;
}

int qld_server_image(qld_server* s, int ticket, float** amp, float** phase) {
    SrvStream* t = get_stream(s, ticket);
    if (!t || t->state != 0) return set_err(QLD_E_INVAL);
    if (t->ctx->pushed < t->N) return set_err(QLD_E_NOT_READY);
    if (amp) *amp = t->amp;
    if (phase) *phase = t->phase;
    return QLD_OK;
}

int qld_server_iq(qld_server* s, int ticket, int32_t* S, int32_t* C) {
    SrvStream* t = get_stream(s, ticket);
    if (!t || t->state != 0) return set_err(QLD_E_INVAL);
    return qld_get_iq(t->ctx, S, C);
}

long long qld_server_frames_pushed(qld_server* s, int ticket) {
    SrvStream* t = get_stream(s, ticket);
    if (!t || t->state != 0) return -1;
    return t->ctx->pushed;
}

long long qld_server_mem_in_use(const qld_server* s) { return s ? s->in_use : -1; }

int qld_server_sync(qld_server* s) {
    if (!s) return set_err(QLD_E_INVAL);
    for (int b = 0; b < 2; ++b)
        if (s->used_valid[b] && cudaEventSynchronize(s->used[b]) != cudaSuccess) return set_err(QLD_E_CUDA);
    return cudaGetLastError() == cudaSuccess ? QLD_OK : set_err(QLD_E_CUDA);
}

int qld_server_num_shapes(void) { return qldk::kNumBatchShapes; }

int qld_server_set_shape(qld_server* s, int index) {
    if (!s || index < 0 || index >= qldk::kNumBatchShapes) return set_err(QLD_E_INVAL);
    if (index != s->shape) {
        wait_ticks(s);  // the graphs are rebuilt at the next tick
        s->shape = index;
        s->graph_valid = false;
    }
    return QLD_OK;
}

int qld_server_shape(const qld_server* s, int* threads, int* vectors_per_thread, int* ctas_per_sm) {
    if (!s) return set_err(QLD_E_INVAL);
    const qldk::BatchShape& sh = qldk::kBatchShapes[s->shape];
    if (threads) *threads = sh.threads;
    if (vectors_per_thread) *vectors_per_thread = sh.vpt;
    if (ctas_per_sm) *ctas_per_sm = sh.ctas_per_sm;
    return QLD_OK;
}

int qld_server_autotune(qld_server* s, void* stream, float* best_us) {
    if (!s) return set_err(QLD_E_INVAL);
    const cudaStream_t st = (cudaStream_t)stream;
    wait_ticks(s);
    // Replicas of the active streams with a 4-frame window: one pushed frame
    // moves the same bytes whatever N is (new and expiring frame, ring
    // write, sums, image).
    std::vector<SrvStream> rep;
    for (const SrvStream& t : s->streams) {
        if (t.state != 0) continue;
        SrvStream r = t;
        r.N = 4;
        r.ctx = qld_create(t.H, t.W, 4, t.pixfmt);
        r.amp = r.phase = nullptr;
        r.pending = nullptr;
        r.pending_count = 0;
        const long long npix = (long long)t.H * t.W;
        void* frame = nullptr;
        if (!r.ctx || cudaMalloc(&r.amp, npix * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&r.phase, npix * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&frame, r.ctx->frame_bytes * 8) != cudaSuccess ||
            cudaMemsetAsync(frame, 0x5A, r.ctx->frame_bytes * 8, st) != cudaSuccess) {
            cudaGetLastError();
            if (frame) cudaFree(frame);
            release_stream(s, r);
            for (SrvStream& x : rep) {
                cudaFree((void*)x.pending);
                release_stream(s, x);
            }
            return set_err(QLD_E_NOMEM);
        }
        r.pending = frame;
        rep.push_back(r);
    }
    if (rep.empty()) return set_err(QLD_E_NOT_READY);
    qldk::BatchParams* pp = new qldk::BatchParams();
    std::memset(pp, 0, sizeof(*pp));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QLD_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = QLD_E_NOMEM;
    const int saved_shape = s->shape;
    float best = 1e30f;
    int best_shape = saved_shape;
    qld_server probe = *s;  // build_items on the replicas with each candidate shape
    probe.streams = rep;
    // Each shape: 3 launches of warm-up, then the best of 3 runs of 8 launches
    // back to back, as ticks run (timing launches one at a time, with a
    // synchronisation after each, measured their latency more than the
    // shape's throughput and let the choice vary from run to run).
    const int warm = 3, run = 8, runs = 3;
    int it = 0;
    auto launch_one = [&](int k) {
        for (SrvStream& r : probe.streams) r.pending_count = 1;
        build_items(&probe, pp->items, &pp->hdr, nullptr);
        // frame (it mod 8) of each replica's 8-frame scratch: consecutive
        // launches read different frames and write different slots
        for (int i = 0; i < pp->hdr.nitems; ++i)
            pp->items[i].a.frames =
                (const uint8_t*)probe.streams[i].pending + (it % 8) * probe.streams[i].ctx->frame_bytes;
        qldk::launch_batch(qldk::kBatchShapes[k], s->num_sms, pp->hdr.ntiles, *pp, s->gate_dev, st);
        for (SrvStream& r : probe.streams) r.ctx->pushed += 1;
        ++it;
    };
    for (int k = 0; rc == QLD_OK && k < qldk::kNumBatchShapes; ++k) {
        probe.shape = k;
        for (int w = 0; w < warm; ++w) launch_one(k);
        float us = 1e30f;
        for (int q = 0; q < runs && rc == QLD_OK; ++q) {
            cudaEventRecord(e0, st);
            for (int l = 0; l < run; ++l) launch_one(k);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = QLD_E_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms * 1e3f / run < us) us = ms * 1e3f / run;
        }
        if (rc == QLD_OK && us < best) {
            best = us;
            best_shape = k;
        }
    }
    for (SrvStream& r : rep) {
        cudaFree((void*)r.pending);
        release_stream(s, r);
    }
    delete pp;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != QLD_OK) {
        cudaGetLastError();
        return set_err(rc);
    }
    qldi::count_launches(qldk::kNumBatchShapes * (warm + run * runs));
    if (best_shape != s->shape) {
        s->shape = best_shape;
        s->graph_valid = false;
    }
    if (best_us) *best_us = best;
    return best_shape;
}

}  // extern "C"
