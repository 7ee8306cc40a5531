// qld_nn_tc.cuh -- the 3x3 convolution forward on the 5th-generation tensor
// cores (tcgen05): implicit GEMM with the accumulator in tensor memory.
//
// CTA tile: M = 128 output pixels x N output channels (N = 32, 64 or 128),
// K = 9 taps x Cin in steps of BK channels of one tap. Operands are staged in
// shared memory in the canonical K-major layout without swizzling: 8 x 16-byte
// "core matrices" (8 rows of 8 bf16), K-adjacent core matrices 128 bytes
// apart (leading byte offset), row-adjacent core-matrix groups BK*16 bytes
// apart (stride byte offset). One thread issues tcgen05.mma (M128 x N x K16,
// BF16 in, FP32 accumulate into TMEM) and commits to an mbarrier per buffer;
// the other threads gather the next K step meanwhile (two buffers). The
// epilogue reads the accumulator with tcgen05.ld (warp w: TMEM lanes
// 32w..32w+31 = pixels), adds the bias, applies ReLU and stores bf16/f32.
// Every wait is bounded: a wait that gives up records 1 in *status, the CTA
// skips its remaining MMAs, drains (bounded) and still frees its TMEM.

#pragma once

#include "qld_nn.cuh"

namespace qldnn {

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; no swizzle (bits 61-63 = 0)
    return d;
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase `parity` of `bar`; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Byte offset of element (row, k) in a K-major no-swizzle operand tile of
// BK columns: core matrix (row / 8, k / 8), row-in-core row % 8.
template <int BK>
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
    return (uint32_t)((row >> 3) * (BK * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int N, int BK>
struct TcSmem {
    __nv_bfloat16 a[2][128 * BK];
    __nv_bfloat16 b[2][N * BK];
    uint64_t bar[2];
    uint32_t tmem;
};

// out = act(conv3x3(in, w) + bias) with wk = weights K-major: wk[tap][co][ci].
template <int N, int BK>
__global__ void __launch_bounds__(128) conv3x3_fwd_tc_kernel(const __nv_bfloat16* __restrict__ in,
                                                             const __nv_bfloat16* __restrict__ wk,
                                                             const float* __restrict__ bias, int B, int H, int W,
                                                             int Cin, int Cout, int relu, __nv_bfloat16* out_bf,
                                                             float* out_f, int* status) {
    __shared__ __align__(1024) TcSmem<N, BK> sm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)B * H * W;
    const long long p0 = (long long)blockIdx.x * 128;
    const int co0 = blockIdx.y * N;
    const int csteps = Cin / BK;
    const int ksteps = 9 * csteps;
    constexpr uint32_t kIdesc = umma_idesc_bf16(128, N);
    constexpr long long kSpin = 1ll << 20;  // about a second of polling at most

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sm.tmem)),
                     "r"(N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;

    // this thread gathers pixel `tid` of the tile
    const long long pm = p0 + tid;
    int py = 0, px = 0;
    long long pb = 0;
    if (pm < P) {
        pb = pm / ((long long)H * W);
        const long long r = pm - pb * H * W;
        py = (int)(r / W);
        px = (int)(r - (long long)py * W);
    }

    bool failed = false;
    for (int ks = 0; ks < ksteps; ++ks) {
        const int buf = ks & 1;
        if (ks >= 2 && !failed) {  // the MMAs of step ks-2 read this buffer
            if (!mbar_wait_bounded(&sm.bar[buf], (uint32_t)(((ks >> 1) - 1) & 1), kSpin)) failed = true;
        }
        // a thread that gave up tells the others through the barrier below
        const int tap = ks / csteps, cc = ks - tap * csteps;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const int yy = py + dy, xx = px + dx;
        const bool ok = pm < P && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const __nv_bfloat16* src = ok ? in + (((pb * H + yy) * W + xx) * Cin + cc * BK) : in;
        unsigned char* abase = reinterpret_cast<unsigned char*>(sm.a[buf]);
#pragma unroll
        for (int c = 0; c < BK / 8; ++c) cp_async16(abase + kmajor_off<BK>(tid, c * 8), src + 8 * c, ok ? 16 : 0);
        unsigned char* bbase = reinterpret_cast<unsigned char*>(sm.b[buf]);
        for (int i = tid; i < N * (BK / 8); i += 128) {
            const int n = i / (BK / 8), c = i % (BK / 8);
            const __nv_bfloat16* ws = wk + (((long long)tap * Cout + co0 + n) * Cin + cc * BK + c * 8);
            cp_async16(bbase + kmajor_off<BK>(n, c * 8), ws, 16);
        }
        cp_async_commit();
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int any_failed = __syncthreads_or(failed ? 1 : 0);
        failed = any_failed != 0;
        if (tid == 0 && !failed) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sm.a[buf]), b0 = smem_u32(sm.b[buf]);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = umma_smem_desc(a0 + kk * 256, 128, BK * 16);
                const uint64_t bd = umma_smem_desc(b0 + kk * 256, 128, BK * 16);
                tc_mma(tmem, ad, bd, kIdesc, (ks > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&sm.bar[buf]);
        }
    }
    // the last step's commit covers every MMA issued before it
    const int last = ksteps - 1;
    bool done = !failed && mbar_wait_bounded(&sm.bar[last & 1], (uint32_t)((last >> 1) & 1), kSpin);
    if (!done) {
        if (tid == 0 && status) atomicExch(status, 1);
        // drain: give in-flight MMAs a bounded chance to finish before freeing
        mbar_wait_bounded(&sm.bar[last & 1], (uint32_t)((last >> 1) & 1), kSpin);
    }
    tc_fence_after();

    // tcgen05.ld is warp-collective: take the TMEM read-out only if every lane got through
    if (__all_sync(0xffffffffu, done)) {
        const long long p = p0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t r[16];
            tc_ld16(trow + (uint32_t)c0, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (p < P) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r[j]) + (bias ? bias[co0 + c0 + j] : 0.f);
                    if (relu) v[j] = fmaxf(v[j], 0.f);
                }
                if (out_bf) {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        pk[j] = *reinterpret_cast<const uint32_t*>(&h2);
                    }
                    uint4* o = reinterpret_cast<uint4*>(out_bf + p * Cout + co0 + c0);
                    o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
                if (out_f) {
                    float4* o = reinterpret_cast<float4*>(out_f + p * Cout + co0 + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(N));
    }
}

// B operands of the tensor-memory kernel from w[tap][ci][co]:
//   forward   (flip = 0): wk[tap][co][ci] = w[tap][ci][co]  (N = Cout, K = Cin)
//   data grad (flip = 1): wk[tap][ci][co] = w[8 - tap][ci][co] (N = Cin, K = Cout)
static __global__ void kmajor_weights_kernel(const __nv_bfloat16* __restrict__ w, int Cin, int Cout, int flip,
                                             __nv_bfloat16* __restrict__ wk) {
    const long long n = 9ll * Cin * Cout;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int tap = (int)(e / ((long long)Cin * Cout));
        const long long r = e - (long long)tap * Cin * Cout;
        const int ci = (int)(r / Cout), co = (int)(r % Cout);
        if (flip)
            wk[((long long)(8 - tap) * Cin + ci) * Cout + co] = w[e];
        else
            wk[((long long)tap * Cout + co) * Cin + ci] = w[e];
    }
}

}  // namespace qldnn

namespace qldnn {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// 16-byte global -> shared copy cached in L1 as well: the nine taps of a tile
// read overlapping rows of the input.
__device__ __forceinline__ void cp_async16_ca(void* smem, const void* gmem, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes));
}

template <int N, int BK, int STAGES>
struct TcPipe {
    static constexpr int kA = 128 * BK * 2;  // bytes of one A tile
    static constexpr int kB = N * BK * 2;    // bytes of one B tile
    static constexpr int kStage = kA + kB;
    static constexpr int kBars = (2 * STAGES + 1) * 8;
    static constexpr int kSmem = STAGES * kStage + kBars + 16;
};

// Warp-specialised version of conv3x3_fwd_tc_kernel. 160 threads: warps 0-3
// gather the K steps into a STAGES-deep ring (each thread: one pixel row of A
// and a share of B) and, LAG steps later, once their copies have landed,
// fence them for the tensor-core (async) proxy and arrive on the step's
// "full" barrier; warp 4 waits on "full", issues the step's BK/16 MMAs
// (M128 x N x K16, whole Cout per tile: N = Cout <= 256) and commits to the
// step's "empty" barrier, which releases the buffer to the producers; a last
// commit to "done" releases the epilogue (warps 0-3, TMEM lanes 32w..32w+31).
// Bounded waits everywhere: a role that gives up sets *status and goes on, so
// every role terminates and TMEM is always freed.
template <int N, int BK, int STAGES>
__global__ void __launch_bounds__(160) conv3x3_fwd_tc2_kernel(const __nv_bfloat16* __restrict__ in,
                                                              const __nv_bfloat16* __restrict__ wk,
                                                              const float* __restrict__ bias, int B, int H, int W,
                                                              int Cin, int Cout, int relu, __nv_bfloat16* out_bf,
                                                              float* out_f, int* status) {
    using L = TcPipe<N, BK, STAGES>;
    constexpr int LAG = STAGES - 2;
    static_assert(LAG >= 1, "need at least three stages");
    extern __shared__ __align__(1024) unsigned char dsm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(dsm + STAGES * L::kStage);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)B * H * W;
    const long long p0 = (long long)blockIdx.x * 128;
    const int csteps = Cin / BK;
    const int ksteps = 9 * csteps;
    constexpr uint32_t kIdesc = umma_idesc_bf16(128, N);
    constexpr long long kSpin = 1ll << 20;

    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int b = 0; b < STAGES; ++b) {
            mbar_init(&full[b], 128);
            mbar_init(&empty[b], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok_all = true;

    if (warp < 4) {
        // ---------------------------------------------------------- producers
        const long long pm = p0 + tid;
        int py = 0, px = 0;
        long long pb = 0;
        if (pm < P) {
            pb = pm / ((long long)H * W);
            const long long r = pm - pb * H * W;
            py = (int)(r / W);
            px = (int)(r - (long long)py * W);
        }
        for (int ks = 0; ks < ksteps; ++ks) {
            const int b = ks % STAGES;
            if (ks >= STAGES && !mbar_wait_bounded(&empty[b], (uint32_t)(((ks / STAGES) - 1) & 1), kSpin))
                ok_all = false;
            const int tap = ks / csteps, cc = ks - tap * csteps;
            const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
            const bool ok = pm < P && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const __nv_bfloat16* src = ok ? in + (((pb * H + yy) * W + xx) * Cin + cc * BK) : in;
            unsigned char* abase = dsm + b * L::kStage;
            unsigned char* bbase = abase + L::kA;
#pragma unroll
            for (int c = 0; c < BK / 8; ++c) cp_async16_ca(abase + kmajor_off<BK>(tid, c * 8), src + 8 * c, ok ? 16 : 0);
            for (int i = tid; i < N * (BK / 8); i += 128) {
                const int n = i / (BK / 8), c = i % (BK / 8);
                cp_async16(bbase + kmajor_off<BK>(n, c * 8),
                           wk + (((long long)tap * Cout + n) * Cin + cc * BK + c * 8), 16);
            }
            cp_async_commit();
            if (ks >= LAG) {
                cp_async_wait<LAG>();
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(&full[(ks - LAG) % STAGES]);
            }
        }
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        for (int k = ksteps - LAG < 0 ? 0 : ksteps - LAG; k < ksteps; ++k) mbar_arrive(&full[k % STAGES]);
    } else if (lane == 0) {
        // ------------------------------------------------------- MMA issuer
        for (int ks = 0; ks < ksteps; ++ks) {
            const int b = ks % STAGES;
            const bool ready = mbar_wait_bounded(&full[b], (uint32_t)((ks / STAGES) & 1), kSpin);
            if (!ready) ok_all = false;
            tc_fence_after();
            if (ready) {
                const uint32_t a0 = smem_u32(dsm + b * L::kStage), b0 = a0 + L::kA;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    tc_mma(tmem, umma_smem_desc(a0 + kk * 256, 128, BK * 16), umma_smem_desc(b0 + kk * 256, 128, BK * 16),
                           kIdesc, (ks > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&empty[b]);
        }
        tc_commit(done);
    }

    if (warp < 4) {
        // --------------------------------------------------------- epilogue
        const bool fin = mbar_wait_bounded(done, 0, kSpin);
        if (!fin) {
            ok_all = false;
            mbar_wait_bounded(done, 0, kSpin);  // bounded drain before TMEM is freed
        }
        tc_fence_after();
        // tcgen05.ld is warp-collective: take the read-out only if every lane got through
        if (__all_sync(0xffffffffu, ok_all)) {
            const long long p = p0 + warp * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t r[16];
                tc_ld16(trow + (uint32_t)c0, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (p < P) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v[j] = __uint_as_float(r[j]) + (bias ? bias[c0 + j] : 0.f);
                        if (relu) v[j] = fmaxf(v[j], 0.f);
                    }
                    if (out_bf) {
                        uint32_t pk[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            pk[j] = *reinterpret_cast<const uint32_t*>(&h2);
                        }
                        uint4* o = reinterpret_cast<uint4*>(out_bf + p * Cout + c0);
                        o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    }
                    if (out_f) {
                        float4* o = reinterpret_cast<float4*>(out_f + p * Cout + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    }
                }
            }
        }
    }
    if (!ok_all && status) atomicExch(status, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(N));
    }
}

}  // namespace qldnn
