// qld_nn_tma.cuh -- persistent, TMA-fed 3x3 convolution forward on the
// 5th-generation tensor cores.
//
// Output tile: 8 rows x 16 columns of one image = M 128 pixels, N = Cout /
// nsplit output channels (32, 64, 128 or 256): when a layer has fewer tiles
// than SMs, nsplit CTAs share each tile, CTA b taking channel slice
// b mod nsplit for all its tiles (gridDim.x is a multiple of nsplit). K runs
// over channel chunks of BK = SWB/2 channels (outer) and the nine taps (inner).
//
// Input staging without im2col: for each channel chunk the tile's input halo
// (10 rows x 16 columns) is loaded three times by the tensor-memory
// accelerator, shifted by one column each (x0-1, x0, x0+1). TMA fills the
// out-of-image borders with zeros, which is exactly the convolution's zero
// padding. In the halo copy for column shift kx, output pixel (y, x) of the
// tile sits in row (y + ky) * 16 + x for tap row ky, so the A operand of tap
// (ky, kx) is that copy starting ky * 16 rows in: a plain offset of the
// matrix descriptor. The nine taps thus read 3 x 160 staged pixel rows instead
// of 9 x 128 gathered ones. Weights (K-major, wk[tap][co][ci]) come in one
// TMA box of N rows x BK channels per tap.
//
// Shared memory: both operands use the swizzled K-major layout TMA writes
// when a box row is exactly the swizzle span (SWB = 128, 64 or 32 bytes):
// 8-row atoms of 8 * SWB bytes. A K16 step inside a row moves the descriptor
// start 32 bytes.
//
// Roles (kConvThreads = 192 threads, persistent over tiles; one CTA per SM,
// or two for some narrow layers):
//   warp 0  one thread issues the TMA loads into a 2-stage halo ring and an
//           SB-stage weight ring of one tap row (three taps) per stage when
//           two such stages fit (mbarrier expect_tx / complete_tx);
//   warp 1  allocates TMEM (two accumulators of N columns), one thread issues
//           tcgen05.mma M128 x N x K16 and commits to the rings' "empty"
//           barriers and, per tile, to the accumulator's "full" barrier;
//   warps 2-5 epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//           lanes 32 (w mod 4) ..), bias, ReLU, bf16/f32 stores and fused
//           outputs, then release the accumulator, so the next tile's MMAs
//           overlap the read-out.
// The weights-resident variant (conv3x3_fwd_tma_wres_kernel) has the same
// roles, loads all the weights once per CTA, and can stack tiles in height
// (SUB) or the three column taps in N (XS).
// Launched early (programmatic stream serialisation), a CTA allocates TMEM,
// sets up its barriers and (weights-resident variant) loads the weights
// while the previous kernel finishes; the producer waits for that kernel
// (griddepcontrol.wait) before the first input load, and every global write
// comes after. Every wait is bounded (about a second of wall time) and also
// gives up once another role has flagged a failure; the producer then waits
// (bounded) for its copies in flight, the MMA thread for its MMAs, and TMEM
// is freed. A failure records 1 in *status.

#pragma once

#include <cuda.h>

#include "qld_nn_tc.cuh"

namespace qldnn {

// Matrix descriptor of a K-major operand in a swizzled layout: rows of SWB
// bytes, 8-row atoms SBO = 8 * SWB bytes apart (leading offset unused).
template <int SWB>
__device__ __forceinline__ uint64_t umma_desc_sw(uint32_t saddr) {
    constexpr uint64_t layout = SWB == 128 ? 2 : (SWB == 64 ? 4 : 6);
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(((8 * SWB) >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

// The descriptor of the same layout at byte offset `off` (a multiple of 16)
// past the one given: the start address is the low 14-bit field in 16-byte
// units, and shared addresses stay below 2^18 bytes, so the field never
// carries into the next one. With `off` a compile-time constant this is one
// 64-bit add per MMA instead of building the descriptor again.
__device__ __forceinline__ uint64_t desc_at(uint64_t desc, uint32_t off) {
    return desc + (uint64_t)(off >> 4);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the kernel before it on the stream is still
// running. pdl_wait returns once that kernel has completed and its writes are
// visible (at once when there is no such dependency); pdl_trigger lets the
// next such kernel launch as soon as every CTA of this one has issued it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` for at most `limit_ns` of wall time (one
// second unless given); with `fail` non-null, also give up as soon as another
// role has set *fail (and set it on a time-out).
__device__ __forceinline__ bool wait_timed(uint64_t* bar, uint32_t parity, volatile int* fail,
                                           uint64_t limit_ns = 1000000000ull) {
    // a phase that has already completed costs one probe: the timer is read
    // (a slow special register, hundreds of cycles on the MMA thread's path)
    // only when the wait is real
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (fail && *fail) return false;
            if (global_ns() - t0 > limit_ns) break;
        }
    }
    if (fail) *fail = 1;
    return false;
}

// Self-test of the failure path of the bounded waits (no fault, no hang):
// lane 0 of warp 0 waits on an mbarrier nothing arrives on, with a short
// limit, and so times out and raises the shared failure flag; lane 0 of warp 1
// waits on another such barrier with a one-minute limit and must leave as soon
// as it sees the flag. out[0] = 1 if the first wait timed out, out[1] = 1 if
// the second gave up because of the flag, out[2] = device nanoseconds the
// kernel took.
__global__ void __launch_bounds__(64) wait_selftest_kernel(uint64_t limit_ns, long long* out) {
    __shared__ uint64_t bars[2];
    __shared__ int fail;
    const uint64_t t0 = global_ns();
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    __syncthreads();
    volatile int* f = &fail;
    bool r0 = true, r1 = true;
    if (threadIdx.x == 0) r0 = wait_timed(&bars[0], 0, f, limit_ns);
    if (threadIdx.x == 32) r1 = wait_timed(&bars[1], 0, f, 60000000000ull);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = r0 ? 0 : 1;
        out[2] = (long long)(global_ns() - t0);
    }
    if (threadIdx.x == 32) out[1] = (!r1 && *f) ? 1 : 0;
}

__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, volatile int* fail) {
    return wait_timed(bar, parity, fail);
}

// Outputs of a persistent TMA convolution's epilogue. Every pointer may be
// null. bf16 outputs are rows of `ld*` channels (>= Cout, a multiple of 8)
// whose first Cout hold this layer: a layer can write straight into a slice
// of a wider (concatenated) tensor.
//   out   [B][H][W] x ldo, the activation (bf16)
//   out_f [B][H][W][Cout] f32 (data gradients)
//   pool  [B][H/2][W/2] x ldp, 2x2 average of the bf16 activations (H, W even)
//   up    [B][2H][2W] x ldu, nearest 2x upsampling of the bf16 activations
//   head  pred[p] = head_b + sum_c act_bf16[p][c] head_w[c] + base[p] (f32; all
//         Cout channels in one CTA), the network's 1x1 output layer
// The pooled and head values use the same operation order as the standalone
// pooling / head / add kernels, so results are bit-identical to running them.
struct ConvEpi {
    __nv_bfloat16* out;
    long long ldo;
    float* out_f;
    __nv_bfloat16* pool;
    long long ldp;
    __nv_bfloat16* up;
    long long ldu;
    const float* head_w;
    const float* head_b;
    const float* base;
    float* pred;
};

// 16 bf16 channels (32 bytes) of one pixel: one 256-bit store when the
// address is 32-byte aligned (v8), else two 16-byte stores. The epilogue's
// lanes are pixels, so a warp's store covers 32 rows of the output tensor:
// the wide store halves the store instructions the memory pipeline takes
// (measured alone: 8 x 64^2, 256 -> 128 22.0 -> 21.0 us; 128 -> 128
// 15.4 -> 14.5 us).
__device__ __forceinline__ void store_row32(__nv_bfloat16* o, const uint32_t* pk, bool v8) {
    if (v8) {
        asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(o), "r"(pk[0]), "r"(pk[1]),
                     "r"(pk[2]), "r"(pk[3]), "r"(pk[4]), "r"(pk[5]), "r"(pk[6]), "r"(pk[7])
                     : "memory");
    } else {
        uint4* o4 = reinterpret_cast<uint4*>(o);
        o4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
}

// Ties 16 registers written by tcgen05.ld to the point after the
// tcgen05.wait::ld before it: the empty statement "redefines" them, so no use
// can be scheduled above the wait.
__device__ __forceinline__ void tc_tie16(uint32_t* r) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]));
}

// Epilogue warps of the persistent TMA convolutions (warps 2-5; warp w may
// read TMEM lanes 32 (w mod 4) .. only). Per tile: wait for its accumulator,
// add the bias, apply ReLU, write the outputs `epi` asks for, release the
// accumulator. Pixel m = 32 (w mod 4) + lane of the tile is (y, x) =
// (m / 16, m mod 16), so a warp holds two whole rows and the 2x2 pooling
// partners of lane l are the lanes l ^ 1, l ^ 16 and l ^ 17. The four lanes
// of a 2x2 block share its pooling: lane role r = (x & 1) + 2 (y & 1) takes
// channel pairs 2r and 2r + 1 of each 16-channel chunk, receiving them from
// its partners as packed bf16 pairs, and sums the block's diagonals first,
// (own + l^17) + (l^1 + l^16), which is the same value in every lane's
// order (the standalone pooling kernels sum the same way). The
// accumulator is read in groups of up to 64 columns (all loads of a group
// issued before one wait); with N <= 64 the bias stays in registers for all
// tiles. A tile is SUB sub-tiles of 8 x 16 pixels stacked in rows, sub-tile h
// in accumulator columns (acc SUB + h) N. The epilogue warps share the SM
// sub-partitions' issue slots with the producer and the MMA-issuing thread,
// whose pace sets the narrow layers' speed, so the read-out is kept to as few
// instructions (and warps) as possible: more epilogue warps measured slower.
constexpr int kEpiWarps = 4;
constexpr int kConvThreads = 64 + 32 * kEpiWarps;

//
// XS (column taps stacked in N, conv3x3_fwd_tma_wres_kernel<..., XS = true>):
// the accumulator of a sub-tile holds 3 N columns, D_kx[m][co] at column
// kx N + co, for the 16 halo columns x0 - 1 .. x0 + 14 of an output tile 14
// columns wide; the output at column x0 + c takes D_0 of halo column c (its
// own lane), D_1 of column c + 1 and D_2 of column c + 2, summed in that order
// ((D_0 + D_1) + D_2) after two shuffles down within the 16-lane row. Lanes
// of halo columns 14 and 15 produce no output (and each other's pooling
// partners, so the pooling exchange stays inside whole 2 x 2 blocks).
//
// EW = 8 (wide layers without a head): two warps per TMEM lane quarter, warp
// w taking accumulator columns [h N/2, (h + 1) N/2) with h = (w - 2) / 4.
template <int N, int SUB = 1, bool BIAS_REG = (N <= 64), bool XS = false, int EW = kEpiWarps>
__device__ __forceinline__ void conv_epilogue(uint32_t tmem, uint64_t* tfull, uint64_t* tempty, volatile int* fail,
                                              int warp, int lane, int ntiles, int tiles_x, int tiles_y, int H, int W,
                                              int Cout, const float* __restrict__ bias, int relu, ConvEpi epi,
                                              int nsplit) {
    constexpr int TW = XS ? 14 : 16;   // output columns per tile
    constexpr int NA = XS ? 3 * N : N; // accumulator columns per sub-tile
    const bool head = epi.head_w != nullptr;
    const int qw = warp & 3;           // TMEM lane quarter this warp may read
    const int m = qw * 32 + lane;
    const int my = m >> 4, mx = m & 15;
    const int co0 = (blockIdx.x % nsplit) * N;  // this CTA's slice of the output channels
    if (bias) bias += co0;
    if (epi.out) epi.out += co0;
    if (epi.out_f) epi.out_f += co0;
    if (epi.pool) epi.pool += co0;
    if (epi.up) epi.up += co0;
    const int role = (lane & 1) | ((lane >> 3) & 2);  // 2x2 block position: x & 1, y & 1
    // pk index of channel pair k (0, 1) of the lane with role r ^ rd, for the
    // lane that sends it to this one across offset rd (1: x, 2: y, 3: both)
    auto pick = [&](const uint32_t* pk, int rd, int k) {
        const int rr = role ^ rd;
        const uint32_t a = rr & 1 ? pk[2 + k] : pk[k];
        const uint32_t b = rr & 1 ? pk[6 + k] : pk[4 + k];
        return rr & 2 ? b : a;
    };
    // accumulator columns per tcgen05.wait::ld (XS: 16 output channels = 48 columns)
    static_assert(EW == 4 || (EW == 8 && !XS && !BIAS_REG && N >= 64), "eight epilogue warps: wide layers only");
    constexpr int NW = N * 4 / EW;                     // accumulator columns this warp reads
    const int cb = EW == 8 ? ((warp - 2) >> 2) * NW : 0;  // the first of them
    constexpr int G = XS ? 16 : (NW < 64 ? NW : 64);
    float bres[BIAS_REG ? N : 1];       // the bias (or 0), for narrow layers
    // wide layers read the bias per 16-channel chunk as four 16-byte
    // read-only loads, issued together, where one scalar load per channel
    // could be ordered behind the output stores (cycle stamps in the
    // epilogue of 8 x 64^2, 256 -> 128 showed 3,000-3,600 cycles per
    // 64-channel group; with this and the 32-byte stores of store_row32 the
    // layer went from 22.4 to 21.2 us and 128 -> 128 from 15.7 to 14.8 us,
    // graph-timed, interleaved against the previous build)
    const bool bias_v4 = bias && (reinterpret_cast<uintptr_t>(bias) & 15u) == 0;
    // 32-byte stores where every pixel row's 16-channel chunks are 32-byte aligned
    const bool out_v8 = (reinterpret_cast<uintptr_t>(epi.out) & 31u) == 0 && (epi.ldo & 15) == 0;
    const bool up_v8 = (reinterpret_cast<uintptr_t>(epi.up) & 31u) == 0 && (epi.ldu & 15) == 0;
    if constexpr (BIAS_REG) {
#pragma unroll
        for (int j = 0; j < N; ++j) bres[j] = bias ? bias[j] : 0.f;
    }
    int it = 0;
    for (int t = blockIdx.x / nsplit; t < ntiles; t += gridDim.x / nsplit) {
        const int acc = it & 1;
        const bool got = wait_or_fail(&tfull[acc], (uint32_t)((it >> 1) & 1), fail);
        if (!__all_sync(0xffffffffu, got)) break;  // tcgen05.ld below is warp-collective
        tc_fence_after();
        const int tx = t % tiles_x, r = t / tiles_x, ty = r % tiles_y, b = r / tiles_y;
#pragma unroll 1
        for (int h = 0; h < SUB; ++h) {  // the tile's 8-row sub-tiles
            const int y = (ty * SUB + h) * 8 + my, x = tx * TW + mx;
            const bool inside = y < H && x < W && (!XS || mx < TW);
            const long long p = ((long long)b * H + y) * W + x;
            const uint32_t taddr = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)((acc * SUB + h) * NA);
            float hacc = head ? *epi.head_b : 0.f;
            // unrolled when XS, so the register-resident bias is indexed
            // with constants
#pragma unroll(XS ? 4 : 1)
            for (int g0 = cb; g0 < cb + NW; g0 += G) {
                uint32_t rg[G];
                if constexpr (XS) {
                    uint32_t r1[16], r2[16];
                    tc_ld16(taddr + (uint32_t)g0, rg);
                    tc_ld16(taddr + (uint32_t)(N + g0), r1);
                    tc_ld16(taddr + (uint32_t)(2 * N + g0), r2);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    tc_tie16(rg);
                    tc_tie16(r1);
                    tc_tie16(r2);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {  // every lane shuffles: warp-uniform
                        const float d1 = __shfl_down_sync(0xffffffffu, __uint_as_float(r1[j]), 1, 16);
                        const float d2 = __shfl_down_sync(0xffffffffu, __uint_as_float(r2[j]), 2, 16);
                        rg[j] = __float_as_uint((__uint_as_float(rg[j]) + d1) + d2);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < G; c += 16) tc_ld16(taddr + (uint32_t)(g0 + c), rg + c);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                    for (int c = 0; c < G; c += 16) tc_tie16(rg + c);
                }
#pragma unroll
                for (int c = 0; c < G; c += 16) {
                    const int c0 = g0 + c;
                    const uint32_t* rr = rg + c;
                    float v[16];
                    float bl[16];  // wide layers: this chunk's bias, read-only loads issued together
                    if constexpr (!BIAS_REG) {
                        if (bias_v4) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + c0) + j);
                                bl[4 * j] = b4.x;
                                bl[4 * j + 1] = b4.y;
                                bl[4 * j + 2] = b4.z;
                                bl[4 * j + 3] = b4.w;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; ++j) bl[j] = bias ? __ldg(bias + c0 + j) : 0.f;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float bj;
                        if constexpr (BIAS_REG) bj = bres[g0 + c + j];
                        else bj = bl[j];
                        v[j] = __uint_as_float(rr[j]) + bj;
                        if (relu) v[j] = fmaxf(v[j], 0.f);
                    }
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        pk[j] = *reinterpret_cast<const uint32_t*>(&h2);
                    }
                    if (epi.out && inside) store_row32(epi.out + p * epi.ldo + c0, pk, out_v8);
                    if (epi.out_f && inside) {
                        float4* o = reinterpret_cast<float4*>(epi.out_f + p * Cout + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    }
                    if (epi.up && inside) {
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            const long long q = ((long long)b * 2 * H + 2 * y + (d >> 1)) * (2ll * W) + 2 * x + (d & 1);
                            store_row32(epi.up + q * epi.ldu + c0, pk, up_v8);
                        }
                    }
                    if (epi.pool) {  // warp-uniform: every lane shuffles
                        uint32_t own[2], v1[2], v16[2], v17[2];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            own[k] = pick(pk, 0, k);
                            v1[k] = __shfl_xor_sync(0xffffffffu, pick(pk, 1, k), 1);
                            v16[k] = __shfl_xor_sync(0xffffffffu, pick(pk, 2, k), 16);
                            v17[k] = __shfl_xor_sync(0xffffffffu, pick(pk, 3, k), 17);
                        }
                        if (inside) {
                            uint32_t o2[2];
#pragma unroll
                            for (int k = 0; k < 2; ++k) {
                                const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&own[k]));
                                const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v1[k]));
                                const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v16[k]));
                                const float2 f3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v17[k]));
                                const float lo = 0.25f * ((f0.x + f3.x) + (f1.x + f2.x));
                                const float hi = 0.25f * ((f0.y + f3.y) + (f1.y + f2.y));
                                const __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
                                o2[k] = *reinterpret_cast<const uint32_t*>(&h2);
                            }
                            const long long pp = ((long long)b * (H / 2) + y / 2) * (W / 2) + x / 2;
                            *reinterpret_cast<uint2*>(epi.pool + pp * epi.ldp + c0 + 4 * role) = make_uint2(o2[0], o2[1]);
                        }
                    }
                    if (head) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {  // the stored (bf16) values, in channel order
                            const float2 t2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk[j]));
                            hacc = fmaf(t2.x, epi.head_w[c0 + 2 * j], hacc);
                            hacc = fmaf(t2.y, epi.head_w[c0 + 2 * j + 1], hacc);
                        }
                    }
                }
            }
            if (head && inside) epi.pred[p] = hacc + epi.base[p];
        }
        tc_fence_before();
        mbar_arrive(&tempty[acc]);
        ++it;
    }
}

template <int N, int SWB>
struct TmaConv {
    static constexpr int BK = SWB / 2;                      // channels per chunk
    static constexpr int HALO = 10 * 16 * SWB;              // one column-shifted halo copy
    static constexpr int SA = 2;                            // halo stages
    static constexpr int kA = SA * 3 * HALO;
    static constexpr int kFree = 232448 - 1024 - kA - 64 * 8 - 16;
    // weight stages of one tap row (three taps: one barrier round trip and
    // one commit per three taps) when two such stages fit beside the halo
    // ring, else of one tap
    static constexpr int TPS = kFree / (3 * N * SWB) >= 2 ? 3 : 1;
    static constexpr int BSTAGE = TPS * N * SWB;
    // weight stages: as many as fit beside the halo ring in 227 KB (at most 12)
    static constexpr int SB = kFree / BSTAGE > 12 ? 12 : kFree / BSTAGE;
    static_assert(SB >= 2, "weight ring too small");
    static constexpr int kB = SB * BSTAGE;
    static constexpr int kBars = (2 * SA + 2 * SB + 5) * 8;
    static constexpr int kSmem = 1024 + kA + kB + kBars + 16;  // 1024: slack to align the base
    static constexpr int kTmemCols = 2 * N;
};

template <int N, int SWB, int EW = kEpiWarps>
__global__ void __launch_bounds__(64 + 32 * EW, 1)
    conv3x3_fwd_tma_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_w,
                           const float* __restrict__ bias, int B, int H, int W, int Cin, int Cout, int relu,
                           const ConvEpi epi, int* status, int nsplit) {
    using L = TmaConv<N, SWB>;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char* dsm = dsm_raw + ((1024u - (smem_u32(dsm_raw) & 1023u)) & 1023u);
    unsigned char* sA = dsm;
    unsigned char* sB = dsm + L::kA;
    uint64_t* fullA = reinterpret_cast<uint64_t*>(sB + L::kB);
    uint64_t* emptyA = fullA + L::SA;
    uint64_t* fullB = emptyA + L::SA;
    uint64_t* emptyB = fullB + L::SB;
    uint64_t* tfull = emptyB + L::SB;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* fail = reinterpret_cast<volatile int*>(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (W + 15) >> 4, tiles_y = (H + 7) >> 3;
    const int ntiles = B * tiles_x * tiles_y;
    const int csteps = Cin / L::BK;
    const int co0 = (blockIdx.x % nsplit) * N;  // this CTA's slice of the output channels
    constexpr uint32_t kIdesc = umma_idesc_bf16(128, N);

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(L::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < L::SA; ++s) {
            mbar_init(&fullA[s], 1);
            mbar_init(&emptyA[s], 1);
        }
        for (int s = 0; s < L::SB; ++s) {
            mbar_init(&fullB[s], 1);
            mbar_init(&emptyB[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 32 * EW);
        }
        mbar_init(drain, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_in)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_w)) : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_trigger();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ TMA producer
            pdl_wait();  // the input (and the output's previous readers) are done
            int ia = 0, ib = 0;
            bool ok = true;
            for (int t = blockIdx.x / nsplit; t < ntiles && ok; t += gridDim.x / nsplit) {
                const int tx = t % tiles_x, r = t / tiles_x, ty = r % tiles_y, b = r / tiles_y;
                const int x0 = tx * 16, y0 = ty * 8;
                for (int cc = 0; cc < csteps && ok; ++cc) {
                    const int sa = ia % L::SA;
                    if (ia >= L::SA && !(ok = wait_or_fail(&emptyA[sa], (uint32_t)(((ia / L::SA) - 1) & 1), fail)))
                        break;
                    mbar_expect_tx(&fullA[sa], 3 * L::HALO);
                    for (int j = 0; j < 3; ++j)
                        tma_load_4d(sA + (sa * 3 + j) * L::HALO, &map_in, &fullA[sa], cc * L::BK, x0 + j - 1, y0 - 1, b);
                    ++ia;
                    for (int g = 0; g < 9 / L::TPS; ++g) {
                        const int sb = ib % L::SB;
                        if (ib >= L::SB && !(ok = wait_or_fail(&emptyB[sb], (uint32_t)(((ib / L::SB) - 1) & 1), fail)))
                            break;
                        mbar_expect_tx(&fullB[sb], L::BSTAGE);
                        for (int tt = 0; tt < L::TPS; ++tt)
                            tma_load_2d(sB + sb * L::BSTAGE + tt * N * SWB, &map_w, &fullB[sb], cc * L::BK,
                                        (g * L::TPS + tt) * Cout + co0);
                        ++ib;
                    }
                }
            }
            // no copy may still be in flight when the CTA leaves: wait for the
            // last load issued into each stage (the earlier ones completed
            // before it could be issued)
            for (int s = 0; s < L::SA; ++s) {
                const int k = ia - 1 - ((ia - 1 - s) % L::SA + L::SA) % L::SA;
                if (k >= 0) wait_timed(&fullA[s], (uint32_t)((k / L::SA) & 1), nullptr);
            }
            for (int s = 0; s < L::SB; ++s) {
                const int k = ib - 1 - ((ib - 1 - s) % L::SB + L::SB) % L::SB;
                if (k >= 0) wait_timed(&fullB[s], (uint32_t)((k / L::SB) & 1), nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // --------------------------------------------------------- MMA issuer
            // As in the weights-resident kernel: counted stages and offset
            // descriptors; one weight barrier per stage of TPS taps.
            const uint64_t adesc0 = umma_desc_sw<SWB>(smem_u32(sA));
            const uint64_t bdesc0 = umma_desc_sw<SWB>(smem_u32(sB));
            int sa = 0, sb = 0, it = 0;
            uint32_t pa = 0, pb = 0;
            bool ok = true;
            for (int t = blockIdx.x / nsplit; t < ntiles && ok; t += gridDim.x / nsplit) {
                const int acc = it & 1;
                if (it >= 2 && !(ok = wait_or_fail(&tempty[acc], (((uint32_t)it >> 1) & 1u) ^ 1u, fail))) break;
                const uint32_t d = tmem + (uint32_t)(acc * N);
                for (int cc = 0; cc < csteps && ok; ++cc) {
                    if (!(ok = wait_or_fail(&fullA[sa], pa, fail))) break;
                    const uint64_t adesc = desc_at(adesc0, (uint32_t)(sa * 3 * L::HALO));
#pragma unroll
                    for (int g = 0; g < 9 / L::TPS; ++g) {
                        if (!(ok = wait_or_fail(&fullB[sb], pb, fail))) break;
                        tc_fence_after();
                        const uint64_t bdesc = desc_at(bdesc0, (uint32_t)(sb * L::BSTAGE));
#pragma unroll
                        for (int tt = 0; tt < L::TPS; ++tt) {
                            const int tap = g * L::TPS + tt;
#pragma unroll
                            for (int kk = 0; kk < L::BK / 16; ++kk)
                                tc_mma(d, desc_at(adesc, (tap % 3) * L::HALO + (tap / 3) * 16 * SWB + kk * 32),
                                       desc_at(bdesc, tt * N * SWB + kk * 32), kIdesc, (cc | tap | kk) ? 1u : 0u);
                        }
                        tc_commit(&emptyB[sb]);
                        if (++sb == L::SB) {
                            sb = 0;
                            pb ^= 1u;
                        }
                    }
                    if (!ok) break;
                    tc_commit(&emptyA[sa]);
                    if (++sa == L::SA) {
                        sa = 0;
                        pa ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(&tfull[acc]);
                ++it;
            }
            // every MMA issued has completed before TMEM can be freed
            tc_commit(drain);
            wait_timed(drain, 0, nullptr);
        }
    } else {
        conv_epilogue<N, 1, (EW == 8 ? false : N <= 64), false, EW>(tmem, tfull, tempty, fail, warp, lane, ntiles,
                                                                     tiles_x, tiles_y, H, W, Cout, bias, relu, epi,
                         nsplit);
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *fail && status) atomicExch(status, 1);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::kTmemCols));
    }
}


// ---------------------------------------------------------------------------
// Weights-resident version for layers whose weights (9 Cin Cout bf16) fit in
// shared memory beside at least two halo stages: the producer loads them once
// per persistent CTA (9 csteps TMA boxes on one barrier) and then streams only
// the halos through an SA-stage ring (SA chosen at launch, at most kMaxSA), so
// neither the L2 nor the ring depth is spent on weights tile after tile.
// Same tiles, operand layouts, MMAs, epilogue and failure handling as
// conv3x3_fwd_tma_kernel. SUB = 2: each tile is two 8 x 16 sub-tiles stacked
// in rows (16 x 16 pixels) that share one 18-row halo load per channel chunk,
// one barrier round trip and the weights of each MMA step, accumulating into
// two accumulators of N columns; the per-tile pipeline costs, which dominate
// narrow (N = 32, 64) layers, are paid once per 256 pixels. With the same
// channel chunks (SWB) the MMAs of each accumulator, and so the results, are
// those of SUB = 1.
//
// XS = true stacks the three column taps kx of a tap row in the MMA's N
// dimension: one MMA M128 x 3N x K16 per tap row ky, sub-tile and K16 step,
// B = the three taps' weight boxes, which lie one after another in shared
// memory (tap 3 ky + kx at box 9 cc + 3 ky + kx), read as one 3N-row operand.
// The halo is loaded once, unshifted, 16 columns from x0 - 1, and a tile
// covers 14 output columns; the epilogue adds the three column groups
// (conv_epilogue). Narrow layers gain because an M128 x N32 x K16 MMA takes
// about as long as an M128 x N96 one.
template <int N, int SWB, int SUB = 1, bool XS = false>
struct TmaConvRes {
    static constexpr int BK = SWB / 2;
    static constexpr int HALO = (8 * SUB + 2) * 16 * SWB;  // one (column-shifted) halo copy of a tile
    static constexpr int ASTAGE = (XS ? 1 : 3) * HALO;
    static constexpr int BSTAGE = N * SWB;
    static constexpr int kMaxSA = 8;
    static constexpr int kBars = (2 * kMaxSA + 6) * 8;
    static constexpr int NA = (XS ? 3 : 1) * N;             // accumulator columns per sub-tile
    static constexpr int TW = XS ? 14 : 16;                 // output columns per tile
    // two accumulators; an allocation is a power of two of at least 32 columns
    static constexpr int kTmemCols = 2 * NA * SUB <= 32    ? 32
                                     : 2 * NA * SUB <= 64  ? 64
                                     : 2 * NA * SUB <= 128 ? 128
                                     : 2 * NA * SUB <= 256 ? 256
                                                           : 512;
    static_assert(2 * NA * SUB <= 512, "accumulators exceed the tensor memory");
    // dynamic shared memory for SA halo stages and Cin input channels
    static constexpr long long smem(int SA, int Cin) {
        return 1024 + (long long)SA * ASTAGE + 9ll * (Cin / BK) * BSTAGE + kBars + 16;
    }
};

// MINB = 2: two CTAs per SM (each within kTwoPerSmSmem of shared memory):
// every MMA-issuing thread feeds a tensor-core queue about one MMA deep and
// pauses for its barriers and commits; with two CTAs on an SM the other
// CTA's MMAs fill those pauses (the narrow layers' MMAs take ~45 cycles, a
// barrier probe ~100), and an early-launched next layer can start on an SM
// while this one's second CTA still runs.
constexpr int kTwoPerSmSmem = 115712;

template <int N, int SWB, int SUB = 1, int MINB = 1, bool XS = false>
__global__ void __launch_bounds__(kConvThreads, MINB)
    conv3x3_fwd_tma_wres_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_w,
                                const float* __restrict__ bias, int B, int H, int W, int Cin, int Cout, int relu,
                                const ConvEpi epi, int* status, int SA, int nsplit) {
    using L = TmaConvRes<N, SWB, SUB, XS>;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char* dsm = dsm_raw + ((1024u - (smem_u32(dsm_raw) & 1023u)) & 1023u);
    const int csteps = Cin / L::BK;
    unsigned char* sA = dsm;
    unsigned char* sW = dsm + SA * L::ASTAGE;
    uint64_t* fullA = reinterpret_cast<uint64_t*>(sW + 9 * csteps * L::BSTAGE);
    uint64_t* emptyA = fullA + L::kMaxSA;
    uint64_t* wfull = emptyA + L::kMaxSA;
    uint64_t* tfull = wfull + 1;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* fail = reinterpret_cast<volatile int*>(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (W + L::TW - 1) / L::TW, tiles_y = (H + 8 * SUB - 1) / (8 * SUB);
    const int ntiles = B * tiles_x * tiles_y;
    const int co0 = (blockIdx.x % nsplit) * N;  // this CTA's slice of the output channels
    constexpr uint32_t kIdesc = umma_idesc_bf16(128, L::NA);

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(L::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < SA; ++s) {
            mbar_init(&fullA[s], 1);
            mbar_init(&emptyA[s], 1);
        }
        mbar_init(wfull, 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 32 * kEpiWarps);
        }
        mbar_init(drain, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_in)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_w)) : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_trigger();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ TMA producer
            mbar_expect_tx(wfull, (uint32_t)(9 * csteps * L::BSTAGE));
            for (int cc = 0; cc < csteps; ++cc)
                for (int tap = 0; tap < 9; ++tap)
                    tma_load_2d(sW + (cc * 9 + tap) * L::BSTAGE, &map_w, wfull, cc * L::BK, tap * Cout + co0);
            // the weights may load while an earlier kernel still runs (an early
            // launch requires that it does not write them); the input may not
            pdl_wait();
            int ia = 0, sa = 0;  // halo loads issued; the stage of the next one
            uint32_t pa = 0;     // phase parity of that stage's use
            bool ok = true;
            for (int t = blockIdx.x / nsplit; t < ntiles && ok; t += gridDim.x / nsplit) {
                const int tx = t % tiles_x, r = t / tiles_x, ty = r % tiles_y, b = r / tiles_y;
                const int x0 = tx * L::TW, y0 = ty * 8 * SUB;
                for (int cc = 0; cc < csteps; ++cc) {
                    if (ia >= SA && !(ok = wait_or_fail(&emptyA[sa], pa ^ 1u, fail))) break;
                    mbar_expect_tx(&fullA[sa], L::ASTAGE);
                    for (int j = 0; j < (XS ? 1 : 3); ++j)
                        tma_load_4d(sA + sa * L::ASTAGE + j * L::HALO, &map_in, &fullA[sa], cc * L::BK, x0 + j - 1,
                                    y0 - 1, b);
                    ++ia;
                    if (++sa == SA) {
                        sa = 0;
                        pa ^= 1u;
                    }
                }
            }
            // no copy may still be in flight when the CTA leaves
            wait_timed(wfull, 0, nullptr);
            for (int s = 0; s < SA; ++s) {
                const int k = ia - 1 - ((ia - 1 - s) % SA + SA) % SA;
                if (k >= 0) wait_timed(&fullA[s], (uint32_t)((k / SA) & 1), nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // --------------------------------------------------------- MMA issuer
            // The tensor core queues about one MMA, so every instruction this
            // thread spends between MMAs is time the pipe may idle: a barrier
            // probe costs ~100 cycles while operands stream out of shared
            // memory. Stages and phases are therefore counted rather than
            // divided out, and descriptors are offsets from precomputed ones.
            bool ok = wait_or_fail(wfull, 0, fail);
            tc_fence_after();
            const uint64_t adesc0 = umma_desc_sw<SWB>(smem_u32(sA));
            const uint64_t bdesc0 = umma_desc_sw<SWB>(smem_u32(sW));
            int sa = 0, it = 0;  // halo stage of the next chunk; tiles done
            uint32_t pa = 0;     // its phase parity
            for (int t = blockIdx.x / nsplit; t < ntiles && ok; t += gridDim.x / nsplit) {
                const int acc = it & 1;
                if (it >= 2 && !(ok = wait_or_fail(&tempty[acc], (((uint32_t)it >> 1) & 1u) ^ 1u, fail))) break;
                const uint32_t d = tmem + (uint32_t)(acc * L::NA * SUB);
                for (int cc = 0; cc < csteps && ok; ++cc) {
                    if (!(ok = wait_or_fail(&fullA[sa], pa, fail))) break;
                    tc_fence_after();
                    const uint64_t adesc = desc_at(adesc0, (uint32_t)(sa * L::ASTAGE));
                    const uint64_t bdesc = desc_at(bdesc0, (uint32_t)(cc * 9 * L::BSTAGE));
                    if constexpr (XS) {
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky) {  // taps 3 ky .. 3 ky + 2 in one 3N-row B operand
#pragma unroll
                            for (int kk = 0; kk < L::BK / 16; ++kk)
#pragma unroll
                                for (int h = 0; h < SUB; ++h)
                                    tc_mma(d + (uint32_t)(h * L::NA),
                                           desc_at(adesc, (ky + 8 * h) * 16 * SWB + kk * 32),
                                           desc_at(bdesc, 3 * ky * L::BSTAGE + kk * 32), kIdesc,
                                           (cc | ky | kk) ? 1u : 0u);
                        }
                    } else {
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                            for (int kk = 0; kk < L::BK / 16; ++kk)
#pragma unroll
                                for (int h = 0; h < SUB; ++h)  // sub-tile h: halo rows from 8 h on
                                    tc_mma(d + (uint32_t)(h * N),
                                           desc_at(adesc, (tap % 3) * L::HALO + (tap / 3 + 8 * h) * 16 * SWB + kk * 32),
                                           desc_at(bdesc, tap * L::BSTAGE + kk * 32), kIdesc, (cc | tap | kk) ? 1u : 0u);
                        }
                    }
                    tc_commit(&emptyA[sa]);
                    if (++sa == SA) {
                        sa = 0;
                        pa ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(&tfull[acc]);
                ++it;
            }
            tc_commit(drain);
            wait_timed(drain, 0, nullptr);
        }
    } else {
        // two CTAs per SM leave 168 registers a thread: the bias of a 64-column
        // layer is then read from memory
        conv_epilogue<N, SUB, (MINB == 1 ? N <= 64 : N <= 32), XS>(tmem, tfull, tempty, fail, warp, lane, ntiles,
                                                                    tiles_x, tiles_y, H, W, Cout, bias, relu, epi,
                                                                    nsplit);
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *fail && status) atomicExch(status, 1);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::kTmemCols));
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores: dW[3 ky + kx][ci][co] +=
//   sum over pixels p of in[p shifted by (ky-1, kx-1)][ci] * g[p][co].
// As a GEMM per tap: D (M = ci, N = co) += A (M x K) B^T (K x N) with K = the
// pixels. Both operands come straight from the NHWC tensors in the layout the
// forward kernel stages them in -- pixel rows of channels -- which for this
// GEMM is MN-major (M resp. N contiguous, K = pixel rows): 8-row atoms of
// 8 * SW bytes at stride SBO along K, blocks of SW/2 channels at stride LBO
// along M or N.
//
// One CTA = one work item (kx, 128-channel block of ci, range of output
// tiles). Per 8 x 16-pixel output tile it TMA-loads the kx-shifted input halo
// (10 x 16 pixels) and the tile's output gradient (8 x 16 pixels x Cout).
// The three tap rows ky of this kx read the halo from pixel row 16 ky on.
//   Cin % 128 == 0 ("channel blocks"): M = 128 channels as two 64-channel
//     blocks (two TMA boxes, LBO = one halo copy); three TMEM accumulators,
//     one per ky.
//   Cin = 16, 32 or 64 ("stacked taps"): M = 128 rows are 128 / Cin tap rows
//     ky of Cin channels each, the ky blocks LBO = 16 pixel rows apart in the
//     same halo copy; ceil(3 Cin / 128) accumulators; rows of ky >= 3 are
//     computed on neighbouring shared memory and dropped.
// At the end the epilogue warps read the accumulators (tcgen05.ld) and add
// them into dW with 16-byte float atomics. Roles, bounded waits and the
// failure path are those of conv3x3_fwd_tma_kernel.
template <int N, int SWA, bool STACK>
struct WgradTma {
    static constexpr int EA = SWA / 2;                         // channels per A block
    static constexpr int SWBB = N >= 64 ? 128 : 64;            // B rows: Cout channels, 64 or 32 per block
    static constexpr int EB = SWBB / 2;
    static constexpr int NBB = N / EB;                         // B blocks
    static constexpr int HALO = 10 * 16 * SWA;                 // one halo copy of one A block
    static constexpr int ABYTES = (STACK ? 1 : 2) * HALO;
    static constexpr int BBYTES = NBB * 128 * SWBB;            // 128 pixel rows per B block
    static constexpr int NACC = STACK ? (3 * EA + 127) / 128 : 3;
    static constexpr int STAGE = ABYTES + BBYTES;
    static constexpr int kPad = 4096;                          // reads past the last A stage stay inside
    static constexpr int kFree = 232448 - 1024 - kPad - 256;
    static constexpr int ST = kFree / STAGE > 6 ? 6 : kFree / STAGE;
    static_assert(ST >= 2, "stage ring too small");
    static constexpr int kSmem = 1024 + ST * STAGE + kPad + 256;
    static constexpr int kCols = NACC * N <= 32 ? 32 : (NACC * N <= 64 ? 64 : (NACC * N <= 128 ? 128 : (NACC * N <= 256 ? 256 : 512)));
};

// Matrix descriptor of an MN-major swizzled operand: LBO = stride between
// channel blocks, SBO = stride between 8-pixel-row groups.
template <int SW>
__device__ __forceinline__ uint64_t umma_desc_mn(uint32_t saddr, uint32_t lbo) {
    constexpr uint64_t layout = SW == 128 ? 2 : (SW == 64 ? 4 : 6);
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(((8 * SW) >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

template <int N, int SWA, bool STACK>
__global__ void __launch_bounds__(192, 1)
    conv3x3_wgrad_tma_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_g,
                             int B, int H, int W, int Cin, int Cout, int nsplit, float* __restrict__ dw,
                             int* status) {
    using L = WgradTma<N, SWA, STACK>;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char* dsm = dsm_raw + ((1024u - (smem_u32(dsm_raw) & 1023u)) & 1023u);
    // [B stages][A stages][pad][barriers]: every operand read, however far a
    // stacked-tap block runs past its halo copy, stays inside the allocation
    unsigned char* sB = dsm;
    unsigned char* sA = dsm + L::ST * L::BBYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sA + L::ST * L::ABYTES + L::kPad);
    uint64_t* empty = full + L::ST;
    uint64_t* done = empty + L::ST;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* fail = reinterpret_cast<volatile int*>(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (W + 15) >> 4, tiles_y = (H + 7) >> 3;
    const long long ntiles = (long long)B * tiles_x * tiles_y;
    const int ncb = STACK ? 1 : Cin / 128;
    const int kx = blockIdx.x % 3;
    const int cb = (blockIdx.x / 3) % ncb;
    const int split = blockIdx.x / (3 * ncb);
    const long long t_begin = ntiles * split / nsplit, t_end = ntiles * (split + 1) / nsplit;
    constexpr uint32_t kIdesc = umma_idesc_bf16(128, N) | (1u << 15) | (1u << 16);  // A and B MN-major

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(L::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < L::ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_in)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_g)) : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_trigger();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------------ TMA producer
            int i = 0;
            bool ok = true;
            for (long long t = t_begin; t < t_end && ok; ++t, ++i) {
                const int s = i % L::ST;
                if (i >= L::ST && !(ok = wait_or_fail(&empty[s], (uint32_t)(((i / L::ST) - 1) & 1), fail))) break;
                const int tx = (int)(t % tiles_x);
                const long long r = t / tiles_x;
                const int ty = (int)(r % tiles_y), b = (int)(r / tiles_y);
                mbar_expect_tx(&full[s], L::STAGE);
                unsigned char* a = sA + s * L::ABYTES;
                unsigned char* g = sB + s * L::BBYTES;
                for (int j = 0; j < (STACK ? 1 : 2); ++j)
                    tma_load_4d(a + j * L::HALO, &map_in, &full[s], cb * 128 + j * 64, tx * 16 + kx - 1, ty * 8 - 1, b);
                for (int j = 0; j < L::NBB; ++j)
                    tma_load_4d(g + j * 128 * L::SWBB, &map_g, &full[s], j * L::EB, tx * 16, ty * 8, b);
            }
            // wait for the last load issued into each stage
            for (int s = 0; s < L::ST; ++s) {
                const int k = i - 1 - ((i - 1 - s) % L::ST + L::ST) % L::ST;
                if (k >= 0) wait_timed(&full[s], (uint32_t)((k / L::ST) & 1), nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // --------------------------------------------------------- MMA issuer
            int i = 0;
            bool ok = true;
            for (long long t = t_begin; t < t_end; ++t, ++i) {
                const int s = i % L::ST;
                if (!(ok = wait_or_fail(&full[s], (uint32_t)((i / L::ST) & 1), fail))) break;
                tc_fence_after();
                constexpr uint32_t lboA = STACK ? 16 * SWA : L::HALO;
                constexpr uint32_t lboB = 128 * L::SWBB;
                constexpr int kyPerAcc = STACK ? 128 / L::EA : 1;
                const uint64_t adesc = umma_desc_mn<SWA>(smem_u32(sA + s * L::ABYTES), lboA);
                const uint64_t bdesc = umma_desc_mn<L::SWBB>(smem_u32(sB + s * L::BBYTES), lboB);
#pragma unroll
                for (int acc = 0; acc < L::NACC; ++acc) {
#pragma unroll
                    for (int k = 0; k < 8; ++k)  // 128 pixels = 8 K16 steps of 16 pixel rows
                        tc_mma(tmem + (uint32_t)(acc * N), desc_at(adesc, (acc * kyPerAcc * 16 + k * 16) * SWA),
                               desc_at(bdesc, k * 16 * L::SWBB), kIdesc, (i > 0 || k > 0) ? 1u : 0u);
                }
                tc_commit(&empty[s]);
            }
            (void)ok;
            tc_commit(done);  // arrives once every MMA issued has completed
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const bool fin = wait_timed(done, 0, nullptr);
        if (!fin) *fail = 1;
        tc_fence_after();
        const int qw = warp & 3;
        const int m = qw * 32 + lane;
        if (__all_sync(0xffffffffu, fin && !*fail) && t_end > t_begin) {
            constexpr int kyPerAcc = STACK ? 128 / L::EA : 1;
#pragma unroll 1
            for (int acc = 0; acc < L::NACC; ++acc) {
                const int ky = STACK ? acc * kyPerAcc + m / L::EA : acc;
                const int ci = STACK ? m % L::EA : cb * 128 + m;
                const bool valid = ky < 3;
                float* drow = dw + ((long long)(3 * ky + kx) * Cin + ci) * Cout;
                const uint32_t taddr = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)(acc * N);
#pragma unroll 1
                for (int c0 = 0; c0 < N; c0 += 16) {
                    uint32_t rr[16];
                    tc_ld16(taddr + (uint32_t)c0, rr);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    if (valid) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            atomicAdd(reinterpret_cast<float4*>(drow + c0 + 4 * j),
                                      make_float4(__uint_as_float(rr[4 * j]), __uint_as_float(rr[4 * j + 1]),
                                                  __uint_as_float(rr[4 * j + 2]), __uint_as_float(rr[4 * j + 3])));
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *fail && status) atomicExch(status, 1);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::kCols));
    }
}

}  // namespace qldnn
