// qld_nn.cuh -- kernels of the learned short-window network.
//
// The paper has no learned component: this network maps the I/Q maps of a
// short window (N = 32) to the amplitude plain QLD reaches with a long window
// (N = 1024), so an image needs far fewer frames. Its 3x3 convolutions are
// implicit GEMMs on the BF16 tensor cores with FP32 accumulation:
//   forward   out[p][co] = sum_{tap,ci} in[p + shift(tap)][ci] w[tap][ci][co]
//             (M = pixels, N = Cout, K = 9 Cin; zero padding 1)
//   data grad the forward kernel on weights flipped in tap and transposed in
//             channels: din = conv(g; w'[8 - tap][co][ci])
//   weight grad dw[tap][ci][co] = sum_p in[p + shift(tap)][ci] g[p][co]
//             (M = Cin, N = Cout, K = pixels, split over CTAs)
// Activations are NHWC bf16 with a channel count that is a multiple of 16.

#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace qldnn {

// ------------------------------------------------------------ primitives --

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte global -> shared copy; src_bytes = 0 fills the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// D (16x8 f32) += A (16x16 bf16, row-major) * B (16x8 bf16, column-major)
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------- forward conv --

// Shared-memory tiles of one K step (16 channels of one tap):
//   A [128 pixels][16 ch]   32-byte rows, 16-byte chunk c stored at c ^ ((row >> 2) & 1)
//   B [16 ch][BN couts]     BN*2-byte rows, chunk c stored at c ^ (row & (BN/8 - 1))
// so the 8 row addresses of every ldmatrix hit distinct banks.
template <int BN>
struct ConvFwdSmem {
    __nv_bfloat16 a[2][128 * 16];
    __nv_bfloat16 b[2][16 * BN];
};

__device__ __forceinline__ int a_swz(int row, int chunk) { return row * 16 + ((chunk ^ ((row >> 2) & 1)) << 3); }
template <int BN>
__device__ __forceinline__ int b_swz(int row, int chunk) {
    return row * BN + ((chunk ^ (row & (BN / 8 - 1))) << 3);
}

// out = act(conv3x3(in, w) + bias). in [B*H*W][Cin] bf16 (Cin % 16 == 0),
// w [9][Cin][Cout] bf16, bias [Cout] f32 or NULL, Cout % BN == 0. Output bf16
// [P][Cout] (out_bf) and/or f32 (out_f). relu: clamp at 0. CTA = 128 threads,
// tile 128 pixels x BN output channels; warp w takes pixels 32w..32w+31.
template <int BN>
__global__ void __launch_bounds__(128) conv3x3_fwd_kernel(const __nv_bfloat16* __restrict__ in,
                                                          const __nv_bfloat16* __restrict__ w,
                                                          const float* __restrict__ bias, int B, int H, int W,
                                                          int Cin, int Cout, int relu, __nv_bfloat16* out_bf,
                                                          float* out_f) {
    __shared__ __align__(128) ConvFwdSmem<BN> sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long P = (long long)B * H * W;
    const long long p0 = (long long)blockIdx.x * 128;
    const int co0 = blockIdx.y * BN;
    const int csteps = Cin / 16;
    const int ksteps = 9 * csteps;

    // this thread's pixel for the A loads
    const long long pm = p0 + tid;
    int py = 0, px = 0;
    long long pb = 0;
    if (pm < P) {
        pb = pm / ((long long)H * W);
        const long long r = pm - pb * H * W;
        py = (int)(r / W);
        px = (int)(r - (long long)py * W);
    }

    auto load_stage = [&](int stage, int ks) {
        const int tap = ks / csteps, cc = ks - tap * csteps;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const int yy = py + dy, xx = px + dx;
        const bool ok = pm < P && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const __nv_bfloat16* src = ok ? in + (((pb * H + yy) * W + xx) * Cin + cc * 16) : in;
#pragma unroll
        for (int c = 0; c < 2; ++c) cp_async16(&sm.a[stage][a_swz(tid, c)], src + 8 * c, ok ? 16 : 0);
        // B: 16 rows x BN columns = 16*BN/8 chunks
        constexpr int BCH = 16 * BN / 8;
        for (int i = tid; i < BCH; i += 128) {
            const int row = i / (BN / 8), ch = i % (BN / 8);
            const __nv_bfloat16* wsrc = w + ((long long)(tap * Cin + cc * 16 + row) * Cout + co0 + ch * 8);
            cp_async16(&sm.b[stage][b_swz<BN>(row, ch)], wsrc, 16);
        }
        cp_async_commit();
    };

    float acc[2][BN / 8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < BN / 8; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    load_stage(0, 0);
    for (int ks = 0; ks < ksteps; ++ks) {
        const int cur = ks & 1;
        if (ks + 1 < ksteps) {
            load_stage(cur ^ 1, ks + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        uint32_t af[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const int j = lane >> 3, i = lane & 7;
            const int row = warp * 32 + mi * 16 + i + 8 * (j & 1);
            ldsm_x4(af[mi], &sm.a[cur][a_swz(row, j >> 1)]);
        }
#pragma unroll
        for (int nj = 0; nj < BN / 16; ++nj) {
            uint32_t bf[4];
            const int j = lane >> 3, i = lane & 7;
            const int row = i + 8 * (j & 1);
            ldsm_x4_t(bf, &sm.b[cur][b_swz<BN>(row, nj * 2 + (j >> 1))]);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                mma_bf16(acc[mi][2 * nj], af[mi], bf);
                mma_bf16(acc[mi][2 * nj + 1], af[mi], bf + 2);
            }
        }
        __syncthreads();
    }

    // epilogue: rows lane/4 (+8), columns 2*(lane%4) (+1) of each 16x8 tile
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long p = p0 + warp * 32 + mi * 16 + (lane >> 2) + 8 * h;
            if (p >= P) continue;
#pragma unroll
            for (int nj = 0; nj < BN / 8; ++nj) {
                const int co = co0 + nj * 8 + 2 * (lane & 3);
                float v0 = acc[mi][nj][2 * h], v1 = acc[mi][nj][2 * h + 1];
                if (bias) {
                    v0 += bias[co];
                    v1 += bias[co + 1];
                }
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (out_bf)
                    *reinterpret_cast<__nv_bfloat162*>(out_bf + p * Cout + co) = __floats2bfloat162_rn(v0, v1);
                if (out_f) *reinterpret_cast<float2*>(out_f + p * Cout + co) = make_float2(v0, v1);
            }
        }
    }
}

// ------------------------------------------------------- weight gradient --

// dw[tap][ci][co] += sum over this CTA's pixels of in[p + shift(tap)][ci] g[p][co]
// for ci in [ci0, ci0 + 16 * MT), co in [co0, co0 + BN). GEMM with M = ci,
// N = co, K = pixels, both operands stored pixel-major in shared memory and
// read with transposing ldmatrix. Each of the 4 warps takes every 4th K step
// of 16 pixels; the warps' partial tiles are summed in shared memory and
// added to dw (f32) with atomics. Grid: (pixel chunks, 9 taps, ci/co tiles).
template <int MT, int BN>
__global__ void __launch_bounds__(128) conv3x3_wgrad_kernel(const __nv_bfloat16* __restrict__ in,
                                                           const __nv_bfloat16* __restrict__ g, int B, int H,
                                                           int W, int Cin, int Cout, int pix_per_cta,
                                                           float* __restrict__ dw) {
    constexpr int BM = 16 * MT;
    __shared__ __align__(128) __nv_bfloat16 sa[4][2][16 * BM];  // [warp][stage][16 pixels][BM ci]
    __shared__ __align__(128) __nv_bfloat16 sb[4][2][16 * BN];  // [warp][stage][16 pixels][BN co]
    __shared__ float red[BM * BN];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long P = (long long)B * H * W;
    const int tap = blockIdx.y;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int ntile_co = Cout / BN;
    const int ci0 = (blockIdx.z / ntile_co) * BM, co0 = (blockIdx.z % ntile_co) * BN;
    const long long pbeg = (long long)blockIdx.x * pix_per_cta;
    const long long pend = pbeg + pix_per_cta < P ? pbeg + pix_per_cta : P;
    const int nsteps = (int)((pend - pbeg + 15) / 16);

    for (int i = tid; i < BM * BN; i += 128) red[i] = 0.f;

    float acc[MT][BN / 8][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < BN / 8; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    // one warp loads its own 16-pixel step: A = in (shifted) [16][BM], B = g [16][BN]
    auto load = [&](int stage, int step) {
        const long long pbase = pbeg + (long long)step * 16;
        constexpr int ACH = 16 * BM / 8, BCH = 16 * BN / 8;
        for (int i = lane; i < ACH + BCH; i += 32) {
            const bool is_a = i < ACH;
            const int ii = is_a ? i : i - ACH;
            const int cpr = is_a ? BM / 8 : BN / 8;  // chunks per row
            const int row = ii / cpr, ch = ii % cpr;
            const long long p = pbase + row;
            const __nv_bfloat16* src = is_a ? in : g;
            int ok = 0;
            if (p < pend) {
                if (is_a) {
                    const long long b = p / ((long long)H * W);
                    const long long r = p - b * H * W;
                    const int y = (int)(r / W), x = (int)(r - (long long)(r / W) * W);
                    const int yy = y + dy, xx = x + dx;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                        src = in + (((b * H + yy) * W + xx) * Cin + ci0 + ch * 8);
                        ok = 16;
                    }
                } else {
                    src = g + (p * Cout + co0 + ch * 8);
                    ok = 16;
                }
            }
            __nv_bfloat16* dst = is_a ? &sa[warp][stage][row * BM + ((ch ^ (row & (BM / 8 - 1))) << 3)]
                                      : &sb[warp][stage][row * BN + ((ch ^ (row & (BN / 8 - 1))) << 3)];
            cp_async16(dst, src, ok);
        }
        cp_async_commit();
    };

    int step = warp;
    if (step < nsteps) load(0, step);
    int stage = 0;
    for (; step < nsteps; step += 4) {
        if (step + 4 < nsteps) {
            load(stage ^ 1, step + 4);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const int j = lane >> 3, i = lane & 7;
#pragma unroll
        for (int mi = 0; mi < MT; ++mi) {
            // A fragment of the transposed tile: smem row k (pixel), column m (ci)
            uint32_t af[4];
            const int krow = i + 8 * (j >> 1);
            const int mch = mi * 2 + (j & 1);
            ldsm_x4_t(af, &sa[warp][stage][krow * BM + ((mch ^ (krow & (BM / 8 - 1))) << 3)]);
#pragma unroll
            for (int nj = 0; nj < BN / 16; ++nj) {
                uint32_t bf[4];
                const int brow = i + 8 * (j & 1);
                const int nch = nj * 2 + (j >> 1);
                ldsm_x4_t(bf, &sb[warp][stage][brow * BN + ((nch ^ (brow & (BN / 8 - 1))) << 3)]);
                mma_bf16(acc[mi][2 * nj], af, bf);
                mma_bf16(acc[mi][2 * nj + 1], af, bf + 2);
            }
        }
        __syncwarp();
        stage ^= 1;
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int nj = 0; nj < BN / 8; ++nj)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = mi * 16 + (lane >> 2) + 8 * h;
                const int n = nj * 8 + 2 * (lane & 3);
                atomicAdd(&red[m * BN + n], acc[mi][nj][2 * h]);
                atomicAdd(&red[m * BN + n + 1], acc[mi][nj][2 * h + 1]);
            }
    __syncthreads();
    for (int e = tid; e < BM * BN; e += 128) {
        const int m = e / BN, n = e % BN;
        atomicAdd(&dw[((long long)tap * Cin + ci0 + m) * Cout + co0 + n], red[e]);
    }
}

}  // namespace qldnn
