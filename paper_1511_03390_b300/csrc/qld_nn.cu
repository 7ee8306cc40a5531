// qld_nn.cu -- C ABI of the learned short-window network's kernels
// (declared in include/qld.h, section "Learned short-window QLD").
//
// Activations: NHWC, bf16, channels a multiple of 16. Gradients: f32 until
// they become the operand of a tensor-core GEMM, then bf16. Weights: f32
// master copies (Adam) and bf16 compute copies [9][Cin][Cout].

#include <atomic>
#include <cstdint>
#include <mutex>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "qld.h"
#include "qld_internal.h"
#include "qld_nn.cuh"
#include "qld_nn_tc.cuh"
#include "qld_nn_tma.cuh"

using qldi::set_err;

namespace {

unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }
bool al(const void* p, unsigned a) { return ((uintptr_t)p % a) == 0; }
int launched(int n) {
    qldi::count_launches(n);
    return cudaGetLastError() == cudaSuccess ? QLD_OK : set_err(QLD_E_CUDA);
}

// w [9][Cin][Cout] -> wt [9][Cout][Cin] with the tap order reversed, so that
// conv(g; wt) is the data gradient of conv(x; w).
__global__ void flip_transpose_kernel(const __nv_bfloat16* __restrict__ w, int Cin, int Cout,
                                      __nv_bfloat16* __restrict__ wt) {
    const long long n = 9ll * Cin * Cout;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int tap = (int)(e / ((long long)Cin * Cout));
        const long long r = e - (long long)tap * Cin * Cout;
        const int ci = (int)(r / Cout), co = (int)(r % Cout);
        wt[((long long)(8 - tap) * Cout + co) * Cin + ci] = w[e];
    }
}

__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ g, long long P, int C, float* __restrict__ db) {
    // thread block = 256 = `lanes` groups of C threads (plus idle ones); each
    // thread sums one channel over a strided range of pixels
    const int lanes = 256 / C;  // C <= 256
    if ((int)threadIdx.x >= lanes * C) return;
    const int c = threadIdx.x % C;
    const int l = threadIdx.x / C;
    float acc = 0.f;
    for (long long p = (long long)blockIdx.x * lanes + l; p < P; p += (long long)gridDim.x * lanes)
        acc += __bfloat162float(g[p * C + c]);
    atomicAdd(&db[c], acc);
}

__global__ void relu_bwd_kernel(const float* __restrict__ g, const __nv_bfloat16* __restrict__ act, long long n,
                                __nv_bfloat16* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(__bfloat162float(act[i]) > 0.f ? g[i] : 0.f);
}

__global__ void avgpool2_fwd_kernel(const __nv_bfloat16* __restrict__ in, int B, int H, int W, int C,
                                    __nv_bfloat16* __restrict__ out) {
    const int h = H / 2, w = W / 2;
    const long long n = (long long)B * h * w * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int x = (int)(r % w);
        r /= w;
        const int y = (int)(r % h);
        const long long b = r / h;
        const long long base = ((b * H + 2 * y) * W + 2 * x) * C + c;
        // the two diagonals of the 2x2 block, then their sum: the same for
        // every order of the four pixels, as the fused convolution epilogue
        // (each of whose lanes starts from its own pixel) computes it
        const float s = (__bfloat162float(in[base]) + __bfloat162float(in[base + (long long)W * C + C])) +
                        (__bfloat162float(in[base + C]) + __bfloat162float(in[base + (long long)W * C]));
        out[e] = __float2bfloat16_rn(0.25f * s);
    }
}

__global__ void avgpool2_bwd_kernel(const float* __restrict__ g, int B, int H, int W, int C, float* __restrict__ out,
                                    int accumulate) {
    const long long n = (long long)B * H * W * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int x = (int)(r % W);
        r /= W;
        const int y = (int)(r % H);
        const long long b = r / H;
        const float v = 0.25f * g[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
        out[e] = accumulate ? out[e] + v : v;
    }
}

__global__ void upsample2_fwd_kernel(const __nv_bfloat16* __restrict__ in, int B, int h, int w, int C,
                                     __nv_bfloat16* __restrict__ out) {
    const long long n = (long long)B * 2 * h * 2 * w * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int x = (int)(r % (2 * w));
        r /= 2 * w;
        const int y = (int)(r % (2 * h));
        const long long b = r / (2 * h);
        out[e] = in[((b * h + y / 2) * w + x / 2) * C + c];
    }
}

__global__ void upsample2_bwd_kernel(const float* __restrict__ g, int B, int h, int w, int C, float* __restrict__ out) {
    const long long n = (long long)B * h * w * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int x = (int)(r % w);
        r /= w;
        const int y = (int)(r % h);
        const long long b = r / h;
        const long long base = ((b * 2 * h + 2 * y) * (2 * w) + 2 * x) * C + c;
        const long long row = (long long)2 * w * C;
        out[e] = g[base] + g[base + C] + g[base + row] + g[base + row + C];
    }
}

__global__ void concat_kernel(const __nv_bfloat16* __restrict__ a, int Ca, const __nv_bfloat16* __restrict__ b,
                              int Cb, long long P, __nv_bfloat16* __restrict__ out) {
    const int C = Ca + Cb;
    const long long n = P * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / C;
        const int c = (int)(e - p * C);
        out[e] = c < Ca ? a[p * Ca + c] : b[p * Cb + (c - Ca)];
    }
}

__global__ void split_kernel(const float* __restrict__ g, long long P, int Ca, int Cb, float* __restrict__ ga,
                             float* __restrict__ gb, int accumulate_b) {
    const int C = Ca + Cb;
    const long long n = P * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / C;
        const int c = (int)(e - p * C);
        if (c < Ca) {
            ga[p * Ca + c] = g[e];
        } else {
            float* d = gb + p * Cb + (c - Ca);
            *d = accumulate_b ? *d + g[e] : g[e];
        }
    }
}

// 1x1 output head: out[p] = b + sum_c in[p][c] w[c] (f32 accumulate).
__global__ void head_fwd_kernel(const __nv_bfloat16* __restrict__ in, const float* __restrict__ w,
                                const float* __restrict__ bp, long long P, int C, float* __restrict__ out) {
    const float b = *bp;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        float acc = b;
        for (int c = 0; c < C; ++c) acc = fmaf(__bfloat162float(in[p * C + c]), w[c], acc);
        out[p] = acc;
    }
}

// head backward: din[p][c] = g[p] w[c]; dw[c] += sum_p in[p][c] g[p]; db += sum_p g[p]
__global__ void head_bwd_kernel(const __nv_bfloat16* __restrict__ in, const float* __restrict__ g,
                                const float* __restrict__ w, long long P, int C, float* __restrict__ din,
                                float* __restrict__ dw, float* __restrict__ db) {
    __shared__ float sdw[256];
    __shared__ float sdb;
    for (int c = threadIdx.x; c < C; c += blockDim.x) sdw[c] = 0.f;
    if (threadIdx.x == 0) sdb = 0.f;
    __syncthreads();
    float pdb = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float gp = g[p];
        pdb += gp;
        for (int c = 0; c < C; ++c) {
            din[p * C + c] = gp * w[c];
            atomicAdd(&sdw[c], __bfloat162float(in[p * C + c]) * gp);
        }
    }
    atomicAdd(&sdb, pdb);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&dw[c], sdw[c]);
    if (threadIdx.x == 0) atomicAdd(db, sdb);
}

// mean squared error over n values: loss += sum (pred - t)^2 / n, grad = 2 (pred - t) / n
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ t, long long n,
                           float* __restrict__ grad, float* __restrict__ loss) {
    float acc = 0.f;
    const float inv = 1.f / (float)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = pred[i] - t[i];
        grad[i] = 2.f * d * inv;
        acc += d * d * inv;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// Adam (Kingma & Ba 2015) on f32 master weights; refreshes the bf16 copy.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16* __restrict__ p_bf) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (p_bf) p_bf[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void cast_bf16_kernel(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void add_kernel(float* __restrict__ y, const float* __restrict__ x, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += x[i];
}

// Network input from the short-window sums: channels (S, C, R) * scale, then
// zeros up to 16 channels. R = sqrt(S^2 + C^2).
// ---- 16-byte (8 x bf16 channel) versions of the forward glue kernels; used
// whenever every channel count involved is a multiple of 8.
__device__ __forceinline__ void unpack8(const uint4 q, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float* f) {
    uint4 q;
    uint32_t* u = reinterpret_cast<uint32_t*>(&q);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
        u[j] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    return q;
}

__global__ void avgpool2_fwd_v8_kernel(const uint4* __restrict__ in, int B, int H, int W, int C8,
                                       uint4* __restrict__ out) {
    const int h = H / 2, w = W / 2;
    const long long n = (long long)B * h * w * C8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C8);
        long long r = e / C8;
        const int x = (int)(r % w);
        r /= w;
        const int y = (int)(r % h);
        const long long b = r / h;
        const long long base = ((b * H + 2 * y) * W + 2 * x) * C8 + c;
        float f0[8], f1[8], f2[8], f3[8], o[8];
        unpack8(__ldg(in + base), f0);
        unpack8(__ldg(in + base + C8), f1);
        unpack8(__ldg(in + base + (long long)W * C8), f2);
        unpack8(__ldg(in + base + (long long)W * C8 + C8), f3);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = 0.25f * ((f0[j] + f3[j]) + (f1[j] + f2[j]));  // diagonals first
        out[e] = pack8(o);
    }
}

__global__ void upsample2_fwd_v8_kernel(const uint4* __restrict__ in, int B, int h, int w, int C8,
                                        uint4* __restrict__ out) {
    const long long n = (long long)B * 2 * h * 2 * w * C8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C8);
        long long r = e / C8;
        const int x = (int)(r % (2 * w));
        r /= 2 * w;
        const int y = (int)(r % (2 * h));
        const long long b = r / (2 * h);
        out[e] = __ldg(in + ((b * h + y / 2) * w + x / 2) * C8 + c);
    }
}

__global__ void concat_v8_kernel(const uint4* __restrict__ a, int Ca8, const uint4* __restrict__ b, int Cb8,
                                 long long P, uint4* __restrict__ out) {
    const int C8 = Ca8 + Cb8;
    const long long n = P * C8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / C8;
        const int c = (int)(e - p * C8);
        out[e] = c < Ca8 ? __ldg(a + p * Ca8 + c) : __ldg(b + p * Cb8 + (c - Ca8));
    }
}

// out[b][Y][X] = [ u[b][Y/2][X/2] (Cu channels) , e[b][Y][X] (Ce channels) ]
// at the full resolution 2h x 2w: nearest 2x upsampling of u fused with the
// channel concatenation.
__global__ void upsample_concat_v8_kernel(const uint4* __restrict__ u, int Cu8, const uint4* __restrict__ e, int Ce8,
                                          int B, int h, int w, uint4* __restrict__ out) {
    const int C8 = Cu8 + Ce8;
    const long long n = (long long)B * 4 * h * w * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / C8;
        const int c = (int)(i - p * C8);
        if (c < Cu8) {
            const int x = (int)(p % (2 * w));
            const long long r = p / (2 * w);
            const int y = (int)(r % (2 * h));
            const long long b = r / (2 * h);
            out[i] = __ldg(u + ((b * h + y / 2) * w + x / 2) * Cu8 + c);
        } else {
            out[i] = __ldg(e + p * Ce8 + (c - Cu8));
        }
    }
}

__global__ void head_fwd_v8_kernel(const uint4* __restrict__ in, const float* __restrict__ w,
                                   const float* __restrict__ bp, long long P, int C8, float* __restrict__ out) {
    const float b = *bp;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        float acc = b;
        for (int g = 0; g < C8; ++g) {
            float f[8];
            unpack8(__ldg(in + p * C8 + g), f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc = fmaf(f[j], __ldg(w + 8 * g + j), acc);
        }
        out[p] = acc;
    }
}

// ---- 16-byte versions of the backward glue kernels (4 f32 / 8 bf16 channels
// per thread), used whenever the channel counts allow.
__global__ void relu_bwd_v4_kernel(const float4* __restrict__ g, const uint2* __restrict__ act, long long n4,
                                   uint2* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 gv = __ldg(g + i);
        const uint2 av = __ldg(act + i);
        const float2 a01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&av.x));
        const float2 a23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&av.y));
        const __nv_bfloat162 o01 = __floats2bfloat162_rn(a01.x > 0.f ? gv.x : 0.f, a01.y > 0.f ? gv.y : 0.f);
        const __nv_bfloat162 o23 = __floats2bfloat162_rn(a23.x > 0.f ? gv.z : 0.f, a23.y > 0.f ? gv.w : 0.f);
        out[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&o01), *reinterpret_cast<const uint32_t*>(&o23));
    }
}

__global__ void avgpool2_bwd_v4_kernel(const float4* __restrict__ g, int B, int H, int W, int C4,
                                       float4* __restrict__ out, int accumulate) {
    const long long n = (long long)B * H * W * C4;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C4);
        long long r = e / C4;
        const int x = (int)(r % W);
        r /= W;
        const int y = (int)(r % H);
        const long long b = r / H;
        const float4 gv = __ldg(g + ((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C4 + c);
        float4 v = make_float4(0.25f * gv.x, 0.25f * gv.y, 0.25f * gv.z, 0.25f * gv.w);
        if (accumulate) {
            const float4 o = out[e];
            v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
        }
        out[e] = v;
    }
}

__global__ void upsample2_bwd_v4_kernel(const float4* __restrict__ g, int B, int h, int w, int C4,
                                        float4* __restrict__ out) {
    const long long n = (long long)B * h * w * C4;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C4);
        long long r = e / C4;
        const int x = (int)(r % w);
        r /= w;
        const int y = (int)(r % h);
        const long long b = r / h;
        const long long base = ((b * 2 * h + 2 * y) * (2 * w) + 2 * x) * C4 + c;
        const long long row = (long long)2 * w * C4;
        const float4 a = __ldg(g + base), b1 = __ldg(g + base + C4), c1 = __ldg(g + base + row),
                     d = __ldg(g + base + row + C4);
        out[e] = make_float4(a.x + b1.x + c1.x + d.x, a.y + b1.y + c1.y + d.y, a.z + b1.z + c1.z + d.z,
                             a.w + b1.w + c1.w + d.w);
    }
}

__global__ void split_v4_kernel(const float4* __restrict__ g, long long P, int Ca4, int Cb4, float4* __restrict__ ga,
                                float4* __restrict__ gb, int accumulate_b) {
    const int C4 = Ca4 + Cb4;
    const long long n = P * C4;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / C4;
        const int c = (int)(e - p * C4);
        const float4 v = __ldg(g + e);
        if (c < Ca4) {
            ga[p * Ca4 + c] = v;
        } else {
            float4* d = gb + p * Cb4 + (c - Ca4);
            if (accumulate_b) {
                const float4 o = *d;
                *d = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
            } else {
                *d = v;
            }
        }
    }
}

// db[c] += sum over pixels of g[p][c] (bf16), C % 8 == 0, C <= 256: each
// thread keeps 8 channel sums in registers over a strided range of pixels,
// the block adds them up in shared memory, then one atomic per channel per
// block (a grid of a few hundred blocks).
__global__ void bias_grad_v8_kernel(const uint4* __restrict__ g, long long P, int C, float* __restrict__ db) {
    __shared__ float sacc[256];
    const int G8 = C / 8;
    const int lanes = 256 / G8;
    for (int c = threadIdx.x; c < C; c += blockDim.x) sacc[c] = 0.f;
    __syncthreads();
    if ((int)threadIdx.x < lanes * G8) {
        const int gi = threadIdx.x % G8;
        const int l = threadIdx.x / G8;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (long long p = (long long)blockIdx.x * lanes + l; p < P; p += (long long)gridDim.x * lanes) {
            float f[8];
            unpack8(__ldg(g + p * G8 + gi), f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += f[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(&sacc[8 * gi + j], acc[j]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], sacc[c]);
}

// ReLU backward fused with the bias gradient: out[p][c] = bf16(act > 0 ? g : 0)
// and db[c] += sum over pixels of that bf16 value (C % 8 == 0, C <= 256);
// the reduction is that of bias_grad_v8_kernel.
__global__ void relu_bwd_bias_v8_kernel(const float4* __restrict__ g, const uint4* __restrict__ act, long long P,
                                        int C, uint4* __restrict__ out, float* __restrict__ db) {
    __shared__ float sacc[256];
    const int G8 = C / 8;
    const int lanes = 256 / G8;
    for (int c = threadIdx.x; c < C; c += blockDim.x) sacc[c] = 0.f;
    __syncthreads();
    if ((int)threadIdx.x < lanes * G8) {
        const int gi = threadIdx.x % G8;
        const int l = threadIdx.x / G8;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (long long p = (long long)blockIdx.x * lanes + l; p < P; p += (long long)gridDim.x * lanes) {
            const long long e = p * G8 + gi;
            const float4 g0 = __ldg(g + 2 * e), g1 = __ldg(g + 2 * e + 1);
            float a[8];
            unpack8(__ldg(act + e), a);
            const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
            float o[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) o[j] = a[j] > 0.f ? gv[j] : 0.f;
            const uint4 q = pack8(o);
            out[e] = q;
            float r[8];
            unpack8(q, r);  // the bias gradient sums the stored (bf16) values
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += r[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(&sacc[8 * gi + j], acc[j]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], sacc[c]);
}

// head backward for CT channels (CT % 8 == 0): one pixel per thread, the
// weight-gradient partials in registers, reduced across the warp with
// shuffles, then per block in shared memory, then one atomic per channel.
template <int CT>
__global__ void head_bwd_v8_kernel(const uint4* __restrict__ in, const float* __restrict__ g,
                                   const float* __restrict__ w, long long P, float4* __restrict__ din,
                                   float* __restrict__ dw, float* __restrict__ db) {
    __shared__ float sdw[CT + 1];
    for (int c = threadIdx.x; c <= CT; c += blockDim.x) sdw[c] = 0.f;
    __syncthreads();
    float acc[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[c] = 0.f;
    float pdb = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float gp = __ldg(g + p);
        pdb += gp;
#pragma unroll
        for (int q = 0; q < CT / 8; ++q) {
            float f[8];
            unpack8(__ldg(in + p * (CT / 8) + q), f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[8 * q + j] = fmaf(f[j], gp, acc[8 * q + j]);
        }
#pragma unroll
        for (int q = 0; q < CT / 4; ++q)
            din[p * (CT / 4) + q] = make_float4(gp * __ldg(w + 4 * q), gp * __ldg(w + 4 * q + 1),
                                                gp * __ldg(w + 4 * q + 2), gp * __ldg(w + 4 * q + 3));
    }
#pragma unroll
    for (int c = 0; c < CT; ++c) {
        float v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sdw[c], v);
    }
    for (int o = 16; o > 0; o >>= 1) pdb += __shfl_xor_sync(0xffffffffu, pdb, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sdw[CT], pdb);
    __syncthreads();
    for (int c = threadIdx.x; c < CT; c += blockDim.x) atomicAdd(&dw[c], sdw[c]);
    if (threadIdx.x == 0) atomicAdd(db, sdw[CT]);
}

// The network's first convolution fused with its input packing. The packed
// input (qldnn_pack_input) has channels (s, c, sqrt(s^2 + c^2)) * scale in
// bf16 and zeros after them, so only the weights of input channels 0..2
// contribute: a 27 x CO contraction per pixel, done here on the FP32 cores
// (tensor-core tiles would multiply 13 zero channels out of 16). A CTA takes
// a 16 x 16 output tile: the three channels of its 18 x 18 input halo are
// computed once into shared memory with exactly the packing's operations,
// each thread accumulates one pixel's CO outputs (taps, then channels, in
// FP32), adds the bias, applies ReLU and stores bf16; the baseline (the
// scaled amplitude, f32) of its pixels is written as qldnn_pack_input does.
// Two FP32 lanes in one 64-bit register for the paired FMA (fma.rn.f32x2:
// each lane rounds as fmaf, one issue slot per pair).
__device__ __forceinline__ unsigned long long splat2(float a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float2 split2(unsigned long long a) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
    return r;
}

template <int CO>
__global__ void __launch_bounds__(128) input_conv3x3_kernel(const int32_t* __restrict__ S, const int32_t* __restrict__ C,
                                                            int B, int H, int W, float scale,
                                                            const __nv_bfloat16* __restrict__ w, int Cin,
                                                            const float* __restrict__ bias, int relu,
                                                            __nv_bfloat16* __restrict__ out, long long ldo,
                                                            float* __restrict__ baseline) {
    // Persistent over tiles (weights staged once per CTA). 128 threads,
    // thread t: pixels (t / 16, t mod 16) and (t / 16 + 8, t mod 16) of the
    // tile, so each weight read from shared memory (4 channels at a time)
    // serves 8 FMAs.
    __shared__ float xin[3][18][18];
    __shared__ float4 ws[27][CO / 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int tiles_x = (W + 15) >> 4, tiles_y = (H + 15) >> 4;
    const long long ntiles = (long long)B * tiles_x * tiles_y;
    float* wsf = reinterpret_cast<float*>(ws);
    for (int i = threadIdx.x; i < 27 * CO; i += 128) {
        const int tc = i / CO, co = i - tc * CO;
        const int tap = tc / 3, ci = tc - tap * 3;
        wsf[i] = __bfloat162float(w[((long long)tap * Cin + ci) * CO + co]);
    }
    // the next layer (launched early, qldnn_conv3x3_fwd_tma_epi) may start
    // its set-up now; it waits for this kernel before reading its output
    asm volatile("griddepcontrol.launch_dependents;" :::);
    for (long long t0 = blockIdx.x; t0 < ntiles; t0 += gridDim.x) {
        long long t = t0;
        const int bx = (int)(t % tiles_x);
        t /= tiles_x;
        const int by = (int)(t % tiles_y);
        const int b = (int)(t / tiles_y);
        const int x0 = bx * 16, y0 = by * 16;
        // the halo's sums: every load issued before any use (3 per thread)
        int32_t sv[3], cv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int i = threadIdx.x + 128 * k;
            const int yy = i / 18, xx = i - yy * 18;
            const int gy = y0 + yy - 1, gx = x0 + xx - 1;
            const bool ok = i < 18 * 18 && gy >= 0 && gy < H && gx >= 0 && gx < W;
            const long long p = ok ? ((long long)b * H + gy) * W + gx : 0;  // in bounds either way
            sv[k] = ok ? __ldg(S + p) : 0;
            cv[k] = ok ? __ldg(C + p) : 0;
        }
        __syncthreads();  // the previous tile's reads of xin are done
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int i = threadIdx.x + 128 * k;
            if (i < 18 * 18) {
                const int yy = i / 18, xx = i - yy * 18;
                const float s0 = (float)sv[k], c0 = (float)cv[k];
                const float r = sqrtf(s0 * s0 + c0 * c0) * scale;
                xin[0][yy][xx] = __bfloat162float(__float2bfloat16_rn(s0 * scale));
                xin[1][yy][xx] = __bfloat162float(__float2bfloat16_rn(c0 * scale));
                xin[2][yy][xx] = __bfloat162float(__float2bfloat16_rn(r));
            }
        }
        __syncthreads();
        unsigned long long a0[CO / 2], a1[CO / 2];  // channel pairs
#pragma unroll
        for (int h = 0; h < CO / 2; ++h) a0[h] = a1[h] = 0ull;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
            for (int ci = 0; ci < 3; ++ci) {
                const unsigned long long xa = splat2(xin[ci][ty + tap / 3][tx + tap % 3]);
                const unsigned long long xb = splat2(xin[ci][ty + 8 + tap / 3][tx + tap % 3]);
                const ulonglong2* wrow = reinterpret_cast<const ulonglong2*>(ws[tap * 3 + ci]);
#pragma unroll
                for (int q = 0; q < CO / 4; ++q) {
                    const ulonglong2 w2 = wrow[q];  // channels (4q, 4q+1) and (4q+2, 4q+3)
                    a0[2 * q] = fma2(xa, w2.x, a0[2 * q]);
                    a0[2 * q + 1] = fma2(xa, w2.y, a0[2 * q + 1]);
                    a1[2 * q] = fma2(xb, w2.x, a1[2 * q]);
                    a1[2 * q + 1] = fma2(xb, w2.y, a1[2 * q + 1]);
                }
            }
        }
        float acc0[CO], acc1[CO];
#pragma unroll
        for (int h = 0; h < CO / 2; ++h) {
            const float2 u = split2(a0[h]), v = split2(a1[h]);
            acc0[2 * h] = u.x;
            acc0[2 * h + 1] = u.y;
            acc1[2 * h] = v.x;
            acc1[2 * h + 1] = v.y;
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int gy = y0 + ty + 8 * half, gx = x0 + tx;
            if (gy >= H || gx >= W) continue;
            const long long p = ((long long)b * H + gy) * W + gx;
            const float* acc = half ? acc1 : acc0;
#pragma unroll
            for (int q = 0; q < CO / 8; ++q) {
                float f[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float v = acc[8 * q + j] + (bias ? bias[8 * q + j] : 0.f);
                    f[j] = relu ? fmaxf(v, 0.f) : v;
                }
                reinterpret_cast<uint4*>(out + p * ldo)[q] = pack8(f);
            }
            if (baseline) {
                const float s0 = (float)S[p], c0 = (float)C[p];
                baseline[p] = sqrtf(s0 * s0 + c0 * c0) * scale;
            }
        }
    }
}

__global__ void pack_input_kernel(const int32_t* __restrict__ S, const int32_t* __restrict__ C, long long n,
                                  float scale, __nv_bfloat16* __restrict__ out, float* __restrict__ baseline) {
    // a first convolution launched early (qldnn_conv3x3_fwd_tma_epi) may set
    // itself up now; it waits for this kernel before it reads the packed input
    asm volatile("griddepcontrol.launch_dependents;" :::);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float s = (float)S[i], c = (float)C[i];
        const float r = sqrtf(s * s + c * c) * scale;
        if (baseline) baseline[i] = r;
        float f[8] = {s * scale, c * scale, r, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint4* o = reinterpret_cast<uint4*>(out + i * 16);  // 16 channels: S, C, R, then zeros
        o[0] = pack8(f);
        o[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 148ll * 32) b = 148ll * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

namespace {
template <int N, int BK>
int launch_tc2(const __nv_bfloat16* x, const __nv_bfloat16* k, const float* bias, int B, int H, int W, int Cin,
               int Cout, int relu, __nv_bfloat16* ob, float* of, int* status, cudaStream_t st) {
    constexpr int STAGES = 4;
    const int smem = qldnn::TcPipe<N, BK, STAGES>::kSmem;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        if (cudaFuncSetAttribute(qldnn::conv3x3_fwd_tc2_kernel<N, BK, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem) != cudaSuccess)
            return set_err(QLD_E_CUDA);
        attr_set = true;
    }
    const long long P = (long long)B * H * W;
    qldnn::conv3x3_fwd_tc2_kernel<N, BK, STAGES><<<nblk(P, 128), 160, smem, st>>>(x, k, bias, B, H, W, Cin, Cout, relu, ob,
                                                                                 of, status);
    return launched(1);
}
}  // namespace

namespace {
// cuTensorMapEncodeTiled, fetched once from the driver through the runtime
// (no link-time dependency on the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

int sm_count(int dev) {
    static std::atomic<int> cache[64];
    if (dev < 0 || dev >= 64) return 0;
    int n = cache[dev].load();
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev].store(n);
    }
    return n;
}

// Launch of `kernel` on `st`; with `early`, with programmatic stream
// serialisation (the kernel may start before the previous one on the stream
// has finished, and waits for it with griddepcontrol.wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_early(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                               bool early, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = early ? attr : nullptr;
    cfg.numAttrs = early ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int N, int SWB, int SUB = 1, int MINB = 1, bool XS = false>
int launch_tma(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout, int relu,
               const qldnn::ConvEpi& epi, int* status, cudaStream_t st, bool force_stream, bool early,
               bool wide_epi = false) {
    using L = qldnn::TmaConv<N, SWB>;
    EncodeTiledFn enc = encode_tiled();
    int dev = 0;
    if (!enc || cudaGetDevice(&dev) != cudaSuccess) return set_err(QLD_E_CUDA);
    const int nsm = sm_count(dev);
    if (nsm <= 0) return set_err(QLD_E_CUDA);
    const CUtensorMapSwizzle sw =
        SWB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : (SWB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    CUtensorMap mi, mw;
    const cuuint64_t gdim[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t gstr[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
    const cuuint32_t box[4] = {(cuuint32_t)L::BK, 16, (cuuint32_t)(8 * SUB + 2), 1};  // a tile's halo rows
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (enc(&mi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(in), gdim, gstr, box, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_err(QLD_E_CUDA);
    const cuuint64_t wdim[2] = {(cuuint64_t)Cin, (cuuint64_t)9 * Cout};
    const cuuint64_t wstr[1] = {(cuuint64_t)Cin * 2};
    const cuuint32_t wbox[2] = {(cuuint32_t)L::BK, (cuuint32_t)N};
    if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(wk), wdim, wstr, wbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_err(QLD_E_CUDA);
    using R = qldnn::TmaConvRes<N, SWB, SUB, XS>;
    const long long ntiles = (long long)B * ((H + 8 * SUB - 1) / (8 * SUB)) * ((W + R::TW - 1) / R::TW);
    const int nsplit = Cout / N;  // CTAs per tile, one output-channel slice each
    long long items = ntiles * nsplit;
    const long long cap = (long long)(MINB * nsm / nsplit) * nsplit;
    const unsigned grid = (unsigned)(items < cap ? items : cap);
    // weights resident in shared memory when they fit beside two or more halo
    // stages (within half of it for two CTAs per SM)
    const long long smem_cap = MINB == 2 ? qldnn::kTwoPerSmSmem : 232448;
    int sa = 0;
    while (sa < R::kMaxSA && R::smem(sa + 1, Cin) <= smem_cap) ++sa;
    if (sa >= 2 && !force_stream) {
        static std::atomic<unsigned long long> attr_res{0};
        if (dev < 64 && !(attr_res.load() >> dev & 1ull)) {
            if (cudaFuncSetAttribute(qldnn::conv3x3_fwd_tma_wres_kernel<N, SWB, SUB, MINB, XS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap) != cudaSuccess)
                return set_err(QLD_E_CUDA);
            attr_res.fetch_or(1ull << dev);
        }
        if (launch_maybe_early(qldnn::conv3x3_fwd_tma_wres_kernel<N, SWB, SUB, MINB, XS>, grid, qldnn::kConvThreads,
                               (size_t)R::smem(sa, Cin),
                               st, early, mi, mw, bias, B, H, W, Cin, Cout, relu, epi, status, sa,
                               nsplit) != cudaSuccess)
            return set_err(QLD_E_CUDA);
        return launched(1);
    }
    // the weight-streaming kernel: 8 x 16 tiles, unstacked taps
    if constexpr (SUB != 1 || MINB != 1 || XS) return set_err(QLD_E_INVAL);
    if constexpr (N >= 64) {
        if (wide_epi) {  // eight epilogue warps, two per TMEM lane quarter
            static std::atomic<unsigned long long> attr8{0};
            if (dev < 64 && !(attr8.load() >> dev & 1ull)) {
                if (cudaFuncSetAttribute(qldnn::conv3x3_fwd_tma_kernel<N, SWB, 8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmem) != cudaSuccess)
                    return set_err(QLD_E_CUDA);
                attr8.fetch_or(1ull << dev);
            }
            if (launch_maybe_early(qldnn::conv3x3_fwd_tma_kernel<N, SWB, 8>, grid, 64 + 32 * 8, (size_t)L::kSmem, st,
                                   early, mi, mw, bias, B, H, W, Cin, Cout, relu, epi, status, nsplit) != cudaSuccess)
                return set_err(QLD_E_CUDA);
            return launched(1);
        }
    }
    static std::atomic<unsigned long long> attr_done{0};  // per instantiation, one bit per device
    if (dev < 64 && !(attr_done.load() >> dev & 1ull)) {
        if (cudaFuncSetAttribute(qldnn::conv3x3_fwd_tma_kernel<N, SWB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 L::kSmem) != cudaSuccess)
            return set_err(QLD_E_CUDA);
        attr_done.fetch_or(1ull << dev);
    }
    if (launch_maybe_early(qldnn::conv3x3_fwd_tma_kernel<N, SWB>, grid, qldnn::kConvThreads, (size_t)L::kSmem, st,
                           early, mi, mw,
                           bias, B, H, W, Cin, Cout, relu, epi, status, nsplit) != cudaSuccess)
        return set_err(QLD_E_CUDA);
    return launched(1);
}

template <int N, int SWA, bool STACK>
int launch_wgrad_tma(const void* in, const void* g, int B, int H, int W, int Cin, int Cout, float* dw, int* status,
                     cudaStream_t st) {
    using L = qldnn::WgradTma<N, SWA, STACK>;
    EncodeTiledFn enc = encode_tiled();
    int dev = 0;
    if (!enc || cudaGetDevice(&dev) != cudaSuccess) return set_err(QLD_E_CUDA);
    const int nsm = sm_count(dev);
    if (nsm <= 0) return set_err(QLD_E_CUDA);
    auto swz = [](int sw) {
        return sw == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : (sw == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    };
    const cuuint32_t one[4] = {1, 1, 1, 1};
    CUtensorMap mi, mg;
    const cuuint64_t idim[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t istr[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
    const cuuint32_t ibox[4] = {(cuuint32_t)L::EA, 16, 10, 1};
    if (enc(&mi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(in), idim, istr, ibox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz(SWA), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_err(QLD_E_CUDA);
    const cuuint64_t gdim[4] = {(cuuint64_t)Cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t gstr[3] = {(cuuint64_t)Cout * 2, (cuuint64_t)W * Cout * 2, (cuuint64_t)H * W * Cout * 2};
    const cuuint32_t gbox[4] = {(cuuint32_t)L::EB, 16, 8, 1};
    if (enc(&mg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(g), gdim, gstr, gbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz(L::SWBB), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_err(QLD_E_CUDA);
    static std::atomic<unsigned long long> attr_done{0};
    if (dev < 64 && !(attr_done.load() >> dev & 1ull)) {
        if (cudaFuncSetAttribute(qldnn::conv3x3_wgrad_tma_kernel<N, SWA, STACK>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmem) != cudaSuccess)
            return set_err(QLD_E_CUDA);
        attr_done.fetch_or(1ull << dev);
    }
    const long long ntiles = (long long)B * ((H + 7) / 8) * ((W + 15) / 16);
    const int ncb = STACK ? 1 : Cin / 128;
    // one wave: about one work item per SM, each a contiguous range of tiles
    long long nsplit = nsm / (3 * ncb);
    if (nsplit < 1) nsplit = 1;
    if (nsplit > ntiles) nsplit = ntiles;
    qldnn::conv3x3_wgrad_tma_kernel<N, SWA, STACK><<<(unsigned)(3 * ncb * nsplit), 192, L::kSmem, st>>>(
        mi, mg, B, H, W, Cin, Cout, (int)nsplit, dw, status);
    return launched(1);
}

// Chooses the variant (weights resident or streamed, CTAs per tile) and the
// template instance of the persistent TMA convolution; mode as in
// qldnn_conv3x3_fwd_tma_mode.
int conv_tma_dispatch(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout,
                      int relu, const qldnn::ConvEpi& epi, int* status, int mode, cudaStream_t st) {
    const int force_stream = mode & 1;
    const int split_mode = (mode >> 4) & 0xF;
    const bool early = ((mode >> 8) & 1) != 0;
    if (split_mode != 0 && split_mode != 1 && split_mode != 2 && split_mode != 4) return set_err(QLD_E_INVAL);
    if (!in || !wk || B < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 ||
        (Cout != 32 && Cout != 64 && Cout != 128 && Cout != 256) || !al(in, 16) || !al(wk, 16) ||
        (long long)B * H * W * Cin >= (1ll << 40))
        return set_err(QLD_E_INVAL);
    const int swb = Cin % 64 == 0 ? 128 : (Cin % 32 == 0 ? 64 : 32);
    // fewer tiles than SMs: split each tile's output channels over 2 or 4 CTAs
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        const int n = sm_count(dev);
        if (n > 0) nsm = n;
    }
    const long long ntiles = (long long)B * ((H + 7) / 8) * ((W + 15) / 16);
    // split only into slices whose weights stay resident: a streamed slice
    // reloads the whole input halo per CTA and runs narrower MMAs (slower)
    auto resident = [&](int nco) {
        const long long halo3 = 3ll * 160 * swb;
        return 1024 + 2 * halo3 + 9ll * Cin * nco * 2 + 256 <= 232448;
    };
    // and only when at most half the SMs would otherwise get a tile: with
    // more, the narrower MMAs and repeated halo loads cost more than it gains
    int nsplit = 1;
    for (int cand = 2; cand <= 4 && 2 * ntiles <= nsm && ntiles * nsplit < nsm; cand *= 2)
        if (Cout / cand >= 32 && resident(Cout / cand)) nsplit = cand;
    // 128-column layers of at most 128 input channels with at most one tile
    // per SM: two CTAs per tile (four when even that leaves 4 tiles per SM
    // free), measured faster whether or not the 64-column slices' weights
    // stay resident (128^2 at batch 1: 64 -> 128 8.95 -> 6.7 us, 128 -> 128
    // 10.5 -> 9.7 us; 8 x 32^2, 128 -> 128 8.5 -> 7.3 us with two instead of
    // four); layers of 256 input channels measured slower split
    if (Cout == 128 && Cin <= 128 && ntiles <= nsm) nsplit = 4 * ntiles <= nsm ? 4 : 2;
    // 64-column layers of 128+ input channels with at most one tile per SM:
    // two 32-column slices, which then stack their column taps (128^2,
    // 128 -> 64 with its fused 2x upsampling 7.8 -> 7.4 us; 8.3 us split
    // without the stacking)
    if (Cout == 64 && Cin >= 128 && ntiles <= nsm) nsplit = 2;
    if (split_mode > 0) nsplit = split_mode;
    if (Cout % nsplit || Cout / nsplit < 32) return set_err(QLD_E_INVAL);
    const int nco = Cout / nsplit;
    // 16 x 16-pixel tiles (two stacked 8 x 16 sub-tiles per pipeline step) for
    // narrow layers with weights resident beside two 18-row halo stages of at
    // most 32 channels, when there are at least two such tiles per SM (mode
    // bit 12 forces them where they apply, bit 13 forbids them). Automatic
    // only for inputs staged in chunks of at most 32 channels anyway: layers
    // of 64+ channels would have to drop from 64- to 32-channel chunks, and
    // measured slower that way (8 x 128^2, 64 -> 64: 554 against 588 TFLOP/s)
    const int swb2 = swb > 64 ? 64 : swb;
    const long long tiles16 = (long long)B * ((H + 15) / 16) * ((W + 15) / 16);
    const bool fits2 = 1024 + 2ll * 3 * 18 * 16 * swb2 + 9ll * Cin * nco * 2 + 256 <= 232448;
    const bool sub2 = nsplit == 1 && nco <= 64 && !force_stream && !((mode >> 13) & 1) && fits2 &&
                      (((mode >> 12) & 1) || (tiles16 >= 2ll * nsm && swb2 == swb));
    // two CTAs per SM for 32- and 64-channel layers (every CTA's MMA thread leaves
    // gaps in the tensor-core queue that the other fills) when the weights and
    // two halo stages fit in half the shared memory, staged in chunks of at
    // most 32 channels, with 16 x 16 tiles if those fit too; by default for
    // 32-column layers whose CTAs get at least two 8 x 16 tiles (mode bit 15
    // forces it where it fits, 64-column layers included; bit 14 forbids it).
    // Measured against one CTA per SM in one process: 512^2 64 -> 32 channels
    // 21.7 -> 18.6 us, 32 -> 32 13.7 -> 13.2 us, and, since the wide bias
    // loads and 32-byte stores of the epilogue, the 16-channel first layer
    // too (10.9 -> 9.7 us; 12.0 -> 12.4 us before those); slower for 256^2,
    // 32 -> 64 (8.7 -> 11.4 us).
    // A second MMA-issuing thread in one CTA, taking every other tile,
    // measured no faster on any layer: the gain is not the second issuer.
    auto fits_two = [&](int sub) {
        return 1024 + 2ll * 3 * (8 * sub + 2) * 16 * swb2 + 9ll * Cin * nco * 2 + 256 <= qldnn::kTwoPerSmSmem;
    };
    const long long tiles8 = ntiles;
    // column taps stacked in N (conv3x3_fwd_tma_wres_kernel<..., XS = true>,
    // 14-column tiles, one unshifted halo copy per channel chunk) for 32- and
    // 64-column slices: mode bit 16 asks for it, bit 17 forbids it. Bits 12-15
    // choose its tile height and CTAs per SM as for the unstacked kernel; two
    // CTAs per SM and 16-row tiles exclude each other (the accumulators of
    // 3 x 32 columns, two per CTA, take the tensor memory). By default where
    // the MMAs outweigh its longer epilogue (three column groups read, two
    // shuffles per channel): 32-column layers of at least 64 input channels
    // with at least eight of its tiles per SM, 64-column ones of at least 128
    // with at least two (measured, graphs of 20 launches: 512^2, 64 -> 32
    // 18.6 -> 13.6 us; 256^2, 128 -> 64 15.7 -> 12.8 us; slower: 512^2,
    // 16 -> 32 12.0 -> 12.6 us; 256^2, 64 -> 64 9.6 -> 11.6 us; 128^2,
    // 128 -> 64 (160 stacked tiles for 148 SMs) 7.3 -> 8.1 us; 256^2, 64 -> 32
    // (4 tiles per SM) 9.0 -> 6.8 us alone but 12.1 -> 13.0 us with the fused
    // 2x upsampling of the inference network, whose stores dominate). The
    // choice depends on the shape alone, so a layer gives the same result
    // with fused and with separate outputs.
    auto fits_xs = [&](int sub, int sw, long long cap) {  // resident weights and two halo stages
        return 1024 + 2ll * (8 * sub + 2) * 16 * sw + 9ll * Cin * nco * 2 + 256 <= cap;
    };
    const long long tx14 = (W + 13) / 14;
    const long long xt8 = (long long)B * ((H + 7) / 8) * tx14, xt16 = (long long)B * ((H + 15) / 16) * tx14;
    // (and 32-column slices of 128+ input channels at any tile count: 64^2,
    // 128 -> 128 in four slices 5.4 -> 4.6 us, with its fused upsampling 6.1 ->
    // 5.65 us)
    const bool xs_auto = (nco == 32 && Cin >= 64 && xt8 * nsplit >= 8ll * nsm) || (nco == 32 && Cin >= 128) ||
                         (nco == 64 && Cin >= 128 && xt8 * nsplit >= 2ll * nsm);
    const bool xs = (nco == 32 || nco == 64) && !force_stream && !((mode >> 17) & 1) && fits_xs(1, swb2, 232448) &&
                    (((mode >> 16) & 1) || xs_auto);
    if (xs) {
        const int sw = fits_xs(1, swb, 232448) ? swb : swb2;
        const bool xtwo = nco == 32 && !((mode >> 14) & 1) && fits_xs(1, sw, qldnn::kTwoPerSmSmem) &&
                          (((mode >> 15) & 1) || (Cin >= 32 && xt8 >= 4ll * nsm));
        const bool xsub2 = nco == 32 && !xtwo && !((mode >> 13) & 1) && fits_xs(2, sw, 232448) &&
                           (((mode >> 12) & 1) || xt16 >= 2ll * nsm);
#define QLD_XS(SS)                                                                                                  \
    if (sw == SS) {                                                                                                 \
        if (nco == 64)                                                                                              \
            return launch_tma<64, SS, 1, 1, true>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false,   \
                                                  early);                                                           \
        if (xtwo)                                                                                                   \
            return launch_tma<32, SS, 1, 2, true>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false,   \
                                                  early);                                                           \
        if (xsub2)                                                                                                  \
            return launch_tma<32, SS, 2, 1, true>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false,   \
                                                  early);                                                           \
        return launch_tma<32, SS, 1, 1, true>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false,       \
                                              early);                                                               \
    }
        QLD_XS(32) QLD_XS(64) QLD_XS(128)
#undef QLD_XS
        return set_err(QLD_E_INVAL);
    }
    const bool two = nsplit == 1 && (nco == 32 || nco == 64) && !force_stream && !((mode >> 14) & 1) && fits_two(1) &&
                     (((mode >> 15) & 1) || (nco == 32 && tiles8 >= 4ll * nsm));
    if (two && nco == 64)  // 8 x 16 tiles only: 16 x 16 ones do not fit twice with 64-column weights
        return swb2 == 32 ? launch_tma<64, 32, 1, 2>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false, early)
                          : launch_tma<64, 64, 1, 2>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false, early);
    if (two) {
        const bool two_sub2 = !((mode >> 13) & 1) && fits_two(2) && (((mode >> 12) & 1) || tiles16 >= 4ll * nsm);
        if (swb2 == 32)
            return two_sub2 ? launch_tma<32, 32, 2, 2>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false, early)
                            : launch_tma<32, 32, 1, 2>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false, early);
        return two_sub2 ? launch_tma<32, 64, 2, 2>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false, early)
                        : launch_tma<32, 64, 1, 2>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false, early);
    }
#define QLD_TMA2(NN, SS)                                                                                            \
    if (sub2 && nco == NN && swb2 == SS)                                                                               \
        return launch_tma<NN, SS, 2>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, false, early);
    QLD_TMA2(32, 32) QLD_TMA2(32, 64) QLD_TMA2(64, 32) QLD_TMA2(64, 64)
#undef QLD_TMA2
    // weight-streaming layers of 64+ columns without a head: eight epilogue
    // warps, two per accumulator lane quarter, each reading half the columns
    // (mode bit 19 forbids them; bit 18 is the default here). Measured, graphs
    // of 20 launches, four against eight warps: 8 x 64^2, 64 -> 128 12.8 ->
    // 10.0 us, 128 -> 128 14.9 -> 13.05 us, 256 -> 128 20.9 -> 20.2 us;
    // 128^2, 256 -> 128 14.1 -> 12.7 us; no shape slower. Their read-out, one
    // warp per lane quarter, had been the last tile's tail (cycle stamps: 7,000
    // cycles for a 128-column tile after its last MMA). The weights-resident
    // kernel's 64- and 128-column layers measured no faster with eight
    // (256^2, 64 -> 64 9.7 -> 10.2 us; 8 x 128^2, 64 -> 64 13.9 -> 14.3 us).
    const bool wide_epi = nco >= 64 && !epi.head_w && !((mode >> 19) & 1);
#define QLD_TMA(NN, SS) \
    if (nco == NN && swb == SS)                                                                                      \
        return launch_tma<NN, SS>(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, st, force_stream != 0, early, \
                                  wide_epi);
    QLD_TMA(32, 32) QLD_TMA(32, 64) QLD_TMA(32, 128)
    QLD_TMA(64, 32) QLD_TMA(64, 64) QLD_TMA(64, 128)
    QLD_TMA(128, 32) QLD_TMA(128, 64) QLD_TMA(128, 128)
    QLD_TMA(256, 32) QLD_TMA(256, 64) QLD_TMA(256, 128)
#undef QLD_TMA
    return set_err(QLD_E_INVAL);
}
}  // namespace

extern "C" {

int qldnn_conv3x3_fwd(const void* in, const void* w, const float* bias, int B, int H, int W, int Cin, int Cout,
                      int relu, void* out_bf16, float* out_f32, void* stream) {
    if (!in || !w || (!out_bf16 && !out_f32) || B < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 32 ||
        Cout % 32 || !al(in, 16) || !al(w, 16) || !al(out_bf16, 4) || !al(out_f32, 8))
        return set_err(QLD_E_INVAL);
    const long long P = (long long)B * H * W;
    const cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16* x = (const __nv_bfloat16*)in;
    const __nv_bfloat16* k = (const __nv_bfloat16*)w;
    if (Cout % 64 == 0)
        qldnn::conv3x3_fwd_kernel<64><<<dim3(nblk(P, 128), Cout / 64), 128, 0, st>>>(
            x, k, bias, B, H, W, Cin, Cout, relu, (__nv_bfloat16*)out_bf16, out_f32);
    else
        qldnn::conv3x3_fwd_kernel<32><<<dim3(nblk(P, 128), Cout / 32), 128, 0, st>>>(
            x, k, bias, B, H, W, Cin, Cout, relu, (__nv_bfloat16*)out_bf16, out_f32);
    return launched(1);
}

int qldnn_conv3x3_wgrad(const void* in, const void* g, int B, int H, int W, int Cin, int Cout, float* dw,
                        void* stream) {
    if (!in || !g || !dw || B < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 32 || Cout % 32 ||
        !al(in, 16) || !al(g, 16))
        return set_err(QLD_E_INVAL);
    const long long P = (long long)B * H * W;
    const cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16* x = (const __nv_bfloat16*)in;
    const __nv_bfloat16* y = (const __nv_bfloat16*)g;
    const int MT = Cin % 32 == 0 ? 2 : 1;
    const int BN = Cout % 64 == 0 ? 64 : 32;
    const int tiles = (Cin / (16 * MT)) * (Cout / BN);
    // pixel chunk per CTA: enough CTAs to fill the GPU twice over
    long long chunk = (P * 9 * tiles) / (148ll * 8);
    chunk = chunk < 256 ? 256 : (chunk > 16384 ? 16384 : chunk);
    chunk = (chunk + 63) / 64 * 64;
    const dim3 grid(nblk(P, (int)chunk), 9, tiles);
    if (MT == 2 && BN == 64) qldnn::conv3x3_wgrad_kernel<2, 64><<<grid, 128, 0, st>>>(x, y, B, H, W, Cin, Cout, (int)chunk, dw);
    else if (MT == 2) qldnn::conv3x3_wgrad_kernel<2, 32><<<grid, 128, 0, st>>>(x, y, B, H, W, Cin, Cout, (int)chunk, dw);
    else if (BN == 64) qldnn::conv3x3_wgrad_kernel<1, 64><<<grid, 128, 0, st>>>(x, y, B, H, W, Cin, Cout, (int)chunk, dw);
    else qldnn::conv3x3_wgrad_kernel<1, 32><<<grid, 128, 0, st>>>(x, y, B, H, W, Cin, Cout, (int)chunk, dw);
    return launched(1);
}

int qldnn_conv3x3_dgrad(const void* g, const void* w, int B, int H, int W, int Cin, int Cout, void* wt_scratch,
                        void* din_bf16, float* din_f32, void* stream) {
    // the layer maps Cin -> Cout; its data gradient maps Cout -> Cin
    if (!g || !w || !wt_scratch || Cout % 16 || Cin % 32 || Cin < 32) return set_err(QLD_E_INVAL);
    const cudaStream_t st = (cudaStream_t)stream;
    const long long n = 9ll * Cin * Cout;
    flip_transpose_kernel<<<grid_for(n), 256, 0, st>>>((const __nv_bfloat16*)w, Cin, Cout,
                                                        (__nv_bfloat16*)wt_scratch);
    if (launched(1) != QLD_OK) return QLD_E_CUDA;
    return qldnn_conv3x3_fwd(g, wt_scratch, nullptr, B, H, W, Cout, Cin, 0, din_bf16, din_f32, stream);
}

int qldnn_bias_grad(const void* g, long long P, int C, float* db, void* stream) {
    if (!g || !db || C < 1 || C > 256) return set_err(QLD_E_INVAL);
    if (C % 8 == 0 && al(g, 16)) {
        const long long rows_per_block = 256 / (C / 8);
        long long nb = (P + rows_per_block - 1) / rows_per_block;
        if (nb > 296) nb = 296;
        if (nb < 1) nb = 1;
        bias_grad_v8_kernel<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>((const uint4*)g, P, C, db);
    } else {
        bias_grad_kernel<<<grid_for(P / (256 / C) + 1), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)g, P,
                                                                                        C, db);
    }
    return launched(1);
}

int qldnn_relu_bwd(const float* g, const void* act, long long n, void* out_bf16, void* stream) {
    if (!g || !act || !out_bf16 || n < 0) return set_err(QLD_E_INVAL);
    if (n % 4 == 0 && al(g, 16) && al(act, 8) && al(out_bf16, 8))
        relu_bwd_v4_kernel<<<grid_for(n / 4), 256, 0, (cudaStream_t)stream>>>((const float4*)g, (const uint2*)act,
                                                                               n / 4, (uint2*)out_bf16);
    else
        relu_bwd_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(g, (const __nv_bfloat16*)act, n,
                                                                         (__nv_bfloat16*)out_bf16);
    return launched(1);
}

int qldnn_relu_bwd_bias(const float* g, const void* act, long long P, int C, void* out_bf16, float* db,
                        void* stream) {
    if (!g || !act || !out_bf16 || !db || P < 0 || C < 8 || C > 256 || C % 8 || !al(g, 16) || !al(act, 16) ||
        !al(out_bf16, 16))
        return set_err(QLD_E_INVAL);
    const long long rows_per_block = 256 / (C / 8);
    long long nb = (P + rows_per_block - 1) / rows_per_block;
    if (nb > 296) nb = 296;
    if (nb < 1) nb = 1;
    relu_bwd_bias_v8_kernel<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>((const float4*)g, (const uint4*)act, P, C,
                                                                             (uint4*)out_bf16, db);
    return launched(1);
}

int qldnn_avgpool2(const void* in, int B, int H, int W, int C, void* out, void* stream) {
    if (!in || !out || H % 2 || W % 2) return set_err(QLD_E_INVAL);
    if (C % 8 == 0 && al(in, 16) && al(out, 16))
        avgpool2_fwd_v8_kernel<<<grid_for((long long)B * H * W * C / 32), 256, 0, (cudaStream_t)stream>>>(
            (const uint4*)in, B, H, W, C / 8, (uint4*)out);
    else
        avgpool2_fwd_kernel<<<grid_for((long long)B * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>(
            (const __nv_bfloat16*)in, B, H, W, C, (__nv_bfloat16*)out);
    return launched(1);
}

int qldnn_avgpool2_bwd(const float* g, int B, int H, int W, int C, float* out, int accumulate, void* stream) {
    if (!g || !out || H % 2 || W % 2) return set_err(QLD_E_INVAL);
    if (C % 4 == 0 && al(g, 16) && al(out, 16))
        avgpool2_bwd_v4_kernel<<<grid_for((long long)B * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>(
            (const float4*)g, B, H, W, C / 4, (float4*)out, accumulate);
    else
        avgpool2_bwd_kernel<<<grid_for((long long)B * H * W * C), 256, 0, (cudaStream_t)stream>>>(g, B, H, W, C, out,
                                                                                                   accumulate);
    return launched(1);
}

int qldnn_upsample2(const void* in, int B, int h, int w, int C, void* out, void* stream) {
    if (!in || !out) return set_err(QLD_E_INVAL);
    if (C % 8 == 0 && al(in, 16) && al(out, 16))
        upsample2_fwd_v8_kernel<<<grid_for(4ll * B * h * w * C / 8), 256, 0, (cudaStream_t)stream>>>(
            (const uint4*)in, B, h, w, C / 8, (uint4*)out);
    else
        upsample2_fwd_kernel<<<grid_for(4ll * B * h * w * C), 256, 0, (cudaStream_t)stream>>>(
            (const __nv_bfloat16*)in, B, h, w, C, (__nv_bfloat16*)out);
    return launched(1);
}

int qldnn_upsample2_bwd(const float* g, int B, int h, int w, int C, float* out, void* stream) {
    if (!g || !out) return set_err(QLD_E_INVAL);
    if (C % 4 == 0 && al(g, 16) && al(out, 16))
        upsample2_bwd_v4_kernel<<<grid_for((long long)B * h * w * C / 4), 256, 0, (cudaStream_t)stream>>>(
            (const float4*)g, B, h, w, C / 4, (float4*)out);
    else
        upsample2_bwd_kernel<<<grid_for((long long)B * h * w * C), 256, 0, (cudaStream_t)stream>>>(g, B, h, w, C, out);
    return launched(1);
}

int qldnn_concat(const void* a, int Ca, const void* b, int Cb, long long P, void* out, void* stream) {
    if (!a || !b || !out) return set_err(QLD_E_INVAL);
    if (Ca % 8 == 0 && Cb % 8 == 0 && al(a, 16) && al(b, 16) && al(out, 16))
        concat_v8_kernel<<<grid_for(P * (Ca + Cb) / 8), 256, 0, (cudaStream_t)stream>>>(
            (const uint4*)a, Ca / 8, (const uint4*)b, Cb / 8, P, (uint4*)out);
    else
        concat_kernel<<<grid_for(P * (Ca + Cb)), 256, 0, (cudaStream_t)stream>>>(
            (const __nv_bfloat16*)a, Ca, (const __nv_bfloat16*)b, Cb, P, (__nv_bfloat16*)out);
    return launched(1);
}

int qldnn_upsample_concat(const void* u, int Cu, const void* e, int Ce, int B, int h, int w, void* out, void* stream) {
    if (!u || !e || !out || B < 1 || h < 1 || w < 1 || Cu < 8 || Ce < 8 || Cu % 8 || Ce % 8 || !al(u, 16) ||
        !al(e, 16) || !al(out, 16))
        return set_err(QLD_E_INVAL);
    upsample_concat_v8_kernel<<<grid_for(4ll * B * h * w * (Cu + Ce) / 8), 256, 0, (cudaStream_t)stream>>>(
        (const uint4*)u, Cu / 8, (const uint4*)e, Ce / 8, B, h, w, (uint4*)out);
    return launched(1);
}

int qldnn_split(const float* g, long long P, int Ca, int Cb, float* ga, float* gb, int accumulate_b, void* stream) {
    if (!g || !ga || !gb) return set_err(QLD_E_INVAL);
    if (Ca % 4 == 0 && Cb % 4 == 0 && al(g, 16) && al(ga, 16) && al(gb, 16))
        split_v4_kernel<<<grid_for(P * (Ca + Cb) / 4), 256, 0, (cudaStream_t)stream>>>(
            (const float4*)g, P, Ca / 4, Cb / 4, (float4*)ga, (float4*)gb, accumulate_b);
    else
        split_kernel<<<grid_for(P * (Ca + Cb)), 256, 0, (cudaStream_t)stream>>>(g, P, Ca, Cb, ga, gb, accumulate_b);
    return launched(1);
}

int qldnn_head(const void* in, const float* w, const float* b, long long P, int C, float* out, void* stream) {
    if (!in || !w || !b || !out || C > 256) return set_err(QLD_E_INVAL);
    if (C % 8 == 0 && al(in, 16))
        head_fwd_v8_kernel<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>((const uint4*)in, w, b, P, C / 8, out);
    else
        head_fwd_kernel<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)in, w, b, P, C, out);
    return launched(1);
}

int qldnn_head_bwd(const void* in, const float* g, const float* w, long long P, int C, float* din, float* dw,
                   float* db, void* stream) {
    if (!in || !g || !w || !din || !dw || !db || C > 256) return set_err(QLD_E_INVAL);
    const bool v8 = al(in, 16) && al(din, 16);
    long long nb = (P + 255) / 256;
    if (nb > 296) nb = 296;
    if (nb < 1) nb = 1;
    if (v8 && C == 32)
        head_bwd_v8_kernel<32><<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>((const uint4*)in, g, w, P, (float4*)din,
                                                                               dw, db);
    else if (v8 && C == 16)
        head_bwd_v8_kernel<16><<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>((const uint4*)in, g, w, P, (float4*)din,
                                                                               dw, db);
    else
        head_bwd_kernel<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)in, g, w, P, C, din, dw,
                                                                      db);
    return launched(1);
}

int qldnn_mse(const float* pred, const float* target, long long n, float* grad, float* loss, void* stream) {
    if (!pred || !target || !grad || !loss || n < 1) return set_err(QLD_E_INVAL);
    mse_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(pred, target, n, grad, loss);
    return launched(1);
}

int qldnn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
               int t, void* p_bf16, void* stream) {
    if (!p || !g || !m || !v || n < 0 || t < 1) return set_err(QLD_E_INVAL);
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2,
                                                                (__nv_bfloat16*)p_bf16);
    return launched(1);
}

int qldnn_cast_bf16(const float* x, long long n, void* y, void* stream) {
    if (!x || !y || n < 0) return set_err(QLD_E_INVAL);
    cast_bf16_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, n, (__nv_bfloat16*)y);
    return launched(1);
}

int qldnn_add(float* y, const float* x, long long n, void* stream) {
    if (!x || !y || n < 0) return set_err(QLD_E_INVAL);
    add_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(y, x, n);
    return launched(1);
}

int qldnn_pack_input(const int32_t* S, const int32_t* C, long long npix, float scale, void* out, float* baseline,
                     void* stream) {
    if (!S || !C || !out || npix < 0 || !al(out, 16)) return set_err(QLD_E_INVAL);
    pack_input_kernel<<<grid_for(npix), 256, 0, (cudaStream_t)stream>>>(S, C, npix, scale, (__nv_bfloat16*)out,
                                                                         baseline);
    return launched(1);
}

int qldnn_input_conv3x3(const int32_t* S, const int32_t* C, int B, int H, int W, float scale, const void* w,
                        int Cin, int Cout, const float* bias, int relu, void* out_bf16, long long ldo, float* baseline,
                        void* stream) {
    if (!S || !C || !w || !out_bf16 || B < 1 || H < 1 || W < 1 || Cin < 3 || (Cout != 32 && Cout != 64) ||
        ldo < Cout || ldo % 8 || !al(out_bf16, 16) || !al(baseline, 4))
        return set_err(QLD_E_INVAL);
    const long long tiles = (long long)B * ((H + 15) / 16) * ((W + 15) / 16);
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess && sm_count(dev) > 0) nsm = sm_count(dev);
    const long long grid = tiles < 4ll * nsm ? tiles : 4ll * nsm;  // persistent: 4 CTAs per SM
    const cudaStream_t st = (cudaStream_t)stream;
    if (Cout == 32)
        input_conv3x3_kernel<32><<<(unsigned)grid, 128, 0, st>>>(S, C, B, H, W, scale, (const __nv_bfloat16*)w, Cin,
                                                                  bias, relu, (__nv_bfloat16*)out_bf16, ldo, baseline);
    else
        input_conv3x3_kernel<64><<<(unsigned)grid, 128, 0, st>>>(S, C, B, H, W, scale, (const __nv_bfloat16*)w, Cin,
                                                                  bias, relu, (__nv_bfloat16*)out_bf16, ldo, baseline);
    return launched(1);
}

int qldnn_kmajor_weights(const void* w, int Cin, int Cout, int flip, void* wk, void* stream) {
    if (!w || !wk || Cin < 1 || Cout < 1) return set_err(QLD_E_INVAL);
    qldnn::kmajor_weights_kernel<<<grid_for(9ll * Cin * Cout), 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)w, Cin, Cout, flip, (__nv_bfloat16*)wk);
    return launched(1);
}

int qldnn_conv3x3_fwd_tc(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout,
                         int relu, void* out_bf16, float* out_f32, int* status, void* stream) {
    if (!in || !wk || (!out_bf16 && !out_f32) || B < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 32 ||
        Cout % 32 || !al(in, 16) || !al(wk, 16) || !al(out_bf16, 16) || !al(out_f32, 16))
        return set_err(QLD_E_INVAL);
    const long long P = (long long)B * H * W;
    const cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16* x = (const __nv_bfloat16*)in;
    const __nv_bfloat16* k = (const __nv_bfloat16*)wk;
    __nv_bfloat16* ob = (__nv_bfloat16*)out_bf16;
    const unsigned gx = nblk(P, 128);
    const bool bk32 = Cin % 32 == 0;
    if (Cout % 128 == 0) {
        if (bk32) qldnn::conv3x3_fwd_tc_kernel<128, 32><<<dim3(gx, Cout / 128), 128, 0, st>>>(x, k, bias, B, H, W, Cin, Cout, relu, ob, out_f32, status);
        else qldnn::conv3x3_fwd_tc_kernel<128, 16><<<dim3(gx, Cout / 128), 128, 0, st>>>(x, k, bias, B, H, W, Cin, Cout, relu, ob, out_f32, status);
    } else if (Cout % 64 == 0) {
        if (bk32) qldnn::conv3x3_fwd_tc_kernel<64, 32><<<dim3(gx, Cout / 64), 128, 0, st>>>(x, k, bias, B, H, W, Cin, Cout, relu, ob, out_f32, status);
        else qldnn::conv3x3_fwd_tc_kernel<64, 16><<<dim3(gx, Cout / 64), 128, 0, st>>>(x, k, bias, B, H, W, Cin, Cout, relu, ob, out_f32, status);
    } else {
        if (bk32) qldnn::conv3x3_fwd_tc_kernel<32, 32><<<dim3(gx, Cout / 32), 128, 0, st>>>(x, k, bias, B, H, W, Cin, Cout, relu, ob, out_f32, status);
        else qldnn::conv3x3_fwd_tc_kernel<32, 16><<<dim3(gx, Cout / 32), 128, 0, st>>>(x, k, bias, B, H, W, Cin, Cout, relu, ob, out_f32, status);
    }
    return launched(1);
}


int qldnn_conv3x3_fwd_tc2(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout,
                          int relu, void* out_bf16, float* out_f32, int* status, void* stream) {
    if (!in || !wk || (!out_bf16 && !out_f32) || B < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 ||
        (Cout != 32 && Cout != 64 && Cout != 128 && Cout != 256) || !al(in, 16) || !al(wk, 16) ||
        !al(out_bf16, 16) || !al(out_f32, 16))
        return set_err(QLD_E_INVAL);
    const __nv_bfloat16* x = (const __nv_bfloat16*)in;
    const __nv_bfloat16* k = (const __nv_bfloat16*)wk;
    __nv_bfloat16* ob = (__nv_bfloat16*)out_bf16;
    const cudaStream_t st = (cudaStream_t)stream;
    const int bk = Cin % 64 == 0 ? 64 : (Cin % 32 == 0 ? 32 : 16);
#define QLD_TC2(NN, KK) \
    if (Cout == NN && bk == KK) return launch_tc2<NN, KK>(x, k, bias, B, H, W, Cin, Cout, relu, ob, out_f32, status, st);
    QLD_TC2(32, 16) QLD_TC2(32, 32) QLD_TC2(32, 64)
    QLD_TC2(64, 16) QLD_TC2(64, 32) QLD_TC2(64, 64)
    QLD_TC2(128, 16) QLD_TC2(128, 32) QLD_TC2(128, 64)
    QLD_TC2(256, 16) QLD_TC2(256, 32) QLD_TC2(256, 64)
#undef QLD_TC2
    return set_err(QLD_E_INVAL);
}

int qldnn_conv3x3_fwd_tma_mode(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin,
                               int Cout, int relu, void* out_bf16, float* out_f32, int* status, int mode,
                               void* stream);

int qldnn_conv3x3_fwd_tma(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin, int Cout,
                          int relu, void* out_bf16, float* out_f32, int* status, void* stream) {
    return qldnn_conv3x3_fwd_tma_mode(in, wk, bias, B, H, W, Cin, Cout, relu, out_bf16, out_f32, status, 0, stream);
}

int qldnn_conv3x3_fwd_tma_mode(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin,
                               int Cout, int relu, void* out_bf16, float* out_f32, int* status, int mode,
                               void* stream) {
    // mode: bit 0 forces the weight-streaming variant; bits 4.. (if non-zero)
    // force the number of CTAs per tile (1, 2 or 4); bit 8 early launch;
    // bits 12-19 the variant choices documented in qld.h; no other bits
    if (mode & ~(1 | (0xF << 4) | (1 << 8) | (0xFF << 12))) return set_err(QLD_E_INVAL);
    if (!out_bf16 && !out_f32) return set_err(QLD_E_INVAL);
    if (!al(out_bf16, 16) || !al(out_f32, 16)) return set_err(QLD_E_INVAL);
    qldnn::ConvEpi epi{};
    epi.out = (__nv_bfloat16*)out_bf16;
    epi.ldo = Cout;
    epi.out_f = out_f32;
    return conv_tma_dispatch(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, mode, (cudaStream_t)stream);
}

int qldnn_conv3x3_fwd_tma_epi(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin,
                              int Cout, int relu, void* out_bf16, long long ldo, void* pool_bf16, void* up_bf16,
                              long long ldu, const float* head_w, const float* head_b, const float* baseline,
                              float* pred, int* status, int flags, void* stream) {
    return qldnn_conv3x3_fwd_tma_epi_mode(in, wk, bias, B, H, W, Cin, Cout, relu, out_bf16, ldo, pool_bf16, up_bf16,
                                          ldu, head_w, head_b, baseline, pred, status, flags, 0, stream);
}

int qldnn_conv3x3_fwd_tma_epi_mode(const void* in, const void* wk, const float* bias, int B, int H, int W, int Cin,
                                   int Cout, int relu, void* out_bf16, long long ldo, void* pool_bf16, void* up_bf16,
                                   long long ldu, const float* head_w, const float* head_b, const float* baseline,
                                   float* pred, int* status, int flags, int mode, void* stream) {
    if (flags & ~QLDNN_EARLY_LAUNCH) return set_err(QLD_E_INVAL);
    // variant bits and (without a head, which needs one CTA per tile) the
    // CTAs per tile; early launch is a flag
    if (mode & ~((0xF << 4) | (0xF << 12) | (0xF << 16) | 1)) return set_err(QLD_E_INVAL);
    const bool head = head_w || head_b || baseline || pred;
    if (head && (mode & (0xF << 4))) return set_err(QLD_E_INVAL);
    if (!out_bf16 && !pool_bf16 && !up_bf16 && !head) return set_err(QLD_E_INVAL);
    if (out_bf16 && (!al(out_bf16, 16) || ldo < Cout || ldo % 8)) return set_err(QLD_E_INVAL);
    if (pool_bf16 && (!al(pool_bf16, 16) || H % 2 || W % 2)) return set_err(QLD_E_INVAL);
    if (up_bf16 && (!al(up_bf16, 16) || ldu < Cout || ldu % 8)) return set_err(QLD_E_INVAL);
    if (head && (!head_w || !head_b || !baseline || !pred)) return set_err(QLD_E_INVAL);
    qldnn::ConvEpi epi{};
    epi.out = (__nv_bfloat16*)out_bf16;
    epi.ldo = ldo;
    epi.pool = (__nv_bfloat16*)pool_bf16;
    epi.ldp = Cout;
    epi.up = (__nv_bfloat16*)up_bf16;
    epi.ldu = ldu;
    epi.head_w = head_w;
    epi.head_b = head_b;
    epi.base = baseline;
    epi.pred = pred;
    // the head needs every output channel of a pixel in one CTA
    mode |= (head ? (1 << 4) : 0) | ((flags & QLDNN_EARLY_LAUNCH) ? (1 << 8) : 0);
    return conv_tma_dispatch(in, wk, bias, B, H, W, Cin, Cout, relu, epi, status, mode, (cudaStream_t)stream);
}

int qldnn_conv3x3_wgrad_tma(const void* in, const void* g, int B, int H, int W, int Cin, int Cout, float* dw,
                            int* status, void* stream) {
    const bool stack = Cin == 16 || Cin == 32 || Cin == 64;
    if (!in || !g || !dw || B < 1 || H < 1 || W < 1 || !(stack || (Cin % 128 == 0 && Cin > 0)) ||
        (Cout != 32 && Cout != 64 && Cout != 128) || !al(in, 16) || !al(g, 16) || !al(dw, 16) ||
        (long long)B * H * W * (Cin > Cout ? Cin : Cout) >= (1ll << 40))
        return set_err(QLD_E_INVAL);
    const cudaStream_t st = (cudaStream_t)stream;
#define QLD_WG(NN, CI, SW, STK) \
    if (Cout == NN && (STK ? Cin == CI : !stack)) return launch_wgrad_tma<NN, SW, STK>(in, g, B, H, W, Cin, Cout, dw, status, st);
    QLD_WG(32, 16, 32, true) QLD_WG(32, 32, 64, true) QLD_WG(32, 64, 128, true) QLD_WG(32, 0, 128, false)
    QLD_WG(64, 16, 32, true) QLD_WG(64, 32, 64, true) QLD_WG(64, 64, 128, true) QLD_WG(64, 0, 128, false)
    QLD_WG(128, 16, 32, true) QLD_WG(128, 32, 64, true) QLD_WG(128, 64, 128, true) QLD_WG(128, 0, 128, false)
#undef QLD_WG
    return set_err(QLD_E_INVAL);
}

int qldnn_wait_selftest(long long limit_ns, long long* out, void* stream) {
    if (!out || limit_ns < 1000 || limit_ns > 2000000000ll || !al(out, 8)) return set_err(QLD_E_INVAL);
    qldnn::wait_selftest_kernel<<<1, 64, 0, (cudaStream_t)stream>>>((uint64_t)limit_ns, out);
    return launched(1);
}

int qldnn_zero(void* p, long long bytes, void* stream) {
    if (!p || bytes < 0) return set_err(QLD_E_INVAL);
    return cudaMemsetAsync(p, 0, (size_t)bytes, (cudaStream_t)stream) == cudaSuccess ? QLD_OK : set_err(QLD_E_CUDA);
}

}  // extern "C"
