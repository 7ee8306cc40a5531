// qldscene.cu -- GPU twin of the seeded scene generator (qldscene/scene.py).
//
// Input generation for tests and benchmarks only; it holds no QLD
// arithmetic and shares nothing with the QLD library. For every pixel p and
// absolute frame index s it evaluates, in integers only,
//     x = clip((mu + ((sd * Z) >> 16) + 2^15) >> 16, 0, maxv)
// where (mu, sd) = (mu1, sd1) when the source is on ((s - off) mod 4 < 2)
// and (mu0, sd0) otherwise, all Q16, and Z (Q16) is the sum of twelve
// Philox4x32-10 words (counter (p, s_lo, j, s_hi), j = 0..2; key (k0, k1))
// minus 6 * 2^32, shifted right by 16. The numpy generator computes the
// same expression, so both produce identical frames.

#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

__device__ __forceinline__ uint64_t philox_sum4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c0, c1, c2, c3, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return (uint64_t)c0 + c1 + c2 + c3;
}

template <typename T>
__global__ void generate_kernel(T* __restrict__ out, long long npix, long long out_stride, long long s_first,
                                int count, const int32_t* __restrict__ mu0, const int32_t* __restrict__ mu1,
                                const int32_t* __restrict__ sd0, const int32_t* __restrict__ sd1, int off,
                                uint32_t k0, uint32_t k1, int maxv) {
    const long long total = npix * (long long)count;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / npix;
        const long long p = e - i * npix;
        const long long s = s_first + i;
        const bool on = ((((s - off) % 4) + 4) % 4) < 2;
        const int64_t mu = on ? mu1[p] : mu0[p];
        const int64_t sd = on ? sd1[p] : sd0[p];
        uint64_t tot = 0;
        for (uint32_t j = 0; j < 3; ++j)
            tot += philox_sum4((uint32_t)p, (uint32_t)(s & 0xFFFFFFFFll), j, (uint32_t)((unsigned long long)s >> 32),
                               k0, k1);
        const int64_t z = ((int64_t)tot - 6ll * (1ll << 32)) >> 16;
        int64_t v = (mu + ((sd * z) >> 16) + (1 << 15)) >> 16;
        v = v < 0 ? 0 : (v > maxv ? maxv : v);
        out[i * out_stride + p] = (T)v;
    }
}

// One pass of a separable blur with zero padding: out[y][x] = sum over
// t = -r..r of taps[t + r] * in at (y, x + t) (rows) or (y + t, x) (columns).
__global__ void blur_pass_kernel(const float* __restrict__ in, float* __restrict__ out, int H, int W,
                                 const float* __restrict__ taps, int r, int along_rows) {
    const long long n = (long long)H * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(e / W), x = (int)(e - (long long)y * W);
        float acc = 0.f;
        for (int t = -r; t <= r; ++t) {
            const int yy = along_rows ? y : y + t, xx = along_rows ? x + t : x;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) acc = fmaf(taps[t + r], in[(long long)yy * W + xx], acc);
        }
        out[e] = acc;
    }
}

}  // namespace

extern "C" {

// Separable blur of an H x W float image on the device (zero padding): the
// row pass into tmp, the column pass into out (each H x W floats; out may not
// alias in or tmp). taps holds 2r + 1 device floats. Returns 0, -1 on bad
// arguments, or the CUDA error code of the launches.
int qs_blur(const float* in, float* tmp, float* out, int H, int W, const float* taps, int r, void* stream) {
    if (!in || !tmp || !out || !taps || H < 1 || W < 1 || r < 0 || out == in || out == tmp || tmp == in) return -1;
    const long long n = (long long)H * W;
    long long blocks = (n + 255) / 256;
    if (blocks > 148ll * 64) blocks = 148ll * 64;
    cudaStream_t st = (cudaStream_t)stream;
    blur_pass_kernel<<<(unsigned)blocks, 256, 0, st>>>(in, tmp, H, W, taps, r, 1);
    blur_pass_kernel<<<(unsigned)blocks, 256, 0, st>>>(tmp, out, H, W, taps, r, 0);
    return (int)cudaGetLastError();
}

// Writes frames s_first .. s_first+count-1 of the scene to out (device),
// frame i at out + i*out_stride elements. pixfmt 1 = uint8, 2 = uint16.
// mu0/mu1/sd0/sd1 are device int32 arrays of npix Q16 values. Returns 0, -1
// on bad arguments, or the CUDA error code of the launch.
int qs_generate(void* out, int pixfmt, long long npix, long long out_stride, long long s_first, int count,
                const int32_t* mu0, const int32_t* mu1, const int32_t* sd0, const int32_t* sd1, int phase_offset,
                unsigned key0, unsigned key1, int maxv, void* stream) {
    if (!out || !mu0 || !mu1 || !sd0 || !sd1 || npix <= 0 || count < 0 || out_stride < npix) return -1;
    if (count == 0) return 0;
    const long long total = npix * (long long)count;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 148ll * 64) blocks = 148ll * 64;
    cudaStream_t st = (cudaStream_t)stream;
    if (pixfmt == 1) {
        generate_kernel<uint8_t><<<(unsigned)blocks, threads, 0, st>>>((uint8_t*)out, npix, out_stride, s_first,
                                                                     count, mu0, mu1, sd0, sd1, phase_offset,
                                                                     key0, key1, maxv);
    } else if (pixfmt == 2) {
        generate_kernel<uint16_t><<<(unsigned)blocks, threads, 0, st>>>((uint16_t*)out, npix, out_stride, s_first,
                                                                      count, mu0, mu1, sd0, sd1, phase_offset,
                                                                      key0, key1, maxv);
    } else {
        return -1;
    }
    return (int)cudaGetLastError();
}

}  // extern "C"
