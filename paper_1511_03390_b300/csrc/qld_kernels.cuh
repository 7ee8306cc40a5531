// qld_kernels.cuh -- sm_103a kernels of the QLD library.
//
// Hot path (per pixel, per frame s of the stream, window of N frames):
//   push:   x_old = ring[s mod N]; ring[s mod N] = x_s; d = x_s - x_old;
//           S += sin(pi s/2) d, C += cos(pi s/2) d        (int32, exact)
//   image:  R = sqrt(S^2 + C^2), phase = atan2(-S, C)      (float32)
//   bin:    X_k = sum_{slots j} ring[j] exp(-2 pi i k j / N), out = |X_k|^2
// (Methods, "Numerical simulations", the equations for R(j,k) and the FFT
// map; SI, "Timing sequence" item 3 and the closing paragraph on the sliding
// buffer of N frames.)
//
// All three are HBM-streaming kernels: pixels are independent, frames are
// contiguous rows, and every thread owns one vector of pixels -- 16 bytes
// (8 uint16 or 16 uint8 pixels) or, for packed 12-bit data, 24 bytes (16
// pixels) -- so loads and stores are wide and fully coalesced.

#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qldk {

constexpr int kVecBytes = 16;

// Tag type of the packed 12-bit pixel format: two pixels in three bytes,
// least significant bits first (GenICam Mono12p), so pixel i of a run is
// bits [12 i, 12 i + 12) of the little-endian byte string.
struct p12_t {};

// 24 bytes = 16 packed 12-bit pixels.
struct P12Vec {
    uint32_t w[6];
};

// uint8 and packed 12-bit frames in vectors of 8 pixels (8 and 12 bytes), for
// the DFT-bin kernel and the multi-stream batch push: with 16-pixel vectors
// those need over 100 registers per thread, too few warps to keep the loads
// in flight. The single-stream push kernel keeps 16-pixel vectors.
struct u8h_t {};
struct p12h_t {};
struct P12Half {
    uint32_t w[3];
};

// Per-format vector traits: Vec, bytes per vector VB, pixels per vector VP,
// and streaming load / store of one vector (cache-streaming hints: every
// frame byte is touched once per kernel).
template <typename T>
struct Fmt;

template <>
struct Fmt<uint8_t> {
    using Vec = uint4;
    static constexpr int VB = 16, VP = 16, ALIGN = 16;
    static __device__ __forceinline__ Vec load(const uint8_t* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
    static __device__ __forceinline__ void store(uint8_t* p, const Vec& v) { __stcs(reinterpret_cast<uint4*>(p), v); }
    static __device__ __forceinline__ Vec zero() { return make_uint4(0, 0, 0, 0); }
};

template <>
struct Fmt<uint16_t> {
    using Vec = uint4;
    static constexpr int VB = 16, VP = 8, ALIGN = 16;
    static __device__ __forceinline__ Vec load(const uint8_t* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
    static __device__ __forceinline__ void store(uint8_t* p, const Vec& v) { __stcs(reinterpret_cast<uint4*>(p), v); }
    static __device__ __forceinline__ Vec zero() { return make_uint4(0, 0, 0, 0); }
};

template <>
struct Fmt<p12_t> {
    using Vec = P12Vec;
    static constexpr int VB = 24, VP = 16, ALIGN = 8;
    static __device__ __forceinline__ Vec load(const uint8_t* p) {
        const uint2* q = reinterpret_cast<const uint2*>(p);
        const uint2 a = __ldcs(q), b = __ldcs(q + 1), c = __ldcs(q + 2);
        return P12Vec{{a.x, a.y, b.x, b.y, c.x, c.y}};
    }
    static __device__ __forceinline__ void store(uint8_t* p, const Vec& v) {
        uint2* q = reinterpret_cast<uint2*>(p);
        __stcs(q, make_uint2(v.w[0], v.w[1]));
        __stcs(q + 1, make_uint2(v.w[2], v.w[3]));
        __stcs(q + 2, make_uint2(v.w[4], v.w[5]));
    }
    static __device__ __forceinline__ Vec zero() { return P12Vec{{0, 0, 0, 0, 0, 0}}; }
};

template <>
struct Fmt<u8h_t> {
    using Vec = uint2;
    static constexpr int VB = 8, VP = 8, ALIGN = 8;
    static __device__ __forceinline__ Vec load(const uint8_t* p) { return __ldcs(reinterpret_cast<const uint2*>(p)); }
    static __device__ __forceinline__ void store(uint8_t* p, const Vec& v) { __stcs(reinterpret_cast<uint2*>(p), v); }
    static __device__ __forceinline__ Vec zero() { return make_uint2(0u, 0u); }
};

template <>
struct Fmt<p12h_t> {
    using Vec = P12Half;
    static constexpr int VB = 12, VP = 8, ALIGN = 4;
    static __device__ __forceinline__ Vec load(const uint8_t* p) {
        const unsigned int* q = reinterpret_cast<const unsigned int*>(p);
        return P12Half{{__ldcs(q), __ldcs(q + 1), __ldcs(q + 2)}};
    }
    static __device__ __forceinline__ void store(uint8_t* p, const Vec& v) {
        unsigned int* q = reinterpret_cast<unsigned int*>(p);
        __stcs(q, v.w[0]);
        __stcs(q + 1, v.w[1]);
        __stcs(q + 2, v.w[2]);
    }
    static __device__ __forceinline__ Vec zero() { return P12Half{{0u, 0u, 0u}}; }
};

// Vector format the DFT-bin kernel reads a pixel format with.
template <typename T>
struct BinFmt {
    using type = T;
};
template <>
struct BinFmt<uint8_t> {
    using type = u8h_t;
};
template <>
struct BinFmt<p12_t> {
    using type = p12h_t;
};

// ---------------------------------------------------------------- helpers --

// Raw bits of pixel q of a vector (q is a compile-time constant after
// unrolling, so the word selection and shifts fold away).
__device__ __forceinline__ uint32_t raw_pix(const uint4& v, int q, uint16_t*) {
    const uint32_t w = (q < 2) ? v.x : (q < 4) ? v.y : (q < 6) ? v.z : v.w;
    return (q & 1) ? (w >> 16) : (w & 0xFFFFu);
}
__device__ __forceinline__ uint32_t raw_pix(const uint4& v, int q, uint8_t*) {
    const uint32_t w = (q < 4) ? v.x : (q < 8) ? v.y : (q < 12) ? v.z : v.w;
    return (w >> (8 * (q & 3))) & 0xFFu;
}
__device__ __forceinline__ uint32_t raw_pix(const uint2& v, int q, u8h_t*) {
    const uint32_t w = (q < 4) ? v.x : v.y;
    return (w >> (8 * (q & 3))) & 0xFFu;
}
__device__ __forceinline__ uint32_t raw_pix(const P12Half& v, int q, p12h_t*) {
    const int o = 12 * q;  // bit offset of pixel q in the 96-bit vector
    const int wi = o >> 5;
    const uint32_t lo = v.w[wi];
    const uint32_t hi = (wi + 1 < 3) ? v.w[wi + 1] : 0u;
    return __funnelshift_r(lo, hi, o & 31) & 0xFFFu;
}
__device__ __forceinline__ uint32_t raw_pix(const P12Vec& v, int q, p12_t*) {
    const int o = 12 * q;  // bit offset of pixel q in the 192-bit vector
    const int wi = o >> 5;
    const uint32_t lo = v.w[wi];
    const uint32_t hi = (wi + 1 < 6) ? v.w[wi + 1] : 0u;
    return __funnelshift_r(lo, hi, o & 31) & 0xFFFu;
}

// Pixel q of a vector as an int.
template <typename T>
__device__ __forceinline__ int pix(const typename Fmt<T>::Vec& v, int q) {
    return (int)raw_pix(v, q, (T*)nullptr);
}

// Pixel q of a vector as an exact float: the integer bits are placed in the
// mantissa of 2^23 and 2^23 is subtracted (exact for values below 2^23); for
// uint8 / uint16 one byte permute builds the float bits.
template <typename T>
__device__ __forceinline__ float pixf(const typename Fmt<T>::Vec& v, int q) {
    return __uint_as_float(raw_pix(v, q, (T*)nullptr) | 0x4B000000u) - 8388608.0f;
}
template <>
__device__ __forceinline__ float pixf<uint16_t>(const uint4& v, int q) {
    const uint32_t w = (q < 2) ? v.x : (q < 4) ? v.y : (q < 6) ? v.z : v.w;
    const uint32_t b = __byte_perm(w, 0x4B000000u, (q & 1) ? 0x7632u : 0x7610u);
    return __uint_as_float(b) - 8388608.0f;
}
template <>
__device__ __forceinline__ float pixf<u8h_t>(const uint2& v, int q) {
    const uint32_t w = (q < 4) ? v.x : v.y;
    const uint32_t b = __byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)(q & 3));
    return __uint_as_float(b) - 8388608.0f;
}
template <>
__device__ __forceinline__ float pixf<uint8_t>(const uint4& v, int q) {
    const uint32_t w = (q < 4) ? v.x : (q < 8) ? v.y : (q < 12) ? v.z : v.w;
    const uint32_t b = __byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)(q & 3));
    return __uint_as_float(b) - 8388608.0f;
}

// Float bits of pixel q of a vector placed in the mantissa of 2^23:
// subtracting 2^23 afterwards gives the pixel value exactly.
template <typename T>
__device__ __forceinline__ uint32_t pixbits(const typename Fmt<T>::Vec& v, int q) {
    return raw_pix(v, q, (T*)nullptr) | 0x4B000000u;
}
template <>
__device__ __forceinline__ uint32_t pixbits<uint16_t>(const uint4& v, int q) {
    const uint32_t w = (q < 2) ? v.x : (q < 4) ? v.y : (q < 6) ? v.z : v.w;
    return __byte_perm(w, 0x4B000000u, (q & 1) ? 0x7632u : 0x7610u);
}
template <>
__device__ __forceinline__ uint32_t pixbits<u8h_t>(const uint2& v, int q) {
    const uint32_t w = (q < 4) ? v.x : v.y;
    return __byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)(q & 3));
}

// Two FP32 lanes in one 64-bit register (low = even pixel, high = odd) for
// the paired FP32 instructions (add / sub / fma .f32x2): each lane rounds
// exactly as the scalar instruction, at one issue slot per pair.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_bits(uint32_t lo, uint32_t hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ f32x2 f2_splat(float a) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float2 f2_split(f32x2 a) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Float bits b[q] of the pixels of a vector for the DFT bin: pixel q is
// exactly b[q] - bin_offset<T>(q) as floats. Generic formats place the
// integer in the mantissa of 2^23 (pixbits).
template <typename T>
__device__ __forceinline__ void bin_bits(const typename Fmt<T>::Vec& v, uint32_t (&b)[Fmt<T>::VP]) {
#pragma unroll
    for (int q = 0; q < Fmt<T>::VP; ++q) b[q] = pixbits<T>(v, q);
}
template <typename T>
__device__ __forceinline__ constexpr float bin_offset(int) {
    return 8388608.0f;
}

__device__ __forceinline__ uint32_t mul_hi_add(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t mul_lo(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Packed 12-bit: the 8 fields of the words w0, w1, w2 sit at bits [0,12),
// [12,24), [24,36), [36,48), [48,60), [60,72), [72,84), [84,96) of the
// 96-bit vector. The integer ALU is the busiest pipe of the bin kernel on
// this format, so the fields are cut with as few ALU instructions as
// possible:
//  - a field wholly inside the mantissa (bits [s, s+12) with s + 12 <= 23:
//    pixels 0, 3, 6 at s = 0, 4, 8) is masked in place and given the
//    exponent of 2^(23-s), which makes the float 2^(23-s) + p exactly;
//  - a field at the top of a word (pixels 1, 4 after a left shift by a
//    multiply, pixel 7 as it is) comes down by a multiply-high whose addend is
//    the exponent of 2^23: these run on the multiply pipe, not the ALU;
//  - the two fields that straddle words (pixels 2, 5) take a funnel shift
//    and a mask.
template <>
__device__ __forceinline__ void bin_bits<p12h_t>(const P12Half& v, uint32_t (&b)[8]) {
    const uint32_t w0 = v.w[0], w1 = v.w[1], w2 = v.w[2];
    constexpr uint32_t e23 = 0x4B000000u;  // exponent bits of 2^23
    b[0] = (w0 & 0xFFFu) | e23;
    b[1] = mul_hi_add(mul_lo(w0, 1u << 8), 1u << 12, e23);
    b[2] = (__funnelshift_r(w0, w1, 24) & 0xFFFu) | e23;
    b[3] = (w1 & 0xFFF0u) | ((127u + 19u) << 23);
    b[4] = mul_hi_add(mul_lo(w1, 1u << 4), 1u << 12, e23);
    b[5] = (__funnelshift_r(w1, w2, 28) & 0xFFFu) | e23;
    b[6] = (w2 & 0xFFF00u) | ((127u + 15u) << 23);
    b[7] = mul_hi_add(w2, 1u << 12, e23);
}
template <>
__device__ __forceinline__ constexpr float bin_offset<p12h_t>(int q) {
    return q == 3 ? 524288.0f : q == 6 ? 32768.0f : 8388608.0f;
}

// Frames per load group of the DFT bin (loads in flight per thread): the
// 8- and 12-byte vectors of uint8 and packed 12-bit frames take eight, so a
// thread keeps as many bytes in flight as with four 16-byte uint16 vectors
// (measured on 1024^2 frames, N = 1024: uint8 +6 %, packed 12-bit +7 %).
//
// INCR: frame pointers advanced by increments, whole groups without bounds
// checks. The uint8 bin is bound by instruction issue, and ~40 % of its
// instructions were per-frame address arithmetic and bounds checks (ncu
// opcode counts: 41 instructions per thread and frame, of which 8 byte
// permutes, 8 paired FMAs, 4.5 paired adds and 2 loads); with INCR it went
// from 221.9 to 196.8 us at 1024^2, N = 1024 (0.75 -> 0.85 of the copy
// peak), bit-identical. The uint16 bin, already at the copy rate, measured
// slower that way (317 -> 336 us) and keeps indexed addresses.
template <typename T>
struct BinGroup {
    static constexpr int UF = 4;
    static constexpr bool INCR = false;
};
template <>
struct BinGroup<u8h_t> {
    static constexpr int UF = 8;
    static constexpr bool INCR = true;
};
template <>
struct BinGroup<p12h_t> {
    static constexpr int UF = 8;
    static constexpr bool INCR = true;
};

// Adds d = x_new - x_old of one frame with absolute index residue r = s mod 4
// to the quadrature sums: sin(pi s/2) = 1, 0, -1, 0 and cos(pi s/2) = 0, -1,
// 0, 1 for r = 1, 2, 3, 0, so exactly one of S, C changes. r is the same for
// every thread of a launch, so the switch does not diverge.
template <typename T, bool HAS_OLD>
__device__ __forceinline__ void accumulate(int32_t* sacc, int32_t* cacc, const typename Fmt<T>::Vec& xn,
                                           const typename Fmt<T>::Vec& xo, int r) {
    constexpr int VP = Fmt<T>::VP;
    switch (r) {
        case 1:
#pragma unroll
            for (int q = 0; q < VP; ++q) sacc[q] += pix<T>(xn, q) - (HAS_OLD ? pix<T>(xo, q) : 0);
            break;
        case 2:
#pragma unroll
            for (int q = 0; q < VP; ++q) cacc[q] -= pix<T>(xn, q) - (HAS_OLD ? pix<T>(xo, q) : 0);
            break;
        case 3:
#pragma unroll
            for (int q = 0; q < VP; ++q) sacc[q] -= pix<T>(xn, q) - (HAS_OLD ? pix<T>(xo, q) : 0);
            break;
        default:
#pragma unroll
            for (int q = 0; q < VP; ++q) cacc[q] += pix<T>(xn, q) - (HAS_OLD ? pix<T>(xo, q) : 0);
            break;
    }
}

// R = sqrt(S^2 + C^2) in float32. S and C convert exactly while |S|, |C| <
// 2^24 (every window of 12-bit data up to N = 16384); beyond that the
// conversion adds at most 2^-24 relative error, so R stays within about
// 2e-7 of its exact value either way.
__device__ __forceinline__ float amplitude(int32_t s, int32_t c) {
    const float fs = (float)s;
    const float fc = (float)c;
    return sqrtf(fmaf(fs, fs, fc * fc));
}

// arctan on [0, 1] by the polynomial of Hastings, "Approximations for Digital
// Computers" (1955), as tabulated in Abramowitz & Stegun, Handbook of
// Mathematical Functions, 4.4.49: atan x = x (1 + sum_{k=1..8} a_{2k} x^{2k})
// with |error| <= 2e-8 for 0 <= x <= 1.
__device__ __forceinline__ float atan_unit(float x) {
    const float t = x * x;
    float p = 0.0028662257f;
    p = fmaf(p, t, -0.0161657367f);
    p = fmaf(p, t, 0.0429096138f);
    p = fmaf(p, t, -0.0752896400f);
    p = fmaf(p, t, 0.1065626393f);
    p = fmaf(p, t, -0.1420889944f);
    p = fmaf(p, t, 0.1999355085f);
    p = fmaf(p, t, -0.3333314528f);
    p = fmaf(p, t, 1.0f);
    return x * p;
}

// atan2(y, x) in (-pi, pi]: the ratio of the smaller to the larger
// magnitude goes through atan_unit, then the octant is restored (pi/2 - r
// above the diagonal, pi - r for x < 0, the sign of y last), so y = +0 with
// x < 0 gives +pi and x = y = 0 gives 0. Error about 4e-7 rad (float32
// rounding of the reduction and of pi).
__device__ __forceinline__ float atan2_unit_poly(float y, float x) {
    const float ay = fabsf(y), ax = fabsf(x);
    const float mx = fmaxf(ay, ax), mn = fminf(ay, ax);
    const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    float r = atan_unit(a);
    if (ay > ax) r = 1.57079632679489662f - r;
    if (x < 0.f) r = 3.14159265358979324f - r;
    return (y < 0.f) ? -r : r;
}

// phase = atan2(-S, C), with the negation done on the integer so S = 0 gives
// y = +0 (C < 0 then gives +pi).
__device__ __forceinline__ float phase_of(int32_t s, int32_t c) {
    return atan2_unit_poly((float)(-s), (float)c);
}

// ------------------------------------------------------------------- push --

struct PushArgs {
    const uint8_t* frames;  // first frame applied
    long long frame_stride; // bytes between consecutive input frames
    int nf;                 // frames applied
    long long s_first;      // absolute index of the first applied frame
    uint8_t* ring;          // N slots
    long long slot_stride;  // bytes between ring slots (multiple of 256)
    int N;
    int32_t* S;             // sums, padded to a multiple of 64 pixels
    int32_t* C;
    long long nvec;         // 16-byte vectors per frame (vector path) or pixels (scalar path)
    long long npix;
    float* amp;             // epilogue outputs (may be NULL)
    float* phase;
    int out_aligned;        // amp and phase are 16-byte aligned (or NULL)
};

// Push of the vector v of every applied frame (vector path: frames aligned to
// Fmt<T>::ALIGN and frame_stride a multiple of Fmt<T>::VB). RESET: the
// window is rebuilt from the applied frames alone (a push of at least N
// frames), so the sums start at zero and the expiring slots are not read.
// EPI: also write the amplitude / phase image.
// GROUP4: frames are taken four at a time with all eight loads issued before
// any store (the single-stream push kernel, where one push carries several
// frames); without it one frame at a time, which needs far fewer registers
// (the batch kernel, whose pushes carry one frame per stream per tick).
template <typename T, bool RESET, bool EPI, bool GROUP4 = true>
__device__ __forceinline__ void push_vector(const PushArgs& a, long long v) {
    using F = Fmt<T>;
    using Vec = typename F::Vec;
    constexpr int VP = F::VP;
    const long long off = v * F::VB;
    const long long p0 = v * VP;

    // Frame s moves S when s is odd and C when s is even (accumulate), so a
    // push of one frame leaves one of the sums as it was: that one is not
    // stored, and not read unless the image needs it. The same for every
    // thread of a launch.
    const bool chS = RESET || a.nf > 1 || (a.s_first & 1);
    const bool chC = RESET || a.nf > 1 || !(a.s_first & 1);

    int32_t sacc[VP], cacc[VP];
    if (RESET) {
#pragma unroll
        for (int q = 0; q < VP; ++q) sacc[q] = cacc[q] = 0;
    } else {
#pragma unroll
        for (int q = 0; q < VP; q += 4) {
            int4 s4 = make_int4(0, 0, 0, 0), c4 = make_int4(0, 0, 0, 0);
            if (EPI || chS) s4 = *reinterpret_cast<const int4*>(a.S + p0 + q);
            if (EPI || chC) c4 = *reinterpret_cast<const int4*>(a.C + p0 + q);
            sacc[q] = s4.x; sacc[q + 1] = s4.y; sacc[q + 2] = s4.z; sacc[q + 3] = s4.w;
            cacc[q] = c4.x; cacc[q + 1] = c4.y; cacc[q + 2] = c4.z; cacc[q + 3] = c4.w;
        }
    }

    const uint8_t* src = a.frames + off;
    uint8_t* ring = a.ring + off;
    int f = 0;
    // Groups of four frames: all loads are issued before any store so eight
    // 128-bit loads per thread are in flight.
    for (; GROUP4 && f + 4 <= a.nf; f += 4) {
        Vec xn[4], xo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xo[u] = F::zero();
        long long slot[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long s = a.s_first + f + u;
            slot[u] = s % a.N;
            xn[u] = F::load(src + (long long)(f + u) * a.frame_stride);
        }
        if (!RESET) {
#pragma unroll
            for (int u = 0; u < 4; ++u) xo[u] = F::load(ring + slot[u] * a.slot_stride);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) F::store(ring + slot[u] * a.slot_stride, xn[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            accumulate<T, !RESET>(sacc, cacc, xn[u], xo[u], (int)((a.s_first + f + u) & 3));
    }
    for (; f < a.nf; ++f) {
        const long long s = a.s_first + f;
        const long long slot = s % a.N;
        const Vec xn = F::load(src + (long long)f * a.frame_stride);
        Vec xo = F::zero();
        if (!RESET) xo = F::load(ring + slot * a.slot_stride);
        F::store(ring + slot * a.slot_stride, xn);
        accumulate<T, !RESET>(sacc, cacc, xn, xo, (int)(s & 3));
    }

#pragma unroll
    for (int q = 0; q < VP; q += 4) {
        if (chS) *reinterpret_cast<int4*>(a.S + p0 + q) = make_int4(sacc[q], sacc[q + 1], sacc[q + 2], sacc[q + 3]);
        if (chC) *reinterpret_cast<int4*>(a.C + p0 + q) = make_int4(cacc[q], cacc[q + 1], cacc[q + 2], cacc[q + 3]);
    }

    if (EPI) {
        if (a.amp) {
            if (a.out_aligned) {
#pragma unroll
                for (int q = 0; q < VP; q += 4)
                    __stcs(reinterpret_cast<float4*>(a.amp + p0 + q),
                           make_float4(amplitude(sacc[q], cacc[q]), amplitude(sacc[q + 1], cacc[q + 1]),
                                       amplitude(sacc[q + 2], cacc[q + 2]), amplitude(sacc[q + 3], cacc[q + 3])));
            } else {
#pragma unroll
                for (int q = 0; q < VP; ++q) a.amp[p0 + q] = amplitude(sacc[q], cacc[q]);
            }
        }
        if (a.phase) {
            if (a.out_aligned) {
#pragma unroll
                for (int q = 0; q < VP; q += 4)
                    __stcs(reinterpret_cast<float4*>(a.phase + p0 + q),
                           make_float4(phase_of(sacc[q], cacc[q]), phase_of(sacc[q + 1], cacc[q + 1]),
                                       phase_of(sacc[q + 2], cacc[q + 2]), phase_of(sacc[q + 3], cacc[q + 3])));
            } else {
#pragma unroll
                for (int q = 0; q < VP; ++q) a.phase[p0 + q] = phase_of(sacc[q], cacc[q]);
            }
        }
    }
}

// uint16 pushes are held to 72 registers, seven 128-thread CTAs per SM, so a
// 1024^2 frame (1024 CTAs) runs in one wave over 148 SMs; the other formats
// keep the compiler's choice (0 = no minimum).
template <typename T>
constexpr int push_min_ctas() { return sizeof(T) == 2 ? 7 : 0; }

template <typename T, bool RESET, bool EPI>
__global__ void __launch_bounds__(128, push_min_ctas<T>()) push_vec_kernel(const PushArgs a) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < a.nvec) push_vector<T, RESET, EPI>(a, v);
}

// Scalar path for inputs that are not 16-byte aligned or whose frame size is
// not a multiple of 16 bytes: one pixel per thread.
template <typename T, bool RESET, bool EPI>
__global__ void __launch_bounds__(256) push_scalar_kernel(const PushArgs a) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npix) return;
    int32_t sacc = RESET ? 0 : a.S[p];
    int32_t cacc = RESET ? 0 : a.C[p];
    const T* src = reinterpret_cast<const T*>(a.frames) + p;
    for (int f = 0; f < a.nf; ++f) {
        const long long s = a.s_first + f;
        T* slotp = reinterpret_cast<T*>(a.ring + (s % a.N) * a.slot_stride) + p;
        const int xn = (int)*reinterpret_cast<const T*>(reinterpret_cast<const uint8_t*>(src) +
                                                        (long long)f * a.frame_stride);
        const int xo = RESET ? 0 : (int)*slotp;
        *slotp = (T)xn;
        const int d = xn - xo;
        switch ((int)(s & 3)) {
            case 1: sacc += d; break;
            case 2: cacc -= d; break;
            case 3: sacc -= d; break;
            default: cacc += d; break;
        }
    }
    a.S[p] = sacc;
    a.C[p] = cacc;
    if (EPI) {
        if (a.amp) a.amp[p] = amplitude(sacc, cacc);
        if (a.phase) a.phase[p] = phase_of(sacc, cacc);
    }
}

// Scalar path for packed 12-bit frames that are not 8-byte aligned or whose
// size is not a multiple of 24 bytes: one pixel pair (3 bytes) per thread,
// so no two threads write the same byte of a ring slot.
template <bool RESET, bool EPI>
__global__ void __launch_bounds__(256) push_scalar_p12_kernel(const PushArgs a) {
    const long long pr = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * pr >= a.npix) return;
    const long long p = 2 * pr;
    int32_t s0 = RESET ? 0 : a.S[p], s1 = RESET ? 0 : a.S[p + 1];
    int32_t c0 = RESET ? 0 : a.C[p], c1 = RESET ? 0 : a.C[p + 1];
    for (int f = 0; f < a.nf; ++f) {
        const long long s = a.s_first + f;
        const uint8_t* src = a.frames + (long long)f * a.frame_stride + 3 * pr;
        uint8_t* slotp = a.ring + (s % a.N) * a.slot_stride + 3 * pr;
        const uint32_t b0 = src[0], b1 = src[1], b2 = src[2];
        const int n0 = (int)(b0 | ((b1 & 0xFu) << 8)), n1 = (int)((b1 >> 4) | (b2 << 4));
        int o0 = 0, o1 = 0;
        if (!RESET) {
            const uint32_t q0 = slotp[0], q1 = slotp[1], q2 = slotp[2];
            o0 = (int)(q0 | ((q1 & 0xFu) << 8));
            o1 = (int)((q1 >> 4) | (q2 << 4));
        }
        slotp[0] = (uint8_t)b0;
        slotp[1] = (uint8_t)b1;
        slotp[2] = (uint8_t)b2;
        const int d0 = n0 - o0, d1 = n1 - o1;
        switch ((int)(s & 3)) {
            case 1: s0 += d0; s1 += d1; break;
            case 2: c0 -= d0; c1 -= d1; break;
            case 3: s0 -= d0; s1 -= d1; break;
            default: c0 += d0; c1 += d1; break;
        }
    }
    a.S[p] = s0;
    a.S[p + 1] = s1;
    a.C[p] = c0;
    a.C[p + 1] = c1;
    if (EPI) {
        if (a.amp) {
            a.amp[p] = amplitude(s0, c0);
            a.amp[p + 1] = amplitude(s1, c1);
        }
        if (a.phase) {
            a.phase[p] = phase_of(s0, c0);
            a.phase[p + 1] = phase_of(s1, c1);
        }
    }
}

// ------------------------------------------------------------------ image --

// Four pixels per thread; S and C are padded so the int4 loads stay in bounds.
static __global__ void __launch_bounds__(256) image_kernel(const int32_t* __restrict__ S, const int32_t* __restrict__ C,
                                                    long long npix, float* __restrict__ amp,
                                                    float* __restrict__ phase, int out_aligned) {
    const long long p0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (p0 >= npix) return;
    const int4 s4 = *reinterpret_cast<const int4*>(S + p0);
    const int4 c4 = *reinterpret_cast<const int4*>(C + p0);
    const int32_t s[4] = {s4.x, s4.y, s4.z, s4.w};
    const int32_t c[4] = {c4.x, c4.y, c4.z, c4.w};
    const bool full = out_aligned && p0 + 4 <= npix;
    if (amp) {
        if (full) {
            __stcs(reinterpret_cast<float4*>(amp + p0), make_float4(amplitude(s[0], c[0]), amplitude(s[1], c[1]),
                                                                     amplitude(s[2], c[2]), amplitude(s[3], c[3])));
        } else {
            for (int q = 0; q < 4 && p0 + q < npix; ++q) amp[p0 + q] = amplitude(s[q], c[q]);
        }
    }
    if (phase) {
        if (full) {
            __stcs(reinterpret_cast<float4*>(phase + p0), make_float4(phase_of(s[0], c[0]), phase_of(s[1], c[1]),
                                                                       phase_of(s[2], c[2]), phase_of(s[3], c[3])));
        } else {
            for (int q = 0; q < 4 && p0 + q < npix; ++q) phase[p0 + q] = phase_of(s[q], c[q]);
        }
    }
}

// --------------------------------------------------------------- DFT bin --

// Twiddles of bin k for ring slot j: exp(-2 pi i k j / N), with (k j) mod N
// reduced in integers, evaluated in FP64 and rounded to float. Slot j holds
// the frame whose absolute index s satisfies s = j (mod N), and
// exp(-2 pi i k s / N) depends only on (k s) mod N, so slot order needs no
// window rotation.
static __global__ void twiddle_kernel(float2* __restrict__ tw, int N, int k) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const long long m = ((long long)k * j) % N;
    double sn, cs;
    sincospi(2.0 * (double)m / (double)N, &sn, &cs);
    tw[j] = make_float2((float)cs, (float)(-sn));
}

// Output of bin_kernel: the power |X|^2, or the amplitude |X| and phase
// arg X (the general-frequency lock-in R and atan2(-S, C), since with
// twiddles (cos, -sin) the real part is C and the imaginary part -S).
enum BinOut { kBinPower = 0, kBinAmpPhase = 1 };

// Pixel-tiled single-bin DFT over the N ring slots. A CTA of NT threads
// covers PV = 2^PV_LOG pixel vectors and splits the time axis into NT/PV
// slices: thread t takes vector t mod PV and frames j = t/PV, t/PV + NT/PV,
// ..., BinGroup<T>::UF loads in flight. Each thread accumulates in float32, flushing a
// partial every 16 frames into a running sum to keep rounding small. When
// PV < 32 one warp holds 32/PV time slices of the same pixels and they are
// combined with warp shuffles; the warps' partials are then combined in
// shared memory.
//
// PUSH: one step of the hot path in one launch. Before the DFT bin the
// kernel pushes a.nf frames (1 <= nf <= N, the window full afterwards; the
// ring is a.ring with slots slot_stride == a.slot_stride apart) and writes the
// amplitude / phase image. Time slice ts reads ring slots j = ts, ts + TS,
// ...; the thread of slice ts pushes exactly the frames whose slot lies in its
// slice, so every slot it then reads was written by itself (program order)
// and by no other thread. The changes of S and C (exact int32) are summed over
// the slices in shared memory before S, C and the image are written. The bin
// loop is the same code as without PUSH: results are bit-identical to
// push_vec_kernel with the image epilogue followed by the DFT bin.
template <typename T, int PV_LOG, int NT, int OUT, bool PUSH = false>
__global__ void __launch_bounds__(NT) bin_kernel(const uint8_t* __restrict__ ring, long long slot_stride, int N,
                                                 const float2* __restrict__ tw, long long nvec, long long npix,
                                                 float* __restrict__ out, float* __restrict__ out2,
                                                 const PushArgs a) {
    using F = Fmt<T>;
    constexpr int VP = F::VP;
    constexpr int PV = 1 << PV_LOG;
    constexpr int TS = NT / PV;
    constexpr int NW = NT / 32;
    static_assert(PV >= 4 && PV <= 32 && NT % 32 == 0 && TS >= 1, "bad bin_kernel geometry");
    __shared__ float2 red[NW][PV * VP];
    __shared__ int2 dsc[PUSH ? TS : 1][PUSH ? PV * VP : 1];  // push changes of (S, C) per slice

    const int t = threadIdx.x;
    const int pv = t & (PV - 1);
    const int ts = t >> PV_LOG;
    const long long v = (long long)blockIdx.x * PV + pv;

    if constexpr (PUSH) {
        int32_t ds[VP], dc[VP];
#pragma unroll
        for (int q = 0; q < VP; ++q) ds[q] = dc[q] = 0;
        if (v < nvec) {
            const long long off = v * F::VB;
            const long long slot0 = a.s_first % N;
            for (int f = 0; f < a.nf; ++f) {
                long long slot = slot0 + f;
                if (slot >= N) slot -= N;
                if ((int)(slot % TS) != ts) continue;
                const typename F::Vec xn = F::load(a.frames + off + (long long)f * a.frame_stride);
                const typename F::Vec xo = F::load(a.ring + off + slot * a.slot_stride);
                F::store(a.ring + off + slot * a.slot_stride, xn);
                accumulate<T, true>(ds, dc, xn, xo, (int)((a.s_first + f) & 3));
            }
        }
#pragma unroll
        for (int q = 0; q < VP; ++q) dsc[ts][pv * VP + q] = make_int2(ds[q], dc[q]);
        __syncthreads();
        const long long pb = (long long)blockIdx.x * PV * VP;
        for (int e = t; e < PV * VP; e += NT) {
            const long long p = pb + e;
            if (p >= npix) continue;
            int32_t sum_s = 0, sum_c = 0;
#pragma unroll
            for (int k = 0; k < TS; ++k) {
                const int2 d = dsc[k][e];
                sum_s += d.x;
                sum_c += d.y;
            }
            const int32_t S = a.S[p] + sum_s, C = a.C[p] + sum_c;
            a.S[p] = S;
            a.C[p] = C;
            if (a.amp) a.amp[p] = amplitude(S, C);
            if (a.phase) a.phase[p] = phase_of(S, C);
        }
    }

    // Pixel pairs (2h, 2h+1) share one f32x2 register per accumulator.
    static_assert(VP % 2 == 0, "pixel pairs");
    constexpr int VH = VP / 2;
    f32x2 re2[VH], im2[VH];
#pragma unroll
    for (int h = 0; h < VH; ++h) re2[h] = im2[h] = 0ull;

    if (v < nvec) {
        // with PUSH the ring is read through a.ring, the pointer the push
        // wrote through (the __restrict__ parameter must not alias a store)
        const uint8_t* base = (PUSH ? (const uint8_t*)a.ring : ring) + v * F::VB;
        f32x2 koff[VH];
#pragma unroll
        for (int h = 0; h < VH; ++h)
            koff[h] = f2_bits(__float_as_uint(bin_offset<T>(2 * h)), __float_as_uint(bin_offset<T>(2 * h + 1)));
        constexpr int UF = BinGroup<T>::UF;
        // UF frames of the thread into its partial sums
        auto mac = [&](const typename F::Vec* x, const float2* w, f32x2* pr2, f32x2* pi2) {
#pragma unroll
            for (int u = 0; u < UF; ++u) {
                const f32x2 wr = f2_splat(w[u].x), wi = f2_splat(w[u].y);
                uint32_t b[VP];
                bin_bits<T>(x[u], b);
#pragma unroll
                for (int h = 0; h < VH; ++h) {
                    const f32x2 xf = f2_sub(f2_bits(b[2 * h], b[2 * h + 1]), koff[h]);
                    pr2[h] = f2_fma(xf, wr, pr2[h]);
                    pi2[h] = f2_fma(xf, wi, pi2[h]);
                }
            }
        };
        int j = ts;
        if constexpr (BinGroup<T>::INCR) {
            // 8-pixel vectors: frame pointers advanced by increments (no
            // per-frame 64-bit index products) and whole groups of UF frames
            // loaded without bounds checks, only the last, partial group
            // checking j < N; the arithmetic per frame is that of the
            // indexed loop below
            const long long step = (long long)TS * slot_stride;
            const uint8_t* px = base + (long long)ts * slot_stride;
            const float2* pw = tw + ts;
            while (j < N) {
                f32x2 pr2[VH], pi2[VH];
#pragma unroll
                for (int h = 0; h < VH; ++h) pr2[h] = pi2[h] = 0ull;
                for (int g = 0; g < 16 / UF && j < N; ++g, j += UF * TS) {
                    typename F::Vec x[UF];
                    float2 w[UF];
                    if (j + (UF - 1) * TS < N) {
                        const uint8_t* q = px;
#pragma unroll
                        for (int u = 0; u < UF; ++u) {
                            x[u] = F::load(q);
                            w[u] = __ldg(pw + u * TS);
                            q += step;
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < UF; ++u) {
                            if (j + u * TS < N) {
                                x[u] = F::load(px + u * step);
                                w[u] = __ldg(pw + u * TS);
                            } else {
                                x[u] = F::zero();
                                w[u] = make_float2(0.f, 0.f);
                            }
                        }
                    }
                    px += UF * step;
                    pw += UF * TS;
                    mac(x, w, pr2, pi2);
                }
#pragma unroll
                for (int h = 0; h < VH; ++h) {
                    re2[h] = f2_add(re2[h], pr2[h]);
                    im2[h] = f2_add(im2[h], pi2[h]);
                }
            }
        } else {
            while (j < N) {
                f32x2 pr2[VH], pi2[VH];
#pragma unroll
                for (int h = 0; h < VH; ++h) pr2[h] = pi2[h] = 0ull;
                // Up to 16 frames (16 / UF groups of UF) into the partial.
                for (int g = 0; g < 16 / UF && j < N; ++g, j += UF * TS) {
                    typename F::Vec x[UF];
                    float2 w[UF];
#pragma unroll
                    for (int u = 0; u < UF; ++u) {
                        const int jj = j + u * TS;
                        if (jj < N) {
                            x[u] = F::load(base + (long long)jj * slot_stride);
                            w[u] = __ldg(tw + jj);
                        } else {
                            x[u] = F::zero();
                            w[u] = make_float2(0.f, 0.f);
                        }
                    }
                    mac(x, w, pr2, pi2);
                }
#pragma unroll
                for (int h = 0; h < VH; ++h) {
                    re2[h] = f2_add(re2[h], pr2[h]);
                    im2[h] = f2_add(im2[h], pi2[h]);
                }
            }
        }
    }
    float re[VP], im[VP];
#pragma unroll
    for (int h = 0; h < VH; ++h) {
        const float2 a = f2_split(re2[h]), b = f2_split(im2[h]);
        re[2 * h] = a.x;
        re[2 * h + 1] = a.y;
        im[2 * h] = b.x;
        im[2 * h + 1] = b.y;
    }

    if (PV < 32) {
#pragma unroll
        for (int o = 16; o >= PV; o >>= 1) {
#pragma unroll
            for (int q = 0; q < VP; ++q) {
                re[q] += __shfl_xor_sync(0xFFFFFFFFu, re[q], o);
                im[q] += __shfl_xor_sync(0xFFFFFFFFu, im[q], o);
            }
        }
    }
    const int warp = t >> 5;
    const bool rep = (PV >= 32) || (((t & 31) >> PV_LOG) == 0);
    if (rep) {
#pragma unroll
        for (int q = 0; q < VP; ++q) red[warp][pv * VP + q] = make_float2(re[q], im[q]);
    }
    __syncthreads();
    const long long pbase = (long long)blockIdx.x * PV * VP;
    for (int e = t; e < PV * VP; e += NT) {
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const float2 r = red[w][e];
            a += r.x;
            b += r.y;
        }
        const long long p = pbase + e;
        if (p < npix) {
            if (OUT == kBinPower) {
                out[p] = a * a + b * b;
            } else {
                if (out) out[p] = sqrtf(fmaf(a, a, b * b));
                if (out2) out2[p] = atan2_unit_poly(b, a);
            }
        }
    }
}

// Launch geometry of bin_kernel: log2 of the pixel vectors per CTA. 32
// vectors in 128-thread CTAs (4 time slices) when the grid still has two
// CTAs per SM; fewer vectors in 256-thread CTAs (more time slices, reduced
// with warp shuffles) for small frames so the grid still covers the GPU.
inline int fftbin_pv_log(long long nvec) {
    int pv_log = 5;
    while (pv_log > 2 && (nvec + (1ll << pv_log) - 1) / (1ll << pv_log) < 296) --pv_log;
    return pv_log;
}

// Enqueues bin_kernel over `N` frames (frame j at base + j * stride) of
// frame_bytes bytes and npix pixels each, twiddles tw[j]; writes the power
// into out (OUT = kBinPower) or the amplitude into out and the phase into
// out2 (OUT = kBinAmpPhase; either may be NULL). Frames are read in vectors
// of BinFmt<T>; the last vector may run past frame_bytes (inside the ring
// slot's padding, or exactly to the end when frame_bytes is a multiple of
// 16), and pixels beyond npix are not written.
template <typename T, int OUT>
inline void launch_bin(const uint8_t* base, long long stride, int N, const float2* tw, long long frame_bytes,
                       long long npix, float* out, float* out2, cudaStream_t st) {
    using B = typename BinFmt<T>::type;
    const long long nvec = (frame_bytes + Fmt<B>::VB - 1) / Fmt<B>::VB;
    const int pv_log = fftbin_pv_log(nvec);
    const unsigned grid = (unsigned)((nvec + (1ll << pv_log) - 1) >> pv_log);
    switch (pv_log) {
        case 5: bin_kernel<B, 5, 128, OUT><<<grid, 128, 0, st>>>(base, stride, N, tw, nvec, npix, out, out2, {}); break;
        case 4: bin_kernel<B, 4, 256, OUT><<<grid, 256, 0, st>>>(base, stride, N, tw, nvec, npix, out, out2, {}); break;
        case 3: bin_kernel<B, 3, 256, OUT><<<grid, 256, 0, st>>>(base, stride, N, tw, nvec, npix, out, out2, {}); break;
        default: bin_kernel<B, 2, 256, OUT><<<grid, 256, 0, st>>>(base, stride, N, tw, nvec, npix, out, out2, {}); break;
    }
}

// Twiddles of a lock-in at omega * dt = omega_dt radians per frame for the
// frames with absolute indices s0 .. s0+N-1: tw[j] = (cos, -sin) of
// omega_dt * (s0 + j), evaluated in FP64 and rounded to float.
static __global__ void lockin_table_kernel(float2* __restrict__ tw, int N, double omega_dt, long long s0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double sn, cs;
    sincos(omega_dt * (double)(s0 + j), &sn, &cs);
    tw[j] = make_float2((float)cs, (float)(-sn));
}

}  // namespace qldk
