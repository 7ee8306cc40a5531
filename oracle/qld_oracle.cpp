// qld_oracle.cpp -- CPU oracle for quadrature lock-in discrimination (QLD).
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct
// restatement of what the QLD hot path computes, written from the paper's
// definitions (Methods, "Numerical simulations"; Supplementary Information,
// "Timing sequence for hybrid parallelisation"). Only the test suite, the
// smoke check in __graft_entry__ and bench.py's CPU-baseline leg may load it.
// It shares no code, header, table or helper with the CUDA library, and it
// never includes anything from it.
//
// Conventions (readings of points the paper leaves open):
//  * Sampling at four samples per modulation period: omega * t_s = pi * s / 2.
//  * s is the absolute 1-based index of a frame in the stream (Methods:
//    t_s = s * dt, s = 1, 2, ...). A window of N frames whose first frame
//    has absolute index s0 covers s = s0 .. s0 + N - 1.
//  * Quadrature sums (Methods, the equation defining R(j,k)):
//        S = sum_s I(s) * sin(omega t_s),   C = sum_s I(s) * cos(omega t_s)
//    computed exactly in int64, from scratch for every window.
//  * R = sqrt(S^2 + C^2) (Methods); phase = atan2(-S, C), the argument of the
//    DFT bin k = N/4 under the absolute-index convention (the paper defines no
//    phase image). S = C = 0 gives phase 0.
//  * DFT bin (Methods, FFT discrimination): X_k = sum_s I(s) exp(-2 pi i k s / N)
//    over the window, with (k * s) mod N reduced in integers before the FP64
//    cos/sin; the map is |X_k|^2.
//  * General-frequency lock-in (Methods, Fig. 1 frequencies): the same sums
//    with sin/cos(omega s dt) tabulated in FP64 for any omega dt.
//  * Contrast-to-noise ratio (Methods, CNR equation and the "surround" figure).
//
// Every array is a window of N frames laid out frame-major: frame i of the
// window starts at x + i * stride (elements), and pixels 0 .. npix-1 of a
// frame are contiguous. All arithmetic is int64 or IEEE double.

#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

// Precomputed reference arrays (Methods: "values of sin(omega t_s) and
// cos(omega t_s) being read from pre-calculated arrays"; SI item 1: tables
// "appropriate for the choice of lock-in and sampling frequencies"). With
// omega t_s = pi s / 2 the functions have period 4 in s and take the exact
// integer values sin(pi r / 2), cos(pi r / 2) for r = s mod 4.
struct RefTables {
    int64_t sin_r[4];
    int64_t cos_r[4];
    RefTables() {
        for (int r = 0; r < 4; ++r) {
            const double arg = M_PI * 0.5 * (double)r;
            sin_r[r] = (int64_t)std::llround(std::sin(arg));
            cos_r[r] = (int64_t)std::llround(std::cos(arg));
        }
    }
};
const RefTables kTables;

inline int residue4(int64_t s) { return (int)(((s % 4) + 4) % 4); }

template <typename T>
void quadrature_sums(const T* x, int64_t stride, int64_t npix, int N, int64_t s0,
                     int64_t* S, int64_t* C) {
    for (int64_t p = 0; p < npix; ++p) {
        int64_t sin_acc = 0, cos_acc = 0;
        for (int i = 0; i < N; ++i) {
            const int64_t s = s0 + i;
            const int64_t I = (int64_t)x[(int64_t)i * stride + p];
            sin_acc += I * kTables.sin_r[residue4(s)];
            cos_acc += I * kTables.cos_r[residue4(s)];
        }
        S[p] = sin_acc;
        C[p] = cos_acc;
    }
}

template <typename T>
void dft_bin(const T* x, int64_t stride, int64_t npix, int N, int64_t s0, int64_t k,
             double* re, double* im, double* power) {
    // Per-window twiddles exp(-2 pi i k s / N) for s = s0 .. s0+N-1, with the
    // angle index (k*s) mod N reduced exactly in integers.
    std::vector<double> cr(N), ci(N);
    for (int i = 0; i < N; ++i) {
        const int64_t s = s0 + i;
        int64_t m = ((k % N) * (s % N)) % N;
        if (m < 0) m += N;
        const double theta = 2.0 * M_PI * (double)m / (double)N;
        cr[i] = std::cos(theta);
        ci[i] = -std::sin(theta);
    }
    for (int64_t p = 0; p < npix; ++p) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < N; ++i) {
            const double I = (double)x[(int64_t)i * stride + p];
            a += I * cr[i];
            b += I * ci[i];
        }
        if (re) re[p] = a;
        if (im) im[p] = b;
        if (power) power[p] = a * a + b * b;
    }
}

// Splits pixels [0, npix) into nthreads contiguous ranges (rows of the image
// are contiguous runs of pixels, so this is a row partition) and runs fn on
// each range in its own std::thread.
template <typename Fn>
void run_partitioned(int64_t npix, int nthreads, Fn fn) {
    if (nthreads <= 1 || npix < 2) {
        fn((int64_t)0, npix);
        return;
    }
    if ((int64_t)nthreads > npix) nthreads = (int)npix;
    std::vector<std::thread> pool;
    pool.reserve(nthreads);
    const int64_t chunk = (npix + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        const int64_t lo = (int64_t)t * chunk;
        const int64_t hi = lo + chunk < npix ? lo + chunk : npix;
        if (lo >= hi) break;
        pool.emplace_back([=] { fn(lo, hi - lo); });
    }
    for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

// Reference arrays sin(pi r/2), cos(pi r/2), r = 0..3 (Methods; SI item 1).
void orc_reference_tables(int64_t* sin_r, int64_t* cos_r) {
    for (int r = 0; r < 4; ++r) {
        sin_r[r] = kTables.sin_r[r];
        cos_r[r] = kTables.cos_r[r];
    }
}

// Quadrature sums S, C of a window (Methods, definition of R(j,k)), int64.
// pixfmt 1 = uint8 frames, 2 = uint16 frames. Returns 0, or -1 on bad args.
int orc_quadrature_sums(const void* x, int pixfmt, int64_t stride, int64_t npix, int N,
                        int64_t s0, int64_t* S, int64_t* C, int nthreads) {
    if (!x || !S || !C || N < 1 || npix < 0 || stride < npix) return -1;
    if (pixfmt == 1) {
        const uint8_t* xb = (const uint8_t*)x;
        run_partitioned(npix, nthreads, [&](int64_t lo, int64_t n) {
            quadrature_sums(xb + lo, stride, n, N, s0, S + lo, C + lo);
        });
    } else if (pixfmt == 2) {
        const uint16_t* xh = (const uint16_t*)x;
        run_partitioned(npix, nthreads, [&](int64_t lo, int64_t n) {
            quadrature_sums(xh + lo, stride, n, N, s0, S + lo, C + lo);
        });
    } else {
        return -1;
    }
    return 0;
}

// Amplitude R = [S^2 + C^2]^(1/2) (Methods) and phase atan2(-S, C), FP64.
// The negation is taken on the integer so that S = 0 gives +0 and the phase
// lies in (-pi, pi].
int orc_amplitude_phase(const int64_t* S, const int64_t* C, int64_t npix, double* R,
                        double* phase) {
    if (!S || !C || npix < 0) return -1;
    for (int64_t p = 0; p < npix; ++p) {
        const double s = (double)S[p];
        const double c = (double)C[p];
        if (R) R[p] = std::sqrt(s * s + c * c);
        if (phase) {
            if (S[p] == 0 && C[p] == 0) {
                phase[p] = 0.0;
            } else {
                phase[p] = std::atan2((double)(-S[p]), c);
            }
        }
    }
    return 0;
}

// DFT bin k of each pixel's time series over the window (Methods, FFT
// discrimination): X_k = sum_s I(s) exp(-2 pi i k s / N), FP64. Any of re,
// im, power may be NULL. k is taken modulo N.
int orc_dft_bin(const void* x, int pixfmt, int64_t stride, int64_t npix, int N, int64_t s0,
                int64_t k, double* re, double* im, double* power, int nthreads) {
    if (!x || N < 1 || npix < 0 || stride < npix) return -1;
    auto off = [](double* a, int64_t lo) { return a ? a + lo : (double*)nullptr; };
    if (pixfmt == 1) {
        const uint8_t* xb = (const uint8_t*)x;
        run_partitioned(npix, nthreads, [&](int64_t lo, int64_t n) {
            dft_bin(xb + lo, stride, n, N, s0, k, off(re, lo), off(im, lo), off(power, lo));
        });
    } else if (pixfmt == 2) {
        const uint16_t* xh = (const uint16_t*)x;
        run_partitioned(npix, nthreads, [&](int64_t lo, int64_t n) {
            dft_bin(xh + lo, stride, n, N, s0, k, off(re, lo), off(im, lo), off(power, lo));
        });
    } else {
        return -1;
    }
    return 0;
}

// Lock-in at an arbitrary frequency (Methods, R(j,k) with the values of
// sin(omega_i t_s) and cos(omega_i t_s) read from pre-calculated arrays;
// t_s = s dt). omega_dt = omega * dt in radians per frame; the window holds
// frames s0 .. s0+N-1. S = sum I sin(omega t_s), C = sum I cos(omega t_s),
// R = sqrt(S^2 + C^2), phase = atan2(-S, C), all FP64. Any output may be NULL.
int orc_lockin_general(const void* x, int pixfmt, int64_t stride, int64_t npix, int N, int64_t s0,
                       double omega_dt, double* S, double* C, double* R, double* phase, int nthreads) {
    if (!x || N < 1 || npix < 0 || stride < npix || (pixfmt != 1 && pixfmt != 2)) return -1;
    std::vector<double> sin_t(N), cos_t(N);
    for (int i = 0; i < N; ++i) {
        const double arg = omega_dt * (double)(s0 + i);
        sin_t[i] = std::sin(arg);
        cos_t[i] = std::cos(arg);
    }
    run_partitioned(npix, nthreads, [&](int64_t lo, int64_t n) {
        for (int64_t p = lo; p < lo + n; ++p) {
            double a = 0.0, b = 0.0;
            for (int i = 0; i < N; ++i) {
                const int64_t idx = (int64_t)i * stride + p;
                const double I = pixfmt == 1 ? (double)((const uint8_t*)x)[idx] : (double)((const uint16_t*)x)[idx];
                a += I * sin_t[i];
                b += I * cos_t[i];
            }
            if (S) S[p] = a;
            if (C) C[p] = b;
            if (R) R[p] = std::sqrt(a * a + b * b);
            if (phase) phase[p] = (a == 0.0 && b == 0.0) ? 0.0 : std::atan2(-a, b);
        }
    });
    return 0;
}

// Contrast-to-noise ratio (Methods, "Estimation of Contrast-to-noise-ratio"):
// the source is the m x m block with top-left corner (r0, c0) of the H x W
// image; the surround is the m-pixel-wide square ring around it, i.e. the
// 3m x 3m block centred on the source minus the source (8 m^2 pixels).
// CNR = (mean_source - mean_surround) / sqrt(mean over the surround of
// (I - mean_surround)^2). Returns -1 if the ring leaves the image.
int orc_cnr(const double* img, int H, int W, int r0, int c0, int m, double* cnr) {
    if (!img || !cnr || m < 1 || r0 - m < 0 || c0 - m < 0 || r0 + 2 * m > H || c0 + 2 * m > W) return -1;
    double src = 0.0;
    for (int r = r0; r < r0 + m; ++r)
        for (int c = c0; c < c0 + m; ++c) src += img[(int64_t)r * W + c];
    src /= (double)m * m;
    double sur = 0.0;
    int64_t count = 0;
    for (int r = r0 - m; r < r0 + 2 * m; ++r)
        for (int c = c0 - m; c < c0 + 2 * m; ++c) {
            const bool in_source = r >= r0 && r < r0 + m && c >= c0 && c < c0 + m;
            if (in_source) continue;
            sur += img[(int64_t)r * W + c];
            ++count;
        }
    sur /= (double)count;
    double var = 0.0;
    for (int r = r0 - m; r < r0 + 2 * m; ++r)
        for (int c = c0 - m; c < c0 + 2 * m; ++c) {
            const bool in_source = r >= r0 && r < r0 + m && c >= c0 && c < c0 + m;
            if (in_source) continue;
            const double d = img[(int64_t)r * W + c] - sur;
            var += d * d;
        }
    var /= (double)count;
    *cnr = (src - sur) / std::sqrt(var);
    return 0;
}

// ---- 3x3 convolution (the learned short-window network) ------------------
// Not in the paper: the network maps short-window I/Q maps to the long-window
// amplitude. Cross-correlation with zero padding 1, NHWC activations and
// weights w[ky][kx][ci][co]:
//   out[b][y][x][co] = bias[co] + sum_{ky,kx,ci} in[b][y+ky-1][x+kx-1][ci] w[ky][kx][ci][co]
// Backward of a loss L with g = dL/dout:
//   din[b][y][x][ci]  = sum_{ky,kx,co} g[b][y-ky+1][x-kx+1][co] w[ky][kx][ci][co]
//   dw[ky][kx][ci][co] = sum_{b,y,x} in[b][y+ky-1][x+kx-1][ci] g[b][y][x][co]
//   dbias[co]          = sum_{b,y,x} g[b][y][x][co]
// All FP64, plain loops in that order; out-of-range taps are zero.
int orc_conv3x3_fwd(const double* in, const double* w, const double* bias, int B, int H, int W, int Cin, int Cout,
                    double* out) {
    if (!in || !w || !out || B < 1 || H < 1 || W < 1 || Cin < 1 || Cout < 1) return -1;
    for (int b = 0; b < B; ++b)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int co = 0; co < Cout; ++co) {
                    double acc = bias ? bias[co] : 0.0;
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            const int yy = y + ky - 1, xx = x + kx - 1;
                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            for (int ci = 0; ci < Cin; ++ci)
                                acc += in[(((int64_t)b * H + yy) * W + xx) * Cin + ci] *
                                       w[((int64_t)(ky * 3 + kx) * Cin + ci) * Cout + co];
                        }
                    out[(((int64_t)b * H + y) * W + x) * Cout + co] = acc;
                }
    return 0;
}

int orc_conv3x3_bwd(const double* in, const double* w, const double* g, int B, int H, int W, int Cin, int Cout,
                    double* din, double* dw, double* dbias) {
    if (!in || !w || !g || B < 1 || H < 1 || W < 1 || Cin < 1 || Cout < 1) return -1;
    if (din) {
        for (int b = 0; b < B; ++b)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    for (int ci = 0; ci < Cin; ++ci) {
                        double acc = 0.0;
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx) {
                                const int yy = y - ky + 1, xx = x - kx + 1;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                                for (int co = 0; co < Cout; ++co)
                                    acc += g[(((int64_t)b * H + yy) * W + xx) * Cout + co] *
                                           w[((int64_t)(ky * 3 + kx) * Cin + ci) * Cout + co];
                            }
                        din[(((int64_t)b * H + y) * W + x) * Cin + ci] = acc;
                    }
    }
    if (dw) {
        for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx)
                for (int ci = 0; ci < Cin; ++ci)
                    for (int co = 0; co < Cout; ++co) {
                        double acc = 0.0;
                        for (int b = 0; b < B; ++b)
                            for (int y = 0; y < H; ++y)
                                for (int x = 0; x < W; ++x) {
                                    const int yy = y + ky - 1, xx = x + kx - 1;
                                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                                    acc += in[(((int64_t)b * H + yy) * W + xx) * Cin + ci] *
                                           g[(((int64_t)b * H + y) * W + x) * Cout + co];
                                }
                        dw[((int64_t)(ky * 3 + kx) * Cin + ci) * Cout + co] = acc;
                    }
    }
    if (dbias) {
        for (int co = 0; co < Cout; ++co) {
            double acc = 0.0;
            for (int64_t p = 0; p < (int64_t)B * H * W; ++p) acc += g[p * Cout + co];
            dbias[co] = acc;
        }
    }
    return 0;
}

}  // extern "C"
