"""Pins for the CPU oracle: facts fixed by the paper's definitions and by
mathematics, not by the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` instance and raises
AssertionError when that oracle disagrees with the pinned fact. They are run
against the real oracle (tests/test_oracle_pins.py) and against deliberately
broken copies of it (tests/test_oracle_mutants.py), where every copy must fail
at least one pin.

Notation (Methods, "Numerical simulations"; four samples per period):
omega t_s = pi s / 2, sigma_s = sin(pi s / 2) = 1, 0, -1, 0 and
gamma_s = cos(pi s / 2) = 0, -1, 0, 1 for s mod 4 = 1, 2, 3, 0;
S = sum sigma_s x_s, C = sum gamma_s x_s, R = sqrt(S^2 + C^2),
phase = atan2(-S, C); X_k = sum_s x_s exp(-2 pi i k s / N).
"""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _assert_eq(a, b, what):
    a = np.asarray(a)
    b = np.asarray(b)
    if not np.array_equal(a, b):
        raise AssertionError("%s: got %r expected %r" % (what, a.ravel()[:8], b.ravel()[:8]))


def _assert_close(a, b, rtol, atol, what):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if not np.allclose(a, b, rtol=rtol, atol=atol):
        i = int(np.argmax(np.abs(a - b).ravel()))
        raise AssertionError("%s: max err at %d: got %r expected %r" % (what, i, a.ravel()[i], b.ravel()[i]))


def pin_reference_tables(o):
    # sin(0), sin(pi/2), sin(pi), sin(3pi/2) and the cosines of the same angles.
    s, c = o.reference_tables()
    _assert_eq(s, [0, 1, 0, -1], "sin table")
    _assert_eq(c, [1, 0, -1, 0], "cos table")


# Square wave of height a, high on two consecutive residues of s mod 4, on a
# background B. Per period the sums are read off sigma/gamma by hand:
#   high {1,2}: S = a*1 + a*0 = +a,  C = a*0 + a*(-1) = -a, phase = atan2(-a,-a) = -3pi/4
#   high {2,3}: S = 0 - a     = -a,  C = -a + 0       = -a, phase = atan2( a,-a) = +3pi/4
#   high {3,0}: S = -a + 0    = -a,  C = 0 + a        = +a, phase = atan2( a, a) = +pi/4
#   high {0,1}: S = 0 + a     = +a,  C = a + 0        = +a, phase = atan2(-a, a) = -pi/4
# The background contributes nothing (each table sums to zero over a period),
# and R = sqrt(2) a P for P = N/4 periods, whatever the phase.
SQUARE_WAVE_TABLE = {
    (1, 2): (+1, -1, -3 * math.pi / 4),
    (2, 3): (-1, -1, +3 * math.pi / 4),
    (3, 0): (-1, +1, +math.pi / 4),
    (0, 1): (+1, +1, -math.pi / 4),
}


def pin_square_wave(o):
    for (r1, r2), (ks, kc, ph) in SQUARE_WAVE_TABLE.items():
        for N, s0, a, B in [(8, 1, 2, 100), (64, 1, 2, 100), (64, 7, 5, 0), (1024, 1234, 3, 4000),
                            (12, 3, 255, 0)]:
            P = N // 4
            s = np.arange(s0, s0 + N)
            high = ((s % 4) == r1) | ((s % 4) == r2)
            x = (B + a * high).astype(np.uint16).reshape(N, 1)
            S, C, R, phase = o.qld(x, s0=s0)
            _assert_eq(S, [ks * a * P], "square wave S %s N=%d s0=%d" % ((r1, r2), N, s0))
            _assert_eq(C, [kc * a * P], "square wave C %s N=%d s0=%d" % ((r1, r2), N, s0))
            _assert_close(R, [math.sqrt(2.0) * a * P], 1e-14, 0, "square wave R")
            _assert_close(phase, [ph], 0, 1e-14, "square wave phase")


# Integer tone x_s = B + A cos(pi s/2 + phi0) with A cos(phi0) = c and
# A sin(phi0) = d integers: cos(pi s/2 + phi0) expands to
# c*cos(pi s/2) - d*sin(pi s/2). Summing over whole periods, where
# sum sin^2 = sum cos^2 = N/2 and sum sin*cos = sum sin = sum cos = 0:
#   S = -(N/2) d,  C = (N/2) c,  R = (N/2) sqrt(c^2+d^2) = (N/2) A,  phase = phi0.
def pin_tone(o):
    for (c, d) in [(3, 4), (-5, 12), (7, 0), (0, -9), (-8, -6), (1, 1)]:
        for N, s0 in [(4, 1), (16, 2), (64, 3), (256, 4), (40, 1001)]:
            s = np.arange(s0, s0 + N, dtype=np.float64)
            tone = c * np.cos(np.pi * s / 2) - d * np.sin(np.pi * s / 2)
            x = (100 + np.rint(tone)).astype(np.uint8).reshape(N, 1, 1)
            S, C, R, phase = o.qld(x, s0=s0)
            _assert_eq(S.ravel(), [-(N // 2) * d], "tone S (c,d)=%s N=%d s0=%d" % ((c, d), N, s0))
            _assert_eq(C.ravel(), [(N // 2) * c], "tone C (c,d)=%s N=%d s0=%d" % ((c, d), N, s0))
            _assert_close(R.ravel(), [(N / 2) * math.hypot(c, d)], 1e-14, 0, "tone R")
            _assert_close(phase.ravel(), [math.atan2(d, c)], 0, 1e-14, "tone phase")


# Constant background, the Nyquist tone B + a(-1)^s and any period-2 sequence
# carry nothing at f_s/4: S = C = 0 exactly, so R = 0 and phase = 0.
def pin_zeros(o):
    rng = np.random.default_rng(5)
    for N, s0 in [(4, 1), (32, 6), (1024, 99)]:
        s = np.arange(s0, s0 + N)
        cols = [np.full(N, 77), 100 + 9 * (-1) ** s]
        u, v = rng.integers(0, 4096, 2)
        cols.append(np.where(s % 2 == 0, u, v))
        x = np.stack(cols, axis=1).astype(np.uint16)
        S, C, R, phase = o.qld(x, s0=s0)
        _assert_eq(S, [0, 0, 0], "zeros S")
        _assert_eq(C, [0, 0, 0], "zeros C")
        _assert_eq(R, [0.0, 0.0, 0.0], "zeros R")
        _assert_eq(phase, [0.0, 0.0, 0.0], "zeros phase")


# Ramp x_s = s pins the time origin and the signs. Over four frames s0..s0+3,
# by hand from the tables:
#   s0 = 1 mod 4: S = 1 - 3 = -2,  C = -2 + 4 = +2
#   s0 = 2 mod 4: S = -3 + 5 = +2, C = -2 + 4 = +2
#   s0 = 3 mod 4: S = -3 + 5 = +2, C = 4 - 6  = -2
#   s0 = 0 mod 4: S = 5 - 7 = -2,  C = 4 - 6  = -2
# Shifting the block by 4 adds 4 * (table sum) = 0, so a window of P periods
# gives P times these values.
RAMP_TABLE = {1: (-2, +2), 2: (+2, +2), 3: (+2, -2), 0: (-2, -2)}


def pin_ramp(o):
    for s0 in [1, 2, 3, 4, 5, 10, 11, 100, 4093]:
        for N in [4, 8, 64, 256]:
            x = np.arange(s0, s0 + N).astype(np.uint16).reshape(N, 1)
            S, C = o.quadrature_sums(x, s0=s0)
            es, ec = RAMP_TABLE[s0 % 4]
            P = N // 4
            _assert_eq(S, [es * P], "ramp S s0=%d N=%d" % (s0, N))
            _assert_eq(C, [ec * P], "ramp C s0=%d N=%d" % (s0, N))


# The sums are linear in the frames and blind to a constant offset (a whole
# number of periods sums each table to 0), exactly, in integers:
# S(a x + b y + c) = a S(x) + b S(y), and the same for C; the DFT bin is
# linear too and its offset term vanishes for k != 0.
def pin_linearity_and_offset(o):
    rng = np.random.default_rng(21)
    for N, s0 in [(8, 3), (64, 1), (256, 1002)]:
        x = rng.integers(0, 1000, (N, 5)).astype(np.int64)
        y = rng.integers(0, 1000, (N, 5)).astype(np.int64)
        z = 3 * x + 2 * y + 7  # <= 5007: fits uint16
        Sx, Cx = o.quadrature_sums(x.astype(np.uint16), s0=s0)
        Sy, Cy = o.quadrature_sums(y.astype(np.uint16), s0=s0)
        Sz, Cz = o.quadrature_sums(z.astype(np.uint16), s0=s0)
        _assert_eq(Sz, 3 * np.asarray(Sx) + 2 * np.asarray(Sy), "linearity S N=%d" % N)
        _assert_eq(Cz, 3 * np.asarray(Cx) + 2 * np.asarray(Cy), "linearity C N=%d" % N)
        for k in (1, N // 4, N // 2 - 1):
            rx, ix, _ = o.dft_bin(x.astype(np.uint16), k, s0=s0)
            ry, iy, _ = o.dft_bin(y.astype(np.uint16), k, s0=s0)
            rz, iz, _ = o.dft_bin(z.astype(np.uint16), k, s0=s0)
            scale = float(np.abs(z).sum(axis=0).max())
            _assert_close(rz, 3 * np.asarray(rx) + 2 * np.asarray(ry), 0, 1e-12 * scale, "DFT linearity re")
            _assert_close(iz, 3 * np.asarray(ix) + 2 * np.asarray(iy), 0, 1e-12 * scale, "DFT linearity im")


# Noise only: for frames of i.i.d. integer noise of variance v, S and C are
# sums of N/2 terms +-x each, so E[S^2] = E[C^2] = (N/2) v and E[R^2] = N v.
# Uniform integers on 0..M have v = ((M+1)^2 - 1) / 12; over 20,000 pixels the
# sample mean of R^2 is within 3 % of N v with overwhelming probability (its
# relative standard deviation is about 1 / sqrt(20000) = 0.7 %).
def pin_noise_power(o):
    rng = np.random.default_rng(22)
    M = 255
    v = ((M + 1) ** 2 - 1) / 12.0
    for N, s0 in [(16, 1), (64, 7)]:
        x = rng.integers(0, M + 1, (N, 20000)).astype(np.uint16)
        S, C = o.quadrature_sums(x, s0=s0)
        S = np.asarray(S, np.float64)
        C = np.asarray(C, np.float64)
        r2 = float(np.mean(S * S + C * C))
        if abs(r2 / (N * v) - 1) > 0.03:
            raise AssertionError("noise power N=%d: mean R^2 %.1f, expected N v = %.1f" % (N, r2, N * v))
        if abs(np.mean(S * S) / (N / 2 * v) - 1) > 0.04 or abs(np.mean(C * C) / (N / 2 * v) - 1) > 0.04:
            raise AssertionError("noise power N=%d: S and C should each carry half" % N)


# Against numpy's FFT of the window y_i = x_{s0+i}: Y_k = sum_i y_i e^{-2 pi i k i/N},
# so the absolute-index bin is X_k = e^{-2 pi i k s0 / N} Y_k.
def pin_dft_vs_numpy(o):
    rng = np.random.default_rng(11)
    for N in [4, 8, 12, 16, 20]:
        for s0 in [1, 3, 22]:
            x = rng.integers(0, 4096, size=(N, 5)).astype(np.uint16)
            Y = np.fft.fft(x.astype(np.float64), axis=0)
            for k in range(N):
                re, im, pw = o.dft_bin(x, k, s0=s0)
                X = Y[k] * np.exp(-2j * np.pi * k * s0 / N)
                scale = float(x.astype(np.float64).sum())
                _assert_close(re, X.real, 0, 1e-12 * scale, "dft re N=%d k=%d s0=%d" % (N, k, s0))
                _assert_close(im, X.imag, 0, 1e-12 * scale, "dft im N=%d k=%d s0=%d" % (N, k, s0))
                _assert_close(pw, np.abs(Y[k]) ** 2, 1e-12, 1e-12 * scale ** 2, "dft power")


# Parseval: sum_k |X_k|^2 = N sum_s x_s^2.
def pin_parseval(o):
    rng = np.random.default_rng(12)
    for N in [4, 8, 16, 24]:
        x = rng.integers(0, 256, size=(N, 7)).astype(np.uint8)
        tot = np.zeros(7)
        for k in range(N):
            tot += o.dft_bin(x, k, s0=2)[2]
        _assert_close(tot, N * (x.astype(np.float64) ** 2).sum(axis=0), 1e-12, 0, "parseval")


# X_{N/4} = sum x_s (cos(pi s/2) - i sin(pi s/2)) = C - i S, X_0 = sum x_s,
# X_{N/2} = sum (-1)^s x_s.
def pin_dft_identities(o):
    rng = np.random.default_rng(13)
    for N, s0 in [(8, 1), (64, 5), (1024, 3)]:
        x = rng.integers(0, 4096, size=(N, 6)).astype(np.uint16)
        S, C = o.quadrature_sums(x, s0=s0)
        re, im, pw = o.dft_bin(x, N // 4, s0=s0)
        scale = float(x.astype(np.float64).sum())
        _assert_close(re, C, 0, 1e-12 * scale, "X_{N/4} real part = C")
        _assert_close(im, -S, 0, 1e-12 * scale, "X_{N/4} imaginary part = -S")
        _assert_close(pw, S.astype(np.float64) ** 2 + C.astype(np.float64) ** 2, 1e-12, 1e-9,
                      "|X_{N/4}|^2 = S^2 + C^2")
        re0, im0, _ = o.dft_bin(x, 0, s0=s0)
        _assert_close(re0, x.astype(np.float64).sum(axis=0), 0, 1e-9, "X_0")
        _assert_close(im0, 0.0, 0, 1e-9, "X_0 imaginary")
        sgn = (-1.0) ** np.arange(s0, s0 + N)
        reh, imh, _ = o.dft_bin(x, N // 2, s0=s0)
        _assert_close(reh, (sgn[:, None] * x).sum(axis=0), 0, 1e-9 * scale, "X_{N/2}")
        _assert_close(imh, 0.0, 0, 1e-9 * scale, "X_{N/2} imaginary")


def pin_amplitude_phase_cases(o):
    S = np.array([0, 0, 3, -1, 0, 5, -7], np.int64)
    C = np.array([0, -4, 4, 0, 9, 0, -7], np.int64)
    R, ph = o.amplitude_phase(S, C)
    _assert_close(R, [0, 4, 5, 1, 9, 5, 7 * math.sqrt(2)], 1e-15, 0, "R cases")
    # S = 0, C < 0 lies on the branch cut: the phase is +pi (range (-pi, pi]).
    _assert_close(ph, [0, math.pi, math.atan2(-3, 4), math.pi / 2, 0, -math.pi / 2, 3 * math.pi / 4],
                  0, 1e-15, "phase cases")
    big = np.array([2 ** 31 - 1], np.int64)
    Rb, _ = o.amplitude_phase(big, big)
    _assert_close(Rb, [(2 ** 31 - 1) * math.sqrt(2)], 1e-15, 0, "R at the int32 limit")


def pin_threads_agree(o):
    rng = np.random.default_rng(14)
    x = rng.integers(0, 65536, size=(32, 1001)).astype(np.uint16)
    S1, C1 = o.quadrature_sums(x, s0=9, nthreads=1)
    S4, C4 = o.quadrature_sums(x, s0=9, nthreads=4)
    _assert_eq(S4, S1, "threaded S")
    _assert_eq(C4, C1, "threaded C")
    p1 = o.dft_bin(x, 3, s0=9, nthreads=1)[2]
    p4 = o.dft_bin(x, 3, s0=9, nthreads=7)[2]
    _assert_eq(p4, p1, "threaded dft")


def load_golden(name):
    """Parse a tests/golden fixture: '#' comments, then 'key: v v v' lines."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, vals = line.split(":", 1)
            out[key.strip()] = [int(v) for v in vals.split()]
    return out


def pin_golden_worked_example(o):
    g = load_golden("qld_worked_example.txt")
    N = g["N"][0]
    npix = g["npix"][0]
    s0 = g["s0"][0]
    x = np.array(g["frames"], np.uint16).reshape(N, npix)
    S, C = o.quadrature_sums(x, s0=s0)
    _assert_eq(S, g["S"], "golden S")
    _assert_eq(C, g["C"], "golden C")
    R, _ = o.amplitude_phase(S, C)
    _assert_close(R ** 2, g["R2"], 1e-13, 0, "golden R^2")
    _assert_close(o.dft_bin(x, 0, s0=s0)[0], g["X0"], 0, 1e-9, "golden X_0")
    _assert_close(o.dft_bin(x, N // 2, s0=s0)[0], g["XN2"], 0, 1e-9, "golden X_{N/2}")


# General-frequency lock-in (Methods, Fig. 1 frequencies). At omega dt = pi/2
# it is the four-samples-per-period QLD.
def pin_lockin_general_quarter_rate(o):
    rng = np.random.default_rng(21)
    x = rng.integers(0, 4096, size=(64, 9)).astype(np.uint16)
    S, C, R, ph = o.lockin_general(x, math.pi / 2, s0=7)
    Si, Ci = o.quadrature_sums(x, s0=7)
    tol = 1e-12 * float(x.astype(np.float64).sum())
    _assert_close(S, Si, 0, tol, "general lock-in at pi/2: S")
    _assert_close(C, Ci, 0, tol, "general lock-in at pi/2: C")
    R_i, ph_i = o.amplitude_phase(Si, Ci)
    _assert_close(R, R_i, 1e-12, 0, "general lock-in at pi/2: R")
    _assert_close(ph, ph_i, 0, 1e-9, "general lock-in at pi/2: phase")


# Tone x_s = B + A cos(w s + phi0), rounded to integers, with w = 2 pi p / N so the
# window holds p whole periods. Over whole periods sum sin(w s) = sum cos(w s) = 0,
# sum sin^2 = sum cos^2 = N/2 and sum sin cos = 0, so the lock-in at w gives
# S = -(N/2) A sin(phi0), C = (N/2) A cos(phi0), R = (N/2) A; at any other
# w' = 2 pi p' / N (p' != p, N - p, 0) S = C = 0. Rounding each sample moves S
# and C by at most N/2.
def pin_lockin_general_tone_and_orthogonality(o):
    for N, p, pw, s0, phi0 in [(64, 5, 9, 1, 0.7), (82, 19, 23, 4, -2.0), (100, 23, 29, 11, 2.9)]:
        A, B = 10000.0, 20000.0
        s = np.arange(s0, s0 + N, dtype=np.float64)
        w = 2 * math.pi * p / N
        x = np.rint(B + A * np.cos(w * s + phi0)).astype(np.uint16).reshape(N, 1)
        S, C, R, ph = o.lockin_general(x, w, s0=s0)
        bound = N / 2 + 1e-6
        _assert_close(S, [-(N / 2) * A * math.sin(phi0)], 0, bound, "tone S")
        _assert_close(C, [(N / 2) * A * math.cos(phi0)], 0, bound, "tone C")
        _assert_close(R, [(N / 2) * A], 0, bound, "tone R")
        _assert_close(ph, [phi0], 0, 2 * bound / (N / 2 * A), "tone phase")
        So, Co, Ro, _ = o.lockin_general(x, 2 * math.pi * pw / N, s0=s0)
        _assert_close(Ro, [0.0], 0, math.sqrt(2) * bound, "off-frequency tone gives zero")


# At w = 2 pi k / N the lock-in is the DFT bin: C - iS = X_k (numpy's FFT of the
# window times exp(-2 pi i k s0 / N) for the absolute frame index).
def pin_lockin_general_is_dft_bin(o):
    rng = np.random.default_rng(22)
    for N, s0 in [(12, 1), (41, 5), (82, 2)]:
        x = rng.integers(0, 256, size=(N, 4)).astype(np.uint8)
        Y = np.fft.fft(x.astype(np.float64), axis=0)
        for k in [0, 1, N // 3, N - 1]:
            S, C, R, ph = o.lockin_general(x, 2 * math.pi * k / N, s0=s0)
            X = Y[k] * np.exp(-2j * np.pi * k * s0 / N)
            scale = float(x.astype(np.float64).sum())
            _assert_close(C, X.real, 0, 1e-11 * scale, "lock-in = DFT real part")
            _assert_close(-S, X.imag, 0, 1e-11 * scale, "lock-in = DFT imaginary part")


def _load_cnr_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "cnr_surround_example.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split(":", 1)
                vals[k.strip()] = [int(t) for t in v.split()]
    H, W = vals["H"][0], vals["W"][0]
    A = np.array([vals["A_row%02d" % r] for r in range(H)], np.float64)
    B = np.array([vals["B_row%02d" % r] for r in range(H)], np.float64)
    return vals, A, B


def pin_cnr_worked_example(o):
    vals, A, B = _load_cnr_golden()
    r0, c0, m = vals["r0"][0], vals["c0"][0], vals["m"][0]
    _assert_close([o.cnr(A, r0, c0, m) ** 2], vals["A_cnr_sq"], 1e-12, 0, "CNR case A")
    _assert_close([o.cnr(B, r0, c0, m) ** 2], vals["B_cnr_sq"], 1e-12, 0, "CNR case B")
    # CNR is unchanged by an offset, a positive scale, or pixels outside the ring
    A2 = 3.5 * A + 17.0
    A2[0, :] = -1e6
    A2[:, -1] = 1e6
    _assert_close([o.cnr(A2, r0, c0, m)], [8.0], 1e-12, 0, "CNR invariances")
    try:
        o.cnr(A, 1, 1, 4)
    except ValueError:
        pass
    else:
        raise AssertionError("a ring leaving the image must be rejected")


# 3x3 convolution (learned short-window network). The backward-data map is
# the adjoint of the forward map: <conv(x), g> = <x, conv_bwd_data(g)>; the
# weight gradient follows from linearity in w: <dw(x, g), v> = <conv(x; v), g>
# (bias-free); the bias gradient is the sum of g.
def pin_conv_adjoint_and_linearity(o):
    rng = np.random.default_rng(31)
    for B, H, W, Cin, Cout in [(1, 5, 7, 2, 3), (2, 4, 4, 3, 1), (1, 1, 6, 1, 2)]:
        x = rng.standard_normal((B, H, W, Cin))
        w = rng.standard_normal((3, 3, Cin, Cout))
        g = rng.standard_normal((B, H, W, Cout))
        v = rng.standard_normal((3, 3, Cin, Cout))
        y = o.conv3x3(x, w)
        dx, dw, db = o.conv3x3_backward(x, w, g)
        _assert_close([np.sum(y * g)], [np.sum(x * dx)], 1e-12, 1e-12, "conv adjoint")
        _assert_close([np.sum(dw * v)], [np.sum(o.conv3x3(x, v) * g)], 1e-12, 1e-12, "weight-gradient linearity")
        _assert_close(db, g.sum(axis=(0, 1, 2)), 1e-12, 1e-12, "bias gradient")
        bias = rng.standard_normal(Cout)
        _assert_close(o.conv3x3(x, w, bias), y + bias, 1e-12, 1e-12, "bias added")


# Closed forms: the delta kernel (w[1][1] = identity) copies the input; an
# all-ones kernel on a constant c image of Cin channels gives 9 Cin c inside,
# 6 Cin c on edges and 4 Cin c at corners (zero padding); against scipy's
# correlate2d (a library routine) for one channel pair.
def pin_conv_closed_forms(o):
    rng = np.random.default_rng(32)
    x = rng.standard_normal((2, 6, 5, 3))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[1, 1, c, c] = 1.0
    _assert_close(o.conv3x3(x, w), x, 0, 1e-15, "delta kernel")
    c = 2.5
    y = o.conv3x3(np.full((1, 5, 6, 4), c), np.ones((3, 3, 4, 1)))[0, :, :, 0]
    exp = np.full((5, 6), 9 * 4 * c)
    exp[0, :] = exp[-1, :] = 6 * 4 * c
    exp[:, 0] = exp[:, -1] = 6 * 4 * c
    exp[0, 0] = exp[0, -1] = exp[-1, 0] = exp[-1, -1] = 4 * 4 * c
    _assert_close(y, exp, 1e-14, 0, "constant image, all-ones kernel")
    from scipy.signal import correlate2d

    x1 = rng.standard_normal((1, 7, 9, 1))
    w1 = rng.standard_normal((3, 3, 1, 1))
    _assert_close(o.conv3x3(x1, w1)[0, :, :, 0], correlate2d(x1[0, :, :, 0], w1[:, :, 0, 0], mode="same"), 1e-12,
                  1e-12, "scipy correlate2d")


ALL_PINS = [
    pin_reference_tables,
    pin_square_wave,
    pin_tone,
    pin_zeros,
    pin_linearity_and_offset,
    pin_noise_power,
    pin_ramp,
    pin_dft_vs_numpy,
    pin_parseval,
    pin_dft_identities,
    pin_amplitude_phase_cases,
    pin_threads_agree,
    pin_golden_worked_example,
    pin_lockin_general_quarter_rate,
    pin_lockin_general_tone_and_orthogonality,
    pin_lockin_general_is_dft_bin,
    pin_cnr_worked_example,
    pin_conv_adjoint_and_linearity,
    pin_conv_closed_forms,
]
