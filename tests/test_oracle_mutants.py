"""Plants plausible mistakes in copies of the CPU oracle and checks that the
pin suite catches every one (each mutant must fail at least one pin).

The mutants are built on the CPU from text edits of qld_oracle.cpp in a
temporary directory; the real oracle is never modified.
"""
import os
import subprocess

import pytest

import oracle
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "qld_oracle.cpp")

# (name, text to replace, replacement). Each edit is a mistake someone could
# plausibly make when writing the oracle from the paper.
MUTANTS = [
    ("sin_cos_transposed", "sin_r[r] = (int64_t)std::llround(std::sin(arg));",
     "sin_r[r] = (int64_t)std::llround(std::cos(arg));"),
    ("cos_sign_flipped", "cos_r[r] = (int64_t)std::llround(std::cos(arg));",
     "cos_r[r] = -(int64_t)std::llround(std::cos(arg));"),
    ("zero_based_time", "const int64_t s = s0 + i;\n            const int64_t I",
     "const int64_t s = s0 + i - 1;\n            const int64_t I"),
    ("dropped_cos_term", "cos_acc += I * kTables.cos_r[residue4(s)];", ""),
    ("last_frame_dropped", "for (int i = 0; i < N; ++i) {\n            const int64_t s = s0 + i;\n            const int64_t I",
     "for (int i = 0; i < N - 1; ++i) {\n            const int64_t s = s0 + i;\n            const int64_t I"),
    ("phase_sign", "std::atan2((double)(-S[p]), c)", "std::atan2((double)(S[p]), c)"),
    ("phase_operands_swapped", "std::atan2((double)(-S[p]), c)", "std::atan2(c, (double)(-S[p]))"),
    ("amplitude_dropped_term", "std::sqrt(s * s + c * c)", "std::sqrt(s * s + s * s)"),
    ("amplitude_no_sqrt", "std::sqrt(s * s + c * c)", "(s * s + c * c)"),
    ("phase_negzero_branch", "std::atan2((double)(-S[p]), c)", "std::atan2(-s, c)"),
    ("dft_conjugated", "ci[i] = -std::sin(theta);", "ci[i] = std::sin(theta);"),
    ("dft_window_relative_index", "int64_t m = ((k % N) * (s % N)) % N;",
     "int64_t m = ((k % N) * (i % N)) % N;"),
    ("dft_power_term", "power[p] = a * a + b * b;", "power[p] = a * a + b;"),
    ("dft_half_angle", "const double theta = 2.0 * M_PI * (double)m / (double)N;",
     "const double theta = M_PI * (double)m / (double)N;"),
    ("lockin_sin_cos_swapped", "a += I * sin_t[i];\n                b += I * cos_t[i];",
     "a += I * cos_t[i];\n                b += I * sin_t[i];"),
    ("lockin_zero_based_time", "const double arg = omega_dt * (double)(s0 + i);",
     "const double arg = omega_dt * (double)(s0 + i - 1);"),
    ("cnr_ring_includes_source", "            if (in_source) continue;\n            sur += img",
     "            sur += img"),
    ("cnr_deviation_about_source_mean", "const double d = img[(int64_t)r * W + c] - sur;",
     "const double d = img[(int64_t)r * W + c] - src;"),
    ("cnr_ring_one_pixel_short", "for (int r = r0 - m; r < r0 + 2 * m; ++r)\n        for (int c = c0 - m; c < c0 + 2 * m; ++c) {\n            const bool in_source = r >= r0 && r < r0 + m && c >= c0 && c < c0 + m;\n            if (in_source) continue;\n            sur",
     "for (int r = r0 - m; r < r0 + 2 * m; ++r)\n        for (int c = c0 - m; c < c0 + 2 * m - 1; ++c) {\n            const bool in_source = r >= r0 && r < r0 + m && c >= c0 && c < c0 + m;\n            if (in_source) continue;\n            sur"),
    ("conv_flipped_taps", "const int yy = y + ky - 1, xx = x + kx - 1;\n                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;\n                            for (int ci = 0; ci < Cin; ++ci)\n                                acc += in",
     "const int yy = y - ky + 1, xx = x - kx + 1;\n                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;\n                            for (int ci = 0; ci < Cin; ++ci)\n                                acc += in"),
    ("conv_bwd_data_unflipped", "const int yy = y - ky + 1, xx = x - kx + 1;", "const int yy = y + ky - 1, xx = x + kx - 1;"),
    ("conv_wgrad_transposed_channels", "dw[((int64_t)(ky * 3 + kx) * Cin + ci) * Cout + co] = acc;",
     "dw[((int64_t)(ky * 3 + kx) * Cin + (ci + 1) % Cin) * Cout + co] = acc;"),
    ("conv_bias_dropped", "double acc = bias ? bias[co] : 0.0;", "double acc = 0.0;"),
    ("threads_last_range_lost", "for (int t = 0; t < nthreads; ++t) {", "for (int t = 0; t < nthreads - 1; ++t) {"),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, source, name, old, new):
    assert source.count(old) == 1, "mutation site for %s not found exactly once" % name
    mutated = source.replace(old, new)
    src = tmp_path / ("%s.cpp" % name)
    src.write_text(mutated)
    lib = tmp_path / ("lib%s.so" % name)
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread", str(src), "-o", str(lib)],
                   check=True)
    o = oracle.Oracle(str(lib))
    failed = []
    for pin in ALL_PINS:
        try:
            pin(o)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "mutant %s passed every pin" % name
