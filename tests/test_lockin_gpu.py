"""General-frequency lock-in (qld_lockin_table + qld_lockin_frames) against
the CPU oracle, and the Fig. 1 analog: QLD and FFT discrimination of the
23 Hz source among sources at 20, 23, 26 and 29 Hz, scored by the paper's
contrast-to-noise ratio."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from qld_check import check_lockin, check_power

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gpu_lockin(x, H, W, omega_dt, s0=1):
    """Amplitude and phase images of the lock-in over the frames x (N, H*W)."""
    N = x.shape[0]
    fmt = 1 if x.dtype == np.uint8 else 2
    dev = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(N, -1)).cuda()
    table = torch.empty(2 * N, dtype=torch.float32, device="cuda")
    amp = torch.empty(H * W, dtype=torch.float32, device="cuda")
    ph = torch.empty_like(amp)
    q.qld_lockin_table(omega_dt, s0, N, table)
    q.qld_lockin_frames(dev, H, W, N, fmt, table, amp, ph)
    torch.cuda.synchronize()
    return amp.cpu().numpy(), ph.cpu().numpy(), table.cpu().numpy()


@pytest.mark.parametrize("H,W,N,fmt,omega_dt,s0", [
    (64, 64, 82, 2, 2 * math.pi * 23 / 100, 1),
    (40, 96, 41, 1, 2 * math.pi * 29 / 100, 5),
    (128, 256, 1000, 2, 0.3, 123456),
    (16, 8, 7, 2, 2.5, 1),
    (1, 8, 1, 2, 1.0, 3),
    (256, 320, 64, 1, math.pi / 2, 9),
])
def test_lockin_matches_oracle(H, W, N, fmt, omega_dt, s0):
    rng = np.random.default_rng(N + H)
    hi = 256 if fmt == 1 else 4096
    x = rng.integers(0, hi, size=(N, H * W)).astype(np.uint8 if fmt == 1 else np.uint16)
    amp, ph, table = gpu_lockin(x, H, W, omega_dt, s0)
    S, C, R, phr = oracle.lockin_general(x, omega_dt, s0=s0)
    check_lockin(amp, ph, R, phr, x.astype(np.int64).sum(axis=0), "N=%d" % N)
    arg = omega_dt * np.arange(s0, s0 + N, dtype=np.float64)
    assert np.abs(table[0::2] - np.cos(arg)).max() <= 6e-8
    assert np.abs(table[1::2] + np.sin(arg)).max() <= 6e-8


def test_lockin_at_a_bin_equals_the_ring_dft_bin():
    """With omega dt = 2 pi k / N over the window s = 1..N, |X|^2 from the
    lock-in equals qld_fft_bin on a context holding the same frames."""
    H, W, N, k = 96, 128, 64, 5
    rng = np.random.default_rng(77)
    x = rng.integers(0, 4096, size=(N, H * W)).astype(np.uint16)
    amp, _, _ = gpu_lockin(x, H, W, 2 * math.pi * k / N, 1)
    ctx = q.qld_create(H, W, N, q.QLD_U16)
    q.qld_push_frames(ctx, torch.from_numpy(x).cuda(), N)
    out = torch.empty(H * W, dtype=torch.float32, device="cuda")
    q.qld_fft_bin(ctx, k, out)
    q.qld_sync(ctx)
    check_power(amp.astype(np.float64) ** 2, out.cpu().numpy().astype(np.float64), x.astype(np.int64).sum(0))
    ctx.destroy()


def test_lockin_rejects_bad_arguments():
    """The C ABI's own validation (called directly, below the binding)."""
    t = torch.empty(64, dtype=torch.float32, device="cuda")
    f = torch.zeros(8 * 16 * 2 * 8, dtype=torch.uint8, device="cuda")
    a = torch.empty(16 * 8, dtype=torch.float32, device="cuda")
    F, T, A = f.data_ptr(), t.data_ptr(), a.data_ptr()
    bad = [(F, 8, 16, 0, 2, T, A, None),      # N = 0
           (F, 8, 16, 8, 3, T, A, None),      # unknown pixel format
           (F, 8, 16, 8, 2, T, None, None),   # no output
           (F, 3, 3, 2, 1, T, A, None),       # frame of 9 bytes: not a multiple of 16
           (F + 4, 8, 16, 8, 2, T, A, None),  # frames not 16-byte aligned
           (None, 8, 16, 8, 2, T, A, None),   # no frames
           (F, 8, 16, 8, 2, None, A, None)]   # no table
    for args in bad:
        assert q.lib.qld_lockin_frames(*args, None) == q.QLD_E_INVAL
    assert q.lib.qld_lockin_table(1.0, 1, 0, T, None) == q.QLD_E_INVAL
    assert q.lib.qld_lockin_table(1.0, 1, 8, None, None) == q.QLD_E_INVAL


# ---- Fig. 1 analog --------------------------------------------------------
# Methods, "Numerical simulations": an n x n frame with five non-overlapping
# m x m sources, four modulated at 20, 23, 26, 29 Hz as 0.5 (1 + sin(w t_s))
# (the paper's "0.5 + sin" read as a non-negative intensity), one constant,
# plus uniform noise U[0, X] on every pixel of every frame; N = 82 and 41
# frames; t_s = s dt. The paper gives neither dt nor n, m or X: here n = 96,
# m = 8, X = 4, and intensities are stored as counts (x 100) in uint16.
FIG1_FREQS = [20.0, 23.0, 26.0, 29.0]
FIG1_POS = [(16, 16), (16, 56), (56, 16), (56, 56), (36, 36)]
FIG1_N, FIG1_M = 96, 8


def fig1_frames(N, X, fs, seed):
    rng = np.random.default_rng(seed)
    s = np.arange(1, N + 1)
    n, m = FIG1_N, FIG1_M
    img = np.zeros((N, n, n))
    for (r, c), f in zip(FIG1_POS[:4], FIG1_FREQS):
        img[:, r:r + m, c:c + m] += (0.5 * (1 + np.sin(2 * math.pi * f * s / fs)))[:, None, None]
    r, c = FIG1_POS[4]
    img[:, r:r + m, c:c + m] += 0.5
    img += rng.uniform(0, X, size=img.shape)
    return np.rint(100 * img).astype(np.uint16).reshape(N, n * n)


def fig1_cnrs(fs, seed=11, X=4.0):
    n, m = FIG1_N, FIG1_M
    x = fig1_frames(82, X, fs, seed)
    sumx = x.astype(np.int64).sum(axis=0)
    maps = {}
    for name, frames, w in [("qld82", x, 2 * math.pi * 23 / fs), ("qld41", x[:41], 2 * math.pi * 23 / fs),
                            ("wrong31", x, 2 * math.pi * 31 / fs),
                            ("fft82", x, 2 * math.pi * round(23 * 82 / fs) / 82)]:
        amp, ph, _ = gpu_lockin(frames, n, n, w)
        S, C, R, phr = oracle.lockin_general(frames, w)
        check_lockin(amp, ph, R, phr, frames.astype(np.int64).sum(axis=0), name)
        maps[name] = amp.astype(np.float64).reshape(n, n)
    r0, c0 = FIG1_POS[1]
    cnr = {k: oracle.cnr(v, r0, c0, m) for k, v in maps.items()}
    cnr["fft82_power"] = oracle.cnr(maps["fft82"] ** 2, r0, c0, m)
    return cnr


def test_fig1_analog_source_between_fft_bins():
    """At 102 frames/s, 23 Hz lies half way between the N = 82 bins (18.49 *
    fs/N): QLD at the exact frequency shows the source with a higher CNR than
    the FFT's nearest bin (as |F| or |F|^2), QLD on N/2 frames is at least as
    good as the FFT on N, and QLD at 31 Hz shows no source."""
    c = fig1_cnrs(fs=102.0)
    assert c["qld82"] > 1.5 * c["fft82"] and c["qld82"] > 1.5 * c["fft82_power"]
    assert c["qld41"] >= c["fft82_power"]
    assert c["qld82"] > c["qld41"]
    assert abs(c["wrong31"]) < 0.5 < c["qld41"]


def test_fig1_analog_source_on_an_fft_bin():
    """At 100 frames/s, 23 Hz is 0.14 bin from bin 19: the FFT amplitude
    |F| then matches QLD's CNR (QLD at a bin frequency is the DFT there)."""
    c = fig1_cnrs(fs=100.0)
    assert abs(c["fft82"] - c["qld82"]) < 0.1 * c["qld82"]
    assert abs(c["wrong31"]) < 0.5


def test_lockin_full_size_sampled_pixels():
    """The size bench.py times: 1024 caller frames of 1024x1024 uint16 (fog
    scene from the device generator) at 23 Hz sampled at 102 frames/s;
    sampled pixels against the oracle on frames regenerated on the host."""
    from qldscene import DeviceScene, scene_fog

    H = W = 1024
    N = 1024
    s0 = 1
    omega_dt = 2 * math.pi * 23 / 102
    sc = scene_fog(6, seed=1002, H=H, W=W)
    frames = torch.empty((N, H, W), dtype=torch.uint16, device="cuda")
    DeviceScene(sc).generate_into(frames, s0, N)
    table = torch.empty(2 * N, dtype=torch.float32, device="cuda")
    amp = torch.empty(H * W, dtype=torch.float32, device="cuda")
    ph = torch.empty_like(amp)
    q.qld_lockin_table(omega_dt, s0, N, table)
    q.qld_lockin_frames(frames, H, W, N, q.QLD_U16, table, amp, ph)
    torch.cuda.synchronize()
    rng = np.random.default_rng(77)
    pix = np.unique(np.concatenate([rng.choice(H * W, 2048, replace=False),
                                    rng.choice(np.flatnonzero(sc.mask.ravel()), 256, replace=False), [0, H * W - 1]]))
    win = sc.frames(s0, N, pix=pix)
    S, C, R, phr = oracle.lockin_general(win, omega_dt, s0=s0)
    check_lockin(amp.cpu().numpy()[pix], ph.cpu().numpy()[pix], R, phr, win.astype(np.int64).sum(axis=0), "full size")
    del frames
