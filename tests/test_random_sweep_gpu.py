"""Seeded random sweep of the ring path and the general-frequency lock-in
against the oracle: pixel format, frame shape (ragged widths, odd pixel
counts, single rows; the lock-in takes frames of whole 16-byte vectors),
window length, push counts (0, 1, bursts longer than the window), fused and
plain pushes (a fused push that would leave the window short must be refused
untouched), aligned and unaligned frame addresses, and DFT bins anywhere in
[0, N). Each case is one seed, so a failure names its configuration and
reruns alone."""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from qld_check import Stream, check_amp_phase, check_lockin
from test_lockin_gpu import gpu_lockin

pytestmark = pytest.mark.gpu

# more cases with QLD_SWEEP_CASES=n (the ring sweep; the lock-in one gets n / 2.5)
RING_CASES = int(os.environ.get("QLD_SWEEP_CASES", "40"))
LOCKIN_CASES = max(16, int(RING_CASES / 2.5))


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ring_case(seed):
    rng = np.random.default_rng(1000 + seed)
    fmt = int(rng.choice([q.QLD_U8, q.QLD_U16, q.QLD_P12]))
    H = int(rng.choice([1, 2, 3, int(rng.integers(4, 97))]))
    W = int(rng.integers(1, 161))
    if fmt == q.QLD_P12 and (H * W) % 2:
        W += 1
    N = int(rng.choice([4, 8, 12, 16, 20, 32, 64]))
    # byte offset of the frames in their buffer: uint16 needs 2-byte alignment,
    # other offsets take the scalar path
    offset = int(rng.choice([0, 0, 8, 2, 6])) if fmt != q.QLD_U8 else int(rng.choice([0, 0, 1, 5, 8]))
    counts = [int(c) for c in rng.choice([0, 1, 2, 3, 4, 5, N - 1, N, N + 3, 2 * N + 1], size=6)]
    return fmt, H, W, N, offset, counts, rng


@pytest.mark.parametrize("seed", range(RING_CASES))
def test_ring_random_configuration(seed):
    fmt, H, W, N, offset, counts, rng = ring_case(seed)
    hi = 256 if fmt == q.QLD_U8 else 4096
    st = Stream(H, W, N, fmt)
    try:
        for i, count in enumerate(counts):
            x = rng.integers(0, hi, size=(count, H * W))
            fused = bool(rng.integers(0, 2)) and count > 0
            if fused and st.frames.shape[0] + count < N:
                # a fused push that would leave the window short is refused
                # before any frame moves
                before = q.qld_frames_pushed(st.ctx)
                with pytest.raises(q.QLDError) as e:
                    st.push(x, offset=offset, fused=True)
                assert e.value.status == q.QLD_E_NOT_READY
                assert q.qld_frames_pushed(st.ctx) == before
                fused = False
            img = st.push(x, offset=offset, fused=fused)
            full = st.frames.shape[0] >= N
            bins = tuple(int(k) for k in rng.choice(N, size=2, replace=False)) if full else ()
            st.check(bins=bins)
            if img is not None and full:
                win, s0 = st.window()
                S_r, C_r = oracle.quadrature_sums(win, s0=s0)
                R, phr = oracle.amplitude_phase(S_r, C_r)
                check_amp_phase(img[0], img[1], R, phr, "fused push %d" % i)
    finally:
        st.ctx.destroy()


@pytest.mark.parametrize("seed", range(LOCKIN_CASES))
def test_lockin_random_configuration(seed):
    rng = np.random.default_rng(5000 + seed)
    fmt = int(rng.choice([q.QLD_U8, q.QLD_U16]))
    H = int(rng.integers(1, 65))
    W = int(rng.integers(1, 9)) * (16 if fmt == q.QLD_U8 else 8)  # frames of whole 16-byte vectors
    N = int(rng.choice([1, 2, 3, 7, int(rng.integers(8, 400))]))
    omega_dt = float(rng.uniform(1e-3, math.pi))
    s0 = int(rng.integers(1, 10 ** 6))
    hi = 256 if fmt == q.QLD_U8 else 4096
    x = rng.integers(0, hi, size=(N, H * W)).astype(np.uint8 if fmt == q.QLD_U8 else np.uint16)
    amp, ph, _ = gpu_lockin(x, H, W, omega_dt, s0)
    _, _, R, phr = oracle.lockin_general(x, omega_dt, s0=s0)
    check_lockin(amp, ph, R, phr, x.astype(np.int64).sum(axis=0), "seed %d N=%d" % (seed, N))
