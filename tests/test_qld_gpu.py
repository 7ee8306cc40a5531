"""Parity of the CUDA path (through the C ABI) with the CPU oracle on small
and ragged shapes, every edge case of the boundary, and the sliding window
checked against a from-scratch recompute after every push."""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from qld_check import Stream, dev_bytes, get_bin, get_image, get_iq
from qldscene import scene_plain

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rand_frames(rng, n, H, W, fmt, hi=None):
    hi = hi if hi is not None else (256 if fmt == 1 else 4096)
    return rng.integers(0, hi, size=(n, H * W)).astype(np.uint8 if fmt == 1 else np.uint16)


def test_block_mode_plain_scene_128x128_u8_N64():
    """128x128 uint8 frames, N = 64, one image from one push of N frames:
    the plain-QLD workload, whole frame against the oracle."""
    sc = scene_plain()
    x = sc.frames(1, 64)
    st = Stream(128, 128, 64, 1)
    st.push(x)
    st.check(bins=(16, 0, 1, 32, 63))
    # The mask square/disk is modulated: its amplitude stands above the rest.
    amp, _ = get_image(st.ctx)
    m = sc.mask.ravel() == 1
    assert amp[m].mean() > 1.5 * amp[~m].mean()


@pytest.mark.parametrize("H,W,fmt", [(37, 100, 2), (48, 80, 2), (33, 65, 1), (64, 64, 1), (1, 17, 1), (3, 8, 2)])
@pytest.mark.parametrize("N", [4, 16])
def test_sliding_equals_recompute_every_step(H, W, fmt, N):
    rng = np.random.default_rng(H * 1000 + W * 10 + N)
    st = Stream(H, W, N, fmt)
    st.check()
    for count in [1, 2, 3, 1, 4, 5, 0, 2, 7, N, 1, 3, N + 1, 2 * N + 3, 1, 4, 4, 4]:
        st.push(rand_frames(rng, count, H, W, fmt))
        st.check(bins=(N // 4, 1) if st.frames.shape[0] >= N else ())


@pytest.mark.parametrize("H,W,N,fmt", [(256, 256, 64, 2), (512, 512, 32, 2), (200, 160, 128, 1), (100, 37, 64, 2)])
def test_dft_bins_several_tiles(H, W, N, fmt):
    """Shapes spanning every CTA layout of the DFT-bin kernel (32, 16, 8, 4
    pixel vectors per CTA) and a ragged last vector."""
    rng = np.random.default_rng(N + H)
    st = Stream(H, W, N, fmt)
    st.push(rand_frames(rng, N + 5, H, W, fmt))
    st.check(bins=(0, 1, N // 4, N // 2, N - 1, 7 % N))


def test_vector_and_scalar_paths_agree_on_unaligned_input():
    rng = np.random.default_rng(3)
    H, W, N = 16, 64, 8
    for fmt, offsets in [(1, [0, 1, 3, 16]), (2, [0, 2, 6, 16])]:
        ref = None
        for off in offsets:
            st = Stream(H, W, N, fmt)
            x = rand_frames(np.random.default_rng(9), 3 * N + 2, H, W, fmt)
            for chunk in np.array_split(x, 5):
                st.push(chunk, offset=off)
            st.check(bins=(2,))
            S, C = get_iq(st.ctx)
            if ref is None:
                ref = (S, C)
            else:
                assert (S == ref[0]).all() and (C == ref[1]).all()


def test_uint16_odd_address_is_rejected():
    st = Stream(4, 8, 4, 2)
    x = np.zeros((1, 32), np.uint16)
    buf, addr = dev_bytes(x, 1)
    assert addr % 2 == 1
    with pytest.raises(q.QLDError) as e:
        q.qld_push_frames(st.ctx, addr, 1)
    assert e.value.status == q.QLD_E_INVAL
    assert q.qld_frames_pushed(st.ctx) == 0


def test_not_ready_until_window_full_and_bad_bin():
    st = Stream(8, 16, 8, 1)
    out = torch.empty(128, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(1)
    st.push(rand_frames(rng, 7, 8, 16, 1))
    for call in (lambda: q.qld_image(st.ctx, out), lambda: q.qld_fft_bin(st.ctx, 2, out)):
        with pytest.raises(q.QLDError) as e:
            call()
        assert e.value.status == q.QLD_E_NOT_READY
    buf, addr = dev_bytes(rand_frames(rng, 0, 8, 16, 1))
    with pytest.raises(q.QLDError) as e:
        q.qld_push_image(st.ctx, addr, 0, None, out, None)
    assert e.value.status == q.QLD_E_NOT_READY
    st.check()  # partial window: the sums of the 7 frames pushed so far
    st.push(rand_frames(rng, 1, 8, 16, 1))
    st.check(bins=(2,))
    for k in (-1, 8, 100):
        with pytest.raises(q.QLDError) as e:
            q.qld_fft_bin(st.ctx, k, out)
        assert e.value.status == q.QLD_E_INVAL


def test_fused_push_image_matches_separate_calls():
    rng = np.random.default_rng(5)
    H, W, N = 64, 128, 16
    a = Stream(H, W, N, 2)
    b = Stream(H, W, N, 2)
    x = rand_frames(rng, N, H, W, 2)
    a.push(x)
    b.push(x)
    for _ in range(5):
        y = rand_frames(rng, 4, H, W, 2)
        amp_f, ph_f = a.push(y, fused=True)
        b.push(y)
        amp_s, ph_s = get_image(b.ctx)
        assert np.array_equal(amp_f, amp_s) and np.array_equal(ph_f, ph_s)
        a.check()


def test_reset_and_independent_contexts():
    rng = np.random.default_rng(8)
    a = Stream(32, 32, 8, 1)
    b = Stream(32, 32, 12, 2)
    for _ in range(3):
        a.push(rand_frames(rng, 5, 32, 32, 1))
        b.push(rand_frames(rng, 7, 32, 32, 2))
    a.check(bins=(2,))
    b.check(bins=(3,))
    q.qld_reset(a.ctx)
    a.frames = a.frames[:0]
    a.check()
    a.push(rand_frames(rng, 9, 32, 32, 1))
    a.check(bins=(2, 5))
    b.check(bins=(3,))


def test_extreme_values_uint16_largest_window():
    """N = 65536 with full-scale 16-bit frames: |S|, |C| reach (N/4) * 65535."""
    N, H, W = 65536, 1, 8
    s = np.arange(1, N + 1)
    x = np.where((s % 4 == 1) | (s % 4 == 0), 65535, 0).astype(np.uint16)
    x = np.repeat(x[:, None], H * W, axis=1)
    st = Stream(H, W, N, 2)
    st.push(x)
    S, C = get_iq(st.ctx)
    assert (S == (N // 4) * 65535).all() and (C == (N // 4) * 65535).all()
    st.check(bins=(N // 4, 1))
    st.push(x[:3])
    st.check()


def test_push_on_a_side_stream():
    rng = np.random.default_rng(4)
    H, W, N = 64, 64, 8
    st = Stream(H, W, N, 2)
    x = rand_frames(rng, 12, H, W, 2)
    side = torch.cuda.Stream()
    buf, addr = dev_bytes(x)
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        q.qld_push_frames(st.ctx, addr, 12, side)
        assert q.qld_stream(st.ctx) == side.cuda_stream
        amp = torch.empty(H * W, dtype=torch.float32, device="cuda")
        q.qld_image(st.ctx, amp, None)
    side.synchronize()
    st.frames = x
    st.check(bins=(2,))
    R = oracle.qld(x[-N:].reshape(N, H * W), s0=12 - N + 1)[2]
    assert np.allclose(amp.cpu().numpy(), R, rtol=1e-6, atol=0)


def test_host_buffer_variants_match_device_variants():
    rng = np.random.default_rng(6)
    H, W, N = 96, 64, 16
    x = rand_frames(rng, N + 8, H, W, 2)
    a = Stream(H, W, N, 2)
    a.push(x)
    ctx = q.qld_create(H, W, N, 2)
    host = torch.from_numpy(x.copy()).pin_memory()
    q.qld_push_frames_host(ctx, host.data_ptr(), x.shape[0])
    amp_h = torch.empty(H * W, dtype=torch.float32).pin_memory()
    ph_h = torch.empty_like(amp_h).pin_memory()
    pw_h = torch.empty_like(amp_h).pin_memory()
    q.qld_image_host(ctx, amp_h, ph_h)
    q.qld_fft_bin_host(ctx, 5, pw_h)
    q.qld_sync(ctx)
    amp_d, ph_d = get_image(a.ctx)
    assert np.array_equal(amp_h.numpy(), amp_d) and np.array_equal(ph_h.numpy(), ph_d)
    assert np.array_equal(pw_h.numpy(), get_bin(a.ctx, 5))
    # pageable host memory works too (the copy is then synchronous)
    y = rand_frames(rng, 3, H, W, 2)
    q.qld_push_frames_host(ctx, y, 3)
    a.push(y)
    q.qld_sync(ctx)
    Sa, Ca = get_iq(a.ctx)
    Sb, Cb = get_iq(ctx)
    assert np.array_equal(Sa, Sb) and np.array_equal(Ca, Cb)
    ctx.destroy()


def test_dft_quarter_bin_equals_squared_sums_on_device():
    """X_{N/4} = C - iS: the DFT-bin kernel and the lock-in sums agree."""
    rng = np.random.default_rng(10)
    H, W, N = 128, 96, 256
    st = Stream(H, W, N, 2)
    st.push(rand_frames(rng, N + 2, H, W, 2))
    S, C = get_iq(st.ctx)
    p = get_bin(st.ctx, N // 4).astype(np.float64)
    ref = S.astype(np.float64) ** 2 + C.astype(np.float64) ** 2
    assert np.allclose(p, ref, rtol=3e-7, atol=0)


def test_memory_budget_and_accounting_on_device():
    base = q.qld_mem_in_use()
    fp = q.qld_footprint_bytes(64, 64, 16, 2)
    ctx = q.qld_create(64, 64, 16, 2)
    assert q.qld_mem_in_use() == base + fp
    q.qld_set_mem_budget(base + fp + fp // 2)
    try:
        with pytest.raises(q.QLDError) as e:
            q.qld_create(64, 64, 16, 2)
        assert e.value.status == q.QLD_E_NOMEM
    finally:
        q.qld_set_mem_budget(0)
    ctx.destroy()
    assert q.qld_mem_in_use() == base


def _frames_for_sums(S1, C1, P):
    """Frames whose window of N = 4P frames (s = 1..4P) has S = P*S1 and
    C = P*C1 per pixel: per period x1 - x3 = S1 and x4 - x2 = C1."""
    x1 = np.where(S1 > 0, S1, 0)
    x3 = np.where(S1 < 0, -S1, 0)
    x4 = np.where(C1 > 0, C1, 0)
    x2 = np.where(C1 < 0, -C1, 0)
    period = np.stack([x1, x2, x3, x4]).astype(np.uint16)
    return np.tile(period, (P, 1))


@pytest.mark.parametrize("P", [1, 3, 16384])
def test_amplitude_phase_on_every_octant_axis_and_extreme(P):
    """Chosen (S, C) pairs -- zero, both axes with both signs, the diagonals,
    points near every octant boundary, full-scale values, random pairs --
    through the push kernel's fused epilogue and the image kernel."""
    rng = np.random.default_rng(P)
    m = 65535
    pairs = [(0, 0), (0, 5), (0, -5), (5, 0), (-5, 0), (7, 7), (-7, 7), (7, -7), (-7, -7), (m, m), (-m, m),
             (m, -m), (-m, -m), (m, 0), (0, -m), (1, m), (m, 1), (-1, -m), (m - 1, m), (m, m - 1), (-m, m - 1),
             (1, 0), (0, 1), (-1, 0), (0, -1)]
    S1 = np.array([p[0] for p in pairs] + list(rng.integers(-m, m + 1, 999)), np.int64)
    C1 = np.array([p[1] for p in pairs] + list(rng.integers(-m, m + 1, 999)), np.int64)
    W = S1.size
    N = 4 * P
    x = _frames_for_sums(S1, C1, P)
    st = Stream(1, W, N, 2)
    amp_f, ph_f = (None, None)
    st.push(x[:-1])
    amp_f, ph_f = st.push(x[-1:], fused=True)
    S, C = get_iq(st.ctx)
    assert np.array_equal(S, P * S1) and np.array_equal(C, P * C1)
    R, ph = oracle.amplitude_phase(S, C)
    from qld_check import check_amp_phase

    check_amp_phase(amp_f, ph_f, R, ph, "fused epilogue")
    amp, phs = get_image(st.ctx)
    check_amp_phase(amp, phs, R, ph, "image kernel")
    assert phs[pairs.index((0, -5))] == np.float32(np.pi)  # S = 0, C < 0: +pi on the branch cut


def test_pipelined_host_path_many_steps_without_sync():
    """Twelve steps of host push + image + DFT bin queued without any sync:
    the staging and the four output buffers are reused while copies overlap
    kernels, and every step's host results must equal the device path's."""
    rng = np.random.default_rng(12)
    H, W, N, steps = 128, 96, 16, 12
    x = rand_frames(rng, N + 4 * steps, H, W, 2)
    host = torch.from_numpy(x.copy()).pin_memory()
    ctx = q.qld_create(H, W, N, 2)
    q.qld_push_frames_host(ctx, host[:N], N)
    outs = [tuple(torch.empty(H * W, dtype=torch.float32).pin_memory() for _ in range(3)) for _ in range(steps)]
    for i in range(steps):
        q.qld_push_frames_host(ctx, host[N + 4 * i:N + 4 * i + 4], 4)
        q.qld_image_host(ctx, outs[i][0], outs[i][1])
        q.qld_fft_bin_host(ctx, 3, outs[i][2])
    q.qld_sync(ctx)
    ref = Stream(H, W, N, 2)
    ref.push(x[:N])
    for i in range(steps):
        ref.push(x[N + 4 * i:N + 4 * i + 4])
        amp, ph = get_image(ref.ctx)
        assert np.array_equal(outs[i][0].numpy(), amp) and np.array_equal(outs[i][1].numpy(), ph), i
        assert np.array_equal(outs[i][2].numpy(), get_bin(ref.ctx, 3)), i
    ctx.destroy()


@pytest.mark.parametrize("H,W,fmt,N", [(128, 128, 1, 64), (37, 40, 2, 16), (30, 64, 3, 8), (64, 96, 1, 256),
                                       (5, 24, 2, 4), (256, 256, 2, 256)])
def test_block_push_equals_the_scalar_path_and_the_oracle(H, W, fmt, N):
    """Pushes of at least N frames into frames of at most 2^20 pixels run the
    block-mode kernel (time slices reduced in shared memory) when the frames
    are 16-byte aligned; the same frames a few bytes off run the one-pixel
    scalar kernel. Sums, images and DFT bins agree bit for bit, and with the
    oracle; both plain and fused pushes, exactly N and more than N frames, and
    sliding pushes afterwards."""
    rng = np.random.default_rng(H * W + N + fmt)
    a, b = Stream(H, W, N, fmt), Stream(H, W, N, fmt)
    try:
        for count, fused in [(N, True), (N + 5, False), (3, False), (2 * N + 1, True), (1, True)]:
            x = rand_frames(rng, count, H, W, fmt)
            ra = a.push(x, offset=0, fused=fused)
            rb = b.push(x, offset={1: 1, 2: 2, 3: 4}[fmt], fused=fused)
            if fused:
                assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
            Sa, Ca = get_iq(a.ctx)
            Sb, Cb = get_iq(b.ctx)
            assert np.array_equal(Sa, Sb) and np.array_equal(Ca, Cb)
            a.check(bins=(N // 4, 1))
        assert np.array_equal(get_bin(a.ctx, 3 % N), get_bin(b.ctx, 3 % N))
    finally:
        a.ctx.destroy()
        b.ctx.destroy()
