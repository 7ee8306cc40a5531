"""qld_step (push + amplitude/phase image + DFT bin) against the same step as
two calls (qld_push_image, qld_fft_bin) on a twin context: sums, images and
DFT powers bit for bit, on the single-kernel path (uint16, every CTA layout)
and on the two-kernel path it takes for uint8, packed 12-bit, unaligned and
ragged frames, plus the oracle on the qld_step context, the argument checks,
and the benchmark's full size."""
import numpy as np
import pytest
import torch

import paper_1511_03390_b300 as q
from qld_check import Stream, dev_bytes, get_iq, pack12

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def step_both(a, b, x, k, offset=0):
    """One step of `x` on Stream a through qld_step and on Stream b through
    the two calls; asserts identical outputs and returns a's (amp, phase,
    power)."""
    x = np.asarray(x, a.dtype).reshape(-1, a.H * a.W)
    buf, addr = dev_bytes(pack12(x) if a.fmt == q.QLD_P12 else x, offset)
    n = x.shape[0]
    out = [torch.full((a.H * a.W,), -1.0, dtype=torch.float32, device="cuda") for _ in range(6)]
    q.qld_step(a.ctx, addr, n, k, out[2], None, out[0], out[1])
    q.qld_push_image(b.ctx, addr, n, None, out[3], out[4])
    q.qld_fft_bin(b.ctx, k, out[5])
    torch.cuda.synchronize()
    del buf
    a.frames = np.concatenate([a.frames, x], axis=0)
    b.frames = np.concatenate([b.frames, x], axis=0)
    got = [o.cpu().numpy() for o in out]
    for i, what in enumerate(("amplitude", "phase", "power")):
        assert np.array_equal(got[i], got[i + 3]), "%s differs from the two-call step" % what
    Sa, Ca = get_iq(a.ctx)
    Sb, Cb = get_iq(b.ctx)
    assert np.array_equal(Sa, Sb) and np.array_equal(Ca, Cb)
    assert q.qld_frames_pushed(a.ctx) == q.qld_frames_pushed(b.ctx) == a.frames.shape[0]
    return got[:3]


@pytest.mark.parametrize("H,W,fmt,N,offset", [
    (512, 512, q.QLD_U16, 16, 0),   # 32 vectors per CTA, 4 time slices
    (64, 96, q.QLD_U16, 32, 0),     # small frame: 4 vectors per CTA, 64 time slices
    (128, 128, q.QLD_U16, 12, 0),   # 16 vectors per CTA
    (256, 256, q.QLD_U8, 16, 0),
    (40, 48, q.QLD_U8, 8, 8),
    (256, 256, q.QLD_P12, 16, 0),
    (30, 64, q.QLD_P12, 8, 4),
    (37, 100, q.QLD_U16, 8, 0),     # 7400-byte frames: not whole 16-byte vectors -> two kernels
    (37, 100, q.QLD_U8, 8, 0),
    (37, 100, q.QLD_P12, 8, 0),
    (64, 64, q.QLD_U16, 8, 2),      # unaligned frames -> two kernels
])
def test_step_equals_push_image_then_fft_bin(H, W, fmt, N, offset):
    rng = np.random.default_rng(H * W + N + fmt)
    hi = 256 if fmt == q.QLD_U8 else 4096
    a, b = Stream(H, W, N, fmt), Stream(H, W, N, fmt)
    try:
        fill = rng.integers(0, hi, size=(N - 1, H * W))
        a.push(fill)
        b.push(fill)
        for count, k in [(1, N // 4), (4, 1), (3, N - 1), (N, 0), (5, N // 2), (2, N // 4), (N + 3, 1)]:
            step_both(a, b, rng.integers(0, hi, size=(count, H * W)), k, offset)
            a.check(bins=(k,))
    finally:
        a.ctx.destroy()
        b.ctx.destroy()


def test_step_argument_checks_leave_the_context_untouched():
    H, W, N = 32, 32, 8
    ctx = q.qld_create(H, W, N, q.QLD_U16)
    try:
        x = torch.randint(0, 4096, (N, H * W), dtype=torch.int16, device="cuda")
        pw = torch.empty(H * W, dtype=torch.float32, device="cuda")
        with pytest.raises(q.QLDError) as e:
            q.qld_step(ctx, x, N - 1, 1, pw)  # window would not be full
        assert e.value.status == q.QLD_E_NOT_READY
        assert q.qld_frames_pushed(ctx) == 0
        q.qld_push_frames(ctx, x, N)
        for count, k in [(1, N), (1, -1)]:
            with pytest.raises(q.QLDError) as e:
                q.qld_step(ctx, x, count, k, pw)
            assert e.value.status == q.QLD_E_INVAL
        assert q.lib.qld_step(ctx.handle, x.data_ptr(), 0, None, None, None, 1, pw.data_ptr()) == q.QLD_E_INVAL
        assert q.lib.qld_step(ctx.handle, x.data_ptr(), 1, None, None, None, 1, None) == q.QLD_E_INVAL
        assert q.lib.qld_step(ctx.handle, x.data_ptr(), 1, None, None, None, 1, pw.data_ptr() + 2) == q.QLD_E_INVAL
        assert q.qld_frames_pushed(ctx) == N
    finally:
        ctx.destroy()


def test_step_full_size_1024x1024_N1024_by_4():
    """The benchmark's step shape: 1024^2 uint16, N = 1024, 4 frames a step."""
    H = W = 1024
    N = 1024
    a = q.qld_create(H, W, N, q.QLD_U16)
    b = q.qld_create(H, W, N, q.QLD_U16)
    try:
        g = torch.Generator(device="cuda").manual_seed(7)
        fill = torch.randint(0, 4096, (N, H * W), dtype=torch.int16, device="cuda", generator=g)
        q.qld_push_frames(a, fill, N)
        q.qld_push_frames(b, fill, N)
        del fill
        outs = [torch.empty(H * W, dtype=torch.float32, device="cuda") for _ in range(6)]
        for step in range(3):
            x = torch.randint(0, 4096, (4, H * W), dtype=torch.int16, device="cuda", generator=g)
            q.qld_step(a, x, 4, N // 4, outs[2], None, outs[0], outs[1])
            q.qld_push_image(b, x, 4, None, outs[3], outs[4])
            q.qld_fft_bin(b, N // 4, outs[5])
            torch.cuda.synchronize()
            for i in range(3):
                assert torch.equal(outs[i], outs[i + 3]), "step %d output %d" % (step, i)
        Sa, Ca = get_iq(a)
        Sb, Cb = get_iq(b)
        assert np.array_equal(Sa, Sb) and np.array_equal(Ca, Cb)
    finally:
        a.destroy()
        b.destroy()


@pytest.mark.parametrize("H,W,fmt,N,count", [
    (256, 256, q.QLD_U16, 16, 4),    # one kernel
    (256, 256, q.QLD_U8, 16, 3),     # two kernels
    (128, 256, q.QLD_P12, 8, 2),
    (1024, 1024, q.QLD_U16, 32, 40),  # 80 MiB of frames: the three host calls
])
def test_step_host_equals_step_on_device(H, W, fmt, N, count):
    rng = np.random.default_rng(H + W + fmt + count)
    hi = 256 if fmt == q.QLD_U8 else 4096
    a, b = q.qld_create(H, W, N, fmt), q.qld_create(H, W, N, fmt)
    npix = H * W
    try:
        def raw(x):
            x = x.astype(np.uint8 if fmt == q.QLD_U8 else np.uint16)
            return np.ascontiguousarray(pack12(x) if fmt == q.QLD_P12 else x).view(np.uint8).reshape(x.shape[0], -1)

        fill = raw(rng.integers(0, hi, size=(N, npix)))
        q.qld_push_frames(a, torch.from_numpy(fill).cuda(), N)
        q.qld_push_frames(b, torch.from_numpy(fill).cuda(), N)
        host_out = [torch.empty(npix, dtype=torch.float32).pin_memory() for _ in range(3)]
        dev_out = [torch.empty(npix, dtype=torch.float32, device="cuda") for _ in range(3)]
        for step in range(3):
            x = raw(rng.integers(0, hi, size=(count, npix)))
            xh = torch.from_numpy(x).pin_memory()
            q.qld_step_host(a, xh, count, N // 4 + step, host_out[2], None, host_out[0], host_out[1])
            q.qld_step(b, xh.cuda(), count, N // 4 + step, dev_out[2], None, dev_out[0], dev_out[1])
            q.qld_sync(a)
            torch.cuda.synchronize()
            for i in range(3):
                assert torch.equal(host_out[i], dev_out[i].cpu()), "step %d output %d" % (step, i)
        Sa, Ca = get_iq(a)
        Sb, Cb = get_iq(b)
        assert np.array_equal(Sa, Sb) and np.array_equal(Ca, Cb)
    finally:
        a.destroy()
        b.destroy()


def test_step_fills_a_window_that_was_almost_empty():
    """qld_step of exactly N frames onto a window holding 2: one kernel whose
    expiring slots are partly the ring's zeros."""
    H, W, N = 64, 64, 16
    rng = np.random.default_rng(5)
    a, b = Stream(H, W, N, q.QLD_U16), Stream(H, W, N, q.QLD_U16)
    try:
        first = rng.integers(0, 4096, size=(2, H * W))
        a.push(first)
        b.push(first)
        step_both(a, b, rng.integers(0, 4096, size=(N, H * W)), 3)
        a.check(bins=(3, N // 4))
    finally:
        a.ctx.destroy()
        b.ctx.destroy()
