"""Parity at the benchmark workloads' full sizes, in the launch
configuration bench.py times, on sampled pixels.

Frames are generated on the device by the seeded scene generator; the
oracle's inputs for the sampled pixels are generated independently on the
host by the numpy twin of that generator (identical integers), never read
back from the device. Pixels are independent, so a window restricted to
sampled pixels is an exact sub-problem.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from qld_check import check_amp_phase, check_power, check_sums, get_bin, get_image, get_iq
from qldscene import DeviceScene, scene_fog

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def sample_pixels(scene, n, seed):
    rng = np.random.default_rng(seed)
    mask_pix = np.flatnonzero(scene.mask.ravel())
    pix = np.concatenate([rng.choice(scene.npix, n, replace=False),
                          rng.choice(mask_pix, min(256, mask_pix.size), replace=False),
                          [0, scene.npix - 1]])
    return np.unique(pix)


def fill(ctx, dscene, N, chunk):
    """Pushes frames 1..N in chunks generated on the device."""
    sc = dscene.scene
    dt = torch.uint8 if sc.pixfmt == 1 else torch.uint16
    pool = torch.empty((chunk, sc.H, sc.W), dtype=dt, device="cuda")
    s = 1
    while s <= N:
        n = min(chunk, N - s + 1)
        dscene.generate_into(pool[:n], s, n)
        q.qld_push_frames(ctx, pool[:n], n)
        s += n
    return pool


def sampled_check(ctx, scene, T, N, pix, bins, amp_ph=None):
    s0 = T - N + 1
    win = scene.frames(s0, N, pix=pix)
    S_r, C_r = oracle.quadrature_sums(win, s0=s0)
    S_g, C_g = get_iq(ctx)
    check_sums(S_g[pix], C_g[pix], S_r, C_r, "T=%d" % T)
    R, phr = oracle.amplitude_phase(S_r, C_r)
    amp, ph = amp_ph if amp_ph is not None else get_image(ctx)
    check_amp_phase(amp[pix], ph[pix], R, phr, "T=%d" % T)
    sumx = win.astype(np.int64).sum(axis=0)
    for k in bins:
        p = get_bin(ctx, k)
        check_power(p[pix], oracle.dft_bin(win, k, s0=s0)[2], sumx, "T=%d k=%d" % (T, k))


@pytest.mark.parametrize("od", [4, 6, 8])
def test_fog_1024x1024_u16_N1024_sliding_by_4(od):
    """1024x1024 12-bit frames, N = 1024, window advanced 4 frames per step
    with the fused push+image call, QLD image and DFT bins k = N/4 and
    k = N/4 + 1 each step (the step bench.py times)."""
    H = W = 1024
    N = 1024
    sc = scene_fog(od, H=H, W=W)
    ds = DeviceScene(sc)
    ctx = q.qld_create(H, W, N, q.QLD_U16)
    fill(ctx, ds, N, 256)
    pix = sample_pixels(sc, 2048, od)
    sampled_check(ctx, sc, N, N, pix, bins=(N // 4,))
    step = torch.empty((4, H, W), dtype=torch.uint16, device="cuda")
    amp = torch.empty(H * W, dtype=torch.float32, device="cuda")
    ph = torch.empty_like(amp)
    T = N
    for i in range(3):
        ds.generate_into(step, T + 1, 4)
        q.qld_push_image(ctx, step, 4, None, amp, ph)
        T += 4
    q.qld_sync(ctx)
    sampled_check(ctx, sc, T, N, pix, bins=(N // 4, N // 4 + 1, 3),
                  amp_ph=(amp.cpu().numpy(), ph.cpu().numpy()))
    ctx.destroy()


def test_step_fog_1024x1024_u16_N1024_by_4_one_launch_against_the_oracle():
    """The kernel bench.py times, at the shape it times it: qld_step (push,
    image and DFT bin k = N/4 in one launch) on the OD 6 fog scene, 1024^2
    uint16, N = 1024, 4 frames a step. After each of three steps, the step's
    own amplitude, phase and power outputs and the context's sums on 2048+
    sampled pixels against the oracle on frames regenerated on the host."""
    H = W = 1024
    N = 1024
    sc = scene_fog(6, H=H, W=W)
    ds = DeviceScene(sc)
    ctx = q.qld_create(H, W, N, q.QLD_U16)
    fill(ctx, ds, N, 256)
    pix = sample_pixels(sc, 2048, 1006)
    step = torch.empty((4, H, W), dtype=torch.uint16, device="cuda")
    amp = torch.empty(H * W, dtype=torch.float32, device="cuda")
    ph = torch.empty_like(amp)
    pw = torch.empty_like(amp)
    T = N
    launches0 = q.qld_launch_count()
    for i in range(3):
        ds.generate_into(step, T + 1, 4)
        q.qld_step(ctx, step, 4, N // 4, pw, None, amp, ph)
        T += 4
        q.qld_sync(ctx)
        s0 = T - N + 1
        win = sc.frames(s0, N, pix=pix)
        S_r, C_r = oracle.quadrature_sums(win, s0=s0)
        S_g, C_g = get_iq(ctx)
        check_sums(S_g[pix], C_g[pix], S_r, C_r, "step %d" % i)
        R, phr = oracle.amplitude_phase(S_r, C_r)
        check_amp_phase(amp.cpu().numpy()[pix], ph.cpu().numpy()[pix], R, phr, "step %d" % i)
        check_power(pw.cpu().numpy()[pix], oracle.dft_bin(win, N // 4, s0=s0)[2],
                    win.astype(np.int64).sum(axis=0), "step %d" % i)
    # one launch per step after the first (which also fills the twiddle table)
    assert q.qld_launch_count() - launches0 == 3 + 1
    ctx.destroy()


def _pack12_device(x):
    """[n, H, W] uint16 (values < 4096) -> [n, H*W*3/2] uint8, two pixels in
    three bytes, least significant bits first (the QLD_P12 layout)."""
    n = x.shape[0]
    xi = x.reshape(n, -1).view(torch.int16).to(torch.int32) & 0xFFFF
    a, b = xi[:, 0::2], xi[:, 1::2]
    return torch.stack([a & 0xFF, (a >> 8) | ((b & 0xF) << 4), b >> 4], dim=-1).to(torch.uint8).reshape(n, -1)


def test_fog_1024x1024_packed12_N1024_sliding_by_4():
    """The benchmark step on packed 12-bit frames at full size (the packed12
    block of bench.py): the window filled with packed frames, then three
    fused push+image steps of 4 frames; sampled pixels against the oracle on
    the unpacked frames regenerated on the host, DFT bins included."""
    H = W = 1024
    N = 1024
    sc = scene_fog(6, H=H, W=W)
    ds = DeviceScene(sc)
    ctx = q.qld_create(H, W, N, q.QLD_P12)
    buf = torch.empty((256, H, W), dtype=torch.uint16, device="cuda")
    s = 1
    while s <= N:
        ds.generate_into(buf, s, 256)
        q.qld_push_frames(ctx, _pack12_device(buf), 256)
        s += 256
    pix = sample_pixels(sc, 2048, 66)
    amp = torch.empty(H * W, dtype=torch.float32, device="cuda")
    ph = torch.empty_like(amp)
    T = N
    for i in range(3):
        ds.generate_into(buf[:4], T + 1, 4)
        q.qld_push_image(ctx, _pack12_device(buf[:4]), 4, None, amp, ph)
        T += 4
    q.qld_sync(ctx)
    sampled_check(ctx, sc, T, N, pix, bins=(N // 4, N // 4 + 1, 3), amp_ph=(amp.cpu().numpy(), ph.cpu().numpy()))
    ctx.destroy()


def test_640x480_u8_N256_full_frame():
    """640x480 uint8, N = 256: whole frame against the oracle (random frames,
    pushed in uneven batches)."""
    H, W, N = 480, 640, 256
    rng = np.random.default_rng(640)
    x = rng.integers(0, 256, size=(N + 3, H * W)).astype(np.uint8)
    ctx = q.qld_create(H, W, N, q.QLD_U8)
    dx = torch.from_numpy(x).cuda()
    done = 0
    for n in (100, 1, 150, 7, 1):
        q.qld_push_frames(ctx, dx[done:done + n], n)
        done += n
    T = N + 3
    assert done == T
    win = x[T - N:]
    S_r, C_r = oracle.quadrature_sums(win, s0=T - N + 1, nthreads=8)
    S_g, C_g = get_iq(ctx)
    check_sums(S_g, C_g, S_r, C_r)
    amp, ph = get_image(ctx)
    R, phr = oracle.amplitude_phase(S_r, C_r)
    check_amp_phase(amp, ph, R, phr)
    p = get_bin(ctx, N // 4 + 5)
    check_power(p, oracle.dft_bin(win, N // 4 + 5, s0=T - N + 1, nthreads=8)[2], win.astype(np.int64).sum(0))
    ctx.destroy()


@pytest.mark.parametrize("H,W,N", [(1024, 1280, 1024), (2048, 2048, 2048)])
def test_serving_stream_shapes_u16(H, W, N):
    """The uint16 camera-stream shapes (1280x1024 N = 1024, 2048x2048
    N = 2048), one new frame per push, sampled pixels."""
    sc = scene_fog(6, seed=1003, H=H, W=W)
    ds = DeviceScene(sc)
    ctx = q.qld_create(H, W, N, q.QLD_U16)
    fill(ctx, ds, N, 128)
    one = torch.empty((1, H, W), dtype=torch.uint16, device="cuda")
    T = N
    for _ in range(5):
        ds.generate_into(one, T + 1, 1)
        q.qld_push_frames(ctx, one, 1)
        T += 1
    pix = sample_pixels(sc, 1024, H)
    sampled_check(ctx, sc, T, N, pix, bins=(N // 4, 1))
    ctx.destroy()


@pytest.mark.large
def test_large_4096x4096_u16_N2048_ring_68GB():
    """4096x4096 uint16, N = 2048: a 68.7 GB ring (64-bit offsets), one new
    frame per step, sampled pixels over full windows."""
    H = W = 4096
    N = 2048
    free, _ = torch.cuda.mem_get_info()
    need = q.qld_footprint_bytes(H, W, N, q.QLD_U16) + (4 << 30)
    if free < need:
        pytest.skip("needs %.1f GB free device memory" % (need / 1e9))
    sc = scene_fog(5, seed=1005, H=H, W=W)
    ds = DeviceScene(sc)
    ctx = q.qld_create(H, W, N, q.QLD_U16)
    pool = fill(ctx, ds, N, 64)
    pix = sample_pixels(sc, 4096, 5)  # a seeded subset of >= 4096 pixels, plus mask pixels and both corners
    T = N
    one = pool[:1]
    amp = torch.empty(H * W, dtype=torch.float32, device="cuda")
    ph = torch.empty_like(amp)
    for _ in range(2):
        ds.generate_into(one, T + 1, 1)
        q.qld_push_image(ctx, one, 1, None, amp, ph)
        T += 1
    q.qld_sync(ctx)
    sampled_check(ctx, sc, T, N, pix, bins=(N // 4,), amp_ph=(amp.cpu().numpy(), ph.cpu().numpy()))
    del pool
    ctx.destroy()


SERVING_MIX = [(480, 640, 256, q.QLD_U8)] * 2 + [(1024, 1280, 1024, q.QLD_U16)] * 4 + [(2048, 2048, 2048, q.QLD_U16)] * 2


@pytest.mark.large
def test_serving_mix_full_size_sampled_pixels():
    """The eight-stream serving mix at full size (45.5 GB of rings) through
    qld_server: the windows filled by the server's own batched ticks (64
    frames per stream per tick), then three single-frame ticks; sampled
    pixels of every stream against the oracle (sums bit-exact, images within
    tolerance)."""
    from qldscene import scene_plain

    budget = sum(q.qld_footprint_bytes(*m) + 8 * m[0] * m[1] for m in SERVING_MIX)
    free, _ = torch.cuda.mem_get_info()
    if free < budget + (6 << 30):
        pytest.skip("needs %.1f GB free device memory" % ((budget + (6 << 30)) / 1e9))
    srv = q.qld_server_create(budget)
    tickets = [q.qld_server_request(srv, *m) for m in SERVING_MIX]
    assert all(q.qld_server_state(srv, t) == 0 for t in tickets)
    scenes = [scene_plain(seed=2003 + i, H=m[0], W=m[1]) if m[3] == q.QLD_U8 else
              scene_fog(6, seed=2003 + i, H=m[0], W=m[1]) for i, m in enumerate(SERVING_MIX)]
    dss = [DeviceScene(sc) for sc in scenes]
    chunk = 64
    pools = [torch.empty((chunk, m[0], m[1]), dtype=torch.uint8 if m[3] == q.QLD_U8 else torch.uint16,
                         device="cuda") for m in SERVING_MIX]
    pushed = [0] * len(SERVING_MIX)
    targets = [m[2] + 3 for m in SERVING_MIX]
    while min(p - t for p, t in zip(pushed, targets)) < 0:
        subs = []
        for i, m in enumerate(SERVING_MIX):
            left = targets[i] - pushed[i]
            n = min(chunk, left) if pushed[i] < m[2] else min(1, left)
            if n:
                dss[i].generate_into(pools[i][:n], pushed[i] + 1, n)
                subs.append((tickets[i], pools[i][:n], n))
                pushed[i] += n
        q.qld_server_submit_many(srv, subs)
        q.qld_server_tick(srv)
        q.qld_server_sync(srv)  # the pools are refilled for the next tick
    for i, (t, m) in enumerate(zip(tickets, SERVING_MIX)):
        H, W, N, fmt = m
        npix = H * W
        assert q.qld_server_frames_pushed(srv, t) == pushed[i]
        S = torch.empty(npix, dtype=torch.int32, device="cuda")
        C = torch.empty_like(S)
        q.qld_server_iq(srv, t, S, C)
        a, p = q.qld_server_image(srv, t)
        amp = torch.empty(npix, dtype=torch.float32, device="cuda")
        ph = torch.empty_like(amp)
        for addr, dst in ((a, amp), (p, ph)):
            src = torch.as_tensor(_DeviceView(addr, npix), device="cuda")
            dst.copy_(src)
        torch.cuda.synchronize()
        pix = sample_pixels(scenes[i], 512, 100 + i)
        T = pushed[i]
        s0 = T - N + 1
        win = scenes[i].frames(s0, N, pix=pix)
        S_r, C_r = oracle.quadrature_sums(win, s0=s0)
        check_sums(S.cpu().numpy()[pix], C.cpu().numpy()[pix], S_r, C_r, "stream %d" % i)
        R, phr = oracle.amplitude_phase(S_r, C_r)
        check_amp_phase(amp.cpu().numpy()[pix], ph.cpu().numpy()[pix], R, phr, "stream %d" % i)
    del pools
    srv.destroy()


class _DeviceView:
    """A zero-copy float32 view of library-owned device memory for torch."""

    def __init__(self, addr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (addr, False), "version": 3}
