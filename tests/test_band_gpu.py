"""Row bands of one camera stream (qld_create_band) against the whole frame.

Pixels are independent (Methods, "Numerical simulations": one time series
per pixel), so a frame cut into row bands, each band a context with its own
ring and sums, must reproduce the whole-frame context row for row: the int32
sums, the amplitude / phase images and the DFT bins bit for bit, through
every push call (plain, fused with the image, the one-launch step, and the
host-buffer variants). Several band contexts share one GPU here, fed the same
whole frames; on several GPUs each would hold one band. The bands are also
checked directly against the oracle on sampled pixels of a scene.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from qld_check import check_amp_phase, check_power, check_sums, dev_bytes, get_bin, get_image, get_iq, pack12

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _raw(x, fmt):
    x = x.astype(np.uint8 if fmt == q.QLD_U8 else np.uint16)
    return np.ascontiguousarray(pack12(x) if fmt == q.QLD_P12 else x).view(np.uint8).reshape(x.shape[0], -1)


def _outputs(ctx, bins):
    S, C = get_iq(ctx)
    amp, ph = get_image(ctx)
    return [S, C, amp, ph] + [get_bin(ctx, k) for k in bins]


@pytest.mark.parametrize("H,W,fmt,N,cuts", [
    (100, 64, q.QLD_U16, 16, (37,)),           # band starts 16-byte aligned: vector path, one-launch step
    (100, 50, q.QLD_U16, 8, (3, 51, 99)),      # unaligned band starts: scalar path, a one-row band
    (64, 96, q.QLD_U8, 12, (16, 48)),
    (90, 64, q.QLD_P12, 8, (45,)),             # packed 12-bit, 24-byte vectors
    (31, 30, q.QLD_P12, 4, (9,)),              # packed, bands of odd row counts on an even width
])
def test_bands_reproduce_the_whole_frame(H, W, fmt, N, cuts):
    rng = np.random.default_rng(H * W + N + fmt)
    hi = 256 if fmt == q.QLD_U8 else 4096
    edges = [0, *cuts, H]
    whole = q.qld_create(H, W, N, fmt)
    bands = [q.qld_create_band(H, W, N, fmt, r0, r1 - r0) for r0, r1 in zip(edges[:-1], edges[1:])]
    for b, (r0, r1) in zip(bands, zip(edges[:-1], edges[1:])):
        assert (b.H, b.W, b.H_total, b.row0) == (r1 - r0, W, H, r0)
        assert b.frame_pitch == whole.frame_bytes
    npix = H * W
    outs = {}
    try:
        frames = []
        # plain pushes, fused push + image, the one-launch step, of uneven counts
        for call, count, k in [("push", N - 1, None), ("push", 3, None), ("image", 1, None), ("step", 4, N // 4),
                               ("step", 1, 1), ("push", N + 2, None), ("step", N, N - 1), ("image", 5, None)]:
            x = rng.integers(0, hi, size=(count, npix))
            frames.append(x)
            buf, addr = dev_bytes(_raw(x, fmt))
            for ctx in [whole] + bands:
                o = [torch.full((ctx.npix,), -7.0, dtype=torch.float32, device="cuda") for _ in range(3)]
                if call == "push":
                    q.qld_push_frames(ctx, addr, count)
                elif call == "image":
                    q.qld_push_image(ctx, addr, count, None, o[0], o[1])
                else:
                    q.qld_step(ctx, addr, count, k, o[2], None, o[0], o[1])
                outs[id(ctx)] = o
            torch.cuda.synchronize()
            del buf
            if call != "push":  # the call's own outputs, band by band
                for i in range(2 if call == "image" else 3):
                    got = np.concatenate([outs[id(b)][i].cpu().numpy() for b in bands])
                    assert np.array_equal(got, outs[id(whole)][i].cpu().numpy()), (call, i)
        bins = (N // 4, 1, N - 1)
        want = _outputs(whole, bins)
        got = [_outputs(b, bins) for b in bands]
        for i in range(len(want)):
            assert np.array_equal(np.concatenate([g[i] for g in got]), want[i]), "output %d" % i
        # and the whole frame against the oracle (so every band is, row for row)
        x = np.concatenate(frames)[-N:].astype(np.uint8 if fmt == q.QLD_U8 else np.uint16)
        T = sum(f.shape[0] for f in frames)
        S_r, C_r = oracle.quadrature_sums(x, s0=T - N + 1)
        check_sums(want[0], want[1], S_r, C_r)
        R, phr = oracle.amplitude_phase(S_r, C_r)
        check_amp_phase(want[2], want[3], R, phr)
        check_power(want[4], oracle.dft_bin(x, N // 4, s0=T - N + 1)[2], x.astype(np.int64).sum(axis=0))
    finally:
        whole.destroy()
        for b in bands:
            b.destroy()


@pytest.mark.parametrize("fmt", [q.QLD_U16, q.QLD_U8, q.QLD_P12])
def test_band_host_pushes_copy_only_the_band(fmt):
    """qld_push_frames_host and qld_step_host on bands take whole host frames
    (strided copies of the band's rows) and equal the whole-frame context."""
    H, W, N = 96, 128, 8
    rng = np.random.default_rng(fmt)
    hi = 256 if fmt == q.QLD_U8 else 4096
    edges = [0, 40, 96]
    whole = q.qld_create(H, W, N, fmt)
    bands = [q.qld_create_band(H, W, N, fmt, r0, r1 - r0) for r0, r1 in zip(edges[:-1], edges[1:])]
    try:
        fill = torch.from_numpy(_raw(rng.integers(0, hi, size=(N, H * W)), fmt)).pin_memory()
        for ctx in [whole] + bands:
            q.qld_push_frames_host(ctx, fill, N)
        for step in range(3):
            x = torch.from_numpy(_raw(rng.integers(0, hi, size=(3, H * W)), fmt)).pin_memory()
            res = []
            for ctx in [whole] + bands:
                o = [torch.empty(ctx.npix, dtype=torch.float32).pin_memory() for _ in range(3)]
                q.qld_step_host(ctx, x, 3, N // 4 + step, o[2], None, o[0], o[1])
                q.qld_sync(ctx)
                res.append(o)
            for i in range(3):
                assert torch.equal(torch.cat([r[i] for r in res[1:]]), res[0][i]), (step, i)
        want = get_iq(whole)
        for i in range(2):
            assert np.array_equal(np.concatenate([get_iq(b)[i] for b in bands]), want[i])
    finally:
        whole.destroy()
        for b in bands:
            b.destroy()


def test_bands_of_a_scene_against_the_oracle():
    """Four bands of a 512x512 fog scene (OD 6), N = 256, filled and then slid
    by the one-launch step; sampled pixels of every band against the oracle
    on frames regenerated on the host."""
    from qldscene import DeviceScene, scene_fog

    H = W = 512
    N = 256
    sc = scene_fog(6, seed=1007, H=H, W=W)
    ds = DeviceScene(sc)
    edges = [0, 128, 256, 384, 512]
    bands = [q.qld_create_band(H, W, N, q.QLD_U16, r0, r1 - r0) for r0, r1 in zip(edges[:-1], edges[1:])]
    try:
        pool = torch.empty((64, H, W), dtype=torch.uint16, device="cuda")
        for s in range(1, N + 1, 64):
            ds.generate_into(pool, s, 64)
            for b in bands:
                q.qld_push_frames(b, pool, 64)
        T = N
        outs = [[torch.empty(b.npix, dtype=torch.float32, device="cuda") for _ in range(3)] for b in bands]
        for _ in range(2):
            ds.generate_into(pool[:4], T + 1, 4)
            for b, o in zip(bands, outs):
                q.qld_step(b, pool[:4], 4, N // 4, o[2], None, o[0], o[1])
            T += 4
        torch.cuda.synchronize()
        rng = np.random.default_rng(1007)
        s0 = T - N + 1
        for bi, (b, o) in enumerate(zip(bands, outs)):
            r0 = edges[bi]
            local = np.unique(np.concatenate([rng.choice(b.npix, 512, replace=False), [0, b.npix - 1]]))
            win = sc.frames(s0, N, pix=local + r0 * W)
            S_r, C_r = oracle.quadrature_sums(win, s0=s0)
            S_g, C_g = get_iq(b)
            check_sums(S_g[local], C_g[local], S_r, C_r, "band %d" % bi)
            R, phr = oracle.amplitude_phase(S_r, C_r)
            check_amp_phase(o[0].cpu().numpy()[local], o[1].cpu().numpy()[local], R, phr, "band %d" % bi)
            check_power(o[2].cpu().numpy()[local], oracle.dft_bin(win, N // 4, s0=s0)[2],
                        win.astype(np.int64).sum(axis=0), "band %d" % bi)
    finally:
        for b in bands:
            b.destroy()


def test_band_rejects_bad_arguments_and_counts_its_own_footprint():
    with pytest.raises(q.QLDError) as e:
        q.qld_create_band(64, 64, 8, q.QLD_U16, 60, 8)
    assert e.value.status == q.QLD_E_INVAL
    before = q.qld_mem_in_use()
    b = q.qld_create_band(1024, 256, 64, q.QLD_U16, 256, 128)
    try:
        assert q.qld_mem_in_use() - before == q.qld_footprint_bytes(128, 256, 64, q.QLD_U16)
    finally:
        b.destroy()
    assert q.qld_mem_in_use() == before
