"""Serving several streams with continuous batching: each stream's results in
the mix equal its results alone (and the oracle's), admission follows the HBM
budget in arrival order, streams join while earlier ticks run, and the
autotuner's choice leaves results unchanged."""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from qld_check import pack12

pytestmark = pytest.mark.gpu

# (H, W, N, pixfmt): uneven sizes, windows and formats
MIX = [(48, 64, 16, q.QLD_U8), (64, 80, 32, q.QLD_U16), (32, 48, 8, q.QLD_P12), (96, 128, 64, q.QLD_U16),
       (40, 64, 12, q.QLD_U8)]


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def frames_for(rng, H, W, fmt, n):
    hi = 256 if fmt == q.QLD_U8 else 4096
    x = rng.integers(0, hi, size=(n, H * W)).astype(np.uint8 if fmt == q.QLD_U8 else np.uint16)
    raw = pack12(x) if fmt == q.QLD_P12 else x
    dev = torch.from_numpy(np.ascontiguousarray(raw).view(np.uint8).reshape(n, -1)).cuda()
    return x, dev


class _DevArray:
    """A zero-copy view of library-owned device memory for torch."""

    def __init__(self, addr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (addr, False), "version": 3}


def server_images(srv, ticket, npix):
    a, p = q.qld_server_image(srv, ticket)
    torch.cuda.synchronize()
    amp = torch.as_tensor(_DevArray(a, npix, "<f4"), device="cuda").cpu().numpy()
    ph = torch.as_tensor(_DevArray(p, npix, "<f4"), device="cuda").cpu().numpy()
    return amp, ph


def server_iq(srv, ticket, npix):
    S = torch.empty(npix, dtype=torch.int32, device="cuda")
    C = torch.empty_like(S)
    q.qld_server_iq(srv, ticket, S, C)
    torch.cuda.synchronize()
    return S.cpu().numpy(), C.cpu().numpy()


def ctx_state(ctx):
    S = torch.empty(ctx.npix, dtype=torch.int32, device="cuda")
    C = torch.empty_like(S)
    amp = torch.empty(ctx.npix, dtype=torch.float32, device="cuda")
    ph = torch.empty_like(amp)
    q.qld_get_iq(ctx, S, C)
    q.qld_image(ctx, amp, ph)
    q.qld_sync(ctx)
    return S.cpu().numpy(), C.cpu().numpy(), amp.cpu().numpy(), ph.cpu().numpy()


def run_mix(autotune=False, ticks=10, seed=0, batched=False, shape=None, late=0):
    """`shape`: a fixed launch shape; `late`: the last `late` streams of the
    mix are requested only at tick 3, after the tick graphs were built."""
    rng = np.random.default_rng(seed)
    srv = q.qld_server_create(1 << 36)
    if shape is not None:
        q.qld_server_set_shape(srv, shape)
    early = len(MIX) - late
    tickets = [q.qld_server_request(srv, *m) for m in MIX[:early]] + [None] * late
    assert all(q.qld_server_state(srv, t) == 0 for t in tickets[:early])
    alone = [q.qld_create(*m) for m in MIX]
    history = [np.zeros((0, m[0] * m[1]), np.uint8 if m[3] == q.QLD_U8 else np.uint16) for m in MIX]
    keep = []
    batch = q.SubmitBatch(len(MIX))
    for tick in range(ticks):
        if late and tick == 3:
            for i in range(early, len(MIX)):
                tickets[i] = q.qld_server_request(srv, *MIX[i])
                assert q.qld_server_state(srv, tickets[i]) == 0
        nb = 0
        for i, (t, m) in enumerate(zip(tickets, MIX)):
            if t is None:
                continue
            H, W, N, fmt = m
            pattern = [1, 2, 0, 3, 1, N + 1, 1, 4, 0, 2]
            count = pattern[(tick + i) % len(pattern)] if tick < ticks - 1 else 1
            if late and tick == 3 and i >= early:
                count = N  # a late stream fills its window on the tick it joins
            if count == 0:
                continue
            x, dev = frames_for(rng, H, W, fmt, count)
            keep.append(dev)
            if batched:
                batch.set(nb, srv, t, dev, count)
                nb += 1
            else:
                q.qld_server_submit(srv, t, dev, count)
            q.qld_push_frames(alone[i], dev, count)
            history[i] = np.concatenate([history[i], x])
        if batched:
            batch.submit(srv, nb)
        assert q.qld_server_tick(srv) >= 1
        if autotune and tick == 2:
            k, us = q.qld_server_autotune(srv)
            assert 0 <= k and us > 0
    q.qld_server_sync(srv)
    for i, (t, m) in enumerate(zip(tickets, MIX)):
        H, W, N, fmt = m
        npix = H * W
        assert q.qld_server_frames_pushed(srv, t) == history[i].shape[0]
        S, C = server_iq(srv, t, npix)
        amp, ph = server_images(srv, t, npix)
        Sa, Ca, ampa, pha = ctx_state(alone[i])
        assert np.array_equal(S, Sa) and np.array_equal(C, Ca), "sums differ in the mix for stream %d" % i
        assert np.array_equal(amp, ampa) and np.array_equal(ph, pha), "images differ in the mix for stream %d" % i
        win = history[i][-N:]
        S_r, C_r = oracle.quadrature_sums(win, s0=history[i].shape[0] - N + 1)
        assert np.array_equal(S, S_r) and np.array_equal(C, C_r)
        alone[i].destroy()
    srv.destroy()


def test_each_stream_in_the_mix_equals_it_alone():
    run_mix()


def test_autotuned_shape_gives_the_same_results():
    run_mix(autotune=True, seed=1)


@pytest.mark.parametrize("shape", range(16))
def test_every_launch_shape_gives_the_same_results(shape):
    """Each candidate shape, persistent or one CTA per tile, with two streams
    admitted after the tick graphs were built (a one-CTA-per-tile grid must
    grow to cover them)."""
    if shape >= q.qld_server_num_shapes():
        pytest.skip("%d launch shapes" % q.qld_server_num_shapes())
    run_mix(seed=20 + shape, shape=shape, late=2)


def test_set_shape_rejects_bad_indices():
    srv = q.qld_server_create(1 << 30)
    try:
        for bad in (-1, q.qld_server_num_shapes()):
            assert q.lib.qld_server_set_shape(srv.handle, bad) == q.QLD_E_INVAL
        q.qld_server_set_shape(srv, q.qld_server_num_shapes() - 1)
        assert q.qld_server_shape(srv)[2] == 0  # the last shapes are one CTA per tile
    finally:
        srv.destroy()


def test_submit_many_equals_single_submits():
    run_mix(seed=2, batched=True)


def test_submit_many_takes_all_or_nothing():
    rng = np.random.default_rng(6)
    srv = q.qld_server_create(1 << 34)
    a = q.qld_server_request(srv, 32, 64, 8, q.QLD_U16)
    b = q.qld_server_request(srv, 16, 32, 4, q.QLD_U8)
    _, da = frames_for(rng, 32, 64, q.QLD_U16, 1)
    _, db = frames_for(rng, 16, 32, q.QLD_U8, 1)
    batch = q.SubmitBatch(3)
    batch.set(0, srv, a, da, 1)
    batch.set(1, srv, b, db, 1)
    batch.set(2, srv, a, da, 1)  # the same stream twice in one tick
    with pytest.raises(q.QLDError) as e:
        batch.submit(srv, 3)
    assert e.value.status == q.QLD_E_INVAL
    assert q.qld_server_tick(srv) == 0  # nothing was taken
    q.qld_server_submit_many(srv, [(a, da, 1), (b, db)])
    assert q.qld_server_tick(srv) == 2
    q.qld_server_sync(srv)
    assert q.qld_server_frames_pushed(srv, a) == 1 and q.qld_server_frames_pushed(srv, b) == 1
    srv.destroy()


def test_admission_by_budget_in_arrival_order():
    fa = q.qld_footprint_bytes(64, 64, 64, q.QLD_U16) + 2 * 64 * 64 * 4
    fb = q.qld_footprint_bytes(32, 32, 16, q.QLD_U8) + 2 * 32 * 32 * 4
    srv = q.qld_server_create(2 * fa + fb // 2)
    a = q.qld_server_request(srv, 64, 64, 64, q.QLD_U16)
    b = q.qld_server_request(srv, 64, 64, 64, q.QLD_U16)
    c = q.qld_server_request(srv, 64, 64, 64, q.QLD_U16)  # does not fit: waits
    d = q.qld_server_request(srv, 32, 32, 16, q.QLD_U8)   # would fit, but arrived after c: waits too
    assert [q.qld_server_state(srv, t) for t in (a, b, c, d)] == [0, 0, 1, 1]
    assert q.qld_server_mem_in_use(srv) == 2 * fa
    rng = np.random.default_rng(4)
    x, dev = frames_for(rng, 64, 64, q.QLD_U16, 2)
    with pytest.raises(q.QLDError) as e:
        q.qld_server_submit(srv, c, dev, 2)
    assert e.value.status == q.QLD_E_NOT_READY
    with pytest.raises(q.QLDError) as e:
        q.qld_server_request(srv, 1024, 1024, 4096, q.QLD_U16)  # larger than the whole budget
    assert e.value.status == q.QLD_E_NOMEM
    q.qld_server_submit(srv, a, dev, 2)
    q.qld_server_tick(srv)
    q.qld_server_close(srv, a)  # frees room: c is admitted, then d does not fit behind it
    assert [q.qld_server_state(srv, t) for t in (a, b, c, d)] == [-1, 0, 0, 1]
    q.qld_server_close(srv, b)
    assert q.qld_server_state(srv, d) == 0
    assert q.qld_server_mem_in_use(srv) == fa + fb
    srv.destroy()


def test_stream_admitted_while_ticks_run_joins_the_next_tick():
    rng = np.random.default_rng(5)
    srv = q.qld_server_create(1 << 34)
    a = q.qld_server_request(srv, 64, 96, 8, q.QLD_U16)
    xa, da = frames_for(rng, 64, 96, q.QLD_U16, 8)
    q.qld_server_submit(srv, a, da, 8)
    q.qld_server_tick(srv)                      # no sync: still on the GPU
    b = q.qld_server_request(srv, 48, 32, 4, q.QLD_U8)
    assert q.qld_server_state(srv, b) == 0
    xb, db = frames_for(rng, 48, 32, q.QLD_U8, 5)
    xa2, da2 = frames_for(rng, 64, 96, q.QLD_U16, 1)
    q.qld_server_submit(srv, b, db, 5)
    q.qld_server_submit(srv, a, da2, 1)
    assert q.qld_server_tick(srv) == 2         # both streams in one launch
    q.qld_server_sync(srv)
    for t, hist, H, W, N in [(a, np.concatenate([xa, xa2]), 64, 96, 8), (b, xb, 48, 32, 4)]:
        S, C = server_iq(srv, t, H * W)
        S_r, C_r = oracle.quadrature_sums(hist[-N:], s0=hist.shape[0] - N + 1)
        assert np.array_equal(S, S_r) and np.array_equal(C, C_r)
        amp, ph = server_images(srv, t, H * W)
        R, phr = oracle.amplitude_phase(S_r, C_r)
        assert np.all(np.abs(amp - R) <= 1e-6 * R)
    srv.destroy()


def test_server_rejects_unbatchable_or_bad_requests():
    srv = q.qld_server_create(1 << 30)
    for args in [(3, 5, 8, q.QLD_U8), (4, 4, 6, q.QLD_U16), (2, 10, 8, q.QLD_P12)]:  # 15 B frames; N; 30 B
        with pytest.raises(q.QLDError) as e:
            q.qld_server_request(srv, *args)
        assert e.value.status == q.QLD_E_INVAL
    t = q.qld_server_request(srv, 16, 16, 8, q.QLD_U16)
    buf = torch.zeros(16 * 16 * 2 * 2 + 16, dtype=torch.uint8, device="cuda")
    assert q.lib.qld_server_submit(srv.handle, t, buf.data_ptr() + 4, 1) == q.QLD_E_INVAL  # misaligned
    assert q.qld_server_tick(srv) == 0  # nothing submitted: no launch
    srv.destroy()


# ---- gated ticks: a bounded device wait on a doorbell before the tick ----

def _gated_setup(seed, shape=None):
    rng = np.random.default_rng(seed)
    srv = q.qld_server_create(1 << 34)
    if shape is not None:
        q.qld_server_set_shape(srv, shape)
    mix = MIX[:3]
    tickets = [q.qld_server_request(srv, *m) for m in mix]
    alone = [q.qld_create(*m) for m in mix]
    frames = []
    for (H, W, N, fmt), t, ctx in zip(mix, tickets, alone):
        x, dev = frames_for(rng, H, W, fmt, N + 3)
        frames.append((x, dev))
        q.qld_server_submit(srv, t, dev, N + 3)
        q.qld_push_frames(ctx, dev, N + 3)
    torch.cuda.synchronize()
    return srv, mix, tickets, alone, frames


def _check_against_alone(srv, mix, tickets, alone):
    for (H, W, N, fmt), t, ctx in zip(mix, tickets, alone):
        S, C, amp, ph = ctx_state(ctx)
        S2, C2 = server_iq(srv, t, H * W)
        amp2, ph2 = server_images(srv, t, H * W)
        assert np.array_equal(S, S2) and np.array_equal(C, C2)
        assert np.array_equal(amp, amp2) and np.array_equal(ph, ph2)


def _per_tile_shape():
    for k in range(q.qld_server_num_shapes()):
        srv = q.qld_server_create(1 << 20)
        try:
            q.qld_server_set_shape(srv, k)
            if q.qld_server_shape(srv)[2] == 0:
                return k
        finally:
            srv.destroy()
    return None


@pytest.mark.parametrize("per_tile", [False, True])
def test_gated_tick_times_out_on_a_doorbell_nothing_rings(per_tile):
    srv, mix, tickets, alone, _ = _gated_setup(41, _per_tile_shape() if per_tile else None)
    try:
        bell = torch.zeros(4, dtype=torch.int32, device="cuda")
        with pytest.raises(q.QLDError) as e:
            q.qld_server_tick_gated(srv, bell, 1, 20_000_000)  # 20 ms, nothing writes the bell
        assert e.value.status == q.QLD_E_TIMEOUT
        with pytest.raises(q.QLDError) as e:  # no gated tick has run yet
            q.qld_server_last_gated_us(srv)
        assert e.value.status == q.QLD_E_NOT_READY
        assert all(q.qld_server_frames_pushed(srv, t) == 0 for t in tickets)
        # the submissions are still pending: a plain tick consumes them, and the
        # server's results equal each stream alone
        assert q.qld_server_tick(srv) == len(mix)
        q.qld_server_sync(srv)
        assert all(q.qld_server_frames_pushed(srv, t) == m[2] + 3 for t, m in zip(tickets, mix))
        _check_against_alone(srv, mix, tickets, alone)
        # a bell that already rang lets the tick through at once
        bell.fill_(7)
        keep = []  # submitted frames must stay valid until the tick has run
        for (H, W, N, fmt), t, ctx in zip(mix, tickets, alone):
            x, dev = frames_for(np.random.default_rng(H), H, W, fmt, 2)
            keep.append(dev)
            q.qld_server_submit(srv, t, dev, 2)
            q.qld_push_frames(ctx, dev, 2)
        assert q.qld_server_tick_gated(srv, bell, 7, 1_000_000_000) == len(mix)
        _check_against_alone(srv, mix, tickets, alone)
        assert 0.0 < q.qld_server_last_gated_us(srv) < 1e5  # the tick alone, not the wait
        for bad in [(None, 1, 1000), (bell, 1, 0), (bell, 1, 11 * 10 ** 9), (bell.data_ptr() + 2, 1, 1000)]:
            assert q.lib.qld_server_tick_gated(srv.handle, None, bad[0] if not isinstance(bad[0], torch.Tensor)
                                               else bad[0].data_ptr(), bad[1], bad[2]) == q.QLD_E_INVAL
    finally:
        srv.destroy()
        for c in alone:
            c.destroy()


def test_gated_tick_runs_when_a_host_thread_rings_the_doorbell():
    """A host thread rings a device-memory doorbell with a copy on its own
    non-blocking stream while the calling thread waits in the gated tick,
    which runs on another non-blocking stream."""
    import threading
    import time
    srv, mix, tickets, alone, _ = _gated_setup(43)
    try:
        bell = torch.zeros(4, dtype=torch.int32, device="cuda")
        three = torch.full((4,), 3, dtype=torch.int32).pin_memory()
        tick_stream, side = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        rung = []

        def ring():
            time.sleep(0.05)
            rung.append(time.perf_counter())
            with torch.cuda.stream(side):
                bell.copy_(three, non_blocking=True)
            side.synchronize()

        th = threading.Thread(target=ring)
        t0 = time.perf_counter()
        th.start()
        n = q.qld_server_tick_gated(srv, bell, 3, 2_000_000_000, stream=tick_stream.cuda_stream)
        t1 = time.perf_counter()
        th.join()
        assert n == len(mix)
        assert rung and t1 >= rung[0] and t1 - t0 < 1.5  # it waited for the bell, not for the limit
        assert all(q.qld_server_frames_pushed(srv, t) == m[2] + 3 for t, m in zip(tickets, mix))
        _check_against_alone(srv, mix, tickets, alone)
    finally:
        srv.destroy()
        for c in alone:
            c.destroy()


def test_gated_tick_doorbell_in_mapped_host_memory():
    """The doorbell as a word of mapped pinned host memory (device pointer from
    cudaHostGetDevicePointer), set by the host: the gate's volatile loads see
    it across the bus and the tick runs."""
    import ctypes
    from cuda.bindings import runtime as rt
    srv, mix, tickets, alone, _ = _gated_setup(47)
    err, hptr = rt.cudaHostAlloc(16, rt.cudaHostAllocMapped)
    assert err == rt.cudaError_t.cudaSuccess
    try:
        word = ctypes.c_int.from_address(int(hptr))
        word.value = 5
        err, dptr = rt.cudaHostGetDevicePointer(hptr, 0)
        assert err == rt.cudaError_t.cudaSuccess
        assert q.qld_server_tick_gated(srv, int(dptr), 5, 1_000_000_000) == len(mix)
        _check_against_alone(srv, mix, tickets, alone)
        # a target above the word's value times out, nothing consumed
        keep = []
        for (H, W, N, fmt), t, ctx in zip(mix, tickets, alone):
            x, dev = frames_for(np.random.default_rng(W), H, W, fmt, 1)
            keep.append(dev)
            q.qld_server_submit(srv, t, dev, 1)
            q.qld_push_frames(ctx, dev, 1)
        with pytest.raises(q.QLDError) as e:
            q.qld_server_tick_gated(srv, int(dptr), 6, 5_000_000)
        assert e.value.status == q.QLD_E_TIMEOUT
        word.value = 6
        assert q.qld_server_tick_gated(srv, int(dptr), 6, 1_000_000_000) == len(mix)
        _check_against_alone(srv, mix, tickets, alone)
    finally:
        srv.destroy()
        for c in alone:
            c.destroy()
        rt.cudaFreeHost(hptr)
