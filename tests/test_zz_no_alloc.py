"""The allocation-free DFT-bin entry point against the context-based one and
against the oracle.

qld_fft_bin_frames_noalloc serves callers that cannot allocate device
memory while they run: a fixed-memory real-time camera loop that sizes all
of its buffers once at start-up, or code that must not risk the device-wide
synchronisation cudaMalloc/cudaFree can cause in the middle of a frame
period. Its twiddle table sits in a fixed device array instead of a context.
These tests call it through the C ABI twice in a row, with different bins
and shapes, and compare each result with qld_fft_bin on a fresh context
holding the same frames and with the FP64 oracle, within the DFT-bin
tolerance the other parity tests use; they also run it at its largest
window, and check that a call after the warm-up call allocates nothing. The
file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from qld_check import check_power

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def context_bin(frames_dev, H, W, N, fmt, k):
    ctx = q.qld_create(H, W, N, fmt)
    q.qld_push_frames(ctx, frames_dev, N)
    out = torch.empty(H * W, dtype=torch.float32, device="cuda")
    q.qld_fft_bin(ctx, k, out)
    q.qld_sync(ctx)
    ctx.destroy()
    return out.cpu().numpy().astype(np.float64)


def test_noalloc_matches_context_path_and_oracle_on_two_calls_in_a_row():
    rng = np.random.default_rng(2024)
    cases = [(192, 320, 64, q.QLD_U16, 16, 4096), (96, 128, 256, q.QLD_U8, 37, 256)]
    data = []
    for H, W, N, fmt, k, hi in cases:
        x = rng.integers(0, hi, size=(N, H * W)).astype(np.uint16 if fmt == q.QLD_U16 else np.uint8)
        dev = torch.from_numpy(x.view(np.uint8).reshape(N, -1)).cuda()
        ref = context_bin(dev, H, W, N, fmt, k)
        data.append((H, W, N, fmt, k, x, dev, ref))
    outs = []
    for H, W, N, fmt, k, x, dev, ref in data:  # two calls back to back on the same stream
        out = torch.empty(H * W, dtype=torch.float32, device="cuda")
        q.qld_fft_bin_frames_noalloc(dev, H, W, N, fmt, k, out)
        outs.append(out)
    torch.cuda.synchronize()
    for (H, W, N, fmt, k, x, dev, ref), out in zip(data, outs):
        got = out.cpu().numpy()
        sums = x.astype(np.int64).sum(axis=0)
        check_power(got, ref, sums, "noalloc vs context k=%d" % k)
        # block frame i is frame i + 1 of a fresh stream; |X_k|^2 does not
        # depend on that origin
        check_power(got, oracle.dft_bin(x, k, s0=1)[2], sums, "noalloc vs oracle k=%d" % k)


def test_noalloc_at_its_largest_window_against_the_oracle():
    H, W = 4, 8  # 64-byte uint16 frames: whole 16-byte vectors
    N = q.QLD_NOALLOC_MAX_N
    rng = np.random.default_rng(77)
    x = rng.integers(0, 4096, size=(N, H * W)).astype(np.uint16)
    dev = torch.from_numpy(x.view(np.uint8).reshape(N, -1)).cuda()
    for k in (N // 4, 12345):
        out = torch.empty(H * W, dtype=torch.float32, device="cuda")
        q.qld_fft_bin_frames_noalloc(dev, H, W, N, q.QLD_U16, k, out)
        torch.cuda.synchronize()
        check_power(out.cpu().numpy(), oracle.dft_bin(x, k, s0=1)[2], x.astype(np.int64).sum(axis=0),
                    "noalloc N=%d k=%d" % (N, k))


def test_noalloc_call_after_warm_up_allocates_nothing():
    H, W, N, k = 64, 64, 128, 5
    rng = np.random.default_rng(5)
    x = rng.integers(0, 4096, size=(N, H * W)).astype(np.uint16)
    dev = torch.from_numpy(x.view(np.uint8).reshape(N, -1)).cuda()
    out = torch.empty(H * W, dtype=torch.float32, device="cuda")
    q.qld_fft_bin_frames_noalloc(dev, H, W, N, q.QLD_U16, k, out)  # warm-up: may load code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    acct0 = q.qld_mem_in_use()
    q.qld_fft_bin_frames_noalloc(dev, H, W, N, q.QLD_U16, k + 1, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "device free memory changed by %d bytes" % (free0 - free1)
    assert q.qld_mem_in_use() == acct0
    check_power(out.cpu().numpy(), oracle.dft_bin(x, k + 1, s0=1)[2], x.astype(np.int64).sum(axis=0), "noalloc")


def test_noalloc_rejects_sizes_beyond_its_maximum():
    H, W = 4, 8
    N = q.QLD_NOALLOC_MAX_N + 4
    frames = torch.zeros(N * H * W * 2, dtype=torch.uint8, device="cuda")
    out = torch.empty(H * W, dtype=torch.float32, device="cuda")
    with pytest.raises(q.QLDError) as e:
        q.qld_fft_bin_frames_noalloc(frames, H, W, N, q.QLD_U16, 1, out)
    assert e.value.status == q.QLD_E_INVAL
    with pytest.raises(q.QLDError) as e:
        q.qld_fft_bin_frames_noalloc(frames, H, W, 6, q.QLD_U16, 1, out)  # N not a multiple of 4
    assert e.value.status == q.QLD_E_INVAL
