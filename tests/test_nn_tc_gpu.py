"""The tensor-memory (tcgen05) convolutions (the two-buffer kernel, the
warp-specialised pipelined one and the persistent TMA-fed one in both its
weights-resident and weight-streaming variants) against the FP64 oracle and the warp-MMA
kernel: forward with bias/ReLU and, with flipped weights, the data gradient. Same tolerance as the other convolution tests (FP32 accumulation
relative to sum |x| |w|, plus bf16 output rounding)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q
from test_nn_gpu import ACC, bf16, close

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# conv3x3_fwd_tma keeps small layers' weights resident in shared memory and
# splits small layers' output channels over several CTAs per tile;
# "conv3x3_fwd_tma_stream" forces its weight-streaming variant, "..._split2" /
# "..._split4" force 2 / 4 CTAs per tile, "..._sub2" 16 x 16-pixel tiles (two
# stacked 8 x 16 sub-tiles), "..._two" two CTAs per SM, "..._xs*" the column
# taps stacked in N (14-column tiles; 8-row tiles, 16-row tiles, two CTAs per
# SM; with 2 CTAs per tile), "..._stream" / "..._stream_wide" the
# weight-streaming kernel with four / eight epilogue warps (eight: 64+
# columns, the default there), on every shape they apply to (the others run
# the unstacked or four-warp kernel).
# The automatic choice stacks the column taps of some layers (those with
# many input channels per output column); "..._noxs" and the unstacked
# variants forbid it (mode bit 17).
XS, NOXS = 1 << 16, 1 << 17
KERNELS = ["conv3x3_fwd_tc", "conv3x3_fwd_tc2", "conv3x3_fwd_tma", "conv3x3_fwd_tma_noxs", "conv3x3_fwd_tma_stream",
           "conv3x3_fwd_tma_split2", "conv3x3_fwd_tma_split4", "conv3x3_fwd_tma_sub2", "conv3x3_fwd_tma_two",
           "conv3x3_fwd_tma_two_sub1", "conv3x3_fwd_tma_xs_sub1", "conv3x3_fwd_tma_xs_sub2",
           "conv3x3_fwd_tma_xs_two", "conv3x3_fwd_tma_xs_split2", "conv3x3_fwd_tma_stream_wide"]
MODES = {"conv3x3_fwd_tma_noxs": NOXS, "conv3x3_fwd_tma_stream": 1 | (1 << 19), "conv3x3_fwd_tma_split2": NOXS | (2 << 4),
         "conv3x3_fwd_tma_split4": NOXS | (4 << 4), "conv3x3_fwd_tma_sub2": NOXS | (1 << 12),
         "conv3x3_fwd_tma_two": NOXS | (1 << 15) | (1 << 12), "conv3x3_fwd_tma_two_sub1": NOXS | (1 << 15) | (1 << 13),
         "conv3x3_fwd_tma_xs_sub1": XS | (1 << 13) | (1 << 14), "conv3x3_fwd_tma_xs_sub2": XS | (1 << 12) | (1 << 14),
         "conv3x3_fwd_tma_xs_two": XS | (1 << 15), "conv3x3_fwd_tma_xs_split2": XS | (2 << 4),
         "conv3x3_fwd_tma_stream_wide": NOXS | 1 | (1 << 18)}


def _tc(kernel, Cout):
    if kernel != "conv3x3_fwd_tc" and Cout not in (32, 64, 128, 256):
        pytest.skip("the pipelined kernels cover Cout in {32, 64, 128, 256}")
    if kernel in MODES:
        mode = MODES[kernel]
        if Cout // max(1, (mode >> 4) & 0xF) < 32:
            pytest.skip("at least 32 output channels per CTA")
        return lambda *a: q.nn.conv3x3_fwd_tma_mode(*a, mode)
    return getattr(q.nn, kernel)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("B,H,W,Cin,Cout,relu", [(1, 8, 16, 16, 32, 0), (2, 17, 13, 16, 64, 1), (1, 32, 40, 32, 64, 0),
                                                 (1, 9, 130, 48, 96, 1), (3, 8, 8, 64, 128, 0),
                                                 (1, 24, 24, 256, 128, 1), (2, 19, 21, 128, 256, 1),
                                                 (1, 7, 5, 64, 32, 0), (1, 9, 130, 48, 64, 1),
                                                 (4, 96, 160, 32, 32, 1)])
def test_tc_conv_forward(kernel, B, H, W, Cin, Cout, relu):
    conv = _tc(kernel, Cout)
    rng = np.random.default_rng(B * H + Cin + 1)
    x, xr = bf16(rng.standard_normal((B, H, W, Cin)))
    w, wr = bf16(rng.standard_normal((3, 3, Cin, Cout)) / np.sqrt(9 * Cin))
    bias = torch.from_numpy(rng.standard_normal(Cout).astype(np.float32)).cuda()
    wk = torch.empty(9 * Cin * Cout, dtype=torch.bfloat16, device="cuda")
    q.nn.kmajor_weights(w, Cin, Cout, 0, wk)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out_f = torch.empty((B, H, W, Cout), dtype=torch.float32, device="cuda")
    out_b = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
    conv(x, wk, bias, B, H, W, Cin, Cout, relu, out_b, out_f, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    ref = oracle.conv3x3(xr, wr, bias.cpu().numpy().astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0)
    bound = ACC * oracle.conv3x3(np.abs(xr), np.abs(wr)) + 1e-6
    close(out_f.cpu().numpy(), ref, bound, "tcgen05 forward f32")
    close(out_b.float().cpu().numpy(), ref, bound + 2.0 ** -8 * np.abs(ref), "tcgen05 forward bf16")
    # the warp-MMA kernel agrees within the same bound
    out_m = torch.empty((B, H, W, Cout), dtype=torch.float32, device="cuda")
    q.nn.conv3x3_fwd(x, w, bias, B, H, W, Cin, Cout, relu, None, out_m)
    torch.cuda.synchronize()
    close(out_f.cpu().numpy(), out_m.cpu().numpy().astype(np.float64), 2 * bound, "tcgen05 vs warp MMA")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 11, 14, 32, 32), (1, 24, 20, 64, 32), (1, 16, 16, 128, 256)])
def test_tc_conv_data_gradient(kernel, B, H, W, Cin, Cout):
    conv = _tc(kernel, Cin)
    rng = np.random.default_rng(H * W + 3)
    g, gr = bf16(rng.standard_normal((B, H, W, Cout)))
    w, wr = bf16(rng.standard_normal((3, 3, Cin, Cout)) / np.sqrt(9 * Cin))
    wk = torch.empty(9 * Cin * Cout, dtype=torch.bfloat16, device="cuda")
    q.nn.kmajor_weights(w, Cin, Cout, 1, wk)
    din = torch.empty((B, H, W, Cin), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    conv(g, wk, None, B, H, W, Cout, Cin, 0, None, din, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    xdummy = np.zeros((B, H, W, Cin))
    ref = oracle.conv3x3_backward(xdummy, wr, gr)[0]
    bound = ACC * oracle.conv3x3_backward(xdummy, np.abs(wr), np.abs(gr))[0] + 1e-6
    close(din.cpu().numpy(), ref, bound, "tcgen05 data gradient")


# The weight gradient sums over every pixel (up to ~4e4 products per entry
# here, plus cross-CTA float atomics in no fixed order): FP32 accumulation
# error of order sqrt(n) * 2^-24 * sum |x| |g|, bounded here by 1e-4 * sum |x| |g|.
ACC_W = 1e-4


def _abs_wgrad(x, g):
    """sum over pixels of |x shifted by the tap| |g|: the scale of the
    tolerance (not the reference), by one matrix product per tap."""
    B, H, W, Cin = x.shape
    xp = np.pad(np.abs(x), ((0, 0), (1, 1), (1, 1), (0, 0)))
    ga = np.abs(g).reshape(-1, g.shape[3])
    out = np.empty((3, 3, Cin, g.shape[3]))
    for ky in range(3):
        for kx in range(3):
            out[ky, kx] = xp[:, ky:ky + H, kx:kx + W, :].reshape(-1, Cin).T @ ga
    return out


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 13, 21, 16, 32), (1, 9, 30, 32, 32), (2, 17, 15, 32, 64),
                                            (1, 24, 20, 64, 64), (2, 11, 19, 64, 32), (1, 16, 24, 64, 128),
                                            (1, 20, 18, 128, 128), (2, 9, 33, 256, 128), (1, 12, 16, 128, 64),
                                            (1, 10, 12, 16, 128), (2, 128, 160, 16, 32), (1, 64, 208, 256, 32)])
def test_tma_weight_gradient(B, H, W, Cin, Cout):
    rng = np.random.default_rng(B * 1000 + H * W + Cin + Cout)
    x, xr = bf16(rng.standard_normal((B, H, W, Cin)))
    g, gr = bf16(rng.standard_normal((B, H, W, Cout)))
    dw = torch.zeros(9 * Cin * Cout, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    q.nn.conv3x3_wgrad_tma(x, g, B, H, W, Cin, Cout, dw, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    ref = oracle.conv3x3_backward(xr, np.zeros((3, 3, Cin, Cout)), gr)[1]
    bnd = _abs_wgrad(xr, gr)
    close(dw.cpu().numpy().reshape(3, 3, Cin, Cout), ref, ACC_W * bnd + 1e-6, "tcgen05 weight gradient")
    # accumulates into dw: a second call doubles it
    q.nn.conv3x3_wgrad_tma(x, g, B, H, W, Cin, Cout, dw, status)
    torch.cuda.synchronize()
    close(dw.cpu().numpy().reshape(3, 3, Cin, Cout), 2 * ref, 2 * ACC_W * bnd + 1e-6, "accumulated twice")


def test_tma_weight_gradient_rejects_unsupported_shapes():
    x = torch.zeros(4 * 4 * 48, dtype=torch.bfloat16, device="cuda")
    g = torch.zeros(4 * 4 * 256, dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros(9 * 48 * 256, dtype=torch.float32, device="cuda")
    for cin, cout in [(48, 32), (96, 64), (64, 256), (64, 48)]:
        with pytest.raises(q.QLDError):
            q.nn.conv3x3_wgrad_tma(x, g, 1, 4, 4, cin, cout, dw, None)


def test_bounded_wait_times_out_raises_the_flag_and_leaves_the_context_usable():
    """The failure path of the tcgen05 kernels' bounded waits: a wait on an
    mbarrier nothing arrives on gives up after its limit and raises the
    failure flag, a second role with a one-minute limit leaves at once, and
    the next kernels run normally (no fault, no hang)."""
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    q.nn.wait_selftest(5_000_000, out)  # 5 ms
    torch.cuda.synchronize()
    timed_out, left_on_flag, ns = out.cpu().tolist()
    assert timed_out == 1 and left_on_flag == 1
    assert 5_000_000 <= ns < 1_000_000_000, ns
    # the context is still usable: a convolution afterwards reports no failure
    x = torch.randn(1 * 8 * 16 * 32, device="cuda").to(torch.bfloat16)
    w = (torch.randn(9 * 32 * 32, device="cuda") * 0.05).to(torch.bfloat16)
    wk = torch.empty_like(w)
    q.nn.kmajor_weights(w, 32, 32, 0, wk)
    y = torch.empty(8 * 16 * 32, dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    q.nn.conv3x3_fwd_tma(x, wk, None, 1, 8, 16, 32, 32, 1, y, None, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    with pytest.raises(q.QLDError):
        q.nn.wait_selftest(10, out)  # below the 1 us minimum


@pytest.mark.parametrize("B,H,W,Cin,Cout,relu", [(1, 64, 48, 32, 32, 1), (2, 33, 40, 16, 64, 0), (1, 48, 80, 96, 32, 1),
                                                 (1, 17, 31, 48, 64, 1), (1, 7, 16, 32, 32, 0)])
def test_tma_16x16_tiles_equal_8x16_tiles(B, H, W, Cin, Cout, relu):
    """Two stacked sub-tiles per pipeline step run the same MMAs per
    accumulator as single 8 x 16 tiles when both stage the same channel
    chunks (inputs of at most 32-channel chunks: Cin not a multiple of 64):
    identical outputs, bit for bit. (Multiples of 64 channels run in 32-channel
    chunks with 16 x 16 tiles, 64-channel ones otherwise: the oracle parity
    test covers those.)"""
    rng = np.random.default_rng(H * W + Cin + Cout)
    x, _ = bf16(rng.standard_normal((B, H, W, Cin)))
    w, _ = bf16(rng.standard_normal((3, 3, Cin, Cout)) / np.sqrt(9 * Cin))
    bias = torch.from_numpy(rng.standard_normal(Cout).astype(np.float32)).cuda()
    wk = torch.empty(9 * Cin * Cout, dtype=torch.bfloat16, device="cuda")
    q.nn.kmajor_weights(w, Cin, Cout, 0, wk)
    outs = []
    for mode in (NOXS | (1 << 12), NOXS | (1 << 13), XS | (1 << 12) | (1 << 14), XS | (1 << 13) | (1 << 14)):
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        out_f = torch.full((B, H, W, Cout), float("nan"), dtype=torch.float32, device="cuda")
        out_b = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
        q.nn.conv3x3_fwd_tma_mode(x, wk, bias, B, H, W, Cin, Cout, relu, out_b, out_f, status, mode)
        torch.cuda.synchronize()
        assert status.item() == 0
        outs.append((out_f.cpu(), out_b.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    # stacked column taps: the same between their own tile heights
    assert torch.equal(outs[2][0], outs[3][0]) and torch.equal(outs[2][1], outs[3][1])


@pytest.mark.parametrize("B,H,W,Cin,Cout,relu", [(1, 64, 48, 32, 32, 1), (2, 33, 40, 16, 32, 0), (1, 48, 80, 96, 32, 1),
                                                 (1, 17, 31, 48, 32, 1), (1, 7, 16, 32, 32, 0), (1, 64, 48, 32, 64, 1),
                                                 (2, 33, 40, 16, 64, 0)])
def test_tma_two_ctas_per_sm_equal_one(B, H, W, Cin, Cout, relu):
    """Two CTAs per SM run the same tiles, MMAs and epilogue as one CTA per SM
    with the same channel chunks and tile height: identical outputs, bit for
    bit (Cin not a multiple of 64, so both stage chunks of at most 32)."""
    rng = np.random.default_rng(H * W + Cin + 7)
    x, _ = bf16(rng.standard_normal((B, H, W, Cin)))
    w, _ = bf16(rng.standard_normal((3, 3, Cin, Cout)) / np.sqrt(9 * Cin))
    bias = torch.from_numpy(rng.standard_normal(Cout).astype(np.float32)).cuda()
    wk = torch.empty(9 * Cin * Cout, dtype=torch.bfloat16, device="cuda")
    q.nn.kmajor_weights(w, Cin, Cout, 0, wk)
    for sub in (NOXS | (1 << 12), NOXS | (1 << 13), XS | (1 << 13)):
        outs = []
        for two in (1 << 15, 1 << 14):
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            out_f = torch.full((B, H, W, Cout), float("nan"), dtype=torch.float32, device="cuda")
            out_b = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
            q.nn.conv3x3_fwd_tma_mode(x, wk, bias, B, H, W, Cin, Cout, relu, out_b, out_f, status, sub | two)
            torch.cuda.synchronize()
            assert status.item() == 0
            outs.append((out_f.cpu(), out_b.cpu()))
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(1, 40, 72, 32, 32), (2, 18, 30, 16, 64), (1, 24, 58, 64, 32)])
def test_tma_stacked_column_taps_with_fused_outputs(B, H, W, Cin, Cout):
    """The column-stacked kernel's fused epilogue outputs (2 x 2 average,
    nearest 2x upsampling, the 1x1 head plus baseline) against the same
    operations applied on the CPU to its own bf16 activation, which is itself
    checked against the FP64 oracle; every pooling block and upsampled pixel
    of a tile edge (14-column tiles, W not a multiple of 14) included."""
    rng = np.random.default_rng(H * W + Cin + 11)
    x, xr = bf16(rng.standard_normal((B, H, W, Cin)))
    w, wr = bf16(rng.standard_normal((3, 3, Cin, Cout)) / np.sqrt(9 * Cin))
    bias = torch.from_numpy(rng.standard_normal(Cout).astype(np.float32) * 0.1).cuda()
    wk = torch.empty(9 * Cin * Cout, dtype=torch.bfloat16, device="cuda")
    q.nn.kmajor_weights(w, Cin, Cout, 0, wk)
    hw = torch.from_numpy(rng.standard_normal(Cout).astype(np.float32) * 0.3).cuda()
    hb = torch.tensor([0.25], dtype=torch.float32, device="cuda")
    base = torch.from_numpy(rng.standard_normal(B * H * W).astype(np.float32)).cuda()
    for sub in ((1 << 13) | (1 << 14), (1 << 12) | (1 << 14), 1 << 15):
        out = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
        pool = torch.full((B, H // 2, W // 2, Cout), float("nan"), dtype=torch.bfloat16, device="cuda")
        up = torch.full((B, 2 * H, 2 * W, Cout), float("nan"), dtype=torch.bfloat16, device="cuda")
        pred = torch.full((B * H * W,), float("nan"), dtype=torch.float32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = q.lib.qldnn_conv3x3_fwd_tma_epi_mode(
            x.data_ptr(), wk.data_ptr(), bias.data_ptr(), B, H, W, Cin, Cout, 1, out.data_ptr(), Cout,
            pool.data_ptr(), up.data_ptr(), Cout, hw.data_ptr(), hb.data_ptr(), base.data_ptr(),
            pred.data_ptr(), status.data_ptr(), 0, XS | sub, None)
        assert rc == 0
        torch.cuda.synchronize()
        assert status.item() == 0
        act = out.float().cpu().numpy().astype(np.float64)
        ref = np.maximum(oracle.conv3x3(xr, wr, bias.cpu().numpy().astype(np.float64)), 0)
        bound = ACC * oracle.conv3x3(np.abs(xr), np.abs(wr)) + 1e-6
        close(act, ref, bound + 2.0 ** -8 * np.abs(ref), "stacked-tap activation")
        # the fused outputs from the activation as stored
        a32 = out.float().cpu().numpy()
        blk = a32[:, :H // 2 * 2, :W // 2 * 2].reshape(B, H // 2, 2, W // 2, 2, Cout)
        pw = ((blk[:, :, 0, :, 0] + blk[:, :, 1, :, 1]) + (blk[:, :, 0, :, 1] + blk[:, :, 1, :, 0])) * np.float32(0.25)
        pw = torch.from_numpy(np.ascontiguousarray(pw)).to(torch.bfloat16).float().numpy()
        assert np.array_equal(pool.float().cpu().numpy(), pw)
        uw = np.repeat(np.repeat(a32, 2, axis=1), 2, axis=2)
        assert np.array_equal(up.float().cpu().numpy(), uw)
        hp = np.einsum("bhwc,c->bhw", act, hw.cpu().numpy().astype(np.float64)) + 0.25
        hp = hp.reshape(-1) + base.cpu().numpy()
        scale = np.einsum("bhwc,c->bhw", np.abs(act), np.abs(hw.cpu().numpy())).reshape(-1) + 1
        assert np.all(np.abs(pred.cpu().numpy() - hp) <= 1e-5 * scale)
