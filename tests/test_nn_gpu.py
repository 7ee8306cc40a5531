"""The learned path's kernels against the FP64 CPU oracle: BF16 tensor-core
3x3 convolution forward, data gradient and weight gradient, and the small
layers of the U-Net. Inputs are rounded to bf16 first and the oracle runs on
exactly those values, so the only differences are the FP32 accumulation
(bounded relative to sum |x| |w|, computed by the oracle on absolute values)
and, for bf16 outputs, the final rounding (2^-8 relative)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1511_03390_b300 as q

pytestmark = pytest.mark.gpu
ACC = 2e-5  # FP32 accumulation over at most a few thousand exact products


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def bf16(x):
    """(device bf16 tensor, the same values as float64 numpy)."""
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda().to(torch.bfloat16).contiguous()
    return t, t.float().cpu().numpy().astype(np.float64)


def close(got, ref, bound, what):
    err = np.abs(np.asarray(got, np.float64) - ref)
    ok = err <= bound
    assert ok.all(), "%s: %d bad of %d, worst err %g (bound %g)" % (what, (~ok).sum(), ok.size, err.max(),
                                                                     bound.ravel()[np.argmax(err)] if np.ndim(bound) else bound)


@pytest.mark.parametrize("B,H,W,Cin,Cout,relu", [(2, 17, 13, 16, 32, 1), (1, 32, 40, 32, 64, 0), (1, 9, 130, 48, 96, 1),
                                                 (3, 8, 8, 64, 128, 0)])
def test_conv_forward(B, H, W, Cin, Cout, relu):
    rng = np.random.default_rng(B * H + Cin)
    x, xr = bf16(rng.standard_normal((B, H, W, Cin)))
    w, wr = bf16(rng.standard_normal((3, 3, Cin, Cout)) / np.sqrt(9 * Cin))
    bias = torch.from_numpy(rng.standard_normal(Cout).astype(np.float32)).cuda()
    out_f = torch.empty((B, H, W, Cout), dtype=torch.float32, device="cuda")
    out_b = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
    q.nn.conv3x3_fwd(x, w, bias, B, H, W, Cin, Cout, relu, out_b, out_f)
    torch.cuda.synchronize()
    ref = oracle.conv3x3(xr, wr, bias.cpu().numpy().astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0)
    bound = ACC * oracle.conv3x3(np.abs(xr), np.abs(wr)) + 1e-6
    close(out_f.cpu().numpy(), ref, bound, "conv forward f32")
    close(out_b.float().cpu().numpy(), ref, bound + 2.0 ** -8 * np.abs(ref), "conv forward bf16")


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 11, 14, 32, 32), (1, 24, 20, 64, 32), (1, 7, 33, 96, 48)])
def test_conv_data_gradient(B, H, W, Cin, Cout):
    rng = np.random.default_rng(H * W)
    g, gr = bf16(rng.standard_normal((B, H, W, Cout)))
    w, wr = bf16(rng.standard_normal((3, 3, Cin, Cout)) / np.sqrt(9 * Cin))
    scratch = torch.empty(9 * Cin * Cout, dtype=torch.bfloat16, device="cuda")
    din = torch.empty((B, H, W, Cin), dtype=torch.float32, device="cuda")
    q.nn.conv3x3_dgrad(g, w, B, H, W, Cin, Cout, scratch, None, din)
    torch.cuda.synchronize()
    xdummy = np.zeros((B, H, W, Cin))
    ref = oracle.conv3x3_backward(xdummy, wr, gr)[0]
    bound = ACC * oracle.conv3x3_backward(xdummy, np.abs(wr), np.abs(gr))[0] + 1e-6
    close(din.cpu().numpy(), ref, bound, "conv data gradient")


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 13, 17, 16, 32), (1, 40, 36, 32, 64), (2, 9, 9, 48, 96),
                                            (1, 64, 64, 128, 128)])
def test_conv_weight_gradient(B, H, W, Cin, Cout):
    rng = np.random.default_rng(Cin + Cout + W)
    x, xr = bf16(rng.standard_normal((B, H, W, Cin)))
    g, gr = bf16(rng.standard_normal((B, H, W, Cout)))
    dw = torch.zeros(9 * Cin * Cout, dtype=torch.float32, device="cuda")
    q.nn.conv3x3_wgrad(x, g, B, H, W, Cin, Cout, dw)
    db = torch.zeros(Cout, dtype=torch.float32, device="cuda")
    q.nn.bias_grad(g, B * H * W, Cout, db)
    torch.cuda.synchronize()
    wdummy = np.zeros((3, 3, Cin, Cout))
    _, ref, refb = oracle.conv3x3_backward(xr, wdummy, gr)
    _, bnd, bndb = oracle.conv3x3_backward(np.abs(xr), wdummy, np.abs(gr))
    close(dw.cpu().numpy().reshape(3, 3, Cin, Cout), ref, ACC * bnd + 1e-6, "conv weight gradient")
    close(db.cpu().numpy(), refb, ACC * bndb + 1e-6, "bias gradient")


@pytest.mark.parametrize("C", [16, 32, 12], ids=["8-channel vectors", "32 channels", "scalar"])
def test_small_layers_against_numpy(C):
    rng = np.random.default_rng(7)
    B, H, W = 2, 6, 10
    x, xr = bf16(rng.standard_normal((B, H, W, C)))
    pooled = torch.empty((B, H // 2, W // 2, C), dtype=torch.bfloat16, device="cuda")
    q.nn.avgpool2(x, B, H, W, C, pooled)
    ref = xr.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))
    close(pooled.float().cpu().numpy(), ref, 2.0 ** -8 * np.abs(ref) + 1e-7, "avgpool2")
    g = torch.from_numpy(rng.standard_normal((B, H // 2, W // 2, C)).astype(np.float32)).cuda()
    gp = torch.empty((B, H, W, C), dtype=torch.float32, device="cuda")
    q.nn.avgpool2_bwd(g, B, H, W, C, gp, 0)
    close(gp.cpu().numpy(), 0.25 * np.repeat(np.repeat(g.cpu().numpy(), 2, 1), 2, 2), 1e-7, "avgpool2 backward")
    up = torch.empty((B, 2 * H, 2 * W, C), dtype=torch.bfloat16, device="cuda")
    q.nn.upsample2(x, B, H, W, C, up)
    close(up.float().cpu().numpy(), np.repeat(np.repeat(xr, 2, 1), 2, 2), 0, "upsample2")
    gu = torch.from_numpy(rng.standard_normal((B, 2 * H, 2 * W, C)).astype(np.float32)).cuda()
    gd = torch.empty((B, H, W, C), dtype=torch.float32, device="cuda")
    q.nn.upsample2_bwd(gu, B, H, W, C, gd)
    close(gd.cpu().numpy(), gu.cpu().numpy().reshape(B, H, 2, W, 2, C).sum(axis=(2, 4)), 1e-5, "upsample2 backward")
    y, yr = bf16(rng.standard_normal((B, H, W, 32)))
    cat = torch.empty((B, H, W, C + 32), dtype=torch.bfloat16, device="cuda")
    q.nn.concat(x, C, y, 32, B * H * W, cat)
    close(cat.float().cpu().numpy(), np.concatenate([xr, yr], axis=3), 0, "concat")
    gc = torch.from_numpy(rng.standard_normal((B, H, W, C + 32)).astype(np.float32)).cuda()
    ga = torch.empty((B, H, W, C), dtype=torch.float32, device="cuda")
    gb = torch.ones((B, H, W, 32), dtype=torch.float32, device="cuda")
    q.nn.split(gc, B * H * W, C, 32, ga, gb, 1)
    close(ga.cpu().numpy(), gc.cpu().numpy()[..., :C], 0, "split a")
    close(gb.cpu().numpy(), gc.cpu().numpy()[..., C:] + 1, 1e-7, "split b accumulated")
    # head + mse
    w = torch.from_numpy(rng.standard_normal(C).astype(np.float32)).cuda()
    out = torch.empty(B * H * W, dtype=torch.float32, device="cuda")
    q.nn.head(x, w, torch.tensor([0.5], device="cuda"), B * H * W, C, out)
    ref_out = xr.reshape(-1, C) @ w.cpu().numpy().astype(np.float64) + 0.5
    close(out.cpu().numpy(), ref_out, 1e-5 * (np.abs(xr.reshape(-1, C)) @ np.abs(w.cpu().numpy())) + 1e-6, "head")
    t = torch.from_numpy(rng.standard_normal(B * H * W).astype(np.float32)).cuda()
    grad = torch.empty_like(out)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    q.nn.mse(out, t, B * H * W, grad, loss)
    d = out.cpu().numpy().astype(np.float64) - t.cpu().numpy()
    close(loss.cpu().numpy(), [np.mean(d * d)], 1e-5 * np.mean(d * d), "mse")
    close(grad.cpu().numpy(), 2 * d / d.size, 1e-6 * np.abs(2 * d / d.size) + 1e-9, "mse gradient")
    din = torch.empty((B * H * W, C), dtype=torch.float32, device="cuda")
    dw = torch.zeros(C, dtype=torch.float32, device="cuda")
    db = torch.zeros(1, dtype=torch.float32, device="cuda")
    q.nn.head_bwd(x, grad, w, B * H * W, C, din, dw, db)
    gn = grad.cpu().numpy().astype(np.float64)
    close(din.cpu().numpy(), np.outer(gn, w.cpu().numpy()), 1e-6, "head data gradient")
    close(dw.cpu().numpy(), xr.reshape(-1, C).T @ gn, 1e-5 * (np.abs(xr.reshape(-1, C)).T @ np.abs(gn)) + 1e-7,
          "head weight gradient")
    close(db.cpu().numpy(), [gn.sum()], 1e-5 * np.abs(gn).sum(), "head bias gradient")
    # relu backward, Adam step
    act, actr = bf16(rng.standard_normal((B, H, W, C)))
    gf = torch.from_numpy(rng.standard_normal((B, H, W, C)).astype(np.float32)).cuda()
    gbf = torch.empty((B, H, W, C), dtype=torch.bfloat16, device="cuda")
    q.nn.relu_bwd(gf, act, B * H * W * C, gbf)
    close(gbf.float().cpu().numpy(), np.where(actr > 0, gf.cpu().numpy(), 0), 2.0 ** -8 * np.abs(gf.cpu().numpy()),
          "relu backward")
    p = torch.from_numpy(rng.standard_normal(100).astype(np.float32)).cuda()
    p0 = p.cpu().numpy().astype(np.float64)
    gr = torch.from_numpy(rng.standard_normal(100).astype(np.float32)).cuda()
    m = torch.zeros(100, device="cuda")
    v = torch.zeros(100, device="cuda")
    q.nn.adam(p, gr, m, v, 100, 1e-2, 0.9, 0.999, 1e-8, 1, None)
    gg = gr.cpu().numpy().astype(np.float64)
    # first Adam step: m_hat = g, v_hat = g^2, so p moves by lr * g / (|g| + eps)
    close(p.cpu().numpy(), p0 - 1e-2 * gg / (np.abs(gg) + 1e-8), 1e-6, "adam step")


def test_upsample_concat_matches_upsample_then_concat():
    rng = np.random.default_rng(8)
    B, h, w, Cu, Ce = 2, 5, 7, 16, 24
    u, ur = bf16(rng.standard_normal((B, h, w, Cu)))
    e, er = bf16(rng.standard_normal((B, 2 * h, 2 * w, Ce)))
    out = torch.empty((B, 2 * h, 2 * w, Cu + Ce), dtype=torch.bfloat16, device="cuda")
    q.nn.upsample_concat(u, Cu, e, Ce, B, h, w, out)
    torch.cuda.synchronize()
    want = np.concatenate([np.repeat(np.repeat(ur, 2, 1), 2, 2), er], axis=3)
    close(out.float().cpu().numpy(), want, 0, "upsample_concat")
    with pytest.raises(q.QLDError):
        q.nn.upsample_concat(u, 12, e, Ce, B, h, w, out)


@pytest.mark.parametrize("P,C", [(1000, 32), (333, 96), (4096, 256)])
def test_relu_bwd_bias_matches_the_separate_kernels(P, C):
    """The fused ReLU backward + bias gradient: the masked bf16 gradient is
    bit-identical to qldnn_relu_bwd, the bias gradient is the per-channel sum
    of those bf16 values (FP32 accumulation bound)."""
    rng = np.random.default_rng(P + C)
    g = torch.from_numpy(rng.standard_normal((P, C)).astype(np.float32)).cuda()
    act, _ = bf16(rng.standard_normal((P, C)))
    out_ref = torch.empty((P, C), dtype=torch.bfloat16, device="cuda")
    q.nn.relu_bwd(g, act, P * C, out_ref)
    out = torch.empty_like(out_ref)
    db = torch.full((C,), 0.5, dtype=torch.float32, device="cuda")  # accumulates into db
    q.nn.relu_bwd_bias(g, act, P, C, out, db)
    torch.cuda.synchronize()
    assert torch.equal(out, out_ref)
    o = out_ref.float().cpu().numpy().astype(np.float64)
    want = o.sum(axis=0) + 0.5
    close(db.cpu().numpy(), want, ACC * np.abs(o).sum(axis=0) + 1e-6, "fused bias gradient")
    with pytest.raises(q.QLDError):
        q.nn.relu_bwd_bias(g, act, P, 12, out, db)
