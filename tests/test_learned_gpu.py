"""The learned short-window path on the GPU: the whole U-Net's loss and
parameter gradients (BF16 tensor-core kernels) against the FP64 CPU reference
built from the oracle, and a short training run that lowers the loss and
beats the short-window baseline 32 R_32 on held-out stacks."""
import numpy as np
import pytest
import torch

import paper_1511_03390_b300 as q
from paper_1511_03390_b300 import learned
from unet_reference import RefUNet

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("conv", learned.UNet.CONVS)
def test_unet_gradients_match_the_fp64_reference(conv):
    rng = np.random.default_rng(3)
    B, H, W = 2, 16, 24
    prm = learned.Params(seed=5)
    for k in prm.tensors:  # non-zero biases and head so every path carries gradient
        if k.endswith(".b"):
            prm[k]["p"].copy_(torch.from_numpy(rng.standard_normal(prm[k]["p"].numel()).astype(np.float32) * 0.1))
    prm["head.w"]["p"].copy_(torch.from_numpy(rng.standard_normal(32).astype(np.float32) * 0.3))
    net = learned.UNet(prm, B, H, W, conv=conv)
    S = torch.from_numpy(rng.integers(-3000, 3000, B * H * W).astype(np.int32)).cuda()
    C = torch.from_numpy(rng.integers(-3000, 3000, B * H * W).astype(np.int32)).cuda()
    T = torch.from_numpy(rng.uniform(0, 20, B * H * W).astype(np.float32)).cuda()
    net.pack(S, C)
    net.forward()
    net.loss_and_grad(T)
    prm.zero_grad()
    net.backward()
    torch.cuda.synchronize()
    assert net.status.item() == 0
    x = net.a["x"].float().cpu().numpy().astype(np.float64).reshape(B, H, W, 16)
    base = net.baseline.cpu().numpy().astype(np.float64).reshape(B, H, W)
    # the packed input: (S, C, R) * scale in bf16, R and the baseline from float32
    s, c = S.cpu().numpy().astype(np.float32), C.cpu().numpy().astype(np.float32)
    r32 = np.sqrt(s * s + c * c).astype(np.float32) * np.float32(learned.IN_SCALE)
    assert np.allclose(base.ravel(), r32, rtol=1e-6, atol=0)
    assert np.all(x[..., 3:] == 0)
    ref = RefUNet({k: e["p"].cpu().numpy().astype(np.float64) for k, e in prm.tensors.items()}, round_bf16=True)
    pred = ref.forward(x, base)
    loss, gpred = ref.loss(pred, T.cpu().numpy().astype(np.float64).reshape(B, H, W))
    grads = ref.backward(gpred)
    assert abs(net.loss.item() - loss) <= 2e-3 * loss
    for k, e in prm.tensors.items():
        got = e["g"].cpu().numpy().astype(np.float64)
        want = grads[k]
        rel = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30)
        cos = float(got @ want) / max(np.linalg.norm(got) * np.linalg.norm(want), 1e-30)
        assert rel < 2e-2 and cos > 0.999, (k, rel, cos)
    stagewise_check(net, prm, B, H, W, T)


def stagewise_check(net, prm, B, H, W, T):
    """Every stage of the network's forward and backward pass, elementwise,
    against FP64 recomputed from the GPU's own inputs to that stage (the
    stage's bf16 / float32 tensors read back), so each bound is that stage's
    own arithmetic: a convolution's FP32 accumulation relative to the sum over
    absolute values (ACC, ACC_W of the per-kernel tests) plus the final bf16
    rounding (2^-8 relative); pooling, upsampling, concatenation, split and
    the ReLU mask are emulated exactly. (A bound carried through the whole
    network over absolute weights grows about sqrt(9 Cin) per layer and says
    nothing; the end-to-end check above is the norm one.)"""
    import oracle
    from test_nn_gpu import ACC, close
    from test_nn_tc_gpu import ACC_W
    from unet_reference import LAYERS, bf16r, pool, pool_bwd, up, up_bwd

    U = 2.0 ** -8
    dims = [(H >> l, W >> l) for l in range(4)]
    a = {k: v.float().cpu().numpy().astype(np.float64) for k, v in net.a.items()}
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in net.g.items()}
    level = {"x": 0, "a0": 0, "e0": 0, "p0": 1, "a1": 1, "e1": 1, "p1": 2, "a2": 2, "e2": 2, "p2": 3, "a3": 3,
             "u3": 3, "cat2": 2, "ad2": 2, "u2": 2, "cat1": 1, "ad1": 1, "u1": 1, "cat0": 0, "ad0": 0, "u0": 0,
             "up1": 0, "up2": 1, "up3": 2}

    def t(d, k):
        h, w = dims[level[k]]
        return d[k].reshape(B, h, w, -1)

    def wb(name):
        _, cin, cout = next(l for l in LAYERS if l[0] == name)
        w = prm[name + ".w"]["p"].cpu().numpy().astype(np.float64)
        return bf16r(w).reshape(3, 3, cin, cout), prm[name + ".b"]["p"].cpu().numpy().astype(np.float64)

    # forward: conv + bias + ReLU into bf16, pooling, upsample + concat
    convs = [("c0a", "x", "a0"), ("c0b", "a0", "e0"), ("c1a", "p0", "a1"), ("c1b", "a1", "e1"), ("c2a", "p1", "a2"),
             ("c2b", "a2", "e2"), ("c3a", "p2", "a3"), ("c3b", "a3", "u3"), ("d2a", "cat2", "ad2"),
             ("d2b", "ad2", "u2"), ("d1a", "cat1", "ad1"), ("d1b", "ad1", "u1"), ("d0a", "cat0", "ad0"),
             ("d0b", "ad0", "u0")]
    for name, src, dst in convs:
        w, b = wb(name)
        x = t(a, src)
        ref = np.maximum(oracle.conv3x3(x, w, b), 0)
        bound = ACC * (oracle.conv3x3(np.abs(x), np.abs(w)) + np.abs(b)) + 1e-6
        close(t(a, dst), ref, bound + U * np.abs(ref), "forward " + name)
    for src, dst in (("e0", "p0"), ("e1", "p1"), ("e2", "p2")):
        assert np.array_equal(t(a, dst), bf16r(pool(t(a, src)))), "pool " + dst
    for u, e, dst in (("u3", "e2", "cat2"), ("u2", "e1", "cat1"), ("u1", "e0", "cat0")):
        assert np.array_equal(t(a, dst), np.concatenate([up(t(a, u)), t(a, e)], axis=3)), "concat " + dst
    # head and loss gradient (float32)
    hw = prm["head.w"]["p"].cpu().numpy().astype(np.float64)
    hb = prm["head.b"]["p"].cpu().numpy().astype(np.float64)
    u0 = t(a, "u0")
    base = net.baseline.cpu().numpy().astype(np.float64).reshape(B, H, W)
    pred = u0 @ hw + hb[0] + base
    close(net.pred.cpu().numpy().reshape(B, H, W), pred, ACC * (np.abs(u0) @ np.abs(hw) + abs(hb[0]) + np.abs(base))
          + 1e-6, "head")
    gp = net.gpred.cpu().numpy().astype(np.float64).reshape(B, H, W)
    pr = net.pred.cpu().numpy().astype(np.float64).reshape(B, H, W)
    gref = 2 * (pr - T.cpu().numpy().astype(np.float64).reshape(B, H, W)) / pr.size
    close(gp, gref, 1e-6 * np.abs(gref) + 1e-12, "loss gradient")
    close(t(g, "u0"), gp[..., None] * hw, 1e-6 * np.abs(gp[..., None] * hw) + 1e-12, "head data gradient")
    # sums over pixels: FP32 in any order is within n 2^-24 of the sum of
    # absolute values
    nsum = lambda P: P * 2.0 ** -24  # noqa: E731
    close(prm["head.w"]["g"].cpu().numpy(), np.einsum("bhwc,bhw->c", u0, gp),
          nsum(B * H * W) * np.einsum("bhwc,bhw->c", np.abs(u0), np.abs(gp)) + 1e-9, "head weight gradient")
    close(prm["head.b"]["g"].cpu().numpy(), [gp.sum()], nsum(B * H * W) * np.abs(gp).sum() + 1e-9,
          "head bias gradient")
    # backward through each convolution: ReLU mask into bf16 (exact), weight,
    # bias and data gradients within the FP32 accumulation bound
    for name, src, dst in reversed(convs):
        w, _ = wb(name)
        x, y, gy = t(a, src), t(a, dst), t(g, dst)
        gz = bf16r(np.where(y > 0, gy, 0.0))
        dx, dw, db = oracle.conv3x3_backward(x, w, gz)
        mx, mw, mb = oracle.conv3x3_backward(np.abs(x), np.abs(w), np.abs(gz))
        close(prm[name + ".w"]["g"].cpu().numpy().reshape(dw.shape), dw, ACC_W * mw + 1e-6, "weight gradient " + name)
        close(prm[name + ".b"]["g"].cpu().numpy(), db, nsum(x.shape[0] * x.shape[1] * x.shape[2]) * mb + 1e-6,
              "bias gradient " + name)
        if src != "x":
            close(t(g, src), dx, ACC * mx + 1e-6, "data gradient " + name)
    # the gradient plumbing between the convolutions (float32, exact but for
    # the sums of four in upsample's backward and the pooled adds)
    for cat, upk, e, uk, c in (("cat0", "up1", "e0", "u1", 32), ("cat1", "up2", "e1", "u2", 64),
                               ("cat2", "up3", "e2", "u3", 128)):
        assert np.array_equal(t(g, upk), t(g, cat)[..., :c]), "split " + cat
        close(t(g, uk), up_bwd(t(g, upk)), 1e-6 * up_bwd(np.abs(t(g, upk))) + 1e-12, "upsample backward " + uk)
    for e, c, p in (("e2", 128, "p2"), ("e1", 64, "p1"), ("e0", 32, "p0")):
        cat = {"e0": "cat0", "e1": "cat1", "e2": "cat2"}[e]
        want = t(g, cat)[..., c:] + pool_bwd(t(g, p))
        close(t(g, e), want, 1e-6 * np.abs(want) + 1e-12, "skip + pooling backward " + e)


def test_short_training_run_beats_the_short_window_baseline():
    H = W = 128
    S, C, T, _ = learned.make_dataset(40, H, W, seed=7)
    prm = learned.Params(seed=1)
    hist = learned.train(prm, S[:32], C[:32], T[:32], H, W, steps=300, batch=4, crop=64, lr=2e-3, log_every=50)
    assert hist[-1][1] < 0.5 * hist[0][1]
    ev = learned.evaluate(prm, S[32:], C[32:], T[32:], H, W, batch=2)
    assert ev["network"][0] < ev["baseline"][0], ev
    assert ev["network"][1] > ev["baseline"][1], ev


def test_trained_network_gains_over_the_short_window_baseline():
    """The committed network against plain QLD's own short-window estimate
    32 R_32, both judged by plain QLD over 1024 frames, on stacks from a seed
    the training never saw: the network cuts the relative L2 error several
    times and gains more than 10 dB of PSNR."""
    H = W = 512
    prm = learned.load(learned.WEIGHTS)
    S, C, T, ods = learned.make_dataset(6, H, W, seed=777)
    ev = learned.evaluate(prm, S, C, T, H, W, batch=2)
    net_rel, net_psnr = ev["network"]
    base_rel, base_psnr = ev["baseline"]
    assert net_rel < 0.25 * base_rel, ev
    assert net_psnr > base_psnr + 10.0, ev


def test_graph_replay_matches_eager_forward():
    """The captured pack+forward graph gives bit-identical predictions to the
    eager calls on new inputs written into its input buffers."""
    rng = np.random.default_rng(11)
    B, H, W = 1, 64, 96
    prm = learned.Params(seed=2)
    eager = learned.UNet(prm, B, H, W, inference_only=True)
    graph = learned.UNet(prm, B, H, W, inference_only=True).capture()
    for _ in range(2):
        S = torch.from_numpy(rng.integers(-5000, 5000, B * H * W).astype(np.int32)).cuda()
        C = torch.from_numpy(rng.integers(-5000, 5000, B * H * W).astype(np.int32)).cuda()
        eager.pack(S, C)
        want = eager.forward().clone()
        graph.S_in.copy_(S)
        graph.C_in.copy_(C)
        got = graph.replay()
        torch.cuda.synchronize()
        assert graph.status.item() == 0 and eager.status.item() == 0
        assert torch.equal(got, want)


@pytest.mark.parametrize("B,H,W", [(1, 64, 96), (2, 32, 48)])
def test_fused_inference_forward_matches_the_layer_by_layer_pass(B, H, W):
    """Inference nets fuse pooling, upsample + concat and the head into the
    convolution epilogues; training nets run them as separate kernels. The
    predictions must agree bit for bit."""
    rng = np.random.default_rng(B * H + W)
    prm = learned.Params(seed=9)
    for k in prm.tensors:  # non-zero biases and head
        if k.endswith(".b"):
            prm[k]["p"].copy_(torch.from_numpy(rng.standard_normal(prm[k]["p"].numel()).astype(np.float32) * 0.1))
    prm["head.w"]["p"].copy_(torch.from_numpy(rng.standard_normal(32).astype(np.float32) * 0.3))
    fused = learned.UNet(prm, B, H, W, inference_only=True, fuse_input=False)
    plain = learned.UNet(prm, B, H, W)
    assert fused.fused and not plain.fused
    S = torch.from_numpy(rng.integers(-5000, 5000, B * H * W).astype(np.int32)).cuda()
    C = torch.from_numpy(rng.integers(-5000, 5000, B * H * W).astype(np.int32)).cuda()
    fused.pack(S, C)
    plain.pack(S, C)
    want = plain.forward().clone()
    got = fused.forward()
    torch.cuda.synchronize()
    assert fused.status.item() == 0 and plain.status.item() == 0
    assert torch.equal(got, want)
    # the first layer on the FP32 cores (input packing fused) sums in another
    # order: predictions agree to FP32 accumulation and bf16 storage rounding
    full = learned.UNet(prm, B, H, W, inference_only=True, fuse_input=True)
    full.pack(S, C)
    got2 = full.forward()
    torch.cuda.synchronize()
    assert torch.equal(full.baseline, plain.baseline)
    rel = (torch.linalg.norm(got2 - want) / torch.linalg.norm(want)).item()
    assert rel < 1e-2, rel


@pytest.mark.parametrize("B,H,W,Cout", [(1, 16, 16, 32), (2, 37, 50, 32), (1, 40, 24, 64)])
def test_input_conv_matches_the_oracle_on_the_packed_input(B, H, W, Cout):
    """qldnn_input_conv3x3 = ReLU(conv3x3(pack(S, C)) + bias) against the FP64
    oracle on the packed tensor the GPU builds (16 channels, zeros after 3),
    and its baseline = qldnn_pack_input's."""
    import oracle
    from test_nn_gpu import ACC, bf16, close

    rng = np.random.default_rng(H * W + Cout)
    S = torch.from_numpy(rng.integers(-9000, 9000, B * H * W).astype(np.int32)).cuda()
    C = torch.from_numpy(rng.integers(-9000, 9000, B * H * W).astype(np.int32)).cuda()
    x = torch.empty(B * H * W * 16, dtype=torch.bfloat16, device="cuda")
    base = torch.empty(B * H * W, dtype=torch.float32, device="cuda")
    q.nn.pack_input(S, C, B * H * W, learned.IN_SCALE, x, base)
    w, wr = bf16(rng.standard_normal((3, 3, 16, Cout)) / 12)
    bias = torch.from_numpy(rng.standard_normal(Cout).astype(np.float32) * 0.1).cuda()
    out = torch.empty(B * H * W * Cout, dtype=torch.bfloat16, device="cuda")
    base2 = torch.empty_like(base)
    q.nn.input_conv3x3(S, C, B, H, W, learned.IN_SCALE, w, 16, Cout, bias, 1, out, Cout, base2)
    torch.cuda.synchronize()
    assert torch.equal(base, base2)
    xr = x.float().cpu().numpy().astype(np.float64).reshape(B, H, W, 16)
    ref = np.maximum(oracle.conv3x3(xr, wr, bias.cpu().numpy().astype(np.float64)), 0)
    bound = ACC * oracle.conv3x3(np.abs(xr), np.abs(wr)) + 1e-6
    close(out.float().cpu().numpy().reshape(B, H, W, Cout), ref, bound + 2.0 ** -8 * np.abs(ref), "input conv")


def test_epi_conv_rejects_unknown_flags():
    x = torch.zeros(64 * 64 * 32, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(9 * 32 * 32, dtype=torch.bfloat16, device="cuda")
    out = torch.empty_like(x)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = q.lib.qldnn_conv3x3_fwd_tma_epi(x.data_ptr(), w.data_ptr(), None, 1, 64, 64, 32, 32, 1, out.data_ptr(), 32,
                                         None, None, 32, None, None, None, None, st.data_ptr(), 2, None)
    assert rc == q.QLD_E_INVAL


def test_network_reading_the_context_sums_in_place_equals_the_copied_input():
    """A network captured on a QLD context's own sums (qld_iq_pointers) gives
    the same prediction, bit for bit, as one fed copies of them (qld_get_iq),
    after each of several pushes; the accessor returns the context's live
    buffers."""
    from qldscene import DeviceScene, scene_fog

    H = W = 64
    prm = learned.Params(seed=3)
    ctx = q.qld_create(H, W, learned.N_SHORT, q.QLD_U16)
    try:
        frames = torch.empty((3 * learned.N_SHORT, H, W), dtype=torch.uint16, device="cuda")
        DeviceScene(scene_fog(6, seed=77, H=H, W=W), torch.device("cuda")).generate_into(frames, 1, 3 * learned.N_SHORT)
        Sp, Cp = q.qld_iq_pointers(ctx)
        inplace = learned.UNet(prm, 1, H, W, inference_only=True).capture(Sp, Cp)
        copied = learned.UNet(prm, 1, H, W, inference_only=True).capture()
        st = torch.cuda.current_stream()
        for k in range(3):
            q.qld_push_frames(ctx, frames[k * learned.N_SHORT:(k + 1) * learned.N_SHORT], learned.N_SHORT, st)
            got = inplace.replay().clone()
            q.qld_get_iq(ctx, copied.S_in, copied.C_in)
            want = copied.replay().clone()
            torch.cuda.synchronize()
            assert torch.equal(got, want)
        S = torch.empty(H * W, dtype=torch.int32, device="cuda")
        q.qld_get_iq(ctx, S, None)
        torch.cuda.synchronize()
        assert q.qld_iq_pointers(ctx)[0] == Sp
    finally:
        q.qld_destroy(ctx)
