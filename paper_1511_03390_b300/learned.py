"""Learned short-window QLD.

The paper has no learned component; it motivates shorter time series because
they cut acquisition time and so latency (the tree/cow experiment: sharper
contrast needs longer series, at the cost of a later first image). This
module maps the I/Q maps of a short window (N = 32 frames) to the amplitude
that plain QLD reaches with a long window (N = 1024 frames), using a 4-level
U-Net with 32 base channels (1.06 M parameters) whose convolutions, pooling,
upsampling, head, loss and Adam steps all run in the library's kernels
(qldnn_* in include/qld.h): BF16 tensor-core implicit-GEMM convolutions with
FP32 accumulation, forward and backward. Plain QLD stays the fallback and the
reference: the training targets are plain-QLD amplitudes of simulated stacks, and
the network predicts a correction to the short-window estimate 32 R_32.

Units: network input channels are (S_32, C_32, R_32) * IN_SCALE; targets are
R_1024 * TARGET_SCALE, with TARGET_SCALE = IN_SCALE / 32 so the short-window
baseline 32 R_32 is the input's third channel.
"""
import math

import numpy as np
import torch

from . import QLD_U16, nn, qld_create, qld_get_iq, qld_image, qld_push_frames, qld_reset, qld_sync

N_SHORT = 32
N_LONG = 1024
IN_SCALE = 1.0 / 200.0
TARGET_SCALE = IN_SCALE / N_SHORT
CIN = 16  # input channels: S, C, R, zero padding
EARLY_LAUNCH = 1  # QLDNN_EARLY_LAUNCH (qld.h)

# (name, input channels, output channels); every convolution is 3x3 + ReLU
LAYERS = [("c0a", 16, 32), ("c0b", 32, 32), ("c1a", 32, 64), ("c1b", 64, 64), ("c2a", 64, 128), ("c2b", 128, 128),
          ("c3a", 128, 128), ("c3b", 128, 128), ("d2a", 256, 128), ("d2b", 128, 64), ("d1a", 128, 64),
          ("d1b", 64, 32), ("d0a", 64, 32), ("d0b", 32, 32)]
HEAD_C = 32
# resolution level (0 = full, l = 1/2^l) at which each layer's name prefix runs
LEVEL = {"c0": 0, "c1": 1, "c2": 2, "c3": 3, "d2": 2, "d1": 1, "d0": 0}


class Params:
    """Master f32 weights, bf16 compute copies, gradients and Adam moments."""

    def __init__(self, device="cuda", seed=0):
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.device = torch.device(device)
        self.t = 0
        self.tensors = {}
        for name, cin, cout in LAYERS:
            std = math.sqrt(2.0 / (9 * cin))
            self._add(name + ".w", torch.randn(9 * cin * cout, generator=g) * std, bf16=True)
            self._add(name + ".b", torch.zeros(cout))
        self._add("head.w", torch.randn(HEAD_C, generator=g) * 0.01)
        self._add("head.b", torch.zeros(1))

    def _add(self, name, value, bf16=False):
        d = self.device
        p = value.to(torch.float32).to(d).contiguous()
        ent = {"p": p, "g": torch.zeros_like(p), "m": torch.zeros_like(p), "v": torch.zeros_like(p), "bf": None}
        if bf16:
            ent["bf"] = torch.empty(p.numel(), dtype=torch.bfloat16, device=d)
            ent["wk"] = torch.empty(p.numel(), dtype=torch.bfloat16, device=d)  # [tap][co][ci]
            ent["wf"] = torch.empty(p.numel(), dtype=torch.bfloat16, device=d)  # [8 - tap][ci][co]
            nn.cast_bf16(p, p.numel(), ent["bf"])
        self.tensors[name] = ent
        if bf16:
            self._refresh(name)

    def _refresh(self, name):
        """K-major and tap-flipped bf16 copies for the tensor-memory kernels."""
        cin, cout = next((ci, co) for n, ci, co in LAYERS if n + ".w" == name)
        e = self.tensors[name]
        nn.kmajor_weights(e["bf"], cin, cout, 0, e["wk"])
        nn.kmajor_weights(e["bf"], cin, cout, 1, e["wf"])

    def __getitem__(self, name):
        return self.tensors[name]

    def count(self):
        return sum(e["p"].numel() for e in self.tensors.values())

    def zero_grad(self):
        for e in self.tensors.values():
            nn.zero(e["g"], e["g"].numel() * 4)

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        for name, e in self.tensors.items():
            nn.adam(e["p"], e["g"], e["m"], e["v"], e["p"].numel(), lr, b1, b2, eps, self.t, e["bf"])
            if e["bf"] is not None:
                self._refresh(name)

    def state_dict(self):
        return {k: e["p"].detach().cpu().numpy() for k, e in self.tensors.items()}

    def load_state_dict(self, sd):
        for k, e in self.tensors.items():
            e["p"].copy_(torch.from_numpy(np.asarray(sd[k], np.float32)))
            if e["bf"] is not None:
                nn.cast_bf16(e["p"], e["p"].numel(), e["bf"])
                self._refresh(k)


class UNet:
    """Activations and gradient buffers for one input shape (B, H, W);
    H and W must be multiples of 8. `conv` picks the kernel of the forward
    and data-gradient convolutions: "tma" (default; persistent TMA-fed
    tcgen05 kernel), "tcgen05" (gathering tcgen05 kernel) or "warp_mma"
    (warp-level MMA). The weight gradient runs on the TMA-fed tcgen05 kernel
    unless "warp_mma" is chosen."""

    CONVS = ("tma", "tcgen05", "warp_mma")

    def __init__(self, params, B, H, W, inference_only=False, conv="tma", fuse_input=False):
        assert H % 8 == 0 and W % 8 == 0
        assert conv in self.CONVS, conv
        self.prm = params
        self.conv = conv
        # inference with the TMA kernel: pooling, upsampling + skip concat and
        # the head run inside the convolutions' epilogues, and (fuse_input)
        # the input packing inside a first convolution on the FP32 cores. That
        # one is off by default: the packing kernel plus the tensor-core layer
        # (16 x 16-pixel tiles, launched early) measured faster in the graph
        # at 512^2 (193 against 199 us for the whole forward).
        self.fused = inference_only and conv == "tma"
        self.fuse_input = self.fused and fuse_input
        self._iq = None
        self.status = torch.zeros(1, dtype=torch.int32, device=params.device)
        self.B, self.H, self.W = B, H, W
        d = params.device
        self.dims = [(H >> l, W >> l) for l in range(4)]
        self.P = [B * h * w for h, w in self.dims]
        bf, f32 = torch.bfloat16, torch.float32

        def act(level, c):
            return torch.empty(self.P[level] * c, dtype=bf, device=d)

        def grad(level, c):
            return torch.empty(self.P[level] * c, dtype=f32, device=d)

        self.a = {"x": act(0, CIN), "a0": act(0, 32), "e0": act(0, 32), "p0": act(1, 32), "a1": act(1, 64),
                  "e1": act(1, 64), "p1": act(2, 64), "a2": act(2, 128), "e2": act(2, 128), "p2": act(3, 128),
                  "a3": act(3, 128), "u3": act(3, 128), "cat2": act(2, 256),
                  "ad2": act(2, 128), "u2": act(2, 64), "cat1": act(1, 128), "ad1": act(1, 64),
                  "u1": act(1, 32), "cat0": act(0, 64), "ad0": act(0, 32), "u0": act(0, 32)}
        self.baseline = torch.empty(self.P[0], dtype=f32, device=d)
        self.pred = torch.empty(self.P[0], dtype=f32, device=d)
        if inference_only:
            return
        self.gpred = torch.empty(self.P[0], dtype=f32, device=d)
        self.loss = torch.zeros(1, dtype=f32, device=d)
        self.g = {"u0": grad(0, 32), "ad0": grad(0, 32), "cat0": grad(0, 64), "up1": grad(0, 32), "e0": grad(0, 32),
                  "a0": grad(0, 32), "u1": grad(1, 32), "ad1": grad(1, 64), "cat1": grad(1, 128),
                  "up2": grad(1, 64), "e1": grad(1, 64), "a1": grad(1, 64), "p0": grad(1, 32), "u2": grad(2, 64),
                  "ad2": grad(2, 128), "cat2": grad(2, 256), "up3": grad(2, 128), "e2": grad(2, 128),
                  "a2": grad(2, 128), "p1": grad(2, 64), "u3": grad(3, 128), "a3": grad(3, 128),
                  "p2": grad(3, 128)}
        self.gz = torch.empty(max(self.P[l] * c for l, c in [(0, 32), (1, 64), (2, 128), (3, 128)]), dtype=bf,
                              device=d)
        self.wt = torch.empty(max(9 * ci * co for _, ci, co in LAYERS), dtype=bf, device=d)

    # -- forward ------------------------------------------------------------
    def _conv(self, name, level, x, y):
        _, cin, cout = next(l for l in LAYERS if l[0] == name)
        h, w = self.dims[level]
        if self.conv != "warp_mma":
            fn = nn.conv3x3_fwd_tma if self.conv == "tma" else nn.conv3x3_fwd_tc
            fn(x, self.prm[name + ".w"]["wk"], self.prm[name + ".b"]["p"], self.B, h, w, cin, cout, 1, y, None,
               self.status)
        else:
            nn.conv3x3_fwd(x, self.prm[name + ".w"]["bf"], self.prm[name + ".b"]["p"], self.B, h, w, cin, cout, 1, y,
                           None)

    def capture(self, S=None, C=None):
        """Record input packing and the forward pass as one CUDA graph over
        this object's fixed buffers (inputs: self.S_in, self.C_in, int32
        [B*H*W]); replay() then runs the whole network as one launch on the
        current stream. With S and C given (int32 device tensors, or device
        addresses such as qld_iq_pointers' of a QLD context of the same
        frame size), the graph reads those in place instead. The first,
        uncaptured pass sets the kernels' launch attributes."""
        d = self.prm.device
        if S is None or C is None:
            self.S_in = torch.zeros(self.P[0], dtype=torch.int32, device=d)
            self.C_in = torch.zeros_like(self.S_in)
        else:
            self.S_in, self.C_in = S, C
        side = torch.cuda.Stream(d)
        side.wait_stream(torch.cuda.current_stream(d))
        with torch.cuda.stream(side):
            self.pack(self.S_in, self.C_in)
            self.forward()
        torch.cuda.current_stream(d).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.pack(self.S_in, self.C_in)
            self.forward()
        return self

    def replay(self):
        self.graph.replay()
        return self.pred

    def pack(self, S, C):
        """Network input and baseline from short-window sums (int32 [B*H*W]).
        With the fused input layer this only records S and C: the first
        convolution of forward() packs them itself."""
        if self.fuse_input:
            self._iq = (S, C)
            return
        nn.pack_input(S, C, self.P[0], IN_SCALE, self.a["x"], self.baseline)

    def _conv_epi(self, name, level, x, out=None, ldo=0, pool=None, up=None, ldu=0, head=False):
        _, cin, cout = next(l for l in LAYERS if l[0] == name)
        h, w = self.dims[level]
        hw = hb = base = pred = None
        if head:
            hw, hb, base, pred = self.prm["head.w"]["p"], self.prm["head.b"]["p"], self.baseline, self.pred
        # each layer may start its set-up while the previous one finishes (the
        # weights are constant during inference)
        nn.conv3x3_fwd_tma_epi(x, self.prm[name + ".w"]["wk"], self.prm[name + ".b"]["p"], self.B, h, w, cin, cout, 1,
                               out, ldo or cout, pool, up, ldu or cout, hw, hb, base, pred, self.status,
                               EARLY_LAUNCH)

    def _forward_fused(self):
        """The forward pass with pooling, upsample + skip concatenation and the
        head fused into the convolutions (bit-identical to the unfused pass):
        each encoder block's second convolution writes its activation into the
        skip half of the concat buffer and its 2x2 average into the next
        level's input; each decoder block's second convolution writes its 2x
        upsampling into the first half of the next concat buffer; the last
        one computes the prediction directly."""
        a = self.a
        if self.fuse_input:
            S, C = self._iq
            h, w = self.dims[0]
            nn.input_conv3x3(S, C, self.B, h, w, IN_SCALE, self.prm["c0a.w"]["bf"], CIN, 32, self.prm["c0a.b"]["p"],
                             1, a["a0"], 32, self.baseline)
        else:
            self._conv_epi("c0a", 0, a["x"], out=a["a0"])  # launched early, behind the packing
        self._conv_epi("c0b", 0, a["a0"], out=a["cat0"][32:], ldo=64, pool=a["p0"])
        self._conv("c1a", 1, a["p0"], a["a1"])
        self._conv_epi("c1b", 1, a["a1"], out=a["cat1"][64:], ldo=128, pool=a["p1"])
        self._conv("c2a", 2, a["p1"], a["a2"])
        self._conv_epi("c2b", 2, a["a2"], out=a["cat2"][128:], ldo=256, pool=a["p2"])
        self._conv("c3a", 3, a["p2"], a["a3"])
        self._conv_epi("c3b", 3, a["a3"], up=a["cat2"], ldu=256)
        self._conv("d2a", 2, a["cat2"], a["ad2"])
        self._conv_epi("d2b", 2, a["ad2"], up=a["cat1"], ldu=128)
        self._conv("d1a", 1, a["cat1"], a["ad1"])
        self._conv_epi("d1b", 1, a["ad1"], up=a["cat0"], ldu=64)
        self._conv("d0a", 0, a["cat0"], a["ad0"])
        self._conv_epi("d0b", 0, a["ad0"], head=True)
        return self.pred

    def forward(self):
        if self.fused:
            return self._forward_fused()
        a, B = self.a, self.B
        h, w = self.dims[0]
        self._conv("c0a", 0, a["x"], a["a0"])
        self._conv("c0b", 0, a["a0"], a["e0"])
        nn.avgpool2(a["e0"], B, h, w, 32, a["p0"])
        h, w = self.dims[1]
        self._conv("c1a", 1, a["p0"], a["a1"])
        self._conv("c1b", 1, a["a1"], a["e1"])
        nn.avgpool2(a["e1"], B, h, w, 64, a["p1"])
        h, w = self.dims[2]
        self._conv("c2a", 2, a["p1"], a["a2"])
        self._conv("c2b", 2, a["a2"], a["e2"])
        nn.avgpool2(a["e2"], B, h, w, 128, a["p2"])
        h, w = self.dims[3]
        self._conv("c3a", 3, a["p2"], a["a3"])
        self._conv("c3b", 3, a["a3"], a["u3"])
        nn.upsample_concat(a["u3"], 128, a["e2"], 128, B, h, w, a["cat2"])
        self._conv("d2a", 2, a["cat2"], a["ad2"])
        self._conv("d2b", 2, a["ad2"], a["u2"])
        h, w = self.dims[2]
        nn.upsample_concat(a["u2"], 64, a["e1"], 64, B, h, w, a["cat1"])
        self._conv("d1a", 1, a["cat1"], a["ad1"])
        self._conv("d1b", 1, a["ad1"], a["u1"])
        h, w = self.dims[1]
        nn.upsample_concat(a["u1"], 32, a["e0"], 32, B, h, w, a["cat0"])
        self._conv("d0a", 0, a["cat0"], a["ad0"])
        self._conv("d0b", 0, a["ad0"], a["u0"])
        nn.head(a["u0"], self.prm["head.w"]["p"], self.prm["head.b"]["p"], self.P[0], HEAD_C, self.pred)
        nn.add(self.pred, self.baseline, self.P[0])
        return self.pred

    # -- backward -----------------------------------------------------------
    def _conv_bwd(self, name, level, x, y, gy, gx):
        """ReLU mask, weight and bias gradients, and (if gx) the data gradient."""
        _, cin, cout = next(l for l in LAYERS if l[0] == name)
        h, w = self.dims[level]
        n = self.P[level] * cout
        gz = self.gz[:n]
        nn.relu_bwd_bias(gy, y, self.P[level], cout, gz, self.prm[name + ".b"]["g"])
        if self.conv == "warp_mma":
            nn.conv3x3_wgrad(x, gz, self.B, h, w, cin, cout, self.prm[name + ".w"]["g"])
        else:
            nn.conv3x3_wgrad_tma(x, gz, self.B, h, w, cin, cout, self.prm[name + ".w"]["g"], self.status)
        if gx is not None:
            if self.conv != "warp_mma":
                fn = nn.conv3x3_fwd_tma if self.conv == "tma" else nn.conv3x3_fwd_tc
                fn(gz, self.prm[name + ".w"]["wf"], None, self.B, h, w, cout, cin, 0, None, gx, self.status)
            else:
                nn.conv3x3_dgrad(gz, self.prm[name + ".w"]["bf"], self.B, h, w, cin, cout, self.wt, None, gx)

    def loss_and_grad(self, target):
        nn.zero(self.loss, 4)
        nn.mse(self.pred, target, self.P[0], self.gpred, self.loss)

    def backward(self):
        a, g, B = self.a, self.g, self.B
        nn.head_bwd(a["u0"], self.gpred, self.prm["head.w"]["p"], self.P[0], HEAD_C, g["u0"], self.prm["head.w"]["g"],
                    self.prm["head.b"]["g"])
        self._conv_bwd("d0b", 0, a["ad0"], a["u0"], g["u0"], g["ad0"])
        self._conv_bwd("d0a", 0, a["cat0"], a["ad0"], g["ad0"], g["cat0"])
        nn.split(g["cat0"], self.P[0], 32, 32, g["up1"], g["e0"], 0)
        h, w = self.dims[1]
        nn.upsample2_bwd(g["up1"], B, h, w, 32, g["u1"])
        self._conv_bwd("d1b", 1, a["ad1"], a["u1"], g["u1"], g["ad1"])
        self._conv_bwd("d1a", 1, a["cat1"], a["ad1"], g["ad1"], g["cat1"])
        nn.split(g["cat1"], self.P[1], 64, 64, g["up2"], g["e1"], 0)
        h, w = self.dims[2]
        nn.upsample2_bwd(g["up2"], B, h, w, 64, g["u2"])
        self._conv_bwd("d2b", 2, a["ad2"], a["u2"], g["u2"], g["ad2"])
        self._conv_bwd("d2a", 2, a["cat2"], a["ad2"], g["ad2"], g["cat2"])
        nn.split(g["cat2"], self.P[2], 128, 128, g["up3"], g["e2"], 0)
        h, w = self.dims[3]
        nn.upsample2_bwd(g["up3"], B, h, w, 128, g["u3"])
        self._conv_bwd("c3b", 3, a["a3"], a["u3"], g["u3"], g["a3"])
        self._conv_bwd("c3a", 3, a["p2"], a["a3"], g["a3"], g["p2"])
        h, w = self.dims[2]
        nn.avgpool2_bwd(g["p2"], B, h, w, 128, g["e2"], 1)
        self._conv_bwd("c2b", 2, a["a2"], a["e2"], g["e2"], g["a2"])
        self._conv_bwd("c2a", 2, a["p1"], a["a2"], g["a2"], g["p1"])
        h, w = self.dims[1]
        nn.avgpool2_bwd(g["p1"], B, h, w, 64, g["e1"], 1)
        self._conv_bwd("c1b", 1, a["a1"], a["e1"], g["e1"], g["a1"])
        self._conv_bwd("c1a", 1, a["p0"], a["a1"], g["a1"], g["p0"])
        h, w = self.dims[0]
        nn.avgpool2_bwd(g["p0"], B, h, w, 32, g["e0"], 1)
        self._conv_bwd("c0b", 0, a["a0"], a["e0"], g["e0"], g["a0"])
        self._conv_bwd("c0a", 0, a["x"], a["a0"], g["a0"], None)


# ---- training data: seeded scattering scenes processed by plain QLD -------

def random_scene_tables(rng, H, W, device, bg=2000.0, maxv=4095):
    """Per-pixel Q16 generator tables of a random multi-source fog scene:
    3-8 sources (squares or disks, 8-64 px), ballistic amplitude
    2000 exp(-OD) with OD uniform in [4, 8], diffuse glow bg (0.5 + 0.5
    blur/max) (Gaussian sigma 20 px), shot noise sd = sqrt(mean)."""
    yy = torch.arange(H, device=device, dtype=torch.float32)[:, None]
    xx = torch.arange(W, device=device, dtype=torch.float32)[None, :]
    mask = torch.zeros((H, W), device=device)
    for _ in range(int(rng.integers(3, 9))):
        size = float(rng.integers(8, 65))
        cy, cx = float(rng.uniform(0, H)), float(rng.uniform(0, W))
        if rng.random() < 0.5:
            m = ((yy - cy).abs() <= size / 2) & ((xx - cx).abs() <= size / 2)
        else:
            m = ((yy - cy) ** 2 + (xx - cx) ** 2) <= (size / 2) ** 2
        mask = torch.maximum(mask, m.float())
    from qldscene import blur_device

    blur = blur_device(mask, 20.0)  # the scene generator's own separable CUDA blur
    diffuse = bg * (0.5 + 0.5 * blur / blur.max().clamp_min(1e-12))
    od = float(rng.uniform(4.0, 8.0))
    amp = bg * math.exp(-od)
    mu0 = diffuse
    mu1 = diffuse + amp * mask
    q = 65536.0
    tables = [torch.round(v.flatten() * q).to(torch.int32).contiguous() for v in (mu0, mu1, mu0.sqrt(), mu1.sqrt())]
    return tables, int(rng.integers(0, 4)), od


class StackMaker:
    """Makes training stacks on the device: a scene's N_LONG frames from the
    seeded generator, pushed through plain QLD twice (windows N_SHORT and
    N_LONG); returns the short-window sums and the long-window amplitude."""

    def __init__(self, H, W, device="cuda", chunk=128):
        self.H, self.W = H, W
        self.npix = H * W
        self.device = torch.device(device)
        self.chunk = chunk
        self.frames = torch.empty((chunk, self.npix), dtype=torch.uint16, device=self.device)
        self.ctx_s = qld_create(H, W, N_SHORT, QLD_U16)
        self.ctx_l = qld_create(H, W, N_LONG, QLD_U16)

    def make(self, rng, seed):
        import qldscene

        tables, off, od = random_scene_tables(rng, self.H, self.W, self.device)
        key = (seed & 0xFFFFFFFF, 0x1EA2)
        qld_reset(self.ctx_s)
        qld_reset(self.ctx_l)
        for s0 in range(1, N_LONG + 1, self.chunk):
            qldscene.generate_from_tables(self.frames, 2, self.npix, s0, self.chunk, *tables, off, key, 4095)
            qld_push_frames(self.ctx_s, self.frames, self.chunk)
            qld_push_frames(self.ctx_l, self.frames, self.chunk)
        S = torch.empty(self.npix, dtype=torch.int32, device=self.device)
        C = torch.empty_like(S)
        R = torch.empty(self.npix, dtype=torch.float32, device=self.device)
        qld_get_iq(self.ctx_s, S, C)
        qld_image(self.ctx_l, R, None)
        qld_sync(self.ctx_l)
        return S, C, R, od

    def close(self):
        self.ctx_s.destroy()
        self.ctx_l.destroy()


def make_dataset(n, H=512, W=512, seed=0, device="cuda"):
    """n stacks: short-window sums (int32 [n, H*W]) and scaled long-window
    targets (f32 [n, H*W])."""
    rng = np.random.default_rng(seed)
    mk = StackMaker(H, W, device)
    S = torch.empty((n, H * W), dtype=torch.int32, device=device)
    C = torch.empty_like(S)
    T = torch.empty((n, H * W), dtype=torch.float32, device=device)
    ods = []
    for i in range(n):
        s, c, r, od = mk.make(rng, seed * 1000003 + i)
        S[i].copy_(s)
        C[i].copy_(c)
        T[i].copy_(r * TARGET_SCALE)
        ods.append(od)
    mk.close()
    return S, C, T, np.array(ods)


def crop_batch(S, C, T, idx, ys, xs, crop, H, W):
    """Gathers square crops (input marshalling) into contiguous buffers."""
    B = len(idx)
    Sb = torch.empty((B, crop, crop), dtype=torch.int32, device=S.device)
    Cb = torch.empty_like(Sb)
    Tb = torch.empty((B, crop, crop), dtype=torch.float32, device=S.device)
    for j, (i, y, x) in enumerate(zip(idx, ys, xs)):
        Sb[j] = S[i].view(H, W)[y:y + crop, x:x + crop]
        Cb[j] = C[i].view(H, W)[y:y + crop, x:x + crop]
        Tb[j] = T[i].view(H, W)[y:y + crop, x:x + crop]
    return Sb.reshape(-1), Cb.reshape(-1), Tb.reshape(-1)


def metrics(pred, target):
    """(relative L2 error, PSNR in dB with the target's peak) of numpy arrays."""
    pred = np.asarray(pred, np.float64)
    target = np.asarray(target, np.float64)
    mse = np.mean((pred - target) ** 2)
    rel = math.sqrt(np.sum((pred - target) ** 2) / max(np.sum(target ** 2), 1e-300))
    psnr = 10 * math.log10(max(target.max() ** 2, 1e-300) / max(mse, 1e-300))
    return rel, psnr


def evaluate(params, S, C, T, H, W, batch=2):
    """Network and baseline (32 R_32) metrics over full frames."""
    n = S.shape[0]
    if n < 1:
        raise ValueError("evaluate needs at least one stack")
    nets = {}
    preds, bases = [], []
    for i0 in range(0, n, batch):
        b = min(batch, n - i0)  # the last batch may be short
        if b not in nets:
            nets[b] = UNet(params, b, H, W, inference_only=True)
        net = nets[b]
        net.pack(S[i0:i0 + b].reshape(-1), C[i0:i0 + b].reshape(-1))
        net.forward()
        torch.cuda.synchronize()
        preds.append(net.pred.cpu().numpy().copy())
        bases.append(net.baseline.cpu().numpy().copy())
    t = T[:n].reshape(-1).cpu().numpy()
    p = np.concatenate(preds)
    b = np.concatenate(bases)
    return {"network": metrics(p, t), "baseline": metrics(b, t)}


def train(params, S, C, T, H, W, steps, batch=8, crop=256, lr=1e-3, seed=1, log_every=100, log=None):
    """Adam on random crops of the dataset; cosine learning-rate decay."""
    rng = np.random.default_rng(seed)
    net = UNet(params, batch, crop, crop)
    n = S.shape[0]
    hist = []
    for step in range(steps):
        idx = rng.integers(0, n, batch)
        ys = rng.integers(0, H - crop + 1, batch)
        xs = rng.integers(0, W - crop + 1, batch)
        Sb, Cb, Tb = crop_batch(S, C, T, idx, ys, xs, crop, H, W)
        net.pack(Sb, Cb)
        net.forward()
        net.loss_and_grad(Tb)
        params.zero_grad()
        net.backward()
        params.adam(lr * 0.5 * (1 + math.cos(math.pi * step / max(1, steps))))
        if (step + 1) % log_every == 0 or step == 0:
            loss = float(net.loss.item())
            hist.append((step + 1, loss))
            if log:
                log("step %d loss %.6g" % (step + 1, loss))
    return hist


WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "weights", "unet_n32.npz")


def save(params, path):
    np.savez_compressed(path, **{k.replace(".", "__"): v.astype(np.float32) for k, v in params.state_dict().items()})


def load(path, device="cuda"):
    p = Params(device)
    data = np.load(path)
    p.load_state_dict({k.replace("__", "."): data[k] for k in data.files})
    return p


def main(argv=None):
    """Trains the network on simulated stacks and reports metrics on
    held-out stacks as JSON lines:

        python -m paper_1511_03390_b300.learned --stacks 20000 --steps 20000 --out weights.npz
    """
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser()
    ap.add_argument("--stacks", type=int, default=256, help="training stacks (512x512, N_LONG frames each)")
    ap.add_argument("--eval-stacks", type=int, default=16)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--crop", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--init", default=None, help="weights to start from")
    ap.add_argument("--out", default=None)
    ap.add_argument("--forward", type=int, default=0, metavar="SIZE",
                    help="only time the inference forward of the committed weights on SIZE x SIZE inputs "
                         "(random short-window sums, the network as one CUDA graph) and exit")
    a = ap.parse_args(argv)
    if a.forward:
        dev = torch.device("cuda")
        prm = load(WEIGHTS, dev)
        net = UNet(prm, 1, a.forward, a.forward, inference_only=True).capture()
        g = torch.Generator(device=dev).manual_seed(a.seed)
        npix = a.forward * a.forward
        net.S_in.copy_(torch.randint(-3000, 3000, (npix,), dtype=torch.int32, device=dev, generator=g))
        net.C_in.copy_(torch.randint(-3000, 3000, (npix,), dtype=torch.int32, device=dev, generator=g))
        for _ in range(3):
            net.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            net.replay()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 20
        flops = 2.0 * npix * sum(9 * ci * co / 4 ** LEVEL[n[:2]] for n, ci, co in LAYERS)
        print(json.dumps({"event": "forward", "size": a.forward, "ms": ms, "tflops": flops / ms / 1e9,
                          "status": int(net.status.item())}), flush=True)
        return
    t0 = time.time()
    S, C, T, ods = make_dataset(a.stacks, a.size, a.size, seed=a.seed)
    Se, Ce, Te, odse = make_dataset(a.eval_stacks, a.size, a.size, seed=a.seed + 99991)
    torch.cuda.synchronize()
    t1 = time.time()
    print(json.dumps({"event": "data", "stacks": a.stacks, "eval_stacks": a.eval_stacks, "seconds": t1 - t0}),
          flush=True)
    prm = load(a.init) if a.init else Params(seed=a.seed)
    hist = train(prm, S, C, T, a.size, a.size, a.steps, batch=a.batch, crop=a.crop, lr=a.lr, seed=a.seed + 1,
                 log_every=max(1, a.steps // 20), log=lambda m: print(json.dumps({"event": "train", "msg": m}),
                                                                           flush=True))
    torch.cuda.synchronize()
    t2 = time.time()
    ev = evaluate(prm, Se, Ce, Te, a.size, a.size)
    print(json.dumps({"event": "done", "params": prm.count(), "train_seconds": t2 - t1,
                      "ms_per_step": (t2 - t1) / max(1, a.steps) * 1e3, "loss_first": hist[0][1],
                      "loss_last": hist[-1][1], "eval_network_rel_l2": ev["network"][0],
                      "eval_network_psnr": ev["network"][1], "eval_baseline_rel_l2": ev["baseline"][0],
                      "eval_baseline_psnr": ev["baseline"][1], "od_range": [float(ods.min()), float(ods.max())]}),
          flush=True)
    if a.out:
        save(prm, a.out)


if __name__ == "__main__":
    main()
