"""FP64 CPU reference of the learned path's U-Net (test infrastructure).

Built from the oracle's 3x3 convolution forward/backward and numpy for the
pooling, upsampling, concatenation, 1x1 head and loss; optionally rounds to
bf16 wherever the GPU stores bf16 (activations, the ReLU-masked gradients fed
to the tensor-core GEMMs, weights), so the GPU can be compared layer for layer.
"""
import numpy as np

import oracle

LAYERS = [("c0a", 16, 32), ("c0b", 32, 32), ("c1a", 32, 64), ("c1b", 64, 64), ("c2a", 64, 128), ("c2b", 128, 128),
          ("c3a", 128, 128), ("c3b", 128, 128), ("d2a", 256, 128), ("d2b", 128, 64), ("d1a", 128, 64),
          ("d1b", 64, 32), ("d0a", 64, 32), ("d0b", 32, 32)]


def bf16r(x):
    """Round to the nearest bf16 (ties to even), as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(g):
    return 0.25 * np.repeat(np.repeat(g, 2, 1), 2, 2)


def up(x):
    return np.repeat(np.repeat(x, 2, 1), 2, 2)


def up_bwd(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


class RefUNet:
    def __init__(self, params, round_bf16=True):
        """params: dict name -> float64 arrays (w as [9*Cin*Cout] flat)."""
        self.p = params
        self.r = bf16r if round_bf16 else (lambda v: np.asarray(v, np.float64))

    def w(self, name):
        _, cin, cout = next(l for l in LAYERS if l[0] == name)
        return self.r(self.p[name + ".w"]).reshape(3, 3, cin, cout)

    def conv(self, name, x):
        return self.r(np.maximum(oracle.conv3x3(x, self.w(name), self.p[name + ".b"]), 0.0))

    def forward(self, x, baseline):
        r = self.r
        c = {"x": x}
        c["a0"] = self.conv("c0a", x)
        c["e0"] = self.conv("c0b", c["a0"])
        c["p0"] = r(pool(c["e0"]))
        c["a1"] = self.conv("c1a", c["p0"])
        c["e1"] = self.conv("c1b", c["a1"])
        c["p1"] = r(pool(c["e1"]))
        c["a2"] = self.conv("c2a", c["p1"])
        c["e2"] = self.conv("c2b", c["a2"])
        c["p2"] = r(pool(c["e2"]))
        c["a3"] = self.conv("c3a", c["p2"])
        c["u3"] = self.conv("c3b", c["a3"])
        c["cat2"] = np.concatenate([up(c["u3"]), c["e2"]], axis=3)
        c["ad2"] = self.conv("d2a", c["cat2"])
        c["u2"] = self.conv("d2b", c["ad2"])
        c["cat1"] = np.concatenate([up(c["u2"]), c["e1"]], axis=3)
        c["ad1"] = self.conv("d1a", c["cat1"])
        c["u1"] = self.conv("d1b", c["ad1"])
        c["cat0"] = np.concatenate([up(c["u1"]), c["e0"]], axis=3)
        c["ad0"] = self.conv("d0a", c["cat0"])
        c["u0"] = self.conv("d0b", c["ad0"])
        pred = c["u0"] @ self.p["head.w"] + self.p["head.b"][0] + baseline
        self.c = c
        return pred

    def loss(self, pred, target):
        d = pred - target
        return np.mean(d * d), 2 * d / d.size

    def backward(self, gpred):
        """Gradients of every parameter for dloss/dpred = gpred."""
        c, r = self.c, self.r
        grads = {}
        grads["head.w"] = np.einsum("bhwc,bhw->c", c["u0"], gpred)
        grads["head.b"] = np.array([gpred.sum()])
        gu0 = gpred[..., None] * self.p["head.w"]

        def conv_bwd(name, x, y, gy, need_dx=True):
            gz = r(np.where(y > 0, gy, 0.0))
            dx, dw, db = oracle.conv3x3_backward(x, self.w(name), gz)
            grads[name + ".w"] = dw.reshape(-1)
            grads[name + ".b"] = db
            return dx if need_dx else None

        g = conv_bwd("d0b", c["ad0"], c["u0"], gu0)
        g = conv_bwd("d0a", c["cat0"], c["ad0"], g)
        gup1, ge0 = g[..., :32], g[..., 32:]
        g = conv_bwd("d1b", c["ad1"], c["u1"], up_bwd(gup1))
        g = conv_bwd("d1a", c["cat1"], c["ad1"], g)
        gup2, ge1 = g[..., :64], g[..., 64:]
        g = conv_bwd("d2b", c["ad2"], c["u2"], up_bwd(gup2))
        g = conv_bwd("d2a", c["cat2"], c["ad2"], g)
        gup3, ge2 = g[..., :128], g[..., 128:]
        g = conv_bwd("c3b", c["a3"], c["u3"], up_bwd(gup3))
        g = conv_bwd("c3a", c["p2"], c["a3"], g)
        g = conv_bwd("c2b", c["a2"], c["e2"], ge2 + pool_bwd(g))
        g = conv_bwd("c2a", c["p1"], c["a2"], g)
        g = conv_bwd("c1b", c["a1"], c["e1"], ge1 + pool_bwd(g))
        g = conv_bwd("c1a", c["p0"], c["a1"], g)
        g = conv_bwd("c0b", c["a0"], c["e0"], ge0 + pool_bwd(g))
        conv_bwd("c0a", c["x"], c["a0"], g, need_dx=False)
        return grads
