"""The FP64 U-Net reference's backward pass against central finite
differences of its own forward pass (no rounding): pins the composition of
skip connections, pooling, upsampling and head that the GPU check relies on."""
import numpy as np

from unet_reference import LAYERS, RefUNet


def random_params(rng):
    p = {}
    for name, cin, cout in LAYERS:
        p[name + ".w"] = rng.standard_normal(9 * cin * cout) * np.sqrt(2.0 / (9 * cin))
        p[name + ".b"] = rng.standard_normal(cout) * 0.1
    p["head.w"] = rng.standard_normal(32) * 0.3
    p["head.b"] = np.array([0.2])
    return p


def test_reference_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = random_params(rng)
    x = rng.standard_normal((1, 8, 8, 16))
    base = rng.standard_normal((1, 8, 8))
    target = rng.standard_normal((1, 8, 8))
    net = RefUNet(p, round_bf16=False)
    loss, gpred = net.loss(net.forward(x, base), target)
    grads = net.backward(gpred)
    for name, idx in [("c0a.w", 5), ("c0b.b", 3), ("c2a.w", 1000), ("c3b.w", 77), ("d2a.w", 4321), ("d1a.b", 10),
                      ("d0b.w", 123), ("head.w", 7), ("head.b", 0)]:
        eps = 1e-5
        orig = p[name][idx]
        p[name][idx] = orig + eps
        lp, _ = net.loss(net.forward(x, base), target)
        p[name][idx] = orig - eps
        lm, _ = net.loss(net.forward(x, base), target)
        p[name][idx] = orig
        fd = (lp - lm) / (2 * eps)
        an = grads[name][idx]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-8, (name, idx, fd, an)
