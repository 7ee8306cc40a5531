"""The seeded input generator: Philox known-answer vectors (Salmon et al.,
SC'11, Random123 distribution), scene statistics, and the GPU twin producing
exactly the numpy frames."""
import numpy as np
import pytest

from qldscene import DeviceScene, Scene, scene_fog, scene_plain
from qldscene.philox import philox4x32


def test_philox_known_answers():
    f = 0xFFFFFFFF
    cases = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((f, f, f, f), (f, f), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in cases:
        got = philox4x32(*ctr, *key)
        assert tuple(int(g) for g in got) == want


def test_noise_statistics_and_modulation():
    sc = Scene(64, 64, 2, seed=7, bg=1000.0, amp=0.0, noise="gauss", sigma=30.0, blur_sigma=0)
    x = sc.frames(1, 64).astype(np.float64)
    # blur_sigma 0 with no modulation: mean bg*(0.5+0.5*mask), noise sd 30
    resid = x - x.mean(axis=0, keepdims=True)
    assert abs(resid.std() / 30.0 - 1) < 0.02
    assert abs(np.mean((resid / 30.0) ** 4) - 2.9) < 0.15  # Irwin-Hall(12) kurtosis 3 - 1.2/12
    sc2 = scene_plain()
    s = np.arange(1, 9)
    m = sc2.modulation(s)
    assert m.sum() == 4 and all(m[i] == m[i + 4] for i in range(4))
    assert ((m[:-1] == 1) & (m[1:] == 1)).sum() in (1, 2)  # two consecutive high residues


def test_fog_scene_levels():
    sc = scene_fog(4, H=128, W=128)
    x = sc.frames(1, 32).astype(np.float64)
    assert 900 < x.mean() < 2100 and x.max() <= 4095
    assert abs(sc.amp - 2000 * np.exp(-4)) < 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("make", [lambda: scene_plain(H=96, W=200), lambda: scene_fog(6, H=64, W=72),
                                  lambda: scene_fog(4, H=33, W=17, pixfmt=2, maxv=65535)])
def test_gpu_generator_matches_numpy(make):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = make()
    ds = DeviceScene(sc)
    for s0, n in [(1, 9), (4093, 5), ((1 << 32) - 2, 4)]:
        got = ds.frames(s0, n).cpu().numpy().reshape(n, -1)
        assert np.array_equal(got, sc.frames(s0, n))


@pytest.mark.gpu
def test_device_blur_matches_the_numpy_blur():
    """qldscene.blur_device (the learned simulator's blur) against the host
    scene generator's Gaussian blur of the same mask."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from qldscene import blur_device
    from qldscene.scene import _gauss_blur

    rng = np.random.default_rng(3)
    mask = (rng.random((96, 130)) < 0.1).astype(np.float64)
    want = _gauss_blur(mask, 20.0)
    got = blur_device(torch.from_numpy(mask.astype(np.float32)).cuda(), 20.0).cpu().numpy()
    assert np.allclose(got, want, rtol=1e-4, atol=1e-6 * want.max())
