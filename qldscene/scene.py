"""Seeded synthetic scattered-light scenes (host side, numpy).

A scene is a per-pixel description of a camera looking through a scattering
medium at sources modulated by a 0/1 square wave at a quarter of the frame
rate. It holds no QLD arithmetic: it only makes frames.

Model (per pixel p and absolute 1-based frame index s):
  * M(p): binary ballistic mask, one filled square and one filled disk whose
    side / diameter is a quarter of the shorter image side, at seeded
    positions.
  * D(p) = bg * (0.5 + 0.5 * B(p) / max B), B = Gaussian blur (sigma 20 px)
    of M: the diffuse glow around the sources.
  * m_s = 1 when (s - phase_offset) mod 4 is 0 or 1, else 0: the source
    modulation, four frames per period, with a seeded phase offset 0..3.
  * mean mu(p, s) = D(p) + A * M(p) * m_s, with A the ballistic amplitude
    in counts (A = 2000 * exp(-OD) for the fog scenes).
  * noise: Gaussian with a fixed sigma, or shot noise (sd = sqrt(mu)) in the
    normal limit of the Poisson law (mu >= 1000 counts here, where the two
    differ by a skew below 0.03).
  * x(p, s) = clip(floor(mu + sd * Z + 1/2), 0, maxv), Z from twelve Philox
    uniforms (Irwin-Hall sum minus 6: mean 0, variance 1).

Everything after the per-pixel tables (mu0, mu1, sd0, sd1 in Q16 fixed
point) is integer arithmetic, so this numpy code and the CUDA generator
(csrc/qldscene.cu) produce identical frames for the same scene.
"""
import math

import numpy as np

from .philox import philox4x32

Q = 16
ONE = 1 << Q
KEY_HI_TAG = 0x51ED


class Scene:
    """Per-pixel generator tables for one seeded scene."""

    def __init__(self, H, W, pixfmt, seed, bg, amp, noise="gauss", sigma=5.0, maxv=None,
                 blur_sigma=20.0, key_hi=0):
        self.H, self.W = int(H), int(W)
        self.npix = self.H * self.W
        self.pixfmt = int(pixfmt)
        if self.pixfmt not in (1, 2):
            raise ValueError("pixfmt must be 1 (uint8) or 2 (uint16)")
        self.dtype = np.uint8 if self.pixfmt == 1 else np.uint16
        self.maxv = int(maxv if maxv is not None else (255 if self.pixfmt == 1 else 65535))
        self.seed = int(seed)
        self.key = (self.seed & 0xFFFFFFFF, (KEY_HI_TAG ^ (int(key_hi) << 16)) & 0xFFFFFFFF)
        rng = np.random.default_rng(self.seed)
        self.mask = _mask(self.H, self.W, rng)
        self.phase_offset = int(rng.integers(0, 4))
        blur = _gauss_blur(self.mask.astype(np.float64), blur_sigma)
        peak = blur.max()
        self.diffuse = bg * (0.5 + 0.5 * (blur / peak if peak > 0 else blur))
        self.amp = float(amp)
        mu0 = self.diffuse
        mu1 = self.diffuse + self.amp * self.mask
        if noise == "gauss":
            sd0 = np.full_like(mu0, float(sigma))
            sd1 = np.full_like(mu1, float(sigma))
        elif noise == "shot":
            sd0 = np.sqrt(mu0)
            sd1 = np.sqrt(mu1)
        else:
            raise ValueError("noise must be 'gauss' or 'shot'")
        self.noise = noise
        self.mu0 = np.rint(mu0.ravel() * ONE).astype(np.int32)
        self.mu1 = np.rint(mu1.ravel() * ONE).astype(np.int32)
        self.sd0 = np.rint(sd0.ravel() * ONE).astype(np.int32)
        self.sd1 = np.rint(sd1.ravel() * ONE).astype(np.int32)

    def modulation(self, s):
        """m_s in {0, 1} for absolute frame indices s (array)."""
        s = np.asarray(s, np.int64)
        return (((s - self.phase_offset) % 4) < 2).astype(np.int64)

    def frames(self, s_first, count, pix=None):
        """Frames s_first .. s_first+count-1 as a (count, npix) array, or
        (count, len(pix)) for the pixel indices pix."""
        pix = np.arange(self.npix, dtype=np.int64) if pix is None else np.asarray(pix, np.int64)
        out = np.empty((int(count), pix.size), self.dtype)
        step = max(1, (1 << 22) // max(1, pix.size))
        for i0 in range(0, int(count), step):
            n = min(step, int(count) - i0)
            s = np.arange(int(s_first) + i0, int(s_first) + i0 + n, dtype=np.int64)
            P, Sg = np.meshgrid(pix, s)
            m = self.modulation(Sg) == 1
            mu = np.where(m, self.mu1[P], self.mu0[P]).astype(np.int64)
            sd = np.where(m, self.sd1[P], self.sd0[P]).astype(np.int64)
            z = _irwin_hall_q16(P, Sg, self.key)
            val = mu + ((sd * z) >> Q) + (ONE >> 1)
            out[i0:i0 + n] = np.clip(val >> Q, 0, self.maxv)
        return out

    def frames_hw(self, s_first, count):
        return self.frames(s_first, count).reshape(count, self.H, self.W)


def _irwin_hall_q16(pix, s, key):
    """Sum of twelve Philox uniforms minus 6, in Q16 (floor)."""
    pix = np.asarray(pix, np.uint64)
    s = np.asarray(s, np.uint64)
    tot = np.zeros(np.broadcast(pix, s).shape, np.uint64)
    for j in range(3):
        words = philox4x32(pix, s & np.uint64(0xFFFFFFFF), j, s >> np.uint64(32), key[0], key[1])
        for w in words:
            tot += w.astype(np.uint64)
    return (tot.astype(np.int64) - 6 * (1 << 32)) >> Q


def _mask(H, W, rng):
    side = max(1, min(H, W) // 4)
    m = np.zeros((H, W), np.uint8)
    # square
    y0 = int(rng.integers(0, max(1, H - side + 1)))
    x0 = int(rng.integers(0, max(1, W - side + 1)))
    m[y0:y0 + side, x0:x0 + side] = 1
    # disk of diameter side
    r = side / 2.0
    cy = float(rng.integers(0, max(1, H - side + 1))) + r
    cx = float(rng.integers(0, max(1, W - side + 1))) + r
    yy, xx = np.mgrid[0:H, 0:W]
    m[((yy + 0.5 - cy) ** 2 + (xx + 0.5 - cx) ** 2) <= r * r] = 1
    return m


def _gauss_blur(img, sigma):
    """Separable Gaussian blur, zero padding, kernel truncated at 4 sigma."""
    if sigma <= 0:
        return img.copy()
    rad = int(math.ceil(4 * sigma))
    t = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    out = _conv_rows(img, k)
    out = _conv_rows(out.T, k).T
    return out


def _conv_rows(img, k):
    """Convolve every row with k ('same' size, zero padding) via FFT."""
    n = img.shape[1]
    L = n + len(k) - 1
    nfft = 1 << (L - 1).bit_length()
    F = np.fft.rfft(img, nfft, axis=1) * np.fft.rfft(k, nfft)[None, :]
    full = np.fft.irfft(F, nfft, axis=1)[:, :L]
    off = (len(k) - 1) // 2
    return full[:, off:off + n]


# ---- the scenes of the benchmark configurations -----------------------------

def scene_plain(seed=1001, H=128, W=128):
    """128x128 uint8: mask amplitude 2 counts on a diffuse background of 100
    counts (blur sigma 20 px), Gaussian noise sigma 5, clipped to [0, 255]."""
    return Scene(H, W, 1, seed, bg=100.0, amp=2.0, noise="gauss", sigma=5.0, maxv=255)


def scene_fog(od, seed=1002, H=1024, W=1024, pixfmt=2, maxv=4095):
    """12-bit frames in uint16: ballistic fraction exp(-OD) of a 2000-count
    level over a 2000-count diffuse background, shot noise, clipped to 4095."""
    return Scene(H, W, pixfmt, seed, bg=2000.0, amp=2000.0 * math.exp(-float(od)), noise="shot",
                 maxv=maxv, key_hi=int(round(float(od) * 16)))
