"""Shared helpers of the GPU parity tests: drive the C ABI through the Python
binding, and compare its outputs with the CPU oracle under the stated
tolerances.

Tolerances (the integer sums are exact; the floating-point ones follow from
float32 arithmetic against FP64):
  * S, C: bit-exact.
  * amplitude: |R_gpu - R| <= 1e-6 R, and exactly 0 where S = C = 0.
  * phase: wrap-aware |phi_gpu - phi| <= 2e-6 rad where R > 0, exactly 0
    where S = C = 0. (float32 inputs to atan2 carry a relative error of
    2^-24 and atan2f a few ulp of pi, about 7e-7 rad in all.)
  * DFT bin power P = |X_k|^2: |P_gpu - P| <= 1e-4 P + 2 e sqrt(P) + e^2 with
    e = 1e-6 * sum_s x_s, i.e. |X_k| within 5e-5 relative plus an absolute
    floor of 1e-6 of the pixel's summed counts for near-empty bins.
"""
import numpy as np
import torch

import oracle
import paper_1511_03390_b300 as q

AMP_RTOL = 1e-6
PHASE_ATOL = 2e-6
POW_RTOL = 1e-4
POW_FLOOR = 1e-6


def dev_bytes(x_np, offset=0):
    """Copies a numpy frame array to a device byte buffer at byte `offset`;
    returns (buffer, address)."""
    raw = np.ascontiguousarray(x_np).view(np.uint8).ravel()
    buf = torch.zeros(raw.size + offset + 16, dtype=torch.uint8, device="cuda")
    buf[offset:offset + raw.size].copy_(torch.from_numpy(raw))
    return buf, buf.data_ptr() + offset


def get_iq(ctx):
    S = torch.empty(ctx.npix, dtype=torch.int32, device="cuda")
    C = torch.empty(ctx.npix, dtype=torch.int32, device="cuda")
    q.qld_get_iq(ctx, S, C)
    q.qld_sync(ctx)
    return S.cpu().numpy(), C.cpu().numpy()


def get_image(ctx):
    amp = torch.empty(ctx.npix, dtype=torch.float32, device="cuda")
    ph = torch.empty(ctx.npix, dtype=torch.float32, device="cuda")
    q.qld_image(ctx, amp, ph)
    q.qld_sync(ctx)
    return amp.cpu().numpy(), ph.cpu().numpy()


def get_bin(ctx, k):
    out = torch.empty(ctx.npix, dtype=torch.float32, device="cuda")
    q.qld_fft_bin(ctx, k, out)
    q.qld_sync(ctx)
    return out.cpu().numpy()


def check_sums(S_g, C_g, S_r, C_r, what=""):
    assert np.abs(S_r).max(initial=0) < 2 ** 31 and np.abs(C_r).max(initial=0) < 2 ** 31
    bad = np.flatnonzero((S_g != S_r) | (C_g != C_r))
    assert bad.size == 0, "%s: %d pixels differ, first %d: S %d vs %d, C %d vs %d" % (
        what, bad.size, bad[0], S_g[bad[0]], S_r[bad[0]], C_g[bad[0]], C_r[bad[0]])


def check_amp_phase(amp_g, ph_g, R, ph, what=""):
    amp_g = amp_g.astype(np.float64)
    ph_g = ph_g.astype(np.float64)
    err = np.abs(amp_g - R)
    ok = err <= AMP_RTOL * R
    assert ok.all(), "%s amplitude: %d bad, worst rel %g" % (what, (~ok).sum(), (err / np.maximum(R, 1e-300)).max())
    zero = R == 0
    assert (amp_g[zero] == 0).all() and (ph_g[zero] == 0).all(), what + ": S = C = 0 must give exact zeros"
    d = np.abs(np.angle(np.exp(1j * (ph_g - ph))))
    okp = (d <= PHASE_ATOL) | zero
    assert okp.all(), "%s phase: %d bad, worst %g rad" % (what, (~okp).sum(), d[~zero].max())
    # float32 atan2 returns values in [-fl(pi), fl(pi)], fl(pi) = 3.14159274 > pi
    pi32 = float(np.float32(np.pi))
    assert (ph_g <= pi32).all() and (ph_g >= -pi32).all()


def check_power(p_g, p_r, sumx, what=""):
    p_g = p_g.astype(np.float64)
    e = POW_FLOOR * sumx.astype(np.float64)
    tol = POW_RTOL * p_r + 2 * e * np.sqrt(p_r) + e * e
    err = np.abs(p_g - p_r)
    ok = err <= tol
    assert ok.all(), "%s DFT power: %d bad of %d, worst err/tol %g" % (what, (~ok).sum(), ok.size,
                                                                       (err / np.maximum(tol, 1e-300)).max())


def check_lockin(amp_g, ph_g, R, ph, sumx, what=""):
    """General-frequency lock-in against the FP64 oracle: the DFT-bin
    tolerance on the amplitude (|X| within 5e-5 relative plus a floor of
    1e-6 of the pixel's summed counts), and the phase where the amplitude
    clears that floor, within the angle the same error subtends."""
    amp_g = amp_g.astype(np.float64)
    e = POW_FLOOR * sumx.astype(np.float64)
    tol = 0.5 * POW_RTOL * R + e
    err = np.abs(amp_g - R)
    ok = err <= tol
    assert ok.all(), "%s lock-in amplitude: %d bad of %d, worst err/tol %g" % (what, (~ok).sum(), ok.size,
                                                                               (err / tol).max())
    if ph_g is not None:
        sel = R > 100 * tol
        d = np.abs(np.angle(np.exp(1j * (ph_g.astype(np.float64) - ph))))
        lim = 2 * tol / np.maximum(R, 1e-300) + 1e-6
        okp = (d <= lim) | ~sel
        assert okp.all(), "%s lock-in phase: %d bad" % (what, (~okp).sum())


def pack12(x):
    """Packs 12-bit values (uint16 array, last axis even) two per three bytes,
    least significant bits first (GenICam Mono12p)."""
    x = np.asarray(x, np.uint16)
    assert x.max(initial=0) <= 4095 and x.shape[-1] % 2 == 0
    a = x[..., 0::2].astype(np.uint16)
    b = x[..., 1::2].astype(np.uint16)
    out = np.empty(x.shape[:-1] + (a.shape[-1], 3), np.uint8)
    out[..., 0] = a & 0xFF
    out[..., 1] = (a >> 8) | ((b & 0xF) << 4)
    out[..., 2] = b >> 4
    return out.reshape(x.shape[:-1] + (x.shape[-1] // 2 * 3,))


class Stream:
    """A context plus a host record of every frame pushed, checked against the
    oracle recomputing each window from scratch. For the packed 12-bit format
    the record holds the unpacked values and the pushes send packed bytes."""

    def __init__(self, H, W, N, fmt):
        self.ctx = q.qld_create(H, W, N, fmt)
        self.H, self.W, self.N, self.fmt = H, W, N, fmt
        self.dtype = np.uint8 if fmt == 1 else np.uint16
        self.frames = np.zeros((0, H * W), self.dtype)

    def push(self, x, offset=0, fused=False):
        x = np.asarray(x, self.dtype).reshape(-1, self.H * self.W)
        buf, addr = dev_bytes(pack12(x) if self.fmt == 3 else x, offset)
        if fused:
            amp = torch.empty(self.H * self.W, dtype=torch.float32, device="cuda")
            ph = torch.empty_like(amp)
            q.qld_push_image(self.ctx, addr, x.shape[0], None, amp, ph)
        else:
            q.qld_push_frames(self.ctx, addr, x.shape[0])
        q.qld_sync(self.ctx)
        del buf
        self.frames = np.concatenate([self.frames, x], axis=0)
        if fused:
            return amp.cpu().numpy(), ph.cpu().numpy()
        return None

    def window(self):
        T = self.frames.shape[0]
        n = min(T, self.N)
        return self.frames[T - n:], T - n + 1

    def check(self, bins=()):
        win, s0 = self.window()
        assert q.qld_frames_pushed(self.ctx) == self.frames.shape[0]
        S_g, C_g = get_iq(self.ctx)
        if win.shape[0] == 0:
            assert not S_g.any() and not C_g.any()
            return
        S_r, C_r = oracle.quadrature_sums(win, s0=s0)
        check_sums(S_g, C_g, S_r, C_r, "T=%d" % self.frames.shape[0])
        if win.shape[0] == self.N:
            amp, ph = get_image(self.ctx)
            R, phr = oracle.amplitude_phase(S_r, C_r)
            check_amp_phase(amp, ph, R, phr)
            sumx = win.astype(np.int64).sum(axis=0)
            for k in bins:
                p_g = get_bin(self.ctx, k)
                p_r = oracle.dft_bin(win, k, s0=s0)[2]
                check_power(p_g, p_r, sumx, "k=%d" % k)
