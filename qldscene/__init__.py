"""Seeded synthetic scene generator for QLD tests and benchmarks.

``scene.py`` builds per-pixel tables on the host and evaluates frames with
numpy; ``csrc/qldscene.cu`` is a GPU twin producing identical frames for
large workloads. This module contains no QLD arithmetic and is shared by the
tests (as the source of inputs for both the oracle and the CUDA library) and
by bench.py.
"""
import ctypes
import os
import subprocess

from .scene import Scene, scene_fog, scene_plain  # noqa: F401

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "qldscene.cu")
LIB = os.path.join(HERE, "libqldscene.so")

_lib = None


def build(force=False):
    """Compile the GPU generator for sm_103a into libqldscene.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC", "-shared", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        ll = ctypes.c_longlong
        p = ctypes.c_void_p
        lib.qs_generate.argtypes = [p, ctypes.c_int, ll, ll, ll, ctypes.c_int, p, p, p, p, ctypes.c_int,
                                    ctypes.c_uint, ctypes.c_uint, ctypes.c_int, p]
        lib.qs_generate.restype = ctypes.c_int
        lib.qs_blur.argtypes = [p, p, p, ctypes.c_int, ctypes.c_int, p, ctypes.c_int, p]
        lib.qs_blur.restype = ctypes.c_int
        _lib = lib
    return _lib


def generate_from_tables(out, pixfmt, npix, s_first, count, mu0, mu1, sd0, sd1, phase_offset, key, maxv, stream=None):
    """Frames s_first .. s_first+count-1 from per-pixel Q16 tables already on
    the device (int32 tensors of npix values) into the contiguous device
    tensor `out` (count * npix elements of the pixel format)."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream()
    rc = _load().qs_generate(ctypes.c_void_p(out.data_ptr()), int(pixfmt), int(npix), int(npix), int(s_first),
                             int(count), ctypes.c_void_p(mu0.data_ptr()), ctypes.c_void_p(mu1.data_ptr()),
                             ctypes.c_void_p(sd0.data_ptr()), ctypes.c_void_p(sd1.data_ptr()), int(phase_offset),
                             int(key[0]), int(key[1]), int(maxv), ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise RuntimeError("qs_generate failed with code %d" % rc)
    return out


def blur_device(img, sigma, stream=None):
    """Gaussian blur (std `sigma` pixels, truncated at 4 sigma, zero
    padding) of a contiguous float32 H x W CUDA tensor, by this package's own
    separable kernel; returns a new tensor."""
    import torch

    import math

    H, W = img.shape
    r = int(math.ceil(4 * sigma))
    t = torch.arange(-r, r + 1, device=img.device, dtype=torch.float64)
    k = torch.exp(-0.5 * (t / sigma) ** 2)
    taps = (k / k.sum()).to(torch.float32).contiguous()
    src = img.contiguous().to(torch.float32)
    tmp = torch.empty_like(src)
    out = torch.empty_like(src)
    st = stream if stream is not None else torch.cuda.current_stream(img.device)
    rc = _load().qs_blur(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(tmp.data_ptr()),
                         ctypes.c_void_p(out.data_ptr()), int(H), int(W), ctypes.c_void_p(taps.data_ptr()), r,
                         ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise RuntimeError("qs_blur failed with code %d" % rc)
    return out


class DeviceScene:
    """A Scene's tables resident on a CUDA device, generating frames there."""

    def __init__(self, scene, device="cuda"):
        import torch

        self.scene = scene
        self.device = torch.device(device)
        self.mu0 = torch.from_numpy(scene.mu0).to(self.device)
        self.mu1 = torch.from_numpy(scene.mu1).to(self.device)
        self.sd0 = torch.from_numpy(scene.sd0).to(self.device)
        self.sd1 = torch.from_numpy(scene.sd1).to(self.device)

    def generate_into(self, out, s_first, count, stream=None):
        """Writes frames s_first .. s_first+count-1 into the contiguous device
        tensor out of shape (count, H, W) (or (count, npix))."""
        import torch

        sc = self.scene
        dt = torch.uint8 if sc.pixfmt == 1 else torch.uint16
        if out.dtype != dt or not out.is_contiguous() or out.numel() != count * sc.npix:
            raise ValueError("output tensor must be contiguous %s with %d elements" % (dt, count * sc.npix))
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        rc = _load().qs_generate(ctypes.c_void_p(out.data_ptr()), sc.pixfmt, sc.npix, sc.npix, int(s_first),
                                 int(count), ctypes.c_void_p(self.mu0.data_ptr()),
                                 ctypes.c_void_p(self.mu1.data_ptr()), ctypes.c_void_p(self.sd0.data_ptr()),
                                 ctypes.c_void_p(self.sd1.data_ptr()), sc.phase_offset, sc.key[0], sc.key[1],
                                 sc.maxv, ctypes.c_void_p(st.cuda_stream))
        if rc != 0:
            raise RuntimeError("qs_generate failed with code %d" % rc)
        return out

    def frames(self, s_first, count):
        import torch

        sc = self.scene
        dt = torch.uint8 if sc.pixfmt == 1 else torch.uint16
        out = torch.empty((count, sc.H, sc.W), dtype=dt, device=self.device)
        return self.generate_into(out, s_first, count)
