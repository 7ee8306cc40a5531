"""CPU oracle for quadrature lock-in discrimination (QLD) -- TEST INFRASTRUCTURE.

A ctypes wrapper around ``qld_oracle.cpp``: plain loops over pixels and
frames in int64 / FP64, restating the paper's definitions (Methods,
"Numerical simulations": the quadrature sums and R(j,k); the FFT map
|F(j,k,omega_q)|^2). It is independent of the CUDA library and imports
nothing from it. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.

Array convention: a window is a numpy array ``x`` of shape (N, npix) (or
(N, H, W)) holding frames s0 .. s0+N-1, uint8 or uint16; s is the absolute
1-based frame index of the stream.
"""
import ctypes

import numpy as np

from . import build as _build

_i64 = ctypes.c_int64
_p = ctypes.c_void_p
_int = ctypes.c_int


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _window(x):
    x = np.asarray(x)
    if x.dtype == np.uint8:
        fmt = 1
    elif x.dtype == np.uint16:
        fmt = 2
    else:
        raise TypeError("oracle windows are uint8 or uint16, got %s" % x.dtype)
    N = x.shape[0]
    pix_shape = x.shape[1:]
    flat = np.ascontiguousarray(x.reshape(N, -1))
    return flat, fmt, N, pix_shape


class Oracle:
    """The oracle's functions bound to one compiled copy of qld_oracle.cpp."""

    def __init__(self, lib_path):
        lib = ctypes.CDLL(lib_path)
        lib.orc_reference_tables.argtypes = [_p, _p]
        lib.orc_reference_tables.restype = None
        lib.orc_quadrature_sums.argtypes = [_p, _int, _i64, _i64, _int, _i64, _p, _p, _int]
        lib.orc_quadrature_sums.restype = _int
        lib.orc_amplitude_phase.argtypes = [_p, _p, _i64, _p, _p]
        lib.orc_amplitude_phase.restype = _int
        lib.orc_dft_bin.argtypes = [_p, _int, _i64, _i64, _int, _i64, _i64, _p, _p, _p, _int]
        lib.orc_dft_bin.restype = _int
        lib.orc_lockin_general.argtypes = [_p, _int, _i64, _i64, _int, _i64, ctypes.c_double, _p, _p, _p, _p, _int]
        lib.orc_lockin_general.restype = _int
        lib.orc_cnr.argtypes = [_p, _int, _int, _int, _int, _int, _p]
        lib.orc_cnr.restype = _int
        lib.orc_conv3x3_fwd.argtypes = [_p, _p, _p, _int, _int, _int, _int, _int, _p]
        lib.orc_conv3x3_fwd.restype = _int
        lib.orc_conv3x3_bwd.argtypes = [_p, _p, _p, _int, _int, _int, _int, _int, _p, _p, _p]
        lib.orc_conv3x3_bwd.restype = _int
        self.lib = lib
        self.path = lib_path

    def reference_tables(self):
        """sin(pi r/2), cos(pi r/2) for r = s mod 4 (the pre-calculated arrays)."""
        s = np.zeros(4, np.int64)
        c = np.zeros(4, np.int64)
        self.lib.orc_reference_tables(_ptr(s), _ptr(c))
        return s, c

    def quadrature_sums(self, x, s0=1, nthreads=1):
        """Exact int64 (S, C) of the window x (frames s0 .. s0+N-1)."""
        flat, fmt, N, shape = _window(x)
        npix = flat.shape[1]
        S = np.zeros(npix, np.int64)
        C = np.zeros(npix, np.int64)
        rc = self.lib.orc_quadrature_sums(_ptr(flat), fmt, npix, npix, N, int(s0), _ptr(S), _ptr(C),
                                          int(nthreads))
        if rc != 0:
            raise ValueError("orc_quadrature_sums rejected its arguments")
        return S.reshape(shape), C.reshape(shape)

    def amplitude_phase(self, S, C):
        """FP64 R = sqrt(S^2 + C^2) and phase = atan2(-S, C) from int64 sums."""
        S = np.ascontiguousarray(np.asarray(S, np.int64))
        C = np.ascontiguousarray(np.asarray(C, np.int64))
        R = np.zeros(S.shape, np.float64)
        ph = np.zeros(S.shape, np.float64)
        rc = self.lib.orc_amplitude_phase(_ptr(S), _ptr(C), S.size, _ptr(R), _ptr(ph))
        if rc != 0:
            raise ValueError("orc_amplitude_phase rejected its arguments")
        return R, ph

    def qld(self, x, s0=1, nthreads=1):
        """(S, C, R, phase) of the window x: the whole QLD image computation."""
        S, C = self.quadrature_sums(x, s0, nthreads)
        R, ph = self.amplitude_phase(S, C)
        return S, C, R, ph

    def dft_bin(self, x, k, s0=1, nthreads=1):
        """FP64 (re, im, |X_k|^2) of bin k over the window x (frames s0 .. s0+N-1)."""
        flat, fmt, N, shape = _window(x)
        npix = flat.shape[1]
        re = np.zeros(npix, np.float64)
        im = np.zeros(npix, np.float64)
        pw = np.zeros(npix, np.float64)
        rc = self.lib.orc_dft_bin(_ptr(flat), fmt, npix, npix, N, int(s0), int(k), _ptr(re), _ptr(im),
                                  _ptr(pw), int(nthreads))
        if rc != 0:
            raise ValueError("orc_dft_bin rejected its arguments")
        return re.reshape(shape), im.reshape(shape), pw.reshape(shape)


    def lockin_general(self, x, omega_dt, s0=1, nthreads=1):
        """FP64 (S, C, R, phase) of the lock-in at omega*dt = omega_dt rad/frame."""
        flat, fmt, N, shape = _window(x)
        npix = flat.shape[1]
        out = [np.zeros(npix, np.float64) for _ in range(4)]
        rc = self.lib.orc_lockin_general(_ptr(flat), fmt, npix, npix, N, int(s0), float(omega_dt),
                                         *[_ptr(a) for a in out], int(nthreads))
        if rc != 0:
            raise ValueError("orc_lockin_general rejected its arguments")
        return tuple(a.reshape(shape) for a in out)

    def cnr(self, img, r0, c0, m):
        """Contrast-to-noise ratio of the m x m source at (r0, c0) of img."""
        img = np.ascontiguousarray(np.asarray(img, np.float64))
        H, W = img.shape
        out = np.zeros(1, np.float64)
        rc = self.lib.orc_cnr(_ptr(img), H, W, int(r0), int(c0), int(m), _ptr(out))
        if rc != 0:
            raise ValueError("orc_cnr: the surround ring leaves the image")
        return float(out[0])

    def conv3x3(self, x, w, bias=None):
        """FP64 3x3 convolution, zero padding 1: x [B,H,W,Cin], w [3,3,Cin,Cout]."""
        x = np.ascontiguousarray(x, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        B, H, W, Cin = x.shape
        Cout = w.shape[3]
        assert w.shape == (3, 3, Cin, Cout)
        b = None if bias is None else np.ascontiguousarray(bias, np.float64)
        out = np.zeros((B, H, W, Cout), np.float64)
        rc = self.lib.orc_conv3x3_fwd(_ptr(x), _ptr(w), _ptr(b), B, H, W, Cin, Cout, _ptr(out))
        if rc != 0:
            raise ValueError("orc_conv3x3_fwd rejected its arguments")
        return out

    def conv3x3_backward(self, x, w, g):
        """FP64 (dx, dw, dbias) of a 3x3 convolution for the output gradient g."""
        x = np.ascontiguousarray(x, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        g = np.ascontiguousarray(g, np.float64)
        B, H, W, Cin = x.shape
        Cout = w.shape[3]
        dx = np.zeros_like(x)
        dw = np.zeros_like(w)
        db = np.zeros(Cout, np.float64)
        rc = self.lib.orc_conv3x3_bwd(_ptr(x), _ptr(w), _ptr(g), B, H, W, Cin, Cout, _ptr(dx), _ptr(dw), _ptr(db))
        if rc != 0:
            raise ValueError("orc_conv3x3_bwd rejected its arguments")
        return dx, dw, db


_default = None


def get():
    """The oracle built from this directory's qld_oracle.cpp (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle(_build.build())
    return _default


def reference_tables():
    return get().reference_tables()


def quadrature_sums(x, s0=1, nthreads=1):
    return get().quadrature_sums(x, s0, nthreads)


def amplitude_phase(S, C):
    return get().amplitude_phase(S, C)


def qld(x, s0=1, nthreads=1):
    return get().qld(x, s0, nthreads)


def dft_bin(x, k, s0=1, nthreads=1):
    return get().dft_bin(x, k, s0, nthreads)


def lockin_general(x, omega_dt, s0=1, nthreads=1):
    return get().lockin_general(x, omega_dt, s0, nthreads)


def cnr(img, r0, c0, m):
    return get().cnr(img, r0, c0, m)


def conv3x3(x, w, bias=None):
    return get().conv3x3(x, w, bias)


def conv3x3_backward(x, w, g):
    return get().conv3x3_backward(x, w, g)
