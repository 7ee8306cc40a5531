"""Python binding of the B300 QLD library (libqld.so, C ABI in include/qld.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels. Device buffers are torch CUDA tensors (or raw integer addresses);
streams are torch.cuda.Stream objects, raw cudaStream_t integers, or None for
torch's current stream. The functions carry the C names.

The package refuses to import when libqld.so has not been built: there is no
fallback path. Build it with ``python -m paper_1511_03390_b300.build``.
"""
import ctypes
import os

from . import build as _build

__all__ = [
    "QLD_U8", "QLD_U16", "QLD_P12", "QLD_OK", "QLD_E_INVAL", "QLD_E_NOMEM", "QLD_E_NOT_READY", "QLD_E_CUDA",
    "QLD_E_TIMEOUT", "QLD_MAX_N", "QLDError", "Context", "qld_create", "qld_create_band", "qld_destroy",
    "qld_push_frames",
    "qld_push_image", "qld_image", "qld_fft_bin", "qld_step", "qld_step_host", "qld_push_frames_host", "qld_image_host",
    "qld_fft_bin_host", "qld_get_iq", "qld_iq_pointers", "qld_reset", "qld_frames_pushed", "qld_sync", "qld_stream",
    "qld_strerror", "qld_last_error", "qld_version", "qld_footprint_bytes", "qld_set_mem_budget",
    "qld_mem_in_use", "qld_launch_count", "qld_fft_bin_frames_noalloc", "QLD_NOALLOC_MAX_N",
    "qld_lockin_table", "qld_lockin_frames", "Server", "QLD_SERVER_MAX_STREAMS", "qld_server_create",
    "qld_server_destroy", "qld_server_request", "qld_server_state", "qld_server_close", "qld_server_submit",
    "qld_server_submit_many", "qld_server_tick_gated", "qld_server_last_gated_us",
    "qld_server_num_shapes", "qld_server_set_shape",
    "qld_server_tick", "qld_server_image", "qld_server_iq", "qld_server_frames_pushed", "qld_server_mem_in_use",
    "qld_server_sync", "qld_server_autotune", "qld_server_shape", "nn", "LIB_PATH", "lib",
]

QLD_U8, QLD_U16, QLD_P12 = 1, 2, 3
QLD_OK, QLD_E_INVAL, QLD_E_NOMEM, QLD_E_NOT_READY, QLD_E_CUDA, QLD_E_TIMEOUT = 0, -1, -2, -3, -4, -5
QLD_MAX_N = 65536
QLD_NOALLOC_MAX_N = 16384
QLD_SERVER_MAX_STREAMS = 64

LIB_PATH = _build.LIB
if not _build.up_to_date():
    # Missing, or older than its sources: rebuild in-tree with nvcc.
    try:
        _build.build()
    except Exception as exc:  # no nvcc, or a compile error
        if not os.path.exists(LIB_PATH):
            raise ImportError("libqld.so is not built (%s) and building it failed: %s" % (LIB_PATH, exc))

_p = ctypes.c_void_p
_i = ctypes.c_int
_ll = ctypes.c_longlong

lib = ctypes.CDLL(LIB_PATH)
_SIGS = {
    "qld_create": ([_i, _i, _i, _i], _p),
    "qld_create_band": ([_i, _i, _i, _i, _i, _i], _p),
    "qld_footprint_bytes": ([_i, _i, _i, _i], _ll),
    "qld_set_mem_budget": ([_ll], None),
    "qld_mem_in_use": ([], _ll),
    "qld_launch_count": ([], _ll),
    "qld_destroy": ([_p], None),
    "qld_push_frames": ([_p, _p, _i, _p], _i),
    "qld_push_image": ([_p, _p, _i, _p, _p, _p], _i),
    "qld_image": ([_p, _p, _p], _i),
    "qld_fft_bin": ([_p, _i, _p], _i),
    "qld_step": ([_p, _p, _i, _p, _p, _p, _i, _p], _i),
    "qld_step_host": ([_p, _p, _i, _p, _p, _p, _i, _p], _i),
    "qld_push_frames_host": ([_p, _p, _i, _p], _i),
    "qld_image_host": ([_p, _p, _p], _i),
    "qld_fft_bin_host": ([_p, _i, _p], _i),
    "qld_fft_bin_frames_noalloc": ([_p, _i, _i, _i, _i, _i, _p, _p], _i),
    "qld_lockin_table": ([ctypes.c_double, _ll, _i, _p, _p], _i),
    "qldnn_conv3x3_fwd": ([_p, _p, _p, _i, _i, _i, _i, _i, _i, _p, _p, _p], _i),
    "qldnn_conv3x3_dgrad": ([_p, _p, _i, _i, _i, _i, _i, _p, _p, _p, _p], _i),
    "qldnn_conv3x3_wgrad": ([_p, _p, _i, _i, _i, _i, _i, _p, _p], _i),
    "qldnn_bias_grad": ([_p, _ll, _i, _p, _p], _i),
    "qldnn_relu_bwd": ([_p, _p, _ll, _p, _p], _i),
    "qldnn_relu_bwd_bias": ([_p, _p, _ll, _i, _p, _p, _p], _i),
    "qldnn_avgpool2": ([_p, _i, _i, _i, _i, _p, _p], _i),
    "qldnn_avgpool2_bwd": ([_p, _i, _i, _i, _i, _p, _i, _p], _i),
    "qldnn_upsample2": ([_p, _i, _i, _i, _i, _p, _p], _i),
    "qldnn_upsample2_bwd": ([_p, _i, _i, _i, _i, _p, _p], _i),
    "qldnn_concat": ([_p, _i, _p, _i, _ll, _p, _p], _i),
    "qldnn_upsample_concat": ([_p, _i, _p, _i, _i, _i, _i, _p, _p], _i),
    "qldnn_split": ([_p, _ll, _i, _i, _p, _p, _i, _p], _i),
    "qldnn_head": ([_p, _p, _p, _ll, _i, _p, _p], _i),
    "qldnn_head_bwd": ([_p, _p, _p, _ll, _i, _p, _p, _p, _p], _i),
    "qldnn_mse": ([_p, _p, _ll, _p, _p, _p], _i),
    "qldnn_adam": ([_p, _p, _p, _p, _ll, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _i, _p,
                    _p], _i),
    "qldnn_cast_bf16": ([_p, _ll, _p, _p], _i),
    "qldnn_add": ([_p, _p, _ll, _p], _i),
    "qldnn_pack_input": ([_p, _p, _ll, ctypes.c_float, _p, _p, _p], _i),
    "qldnn_zero": ([_p, _ll, _p], _i),
    "qldnn_kmajor_weights": ([_p, _i, _i, _i, _p, _p], _i),
    "qldnn_conv3x3_fwd_tc": ([_p, _p, _p, _i, _i, _i, _i, _i, _i, _p, _p, _p, _p], _i),
    "qldnn_conv3x3_fwd_tc2": ([_p, _p, _p, _i, _i, _i, _i, _i, _i, _p, _p, _p, _p], _i),
    "qldnn_conv3x3_fwd_tma": ([_p, _p, _p, _i, _i, _i, _i, _i, _i, _p, _p, _p, _p], _i),
    "qldnn_conv3x3_fwd_tma_mode": ([_p, _p, _p, _i, _i, _i, _i, _i, _i, _p, _p, _p, _i, _p], _i),
    "qldnn_wait_selftest": ([_ll, _p, _p], _i),
    "qldnn_input_conv3x3": ([_p, _p, _i, _i, _i, ctypes.c_float, _p, _i, _i, _p, _i, _p, _ll, _p, _p], _i),
    "qldnn_conv3x3_fwd_tma_epi": ([_p, _p, _p, _i, _i, _i, _i, _i, _i, _p, _ll, _p, _p, _ll, _p, _p, _p, _p, _p, _i, _p],
                                  _i),
    "qldnn_conv3x3_fwd_tma_epi_mode": ([_p, _p, _p, _i, _i, _i, _i, _i, _i, _p, _ll, _p, _p, _ll, _p, _p, _p, _p, _p,
                                        _i, _i, _p], _i),
    "qldnn_conv3x3_wgrad_tma": ([_p, _p, _i, _i, _i, _i, _i, _p, _p, _p], _i),
    "qld_server_create": ([_ll, _i], _p),
    "qld_server_destroy": ([_p], None),
    "qld_server_request": ([_p, _i, _i, _i, _i], _i),
    "qld_server_state": ([_p, _i], _i),
    "qld_server_close": ([_p, _i], _i),
    "qld_server_submit": ([_p, _i, _p, _i], _i),
    "qld_server_submit_many": ([_p, _i, _p, _p, _p], _i),
    "qld_server_tick": ([_p, _p], _i),
    "qld_server_tick_gated": ([_p, _p, _p, _i, _ll], _i),
    "qld_server_last_gated_us": ([_p, ctypes.POINTER(ctypes.c_float)], _i),
    "qld_server_num_shapes": ([], _i),
    "qld_server_set_shape": ([_p, _i], _i),
    "qld_server_image": ([_p, _i, ctypes.POINTER(_p), ctypes.POINTER(_p)], _i),
    "qld_server_iq": ([_p, _i, _p, _p], _i),
    "qld_server_frames_pushed": ([_p, _i], _ll),
    "qld_server_mem_in_use": ([_p], _ll),
    "qld_server_sync": ([_p], _i),
    "qld_server_autotune": ([_p, _p, ctypes.POINTER(ctypes.c_float)], _i),
    "qld_server_shape": ([_p, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "qld_lockin_frames": ([_p, _i, _i, _i, _i, _p, _p, _p, _p], _i),
    "qld_get_iq": ([_p, _p, _p], _i),
    "qld_iq_pointers": ([_p, ctypes.POINTER(_p), ctypes.POINTER(_p)], _i),
    "qld_reset": ([_p], _i),
    "qld_frames_pushed": ([_p], _ll),
    "qld_sync": ([_p], _i),
    "qld_stream": ([_p], _p),
    "qld_strerror": ([_i], ctypes.c_char_p),
    "qld_last_error": ([], _i),
    "qld_version": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class QLDError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, lib.qld_strerror(status).decode(), status))


def _check(rc, where):
    if rc != QLD_OK:
        raise QLDError(rc, where)
    return rc


def _addr(buf, nbytes_needed=None, what="buffer"):
    """Device/host address of a tensor, numpy array or integer (None -> NULL)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):  # torch tensor
        if not buf.is_contiguous():
            raise ValueError("%s must be contiguous" % what)
        if nbytes_needed is not None and buf.numel() * buf.element_size() < nbytes_needed:
            raise ValueError("%s holds %d bytes, %d needed" % (what, buf.numel() * buf.element_size(),
                                                               nbytes_needed))
        return buf.data_ptr()
    if hasattr(buf, "__array_interface__"):  # numpy array
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("%s must be C-contiguous" % what)
        if nbytes_needed is not None and buf.nbytes < nbytes_needed:
            raise ValueError("%s holds %d bytes, %d needed" % (what, buf.nbytes, nbytes_needed))
        return buf.__array_interface__["data"][0]
    raise TypeError("unsupported %s type %r" % (what, type(buf)))


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _frame_bytes(npix, pixfmt):
    return npix // 2 * 3 if pixfmt == QLD_P12 else npix * pixfmt


class Context:
    """A qld_ctx handle with its geometry."""

    def __init__(self, handle, H, W, N, pixfmt, H_total=None, row0=0):
        self.handle = handle
        self.H, self.W, self.N, self.pixfmt = H, W, N, pixfmt
        self.npix = H * W
        self.frame_bytes = _frame_bytes(self.npix, pixfmt)
        # a row band reads rows row0 .. row0 + H - 1 of H_total x W frames
        self.H_total = H if H_total is None else H_total
        self.row0 = row0
        self.frame_pitch = _frame_bytes(self.H_total * W, pixfmt)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib.qld_destroy(self.handle)
            except Exception:
                pass
            self.handle = None

    def destroy(self):
        if self.handle:
            lib.qld_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def _h(ctx):
    if ctx is None or not ctx.handle:
        raise ValueError("invalid (destroyed) context")
    return ctx.handle


def qld_create(H, W, N, pixfmt):
    h = lib.qld_create(int(H), int(W), int(N), int(pixfmt))
    if not h:
        raise QLDError(lib.qld_last_error(), "qld_create")
    return Context(h, int(H), int(W), int(N), int(pixfmt))


def qld_create_band(H_total, W, N, pixfmt, row0, rows):
    """A context for rows row0 .. row0 + rows - 1 of H_total x W frames; its
    pushes take whole frames and its images, sums and bins are rows x W."""
    h = lib.qld_create_band(int(H_total), int(W), int(N), int(pixfmt), int(row0), int(rows))
    if not h:
        raise QLDError(lib.qld_last_error(), "qld_create_band")
    return Context(h, int(rows), int(W), int(N), int(pixfmt), H_total=int(H_total), row0=int(row0))


def qld_destroy(ctx):
    ctx.destroy()


def qld_footprint_bytes(H, W, N, pixfmt):
    return lib.qld_footprint_bytes(int(H), int(W), int(N), int(pixfmt))


def qld_set_mem_budget(nbytes):
    lib.qld_set_mem_budget(int(nbytes))


def qld_mem_in_use():
    return lib.qld_mem_in_use()


def qld_launch_count():
    return lib.qld_launch_count()


def _count_of(frames, count, frame_bytes):
    if count is not None:
        return int(count)
    if hasattr(frames, "shape") and len(frames.shape) >= 1:
        nbytes = frames.nbytes if hasattr(frames, "nbytes") else frames.numel() * frames.element_size()
        return nbytes // frame_bytes
    raise ValueError("count is required when frames is a raw address")


def qld_push_frames(ctx, frames, count=None, stream=None):
    n = _count_of(frames, count, ctx.frame_pitch)
    a = _addr(frames, n * ctx.frame_pitch, "frames")
    return _check(lib.qld_push_frames(_h(ctx), a, n, _stream(stream)), "qld_push_frames")


def qld_push_image(ctx, frames, count=None, stream=None, amp=None, phase=None):
    n = _count_of(frames, count, ctx.frame_pitch)
    a = _addr(frames, n * ctx.frame_pitch, "frames")
    return _check(lib.qld_push_image(_h(ctx), a, n, _stream(stream), _addr(amp, 4 * ctx.npix, "amp"),
                                     _addr(phase, 4 * ctx.npix, "phase")), "qld_push_image")


def qld_image(ctx, amp=None, phase=None):
    return _check(lib.qld_image(_h(ctx), _addr(amp, 4 * ctx.npix, "amp"), _addr(phase, 4 * ctx.npix, "phase")),
                  "qld_image")


def qld_fft_bin(ctx, k, out):
    return _check(lib.qld_fft_bin(_h(ctx), int(k), _addr(out, 4 * ctx.npix, "out")), "qld_fft_bin")


def qld_step(ctx, frames, count, k, power, stream=None, amp=None, phase=None):
    """qld_push_image then qld_fft_bin (bin k into `power`) as one kernel."""
    n = _count_of(frames, count, ctx.frame_pitch)
    a = _addr(frames, n * ctx.frame_pitch, "frames")
    return _check(lib.qld_step(_h(ctx), a, n, _stream(stream), _addr(amp, 4 * ctx.npix, "amp"),
                               _addr(phase, 4 * ctx.npix, "phase"), int(k), _addr(power, 4 * ctx.npix, "power")),
                  "qld_step")


def qld_step_host(ctx, frames, count, k, power, stream=None, amp=None, phase=None):
    """qld_step with host frames and host output images (valid after qld_sync)."""
    n = _count_of(frames, count, ctx.frame_pitch)
    a = _addr(frames, n * ctx.frame_pitch, "frames")
    return _check(lib.qld_step_host(_h(ctx), a, n, _stream(stream), _addr(amp, 4 * ctx.npix, "amp"),
                                    _addr(phase, 4 * ctx.npix, "phase"), int(k), _addr(power, 4 * ctx.npix, "power")),
                  "qld_step_host")


def qld_push_frames_host(ctx, frames, count=None, stream=None):
    n = _count_of(frames, count, ctx.frame_pitch)
    a = _addr(frames, n * ctx.frame_pitch, "host frames")
    return _check(lib.qld_push_frames_host(_h(ctx), a, n, _stream(stream)), "qld_push_frames_host")


def qld_image_host(ctx, amp=None, phase=None):
    return _check(lib.qld_image_host(_h(ctx), _addr(amp, 4 * ctx.npix, "amp"), _addr(phase, 4 * ctx.npix, "phase")),
                  "qld_image_host")


def qld_fft_bin_host(ctx, k, out):
    return _check(lib.qld_fft_bin_host(_h(ctx), int(k), _addr(out, 4 * ctx.npix, "out")), "qld_fft_bin_host")


def qld_fft_bin_frames_noalloc(frames, H, W, N, pixfmt, k, out, stream=None):
    """|X_k|^2 over N device frames without any allocation (see qld.h)."""
    nb = int(H) * int(W) * int(pixfmt)
    return _check(lib.qld_fft_bin_frames_noalloc(_addr(frames, int(N) * nb, "frames"), int(H), int(W), int(N),
                                                 int(pixfmt), int(k), _addr(out, 4 * int(H) * int(W), "out"),
                                                 _stream(stream)), "qld_fft_bin_frames_noalloc")


def qld_lockin_table(omega_dt, s0, N, table, stream=None):
    """Fills the device float32 [N][2] table with (cos, -sin)(omega_dt * s), s = s0 .. s0+N-1."""
    return _check(lib.qld_lockin_table(float(omega_dt), int(s0), int(N), _addr(table, 8 * int(N), "table"),
                                       _stream(stream)), "qld_lockin_table")


def qld_lockin_frames(frames, H, W, N, pixfmt, table, amp=None, phase=None, stream=None):
    """Amplitude and phase of the lock-in with `table` over N device frames."""
    npix = int(H) * int(W)
    return _check(lib.qld_lockin_frames(_addr(frames, int(N) * npix * int(pixfmt), "frames"), int(H), int(W), int(N),
                                        int(pixfmt), _addr(table, 8 * int(N), "table"), _addr(amp, 4 * npix, "amp"),
                                        _addr(phase, 4 * npix, "phase"), _stream(stream)), "qld_lockin_frames")


def qld_get_iq(ctx, S=None, C=None):
    return _check(lib.qld_get_iq(_h(ctx), _addr(S, 4 * ctx.npix, "S"), _addr(C, 4 * ctx.npix, "C")), "qld_get_iq")


def qld_iq_pointers(ctx):
    """Device addresses (ints) of the context's own sums S and C (int32
    [H*W]); their contents change with every push."""
    S, C = _p(), _p()
    _check(lib.qld_iq_pointers(_h(ctx), ctypes.byref(S), ctypes.byref(C)), "qld_iq_pointers")
    return S.value, C.value


def qld_reset(ctx):
    return _check(lib.qld_reset(_h(ctx)), "qld_reset")


def qld_frames_pushed(ctx):
    return lib.qld_frames_pushed(_h(ctx))


def qld_sync(ctx):
    return _check(lib.qld_sync(_h(ctx)), "qld_sync")


def qld_stream(ctx):
    return lib.qld_stream(_h(ctx)) or 0


def qld_strerror(status):
    return lib.qld_strerror(int(status)).decode()


def qld_last_error():
    return lib.qld_last_error()


def qld_version():
    return lib.qld_version().decode()


# ---- serving ---------------------------------------------------------------

class Server:
    """A qld_server handle (see qld.h: continuous batching of camera streams)."""

    def __init__(self, handle):
        self.handle = handle
        self.shapes = {}  # ticket -> (H, W, N, pixfmt)

    def destroy(self):
        if self.handle:
            lib.qld_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _sh(srv):
    if srv is None or not srv.handle:
        raise ValueError("invalid (destroyed) server")
    return srv.handle


def qld_server_create(hbm_budget_bytes, max_streams=QLD_SERVER_MAX_STREAMS):
    h = lib.qld_server_create(int(hbm_budget_bytes), int(max_streams))
    if not h:
        raise QLDError(lib.qld_last_error(), "qld_server_create")
    return Server(h)


def qld_server_destroy(srv):
    srv.destroy()


def qld_server_request(srv, H, W, N, pixfmt):
    t = lib.qld_server_request(_sh(srv), int(H), int(W), int(N), int(pixfmt))
    if t < 0:
        raise QLDError(t, "qld_server_request")
    srv.shapes[t] = (int(H), int(W), int(N), int(pixfmt))
    return t


def qld_server_state(srv, ticket):
    return lib.qld_server_state(_sh(srv), int(ticket))


def qld_server_close(srv, ticket):
    return _check(lib.qld_server_close(_sh(srv), int(ticket)), "qld_server_close")


def qld_server_submit(srv, ticket, frames, count=None):
    H, W, N, fmt = srv.shapes[ticket]
    fb = H * W // 2 * 3 if fmt == QLD_P12 else H * W * fmt
    n = _count_of(frames, count, fb)
    return _check(lib.qld_server_submit(_sh(srv), int(ticket), _addr(frames, n * fb, "frames"), n),
                  "qld_server_submit")


class SubmitBatch:
    """Reusable host arrays for qld_server_submit_many: set(i, ticket, frames,
    count) fills entry i (device frames, checked like qld_server_submit),
    submit(srv, n) hands over entries 0..n-1 in one call."""

    def __init__(self, capacity):
        self.tickets = (ctypes.c_int * capacity)()
        self.frames = (ctypes.c_void_p * capacity)()
        self.counts = (ctypes.c_int * capacity)()

    def set(self, i, srv, ticket, frames, count=None):
        H, W, N, fmt = srv.shapes[ticket]
        fb = H * W // 2 * 3 if fmt == QLD_P12 else H * W * fmt
        n = _count_of(frames, count, fb)
        self.tickets[i] = int(ticket)
        self.frames[i] = _addr(frames, n * fb, "frames")
        self.counts[i] = n

    def submit(self, srv, n):
        return _check(lib.qld_server_submit_many(_sh(srv), int(n), self.tickets, self.frames, self.counts),
                      "qld_server_submit_many")


def qld_server_submit_many(srv, submissions):
    """Hands over [(ticket, frames, count or None), ...] in one call."""
    b = SubmitBatch(max(1, len(submissions)))
    for i, sub in enumerate(submissions):
        ticket, frames = sub[0], sub[1]
        b.set(i, srv, ticket, frames, sub[2] if len(sub) > 2 else None)
    return b.submit(srv, len(submissions))


def qld_server_tick(srv, stream=None):
    n = lib.qld_server_tick(_sh(srv), _stream(stream))
    if n < 0:
        raise QLDError(n, "qld_server_tick")
    return n


def qld_server_last_gated_us(srv):
    """GPU microseconds of the last gated tick, doorbell seen -> images complete."""
    us = ctypes.c_float()
    _check(lib.qld_server_last_gated_us(_sh(srv), ctypes.byref(us)), "qld_server_last_gated_us")
    return us.value


def qld_server_tick_gated(srv, doorbell, target, timeout_ns, stream=None):
    """qld_server_tick once *doorbell >= target (device or mapped pinned host
    int32), waiting at most timeout_ns on the GPU; raises QLDError with
    QLD_E_TIMEOUT when the wait ran out (the submissions stay pending)."""
    n = lib.qld_server_tick_gated(_sh(srv), _stream(stream), _addr(doorbell, 4, "doorbell"), int(target),
                                  int(timeout_ns))
    if n < 0:
        raise QLDError(n, "qld_server_tick_gated")
    return n


def qld_server_image(srv, ticket):
    """(amp, phase) device addresses of the stream's latest images."""
    a, p = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.qld_server_image(_sh(srv), int(ticket), ctypes.byref(a), ctypes.byref(p)), "qld_server_image")
    return a.value, p.value


def qld_server_iq(srv, ticket, S=None, C=None):
    H, W, _, _ = srv.shapes[ticket]
    return _check(lib.qld_server_iq(_sh(srv), int(ticket), _addr(S, 4 * H * W, "S"), _addr(C, 4 * H * W, "C")),
                  "qld_server_iq")


def qld_server_frames_pushed(srv, ticket):
    return lib.qld_server_frames_pushed(_sh(srv), int(ticket))


def qld_server_mem_in_use(srv):
    return lib.qld_server_mem_in_use(_sh(srv))


def qld_server_sync(srv):
    return _check(lib.qld_server_sync(_sh(srv)), "qld_server_sync")


def qld_server_autotune(srv, stream=None):
    """Index of the fastest launch shape on the active streams, and its time (us)."""
    us = ctypes.c_float()
    k = lib.qld_server_autotune(_sh(srv), _stream(stream), ctypes.byref(us))
    if k < 0:
        raise QLDError(k, "qld_server_autotune")
    return k, us.value


def qld_server_num_shapes():
    return lib.qld_server_num_shapes()


def qld_server_set_shape(srv, index):
    """Fix the batched kernel's launch shape (an index as the autotuner returns)."""
    return _check(lib.qld_server_set_shape(_sh(srv), index), "qld_server_set_shape")


def qld_server_shape(srv):
    t, v, c = _i(), _i(), _i()
    _check(lib.qld_server_shape(_sh(srv), ctypes.byref(t), ctypes.byref(v), ctypes.byref(c)), "qld_server_shape")
    return t.value, v.value, c.value


class _NN:
    """The network kernels (qldnn_* in qld.h) with tensors or raw addresses as
    pointers; every call enqueues on torch's current stream unless `stream`
    is given, and raises QLDError on a non-OK status."""

    def __getattr__(self, name):
        f = getattr(lib, "qldnn_" + name)

        def call(*args, stream=None):
            conv = [_addr(a) if (a is None or hasattr(a, "data_ptr")) else a for a in args]
            return _check(f(*conv, _stream(stream)), "qldnn_" + name)

        return call


nn = _NN()
