"""The C-ABI library loads on a machine without a GPU, exports every entry
point include/qld.h declares, and rejects bad arguments before touching the
device."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1511_03390_b300 as q

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qld.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qld_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["qld_create", "qld_push_frames", "qld_image", "qld_fft_bin", "qld_destroy", "qld_get_iq",
                     "qld_frames_pushed", "qld_sync", "qld_strerror", "qld_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(q.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", q.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (qld_[a-z0-9_]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_binding_covers_every_declared_function():
    for n in declared_functions():
        assert hasattr(q, n), n


def test_library_is_built_for_sm_103a():
    from paper_1511_03390_b300 import build

    assert "arch=compute_103a,code=sm_103a" in build.NVCC_FLAGS


@pytest.mark.parametrize("H,W,N,fmt", [(0, 4, 8, 1), (4, 0, 8, 1), (4, 4, 6, 1), (4, 4, 0, 1), (4, 4, -4, 2),
                                       (4, 4, 8, 4), (4, 4, 8, 0), (3, 5, 8, 3), (4, 4, 65540, 2),
                                       (65536, 65536, 4, 1)])
def test_create_rejects_bad_arguments(H, W, N, fmt):
    assert q.lib.qld_create(H, W, N, fmt) is None
    assert q.qld_last_error() == q.QLD_E_INVAL
    assert q.qld_footprint_bytes(H, W, N, fmt) == q.QLD_E_INVAL


@pytest.mark.parametrize("H_total,W,N,fmt,row0,rows", [
    (16, 16, 8, 2, 12, 8),    # band runs past the frame
    (16, 16, 8, 2, -1, 4),    # negative start
    (16, 16, 8, 2, 0, 0),     # empty band
    (16, 16, 6, 2, 0, 8),     # bad window
    (16, 15, 8, 3, 1, 2),     # packed band starting mid pixel pair
    (16, 15, 8, 3, 0, 3),     # packed band of an odd pixel count
    (65536, 65536, 4, 1, 0, 1),  # whole frame too large
])
def test_create_band_rejects_bad_arguments(H_total, W, N, fmt, row0, rows):
    assert q.lib.qld_create_band(H_total, W, N, fmt, row0, rows) is None
    assert q.qld_last_error() == q.QLD_E_INVAL


def test_budget_refuses_a_band_by_its_own_footprint():
    band = q.qld_footprint_bytes(256, 1024, 1024, 2)
    q.qld_set_mem_budget(band - 1)
    try:
        assert q.lib.qld_create_band(1024, 1024, 1024, 2, 256, 256) is None
        assert q.qld_last_error() == q.QLD_E_NOMEM
        assert q.qld_mem_in_use() == 0
    finally:
        q.qld_set_mem_budget(0)


def test_footprint():
    # ring: N slots of the frame size rounded up to 256 bytes; two int32 sum
    # planes padded to 64 pixels; N float2 twiddles rounded up to 256 bytes.
    assert q.qld_footprint_bytes(128, 128, 64, 1) == 64 * 16384 + 2 * 4 * 16384 + 512
    assert q.qld_footprint_bytes(1024, 1024, 1024, 2) == 1024 * 2 ** 21 + 2 * 4 * 2 ** 20 + 8192
    assert q.qld_footprint_bytes(1, 17, 4, 1) == 4 * 256 + 2 * 4 * 64 + 256
    # packed 12-bit: 1.5 bytes per pixel, slots a whole number of 24-byte vectors
    assert q.qld_footprint_bytes(1024, 1024, 1024, 3) == 1024 * 3 * 2 ** 19 + 2 * 4 * 2 ** 20 + 8192
    # a 255-byte frame rounds up to 264 (11 vectors of 24 B), then to a 512-byte slot
    assert q.qld_footprint_bytes(1, 170, 4, 3) == 4 * 512 + 2 * 4 * 192 + 256
    big = q.qld_footprint_bytes(4096, 4096, 2048, 2)
    assert big == 2048 * 32 * 2 ** 20 + 2 * 4 * 2 ** 24 + 16384
    assert big > 68.7e9


def test_budget_refuses_before_allocating():
    q.qld_set_mem_budget(1 << 20)
    try:
        assert q.lib.qld_create(1024, 1024, 1024, 2) is None
        assert q.qld_last_error() == q.QLD_E_NOMEM
        assert q.qld_mem_in_use() == 0
    finally:
        q.qld_set_mem_budget(0)


def test_null_context_and_strings():
    assert q.lib.qld_push_frames(None, None, 0, None) == q.QLD_E_INVAL
    assert q.lib.qld_image(None, None, None) == q.QLD_E_INVAL
    assert q.lib.qld_fft_bin(None, 0, None) == q.QLD_E_INVAL
    assert q.lib.qld_iq_pointers(None, None, None) == q.QLD_E_INVAL
    assert q.lib.qld_sync(None) == q.QLD_E_INVAL
    assert q.lib.qld_frames_pushed(None) == -1
    assert q.qld_strerror(q.QLD_E_NOT_READY).startswith("window not full")
    assert q.qld_strerror(12345) == "unknown status"
    assert "sm_103a" in q.qld_version()


def test_c_program_builds_links_and_runs():
    """tests/abi_check.c: the header compiles as pedantic C99 and a C program
    links to libqld.so and gets the right answers from it, no Python or torch
    involved."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    build = os.path.join(root, "_build")
    os.makedirs(build, exist_ok=True)
    exe = os.path.join(build, "abi_check")
    libdir = os.path.dirname(q.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.dirname(HEADER),
                    os.path.join(root, "tests", "abi_check.c"), "-o", exe, "-L", libdir, "-lqld",
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
