"""Packed 12-bit input (QLD_P12, two pixels in three bytes, Mono12p order):
the same sums, images and DFT bins as unpacked data, on the vector path
(frames 8-byte aligned, a multiple of 24 bytes) and the scalar path."""
import numpy as np
import pytest
import torch

import paper_1511_03390_b300 as q
from qld_check import Stream, get_bin, get_image, get_iq, pack12

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_pack12_layout_by_hand():
    # pixels 0xABC, 0x123 -> bytes 0xBC, 0x3A, 0x12 (low byte of p0; high nibble
    # of p0 in the low half, low nibble of p1 in the high half; high byte of p1)
    assert list(pack12(np.array([0xABC, 0x123], np.uint16))) == [0xBC, 0x3A, 0x12]


@pytest.mark.parametrize("H,W,offset", [(64, 96, 0), (48, 80, 8), (37, 100, 0), (6, 7, 0), (64, 96, 1), (16, 32, 5)])
@pytest.mark.parametrize("N", [4, 16])
def test_packed_sliding_equals_recompute_every_step(H, W, offset, N):
    """(37x100: 5550 bytes, not a multiple of 24; 6x7: 63 bytes; offsets 1 and
    5: unaligned frames -- scalar path. The others: vector path.)"""
    rng = np.random.default_rng(H * W + N + offset)
    st = Stream(H, W, N, q.QLD_P12)
    for count in [1, 3, 4, 0, 2, N, 5, 2 * N + 1, 4, 4]:
        st.push(rng.integers(0, 4096, size=(count, H * W)).astype(np.uint16), offset=offset)
        st.check(bins=(N // 4, 1) if st.frames.shape[0] >= N else ())


def test_packed_equals_unpacked_uint16():
    rng = np.random.default_rng(31)
    H, W, N = 128, 192, 64
    a = Stream(H, W, N, q.QLD_P12)
    b = Stream(H, W, N, q.QLD_U16)
    for count in [N, 4, 4, 1, 7]:
        x = rng.integers(0, 4096, size=(count, H * W)).astype(np.uint16)
        a.push(x)
        b.push(x)
        Sa, Ca = get_iq(a.ctx)
        Sb, Cb = get_iq(b.ctx)
        assert np.array_equal(Sa, Sb) and np.array_equal(Ca, Cb)
        ia, ib = get_image(a.ctx), get_image(b.ctx)
        assert np.array_equal(ia[0], ib[0]) and np.array_equal(ia[1], ib[1])
    a.check(bins=(16, 3))
    # Both formats run the DFT bin on 8-pixel vectors with the same pixel
    # floats, twiddles and summation order: bit-identical powers.
    for k in (16, 3, 1):
        assert np.array_equal(get_bin(a.ctx, k), get_bin(b.ctx, k))


def test_packed_rejects_odd_pixel_count_and_sizes_footprint():
    with pytest.raises(q.QLDError) as e:
        q.qld_create(3, 5, 8, q.QLD_P12)
    assert e.value.status == q.QLD_E_INVAL
    # 1024x1024 packed: 1.5 MiB frames (a multiple of 24 and 256 bytes)
    assert q.qld_footprint_bytes(1024, 1024, 1024, q.QLD_P12) == 1024 * 3 * 2 ** 19 + 2 * 4 * 2 ** 20 + 8192
