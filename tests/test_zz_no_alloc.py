"""Labelling without device allocation (vl_ccl_noalloc).

Some callers cannot allocate device memory: cudaMalloc synchronises the whole
GPU, an application may have reserved all device memory for its own pool, or
the memory may belong to another allocator.  vl_ccl_noalloc serves them: the
caller passes the packed mask and the label buffer, and the working memory is
a fixed array inside the library.  This file checks, through the C ABI, that
two calls in a row give exactly the labels of the allocating vl_ccl and of
the CPU oracle's flood fill (labels are integers, so the comparison is
exact), that padding bits set in the caller's buffer are ignored, and that
an image too large for the fixed array is refused.  It is collected last on
purpose and passes both alone and after the other tests.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import context, torch_cuda

pytestmark = pytest.mark.gpu


def _packed(mask: np.ndarray) -> np.ndarray:
    """(H, Wp) uint32 words: LSB-first bits, rows padded to 128 pixels with 0."""
    H, W = mask.shape
    Wp = ((W + 127) // 128) * 4
    padded = np.zeros((H, Wp * 32), np.uint8)
    padded[:, :W] = mask != 0
    return np.packbits(padded, axis=1, bitorder="little").view(np.uint32).copy()


def _labels_with_allocation(mask: np.ndarray, conn: int) -> np.ndarray:
    torch = torch_cuda()
    ctx = context()
    lab = torch.empty(mask.size, dtype=torch.int32, device="cuda")
    ctx.ccl(ctx.mask(mask), lab, conn)
    assert ctx.ccl_status() == 0, ctx.last_error()
    return lab.cpu().numpy().reshape(mask.shape)


def _labels_without_allocation(mask: np.ndarray, conn: int, stream, words_host=None) -> np.ndarray:
    torch = torch_cuda()
    from paper_2010_07284_gb300 import _native as N
    H, W = mask.shape
    words = torch.from_numpy(_packed(mask) if words_host is None else words_host).cuda()
    labels = torch.full((H * W,), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = N.load().vl_ccl_noalloc(words.data_ptr(), H, W, conn, labels.data_ptr(), 1,
                                 stream.cuda_stream)
    assert rc == N.OK, f"vl_ccl_noalloc returned {N.STATUS_NAMES.get(rc, rc)}"
    return labels.cpu().numpy().reshape(H, W)


def test_two_calls_in_a_row_match_the_allocating_entry_point():
    torch = torch_cuda()
    stream = torch.cuda.Stream()
    first = (wl.bernoulli_mask(700, 1500, 0.5, seed=21), 8)
    second = (wl.spiral_mask(1000, 2048), 4)   # reuses the array the first call left behind
    for mask, conn in (first, second):
        got = _labels_without_allocation(mask, conn, stream)
        exp = _labels_with_allocation(mask, conn)
        np.testing.assert_array_equal(got, exp)
        ref, _ = oracle.ccl(mask, conn)
        np.testing.assert_array_equal(got, ref)


def test_padding_bits_in_the_callers_buffer_are_ignored():
    """A caller's packed buffer may hold garbage in the bits past column
    w - 1 of each row (here: every padding bit set, on every row, the last
    one included); the labels must equal those of the clean buffer."""
    torch = torch_cuda()
    stream = torch.cuda.Stream()
    for (H, W), conn in (((300, 1000), 8), ((257, 1100), 4), ((64, 33), 8)):
        mask = wl.bernoulli_mask(H, W, 0.55, seed=H + W)
        words = _packed(mask)
        Wp = words.shape[1]
        bits = np.zeros((H, Wp * 32), np.uint8)
        bits[:, W:] = 1
        words |= np.packbits(bits, axis=1, bitorder="little").view(np.uint32)
        got = _labels_without_allocation(mask, conn, stream, words_host=words)
        ref, _ = oracle.ccl(mask, conn)
        np.testing.assert_array_equal(got, ref)


def test_images_beyond_the_fixed_array_are_refused():
    torch = torch_cuda()
    from paper_2010_07284_gb300 import _native as N
    lib = N.load()
    # 4096 x 4096 needs 512 tiles of 16384 entries: more than the 2^20 held;
    # the call refuses on the host before touching the (small) buffers
    words = torch.zeros(16, dtype=torch.int32, device="cuda")
    labels = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = lib.vl_ccl_noalloc(words.data_ptr(), 4096, 4096, 8, labels.data_ptr(), 1,
                            torch.cuda.current_stream().cuda_stream)
    assert rc == N.ERR_SHAPE
