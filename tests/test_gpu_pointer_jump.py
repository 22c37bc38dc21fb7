"""The paper's pointer-jumping labelling (Sec. 3.3, Alg. 1), kept as an
in-library comparison for the union-find labelling: the partition it
converges to equals the oracle's flood fill (compared after renaming every
component to its minimum linear index), every label names a pixel of its own
component, and concave corners -- the case its reconnect step exists for --
come out whole."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import context, torch_cuda

pytestmark = pytest.mark.gpu


def _run(m, conn, period=16):
    torch = torch_cuda()
    ctx = context()
    lab = torch.empty(m.size, dtype=torch.int32, device="cuda")
    iters = ctx.ccl_pointer_jumping(ctx.mask(m), lab, conn, period=period)
    return lab.cpu().numpy().reshape(m.shape), iters


def _check(m, conn, period=16):
    got, iters = _run(m, conn, period)
    flat, mk = got.ravel(), m.ravel().astype(bool)
    fg = flat >= 0
    np.testing.assert_array_equal(fg, mk)
    assert mk[flat[fg]].all(), "a label names a background pixel"
    # rename each label class to its minimum pixel index
    idx = np.arange(flat.size)
    low = np.full(flat.size, np.iinfo(np.int64).max)
    np.minimum.at(low, flat[fg], idx[fg])
    canon = np.where(fg, low[np.where(fg, flat, 0)], -1).reshape(m.shape)
    exp, _ = oracle.ccl(m, conn)
    np.testing.assert_array_equal(canon, exp)
    # the label of a component is one of its pixels
    assert (exp.ravel()[flat[fg]] == exp.ravel()[fg]).all()
    return iters


@pytest.mark.parametrize("p", [0.3, 0.5, 0.6])
@pytest.mark.parametrize("conn", [8, 4])
def test_random_masks(p, conn):
    m = wl.bernoulli_mask(300, 700, p, seed=int(100 * p) + conn)
    assert _check(m, conn) >= 16


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("name", ["spiral", "checker", "rings"])
def test_adversarial_patterns(name, conn):
    make = {"spiral": wl.spiral_mask, "checker": wl.checkerboard_mask, "rings": wl.rings_mask}[name]
    _check(make(96, 128), conn)


@pytest.mark.parametrize("period", [1, 8, 16])
def test_concave_corners_and_reconnect_periods(period):
    """Combs and U shapes: components whose corners the main iteration alone
    leaves split (pixel (a, b) set with (a+1, b) and (a, b+1), but not
    (a+1, b+1)); the captions' period 8, the text's 16, and every step."""
    m = np.zeros((64, 96), dtype=np.uint8)
    m[5, 5:90] = 1
    for x in range(5, 90, 4):
        m[5:60, x] = 1          # a comb hanging from one bar
    m[62, 0:96] = 1
    m[40:62, 0] = 1
    m[40:62, 95] = 1            # a U along the bottom edge
    for conn in (8, 4):
        _check(m, conn, period)


def test_empty_full_and_single_pixels():
    for m in (np.zeros((17, 33), np.uint8), np.ones((17, 33), np.uint8)):
        for conn in (8, 4):
            _check(m, conn)
    m = np.zeros((9, 40), np.uint8)
    m[::2, ::3] = 1
    _check(m, 8)
    _check(m, 4)


def test_matches_union_find_on_a_large_mask():
    """2048 x 2048 at p = 0.5: the same partition as vl_ccl."""
    torch = torch_cuda()
    m = wl.bernoulli_mask(2048, 2048, 0.5, seed=7)
    ctx = context()
    lab = torch.empty(m.size, dtype=torch.int32, device="cuda")
    ctx.ccl(ctx.mask(m), lab, 8)
    assert ctx.ccl_status() == 0
    uf = lab.cpu().numpy()
    pj, _ = _run(m, 8)
    flat = pj.ravel()
    fg = flat >= 0
    # every union-find component carries exactly one pointer-jumping label
    # and vice versa
    pairs = np.unique(np.stack([uf[fg], flat[fg]]), axis=1)
    assert pairs.shape[1] == len(np.unique(uf[fg])) == len(np.unique(flat[fg]))
