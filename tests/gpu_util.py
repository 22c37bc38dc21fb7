"""Helpers for the GPU parity tests: evaluate a formula through the C ABI and
through the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


_CTX = {}


def context(mode="fused", **kw):
    import paper_2010_07284_gb300 as vg
    key = (mode, tuple(sorted(kw.items())))
    if key not in _CTX:
        _CTX[key] = vg.Context(exec_mode=mode, **kw)
    return _CTX[key]


def gpu_eval(ctx, records, roots, images=(), masks=(), conn=8, mode=None, stream=None):
    """Float images first, then masks, in the image list: node.image of a MASK
    atom is shifted by len(images) by the caller (see ``split_records``)."""
    F = ctx.compile(records, roots, conn)
    ims = [ctx.image(im, stream) for im in images] + [ctx.mask(m, stream) for m in masks]
    res = ctx.eval(F, ims, stream=stream, mode=mode)
    st = res.sync()
    assert st == 0, f"device status {st}: {ctx.last_error()}"
    out = [res.mask(r) for r in range(len(roots))]
    return out, F


def shift_mask_images(records, n_float):
    """The C ABI indexes one image list (floats then masks); the oracle keeps
    two lists.  Shift MASK atoms' image index for the C ABI."""
    out = []
    for (op, a, b, img, ch, t, q) in records:
        if op == "MASK":
            img = img + n_float
        out.append((op, a, b, img, ch, t, q))
    return out


def assert_same(got, exp, what=""):
    for r, (g, e) in enumerate(zip(got, exp)):
        if not np.array_equal(g, e):
            bad = np.argwhere(g != e)
            raise AssertionError(f"{what} root {r}: {len(bad)} of {e.size} pixels differ; "
                                 f"first {bad[:6].tolist()}")


def check_formula(records, roots, images=(), masks=(), conn=8, modes=("fused", "plain"), ctx=None):
    exp = oracle.evaluate(records, roots, list(images), list(masks), conn=conn,
                          shape=(masks[0].shape if masks and not images else None)).masks
    recs = shift_mask_images(records, len(images))
    for mode in modes:
        got, _ = gpu_eval(ctx or context(), recs, roots, images, masks, conn, mode=mode)
        assert_same(got, exp, f"{mode} conn={conn}")
    return exp
