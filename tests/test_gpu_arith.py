"""uint16 images and number terms (the tool's 16-bit pixels and basic
arithmetic, Sec. 3) on the GPU, element by element against the oracle: the
fused executor's arithmetic step and the plain form's one launch per
operation; thresholds, rank codes and percentiles reading uint16 planes and
number images; division by zero (NaN, infinities); the case-study spec on
a 7680 x 7680 uint16 slice as the paper ran it; a batch mixing formats."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import assert_same, check_formula, context, torch_cuda

pytestmark = pytest.mark.gpu


def _two_channel(h, w, seed):
    return np.stack([wl.gaussian_field_image(h, w, seed=seed)[0], wl.uniform_image(h, w, seed=seed)[0]])


@pytest.mark.parametrize("seed,shape,conn", [(0, (131, 1100), 8), (1, (64, 128), 4),
                                             (2, (300, 257), 8), (3, (1, 33), 8),
                                             (4, (517, 2049), 4)])
def test_number_terms_float_images(seed, shape, conn):
    torch_cuda()
    f = wl.arith_dag(80, seed=seed)
    check_formula(wl.formula_to_records(f), f.roots, [_two_channel(*shape, seed)], conn=conn)


@pytest.mark.parametrize("seed,shape", [(5, (200, 700)), (6, (97, 1500))])
def test_number_terms_uint16_with_zero_divisors(seed, shape):
    torch_cuda()
    f = wl.arith_dag(80, seed=seed)
    img = wl.uniform_image_u16(*shape, channels=2, seed=seed)
    img[:, ::5, ::3] = 0   # x / 0 and 0 / 0
    check_formula(wl.formula_to_records(f), f.roots, [img], conn=8)


def test_uint16_random_formula_thresholds_rank_codes_percentiles():
    """A 500-node random formula on a uint16 image with thresholds scaled to
    the 16-bit range (rank codes read the uint16 plane), plus percentiles."""
    torch_cuda()
    f = wl.random_dag(500, seed=4, max_depth=100)
    rec = [(op, a, b, im, ch, float(np.float32(round(t * 65535.0))), q)
           for (op, a, b, im, ch, t, q) in wl.formula_to_records(f)]
    n = len(rec)
    rec += [("PCT_GT", -1, -1, 0, 0, 0.0, 0.9), ("PCT_LT", -1, -1, 0, 0, 0.0, 0.05),
            ("AND", n, n - 1, 0, 0, 0.0, 0.0), ("NOT", n + 1, -1, 0, 0, 0.0, 0.0)]
    roots = list(f.roots) + [n + 2, n + 3]
    img = wl.uniform_image_u16(333, 1030, seed=4)
    img[0, :7, :7] = 65535
    check_formula(rec, roots, [img], conn=8)


def test_uint16_config4_formula_on_scaled_phantoms():
    """The MRI-shaped formula (percentiles, grow, N chains, surrounded,
    touch) on 16-bit phantoms, batched with float phantoms in one launch."""
    torch_cuda()
    f = wl.config4_formula()
    rec = wl.formula_to_records(f)
    sides = wl.mri_side_lengths(12, seed=21)
    imgs = wl.mri_phantom_batch(sides, seed=21)
    imgs = [wl.to_u16(im) if k % 2 == 0 else im for k, im in enumerate(imgs)]
    ctx = context()
    F = ctx.compile(rec, f.roots, 8)
    handles = [ctx.image(im) for im in imgs]
    assert [h.format for h in handles[:2]] == ["u16", "f32"]
    results = ctx.eval_batch([(F, [h]) for h in handles])
    for k, (im, res) in enumerate(zip(imgs, results)):
        assert res.sync() == 0, ctx.last_error()
        exp = oracle.evaluate(rec, f.roots, [im], conn=8).masks
        assert_same([res.mask(r) for r in range(len(f.roots))], exp, f"image {k}")


def test_batch_mixing_number_term_formulas_and_formats():
    torch_cuda()
    ctx = context()
    jobs, expect = [], []
    for k in range(6):
        f = wl.arith_dag(60, seed=30 + k)
        rec = wl.formula_to_records(f)
        shape = (50 + 37 * k, 90 + 101 * k)
        img = _two_channel(*shape, 30 + k)
        if k % 2:
            img = wl.to_u16(np.clip(img, 0.0, 1.0))
        F = ctx.compile(rec, f.roots, 8 if k % 3 else 4)
        jobs.append((F, [ctx.image(img)]))
        expect.append(oracle.evaluate(rec, f.roots, [img], conn=8 if k % 3 else 4).masks)
    for k, res in enumerate(ctx.eval_batch(jobs)):
        assert res.sync() == 0, ctx.last_error()
        assert_same([res.mask(r) for r in range(len(expect[k]))], expect[k], f"job {k}")


def test_nan_ordering_of_percentiles_on_the_gpu():
    """0/0 gives NaN, which sorts after +infinity: the top percentile of a
    quotient with NaN pixels is NaN (no pixel passes), lower ones are the
    order statistics of the numbers."""
    torch_cuda()
    img = np.zeros((2, 40, 150), dtype=np.float32)
    rng = np.random.default_rng(2)
    img[0] = rng.standard_normal((40, 150)).astype(np.float32)
    img[1] = rng.integers(-2, 3, size=(40, 150)).astype(np.float32)   # zeros: x/0, 0/0
    img[0, :3, :3] = 0.0
    rec = [("VALUE", -1, -1, 0, 0, 0, 0), ("VALUE", -1, -1, 0, 1, 0, 0),
           ("DIV", 0, 1, 0, 0, 0, 0)]
    roots = []
    for q in (0.0, 0.3, 0.6, 0.9, 0.99, 1.0):
        rec.append(("PCT_GT", 2, -1, 0, 0, 0.0, q))
        roots.append(len(rec) - 1)
        rec.append(("PCT_LT", 2, -1, 0, 0, 0.0, q))
        roots.append(len(rec) - 1)
    rec.append(("THR_GT", 2, -1, 0, 0, 1.0, 0.0))
    roots.append(len(rec) - 1)
    exp = check_formula(rec, roots, [img], conn=8)
    assert exp[10].sum() == 0 and exp[11].sum() == 0   # q = 1 picks NaN


def test_grow_spec_uint16_7680():
    """The case-study spec exactly as the paper runs it (Sec. 4.2): 16-bit
    pixels, thresholds 62258 and 56360, grow, on a 7680 x 7680 slice."""
    torch_cuda()
    from workloads.images import upscaled_slice
    f = wl.grow_spec_u16_formula()
    rec = wl.formula_to_records(f)
    img = wl.to_u16(upscaled_slice(7680))
    exp = oracle.evaluate(rec, f.roots, [img], conn=8).masks[0]
    assert 0 < exp.sum() < exp.size
    for mode in ("fused", "plain"):
        ctx = context(mode)
        F = ctx.compile(rec, f.roots, 8)
        res = ctx.eval(F, [ctx.image(img)])
        assert res.sync() == 0, ctx.last_error()
        assert_same([res.mask(0)], [exp], f"grow u16 7680 {mode}")


def test_hand_worked_spec_u16_fixture():
    """The case-study spec on the hand-worked 16-bit fixture (pixels on and
    next to both thresholds, a diagonal-only contact): the GPU gives the
    fixture's masks under both adjacencies, fused and plain."""
    torch_cuda()
    import golden_io
    import os
    fx = golden_io.load(os.path.join(golden_io.GOLDEN, "spec_u16.txt"))
    img = fx["image"].astype(np.uint16)[None]
    f = wl.grow_spec_u16_formula()
    for conn, exp in fx["expect"].items():
        check_formula(wl.formula_to_records(f), f.roots, [img], conn=conn)
        ctx = context()
        F = ctx.compile(wl.formula_to_records(f), f.roots, conn)
        res = ctx.eval(F, [ctx.image(img)])
        assert res.sync() == 0
        assert_same([res.mask(0)], [exp], f"fixture conn={conn}")
