"""Volumes on the GPU against the oracle's volume operators, element by
element: N with the 26- and 6-neighbourhoods, rho, and labelling of D x H x W
voxel grids (the paper's 3D outlook, Sec. 1 and Sec. 5), on MRI-shaped
phantom volumes and seeded noise.  Sizes put several labelling tiles in
every slice (rows beyond 32, more than 32 words per row), slices whose height
is and is not a multiple of the tile height, and ragged rows."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import assert_same, context, torch_cuda

pytestmark = pytest.mark.gpu


def _f(op, a=-1, b=-1, image=0, channel=0, t=0.0, q=0.0):
    return (op, a, b, image, channel, t, q)


def _run(records, roots, volumes=(), masks=(), conn=26):
    """The formula on the GPU (per-operator form, the one volumes have)."""
    torch_cuda()
    ctx = context()
    n_vol = len(volumes)
    recs = [(op, a, b, (img + n_vol if op == "MASK" else img), ch, t, q)
            for (op, a, b, img, ch, t, q) in records]
    F = ctx.compile(recs, roots, conn)
    ims = [ctx.volume(v) for v in volumes] + [ctx.mask_volume(m) for m in masks]
    res = ctx.eval(F, ims)
    st = res.sync()
    assert st == 0, f"device status {st}: {ctx.last_error()}"
    return [res.mask(r) for r in range(len(roots))]


@pytest.mark.parametrize("conn", (26, 6))
@pytest.mark.parametrize("shape", [(1, 13, 21), (3, 1, 40), (4, 45, 300), (6, 64, 1100),
                                   (9, 70, 1025)])
def test_near_and_reach_on_noise(conn, shape):
    rng = np.random.default_rng(sum(shape) + conn)
    a = (rng.random(shape) < 0.02).astype(np.uint8)
    b = (rng.random(shape) < (0.35 if conn == 26 else 0.55)).astype(np.uint8)
    recs = [_f("MASK", image=0), _f("MASK", image=1), _f("NEAR", 0), _f("REACH", 0, 1),
            _f("NEAR", 2), _f("GROW", 0, 1), _f("INTERIOR", 1), _f("SURROUNDED", 0, 1)]
    roots = [2, 3, 4, 5, 6, 7]
    got = _run(recs, roots, masks=[a, b], conn=conn)
    exp = oracle.evaluate3(recs, roots, masks=[a, b], conn=conn).masks
    assert_same([g.reshape(shape) for g in got], exp, f"conn={conn} {shape}")


@pytest.mark.parametrize("conn", (26, 6))
def test_segmentation_formula_on_mri_phantom_volumes(conn):
    """The 40-primitive segmentation formula (percentile thresholds over the
    whole volume, grow, N chains, interior, surrounded, touch) on MRI-shaped
    4-channel volumes, float32 and uint16."""
    f = wl.config4_formula()
    rec = wl.formula_to_records(f)
    for (d, h, w), seed in (((12, 48, 56), 0), ((7, 70, 1100), 1)):
        vol = wl.mri_phantom_volume(d, h, w, seed=seed)
        got = _run(rec, f.roots, volumes=[vol], conn=conn)
        exp = oracle.evaluate3(rec, f.roots, volumes=[vol], conn=conn).masks
        assert_same(got, exp, f"float32 conn={conn} {(d, h, w)}")
    vol16 = wl.to_u16(np.clip(wl.mri_phantom_volume(10, 40, 130, seed=3), 0, 1))
    got = _run(rec, f.roots, volumes=[vol16], conn=conn)
    exp = oracle.evaluate3(rec, f.roots, volumes=[vol16], conn=conn).masks
    assert_same(got, exp, f"uint16 conn={conn}")


@pytest.mark.parametrize("conn", (26, 6))
def test_random_formulas_on_volumes(conn):
    for seed in range(4):
        f = wl.random_dag(150, seed=seed, max_depth=40)
        rec = wl.formula_to_records(f)
        vol = wl.uniform_image(5 * 37, 90, seed=seed).reshape(1, 5, 37, 90)
        got = _run(rec, f.roots, volumes=[vol], conn=conn)
        exp = oracle.evaluate3(rec, f.roots, volumes=[vol], conn=conn).masks
        assert_same(got, exp, f"seed {seed} conn={conn}")


@pytest.mark.parametrize("conn", (26, 6))
@pytest.mark.parametrize("shape,p", [((8, 96, 1100), 0.25), ((16, 64, 256), 0.31),
                                     ((5, 33, 2100), 0.5), ((40, 40, 40), 0.2)])
def test_labels_of_noise_volumes(conn, shape, p):
    torch = torch_cuda()
    ctx = context()
    rng = np.random.default_rng(int(p * 100) + conn + shape[0])
    m = (rng.random(shape) < p).astype(np.uint8)
    mv = ctx.mask_volume(m)
    lab = torch.full((m.size,), -7, dtype=torch.int32, device="cuda")
    ctx.ccl(mv, lab, conn)
    assert ctx.ccl_status() == 0, ctx.last_error()
    exp, _ = oracle.ccl3(m, conn)
    np.testing.assert_array_equal(lab.cpu().numpy().reshape(shape), exp)


def test_one_slice_volumes_equal_the_image_path():
    """A volume of depth 1 under 26- (6-) adjacency is the image under 8-
    (4-) adjacency."""
    torch_cuda()
    f = wl.config4_formula()
    rec = wl.formula_to_records(f)
    img = wl.mri_phantom_batch([(90, 700)], seed=5)[0]
    for c3, c2 in ((26, 8), (6, 4)):
        got = _run(rec, f.roots, volumes=[img[:, None]], conn=c3)
        exp = oracle.evaluate(rec, f.roots, [img], conn=c2).masks
        assert_same(got, exp, f"conn {c3} vs {c2}")


def test_volumes_are_refused_by_the_batched_form():
    torch_cuda()
    ctx = context()
    f = wl.config4_formula()
    F = ctx.compile(wl.formula_to_records(f), f.roots, 26)
    vol = ctx.volume(wl.mri_phantom_volume(3, 20, 30, seed=0))
    with pytest.raises(Exception):
        ctx.batch([(F, [vol])])


@pytest.mark.parametrize("conn", (26, 6))
def test_large_volume_percentiles_take_the_grid_wide_select(conn):
    """Above a million voxels the percentile select runs over the whole grid:
    ties, NaN voxels (sorted last) and ranks at both ends, float32 and
    uint16, against the oracle's sort."""
    rng = np.random.default_rng(conn)
    vol = wl.mri_phantom_volume(20, 70, 1100, seed=4)
    vol[0, 3, 5, :40] = np.nan
    vol[1] = np.round(vol[1] * 50) / 50          # many ties
    recs = [_f("PCT_GT", q=0.0), _f("PCT_GT", q=0.95, channel=1), _f("PCT_LT", q=0.5, channel=0),
            _f("PCT_LT", q=1.0, channel=1), _f("PCT_GT", q=0.999, channel=2),
            _f("AND", 1, 2), _f("NEAR", 5)]
    roots = [0, 1, 2, 3, 4, 6]
    got = _run(recs, roots, volumes=[vol], conn=conn)
    exp = oracle.evaluate3(recs, roots, volumes=[vol], conn=conn).masks
    assert_same(got, exp, f"float32 conn={conn}")
    v16 = rng.integers(0, 700, size=(2, 12, 300, 400)).astype(np.uint16)
    got = _run(recs[:2] + [_f("PCT_LT", q=0.3, channel=1)], [0, 1, 2], volumes=[v16], conn=conn)
    exp = oracle.evaluate3(recs[:2] + [_f("PCT_LT", q=0.3, channel=1)], [0, 1, 2],
                           volumes=[v16], conn=conn).masks
    assert_same(got, exp, f"uint16 conn={conn}")


def test_large_image_percentiles_in_the_per_operator_form():
    torch_cuda()
    img = wl.uniform_image(1100, 1000, channels=2, seed=8)
    img[1] = np.round(img[1] * 30) / 30
    img[0, 7, :100] = np.nan
    recs = [_f("PCT_GT", q=0.25), _f("PCT_LT", q=0.75, channel=1), _f("PCT_GT", q=1.0, channel=1)]
    from gpu_util import check_formula
    check_formula(recs, [0, 1, 2], [img], conn=8, modes=("plain", "fused"))
