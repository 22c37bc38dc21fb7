"""Parity at the full sizes of the workloads, element by element against the
oracle: connected components and rho on 8192 x 8192 masks (noise at four
densities around the percolation thresholds, and the adversarial spiral,
checkerboard and rings), the 2000-node random formula at 2048 x 2048 with
4-adjacency, the MRI-shaped batch of 4096 images in one autotuned launch (a
seeded sample of its images checked one by one), and the case-study grow
spec on a 7680 x 7680 slice."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import assert_same, context, torch_cuda

pytestmark = pytest.mark.gpu

S = 8192
PATTERNS = {
    "p30": lambda: wl.bernoulli_mask(S, S, 0.30, seed=1),
    "p41": lambda: wl.bernoulli_mask(S, S, 0.41, seed=2),
    "p50": lambda: wl.bernoulli_mask(S, S, 0.50, seed=3),
    "p60": lambda: wl.bernoulli_mask(S, S, 0.60, seed=4),
    "spiral": lambda: wl.spiral_mask(S, S),
    "checker": lambda: wl.checkerboard_mask(S, S),
    "rings": lambda: wl.rings_mask(S, S),
}
_CACHE = {}


def _pattern(name):
    if name not in _CACHE:
        _CACHE.clear()
        _CACHE[name] = PATTERNS[name]()
    return _CACHE[name]


@pytest.mark.parametrize("conn", (8, 4))
@pytest.mark.parametrize("name", list(PATTERNS))
def test_ccl_8192(name, conn):
    torch = torch_cuda()
    m = _pattern(name)
    ctx = context()
    lab = torch.empty(S * S, dtype=torch.int32, device="cuda")
    ctx.ccl(ctx.mask(m), lab, conn)
    assert ctx.ccl_status() == 0, ctx.last_error()
    got = lab.cpu().numpy().reshape(S, S)
    exp, _ = oracle.ccl(m, conn)
    np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("conn", (8, 4))
@pytest.mark.parametrize("name", ["p41", "p60", "spiral", "rings"])
def test_reach_8192(name, conn):
    """rho phi1[phi2] with phi2 the pattern and phi1 sparse seeds (1e-4)."""
    torch_cuda()
    phi2 = _pattern(name)
    phi1 = wl.bernoulli_mask(S, S, 1e-4, seed=1)
    ctx = context()
    F = ctx.compile([("MASK", -1, -1, 0, 0, 0.0, 0.0), ("MASK", -1, -1, 1, 0, 0.0, 0.0),
                     ("REACH", 0, 1, 0, 0, 0.0, 0.0)], [2], conn)
    res = ctx.eval(F, [ctx.mask(phi1), ctx.mask(phi2)])
    assert res.sync() == 0, ctx.last_error()
    got = res.mask(0)
    exp = oracle.reach(phi1, phi2, conn)
    assert_same([got], [exp], f"reach {name} conn={conn}")


def test_random_formula_2048_seed1_conn4():
    torch_cuda()
    f = wl.random_dag(2000, seed=1)
    rec = wl.formula_to_records(f)
    img = wl.uniform_image(2048, 2048, seed=1)
    exp = oracle.evaluate(rec, f.roots, [img], conn=4).masks
    ctx = context()
    F = ctx.compile(rec, f.roots, 4)
    res = ctx.eval(F, [ctx.image(img)])
    assert res.sync() == 0, ctx.last_error()
    assert_same([res.mask(r) for r in range(len(f.roots))], exp, "seed 1 conn 4")


def test_random_formula_2048_seed2_batched():
    """The third seeded 2000-node formula at full size (2048 x 2048, 8-
    adjacency), in a prepared batch with the tuned tile shape, every root
    against the oracle."""
    torch = torch_cuda()
    import paper_2010_07284_gb300 as vg
    f = wl.random_dag(2000, seed=2)
    rec = wl.formula_to_records(f)
    img = wl.uniform_image(2048, 2048, seed=2)
    exp = oracle.evaluate(rec, f.roots, [img], conn=8).masks
    ctx = vg.Context()
    F = ctx.compile(rec, f.roots, 8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        im = ctx.image(img, s)
        ctx.autotune([(F, [im])], stream=s, reps=1)
        b = ctx.batch([(F, [im])], s)
        b.run(s)
        s.synchronize()
        res = b.result(0)
        assert res.sync() == 0, ctx.last_error()
        got = [res.mask(r) for r in range(len(f.roots))]
        b.close()
    assert_same(got, exp, "seed 2 conn 8")


def test_mri_batch_4096_autotuned():
    """4096 MRI-shaped images (sides 160..512, median 240, 4 channels), the
    fixed 40-primitive formula with percentile thresholds, one persistent
    launch with the autotuner's tile shape, replayed twice; 160 images
    chosen by a seeded draw are compared with the oracle, root by root."""
    torch = torch_cuda()
    import paper_2010_07284_gb300 as vg
    f = wl.config4_formula()
    rec = wl.formula_to_records(f)
    sides = wl.mri_side_lengths(4096, seed=0)
    imgs = wl.mri_phantom_batch_parallel(sides, seed=0)
    ctx = vg.Context()
    F = ctx.compile(rec, f.roots, 8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        handles = [ctx.image(im, s) for im in imgs]
        jobs = [(F, [h]) for h in handles]
        tune = ctx.autotune(jobs, stream=s, reps=1)
        assert all(t["status"] == 0 for t in tune["trials"]), tune
        assert ctx.tile_shape(jobs)["tuned"]
        b = ctx.batch(jobs, s)
        for _ in range(2):
            b.run(s)
        s.synchronize()
        pick = np.random.default_rng(5).choice(len(imgs), size=160, replace=False)
        for k in pick:
            res = b.result(int(k))
            assert res.status_word() == 0
            exp = oracle.evaluate(rec, f.roots, [imgs[k]], conn=8).masks
            assert_same([res.mask(r, s) for r in range(len(f.roots))], exp, f"image {k}")
    ctx.close()


def test_grow_spec_7680_both_forms():
    """The case-study spec of Sec. 4.2 at its timing scale: two thresholds and
    grow on a 7680 x 7680 upscaled MRI-shaped slice (about 60 Mpx)."""
    torch_cuda()
    from workloads.images import upscaled_slice
    f = wl.grow_spec_formula()
    rec = wl.formula_to_records(f)
    img = upscaled_slice(7680)
    exp = oracle.evaluate(rec, f.roots, [img], conn=8).masks[0]
    for mode in ("fused", "plain"):
        ctx = context(mode)
        F = ctx.compile(rec, f.roots, 8)
        res = ctx.eval(F, [ctx.image(img)])
        assert res.sync() == 0, ctx.last_error()
        assert_same([res.mask(0)], [exp], f"grow 7680 {mode}")


def test_ccl_8192_repeated_labellings_agree():
    """Twelve labellings of one 8192 x 8192 mask at 4-adjacency near its
    percolation threshold: every status is clean and every labelling equals
    the oracle's (a race in the tile flatten once left, in about one run in
    twenty, a run one hop short of its root and a bad index in the global
    union-find)."""
    torch = torch_cuda()
    m = wl.bernoulli_mask(S, S, 0.60, seed=4)
    exp = torch.from_numpy(oracle.ccl(m, 4)[0].ravel()).cuda()
    ctx = context()
    mimg = ctx.mask(m)
    lab = torch.empty(S * S, dtype=torch.int32, device="cuda")
    for rep in range(12):
        lab.fill_(-7)
        ctx.ccl(mimg, lab, 4)
        assert ctx.ccl_status() == 0, f"rep {rep}: {ctx.last_error()}"
        assert torch.equal(lab, exp), f"rep {rep}: labels differ"
