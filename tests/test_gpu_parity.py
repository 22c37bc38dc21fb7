"""CUDA path vs the oracle, element by element, through the C ABI.  Masks
must be identical; labels identical after the canonical (minimum linear
index) naming both sides use.  Both execution forms are checked."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import (assert_same, check_formula, context, gpu_eval, shift_mask_images,
                      torch_cuda)

pytestmark = pytest.mark.gpu

CONNS = (4, 8)


def _f(op, a=-1, b=-1, image=0, channel=0, t=0.0, q=0.0):
    return (op, a, b, image, channel, t, q)


# ------------------------------------------------------------ primitives ---

@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (45, 1), (33, 129), (97, 1025), (64, 2048)])
@pytest.mark.parametrize("conn", CONNS)
def test_pointwise_and_near_chains(shape, conn):
    torch_cuda()
    img = wl.uniform_image(*shape, channels=2, seed=shape[0] * 7 + shape[1])
    nodes = [_f("THR_GT", t=0.3), _f("THR_LT", channel=1, t=0.6), _f("AND", 0, 1), _f("NOT", 2),
             _f("NEAR", 3), _f("NEAR", 4), _f("OR", 5, 0), _f("INTERIOR", 6), _f("NEAR", 0),
             _f("TRUE"), _f("FALSE"), _f("AND", 9, 7), _f("OR", 10, 8)]
    check_formula(nodes, [2, 3, 4, 5, 7, 8, 11, 12, 9, 10], [img], conn=conn)


@pytest.mark.parametrize("conn", CONNS)
def test_thresholds_are_strict(conn):
    torch_cuda()
    img = np.full((1, 20, 70), 0.5, np.float32)
    img[0, 3, 4] = np.nextafter(np.float32(0.5), np.float32(1))
    img[0, 5, 6] = np.nextafter(np.float32(0.5), np.float32(0))
    nodes = [_f("THR_GT", t=0.5), _f("THR_LT", t=0.5)]
    check_formula(nodes, [0, 1], [img], conn=conn)


@pytest.mark.parametrize("conn", CONNS)
def test_rank_thresholds_ties_signed_zeros_nan(conn):
    """Eight thresholds on one channel take the rank-code path: pixel values
    equal to thresholds, -0.0 against 0.0 and NaN pixels must give the strict
    float comparisons exactly, in fused groups with halos and plain form."""
    torch_cuda()
    ts = [0.0, -0.0, 0.25, 0.5, 0.5, 0.75, -1.0, 2.0]
    nodes = [_f("THR_GT" if k % 2 == 0 else "THR_LT", t=t) for k, t in enumerate(ts)]
    nodes += [_f("AND", 0, 3), _f("NEAR", 8), _f("OR", 9, 5), _f("NEAR", 10)]
    rng = np.random.default_rng(12)
    vals = np.array([0.0, -0.0, 0.25, 0.5, 0.75, -1.0, 2.0, 0.3, np.nan, -5.0], dtype=np.float32)
    img = rng.choice(vals, size=(1, 131, 1100)).astype(np.float32)
    check_formula(nodes, list(range(len(nodes))), [img], conn=conn)


@pytest.mark.parametrize("shape,p2", [((64, 64), 0.5), ((131, 1100), 0.45), ((300, 2100), 0.6),
                                      ((1, 3000), 0.7), ((2500, 3), 0.7)])
@pytest.mark.parametrize("conn", CONNS)
def test_reach_masks(shape, p2, conn):
    torch_cuda()
    phi1 = wl.bernoulli_mask(*shape, 0.002, seed=1)
    phi2 = wl.bernoulli_mask(*shape, p2, seed=2)
    nodes = [_f("MASK", image=0), _f("MASK", image=1), _f("REACH", 0, 1), _f("GROW", 0, 1),
             _f("SURROUNDED", 1, 0), _f("TOUCH", 1, 0)]
    check_formula(nodes, [2, 3, 4, 5], masks=[phi1, phi2], conn=conn)


@pytest.mark.parametrize("conn", CONNS)
def test_reach_degenerate_cases(conn):
    torch_cuda()
    H, W = 70, 200
    z = np.zeros((H, W), np.uint8)
    one = np.ones((H, W), np.uint8)
    p = wl.bernoulli_mask(H, W, 0.01, seed=3)
    q = wl.bernoulli_mask(H, W, 0.5, seed=4)
    for a, b in [(z, q), (p, z), (p, one), (one, one), (z, z), (one, z), (p, wl.spiral_mask(H, W))]:
        nodes = [_f("MASK", image=0), _f("MASK", image=1), _f("REACH", 0, 1)]
        check_formula(nodes, [2, 0], masks=[a, b], conn=conn)


# ------------------------------------------------------------- formulas ---

@pytest.mark.parametrize("conn", CONNS)
def test_config1_full(conn):
    """512 x 512 smoothed Gaussian field; a = I > 0.6, b = I < 0.3,
    rho(N a)[not b] and not a, surrounded(a, not b)."""
    torch_cuda()
    f = wl.config1_formula()
    img = wl.gaussian_field_image(512, 512, seed=0)
    check_formula(wl.formula_to_records(f), f.roots, [img], conn=conn)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("shape", [(96, 300), (130, 1100)])
def test_random_dags_small(seed, shape):
    torch_cuda()
    f = wl.random_dag(500, seed=seed, max_depth=100)
    img = wl.uniform_image(*shape, seed=seed)
    check_formula(wl.formula_to_records(f), f.roots, [img], conn=8 if seed % 2 == 0 else 4)


def test_sequential_formula():
    torch_cuda()
    f = wl.sequential_dag(300, seed=5)
    img = wl.uniform_image(200, 700, seed=5)
    check_formula(wl.formula_to_records(f), f.roots, [img], conn=8)


def test_config4_formula_batch_vs_single():
    """Percentile thresholds, grow, N chains, interior, surrounded, touch, on
    MRI-shaped phantoms of uneven sizes, in one batched launch."""
    torch_cuda()
    f = wl.config4_formula()
    rec = wl.formula_to_records(f)
    sides = wl.mri_side_lengths(24, seed=11)
    imgs = wl.mri_phantom_batch(sides, seed=11)
    ctx = context()
    F = ctx.compile(rec, f.roots, 8)
    handles = [ctx.image(im) for im in imgs]
    results = ctx.eval_batch([(F, [h]) for h in handles])
    for im, res in zip(imgs, results):
        assert res.sync() == 0
        exp = oracle.evaluate(rec, f.roots, [im], conn=8).masks
        assert_same([res.mask(r) for r in range(len(f.roots))], exp, "batch")


# ----------------------------------------------------- connected components

def _labels_gpu(mask, conn):
    torch = torch_cuda()
    ctx = context()
    m = ctx.mask(mask)
    lab = torch.empty(mask.size, dtype=torch.int32, device="cuda")
    ctx.ccl(m, lab, conn)
    assert ctx.ccl_status() == 0, ctx.last_error()
    return lab.cpu().numpy().reshape(mask.shape)


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("name", ["p30", "p41", "p50", "p60", "spiral", "checker", "rings"])
def test_ccl_labels_match_oracle(name, conn):
    shape = (1000, 2100)
    m = {"p30": lambda: wl.bernoulli_mask(*shape, 0.3, seed=1),
         "p41": lambda: wl.bernoulli_mask(*shape, 0.41, seed=2),
         "p50": lambda: wl.bernoulli_mask(*shape, 0.5, seed=3),
         "p60": lambda: wl.bernoulli_mask(*shape, 0.6, seed=4),
         "spiral": lambda: wl.spiral_mask(*shape),
         "checker": lambda: wl.checkerboard_mask(*shape),
         "rings": lambda: wl.rings_mask(*shape)}[name]()
    got = _labels_gpu(m, conn)
    exp, _ = oracle.ccl(m, conn)
    np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("shape", [(1, 1), (1, 5000), (5000, 1), (31, 33), (33, 1023), (64, 1025)])
def test_ccl_ragged_shapes(shape):
    for conn in CONNS:
        m = wl.bernoulli_mask(*shape, 0.55, seed=shape[1])
        np.testing.assert_array_equal(_labels_gpu(m, conn), oracle.ccl(m, conn)[0])


# --------------------------------------------------------------- failure ---

def test_timeout_status_surfaces_without_faulting():
    """Every device-side dependency wait expires at once (negative spin
    limit): the job reports VL_ERR_TIMEOUT, nothing hangs, and the context
    stays usable."""
    torch_cuda()
    import paper_2010_07284_gb300 as vg
    ctx = vg.Context(spin_limit=-1)
    f = wl.config1_formula()
    F = ctx.compile(wl.formula_to_records(f), f.roots, 8)
    res = ctx.eval(F, [ctx.image(wl.gaussian_field_image(128, 128))])
    assert res.sync() == 6  # VL_ERR_TIMEOUT
    ok = context()
    got, _ = gpu_eval(ok, wl.formula_to_records(f), f.roots, [wl.gaussian_field_image(128, 128)])
    assert len(got) == 2


def test_bad_inputs_are_rejected():
    torch_cuda()
    import paper_2010_07284_gb300 as vg
    ctx = context()
    F = ctx.compile([_f("THR_GT", t=0.5)], [0])
    a = ctx.image(np.zeros((1, 10, 10), np.float32))
    b = ctx.image(np.zeros((1, 11, 10), np.float32))
    m = ctx.mask(np.zeros((10, 10), np.uint8))
    with pytest.raises(vg.VlError):
        ctx.eval(F, [m])                       # mask where a float image is needed
    G = ctx.compile([_f("THR_GT", t=0.5), _f("THR_GT", image=1, t=0.5), _f("AND", 0, 1)], [2])
    with pytest.raises(vg.VlError):
        ctx.eval(G, [a, b])                    # shapes differ
    with pytest.raises(vg.VlError):
        ctx.eval(G, [a])                       # missing image


# ------------------------------------------------------------ full sizes ---

def test_config2_full_size_repeated_replays():
    """2048 x 2048 uniform image, 2000-node random formula, in the launch
    configuration the benchmark times (the autotuner's tile shape for this
    job): the fused batch replayed several times (graph replays reuse
    scratch memory) must keep a clean status and equal the oracle on every
    root each time."""
    torch = torch_cuda()
    import paper_2010_07284_gb300 as vg
    f = wl.random_dag(2000, seed=0)
    rec = wl.formula_to_records(f)
    img = wl.uniform_image(2048, 2048, seed=0)
    exp = oracle.evaluate(rec, f.roots, [img], conn=8).masks
    ctx = vg.Context()
    F = ctx.compile(rec, f.roots, 8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        im = ctx.image(img, s)
        tune = ctx.autotune([(F, [im])], stream=s, reps=1)
        assert all(t["status"] == 0 for t in tune["trials"]), tune
        assert ctx.tile_shape([(F, [im])])["tuned"]
        b = ctx.batch([(F, [im])], s)
        for k in range(3):
            b.run(s)
            s.synchronize()
            res = b.result(0)
            assert res.status_word() == 0
            words = np.empty((len(f.roots), 2048, 2048 // 32), dtype=np.uint32)
            res.masks_into(words, on_device=False, stream=s)
            got = np.unpackbits(words.view(np.uint8), axis=-1, bitorder="little")
            for r in range(len(f.roots)):
                if not np.array_equal(got[r], exp[r]):
                    raise AssertionError(f"replay {k} root {r} differs")
        plain = ctx.eval(F, [im], stream=s, mode="plain")
        assert plain.sync() == 0
        for r in range(0, len(f.roots), 50):
            assert np.array_equal(plain.mask(r, s), exp[r])


@pytest.mark.parametrize("shape", [(65535, 40), (40, 65535)])
def test_longest_sides(shape):
    """Sides at the 65535 limit: labelling tiles, group tiles and the last
    padded word of a row all at their edges; a formula with N, rho, grow and
    a uint16 threshold, and a full labelling."""
    torch = torch_cuda()
    img = wl.uniform_image_u16(*shape, seed=3)
    nodes = [_f("THR_GT", t=60000.0), _f("THR_LT", t=20000.0), _f("NEAR", 0), _f("REACH", 0, 1),
             _f("GROW", 1, 0), _f("AND", 3, 4), _f("NOT", 5)]
    check_formula(nodes, [2, 3, 4, 6], [img], conn=8)
    m = wl.bernoulli_mask(*shape, 0.55, seed=4)
    ctx = context()
    lab = torch.empty(m.size, dtype=torch.int32, device="cuda")
    ctx.ccl(ctx.mask(m), lab, 4)
    assert ctx.ccl_status() == 0
    np.testing.assert_array_equal(lab.cpu().numpy().reshape(shape), oracle.ccl(m, 4)[0])


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["fused", "plain"])
def test_specification_text_on_the_gpu(mode):
    """A specification text (vl_formula_compile_text) evaluated through the
    CUDA path equals the oracle on the node formula it spells out."""
    torch_cuda()
    ctx = context(mode)
    src = """
    load a = "a"
    load b = "b"
    let band(x, lo, hi) = intensity(x) >. lo & intensity(x) <. hi
    let core = band(a, 0.6, 0.95)
    save "grown" grow(core, band(b, 0.2, 0.9))
    save "edge" N(core) & !core | touch(core, intensity(b) >. percentile(intensity(b), 0.8))
    """
    F = ctx.compile_text(src, 8)
    assert F.loads == ["a", "b"] and F.saves == ["grown", "edge"]
    ims = [wl.gaussian_field_image(200, 300, seed=11), wl.gaussian_field_image(200, 300, seed=12)]
    res = ctx.eval(F, [ctx.image(im) for im in ims])
    assert res.sync() == 0, ctx.last_error()
    got = [res.mask(r) for r in range(2)]
    N = lambda op, a=-1, b=-1, image=0, t=0.0, q=0.0: (op, a, b, image, 0, float(np.float32(t)), q)
    nodes = [N("THR_GT", image=0, t=0.6), N("THR_LT", image=0, t=0.95), N("AND", 0, 1),
             N("THR_GT", image=1, t=0.2), N("THR_LT", image=1, t=0.9), N("AND", 3, 4),
             N("GROW", 2, 5), N("NEAR", 2), N("NOT", 2), N("AND", 7, 8),
             N("PCT_GT", image=1, q=0.8), N("TOUCH", 2, 10), N("OR", 9, 11)]
    exp = oracle.evaluate(nodes, [6, 12], ims, conn=8).masks
    assert_same(got, exp, mode)


@pytest.mark.gpu
def test_command_line_runs_a_specification_file(tmp_path):
    """`python -m paper_2010_07284_gb300 SPEC`: loads read NumPy files, saves
    write the masks; the result equals the oracle."""
    torch_cuda()
    from paper_2010_07284_gb300.__main__ import run
    img = wl.gaussian_field_image(64, 96, seed=3)
    roi = np.random.default_rng(0).random((64, 96)) < 0.3
    np.save(tmp_path / "scan.npy", img)
    np.save(tmp_path / "roi.npy", roi)
    (tmp_path / "spec.imgql").write_text(
        'load scan = "scan.npy"\nload roi = "roi.npy"\n'
        'let hot = intensity(scan) >. 0.6\nsave "out.npy" grow(hot, mask(roi) | hot)\n')
    written = run(str(tmp_path / "spec.imgql"))
    got = np.load(written[0])
    nodes = [("THR_GT", -1, -1, 0, 0, float(np.float32(0.6)), 0.0), ("MASK", -1, -1, 0, 0, 0.0, 0.0),
             ("OR", 1, 0, 0, 0, 0.0, 0.0), ("GROW", 0, 2, 0, 0, 0.0, 0.0)]
    exp = oracle.evaluate(nodes, [3], [img], [roi], conn=8).masks[0]
    assert got.dtype == np.bool_ and np.array_equal(got.astype(np.uint8), exp)
