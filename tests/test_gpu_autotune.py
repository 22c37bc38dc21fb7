"""Tile shapes and the autotuner: every tile shape gives the oracle's masks;
the autotuner times every candidate cleanly, keeps the fastest, and later
batches of the same signature take it (also after a save and a load)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import assert_same, check_formula, context, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rows,words", [(16, 8), (32, 16), (64, 16), (16, 32), (7, 3)])
def test_fixed_tile_shapes_match_oracle(rows, words):
    torch_cuda()
    f = wl.random_dag(400, seed=rows + words, max_depth=80)
    img = wl.uniform_image(131, 1100, seed=3)
    ctx = context(tile_rows=rows, tile_words=words)
    check_formula(wl.formula_to_records(f), f.roots, [img], conn=8, ctx=ctx)


def _jobs(ctx, n_images=3, side=(300, 700), seed=0):
    f = wl.random_dag(300, seed=seed, max_depth=60)
    rec = wl.formula_to_records(f)
    F = ctx.compile(rec, f.roots, 8)
    imgs = [wl.uniform_image(side[0] + 7 * k, side[1] - 5 * k, seed=seed + k) for k in range(n_images)]
    handles = [ctx.image(im) for im in imgs]
    return f, rec, F, imgs, handles


def test_autotune_picks_the_fastest_and_later_batches_use_it(tmp_path):
    torch = torch_cuda()
    import paper_2010_07284_gb300 as vg
    ctx = vg.Context()
    f, rec, F, imgs, handles = _jobs(ctx)
    jobs = [(F, [h]) for h in handles]
    before = ctx.tile_shape(jobs)
    assert not before["tuned"]
    s = torch.cuda.Stream()
    out = ctx.autotune(jobs, stream=s, reps=2)
    trials = out["trials"]
    assert len(trials) >= 8
    for t in trials:
        assert t["status"] == 0, f"candidate {t} failed: {ctx.last_error()}"
        assert t["ms"] > 0
    best = out["best"]
    assert best["ms"] == pytest.approx(min(t["ms"] for t in trials))
    now = ctx.tile_shape(jobs)
    assert now["tuned"]
    assert (now["tile_rows"], now["tile_words"], now["ctas_per_sm"]) == \
        (best["tile_rows"], best["tile_words"], best["ctas_per_sm"])
    # the tuned batch still gives the oracle's masks
    results = ctx.eval_batch(jobs)
    for im, res in zip(imgs, results):
        assert res.sync() == 0
        exp = oracle.evaluate(rec, f.roots, [im], conn=8).masks
        assert_same([res.mask(r) for r in range(len(f.roots))], exp, "tuned")
    # the table survives a save and a load into a fresh context
    path = tmp_path / "tiles.txt"
    ctx.save_tuning(path)
    ctx2 = vg.Context()
    F2 = ctx2.compile(rec, f.roots, 8)
    handles2 = [ctx2.image(im) for im in imgs]
    jobs2 = [(F2, [h]) for h in handles2]
    assert not ctx2.tile_shape(jobs2)["tuned"]
    ctx2.load_tuning(path)
    got = ctx2.tile_shape(jobs2)
    assert got["tuned"] and (got["tile_rows"], got["tile_words"]) == (best["tile_rows"], best["tile_words"])
    ctx2.close()
    ctx.close()


def test_fixed_shape_context_refuses_autotune_and_bad_tables(tmp_path):
    torch_cuda()
    import paper_2010_07284_gb300 as vg
    ctx = context(tile_rows=32, tile_words=16)
    f, rec, F, imgs, handles = _jobs(ctx, n_images=1)
    jobs = [(F, [handles[0]])]
    assert ctx.tile_shape(jobs)["tile_words"] == 16
    with pytest.raises(vg.VlError):
        ctx.autotune(jobs)
    bad = tmp_path / "bad.txt"
    bad.write_text("not a table\n")
    with pytest.raises(vg.VlError):
        ctx.load_tuning(bad)
    with pytest.raises(vg.VlError):
        vg.Context(tile_rows=32, tile_words=0)


def test_one_job_batches_can_take_the_per_operator_form(tmp_path):
    """A batch of one job whose formula is tiny takes the per-operator form
    (reported as a 0 x 0 tile); the autotuner tries that form for every
    batch of one job; both forms, replayed, give the oracle's masks; a
    saved table keeps the per-operator choice."""
    torch = torch_cuda()
    import paper_2010_07284_gb300 as vg
    ctx = vg.Context()
    img = wl.gaussian_field_image(300, 700, seed=2)
    h = ctx.image(img)
    tiny = wl.config1_formula()
    F = ctx.compile(wl.formula_to_records(tiny), tiny.roots, 8)
    assert ctx.tile_shape([(F, [h])])["tile_rows"] == 0
    exp = oracle.evaluate(wl.formula_to_records(tiny), tiny.roots, [img], conn=8).masks
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = ctx.batch([(F, [h])], stream)
        for _ in range(3):
            b.run(stream)
        stream.synchronize()
        r = b.result(0)
        assert r.sync() == 0
        assert_same([r.mask(k) for k in range(len(tiny.roots))], exp, "per-operator batch")
        b.close()
    big = wl.sequential_dag(200, seed=4, mix="reach")
    G = ctx.compile(wl.formula_to_records(big), big.roots, 8)
    with torch.cuda.stream(stream):
        tune = ctx.autotune([(G, [h])], stream=stream, reps=1)
        assert any(t["tile_rows"] == 0 and t["status"] == 0 for t in tune["trials"])
        b = ctx.batch([(G, [h])], stream)
        for _ in range(2):
            b.run(stream)
        stream.synchronize()
        r = b.result(0)
        assert r.sync() == 0
        got = [r.mask(k) for k in range(len(big.roots))]
        b.close()
    exp = oracle.evaluate(wl.formula_to_records(big), big.roots, [img], conn=8).masks
    assert_same(got, exp, f"tuned batch ({tune['best']})")
    path = str(tmp_path / "tiles.txt")
    ctx.save_tuning(path)
    ctx2 = vg.Context()
    ctx2.load_tuning(path)
    G2 = ctx2.compile(wl.formula_to_records(big), big.roots, 8)
    h2 = ctx2.image(img)
    assert ctx2.tile_shape([(G2, [h2])])["tile_rows"] == tune["best"]["tile_rows"]
