"""The compiler fuzz formulas (every operator of the ABI, constants, mask
atoms, percentiles and number terms, roots of every kind) evaluated on the
GPU, fused and plain, against the oracle on float32 and uint16 images."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import assert_same, context, torch_cuda
from test_compiler_fuzz import random_formula

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(int(__import__("os").environ.get("VL_GPU_FUZZ_SEEDS", "60"))))
def test_random_formulas_on_the_gpu(seed):
    torch_cuda()
    rng = np.random.default_rng(5000 + seed)
    n_channels = int(rng.integers(1, 3))
    with_mask = seed % 3 == 0
    recs, roots = random_formula(rng, int(rng.integers(5, 120)), n_channels, with_mask)
    H, W = int(rng.integers(1, 90)), int(rng.integers(1, 700))
    conn = 8 if seed % 2 == 0 else 4
    img = rng.random((n_channels, H, W)).astype(np.float32)
    if seed % 4 == 1:
        img = (img * 65535).astype(np.uint16)
    mask = rng.random((H, W)) < 0.4
    recs_o = [(op, a, b, (0 if op == "MASK" else im), ch, t, q)
              for (op, a, b, im, ch, t, q) in recs]
    exp = oracle.evaluate(recs_o, roots, [img], [mask] if with_mask else [], conn=conn).masks
    ctx = context()
    F = ctx.compile(recs, roots, conn)
    ims = [ctx.image(img)] + ([ctx.mask(mask)] if with_mask else [])
    for mode in ("fused", "plain"):
        res = ctx.eval(F, ims, mode=mode)
        assert res.sync() == 0, ctx.last_error()
        assert_same([res.mask(r) for r in range(len(roots))], exp, f"seed {seed} {mode}")


@pytest.mark.parametrize("batch", range(int(__import__("os").environ.get("VL_GPU_FUZZ_BATCHES", "6"))))
def test_random_formula_batches_in_one_launch(batch):
    """Twelve fuzz jobs of different formulas, image sizes, formats and
    adjacencies in one persistent launch (and replayed), against the
    oracle."""
    torch_cuda()
    rng = np.random.default_rng(9000 + batch)
    ctx = context()
    jobs, expect = [], []
    for k in range(12):
        n_channels = int(rng.integers(1, 3))
        with_mask = rng.random() < 0.3
        recs, roots = random_formula(rng, int(rng.integers(5, 150)), n_channels, with_mask)
        H, W = int(rng.integers(1, 300)), int(rng.integers(1, 900))
        conn = 8 if rng.random() < 0.5 else 4
        img = rng.random((n_channels, H, W)).astype(np.float32)
        if rng.random() < 0.3:
            img = (img * 65535).astype(np.uint16)
        mask = rng.random((H, W)) < 0.4
        recs_o = [(op, a, b, (0 if op == "MASK" else im), ch, t, q)
                  for (op, a, b, im, ch, t, q) in recs]
        expect.append(oracle.evaluate(recs_o, roots, [img], [mask] if with_mask else [],
                                      conn=conn).masks)
        F = ctx.compile(recs, roots, conn)
        jobs.append((F, [ctx.image(img)] + ([ctx.mask(mask)] if with_mask else [])))
    b = ctx.batch(jobs)
    for _ in range(2):
        b.run()
        for k, exp in enumerate(expect):
            res = b.result(k)
            assert res.status_word() == 0, ctx.last_error()
            assert_same([res.mask(r) for r in range(len(exp))], exp, f"batch {batch} job {k}")
    b.close()


def test_random_formula_queries_through_the_server():
    """Forty fuzz queries (formulas, sizes, formats, adjacencies) submitted
    to the serving loop in bursts, so that later ones join batches in
    flight; every result equals the oracle's."""
    torch_cuda()
    import time
    import paper_2010_07284_gb300 as vg
    rng = np.random.default_rng(777)
    ctx = context()
    srv = vg.Server(ctx, max_inflight_batches=3, max_batch_jobs=8, batch_window_us=100)
    pending = []
    for k in range(40):
        n_channels = int(rng.integers(1, 3))
        with_mask = rng.random() < 0.3
        recs, roots = random_formula(rng, int(rng.integers(5, 150)), n_channels, with_mask)
        H, W = int(rng.integers(1, 260)), int(rng.integers(1, 800))
        conn = 8 if rng.random() < 0.5 else 4
        img = rng.random((n_channels, H, W)).astype(np.float32)
        if rng.random() < 0.3:
            img = (img * 65535).astype(np.uint16)
        mask = rng.random((H, W)) < 0.4
        recs_o = [(op, a, b, (0 if op == "MASK" else im), ch, t, q)
                  for (op, a, b, im, ch, t, q) in recs]
        exp = oracle.evaluate(recs_o, roots, [img], [mask] if with_mask else [], conn=conn).masks
        F = ctx.compile(recs, roots, conn)
        ims = [ctx.image(img)] + ([ctx.mask(mask)] if with_mask else [])
        pending.append((srv.submit(F, ims), exp, F, ims))
        if k % 8 == 7:
            time.sleep(0.002)
    for t, exp, F, ims in pending:
        st, res = srv.wait(t, timeout_us=60_000_000)
        assert st == 0, f"ticket {t}: status {st}"
        assert_same([res.mask(r) for r in range(len(exp))], exp, f"ticket {t}")
    srv.close()
