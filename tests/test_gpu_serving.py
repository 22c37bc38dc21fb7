"""Serving loop: queries admitted while others run on the GPU give exactly
the masks they give alone; cancellation, rejection and a tight memory budget
leave the other queries untouched."""
from __future__ import annotations

import time

import numpy as np
import pytest

import workloads as wl
from gpu_util import context, torch_cuda

pytestmark = pytest.mark.gpu


def _pool(ctx, n=6, seed=0):
    rng = np.random.default_rng(seed)
    sides = [int(s) for s in rng.integers(96, 700, size=n)]
    imgs = [wl.uniform_image(s, s + int(rng.integers(0, 300)), seed=seed + k) for k, s in enumerate(sides)]
    return [ctx.image(im) for im in imgs]


def _queries(ctx, handles, n, seed=0):
    rng = np.random.default_rng(seed)
    qs = []
    for k in range(n):
        size = int(np.exp(rng.uniform(np.log(10), np.log(300))))
        f = wl.random_dag(size, seed=seed * 1000 + k, max_depth=min(500, size))
        F = ctx.compile(wl.formula_to_records(f), f.roots, 8 if k % 3 else 4)
        qs.append((F, handles[int(rng.integers(0, len(handles)))], len(f.roots)))
    return qs


def _alone(ctx, F, img, n_roots):
    r = ctx.eval(F, [img])
    assert r.sync() == 0
    return [r.mask(q) for q in range(n_roots)]


def test_results_in_the_mix_equal_results_alone():
    torch_cuda()
    import paper_2010_07284_gb300 as vg
    ctx = context()
    handles = _pool(ctx, seed=1)
    qs = _queries(ctx, handles, 40, seed=1)
    srv = vg.Server(ctx, max_inflight_batches=3, max_batch_jobs=8, batch_window_us=100)
    tickets = []
    for k, (F, img, _) in enumerate(qs):
        tickets.append(srv.submit(F, [img]))
        if k % 10 == 9:
            time.sleep(0.002)   # let earlier batches start: later ones join the mix
    for (F, img, nr), t in zip(qs, tickets):
        st, res = srv.wait(t, timeout_us=60_000_000)
        assert st == 0, f"ticket {t}: status {st}"
        got = [res.mask(q) for q in range(nr)]
        exp = _alone(ctx, F, img, nr)
        for g, e in zip(got, exp):
            assert np.array_equal(g, e)
    stats = srv.stats()
    assert stats["completed"] == len(qs)
    assert stats["batches"] >= 2
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    srv.close()


def test_cancel_reject_and_tight_budget():
    torch_cuda()
    import paper_2010_07284_gb300 as vg
    ctx = context()
    handles = _pool(ctx, n=3, seed=2)
    qs = _queries(ctx, handles, 24, seed=2)
    # a budget of one byte: only one query is admitted at a time, the rest queue
    srv = vg.Server(ctx, max_inflight_batches=2, max_batch_jobs=4, memory_budget=1,
                    batch_window_us=0)
    tickets = [srv.submit(F, [img]) for F, img, _ in qs]
    cancelled = set()
    for t in tickets[-6:]:
        if srv.cancel(t) == 0:
            cancelled.add(t)
    bad = ctx.compile([("THR_GT", -1, -1, 0, 0, 0.5, 0), ("THR_GT", -1, -1, 1, 0, 0.5, 0),
                       ("AND", 0, 1, 0, 0, 0, 0)], [2])
    with pytest.raises(vg.VlError):
        srv.submit(bad, [handles[0], handles[1]])   # images of different shapes
    for (F, img, nr), t in zip(qs, tickets):
        st, res = srv.wait(t, timeout_us=60_000_000)
        if t in cancelled:
            assert st == 9  # VL_ERR_CANCELLED
            continue
        assert st == 0
        exp = _alone(ctx, F, img, nr)
        for q in range(nr):
            assert np.array_equal(res.mask(q), exp[q])
    stats = srv.stats()
    assert stats["cancelled"] == len(cancelled)
    assert stats["completed"] == len(qs) - len(cancelled)
    srv.close()


def test_serving_mixes_number_terms_and_uint16_images():
    """Queries with number terms on float and uint16 images served in one
    mix equal the oracle's masks."""
    torch_cuda()
    import oracle
    import paper_2010_07284_gb300 as vg
    ctx = context()
    imgs = []
    for k in range(4):
        im = np.stack([wl.gaussian_field_image(150 + 40 * k, 300 + 70 * k, seed=k)[0],
                       wl.uniform_image(150 + 40 * k, 300 + 70 * k, seed=k)[0]])
        imgs.append(wl.to_u16(np.clip(im, 0.0, 1.0)) if k % 2 else im)
    handles = [ctx.image(im) for im in imgs]
    srv = vg.Server(ctx, max_inflight_batches=2, max_batch_jobs=4, batch_window_us=100)
    jobs = []
    for k in range(12):
        f = wl.arith_dag(50, seed=40 + k)
        rec = wl.formula_to_records(f)
        F = ctx.compile(rec, f.roots, 8)
        j = k % len(imgs)
        jobs.append((rec, f.roots, j, srv.submit(F, [handles[j]])))
    for rec, roots, j, t in jobs:
        st, res = srv.wait(t, timeout_us=60_000_000)
        assert st == 0, f"ticket {t}: status {st}"
        exp = oracle.evaluate(rec, roots, [imgs[j]], conn=8).masks
        for r, e in enumerate(exp):
            assert np.array_equal(res.mask(r), e), f"ticket {t} root {r}"
    srv.close()


def test_large_queries_in_the_mix_match_the_oracle():
    """Queries at the large end of the serving stream -- 2048 x 2048 and
    2304 x 2048 images with formulas of 1000 and more nodes -- submitted
    while a burst of small queries is in flight, checked against the CPU
    oracle root by root; a seeded sample of the small ones too."""
    torch_cuda()
    import oracle
    import paper_2010_07284_gb300 as vg
    ctx = context()
    rng = np.random.default_rng(77)
    small_imgs = [wl.uniform_image(int(s), int(s) + 40, seed=500 + k)
                  for k, s in enumerate(rng.integers(128, 600, size=5))]
    small_h = [ctx.image(im) for im in small_imgs]
    big_imgs = [wl.uniform_image(2048, 2048, seed=601), wl.uniform_image(2304, 2048, seed=602)]
    big_h = [ctx.image(im) for im in big_imgs]
    big_f = [wl.random_dag(1000, seed=611, max_depth=500), wl.random_dag(1400, seed=612, max_depth=500)]
    big_F = [ctx.compile(wl.formula_to_records(f), f.roots, 8) for f in big_f]
    small = []
    for k in range(30):
        n = int(np.exp(rng.uniform(np.log(10), np.log(400))))
        f = wl.random_dag(n, seed=700 + k, max_depth=min(500, n))
        small.append((f, ctx.compile(wl.formula_to_records(f), f.roots, 8), int(rng.integers(0, 5))))
    srv = vg.Server(ctx, max_inflight_batches=3, max_batch_jobs=16, batch_window_us=100)
    tickets = []
    for k, (f, F, i) in enumerate(small):
        tickets.append(("small", k, srv.submit(F, [small_h[i]])))
        if k == 10:
            for j in range(2):
                tickets.append(("big", j, srv.submit(big_F[j], [big_h[j]])))
    got = {}
    for kind, k, t in tickets:
        st, res = srv.wait(t, timeout_us=120_000_000)
        assert st == 0, f"{kind} {k}: status {st}"
        nr = len((big_f[k] if kind == "big" else small[k][0]).roots)
        got[(kind, k)] = [res.mask(q) for q in range(nr)]
        res.close()
    srv.close()
    for j in range(2):
        f = big_f[j]
        exp = oracle.evaluate(wl.formula_to_records(f), f.roots, [big_imgs[j]], conn=8).masks
        for r, (g, e) in enumerate(zip(got[("big", j)], exp)):
            assert np.array_equal(g, e), f"large query {j} root {r}"
    for k in np.random.default_rng(5).choice(len(small), size=8, replace=False):
        f, _, i = small[int(k)]
        exp = oracle.evaluate(wl.formula_to_records(f), f.roots, [small_imgs[i]], conn=8).masks
        for r, (g, e) in enumerate(zip(got[("small", int(k))], exp)):
            assert np.array_equal(g, e), f"small query {k} root {r}"
