"""Seeded fuzzing of the compiler: random formulas mixing every operator the
C ABI accepts -- constants, mask atoms, thresholds and percentiles on
channels and on number terms, + - * /, not, and, or, N, rho, interior,
surrounded, grow, touch -- with roots of every kind, compiled and run
through the tile-accurate plan simulator (in listed and in random
dependency-respecting step orders) against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import plan_sim
import paper_2010_07284_gb300 as vg

BOOL_UNARY = ("NOT", "NEAR", "INTERIOR")
BOOL_BINARY = ("AND", "OR", "REACH", "SURROUNDED", "GROW", "TOUCH")
ARITH = ("ADD", "SUB", "MUL", "DIV")


def random_formula(rng, n_nodes, n_channels, with_mask):
    """Records (op, a, b, image, channel, t, q) and roots.  Image 0 is a
    number image with n_channels channels; image 1 a mask when with_mask."""
    recs, kind = [], []   # kind: "b" mask-valued, "n" number term

    def pick(k):
        idx = [i for i, x in enumerate(kind) if x == k]
        if not idx:
            return None
        # recent nodes more often, any earlier node sometimes
        return idx[-1 - int(rng.integers(0, min(4, len(idx))))] if rng.random() < 0.7 \
            else idx[int(rng.integers(0, len(idx)))]

    while len(recs) < n_nodes:
        r = rng.random()
        ch = int(rng.integers(0, n_channels))
        if r < 0.08:
            recs.append(("VALUE", -1, -1, 0, ch, 0.0, 0.0)); kind.append("n")
        elif r < 0.16 and pick("n") is not None:
            a = pick("n")
            op = ARITH[int(rng.integers(0, 4))]
            if rng.random() < 0.4:
                recs.append((op, a, -1, 0, 0, float(np.float32(rng.uniform(-1.5, 1.5) or 0.5)), 0.0))
            else:
                recs.append((op, a, pick("n"), 0, 0, 0.0, 0.0))
            kind.append("n")
        elif r < 0.30:
            n_src = pick("n") if rng.random() < 0.3 else None
            if rng.random() < 0.5:
                op = "THR_GT" if rng.random() < 0.5 else "THR_LT"
                t = 0.0 if n_src is not None else float(np.float32(rng.random()))
                recs.append((op, -1 if n_src is None else n_src, -1, 0, ch, t, 0.0))
            else:
                op = "PCT_GT" if rng.random() < 0.5 else "PCT_LT"
                q = float(rng.choice([0.0, 0.1, 0.5, 0.9, 1.0]))
                recs.append((op, -1 if n_src is None else n_src, -1, 0, ch, 0.0, q))
            kind.append("b")
        elif r < 0.33:
            recs.append(("TRUE" if rng.random() < 0.5 else "FALSE", -1, -1, 0, 0, 0.0, 0.0))
            kind.append("b")
        elif r < 0.37 and with_mask:
            recs.append(("MASK", -1, -1, 1, 0, 0.0, 0.0)); kind.append("b")
        elif pick("b") is not None:
            if rng.random() < 0.45:
                recs.append((BOOL_UNARY[int(rng.integers(0, 3))], pick("b"), -1, 0, 0, 0.0, 0.0))
            else:
                op = BOOL_BINARY[int(rng.choice(6, p=(0.3, 0.2, 0.2, 0.1, 0.1, 0.1)))]
                recs.append((op, pick("b"), pick("b"), 0, 0, 0.0, 0.0))
            kind.append("b")
    masks = [i for i, k in enumerate(kind) if k == "b"]
    if not masks:
        recs.append(("TRUE", -1, -1, 0, 0, 0.0, 0.0)); kind.append("b")
        masks = [len(recs) - 1]
    n_roots = int(rng.integers(1, min(6, len(masks)) + 1))
    roots = [int(x) for x in rng.choice(masks, size=n_roots, replace=True)]
    return recs, roots


@pytest.mark.parametrize("seed", range(int(__import__("os").environ.get("VL_FUZZ_SEEDS", "100"))))
def test_random_formulas_plan_matches_oracle(seed):
    pytest.importorskip("scipy")
    rng = np.random.default_rng(1000 + seed)
    n_channels = int(rng.integers(1, 3))
    with_mask = seed % 3 == 0
    recs, roots = random_formula(rng, int(rng.integers(5, 90)), n_channels, with_mask)
    H, W = int(rng.integers(1, 45)), int(rng.integers(1, 300))
    conn = 8 if seed % 2 == 0 else 4
    img = rng.random((n_channels, H, W)).astype(np.float32)
    if seed % 5 == 0:
        img = (img * 65535).astype(np.uint16)
    masks = {1: rng.random((H, W)) < 0.4} if with_mask else {}
    # the oracle keeps masks in a list of their own (the mask is its mask
    # 0); the C ABI reads one image list (number image 0, the mask image 1)
    recs_o = [(op, a, b, (0 if op == "MASK" else im), ch, t, q)
              for (op, a, b, im, ch, t, q) in recs]
    exp = oracle.evaluate(recs_o, roots, [img], [masks[1]] if with_mask else [], conn=conn).masks
    F = vg.compile_formula(recs, roots, conn)
    plan = F.plan()
    images = [img, None] if with_mask else [img]
    for order_seed in (None, seed):
        order = plan_sim.random_topological_order(plan, order_seed) if order_seed is not None else None
        got = plan_sim.simulate(plan, images, masks, conn, seed=seed, order=order)
        for r, (g, e) in enumerate(zip(got, exp)):
            assert np.array_equal(g.astype(np.uint8), e), f"seed {seed} root {r} order {order_seed}"
