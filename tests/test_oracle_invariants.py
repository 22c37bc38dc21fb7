"""Algebraic invariants of the oracle's operators (seeded property tests,
CPU only).  Each property follows from the definitions of Sec. 2."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

CONNS = (4, 8)


def _masks(rng, shape, n, lo=0.05, hi=0.7):
    return [(rng.random(shape) < rng.uniform(lo, hi)).astype(np.uint8) for _ in range(n)]


def _surr(a, b, conn):
    nodes = [("MASK", -1, -1, 0, 0, 0.0, 0.0), ("MASK", -1, -1, 1, 0, 0.0, 0.0),
             ("SURROUNDED", 0, 1, 0, 0, 0.0, 0.0)]
    return oracle.evaluate(nodes, [2], masks=[a, b], conn=conn).masks[0]


@pytest.mark.parametrize("conn", CONNS)
def test_near_properties(conn):
    rng = np.random.default_rng(100 + conn)
    for shape in [(1, 1), (5, 9), (33, 17), (40, 40)]:
        a, b = _masks(rng, shape, 2)
        na, nb = oracle.near(a, conn), oracle.near(b, conn)
        assert np.all(na >= a)                                   # phi in N phi
        assert np.array_equal(oracle.near(a | b, conn), na | nb)  # additive
        assert np.all(oracle.near(a & b, conn) <= (na & nb))     # monotone
        assert not oracle.near(np.zeros(shape, np.uint8), conn).any()
        if conn == 4:                                            # cross inside square
            assert np.all(na <= oracle.near(a, 8))


@pytest.mark.parametrize("conn", CONNS)
def test_reach_properties(conn):
    rng = np.random.default_rng(200 + conn)
    for shape in [(1, 1), (1, 12), (6, 7), (30, 31)]:
        p1, p2, q1, q2 = _masks(rng, shape, 4)
        z = np.zeros(shape, np.uint8)
        one = np.ones(shape, np.uint8)
        r = oracle.reach(p1, p2, conn)
        assert np.all(oracle.near(p1, conn) <= r)                        # N phi1 inside
        assert np.array_equal(oracle.reach(p1, z, conn), oracle.near(p1, conn))
        assert not oracle.reach(z, p2, conn).any()
        assert np.array_equal(oracle.reach(p1, one, conn), one if p1.any() else z)
        assert np.all(r <= oracle.reach(p1 | q1, p2, conn))              # monotone in phi1
        assert np.all(r <= oracle.reach(p1, p2 | q2, conn))              # monotone in phi2
        assert np.all(r <= oracle.reach(r, p2, conn))


@pytest.mark.parametrize("conn", CONNS)
def test_surrounded_properties(conn):
    rng = np.random.default_rng(300 + conn)
    for shape in [(4, 4), (9, 13), (24, 24)]:
        a, b = _masks(rng, shape, 2)
        z = np.zeros(shape, np.uint8)
        one = np.ones(shape, np.uint8)
        assert np.array_equal(_surr(a, one, conn), a)       # everything is b
        assert np.array_equal(_surr(one, z, conn), one)     # nowhere to escape to
        assert np.all(_surr(a, b, conn) <= a)
        assert not _surr(z, b, conn).any()


@pytest.mark.parametrize("conn", CONNS)
def test_ccl_labels_are_consistent(conn):
    """The paper's termination predicate (Sec. 3.3): no foreground pixel has a
    foreground neighbour with another label; labels are component minima."""
    rng = np.random.default_rng(400 + conn)
    m = (rng.random((50, 60)) < 0.5).astype(np.uint8)
    lab, n = oracle.ccl(m, conn)
    H, W = m.shape
    for y in range(H):
        for x in range(W):
            if not m[y, x]:
                assert lab[y, x] == -1
                continue
            assert lab[y, x] <= y * W + x
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if conn == 4 and dy and dx:
                        continue
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W and m[yy, xx]:
                        assert lab[yy, xx] == lab[y, x]
    roots = np.unique(lab[lab >= 0])
    assert len(roots) == n
    assert all(lab.ravel()[r] == r for r in roots)
