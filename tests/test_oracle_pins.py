"""Pins of the CPU oracle against things other than itself: hand-worked
fixtures, brute-force path enumeration, relation algebra, textbook routines
and library special cases.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import brute
import golden_io
import workloads as wl

CONNS = (4, 8)


def _f(op, a=-1, b=-1, image=0, channel=0, t=0.0, q=0.0):
    return (op, a, b, image, channel, t, q)


def _eval_binary(op, phi1, phi2, conn):
    nodes = [_f("MASK", image=0), _f("MASK", image=1), _f(op, 0, 1)]
    return oracle.evaluate(nodes, [2], masks=[phi1, phi2], conn=conn).masks[0]


# ------------------------------------------------------------ fixtures ---

@pytest.mark.parametrize("fx", golden_io.all_fixtures(), ids=lambda f: f["path"].split("/")[-1])
def test_golden_fixture(fx):
    op = fx["op"]
    if op == "near":
        for conn, exp in fx["expect"].items():
            np.testing.assert_array_equal(oracle.near(fx["phi"], conn), exp)
    elif op == "reach":
        for conn, exp in fx["expect"].items():
            np.testing.assert_array_equal(oracle.reach(fx["phi1"], fx["phi2"], conn), exp)
    elif op in ("surrounded", "grow", "touch"):
        for conn, exp in fx["expect"].items():
            got = _eval_binary(op.upper(), fx["phi1"], fx["phi2"], conn)
            np.testing.assert_array_equal(got, exp)
    elif op == "ccl":
        for conn, exp in fx["expect"].items():
            lab, _ = oracle.ccl(fx["phi"], conn)
            np.testing.assert_array_equal(lab, exp)
    elif op == "percentile":
        vals = np.array([float(v) for v in fx["kv"][0][1:]], dtype=np.float32)
        for _, q, want in fx["kv"][1:]:
            assert oracle.percentile(vals, float(q)) == float(want)
    elif op == "constants":
        scale = float(fx["kv"][0][1])
        for _, frac, want in fx["kv"][1:]:
            assert round(float(frac) * scale) == int(want)
        spec = wl.grow_spec_formula()
        assert np.float32(spec.nodes[0].t) == np.float32(62258.0 / 65535.0)
        assert np.float32(spec.nodes[1].t) == np.float32(56360.0 / 65535.0)
    elif op == "spec_u16":
        img = fx["image"].astype(np.uint16)[None]
        spec = wl.grow_spec_u16_formula()
        for conn, exp in fx["expect"].items():
            got = oracle.evaluate(wl.formula_to_records(spec), spec.roots, [img], conn=conn).masks[0]
            np.testing.assert_array_equal(got, exp)
    else:
        raise AssertionError(f"unknown fixture op {op}")


# -------------------------------------------------- atoms and booleans ---

def test_threshold_matches_numpy_strict():
    rng = np.random.default_rng(1)
    ch = rng.random((37, 53), dtype=np.float32)
    t = np.float32(0.5)
    ch[3, 4] = t                       # ties must be false both ways
    ch[0, 0] = np.nextafter(t, np.float32(1))
    np.testing.assert_array_equal(oracle.threshold(ch, t, True), (ch > t).astype(np.uint8))
    np.testing.assert_array_equal(oracle.threshold(ch, t, False), (ch < t).astype(np.uint8))
    assert oracle.threshold(ch, t, True)[3, 4] == 0
    assert oracle.threshold(ch, t, False)[3, 4] == 0


def test_boolean_ops_match_numpy():
    rng = np.random.default_rng(2)
    a = rng.random((17, 29)) < 0.5
    b = rng.random((17, 29)) < 0.3
    np.testing.assert_array_equal(oracle.op_not(a), (~a).astype(np.uint8))
    np.testing.assert_array_equal(oracle.op_and(a, b), (a & b).astype(np.uint8))


# ---------------------------------------------------------------- near ---

@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (2, 2), (13, 31), (64, 70)])
def test_near_matches_scipy_dilation(conn, shape):
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(shape[0] * 100 + shape[1] + conn)
    for p in (0.02, 0.2, 0.6):
        m = (rng.random(shape) < p).astype(np.uint8)
        st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
        exp = nd.binary_dilation(m, structure=st, border_value=0).astype(np.uint8)
        np.testing.assert_array_equal(oracle.near(m, conn), exp)


# --------------------------------------------------------------- reach ---

def _tile_batch(phi1_list, phi2, h, w, gap=2):
    """Place many (phi1, phi2) cases in one image, separated by gaps where
    phi1 and phi2 are both false: no phi2 path crosses a gap, so each tile is
    evaluated as if alone (clipping included, since gap pixels are neither
    endpoints nor intermediates)."""
    n = len(phi1_list)
    cols = int(np.ceil(np.sqrt(n)))
    rows = int(np.ceil(n / cols))
    P1 = np.zeros((rows * (h + gap), cols * (w + gap)), np.uint8)
    P2 = np.zeros_like(P1)
    coords = []
    for k, m in enumerate(phi1_list):
        r, c = divmod(k, cols)
        y, x = r * (h + gap), c * (w + gap)
        P1[y:y + h, x:x + w] = m
        P2[y:y + h, x:x + w] = phi2
        coords.append((y, x))
    return P1, P2, coords


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("shape", [(3, 3), (2, 4)])
def test_reach_exhaustive_against_simple_paths(conn, shape):
    """Every (phi1, phi2) pair on a 3x3 (2^18 pairs) and 2x4 (2^16) grid
    against the definition: a simple path from x to a phi1 pixel whose
    intermediate pixels all satisfy phi2."""
    H, W = shape
    n = H * W
    table = brute.simple_path_table(H, W, conn)
    phi1_all = [brute.bits_to_mask(b, H, W) for b in range(1 << n)]
    F1 = np.array([m.ravel() for m in phi1_all], dtype=np.uint8)      # (2^n, n)
    for b2 in range(1 << n):
        phi2 = brute.bits_to_mask(b2, H, W)
        rel = brute.reach_relation(table, n, b2)                       # (n, n)
        exp = (F1.astype(bool) | ((F1 @ rel.T.astype(np.uint8)) > 0)).astype(np.uint8)
        P1, P2, coords = _tile_batch(phi1_all, phi2, H, W)
        got = oracle.reach(P1, P2, conn)
        for k, (y, x) in enumerate(coords):
            g = got[y:y + H, x:x + W].ravel()
            if not np.array_equal(g, exp[k]):
                raise AssertionError(f"conn={conn} phi1={k:#x} phi2={b2:#x}: {g} != {exp[k]}")


@pytest.mark.parametrize("conn", CONNS)
def test_reach_random_small_against_dfs_and_matrix(conn):
    rng = np.random.default_rng(10 + conn)
    for shape in [(4, 4)] * 60 + [(5, 5)] * 25 + [(3, 7)] * 20:
        p1 = rng.uniform(0.03, 0.3)
        p2 = rng.uniform(0.2, 0.7)
        phi1 = (rng.random(shape) < p1).astype(np.uint8)
        phi2 = (rng.random(shape) < p2).astype(np.uint8)
        got = oracle.reach(phi1, phi2, conn)
        np.testing.assert_array_equal(got, brute.reach_by_paths(phi1, phi2, conn))
        np.testing.assert_array_equal(got, brute.reach_by_matrix(phi1, phi2, conn))


@pytest.mark.parametrize("conn", CONNS)
def test_reach_closed_form_via_components(conn):
    """rho phi1[phi2] = N(phi1 or Z), Z the phi2-components meeting N phi1 (the
    argument of Sec. 3.2 reducing rho to connected components), computed with
    scipy's labelling and dilation."""
    nd = pytest.importorskip("scipy.ndimage")
    st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
    rng = np.random.default_rng(20 + conn)
    for shape, p2 in [((64, 64), 0.45), ((50, 77), 0.6), ((31, 33), 0.3)]:
        phi1 = (rng.random(shape) < 0.01).astype(np.uint8)
        phi2 = (rng.random(shape) < p2).astype(np.uint8)
        lab, _ = nd.label(phi2, structure=st)
        n1 = nd.binary_dilation(phi1, structure=st, border_value=0)
        hit = np.unique(lab[n1 & (lab > 0)])
        Z = np.isin(lab, hit) & (lab > 0)
        exp = nd.binary_dilation(phi1.astype(bool) | Z, structure=st, border_value=0)
        np.testing.assert_array_equal(oracle.reach(phi1, phi2, conn), exp.astype(np.uint8))


# ----------------------------------------------------------------- ccl ---

@pytest.mark.parametrize("conn", CONNS)
def test_ccl_matches_two_pass_and_scipy(conn):
    rng = np.random.default_rng(30 + conn)
    nd = None
    try:
        import scipy.ndimage as nd  # noqa
    except Exception:  # pragma: no cover
        pass
    for shape, p in [((1, 1), 1.0), ((1, 40), 0.5), ((40, 1), 0.5), ((48, 48), 0.41),
                     ((37, 61), 0.6), ((64, 64), 0.3)]:
        m = (rng.random(shape) < p).astype(np.uint8)
        lab, count = oracle.ccl(m, conn)
        tp = brute.two_pass_label(m, conn)
        assert brute.same_partition(lab, tp, -1, 0)
        np.testing.assert_array_equal(lab, brute.canonical_min_index(tp, 0))
        assert count == tp.max()
        if nd is not None:
            st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
            sl, k = nd.label(m, structure=st)
            assert k == count
            assert brute.same_partition(lab, sl, -1, 0)


def test_ccl_adversarial_patterns():
    for h, w in [(9, 9), (33, 47), (64, 64)]:
        cb = wl.checkerboard_mask(h, w)
        assert oracle.ccl(cb, 8)[1] == 1
        assert oracle.ccl(cb, 4)[1] == int(cb.sum())
        sp = wl.spiral_mask(h, w)
        assert oracle.ccl(sp, 8)[1] == 1 and oracle.ccl(sp, 4)[1] == 1
        rg = wl.rings_mask(h, w)
        assert oracle.ccl(rg, 8)[1] == wl.rings_count(h, w)
        assert oracle.ccl(rg, 4)[1] == wl.rings_count(h, w)


# ---------------------------------------------------------- percentile ---

def test_percentile_matches_numpy_sort():
    rng = np.random.default_rng(40)
    for n in (1, 2, 7, 1000, 4097):
        v = rng.standard_normal(n).astype(np.float32)
        for q in (0.0, 0.3, 0.5, 0.86, 0.95, 0.999, 1.0):
            k = int(np.floor(q * (n - 1)))
            assert oracle.percentile(v, q) == np.sort(v)[k]


# ------------------------------------------------- derived connectives ---

@pytest.mark.parametrize("conn", CONNS)
def test_surrounded_against_direct_definition(conn):
    rng = np.random.default_rng(50 + conn)
    for shape in [(3, 3)] * 40 + [(4, 4)] * 40 + [(5, 5)] * 20:
        phi1 = (rng.random(shape) < rng.uniform(0.2, 0.7)).astype(np.uint8)
        phi2 = (rng.random(shape) < rng.uniform(0.2, 0.7)).astype(np.uint8)
        got = _eval_binary("SURROUNDED", phi1, phi2, conn)
        np.testing.assert_array_equal(got, brute.surrounded_by_paths(phi1, phi2, conn))


@pytest.mark.parametrize("conn", CONNS)
def test_grow_against_region_contact(conn):
    """grow(a, b): a, plus every b-component that contains or touches an a
    pixel (Sec. 4.2)."""
    nd = pytest.importorskip("scipy.ndimage")
    st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
    rng = np.random.default_rng(60 + conn)
    for shape in [(16, 16), (40, 23), (7, 50)]:
        a = (rng.random(shape) < 0.03).astype(np.uint8)
        b = (rng.random(shape) < 0.55).astype(np.uint8)
        lab, _ = nd.label(b, structure=st)
        touch = nd.binary_dilation(a, structure=st, border_value=0)
        hit = np.unique(lab[touch & (lab > 0)])
        exp = a.astype(bool) | (np.isin(lab, hit) & (lab > 0))
        np.testing.assert_array_equal(_eval_binary("GROW", a, b, conn), exp.astype(np.uint8))


@pytest.mark.parametrize("conn", CONNS)
def test_touch_against_region_contact(conn):
    """touch(a, b): the a pixels whose a-component contains a b pixel or is
    adjacent to one.  Written from the components of a (scipy's labeller)
    and the dilation of b, not from reachability."""
    nd = pytest.importorskip("scipy.ndimage")
    st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
    rng = np.random.default_rng(80 + conn)
    for shape in [(16, 16), (40, 23), (7, 50), (1, 30), (30, 1)]:
        for pa, pb in [(0.55, 0.02), (0.4, 0.05), (0.7, 0.01)]:
            a = (rng.random(shape) < pa).astype(np.uint8)
            b = (rng.random(shape) < pb).astype(np.uint8)
            lab, _ = nd.label(a, structure=st)
            near_b = nd.binary_dilation(b, structure=st, border_value=0)
            hit = np.unique(lab[near_b & (lab > 0)])
            exp = np.isin(lab, hit) & (lab > 0)
            np.testing.assert_array_equal(_eval_binary("TOUCH", a, b, conn), exp.astype(np.uint8))


@pytest.mark.parametrize("conn", CONNS)
def test_touch_against_paths(conn):
    """touch(a, b) on small grids against its meaning by path search: from x
    in a, walk inside a until a b pixel is entered."""
    rng = np.random.default_rng(90 + conn)
    for shape in [(3, 3)] * 60 + [(4, 4)] * 60 + [(5, 5)] * 40 + [(2, 6)] * 20:
        a = (rng.random(shape) < rng.uniform(0.3, 0.8)).astype(np.uint8)
        b = (rng.random(shape) < rng.uniform(0.05, 0.4)).astype(np.uint8)
        np.testing.assert_array_equal(_eval_binary("TOUCH", a, b, conn),
                                      brute.touch_by_paths(a, b, conn))


def test_touch_special_cases():
    """touch(a, false) = false; touch(a, true) = a; touch(a, a) = a;
    touch(false, b) = false."""
    rng = np.random.default_rng(99)
    for conn in CONNS:
        a = (rng.random((9, 11)) < 0.5).astype(np.uint8)
        z, o = np.zeros_like(a), np.ones_like(a)
        np.testing.assert_array_equal(_eval_binary("TOUCH", a, z, conn), z)
        np.testing.assert_array_equal(_eval_binary("TOUCH", a, o, conn), a)
        np.testing.assert_array_equal(_eval_binary("TOUCH", a, a, conn), a)
        np.testing.assert_array_equal(_eval_binary("TOUCH", z, a, conn), z)


@pytest.mark.parametrize("conn", CONNS)
def test_interior_is_erosion(conn):
    nd = pytest.importorskip("scipy.ndimage")
    st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
    rng = np.random.default_rng(70 + conn)
    m = (rng.random((40, 41)) < 0.8).astype(np.uint8)
    nodes = [_f("MASK"), _f("INTERIOR", 0)]
    got = oracle.evaluate(nodes, [1], masks=[m], conn=conn).masks[0]
    # erosion with pixels outside the image counting as "not in phi" being
    # absent: outside pixels do not exist, so they never remove a pixel
    exp = nd.binary_erosion(m, structure=st, border_value=1)
    np.testing.assert_array_equal(got, exp.astype(np.uint8))


# ----------------------------------------------------- DAG plumbing ---

def _compose(nodes, roots, img, conn):
    """Evaluate a formula with independent Python primitives: numpy compares,
    scipy dilation, relation-algebra reach; derived connectives by their
    definitions."""
    nd = pytest.importorskip("scipy.ndimage")
    st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
    N = lambda m: nd.binary_dilation(m, structure=st, border_value=0)
    R = lambda a, b: brute.reach_by_matrix(a, b, conn).astype(bool)
    v = []
    for (op, a, b, image, ch, t, q) in nodes:
        if op == "THR_GT":
            v.append(img[ch] > np.float32(t))
        elif op == "THR_LT":
            v.append(img[ch] < np.float32(t))
        elif op in ("PCT_GT", "PCT_LT"):
            x = img[ch].ravel()
            p = np.sort(x)[int(np.floor(q * (x.size - 1)))]
            v.append(img[ch] > p if op == "PCT_GT" else img[ch] < p)
        elif op == "NOT":
            v.append(~v[a])
        elif op == "AND":
            v.append(v[a] & v[b])
        elif op == "OR":
            v.append(v[a] | v[b])
        elif op == "NEAR":
            v.append(N(v[a]))
        elif op == "REACH":
            v.append(R(v[a], v[b]))
        elif op == "INTERIOR":
            v.append(~N(~v[a]))
        elif op == "SURROUNDED":
            v.append(v[a] & ~R(~(v[a] | v[b]), ~v[b]))
        elif op == "GROW":
            v.append(v[a] | (v[b] & R(v[a], v[b])))
        elif op == "TOUCH":
            v.append(v[a] & R(v[b], v[a]))
        else:
            raise AssertionError(op)
    return [v[r].astype(np.uint8) for r in roots]


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dag_evaluation_matches_composition(conn, seed):
    f = wl.random_dag(120, seed=seed, max_depth=40)
    img = wl.uniform_image(14, 15, seed=seed)
    got = oracle.evaluate(wl.formula_to_records(f), f.roots, [img], conn=conn).masks
    exp = _compose(wl.formula_to_records(f), f.roots, img, conn)
    for g, e in zip(got, exp):
        np.testing.assert_array_equal(g, e)


def test_dag_with_derived_ops_matches_composition():
    f = wl.config4_formula()
    img = wl.mri_phantom_batch([(18, 21)], seed=3)[0]
    for conn in CONNS:
        got = oracle.evaluate(wl.formula_to_records(f), f.roots, [img], conn=conn).masks
        exp = _compose(wl.formula_to_records(f), f.roots, img, conn)
        for g, e in zip(got, exp):
            np.testing.assert_array_equal(g, e)


def test_expansion_counts():
    f = _f
    # or(a, b) -> not a, not b, and, not : 4 nodes beyond the atoms
    prim, _ = oracle.expand([f("MASK", image=0), f("MASK", image=1), f("OR", 0, 1)], [2])
    assert len(prim) == 2 + 4
    # surrounded(a, b) = a and not rho(not(a or b))[not b]: not a, not b, and,
    # not (the or), not (its negation), rho, not, and = 8; not b shared
    prim, _ = oracle.expand([f("MASK", image=0), f("MASK", image=1), f("SURROUNDED", 0, 1)], [2])
    assert len(prim) == 2 + 8
    # identical subtrees are shared; commuted operands are not merged
    prim, roots = oracle.expand([f("MASK"), f("MASK", image=1), f("NEAR", 0), f("NEAR", 0),
                                 f("AND", 2, 1), f("AND", 1, 3)], [4, 5])
    assert len(prim) == 5 and roots == [3, 4]
    assert len(oracle.expand(wl.formula_to_records(wl.config4_formula()),
                             wl.config4_formula().roots)[0]) == 40
