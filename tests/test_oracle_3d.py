"""Pins of the oracle's volume operators (groundwork for 3D volumes, the
paper's outlook beyond 2D slices, Sec. 3 and Sec. 5): N with the 26- and
6-neighbourhoods, rho, and component labelling in D x H x W volumes.  The
references are scipy routines, brute-force path enumeration on tiny
volumes, a fixed-point labelling, and the 2D oracle on one-slice volumes."""
from __future__ import annotations

import numpy as np
import pytest

import brute
import oracle

scipy_nd = pytest.importorskip("scipy.ndimage")


def _struct(conn):
    return scipy_nd.generate_binary_structure(3, 3 if conn == 26 else 1)


@pytest.mark.parametrize("conn", [6, 26])
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (5, 7, 6), (9, 1, 13), (3, 17, 2)])
def test_near3_is_scipy_dilation(conn, shape):
    rng = np.random.default_rng(sum(shape) + conn)
    for p in (0.05, 0.3, 0.7):
        m = (rng.random(shape) < p).astype(np.uint8)
        exp = scipy_nd.binary_dilation(m, structure=_struct(conn), border_value=0).astype(np.uint8)
        np.testing.assert_array_equal(oracle.near3(m, conn), exp)


@pytest.mark.parametrize("conn3,conn2", [(26, 8), (6, 4)])
def test_one_slice_volumes_are_the_2d_operators(conn3, conn2):
    rng = np.random.default_rng(3)
    for _ in range(10):
        a = (rng.random((1, 13, 21)) < 0.2).astype(np.uint8)
        b = (rng.random((1, 13, 21)) < 0.55).astype(np.uint8)
        np.testing.assert_array_equal(oracle.near3(a, conn3)[0], oracle.near(a[0], conn2))
        np.testing.assert_array_equal(oracle.reach3(a, b, conn3)[0], oracle.reach(a[0], b[0], conn2))
        np.testing.assert_array_equal(oracle.ccl3(b, conn3)[0][0], oracle.ccl(b[0], conn2)[0])


@pytest.mark.parametrize("conn", [6, 26])
def test_reach3_exhaustive_on_a_2x2x2_volume(conn):
    """(phi1, phi2) pairs on 2 x 2 x 2 voxels against DFS over simple paths:
    every phi1, with every phi2 for each seventh phi1 and a stride of 37
    through the phi2 otherwise."""
    nb = brute.neighbours3(2, 2, 2, conn)
    for b1 in range(256):
        f1 = np.array([(b1 >> i) & 1 for i in range(8)], np.uint8)
        for b2 in range(0, 256, 1 if b1 % 7 == 0 else 37):
            f2 = np.array([(b2 >> i) & 1 for i in range(8)], np.uint8)
            exp = brute.reach_by_paths_nb(f1, f2, nb)
            got = oracle.reach3(f1.reshape(2, 2, 2), f2.reshape(2, 2, 2), conn).ravel()
            assert np.array_equal(got, exp), (b1, b2)


@pytest.mark.parametrize("conn", [6, 26])
def test_reach3_random_small_against_paths_and_closed_form(conn):
    """Seeded pairs on 2 x 3 x 2 volumes against simple paths; on larger
    volumes against N(phi1 or Z), Z the phi2-components meeting N phi1."""
    rng = np.random.default_rng(conn)
    nb = brute.neighbours3(2, 3, 2, conn)
    for _ in range(60):
        f1 = (rng.random(12) < 0.15).astype(np.uint8)
        f2 = (rng.random(12) < 0.5).astype(np.uint8)
        got = oracle.reach3(f1.reshape(2, 3, 2), f2.reshape(2, 3, 2), conn).ravel()
        assert np.array_equal(got, brute.reach_by_paths_nb(f1, f2, nb))
    st = _struct(conn)
    for _ in range(10):
        a = (rng.random((6, 9, 11)) < 0.03).astype(np.uint8)
        b = (rng.random((6, 9, 11)) < 0.45).astype(np.uint8)
        lab, _ = scipy_nd.label(b, structure=st)
        na = scipy_nd.binary_dilation(a, structure=st, border_value=0)
        hit = np.unique(lab[na & (lab > 0)])
        z = np.isin(lab, hit) & (lab > 0)
        exp = scipy_nd.binary_dilation(a.astype(bool) | z, structure=st, border_value=0)
        np.testing.assert_array_equal(oracle.reach3(a, b, conn), exp.astype(np.uint8))


@pytest.mark.parametrize("conn", [6, 26])
def test_ccl3_matches_fixed_point_labelling_and_scipy(conn):
    rng = np.random.default_rng(11 + conn)
    for shape, p in [((3, 4, 5), 0.5), ((4, 6, 3), 0.3), ((2, 9, 9), 0.6)]:
        m = (rng.random(shape) < p).astype(np.uint8)
        lab, n = oracle.ccl3(m, conn)
        exp = brute.components_nb(m.ravel(), brute.neighbours3(*shape, conn)).reshape(shape)
        np.testing.assert_array_equal(lab, exp)
        sl, sn = scipy_nd.label(m, structure=_struct(conn))
        assert n == sn and brute.same_partition(lab, sl, -1, 0)


def test_ccl3_adjacency_along_the_third_axis():
    """Two slices that touch only through a diagonal in z: one component
    under 26-adjacency, two under 6; a column of voxels along z is one
    component under both."""
    m = np.zeros((2, 3, 3), np.uint8)
    m[0, 0, 0] = 1
    m[1, 1, 1] = 1
    assert oracle.ccl3(m, 26)[1] == 1 and oracle.ccl3(m, 6)[1] == 2
    col = np.zeros((5, 2, 2), np.uint8)
    col[:, 1, 0] = 1
    for conn in (6, 26):
        lab, n = oracle.ccl3(col, conn)
        assert n == 1 and (lab[:, 1, 0] == 2).all()


@pytest.mark.parametrize("conn", [6, 26])
def test_volume_formula_is_a_composition_of_the_pinned_operators(conn):
    """A formula with thresholds, a percentile, a number term, N, rho and
    the derived grow and surrounded on a two-channel volume equals the same
    steps composed by hand from the pinned primitives."""
    rng = np.random.default_rng(5)
    vol = rng.random((2, 4, 9, 11)).astype(np.float32)
    rec = [("THR_GT", -1, -1, 0, 0, 0.8, 0.0), ("PCT_LT", -1, -1, 0, 1, 0.0, 0.4),
           ("VALUE", -1, -1, 0, 0, 0.0, 0.0), ("VALUE", -1, -1, 0, 1, 0.0, 0.0),
           ("SUB", 2, 3, 0, 0, 0.0, 0.0), ("THR_GT", 4, -1, 0, 0, 0.1, 0.0),
           ("NEAR", 0, -1, 0, 0, 0.0, 0.0), ("REACH", 6, 1, 0, 0, 0.0, 0.0),
           ("GROW", 0, 5, 0, 0, 0.0, 0.0), ("SURROUNDED", 5, 0, 0, 0, 0.0, 0.0)]
    got = oracle.evaluate3(rec, [6, 7, 8, 9], [vol], conn=conn).masks
    st = _struct(conn)
    a = vol[0] > np.float32(0.8)
    v1 = np.sort(vol[1].ravel())[int(0.4 * (vol[1].size - 1))]
    b = vol[1] < v1
    c = (vol[0] - vol[1]) > np.float32(0.1)
    n_a = scipy_nd.binary_dilation(a, structure=st, border_value=0)
    r = oracle.reach3(n_a, b, conn).astype(bool)
    grow = a | (c & oracle.reach3(a, c, conn).astype(bool))
    sur = c & ~oracle.reach3(~(c | a), ~a, conn).astype(bool)
    for g, e in zip(got, [n_a, r, grow, sur]):
        np.testing.assert_array_equal(g.astype(bool), e)
