"""Input generators: shapes, determinism and the structural facts the
workloads rely on (CPU only)."""
import numpy as np

import workloads as wl


def test_generators_are_seeded():
    assert np.array_equal(wl.uniform_image(8, 9, 2, seed=3), wl.uniform_image(8, 9, 2, seed=3))
    assert np.array_equal(wl.gaussian_field_image(32, 40, seed=1), wl.gaussian_field_image(32, 40, seed=1))
    a = wl.random_dag(300, seed=4)
    b = wl.random_dag(300, seed=4)
    assert a.nodes == b.nodes and a.roots == b.roots


def test_gaussian_field_range():
    im = wl.gaussian_field_image(64, 64)
    assert im.shape == (1, 64, 64) and im.dtype == np.float32
    assert im.min() == 0.0 and im.max() == 1.0


def test_random_dag_structure():
    f = wl.random_dag(2000, seed=0)
    ops = [n.op for n in f.nodes]
    assert ops[0] in ("THR_GT", "THR_LT")
    frac = {k: sum(o == k for o in ops) / len(ops) for k in set(ops)}
    assert abs(frac["THR_GT"] + frac["THR_LT"] - 0.35) < 0.04
    assert abs(frac["NEAR"] - 0.20) < 0.03 and abs(frac["REACH"] - 0.10) < 0.03
    assert f.depth() <= 500
    consumed = {x for n in f.nodes for x in (n.a, n.b) if x >= 0}
    assert set(f.roots) == set(range(len(f.nodes))) - consumed
    for n in f.nodes:
        if n.op.startswith("THR"):
            assert np.float32(n.t) == n.t


def test_mri_batch_shapes():
    sides = wl.mri_side_lengths(4096)
    assert sides.min() >= 160 and sides.max() <= 512
    assert 225 <= np.median(sides) <= 255
    ims = wl.mri_phantom_batch(sides[:3])
    for im, (h, w) in zip(ims, sides[:3]):
        assert im.shape == (4, h, w) and im.dtype == np.float32


def test_stream_shapes():
    q = wl.poisson_queries(1000, rate_per_s=50.0, seed=1)
    t = np.array([x.arrival_s for x in q])
    assert np.all(np.diff(t) >= 0)
    sizes = np.array([x.n_nodes for x in q])
    assert sizes.min() >= 10 and sizes.max() <= 2000
