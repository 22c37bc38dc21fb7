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


def test_sequential_chains_and_taps():
    for mix in ("mixed", "near", "reach"):
        f = wl.sequential_dag(400, seed=2, mix=mix, taps=25)
        g = wl.sequential_dag(400, seed=2, mix=mix, taps=25)
        assert f.nodes == g.nodes and f.roots == g.roots
        # every operator takes the node before it as its first operand,
        # binary ones a fresh threshold as the second
        for i, n in enumerate(f.nodes[1:], start=1):
            if n.op in ("NOT", "NEAR"):
                assert n.a == i - 1
            elif n.op in ("AND", "REACH"):
                assert n.b == i - 1 and f.nodes[i - 1].op in ("THR_GT", "THR_LT")
        assert f.roots[-1] == len(f.nodes) - 1 and f.roots[:3] == [0, 25, 50]
    ops = [n.op for n in wl.sequential_dag(2000, seed=0, mix="near").nodes]
    assert ops.count("REACH") == 0 and ops.count("NEAR") > ops.count("NOT")
    assert wl.sequential_dag(300, seed=5).roots == [len(wl.sequential_dag(300, seed=5).nodes) - 1]


def test_arith_dag_kinds():
    f = wl.arith_dag(80, seed=1)
    num = set()
    for i, n in enumerate(f.nodes):
        if n.op in wl.NUMBER_OPS:
            num.add(i)
            if n.op != "VALUE":
                assert n.a in num and (n.b < 0 or n.b in num)
        elif n.op in ("THR_GT", "THR_LT", "PCT_GT", "PCT_LT"):
            assert n.a in num
        else:
            assert n.a not in num and n.b not in num
    assert all(r not in num for r in f.roots)


def test_uint16_generators():
    u = wl.uniform_image_u16(7, 9, channels=2, seed=1)
    assert u.dtype == np.uint16 and u.shape == (2, 7, 9)
    q = wl.to_u16(np.array([[-0.1, 0.0, 0.5, 1.0, 1.2]], np.float32))
    assert q.tolist() == [[0, 0, 32768, 65535, 65535]]
    spec = wl.grow_spec_u16_formula()
    assert [n.t for n in spec.nodes[:2]] == [62258.0, 56360.0]


def test_mri_volume_phantom():
    v = wl.mri_phantom_volume(12, 40, 36, seed=2)
    assert v.shape == (4, 12, 40, 36) and v.dtype == np.float32
    assert np.array_equal(v, wl.mri_phantom_volume(12, 40, 36, seed=2))
    # the core is brighter than the background in channel 2, in 3D
    assert v[2].max() > 0.7 and np.median(v[2]) < 0.45
