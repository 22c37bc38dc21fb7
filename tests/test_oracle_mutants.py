"""Planted mistakes: each test copies the oracle's C source, plants one
plausible mistake (a dropped term, a wrong comparison, an off-by-one, a wrong
neighbourhood), builds it on the CPU and checks that the pins reject it.  The
oracle itself is never modified."""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import brute
import golden_io
from exact_f32 import round_f32

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "vl_oracle.c")

MUTANTS = {
    "reach_drops_l0": ("out[i] = phi1[i] ? 1 : 0;", "out[i] = 0;"),
    "reach_ignores_phi2": ("if (phi2[u] && !pushed[u])", "if (!pushed[u])"),
    "reach_needs_phi2_at_x": ("out[u] = 1;                       /* u = pi_0, v = pi_1 */",
                              "if (phi2[u]) out[u] = 1;"),
    "near_not_reflexive": ("if (!is_offset(dy, dx, conn)) continue;\n          int yy = y + dy, xx = x + dx;\n          if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;\n          if (a[",
                           "if (!is_offset(dy, dx, conn) || (dy == 0 && dx == 0)) continue;\n          int yy = y + dy, xx = x + dx;\n          if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;\n          if (a["),
    "cross_is_square": ("if (conn == 4) return (dy == 0) || (dx == 0);", "(void)conn;"),
    "threshold_not_strict": ("out[i] = gt ? (v > t) : (v < t);", "out[i] = gt ? (v >= t) : (v <= t);"),
    "percentile_off_by_one": ("int64_t k = (int64_t)(q * (double)(n - 1));",
                              "int64_t k = (int64_t)(q * (double)(n - 1) + 0.5);"),
    "ccl_labels_by_last_pixel": ("labels[u] = (int32_t)s;", "labels[u] = (int32_t)u;"),
    "sub_operands_swapped": ("case VLO_ARITH_SUB: r = x - y;", "case VLO_ARITH_SUB: r = y - x;"),
    "div_is_mul": ("default: r = x / y;", "default: r = x * y;"),
    "constant_operand_dropped": ("float x = a[i], y = b ? b[i] : c, r;", "float x = a[i], y = b ? b[i] : 0.0f, r;"),
    "add_rounds_to_half": ("case VLO_ARITH_ADD: r = x + y;",
                           "case VLO_ARITH_ADD: r = (float)(_Float16)(x + y);"),
    "nan_sorts_first": ("if (nx || ny) return nx - ny;", "if (nx || ny) return ny - nx;"),
    "faces_as_cube_3d": ("if (conn == 6) return (dz != 0) + (dy != 0) + (dx != 0) <= 1;",
                         "(void)conn;"),
    "near3_skips_z": ("if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;\n              if (a[",
                      "if (zz != z || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;\n              if (a["),
    "reach3_ignores_phi2": ("          if (phi2[u] && !pushed[u]) {", "          if (!pushed[u]) {"),
    "ccl3_labels_by_voxel": ("              labels[u] = (int32_t)s;\n              queue[tail++] = u;\n            }\n          }\n    }\n  }\n  free(queue);\n  return count;\n}\n",
                             "              labels[u] = (int32_t)u;\n              queue[tail++] = u;\n            }\n          }\n    }\n  }\n  free(queue);\n  return count;\n}\n"),
}


def _build(tmp, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation {name} no longer applies"
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new, 1))
    so = os.path.join(tmp, f"{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", so, path])
    lib = C.CDLL(so)
    P = C.c_void_p
    lib.vlo_threshold.argtypes = [P, C.c_int64, C.c_float, C.c_int, P]
    lib.vlo_near.argtypes = [P, C.c_int, C.c_int, C.c_int, P]
    lib.vlo_reach.argtypes = [P, P, C.c_int, C.c_int, C.c_int, P]
    lib.vlo_ccl.argtypes = [P, C.c_int, C.c_int, C.c_int, P]
    lib.vlo_ccl.restype = C.c_int64
    lib.vlo_percentile.argtypes = [P, C.c_int64, C.c_double]
    lib.vlo_percentile.restype = C.c_float
    lib.vlo_arith.argtypes = [C.c_int, P, P, C.c_float, C.c_int64, P]
    lib.vlo_near3.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P]
    lib.vlo_reach3.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P]
    lib.vlo_ccl3.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P]
    lib.vlo_ccl3.restype = C.c_int64
    return lib


def _pins_pass(lib) -> bool:
    """A compact copy of the pins: hand-worked fixtures, brute-force reach,
    scipy-free dilation by definition, strict thresholds, percentile ranks,
    canonical labels."""
    def near(m, conn):
        m = np.ascontiguousarray(m, np.uint8)
        o = np.empty_like(m)
        lib.vlo_near(m.ctypes.data, m.shape[0], m.shape[1], conn, o.ctypes.data)
        return o

    def reach(a, b, conn):
        a = np.ascontiguousarray(a, np.uint8)
        b = np.ascontiguousarray(b, np.uint8)
        o = np.empty_like(a)
        lib.vlo_reach(a.ctypes.data, b.ctypes.data, a.shape[0], a.shape[1], conn, o.ctypes.data)
        return o

    def ccl(m, conn):
        m = np.ascontiguousarray(m, np.uint8)
        o = np.empty(m.shape, np.int32)
        lib.vlo_ccl(m.ctypes.data, m.shape[0], m.shape[1], conn, o.ctypes.data)
        return o

    for fx in golden_io.all_fixtures():
        for conn, exp in fx["expect"].items():
            if fx["op"] == "near" and not np.array_equal(near(fx["phi"], conn), exp):
                return False
            if fx["op"] == "reach" and not np.array_equal(reach(fx["phi1"], fx["phi2"], conn), exp):
                return False
            if fx["op"] == "ccl" and not np.array_equal(ccl(fx["phi"], conn), exp):
                return False
        if fx["op"] == "percentile":
            v = np.array([float(x) for x in fx["kv"][0][1:]], np.float32)
            for _, q, want in fx["kv"][1:]:
                if lib.vlo_percentile(v.ctypes.data, v.size, float(q)) != float(want):
                    return False
    rng = np.random.default_rng(5)
    for conn in (4, 8):
        for _ in range(20):
            a = (rng.random((4, 4)) < 0.2).astype(np.uint8)
            b = (rng.random((4, 4)) < 0.5).astype(np.uint8)
            if not np.array_equal(reach(a, b, conn), brute.reach_by_paths(a, b, conn)):
                return False
            # dilation by its definition: OR over the neighbourhood, pixel included
            nb = brute.neighbours(4, 4, conn)
            exp = np.array([a.ravel()[v] or any(a.ravel()[u] for u in nb[v]) for v in range(16)],
                           np.uint8).reshape(4, 4)
            if not np.array_equal(near(a, conn), exp):
                return False
    ch = np.array([0.25, 0.5, 0.75], np.float32)
    o = np.empty(3, np.uint8)
    lib.vlo_threshold(ch.ctypes.data, 3, C.c_float(0.5), 1, o.ctypes.data)
    if list(o) != [0, 0, 1]:
        return False
    # number terms: exact rational results rounded to binary32, for both an
    # array and a constant second operand
    from fractions import Fraction
    xs = (rng.standard_normal(200) * 1e3).astype(np.float32)
    ys = (rng.standard_normal(200) * 1e-2).astype(np.float32)
    ops = {0: lambda a, b: a + b, 1: lambda a, b: a - b, 2: lambda a, b: a * b,
           3: lambda a, b: a / b}
    for op, fn in ops.items():
        for second in (ys, np.float32(0.3)):
            out = np.empty_like(xs)
            if np.isscalar(second):
                lib.vlo_arith(op, xs.ctypes.data, None, C.c_float(second), xs.size, out.ctypes.data)
                bs = [float(second)] * xs.size
            else:
                lib.vlo_arith(op, xs.ctypes.data, second.ctypes.data, 0.0, xs.size, out.ctypes.data)
                bs = second.tolist()
            want = [round_f32(fn(Fraction(a), Fraction(b))) for a, b in zip(xs.tolist(), bs)]
            if out.tolist() != want:
                return False
    # volumes: dilation by definition, reach by simple paths, labels by a
    # fixed-point relaxation, on small random volumes
    for conn in (6, 26):
        nb = brute.neighbours3(2, 3, 2, conn)
        for _ in range(12):
            a = (rng.random((2, 3, 2)) < 0.2).astype(np.uint8)
            b = (rng.random((2, 3, 2)) < 0.5).astype(np.uint8)
            o = np.empty_like(a)
            lib.vlo_near3(a.ctypes.data, 2, 3, 2, conn, o.ctypes.data)
            af = a.ravel()
            exp = np.array([af[v] or any(af[u] for u in nb[v]) for v in range(12)], np.uint8)
            if not np.array_equal(o.ravel(), exp):
                return False
            lib.vlo_reach3(a.ctypes.data, b.ctypes.data, 2, 3, 2, conn, o.ctypes.data)
            if not np.array_equal(o.ravel(), brute.reach_by_paths_nb(af, b.ravel(), nb)):
                return False
            lab = np.empty((2, 3, 2), np.int32)
            lib.vlo_ccl3(b.ctypes.data, 2, 3, 2, conn, lab.ctypes.data)
            if not np.array_equal(lab.ravel(), brute.components_nb(b.ravel(), nb)):
                return False
    # NaN sorts after every number in a percentile: -1, 0.5, 2, NaN, NaN
    v = np.array([np.nan, 2.0, -1.0, np.nan, 0.5], np.float32)
    if lib.vlo_percentile(v.ctypes.data, v.size, 0.5) != 2.0:
        return False
    return True


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="vlo_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_unmutated_source_passes(tmpdir_mod):
    assert _pins_pass(_build(tmpdir_mod, "clean", "", ""))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(tmpdir_mod, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_build(tmpdir_mod, name, old, new)), f"pins missed mutant {name}"


# ----------------------------------------------- expansion of connectives --
# Planted mistakes in the oracle's expansion of the contact connective
# (oracle/expand.py): a modified copy of the module replaces the expansion
# for the duration of one check; the touch pins must then fail.

EXPAND_SRC = os.path.join(os.path.dirname(SRC), "expand.py")

EXPAND_MUTANTS = {
    "touch_arguments_swapped": ("return self.AND(a, self.REACH(b, a))",
                                "return self.AND(a, self.REACH(a, b))"),
    "touch_without_and": ("return self.AND(a, self.REACH(b, a))", "return self.REACH(b, a)"),
    "touch_is_grow": ("return self.AND(a, self.REACH(b, a))",
                      "return self.OR(a, self.AND(b, self.REACH(a, b)))"),
    "touch_via_near": ("return self.AND(a, self.REACH(b, a))",
                       "return self.AND(a, self.NEAR(b))"),
}


def _touch_pins_pass(expand_fn) -> bool:
    """The touch pins (hand-worked fixture, path search, region contact)
    with the oracle's evaluator running on `expand_fn`."""
    import oracle.oracle as oo
    saved = oo.expand
    oo.expand = expand_fn
    try:
        def touch(a, b, conn):
            nodes = [("MASK", -1, -1, 0, 0, 0.0, 0.0), ("MASK", -1, -1, 1, 0, 0.0, 0.0),
                     ("TOUCH", 0, 1, 0, 0, 0.0, 0.0)]
            return oo.evaluate(nodes, [2], masks=[a, b], conn=conn).masks[0]

        for fx in golden_io.all_fixtures():
            if fx["op"] != "touch":
                continue
            for conn, exp in fx["expect"].items():
                if not np.array_equal(touch(fx["phi1"], fx["phi2"], conn), exp):
                    return False
        rng = np.random.default_rng(7)
        for conn in (4, 8):
            for shape in [(4, 4)] * 15 + [(5, 5)] * 10:
                a = (rng.random(shape) < 0.6).astype(np.uint8)
                b = (rng.random(shape) < 0.15).astype(np.uint8)
                if not np.array_equal(touch(a, b, conn), brute.touch_by_paths(a, b, conn)):
                    return False
        return True
    finally:
        oo.expand = saved


def _load_expand(tmp, name, old, new):
    import importlib.util
    src = open(EXPAND_SRC).read()
    assert old in src, f"mutation {name} no longer applies"
    path = os.path.join(tmp, f"expand_{name}.py")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location(f"expand_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.expand


def test_unmutated_expansion_passes_touch_pins(tmpdir_mod):
    assert _touch_pins_pass(_load_expand(tmpdir_mod, "clean", "", ""))


@pytest.mark.parametrize("name", sorted(EXPAND_MUTANTS))
def test_expansion_mutant_is_rejected(tmpdir_mod, name):
    old, new = EXPAND_MUTANTS[name]
    assert not _touch_pins_pass(_load_expand(tmpdir_mod, name, old, new)), \
        f"touch pins missed mutant {name}"
