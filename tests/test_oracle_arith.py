"""Pins of the oracle's number terms and of uint16 images (the tool's basic
arithmetic and 16-bit unsigned pixels, Sec. 3).  Reading: a uint16 pixel is
its integer value; ADD / SUB / MUL / DIV are IEEE-754 binary32 operations
rounded to nearest even, one rounding per node; thresholds compare strictly;
NaN satisfies no threshold and sorts after +infinity in a percentile.

The expected values here come from exact rational arithmetic (fractions)
rounded to binary32 by the rounding rule written out below, from integer
comparisons, and from IEEE-754's special-case rules -- not from the oracle's
own float code."""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle

from exact_f32 import round_f32


def _bits(f: float) -> int:
    return struct.unpack("<I", struct.pack("<f", f))[0]


def _samples(rng, n):
    """float32 values over the whole range: normals of every binade,
    subnormals, values next to powers of two, small integers."""
    e = rng.integers(-149, 128, size=n)
    m = rng.random(n) + 1.0
    v = (m * np.exp2(e.astype(np.float64))).astype(np.float32)
    v[rng.random(n) < 0.5] *= -1
    v[: n // 10] = rng.integers(-300, 300, size=n // 10).astype(np.float32)
    sub = rng.integers(1, 1 << 23, size=n // 10).astype(np.uint32)
    v[n // 10: 2 * (n // 10)] = sub.view(np.float32)
    return v[np.isfinite(v)]


@pytest.mark.parametrize("op", ["ADD", "SUB", "MUL", "DIV"])
def test_arith_is_correctly_rounded_binary32(op):
    rng = np.random.default_rng({"ADD": 1, "SUB": 2, "MUL": 3, "DIV": 4}[op])
    a = _samples(rng, 4000)
    b = _samples(rng, 4000)[: a.size]
    a = a[: b.size]
    if op == "ADD":  # also operands of close magnitude (cancellation)
        b[:500] = (-a[:500] * np.float32(1.0 + 1e-6)).astype(np.float32)
    if op == "DIV":
        keep = b != 0
        a, b = a[keep], b[keep]
    got = oracle.arith(op, a, b)
    for x, y, g in zip(a.tolist(), b.tolist(), got.tolist()):
        X, Y = Fraction(x), Fraction(y)
        exact = {"ADD": X + Y, "SUB": X - Y, "MUL": X * Y, "DIV": X / Y if Y != 0 else None}[op]
        want = round_f32(exact)
        if want == 0.0 and g == 0.0:
            continue  # the sign of an exact zero is checked separately
        assert _bits(g) == _bits(want), f"{x} {op} {y}: got {g!r}, exact rounding {want!r}"


def test_arith_constant_operand_and_special_cases():
    inf, nan = math.inf, math.nan
    x = np.array([1.0, -1.0, 0.0, -0.0, inf, -inf, 3.0], dtype=np.float32)
    # x / 0: +-inf by the sign of x, NaN for 0/0; inf - inf = NaN; 0 * inf = NaN
    d = oracle.arith("DIV", x, np.float32(0.0))
    assert d[0] == inf and d[1] == -inf and np.isnan(d[2]) and np.isnan(d[3])
    assert d[4] == inf and d[5] == -inf
    s = oracle.arith("SUB", np.array([inf], np.float32), np.array([inf], np.float32))
    assert np.isnan(s[0])
    m = oracle.arith("MUL", np.array([0.0], np.float32), np.array([inf], np.float32))
    assert np.isnan(m[0])
    # exact zeros: x - x = +0 under round to nearest; -0 + -0 = -0
    z = oracle.arith("SUB", x[:2], x[:2])
    assert _bits(float(z[0])) == 0 and _bits(float(z[1])) == 0
    nz = oracle.arith("ADD", np.array([-0.0], np.float32), np.array([-0.0], np.float32))
    assert _bits(float(nz[0])) == 0x80000000
    # the constant operand is the float32 rounding of the given value
    c = oracle.arith("ADD", np.array([0.0], np.float32), 0.1)
    assert _bits(float(c[0])) == _bits(float(np.float32(0.1)))
    # overflow rounds to infinity, gradual underflow keeps subnormals
    big = np.array([np.finfo(np.float32).max], np.float32)
    assert oracle.arith("MUL", big, np.float32(2.0))[0] == inf
    tiny = np.array([np.float32(2.0 ** -126)], np.float32)
    assert oracle.arith("DIV", tiny, np.float32(4.0))[0] == np.float32(2.0 ** -128)


def test_uint16_thresholds_are_integer_comparisons():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 65536, size=(1, 37, 53), dtype=np.uint16)
    img[0, 0, :6] = [0, 65535, 62258, 62259, 56360, 100]
    v = img[0].astype(np.int64)
    for t, gt_int, lt_int in [(62258.0, 62258, 62258), (56360.0, 56360, 56360),
                              (100.5, 100, 101), (0.0, 0, 0), (65535.0, 65535, 65535),
                              (-1.0, -1, -1), (70000.0, 70000, 70000)]:
        rec = [("THR_GT", -1, -1, 0, 0, t, 0.0), ("THR_LT", -1, -1, 0, 0, t, 0.0)]
        gt, lt = oracle.evaluate(rec, [0, 1], [img]).masks
        np.testing.assert_array_equal(gt, (v > gt_int).astype(np.uint8), err_msg=f"> {t}")
        np.testing.assert_array_equal(lt, (v < lt_int).astype(np.uint8), err_msg=f"< {t}")
    # the percentile of a uint16 channel is one of its values, by integer sort
    for q in (0.0, 0.5, 0.86, 0.95, 1.0):
        k = int(q * (v.size - 1))
        assert oracle.percentile(img[0], q) == float(np.sort(v.ravel())[k])


def _exact_number(op, xs, ys):
    return [round_f32({"ADD": Fraction(x) + Fraction(y), "SUB": Fraction(x) - Fraction(y),
                       "MUL": Fraction(x) * Fraction(y), "DIV": Fraction(x) / Fraction(y)}[op])
            for x, y in zip(xs, ys)]


def test_formula_with_number_terms_brute_force():
    """(v0 - v1) / (v0 + c) > t and the median of v0 * v1, on a small
    two-channel image, against exact arithmetic pixel by pixel."""
    rng = np.random.default_rng(11)
    img = (rng.random((2, 6, 7)) * 4.0 - 1.0).astype(np.float32)
    c, t = 0.75, 0.125
    rec = [("VALUE", -1, -1, 0, 0, 0.0, 0.0),           # 0  v0
           ("VALUE", -1, -1, 0, 1, 0.0, 0.0),           # 1  v1
           ("SUB", 0, 1, 0, 0, 0.0, 0.0),               # 2  v0 - v1
           ("ADD", 0, -1, 0, 0, c, 0.0),                # 3  v0 + c
           ("DIV", 2, 3, 0, 0, 0.0, 0.0),               # 4  (v0 - v1) / (v0 + c)
           ("THR_GT", 4, -1, 0, 0, t, 0.0),             # 5
           ("MUL", 0, 1, 0, 0, 0.0, 0.0),               # 6  v0 * v1
           ("PCT_LT", 6, -1, 0, 0, 0.0, 0.5),           # 7  v0 * v1 < its median
           ("NOT", 5, -1, 0, 0, 0.0, 0.0),              # 8
           ("AND", 8, 7, 0, 0, 0.0, 0.0)]               # 9
    got = oracle.evaluate(rec, [5, 7, 9], [img]).masks
    v0, v1 = img[0].ravel().tolist(), img[1].ravel().tolist()
    num = _exact_number("SUB", v0, v1)
    den = _exact_number("ADD", v0, [float(np.float32(c))] * len(v0))
    q = [round_f32(Fraction(a) / Fraction(b)) if b != 0 else math.copysign(math.inf, a)
         for a, b in zip(num, den)]
    e5 = np.array([x > t for x in q], dtype=np.uint8).reshape(6, 7)
    prod = _exact_number("MUL", v0, v1)
    med = sorted(prod)[int(0.5 * (len(prod) - 1))]
    e7 = np.array([p < med for p in prod], dtype=np.uint8).reshape(6, 7)
    np.testing.assert_array_equal(got[0], e5)
    np.testing.assert_array_equal(got[1], e7)
    np.testing.assert_array_equal(got[2], (1 - e5) & e7)


def test_operand_order_of_sub_and_div():
    """v0 - v1 > 0 exactly when v0 > v1 (gradual underflow makes a - b = 0
    only for a = b), and v1 / v0 < 0 exactly when the signs differ."""
    rng = np.random.default_rng(3)
    img = (rng.standard_normal((2, 19, 23)) * 10).astype(np.float32)
    img[1, :3] = img[0, :3]
    rec = [("VALUE", -1, -1, 0, 0, 0.0, 0.0), ("VALUE", -1, -1, 0, 1, 0.0, 0.0),
           ("SUB", 0, 1, 0, 0, 0.0, 0.0), ("THR_GT", 2, -1, 0, 0, 0.0, 0.0),
           ("DIV", 1, 0, 0, 0, 0.0, 0.0), ("THR_LT", 4, -1, 0, 0, 0.0, 0.0)]
    gt, neg = oracle.evaluate(rec, [3, 5], [img]).masks
    np.testing.assert_array_equal(gt, (img[0] > img[1]).astype(np.uint8))
    np.testing.assert_array_equal(neg, ((img[0] > 0) != (img[1] > 0)).astype(np.uint8))


def test_nan_satisfies_no_threshold_and_sorts_last():
    img = np.array([[[0.0, 1.0, 2.0, 0.0, -3.0]]], dtype=np.float32)
    # 0/0 = NaN at pixels 0 and 3
    rec = [("VALUE", -1, -1, 0, 0, 0.0, 0.0), ("DIV", 0, 0, 0, 0, 0.0, 0.0),
           ("THR_GT", 1, -1, 0, 0, 0.5, 0.0), ("THR_LT", 1, -1, 0, 0, 0.5, 0.0),
           ("PCT_GT", 1, -1, 0, 0, 0.0, 0.0), ("PCT_LT", 1, -1, 0, 0, 0.0, 1.0)]
    gt, lt, pmin, pmax = oracle.evaluate(rec, [2, 3, 4, 5], [img]).masks
    # x / x = 1 elsewhere
    assert gt.tolist() == [[0, 1, 1, 0, 1]]
    assert lt.tolist() == [[0, 0, 0, 0, 0]]
    # ascending: 1, 1, 1, NaN, NaN: the minimum is 1; the maximum is NaN
    assert pmin.tolist() == [[0, 0, 0, 0, 0]]
    assert pmax.tolist() == [[0, 0, 0, 0, 0]]
    assert math.isnan(oracle.percentile(np.array([np.nan, 1.0, np.inf], np.float32), 1.0))
    assert oracle.percentile(np.array([np.nan, 1.0, np.inf], np.float32), 0.5) == math.inf


@pytest.mark.parametrize("rec,roots", [
    ([("VALUE", -1, -1, 0, 0, 0, 0)], [0]),                                   # number root
    ([("VALUE", -1, -1, 0, 0, 0, 0), ("NOT", 0, -1, 0, 0, 0, 0)], [1]),       # not of a number
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0), ("ADD", 0, -1, 0, 0, 1, 0),
      ("THR_GT", 1, -1, 0, 0, 0, 0)], [2]),                                  # add of a mask
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0), ("THR_GT", 0, -1, 0, 0, 0, 0)], [1]),  # threshold of a mask
])
def test_number_and_mask_kinds_do_not_mix(rec, roots):
    with pytest.raises(ValueError):
        oracle.expand(rec, roots)


def test_round_f32_agrees_with_numpy_on_doubles():
    """The rounding rule above, on doubles, is numpy's float64 -> float32
    conversion (both round to nearest even)."""
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.standard_normal(2000) * np.exp2(rng.integers(-160, 140, 2000)),
                         [2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** 128 - 2.0 ** 103, 1.0 + 2.0 ** -24]])
    for x in xs.tolist():
        with np.errstate(over="ignore"):
            want = float(np.float32(x))
        assert round_f32(Fraction(x)) == want or (math.isinf(want) and math.isinf(round_f32(Fraction(x))))
