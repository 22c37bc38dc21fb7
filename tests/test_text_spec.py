"""Specification texts (vl_formula_compile_text): the command language of the
paper's tool (Sec. 3) compiled into the same formulas as node arrays.  Each
text is checked against a node formula written out by hand: both plans are
run by the host simulation of the executor and compared with the oracle on
the node formula, on the same images.  Also names, sharing and errors."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import plan_sim
import paper_2010_07284_gb300 as vg

pytest.importorskip("scipy")


def N(op, a=-1, b=-1, image=0, channel=0, t=0.0, q=0.0):
    return (op, a, b, image, channel, float(np.float32(t)), float(q))


def run_text(src, images, conn=8):
    F = vg.compile_text(src, conn)
    return F, plan_sim.simulate(F.plan(), images, {}, conn)


def expect(nodes, roots, images, conn=8):
    return oracle.evaluate(nodes, roots, images, conn=conn).masks


def same(got, exp):
    assert len(got) == len(exp)
    for r, (g, e) in enumerate(zip(got, exp)):
        assert np.array_equal(g.astype(np.uint8), e), f"root {r} differs"


def images(seed, n=1, c=1, h=37, w=150, scale=1.0):
    rng = np.random.default_rng(seed)
    return [(rng.random((c, h, w)) * scale).astype(np.float32) for _ in range(n)]


@pytest.mark.parametrize("conn", [4, 8])
def test_region_growing_spec(conn):
    # two intensity bands of a 16-bit scan and the growth of the brighter
    # one through the other (the case study of Sec. 4.2)
    src = """
    // a 16-bit scan, values 0 .. 65535
    load flair = "flair"
    let bright = intensity(flair) >. 62258
    let candidate = intensity(flair) >. 56360
    save "tumour" grow(bright, candidate)
    """
    ims = images(1, scale=65535.0)
    F, got = run_text(src, ims, conn)
    assert F.loads == ["flair"] and F.saves == ["tumour"]
    nodes = [N("THR_GT", t=62258), N("THR_GT", t=56360), N("GROW", 0, 1)]
    same(got, expect(nodes, [2], ims, conn))


def test_macros_constants_infix_and_two_images():
    src = """
    load a = "first"
    load b = "second"
    let above(x, t) = intensity(x) >. t
    let ring(m) = N(m) & !m
    let core = above(a, 0.7) & !above(b, 0.2)
    save "ring" ring(core) | touch(core, above(b, 0.5))
    save "held" surrounded(core, tt) & (interior(above(a, 0.1)) | ff)
    save "reach" rho(above(a, 0.9), !above(b, 0.8)) & not(core)
    """
    ims = images(2, n=2)
    F, got = run_text(src, ims)
    assert F.loads == ["a", "b"] and F.saves == ["ring", "held", "reach"]
    nodes = [
        N("THR_GT", image=0, t=0.7),   # 0
        N("THR_GT", image=1, t=0.2),   # 1
        N("NOT", 1),                   # 2
        N("AND", 0, 2),                # 3 core
        N("NEAR", 3),                  # 4
        N("NOT", 3),                   # 5
        N("AND", 4, 5),                # 6 ring(core)
        N("THR_GT", image=1, t=0.5),   # 7
        N("TOUCH", 3, 7),              # 8
        N("OR", 6, 8),                 # 9 root 0
        N("TRUE"),                     # 10
        N("SURROUNDED", 3, 10),        # 11
        N("THR_GT", image=0, t=0.1),   # 12
        N("INTERIOR", 12),             # 13
        N("FALSE"),                    # 14
        N("OR", 13, 14),               # 15
        N("AND", 11, 15),              # 16 root 1
        N("THR_GT", image=0, t=0.9),   # 17
        N("THR_GT", image=1, t=0.8),   # 18
        N("NOT", 18),                  # 19
        N("REACH", 17, 19),            # 20
        N("AND", 20, 5),               # 21 root 2
    ]
    same(got, expect(nodes, [9, 16, 21], ims))


def test_percentiles_channels_and_arithmetic():
    src = """
    load im = "rgb"
    let d = red(im) - channel(im, 2)
    let s = (green(im) + 0.25) * 2
    save "p" d >. percentile(d, 0.9)
    save "q" (0.5 - blue(im)) <. 0.1 & s <. 1.5
    save "r" intensity(im) <. percentile(intensity(im), 0.25) | -s >. -1
    """
    ims = images(3, c=3)
    _, got = run_text(src, ims)
    nodes = [
        N("VALUE", channel=0),          # 0 red
        N("VALUE", channel=2),          # 1
        N("SUB", 0, 1),                 # 2 d
        N("PCT_GT", 2, q=0.9),          # 3 root p
        N("VALUE", channel=2),          # 4 (shared with 1 by the compiler)
        N("MUL", 4, -1, t=-1.0),        # 5 -blue
        N("ADD", 5, -1, t=0.5),         # 6 0.5 - blue
        N("THR_LT", 6, t=0.1),          # 7
        N("VALUE", channel=1),          # 8 green
        N("ADD", 8, -1, t=0.25),        # 9
        N("MUL", 9, -1, t=2.0),         # 10 s
        N("THR_LT", 10, t=1.5),         # 11
        N("AND", 7, 11),                # 12 root q
        N("PCT_LT", channel=0, q=0.25),  # 13
        N("MUL", 10, -1, t=-1.0),       # 14 -s
        N("THR_GT", 14, t=-1.0),        # 15
        N("OR", 13, 15),                # 16 root r
    ]
    same(got, expect(nodes, [3, 12, 16], ims))


def test_a_macro_applied_twice_is_shared():
    one = vg.compile_text('load x = "x"\nlet f(m) = N(N(m)) & !m\nsave "o" f(intensity(x) >. 0.5)')
    two = vg.compile_text('load x = "x"\nlet f(m) = N(N(m)) & !m\n'
                          'save "o" f(intensity(x) >. 0.5) & f(intensity(x) >. 0.5)')
    assert one.plan()["sizes"]["n_insns"] == two.plan()["sizes"]["n_insns"]


@pytest.mark.parametrize("src, where", [
    ('load a = "a"\nsave "o" intensity(a) >. ', "line 2"),
    ('load a = "a"\nlet x = intensity(a) >. 1 >. 2\nsave "o" x', "do not chain"),
    ('save "o" intensity(b) >. 1', "unknown name b"),
    ('load a = "a"\nload a = "b"\nsave "o" mask(a)', "already defined"),
    ('load a = "a"\nsave "o" intensity(a)', "save takes a mask"),
    ('load a = "a"\nsave "o" intensity(a) & tt', "takes masks"),
    ('load a = "a"\nlet f(m) = f(m)\nsave "o" f(mask(a))', "deeper than 64"),
    ('load a = "a"\nsave "o" 2 / intensity(a) >. 1', "divided by a number term"),
    ('load a = "a"\nload b = "b"\nsave "o" intensity(a) >. percentile(intensity(b), 0.5)',
     "of the term it is compared with"),
    ('load a = "a"\nsave "o" intensity(a) >. percentile(intensity(a), 1.5)', "in [0, 1]"),
    ('load a = "a"\nlet x = mask(a)', "nothing saved"),
    ('load a = "a"\nprint "v" mask(a)', "print is not supported"),
    ('load a = "a"\nsave "o" grow(mask(a))', "takes 2 arguments"),
    ('load a = "a"\nsave "o" mask(a) $ tt', "unexpected character"),
    ('load a = "a"\nsave "o mask(a)', "unterminated string"),
    ('let = 3', "expected a name"),
])
def test_errors_say_where_and_what(src, where):
    with pytest.raises(vg.VlError) as e:
        vg.compile_text(src)
    assert e.value.code == vg._native.ERR_FORMULA
    assert where in str(e.value), str(e.value)


def test_comments_imports_and_names_of_node_formulas():
    F = vg.compile_text('// a comment\nimport "stdlib.imgql"\nload z = "z" // after\n'
                        'save "all" tt\nsave "none" ff')
    assert F.loads == ["z"] and F.saves == ["all", "none"]
    G = vg.compile_formula([N("TRUE")], [0])
    assert G.loads == [] and G.saves == []


def test_deep_nesting_is_refused_not_a_crash():
    for src in ['load a = "a"\nsave "o" ' + "(" * 5000 + "mask(a)" + ")" * 5000,
                'load a = "a"\nsave "o" ' + "!" * 3000 + "mask(a)"]:
        with pytest.raises(vg.VlError) as e:
            vg.compile_text(src)
        assert "nested deeper than 1000" in str(e.value)
    # 60 macros each applying the previous one: expanded, and shared
    chain = "".join(f"let f{i}(m) = N(m) & f{i - 1}(m)\n" if i else "let f0(m) = N(m)\n"
                    for i in range(60))
    F = vg.compile_text('load a = "a"\n' + chain + 'save "o" f59(mask(a))')
    assert F.saves == ["o"]


def formula_text(recs, roots, with_mask):
    """A node formula spelled as a specification: one `let` per node."""
    lines = ['load img0 = "numbers"'] + (['load img1 = "mask"'] if with_mask else [])
    infix = {"ADD": "+", "SUB": "-", "MUL": "*", "DIV": "/", "AND": "&", "OR": "|"}
    calls = {"NEAR": "N", "INTERIOR": "interior", "REACH": "rho", "SURROUNDED": "surrounded",
             "GROW": "grow", "TOUCH": "touch"}
    for i, (op, a, b, im, ch, t, q) in enumerate(recs):
        chan = f"channel(img{im}, {ch})"
        if op == "VALUE":
            e = chan
        elif op in ("ADD", "SUB", "MUL", "DIV"):
            e = f"n{a} {infix[op]} " + (f"n{b}" if b >= 0 else repr(t))
        elif op in ("THR_GT", "THR_LT"):
            e = f"{f'n{a}' if a >= 0 else chan} {'>.' if op == 'THR_GT' else '<.'} {t!r}"
        elif op in ("PCT_GT", "PCT_LT"):
            term = f"n{a}" if a >= 0 else chan
            e = f"{term} {'>.' if op == 'PCT_GT' else '<.'} percentile({term}, {q!r})"
        elif op in ("TRUE", "FALSE"):
            e = "tt" if op == "TRUE" else "ff"
        elif op == "MASK":
            e = f"mask(img{im})"
        elif op == "NOT":
            e = f"!n{a}"
        elif op in ("AND", "OR"):
            e = f"n{a} {infix[op]} n{b}"
        elif op in ("NEAR", "INTERIOR"):
            e = f"{calls[op]}(n{a})"
        else:
            e = f"{calls[op]}(n{a}, n{b})"
        lines.append(f"let n{i} = {e}")
    lines += [f'save "r{k}" n{r}' for k, r in enumerate(roots)]
    return "\n".join(lines)


@pytest.mark.parametrize("seed", range(40))
def test_random_formulas_spelled_as_text(seed):
    """The compiler's fuzz formulas (every operator, number terms, masks),
    written out as specification text: the text's plan, run by the host
    simulation, equals the oracle on the node formula."""
    from test_compiler_fuzz import random_formula
    rng = np.random.default_rng(5000 + seed)
    n_channels = int(rng.integers(1, 3))
    with_mask = seed % 3 == 0
    recs, roots = random_formula(rng, int(rng.integers(5, 70)), n_channels, with_mask)
    H, W = int(rng.integers(1, 40)), int(rng.integers(1, 260))
    conn = 8 if seed % 2 == 0 else 4
    img = rng.random((n_channels, H, W)).astype(np.float32)
    masks = {1: rng.random((H, W)) < 0.4} if with_mask else {}
    recs_o = [(op, a, b, (0 if op == "MASK" else im), ch, t, q)
              for (op, a, b, im, ch, t, q) in recs]
    exp = oracle.evaluate(recs_o, roots, [img], [masks[1]] if with_mask else [], conn=conn).masks
    F = vg.compile_text(formula_text(recs, roots, with_mask), conn)
    assert len(F.saves) == len(roots)
    got = plan_sim.simulate(F.plan(), [img, None] if with_mask else [img], masks, conn)
    same(got, exp)
