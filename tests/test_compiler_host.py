"""Host logic of the library, on the CPU: the C ABI loads and exports what
include/vl.h declares; the compiler counts primitives like the oracle, rejects
malformed formulas, and its plans -- simulated tile by tile with garbage in
every uncomputed halo row -- give the oracle's masks."""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import plan_sim
import workloads as wl
import paper_2010_07284_gb300 as vg
from paper_2010_07284_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"VL_API\s+[\w\s\*]+?\b(vl_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = N.load()
    declared = _declared_symbols()
    assert len(declared) >= 30
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    bound = {s[0] for s in N.SIGNATURES}
    assert declared <= bound | set(), f"unbound: {sorted(declared - bound)}"


def _rec(f):
    return wl.formula_to_records(f)


@pytest.mark.parametrize("make", [
    lambda: wl.config1_formula(), lambda: wl.config4_formula(), lambda: wl.grow_spec_formula(),
    lambda: wl.random_dag(300, seed=1), lambda: wl.random_dag(2000, seed=0),
    lambda: wl.sequential_dag(200, seed=2)])
def test_primitive_count_matches_oracle(make):
    f = make()
    F = vg.compile_formula(_rec(f), f.roots)
    prim, _ = oracle.expand(_rec(f), f.roots)
    assert F.info()["n_primitive"] == len(prim)
    assert F.info()["n_reach"] == sum(1 for p in prim if p[0] == "REACH")


@pytest.mark.parametrize("nodes,roots,conn,code", [
    ([("NOT", 0, -1, 0, 0, 0, 0)], [0], 8, N.ERR_FORMULA),                       # self operand
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0), ("AND", 0, 5, 0, 0, 0, 0)], [1], 8, N.ERR_FORMULA),
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0)], [3], 8, N.ERR_FORMULA),                 # bad root
    ([("PCT_GT", -1, -1, 0, 0, 0, 1.5)], [0], 8, N.ERR_FORMULA),                 # q > 1
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0)], [0], 5, N.ERR_ARG),                     # conn
    ([(99, -1, -1, 0, 0, 0, 0)], [0], 8, N.ERR_FORMULA),                          # op code
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0), ("MASK", -1, -1, 0, 0, 0, 0),
      ("AND", 0, 1, 0, 0, 0, 0)], [2], 8, N.ERR_FORMULA),                         # image kinds clash
])
def test_malformed_formulas_are_rejected(nodes, roots, conn, code):
    with pytest.raises(N.VlError) as e:
        vg.compile_formula(nodes, roots, conn)
    assert e.value.code == code


def _check_sim(f, images, masks=None, conn=8, seed=0, shuffle=None):
    masks = masks or {}
    F = vg.compile_formula(_rec(f), f.roots, conn)
    plan = F.plan()
    order = plan_sim.random_topological_order(plan, shuffle) if shuffle is not None else None
    got = plan_sim.simulate(plan, images, masks, conn, seed=seed, order=order)
    mlist = [masks[k] for k in sorted(masks)] if masks else []
    # the oracle indexes float images and masks separately
    exp = oracle.evaluate(_rec(f), f.roots, [im for im in images if im is not None], mlist,
                          conn=conn, shape=(next(iter(masks.values())).shape if masks else None)).masks
    for r, (g, e) in enumerate(zip(got, exp)):
        if not np.array_equal(g.astype(np.uint8), e):
            bad = np.argwhere(g.astype(np.uint8) != e)
            raise AssertionError(f"root {r}: {len(bad)} pixels differ, first {bad[:5].tolist()}")
    return plan


@pytest.mark.parametrize("conn", [4, 8])
def test_plan_config1_shape(conn):
    pytest.importorskip("scipy")
    img = wl.gaussian_field_image(130, 200, seed=3)
    _check_sim(wl.config1_formula(), [img], conn=conn)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_plan_random_dags(conn, seed):
    pytest.importorskip("scipy")
    f = wl.random_dag(400, seed=seed, max_depth=60)
    img = wl.uniform_image(70, 1100, seed=seed)   # two tile rows+, two tile columns
    _check_sim(f, [img], conn=conn, seed=seed)


def test_plan_large_random_dag_is_split_and_correct():
    pytest.importorskip("scipy")
    f = wl.random_dag(2000, seed=0)
    img = wl.uniform_image(40, 300, seed=5)
    plan = _check_sim(f, [img], conn=8)
    groups = [s for s in plan["steps"] if s["kind"] == 1]
    assert len(groups) > 1
    assert max(s["halo"] for s in groups) <= 8


def test_plan_sequential_chain_hits_halo_budget():
    pytest.importorskip("scipy")
    nodes = [("THR_GT", -1, -1, 0, 0, 0.7, 0.0)]
    for i in range(40):
        nodes.append(("NEAR", len(nodes) - 1, -1, 0, 0, 0, 0))
    f = wl.Formula([wl.Node(*n) for n in nodes], [len(nodes) - 1])
    img = wl.uniform_image(90, 150, seed=9)
    plan = _check_sim(f, [img], conn=8)
    assert sum(1 for s in plan["steps"] if s["kind"] == 1) >= 5


def test_plan_config4_formula_with_percentiles():
    pytest.importorskip("scipy")
    f = wl.config4_formula()
    img = wl.mri_phantom_batch([(70, 90)], seed=4)[0]
    for conn in (4, 8):
        _check_sim(f, [img], conn=conn)


def test_plan_mask_atoms_constants_and_mask_root():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(7)
    m0 = rng.random((50, 60)) < 0.5
    m1 = rng.random((50, 60)) < 0.02
    nodes = [("MASK", -1, -1, 0, 0, 0, 0), ("MASK", -1, -1, 1, 0, 0, 0),
             ("REACH", 1, 0, 0, 0, 0, 0), ("TRUE", -1, -1, 0, 0, 0, 0),
             ("AND", 2, 3, 0, 0, 0, 0), ("FALSE", -1, -1, 0, 0, 0, 0),
             ("REACH", 0, 5, 0, 0, 0, 0), ("GROW", 1, 0, 0, 0, 0, 0),
             ("REACH", 1, 3, 0, 0, 0, 0)]
    f = wl.Formula([wl.Node(*n) for n in nodes], [4, 0, 6, 7, 8, 3])
    for conn in (4, 8):
        _check_sim(f, [None, None], masks={0: m0, 1: m1}, conn=conn)


# ------------------------------------------------------------- rank codes

def test_rank_tables_encode_every_constant_threshold():
    """Every constant threshold of a channel read by many becomes a rank
    comparison whose bound points back at its own value in the table."""
    f = wl.random_dag(2000, seed=0)
    plan = vg.compile_formula(_rec(f), f.roots, 8).plan()
    tabs, vals = plan["rank_tables"], plan["rank_values"]
    assert len(tabs) == 1 and plan["steps"][0]["kind"] == 6
    t = tabs[0]
    v = vals[t["value_off"]:t["value_off"] + t["m"]]
    assert np.all(np.diff(v) > 0)                       # sorted, distinct
    assert t["nbits"] == int(2 * t["m"] + 1).bit_length()
    thr = [n.t for n in f.nodes if n.op in ("THR_GT", "THR_LT")]
    used = set()
    n_rank = 0
    for s in plan["steps"]:
        if s["kind"] != 1:
            continue
        for ins in plan["insns"][s["insn_off"]:s["insn_off"] + s["insn_cnt"]]:
            assert ins["op"] != 1, "a constant threshold was left direct"
            if ins["op"] != 10:
                continue
            n_rank += 1
            used.add(np.float32(ins["t"]))
            K, lt = ins["image"] & 0xFFFF, ins["b"] & 1
            assert K % 2 == (1 if lt else 0)
            k = (K + 1) // 2 if lt else K // 2              # 1-based position of t
            assert v[k - 1] == np.float32(ins["t"])
            assert ins["channel"] == t["nbits"]
            assert s["rank_mask"] & 1 and s["rank_halo"] >= ins["halo"]
    assert n_rank >= len(thr) * 0.9
    assert t["m"] == len(used)      # exactly the thresholds the plan still reads


def test_few_thresholds_and_percentiles_stay_direct():
    plan = vg.compile_formula(_rec(wl.config1_formula()), wl.config1_formula().roots, 8).plan()
    assert plan["rank_tables"] == [] and all(s["kind"] != 6 for s in plan["steps"])
    f = wl.config4_formula()
    plan = vg.compile_formula(_rec(f), f.roots, 8).plan()
    for ins in plan["insns"]:
        if ins["op"] == 1 and ins["slot"] >= 0:
            continue
        assert ins["op"] != 10 or ins["slot"] < 0


@pytest.mark.parametrize("conn", [4, 8])
def test_rank_thresholds_with_ties_signed_zeros_and_nan(conn):
    """Pixel values equal to thresholds, -0.0 against 0.0, NaN pixels: the
    planned rank comparisons give exactly the strict float comparisons."""
    pytest.importorskip("scipy")
    ts = [0.0, -0.0, 0.25, 0.5, 0.5, 0.75, -1.0, 2.0]
    nodes = []
    for k, t in enumerate(ts):
        nodes.append(("THR_GT" if k % 2 == 0 else "THR_LT", -1, -1, 0, 0, t, 0.0))
    nodes.append(("AND", 0, 3, 0, 0, 0, 0))
    nodes.append(("NEAR", 8, -1, 0, 0, 0, 0))
    f = wl.Formula([wl.Node(*n) for n in nodes], list(range(len(nodes))))
    rng = np.random.default_rng(11)
    img = rng.choice(np.array([0.0, -0.0, 0.25, 0.5, 0.75, -1.0, 2.0, 0.3, np.nan, -5.0],
                              dtype=np.float32), size=(1, 37, 140)).astype(np.float32)
    plan = _check_sim(f, [img], conn=conn)
    assert any(ins["op"] == 10 for ins in plan["insns"])


@pytest.mark.parametrize("shuffle", [1, 2, 3])
def test_step_dependencies_allow_any_respecting_order(shuffle):
    """Steps run in a random order that respects the plan's dependencies
    (as the executor may overlap them) still give the oracle's masks: slot
    reuse, select batches and rank codes are all ordered by the dependencies."""
    pytest.importorskip("scipy")
    f = wl.random_dag(2000, seed=shuffle)
    img = wl.uniform_image(40, 300, seed=shuffle)
    plan = _check_sim(f, [img], conn=8, shuffle=shuffle)
    order = plan_sim.random_topological_order(plan, shuffle)
    assert order != list(range(len(order)))  # the order really differs


def test_step_dependencies_with_percentiles_and_masks():
    pytest.importorskip("scipy")
    f = wl.config4_formula()
    img = wl.mri_phantom_batch([(70, 90)], seed=4)[0]
    for k in range(3):
        _check_sim(f, [img], conn=8, shuffle=10 + k)


# ---------------------------------------------------------- number terms --

def _two_channel(h, w, seed):
    return np.stack([wl.gaussian_field_image(h, w, seed=seed)[0], wl.uniform_image(h, w, seed=seed)[0]])


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("conn", [4, 8])
def test_number_terms_plan_matches_oracle(seed, conn):
    """Random formulas with + - * / over two channels, compared by
    percentiles and sign tests: the planned program (one pass over the
    pixels, registers reused) and any dependency-respecting step order give
    the oracle's masks."""
    pytest.importorskip("scipy")
    f = wl.arith_dag(70, seed=seed)
    img = _two_channel(45, 170, seed)
    plan = _check_sim(f, [img], conn=conn)
    assert plan["steps"][0]["kind"] == 7 and plan["arith"]
    for k in range(2):
        _check_sim(f, [img], conn=conn, shuffle=20 + k)


def test_number_terms_on_uint16_images():
    pytest.importorskip("scipy")
    f = wl.arith_dag(50, seed=9)
    img = wl.uniform_image_u16(33, 140, channels=2, seed=9)
    img[:, ::7, ::5] = 0  # quotients 0/0 and x/0: NaN and infinities
    _check_sim(f, [img], conn=8)


def test_comparing_a_channel_value_is_a_plain_threshold():
    """THR(VALUE(i, c)) is the threshold of the channel itself: shared with
    it, and no arithmetic step."""
    rec = [("VALUE", -1, -1, 0, 1, 0, 0), ("THR_GT", 0, -1, 0, 0, 0.5, 0),
           ("THR_GT", -1, -1, 0, 1, 0.5, 0), ("AND", 1, 2, 0, 0, 0, 0),
           ("PCT_LT", 0, -1, 0, 0, 0, 0.25), ("AND", 3, 4, 0, 0, 0, 0)]
    F = vg.compile_formula(rec, [5])
    p = F.plan()
    assert not p["arith"] and all(s["kind"] != 7 for s in p["steps"])
    assert p["pct"][0]["image"] == 0 and p["pct"][0]["channel"] == 1
    thr = [i for i in p["insns"] if i["op"] == 1 and i["slot"] < 0]
    assert len(thr) == 1 and (thr[0]["image"], thr[0]["channel"]) == (0, 1)
    assert F.info()["n_number_images"] == 0


def test_number_images_follow_the_formula_images_and_dead_terms_vanish():
    rec = [("VALUE", -1, -1, 0, 0, 0, 0), ("VALUE", -1, -1, 2, 0, 0, 0),     # images 0 and 2
           ("MUL", 0, 1, 0, 0, 0, 0), ("THR_GT", 2, -1, 0, 0, 0.25, 0),
           ("ADD", 0, -1, 0, 0, 3.0, 0), ("THR_LT", 4, -1, 0, 0, 1.0, 0),      # dead
           ("MASK", -1, -1, 1, 0, 0, 0), ("AND", 3, 6, 0, 0, 0, 0)]
    F = vg.compile_formula(rec, [7])
    p = F.plan()
    assert p["first_number_image"] == 3 and p["n_number_images"] == 1
    assert [a["op"] for a in p["arith"]] == [0, 0, 3, 5]      # value, value, mul, store
    assert all(a["op"] != 1 for a in p["arith"])               # the dead + is gone
    thr = [i for i in p["insns"] if i["op"] == 1]
    assert [i["image"] for i in thr] == [3]
    # the group comparing the number image waits for the arithmetic step
    arith_step = [k for k, s in enumerate(p["steps"]) if s["kind"] == 7][0]
    for k, s in enumerate(p["steps"]):
        if s["kind"] == 1:
            assert arith_step in p["deps"][k]


def test_rank_table_on_a_number_image():
    """Many constant thresholds of one number term share a rank table that
    reads the number image."""
    pytest.importorskip("scipy")
    nodes = [wl.Node("VALUE", channel=0), wl.Node("VALUE", channel=1), wl.Node("SUB", a=0, b=1)]
    ts = [-0.5, -0.25, 0.0, 0.125, 0.25, 0.5]
    for k, t in enumerate(ts):
        nodes.append(wl.Node("THR_GT" if k % 2 else "THR_LT", a=2, t=t))
    nodes.append(wl.Node("AND", a=3, b=4))
    nodes.append(wl.Node("NEAR", a=9))
    f = wl.Formula(nodes, list(range(3, len(nodes))))
    img = _two_channel(40, 260, 4)
    plan = _check_sim(f, [img], conn=8)
    assert plan["rank_tables"] and plan["rank_tables"][0]["image"] == plan["first_number_image"]


@pytest.mark.parametrize("rec,roots", [
    ([("VALUE", -1, -1, 0, 0, 0, 0)], [0]),                                      # number root
    ([("VALUE", -1, -1, 0, 0, 0, 0), ("NEAR", 0, -1, 0, 0, 0, 0)], [1]),         # N of a number
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0), ("MUL", 0, -1, 0, 0, 2, 0),
      ("THR_GT", 1, -1, 0, 0, 0, 0)], [2]),                                     # * of a mask
    ([("THR_GT", -1, -1, 0, 0, 0.5, 0), ("THR_LT", 0, -1, 0, 0, 0, 0)], [1]),   # threshold of a mask
    ([("VALUE", -1, -1, 0, 0, 0, 0), ("ADD", 0, -1, 0, 0, float("nan"), 0),
      ("THR_GT", 1, -1, 0, 0, 0, 0)], [2]),                                     # NaN constant
    ([("VALUE", -1, -1, 0, 0, 0, 0), ("ADD", 0, 5, 0, 0, 0, 0),
      ("THR_GT", 1, -1, 0, 0, 0, 0)], [2]),                                     # operand after node
])
def test_number_terms_and_masks_do_not_mix(rec, roots):
    with pytest.raises(N.VlError) as e:
        vg.compile_formula(rec, roots)
    assert e.value.code == N.ERR_FORMULA


def test_number_terms_register_limit():
    """17 channel values live at once (each summed only at the end) exceed
    the 16 registers of the arithmetic step: a clean compile error; 16 fit."""
    def chain(k):
        # k channel values, summed from the last one back to the first: all
        # k are live when the first add runs
        rec = [("VALUE", -1, -1, 0, c, 0, 0) for c in range(k)]
        acc = k - 1
        for c in range(k - 2, -1, -1):
            rec.append(("ADD", acc, c, 0, 0, 0, 0))
            acc = len(rec) - 1
        rec.append(("THR_GT", acc, -1, 0, 0, 0.0, 0))
        return rec
    p = vg.compile_formula(chain(16), [len(chain(16)) - 1]).plan()
    assert max(a["dst"] for a in p["arith"]) == 15
    with pytest.raises(N.VlError) as e:
        vg.compile_formula(chain(17), [len(chain(17)) - 1])
    assert e.value.code == N.ERR_FORMULA


# ------------------------------------------------ entry points without GPU --

def test_entry_points_reject_null_handles():
    """Every entry point added for uint16 images, number terms and the
    pointer-jumping comparison returns VL_ERR_ARG for a null handle before
    touching the device."""
    lib = N.load()
    out = C.c_void_p()
    i = C.c_int32()
    data = (C.c_uint16 * 4)()
    assert lib.vl_image_create_u16(None, 2, 2, 1, data, 0, None, C.byref(out)) == N.ERR_ARG
    assert lib.vl_image_format(None, C.byref(i)) == N.ERR_ARG
    assert lib.vl_formula_arith(None, None, C.byref(i), None, None) == N.ERR_ARG
    assert lib.vl_ccl_pointer_jumping(None, None, 8, 16, 0, None, None, C.byref(i)) == N.ERR_ARG


def test_number_term_plan_of_a_compiled_formula_without_context():
    """vl_formula_arith on a host-compiled formula: program, number-image
    count and the index of the first number image."""
    f = wl.arith_dag(40, seed=2)
    F = vg.compile_formula(_rec(f), f.roots)
    p = F.plan()
    assert p["arith"][-1]["op"] == 5                      # ends with a store
    assert p["first_number_image"] == 1                    # one float image read
    stores = [a for a in p["arith"] if a["op"] == 5]
    assert sorted(a["image"] for a in stores) == list(range(p["n_number_images"]))
    assert max(a["dst"] for a in p["arith"]) < 16


@pytest.mark.parametrize("mix", ["mixed", "near", "reach"])
@pytest.mark.parametrize("conn", [4, 8])
def test_sequential_chains_plan_matches_oracle(mix, conn):
    """The chains of Sec. 4.1 (tapped every 20 nodes): deep N runs split at
    the halo budget, rho after rho, in listed and random dependency orders."""
    pytest.importorskip("scipy")
    f = wl.sequential_dag(300, seed=7, mix=mix, taps=20)
    img = wl.gaussian_field_image(40, 300, sigma=8.0, seed=7)
    _check_sim(f, [img], conn=conn)
    _check_sim(f, [img], conn=conn, shuffle=3)

@pytest.mark.parametrize("seed", [0, 1])
def test_group_steps_record_the_buffers_they_use(seed):
    """Each group step's n_bufs is one past the highest tile buffer its
    instructions touch (the executor places the shared-memory stage of rank
    planes right after them, so a lower count would let the stage overwrite
    a live buffer)."""
    f = wl.random_dag(2000, seed=seed)
    p = vg.compile_formula(_rec(f), f.roots, 8).plan()
    ins = p["insns"]
    groups = [s for s in p["steps"] if s["kind"] == 1]
    assert groups
    for s in groups:
        hi = 0
        for i in ins[s["insn_off"]:s["insn_off"] + s["insn_cnt"]]:
            op = i["op"]
            if op != 8:                      # every op but the store writes dst
                hi = max(hi, i["dst"] + 1)
            if op in (3, 4, 5, 6, 8, 9):     # not, and, or, N, store, and-not read a
                hi = max(hi, i["a"] + 1)
            if op in (4, 5, 9):              # and, or, and-not read b
                hi = max(hi, i["b"] + 1)
        assert s["n_bufs"] == hi, (s, hi)
    for s in p["steps"]:
        if s["kind"] != 1:
            assert s["n_bufs"] == 0
