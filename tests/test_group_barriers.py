"""Barrier placement inside fused groups, checked on the CPU.

The group interpreter gives every shared-memory buffer word one owning
thread (word i * bw + j belongs to thread (i * bw + j) mod 512), and the
compiler puts a block barrier (opcode bit 7) before an instruction only
where some thread could touch a word that another thread touched since the
previous barrier.  This test replays every group of a plan word by word
under that ownership -- pointwise ops, loads, constants and rank thresholds
read and write their own words, N reads the 3 x 3 words around its own, a
store reads the core words it owns, the float threshold writes its words
from other lanes -- and reports any read after a write, write after a read,
or write after a write of one word by two threads with no barrier between.
It runs over the tile shapes the autotuner tries: the fixed ones, the
one-wave shapes it adds for a single job (on a 2048 x 2048 image 14 x 32
and 27 x 16), and short last tile rows (an image height that is not a
multiple of the tile height).
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl
import paper_2010_07284_gb300 as vg
from test_compiler_fuzz import random_formula

NT = 512
HMAX = 8
SHAPES = [(32, 32), (64, 16), (32, 16), (16, 32), (16, 16), (64, 8), (32, 8), (16, 8),
          (14, 32), (27, 16), (4, 32), (1, 16)]
OWN_WRITE = {1: False, 2: True, 3: True, 4: True, 5: True, 6: True, 7: True, 9: True, 10: True}


def hazards(plan: dict, th: int, tww: int):
    """Yield (step, instruction, what) for every unsynchronised conflict."""
    bw = tww + 2
    for si, st in enumerate(plan["steps"]):
        if st["kind"] != 1:
            continue
        halo = st["halo"]
        bh = th + 2 * halo
        n = bh * bw
        owner = np.arange(n) % NT
        writer = {}      # buffer -> int8 per word: 0 none, 1 owner, 2 another thread
        rd_own = {}      # buffer -> bool per word: read by its owner
        rd_other = {}    # buffer -> bool per word: read by another thread

        def arr(d, b, dtype):
            if b not in d:
                d[b] = np.zeros(n, dtype)
            return d[b]

        rows = np.arange(n) // bw
        cols = np.arange(n) % bw
        for k in range(st["insn_off"], st["insn_off"] + st["insn_cnt"]):
            ins = plan["insns"][k]
            if ins["sync"]:
                writer.clear(); rd_own.clear(); rd_other.clear()
            op, h = ins["op"], ins["halo"]
            lo, hi = halo - h, halo + th + h
            inr = (rows >= lo) & (rows < hi)
            if op == 8:  # store: reads core words, own mapping
                core = (rows >= halo) & (rows < halo + th) & (cols >= 1) & (cols <= tww)
                w = arr(writer, ins["a"], np.int8)
                if np.any(core & (w == 2)):
                    yield si, k, "store reads a word another thread wrote"
                arr(rd_own, ins["a"], bool)[core] = True
                continue
            reads = []
            if op in (3, 4, 5, 9):
                reads = [ins["a"]] + ([ins["b"]] if op in (4, 5, 9) else [])
            for b in reads:
                if np.any(inr & (arr(writer, b, np.int8) == 2)):
                    yield si, k, f"reads buffer {b} written by another thread"
                arr(rd_own, b, bool)[inr] = True
            if op == 6:  # N: the 3 x 3 words around each own word
                b = ins["a"]
                w = arr(writer, b, np.int8)
                if np.any(inr & (w == 2)):
                    yield si, k, "N reads its centre written by another thread"
                nb = np.zeros(n, bool)
                for di in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        if di == 0 and dj == 0:
                            continue
                        ok = inr & (cols + dj >= 0) & (cols + dj < bw) & (rows + di >= 0) & (rows + di < bh)
                        nb[np.flatnonzero(ok) + di * bw + dj] = True
                if np.any(nb & (w != 0)):
                    yield si, k, "N reads neighbour words written since the last barrier"
                arr(rd_other, b, bool)[nb] = True
                arr(rd_own, b, bool)[inr] = True
            d = ins["dst"]
            w = arr(writer, d, np.int8)
            if OWN_WRITE[op]:
                if np.any(inr & ((w == 2) | arr(rd_other, d, bool))):
                    yield si, k, f"writes buffer {d} another thread touched"
                w[inr & (w == 0)] = 1
            else:
                if np.any(inr & ((w != 0) | arr(rd_own, d, bool) | arr(rd_other, d, bool))):
                    yield si, k, f"threshold writes buffer {d} touched since the last barrier"
                w[inr] = 2


def _plans():
    out = []
    f = wl.random_dag(2000, seed=0)
    out.append(("random-2000", vg.compile_formula(wl.formula_to_records(f), f.roots, 8).plan()))
    f = wl.config4_formula()
    out.append(("mri-40", vg.compile_formula(wl.formula_to_records(f), f.roots, 8).plan()))
    f = wl.sequential_dag(300, seed=1, mix="near")
    out.append(("deep-N", vg.compile_formula(wl.formula_to_records(f), f.roots, 4).plan()))
    for seed in range(30):
        rng = np.random.default_rng(1000 + seed)
        nch = int(rng.integers(1, 3))
        recs, roots = random_formula(rng, int(rng.integers(5, 90)), nch, seed % 3 == 0)
        out.append((f"fuzz-{seed}", vg.compile_formula(recs, roots, 8 if seed % 2 == 0 else 4).plan()))
    return out


@pytest.fixture(scope="module")
def plans():
    return _plans()


@pytest.mark.parametrize("shape", SHAPES)
def test_no_unsynchronised_conflicts(plans, shape):
    for name, plan in plans:
        bad = list(hazards(plan, *shape))
        assert not bad, f"{name} tile {shape}: {bad[:3]}"


def test_barriers_are_elided_and_the_checker_sees_missing_ones(plans):
    name, plan = plans[0]
    n = sum(1 for st in plan["steps"] if st["kind"] == 1
            for k in range(st["insn_off"], st["insn_off"] + st["insn_cnt"]))
    syncs = sum(1 for ins in plan["insns"] if ins["sync"])
    assert syncs < n // 2, f"{syncs} barriers for {n} group instructions"
    # without any barrier the replay must find conflicts
    bare = dict(plan, insns=[dict(i, sync=False) for i in plan["insns"]])
    assert any(True for _ in hazards(bare, 16, 32))
