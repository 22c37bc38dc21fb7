"""Tile-accurate CPU simulation of a compiled plan (test infrastructure).

It runs the host compiler's output -- steps, group instructions with their
halos, slots and selects -- the way the executor does, tile by tile, but in
numpy on boolean pixel arrays.  Buffer rows a tile has not computed hold
random garbage, so an instruction that reads outside its operand's computed
halo shows up as a wrong result.  Component selects use scipy's labelling.
This checks the compiler (expansion, lowering, grouping, halos, slot
liveness), not the CUDA kernels.
"""
from __future__ import annotations

import numpy as np

GTH, GTWW = 32, 32  # default context tile: rows, 32-px words


def _dilate(a: np.ndarray, conn: int) -> np.ndarray:
    """Dilation inside the array; outside counts as false."""
    p = np.pad(a, 1)
    out = a.copy()
    H, W = a.shape
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if conn == 4 and dy and dx:
                continue
            out |= p[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    return out


def _select(phi1, phi2, conn):
    import scipy.ndimage as nd
    st = np.ones((3, 3), bool) if conn == 8 else nd.generate_binary_structure(2, 1)
    lab, _ = nd.label(phi2, structure=st)
    hit = np.unique(lab[_dilate(phi1, conn) & (lab > 0)])
    return np.isin(lab, hit) & (lab > 0)


def random_topological_order(plan: dict, seed: int):
    """A random order of the plan's steps that respects its dependencies
    (what the persistent executor may run, step by step)."""
    rng = np.random.default_rng(seed)
    deps = plan["deps"]
    n = len(deps)
    users = [[] for _ in range(n)]
    indeg = [len(set(d)) for d in deps]
    for s, d in enumerate(deps):
        for x in set(d):
            users[x].append(s)
    ready = [s for s in range(n) if indeg[s] == 0]
    order = []
    while ready:
        k = int(rng.integers(0, len(ready)))
        s = ready.pop(k)
        order.append(s)
        for u in users[s]:
            indeg[u] -= 1
            if indeg[u] == 0:
                ready.append(u)
    assert len(order) == n, "dependency cycle"
    return order


def simulate(plan: dict, images, masks_by_image: dict, conn: int, seed: int = 0,
             tile_rows: int = GTH, tile_words: int = GTWW, order=None):
    """images: list of (C, H, W) float32 arrays (None for mask images);
    masks_by_image: {image index: (H, W) bool}.  Steps run in `order` (default:
    the listed order).  Returns one bool mask per root."""
    rng = np.random.default_rng(seed)
    some = next(x for x in images if x is not None) if any(x is not None for x in images) else None
    H, W = some.shape[1:] if some is not None else next(iter(masks_by_image.values())).shape
    Wp = ((W + 127) // 128) * 4
    sz = plan["sizes"]
    n_slots = sz["n_inter_slots"] + sz["n_root_slots"] + sz["n_mask_slots"]
    GARB = object()
    slots = [GARB] * n_slots
    base_mask = sz["n_inter_slots"] + sz["n_root_slots"]
    for k, img in enumerate(plan["mask_slot_images"]):
        slots[base_mask + k] = masks_by_image[img].astype(bool)
    # number images (step kind 7) follow the formula's own images
    first_num = plan.get("first_number_image", len(images))
    nums = {}

    def img_of(k):
        if k >= first_num:
            if k - first_num not in nums:
                raise AssertionError("a number image is read before the step that writes it")
            return nums[k - first_num]
        return np.asarray(images[k], dtype=np.float32)

    pct = {}
    insns = plan["insns"]
    sels = plan["selects"]
    pending_sel = {}
    for si in (order if order is not None else range(len(plan["steps"]))):
        st = plan["steps"][si]
        kind = st["kind"]
        if kind == 7:  # number terms: the program on every pixel, in float32
            regs = {}
            for A in plan["arith"]:
                if A["op"] == 0:
                    regs[A["dst"]] = img_of(A["image"])[A["channel"]].astype(np.float32)
                elif A["op"] == 5:
                    nums[A["image"]] = regs[A["a"]][None].copy()
                else:
                    u = regs[A["a"]]
                    w = np.float32(A["c"]) if A["b"] == 255 else regs[A["b"]]
                    with np.errstate(all="ignore"):
                        regs[A["dst"]] = {1: np.add, 2: np.subtract, 3: np.multiply,
                                          4: np.divide}[A["op"]](u, w).astype(np.float32)
            continue
        if kind == 0:  # percentiles (numpy sorts NaN last)
            for d in plan["pct"]:
                v = np.sort(img_of(d["image"])[d["channel"]].ravel())
                pct[d["slot"]] = v[int(np.floor(d["q"] * (v.size - 1)))]
            continue
        if kind == 1:
            halo = st["halo"]
            prog = insns[st["insn_off"]:st["insn_off"] + st["insn_cnt"]]
            outs = {}
            for r0 in range(0, H, tile_rows):
                th = min(tile_rows, H - r0)
                for w0 in range(0, Wp, tile_words):
                    tww = min(tile_words, Wp - w0)
                    x0 = 32 * w0
                    bh, bwpx = th + 2 * halo, 32 * (tww + 2)
                    rows = np.arange(r0 - halo, r0 - halo + bh)
                    cols = np.arange(x0 - 32, x0 - 32 + bwpx)
                    inimg = ((rows >= 0) & (rows < H))[:, None] & ((cols >= 0) & (cols < W))[None, :]
                    rr = np.clip(rows, 0, H - 1)
                    cc = np.clip(cols, 0, W - 1)
                    bufs = {}

                    def buf(b):
                        if b not in bufs:
                            bufs[b] = rng.random((bh, bwpx)) < 0.5
                        return bufs[b]

                    for ins in prog:
                        op, h = ins["op"], ins["halo"]
                        lo, hi = halo - h, halo + th + h
                        if op == 8:  # store core
                            s = ins["slot"]
                            if slots[s] is GARB or not isinstance(slots[s], np.ndarray):
                                slots[s] = rng.random((H, W)) < 0.5
                            a = buf(ins["a"])
                            cw = min(32 * tww, W - x0)
                            slots[s][r0:r0 + th, x0:x0 + cw] = a[halo:halo + th, 32:32 + cw]
                            outs[s] = True
                            continue
                        if op == 1:
                            ch = img_of(ins["image"])[ins["channel"]]
                            if ins["slot"] >= 0 and ins["slot"] not in pct:
                                raise AssertionError(f"step {si}: percentile read before it is computed")
                            t = pct[ins["slot"]] if ins["slot"] >= 0 else np.float32(ins["t"])
                            v = ch[rr][:, cc]
                            val = (v < t) if ins["b"] & 1 else (v > t)
                        elif op == 10:  # threshold by rank code
                            tab = plan["rank_tables"][ins["a"]]
                            vals = plan["rank_values"][tab["value_off"]:tab["value_off"] + tab["m"]]
                            v = img_of(tab["image"])[tab["channel"]][rr][:, cc]
                            nan = np.isnan(v)
                            below = np.searchsorted(vals, np.where(nan, 0, v), side="left")
                            hit = vals[np.minimum(below, tab["m"] - 1)] == v
                            code = np.where(nan, 0, 2 * below + ((below < tab["m"]) & hit))
                            ge = code >= (ins["image"] & 0xFFFF)
                            val = (~ge & ~nan) if ins["b"] & 1 else ge
                        elif op == 2:
                            src = slots[ins["slot"]]
                            if src is GARB:
                                raise AssertionError(f"step {si}: load of a slot never written")
                            val = src[rr][:, cc]
                        elif op == 3:
                            val = ~buf(ins["a"])
                        elif op == 4:
                            val = buf(ins["a"]) & buf(ins["b"])
                        elif op == 5:
                            val = buf(ins["a"]) | buf(ins["b"])
                        elif op == 9:
                            val = buf(ins["a"]) & ~buf(ins["b"])
                        elif op == 6:
                            a = buf(ins["a"]).copy()
                            val = _dilate(a, conn)
                        elif op == 7:
                            val = np.full((bh, bwpx), bool(ins["b"]))
                        else:
                            raise AssertionError(f"unknown op {op}")
                        val = val & inimg
                        d = buf(ins["dst"]).copy()
                        d[lo:hi] = val[lo:hi]
                        bufs[ins["dst"]] = d
        elif kind == 2:  # select batch, first pass: inputs are read here
            for j in range(st["sel_cnt"]):
                s = sels[st["sel_off"] + j]
                a, b = slots[s["phi1_slot"]], slots[s["phi2_slot"]]
                if a is GARB or b is GARB:
                    raise AssertionError(f"step {si}: select reads an unwritten slot")
                pending_sel[st["sel_off"] + j] = (a.copy(), b.copy())
        elif kind == 5:  # final pass: inputs must be unchanged, Z written
            for j in range(st["sel_cnt"]):
                k = st["sel_off"] + j
                s = sels[k]
                a0, b0 = pending_sel.pop(k)
                if not (np.array_equal(a0, slots[s["phi1_slot"]]) and
                        np.array_equal(b0, slots[s["phi2_slot"]])):
                    raise AssertionError(f"step {si}: select input overwritten mid-select")
                slots[s["z_slot"]] = _select(a0, b0, conn)
    return [slots[s].copy() for s in plan["root_slots"]]
