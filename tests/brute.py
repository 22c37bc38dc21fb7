"""Brute-force and textbook checkers used to pin the oracle.

Nothing here calls the oracle or the CUDA library; every function restates a
definition of the paper directly (path enumeration, matrix closure) or is a
textbook routine (two-pass labelling), for tiny inputs only.
"""
from __future__ import annotations

import itertools
from collections import defaultdict
from typing import Dict, List, Tuple

import numpy as np


def neighbours(H: int, W: int, conn: int) -> List[List[int]]:
    """Adjacency lists (pixel itself excluded) of the H x W grid."""
    out = []
    for y in range(H):
        for x in range(W):
            lst = []
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dy == 0 and dx == 0:
                        continue
                    if conn == 4 and dy != 0 and dx != 0:
                        continue
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W:
                        lst.append(yy * W + xx)
            out.append(lst)
    return out


def adjacency_matrix(H: int, W: int, conn: int) -> np.ndarray:
    n = H * W
    A = np.zeros((n, n), dtype=bool)
    for v, lst in enumerate(neighbours(H, W, conn)):
        A[v, lst] = True
    return A


# ------------------------------------------------------ path enumeration ---

def simple_path_table(H: int, W: int, conn: int) -> Dict[Tuple[int, int], List[int]]:
    """For every ordered pair (x, y), x != y, the minimal sets (bitmasks over
    pixels) of intermediate pixels pi_1..pi_{l-1} over all simple paths
    x = pi_0, ..., pi_l = y.  Exhaustive DFS: only for grids of <= 9 pixels."""
    nb = neighbours(H, W, conn)
    table: Dict[Tuple[int, int], set] = defaultdict(set)

    def dfs(x: int, cur: int, visited: int, inner: int) -> None:
        for u in nb[cur]:
            if visited >> u & 1:
                continue
            table[(x, u)].add(inner)
            dfs(x, u, visited | (1 << u), inner | (1 << u))

    for x in range(H * W):
        dfs(x, x, 1 << x, 0)
    out = {}
    for k, sets in table.items():
        s = sorted(sets, key=lambda m: bin(m).count("1"))
        minimal: List[int] = []
        for m in s:
            if not any((mm & m) == mm for mm in minimal):
                minimal.append(m)
        out[k] = minimal
    return out


def reach_relation(table, n: int, phi2_bits: int) -> np.ndarray:
    """rel[x, y]: a path from x to y exists whose intermediates are phi2."""
    rel = np.zeros((n, n), dtype=bool)
    for (x, y), sets in table.items():
        if any((m & ~phi2_bits) == 0 for m in sets):
            rel[x, y] = True
    return rel


def reach_by_paths(phi1: np.ndarray, phi2: np.ndarray, conn: int) -> np.ndarray:
    """rho phi1[phi2] by DFS over simple paths from each pixel (Sec. 2: pi_0 =
    x, pi_l in phi1, pi_1..pi_{l-1} in phi2).  Walks with repeats shortcut to
    simple paths with fewer intermediates, so simple paths suffice."""
    H, W = phi1.shape
    f1 = phi1.ravel().astype(bool)
    f2 = phi2.ravel().astype(bool)
    nb = neighbours(H, W, conn)
    out = np.zeros(H * W, dtype=np.uint8)

    def dfs(cur: int, visited: int) -> bool:
        for u in nb[cur]:
            if visited >> u & 1:
                continue
            if f1[u]:
                return True
            if f2[u] and dfs(u, visited | (1 << u)):
                return True
        return False

    for x in range(H * W):
        out[x] = 1 if (f1[x] or dfs(x, 1 << x)) else 0
    return out.reshape(H, W)


def touch_by_paths(phi1: np.ndarray, phi2: np.ndarray, conn: int) -> np.ndarray:
    """Contact by its meaning: x is in phi1 and a path pi_0 = x, ..., pi_l
    (l >= 0) exists that stays inside phi1 up to pi_{l-1} and ends on a phi2
    pixel pi_l -- phi1's region around x meets phi2 or borders it (Sec. 2
    names contact among the derived connectives).  DFS over phi1 pixels."""
    H, W = phi1.shape
    f1 = phi1.ravel().astype(bool)
    f2 = phi2.ravel().astype(bool)
    nb = neighbours(H, W, conn)
    out = np.zeros(H * W, dtype=np.uint8)
    for x in range(H * W):
        if not f1[x]:
            continue
        seen = {x}
        stack = [x]
        hit = False
        while stack and not hit:
            v = stack.pop()
            if f2[v]:
                hit = True
                break
            for u in nb[v]:
                if f2[u]:
                    hit = True
                    break
                if f1[u] and u not in seen:
                    seen.add(u)
                    stack.append(u)
        out[x] = 1 if hit else 0
    return out.reshape(H, W)


def surrounded_by_paths(phi1: np.ndarray, phi2: np.ndarray, conn: int) -> np.ndarray:
    """Direct definition: x in phi1 and no path pi from x with l >= 1,
    pi_1..pi_l outside phi2 and pi_l outside phi1 (every way out of phi1
    meets phi2)."""
    H, W = phi1.shape
    f1 = phi1.ravel().astype(bool)
    f2 = phi2.ravel().astype(bool)
    nb = neighbours(H, W, conn)
    out = np.zeros(H * W, dtype=np.uint8)

    def escapes(cur: int, visited: int) -> bool:
        for u in nb[cur]:
            if visited >> u & 1 or f2[u]:
                continue
            if not f1[u]:
                return True
            if escapes(u, visited | (1 << u)):
                return True
        return False

    for x in range(H * W):
        out[x] = 1 if (f1[x] and not escapes(x, 1 << x)) else 0
    return out.reshape(H, W)


# ------------------------------------------------------ matrix closures ---

def closure(M: np.ndarray) -> np.ndarray:
    """Reflexive-transitive closure of a boolean relation by squaring."""
    n = M.shape[0]
    T = M | np.eye(n, dtype=bool)
    while True:
        T2 = T | ((T.astype(np.uint8) @ T.astype(np.uint8)) > 0)
        if (T2 == T).all():
            return T
        T = T2


def reach_by_matrix(phi1: np.ndarray, phi2: np.ndarray, conn: int) -> np.ndarray:
    """rho via relation algebra: x reaches phi1 directly (l <= 1) or steps to a
    phi2 pixel u, walks inside phi2 to v, and steps from v into phi1."""
    H, W = phi1.shape
    A = adjacency_matrix(H, W, conn)
    f1 = phi1.ravel().astype(bool)
    f2 = phi2.ravel().astype(bool)
    inner = A & f2[:, None] & f2[None, :]
    T = closure(inner) & f2[:, None] & f2[None, :]
    u8 = lambda m: m.astype(np.uint8)
    step1 = (u8(A) @ u8(f1)) > 0                        # l = 1
    into_phi1 = (u8(A) @ u8(f1)) > 0                     # v adjacent to phi1
    via = (u8(A & f2[None, :]) @ u8((u8(T) @ u8(into_phi1 & f2)) > 0)) > 0
    return (f1 | step1 | via).astype(np.uint8).reshape(H, W)


# ---------------------------------------------------- textbook labelling ---

def two_pass_label(m: np.ndarray, conn: int) -> np.ndarray:
    """Classic two-pass labelling (raster scan with an equivalence table, then
    relabelling); returns labels 1..k in first-scan order, 0 background."""
    H, W = m.shape
    lab = np.zeros((H, W), dtype=np.int64)
    parent = [0]

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    def union(a, b):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)

    prev = [(-1, 0), (0, -1)] if conn == 4 else [(-1, -1), (-1, 0), (-1, 1), (0, -1)]
    for y in range(H):
        for x in range(W):
            if not m[y, x]:
                continue
            ls = []
            for dy, dx in prev:
                yy, xx = y + dy, x + dx
                if 0 <= yy < H and 0 <= xx < W and lab[yy, xx]:
                    ls.append(lab[yy, xx])
            if not ls:
                parent.append(len(parent))
                lab[y, x] = len(parent) - 1
            else:
                lab[y, x] = min(ls)
                for l in ls:
                    union(lab[y, x], l)
    out = np.zeros_like(lab)
    remap = {}
    for y in range(H):
        for x in range(W):
            if lab[y, x]:
                r = find(lab[y, x])
                if r not in remap:
                    remap[r] = len(remap) + 1
                out[y, x] = remap[r]
    return out


def canonical_min_index(lab: np.ndarray, background: int = 0) -> np.ndarray:
    """Rename each component to its minimum linear index; background -> -1."""
    flat = lab.ravel()
    out = np.full(flat.shape, -1, dtype=np.int64)
    first = {}
    for i, v in enumerate(flat):
        if v == background:
            continue
        if v not in first:
            first[v] = i
        out[i] = first[v]
    return out.reshape(lab.shape)


def same_partition(a: np.ndarray, b: np.ndarray, bg_a: int, bg_b: int) -> bool:
    """Two labellings describe the same partition (background matched)."""
    fa, fb = a.ravel(), b.ravel()
    if not np.array_equal(fa == bg_a, fb == bg_b):
        return False
    fwd, bwd = {}, {}
    for x, y in zip(fa.tolist(), fb.tolist()):
        if x == bg_a:
            continue
        if fwd.setdefault(x, y) != y or bwd.setdefault(y, x) != x:
            return False
    return True


# ------------------------------------------------------------ fixtures ---

def all_masks(H: int, W: int):
    n = H * W
    for bits in range(1 << n):
        yield bits, np.array([(bits >> i) & 1 for i in range(n)],
                             dtype=np.uint8).reshape(H, W)


def bits_to_mask(bits: int, H: int, W: int) -> np.ndarray:
    return np.array([(bits >> i) & 1 for i in range(H * W)], dtype=np.uint8).reshape(H, W)


# ------------------------------------------------------------ 3D volumes ---

def neighbours3(D: int, H: int, W: int, conn: int) -> List[List[int]]:
    """Adjacency lists (voxel itself excluded) of a D x H x W volume: 26 =
    every voxel of the 3x3x3 cube around, 6 = the voxels sharing a face."""
    out = []
    for z in range(D):
        for y in range(H):
            for x in range(W):
                lst = []
                for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
                    if (dz, dy, dx) == (0, 0, 0):
                        continue
                    if conn == 6 and abs(dz) + abs(dy) + abs(dx) != 1:
                        continue
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if 0 <= zz < D and 0 <= yy < H and 0 <= xx < W:
                        lst.append((zz * H + yy) * W + xx)
                out.append(lst)
    return out


def reach_by_paths_nb(f1: np.ndarray, f2: np.ndarray, nb: List[List[int]]) -> np.ndarray:
    """rho phi1[phi2] on any graph given by adjacency lists, by DFS over
    simple paths (flat 0/1 arrays)."""
    n = len(nb)
    f1 = f1.astype(bool)
    f2 = f2.astype(bool)
    out = np.zeros(n, dtype=np.uint8)

    def dfs(cur: int, visited: int) -> bool:
        for u in nb[cur]:
            if visited >> u & 1:
                continue
            if f1[u]:
                return True
            if f2[u] and dfs(u, visited | (1 << u)):
                return True
        return False

    for x in range(n):
        out[x] = 1 if (f1[x] or dfs(x, 1 << x)) else 0
    return out


def components_nb(m: np.ndarray, nb: List[List[int]]) -> np.ndarray:
    """Component ids by repeated relaxation to the minimum index over the
    graph's edges until nothing changes (a fixed-point definition, no queue):
    label = minimum index of the component, background -1."""
    f = m.astype(bool)
    lab = np.where(f, np.arange(len(nb)), -1)
    changed = True
    while changed:
        changed = False
        for v in range(len(nb)):
            if not f[v]:
                continue
            for u in nb[v]:
                if f[u] and lab[u] < lab[v]:
                    lab[v] = lab[u]
                    changed = True
    return lab
