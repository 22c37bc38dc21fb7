"""Expansion of derived connectives into the primitive grammar, with
structural sharing -- oracle side (test infrastructure only).

The primitive grammar is Eq. (def:syntax): p | not | and | N | rho.  The paper
names interior, surroundedness, contact (Sec. 2) and grow (Sec. 4.2) as derived
from these without printing the formulas; the definitions used here are the
readings listed below.

  or(a, b)          = not(and(not a, not b))
  interior(a)       = not N not a                       (erosion, Sec. 2)
  surrounded(a, b)  = a and not rho(not(a or b))[not b]
      x satisfies it iff x |= a and every path leaving a passes through b
      before (or when) it reaches a pixel outside a.
  grow(a, b)        = a or (b and rho a[b])             (Sec. 4.2: a's
      pixels, plus the b-regions in contact with a)
  touch(a, b)       = a and rho b[a]

Sharing: a node is identified by its operator, its (already shared) operand
ids and, for atoms, its parameters; two identical nodes become one.  No
algebraic rewriting (double negation, commutativity, idempotence) is done.
"""
from __future__ import annotations

import struct
from typing import Dict, List, Sequence, Tuple

PRIMS = ("TRUE", "FALSE", "THR_GT", "THR_LT", "PCT_GT", "PCT_LT", "MASK",
         "NOT", "AND", "NEAR", "REACH")
ATOMS = ("TRUE", "FALSE", "THR_GT", "THR_LT", "PCT_GT", "PCT_LT", "MASK")

# A primitive node: (op, a, b, image, channel, t, q)
PNode = Tuple[str, int, int, int, int, float, float]


class _Builder:
    def __init__(self) -> None:
        self.nodes: List[PNode] = []
        self.index: Dict[tuple, int] = {}

    def _key(self, nd: PNode) -> tuple:
        op, a, b, img, ch, t, q = nd
        if op in ("TRUE", "FALSE"):
            return (op,)
        if op == "MASK":
            return (op, img)
        if op in ("THR_GT", "THR_LT"):
            return (op, img, ch, struct.pack("<f", t))
        if op in ("PCT_GT", "PCT_LT"):
            return (op, img, ch, struct.pack("<d", q))
        return (op, a, b)

    def add(self, op: str, a: int = -1, b: int = -1, image: int = 0,
            channel: int = 0, t: float = 0.0, q: float = 0.0) -> int:
        nd = (op, a, b, image, channel, t, q)
        k = self._key(nd)
        if k in self.index:
            return self.index[k]
        self.nodes.append(nd)
        self.index[k] = len(self.nodes) - 1
        return self.index[k]

    # derived connectives ------------------------------------------------
    def NOT(self, a):
        return self.add("NOT", a)

    def AND(self, a, b):
        return self.add("AND", a, b)

    def OR(self, a, b):
        return self.NOT(self.AND(self.NOT(a), self.NOT(b)))

    def NEAR(self, a):
        return self.add("NEAR", a)

    def REACH(self, a, b):
        return self.add("REACH", a, b)

    def INTERIOR(self, a):
        return self.NOT(self.NEAR(self.NOT(a)))

    def SURROUNDED(self, a, b):
        return self.AND(a, self.NOT(self.REACH(self.NOT(self.OR(a, b)), self.NOT(b))))

    def GROW(self, a, b):
        return self.OR(a, self.AND(b, self.REACH(a, b)))

    def TOUCH(self, a, b):
        return self.AND(a, self.REACH(b, a))


def expand(nodes: Sequence, roots: Sequence[int]):
    """Return (primitive nodes, root ids).  ``nodes`` are records with fields
    (op, a, b, image, channel, t, q) in topological order."""
    bld = _Builder()
    ids: List[int] = []
    for i, nd in enumerate(nodes):
        op, a, b, img, ch, t, q = tuple(nd)
        if op in ATOMS:
            ids.append(bld.add(op, image=int(img), channel=int(ch),
                               t=float(t), q=float(q)))
            continue
        if not (0 <= a < i) or (op not in ("NOT", "NEAR", "INTERIOR") and not (0 <= b < i)):
            raise ValueError(f"node {i}: operands must precede the node")
        A = ids[a]
        B = ids[b] if b >= 0 else -1
        fn = getattr(bld, op, None)
        if fn is None:
            raise ValueError(f"node {i}: unknown operator {op}")
        ids.append(fn(A) if op in ("NOT", "NEAR", "INTERIOR") else fn(A, B))
    return bld.nodes, [ids[r] for r in roots]
