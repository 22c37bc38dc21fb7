"""Expansion of derived connectives into the primitive grammar, with
structural sharing -- oracle side (test infrastructure only).

The primitive grammar is Eq. (1) of Sec. 2: p | not | and | N | rho.  The paper
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

Number terms (the tool offers basic arithmetic beside the SLCS primitives,
on 16-bit unsigned images, Sec. 3): VALUE reads one channel of an image as
numbers (uint16 pixels are their integer values);
ADD / SUB / MUL / DIV combine two number terms, or a term and the float32
constant t (when b = -1), pixel by pixel in IEEE-754 binary32 with
round-to-nearest-even.  A threshold or percentile atom whose a >= 0 compares
the number term a instead of an image channel.  Masks and numbers do not
mix: boolean connectives take masks, arithmetic takes numbers, roots are
masks.

Sharing: a node is identified by its operator, its (already shared) operand
ids and, for atoms, its parameters; two identical nodes become one.  No
algebraic rewriting (double negation, commutativity, idempotence) is done.
"""
from __future__ import annotations

import struct
from typing import Dict, List, Sequence, Tuple

PRIMS = ("TRUE", "FALSE", "THR_GT", "THR_LT", "PCT_GT", "PCT_LT", "MASK",
         "NOT", "AND", "NEAR", "REACH", "VALUE", "ADD", "SUB", "MUL", "DIV")
ATOMS = ("TRUE", "FALSE", "THR_GT", "THR_LT", "PCT_GT", "PCT_LT", "MASK")
ARITH = ("ADD", "SUB", "MUL", "DIV")
NUMBER_OPS = ("VALUE",) + ARITH

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
            if a >= 0:
                return (op, "number", a, struct.pack("<f", t))
            return (op, img, ch, struct.pack("<f", t))
        if op in ("PCT_GT", "PCT_LT"):
            if a >= 0:
                return (op, "number", a, struct.pack("<d", q))
            return (op, img, ch, struct.pack("<d", q))
        if op == "VALUE":
            return (op, img, ch)
        if op in ARITH and b < 0:
            return (op, a, "const", struct.pack("<f", t))
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
    number: List[bool] = []   # is node i a number term
    for i, nd in enumerate(nodes):
        op, a, b, img, ch, t, q = tuple(nd)
        a, b = int(a), int(b)
        if op in ATOMS:
            if op in ("THR_GT", "THR_LT", "PCT_GT", "PCT_LT") and a >= 0:
                if not (a < i and number[a]):
                    raise ValueError(f"node {i}: a threshold operand must be an earlier number term")
                ids.append(bld.add(op, a=ids[a], t=float(t), q=float(q)))
            else:
                ids.append(bld.add(op, image=int(img), channel=int(ch),
                                   t=float(t), q=float(q)))
            number.append(False)
            continue
        if op == "VALUE":
            ids.append(bld.add(op, image=int(img), channel=int(ch)))
            number.append(True)
            continue
        if op in ARITH:
            if not (0 <= a < i and number[a]) or (b >= 0 and not (b < i and number[b])):
                raise ValueError(f"node {i}: arithmetic operands must be earlier number terms")
            ids.append(bld.add(op, a=ids[a], b=ids[b] if b >= 0 else -1,
                               t=float(t) if b < 0 else 0.0))
            number.append(True)
            continue
        if not (0 <= a < i) or (op not in ("NOT", "NEAR", "INTERIOR") and not (0 <= b < i)):
            raise ValueError(f"node {i}: operands must precede the node")
        if number[a] or (op not in ("NOT", "NEAR", "INTERIOR") and number[b]):
            raise ValueError(f"node {i}: a connective needs masks, not number terms")
        A = ids[a]
        B = ids[b] if b >= 0 else -1
        fn = getattr(bld, op, None)
        if fn is None:
            raise ValueError(f"node {i}: unknown operator {op}")
        ids.append(fn(A) if op in ("NOT", "NEAR", "INTERIOR") else fn(A, B))
        number.append(False)
    for r in roots:
        if number[r]:
            raise ValueError(f"root {r} is a number term, not a mask")
    return bld.nodes, [ids[r] for r in roots]
