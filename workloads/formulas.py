"""Formula DAGs shaped like the paper's test formulas.

Grammar of the logic (Eq. (1) of Sec. 2): p | not phi | phi1 and phi2 |
N phi | rho phi1[phi2].  Atomic propositions are thresholds on an image
feature (Sec. 2 and the segmentation spec of Fig. "specification").  Derived
connectives (interior, surrounded, grow, touch, or) are kept as named nodes
here: each evaluator expands them with its own code.

A node is ``Node(op, a, b, image, channel, t, q)``:
  * op       -- one of ``OPS``
  * a, b     -- operand node indices (< own index), -1 when unused
  * image    -- which input image an atom reads (index into the image list)
  * channel  -- which channel of that image an atom reads
  * t        -- threshold constant, already rounded to float32
  * q        -- percentile level in [0, 1] for PCT_* atoms (float64)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, NamedTuple

import numpy as np

PRIMITIVE_OPS = ("TRUE", "FALSE", "THR_GT", "THR_LT", "PCT_GT", "PCT_LT",
                 "MASK", "NOT", "AND", "NEAR", "REACH")
DERIVED_OPS = ("OR", "INTERIOR", "SURROUNDED", "GROW", "TOUCH")
# number terms: VALUE reads a channel; ADD/SUB/MUL/DIV take two terms, or a
# term and the constant t when b = -1; THR_*/PCT_* with a >= 0 compare term a
NUMBER_OPS = ("VALUE", "ADD", "SUB", "MUL", "DIV")
OPS = PRIMITIVE_OPS + DERIVED_OPS + NUMBER_OPS
UNARY = ("NOT", "NEAR", "INTERIOR")
BINARY = ("AND", "REACH", "OR", "SURROUNDED", "GROW", "TOUCH")
ATOMS = ("TRUE", "FALSE", "THR_GT", "THR_LT", "PCT_GT", "PCT_LT", "MASK")


class Node(NamedTuple):
    op: str
    a: int = -1
    b: int = -1
    image: int = 0
    channel: int = 0
    t: float = 0.0
    q: float = 0.0


def f32(x: float) -> float:
    """Round a Python float to the nearest float32 and return it as float."""
    return float(np.float32(x))


@dataclass
class Formula:
    nodes: List[Node]
    roots: List[int]
    name: str = ""
    meta: dict = field(default_factory=dict)

    def validate(self) -> None:
        n = len(self.nodes)
        for i, nd in enumerate(self.nodes):
            if nd.op not in OPS:
                raise ValueError(f"node {i}: unknown op {nd.op}")
            if nd.op in UNARY and not (0 <= nd.a < i):
                raise ValueError(f"node {i}: bad operand {nd.a}")
            if nd.op in BINARY and not (0 <= nd.a < i and 0 <= nd.b < i):
                raise ValueError(f"node {i}: bad operands {nd.a},{nd.b}")
            if nd.op in NUMBER_OPS[1:] and not (0 <= nd.a < i and nd.b < i):
                raise ValueError(f"node {i}: bad operands {nd.a},{nd.b}")
        for r in self.roots:
            if not 0 <= r < n:
                raise ValueError(f"bad root {r}")

    def depth(self) -> int:
        d = [0] * len(self.nodes)
        for i, nd in enumerate(self.nodes):
            ops = [x for x in (nd.a, nd.b) if x >= 0 and nd.op not in ATOMS]
            d[i] = 1 + max((d[x] for x in ops), default=0)
        return max(d) if d else 0

    def n_images(self) -> int:
        return 1 + max((nd.image for nd in self.nodes if nd.op in ATOMS), default=0)


# Kind mix of the large random formulas: 35 % thresholds, 35 % not/and (split
# evenly), 20 % near, 10 % reachability.
_RANDOM_KINDS = ("THR", "NOT", "AND", "NEAR", "REACH")
_RANDOM_PROBS = (0.35, 0.175, 0.175, 0.20, 0.10)


def random_dag(n_nodes: int = 2000, seed: int = 0, max_depth: int = 500,
               p_local: float = 0.7, window: int = 4, n_images: int = 1,
               n_channels: int = 1) -> Formula:
    """A random formula DAG in the style of the paper's "random" large formulas
    (Sec. 4.1: operators composed in various ways over the images).

    Node 0 is a threshold.  Each operand is, with probability ``p_local``, one
    of the last ``window`` nodes, otherwise any earlier node; operand draws that
    would exceed ``max_depth`` are redrawn.  Roots are the nodes nobody
    consumes.
    """
    rng = np.random.default_rng(seed)
    nodes: List[Node] = []
    depth: List[int] = []
    consumed = np.zeros(n_nodes, dtype=bool)

    def draw_operand(i: int) -> int:
        if rng.random() < p_local:
            lo = max(0, i - window)
            return int(rng.integers(lo, i))
        return int(rng.integers(0, i))

    for i in range(n_nodes):
        kind = "THR" if i == 0 else _RANDOM_KINDS[rng.choice(5, p=_RANDOM_PROBS)]
        if kind == "THR":
            op = "THR_GT" if rng.random() < 0.5 else "THR_LT"
            t = f32(rng.random())
            img = int(rng.integers(0, n_images)) if n_images > 1 else 0
            ch = int(rng.integers(0, n_channels)) if n_channels > 1 else 0
            nodes.append(Node(op, image=img, channel=ch, t=t))
            depth.append(1)
            continue
        arity = 1 if kind in ("NOT", "NEAR") else 2
        for _ in range(10000):
            ops = [draw_operand(i) for _ in range(arity)]
            d = 1 + max(depth[x] for x in ops)
            if d <= max_depth:
                break
        else:  # pragma: no cover - node 0 always has depth 1
            ops = [0] * arity
            d = 2
        for x in ops:
            consumed[x] = True
        if arity == 1:
            nodes.append(Node(kind, a=ops[0]))
        else:
            nodes.append(Node(kind, a=ops[0], b=ops[1]))
        depth.append(d)
    roots = [i for i in range(n_nodes) if not consumed[i]]
    f = Formula(nodes, roots, name=f"random{n_nodes}_s{seed}",
                meta={"seed": seed, "max_depth": max_depth})
    f.validate()
    return f


# Operator mixes of the sequential chains: weights of (NOT, NEAR, AND, REACH).
CHAIN_MIXES = {
    "mixed": (0.3, 0.3, 0.25, 0.15),
    # deep N chains: long runs of dilations cut by complements, which stress
    # the halo of fused groups (a dilation of a complement is an erosion)
    "near": (0.3, 0.65, 0.05, 0.0),
    # reachability after reachability: every rho waits for the one before
    "reach": (0.3, 0.1, 0.2, 0.4),
}


def sequential_dag(n_nodes: int = 500, seed: int = 0, mix: str = "mixed",
                   taps: int = 0) -> Formula:
    """A sequential formula f(g(...(x))) (Sec. 4.1): every operator takes the
    previous node as its first operand; binary operators take a fresh
    threshold as the second.  `mix` picks the operator weights (CHAIN_MIXES).
    The root is the last node; with `taps` > 0 every taps-th node is an output
    too (chains often end in an all-true or all-false mask, the taps show the
    states on the way)."""
    rng = np.random.default_rng(seed)
    p = CHAIN_MIXES[mix]
    nodes = [Node("THR_GT", t=f32(rng.random()))]
    while len(nodes) < n_nodes:
        kind = ("NOT", "NEAR", "AND", "REACH")[rng.choice(4, p=p)]
        prev = len(nodes) - 1
        if kind in ("NOT", "NEAR"):
            nodes.append(Node(kind, a=prev))
        else:
            op = "THR_GT" if rng.random() < 0.5 else "THR_LT"
            nodes.append(Node(op, t=f32(rng.random())))
            nodes.append(Node(kind, a=prev, b=len(nodes) - 1))
    name = f"seq{n_nodes}_s{seed}" if mix == "mixed" else f"seq-{mix}{n_nodes}_s{seed}"
    roots = list(range(0, len(nodes) - 1, taps)) if taps > 0 else []
    f = Formula(nodes, roots + [len(nodes) - 1], name=name,
                meta={"seed": seed, "mix": mix, "taps": taps})
    f.validate()
    return f


def config1_formula() -> Formula:
    """a = I > 0.6, b = I < 0.3, out = rho(N a)[not b] and not a, plus
    surrounded(a, not b); two roots."""
    n = [
        Node("THR_GT", t=f32(0.6)),   # 0 a
        Node("THR_LT", t=f32(0.3)),   # 1 b
        Node("NEAR", a=0),            # 2 N a
        Node("NOT", a=1),             # 3 not b
        Node("REACH", a=2, b=3),      # 4 rho (N a)[not b]
        Node("NOT", a=0),             # 5 not a
        Node("AND", a=4, b=5),        # 6 out
        Node("SURROUNDED", a=0, b=3), # 7 surrounded(a, not b)
    ]
    f = Formula(n, [6, 7], name="config1")
    f.validate()
    return f


def grow_spec_formula(t_hyper: float = 62258.0 / 65535.0,
                      t_very: float = 56360.0 / 65535.0) -> Formula:
    """The segmentation spec of Fig. "specification": two intensity thresholds
    (0.95 and 0.86 of full scale) and gtv = grow(hI, vI)."""
    n = [Node("THR_GT", t=f32(t_hyper)), Node("THR_GT", t=f32(t_very)),
         Node("GROW", a=0, b=1)]
    f = Formula(n, [2], name="grow_spec")
    f.validate()
    return f


def config4_formula() -> Formula:
    """Fixed segmentation formula for the batched MRI-slice workload, modelled
    on the paper's spec (percentile-normalised thresholds, grow as semantic
    noise removal) and extended with near chains, interior, surrounded and a
    touch test.  Channels: 0 FLAIR-like (oedema and core bright), 1 rim
    bright, 2 core bright, 3 plain brain background.  It expands to 40
    primitive nodes (threshold, not, and, N, rho) after CSE."""
    n: List[Node] = []

    def add(*args, **kw) -> int:
        n.append(Node(*args, **kw))
        return len(n) - 1

    hI = add("PCT_GT", channel=0, q=0.95)
    vI = add("PCT_GT", channel=0, q=0.86)
    gtv = add("GROW", a=hI, b=vI)
    rim = add("PCT_GT", channel=1, q=0.97)
    core = add("PCT_GT", channel=2, q=0.98)
    brain = add("PCT_GT", channel=3, q=0.30)
    dark = add("THR_LT", channel=3, t=f32(0.08))
    n1 = add("NEAR", a=gtv)
    n2 = add("NEAR", a=n1)
    n3 = add("NEAR", a=n2)
    closed = add("INTERIOR", a=n3)
    roi = add("AND", a=closed, b=brain)
    nd = add("NOT", a=dark)
    seg = add("AND", a=roi, b=nd)
    sur = add("SURROUNDED", a=core, b=rim)
    tch = add("TOUCH", a=rim, b=core)
    act = add("OR", a=sur, b=tch)
    inner = add("INTERIOR", a=gtv)
    ninner = add("NOT", a=inner)
    edge = add("AND", a=gtv, b=ninner)
    f = Formula(n, [seg, act, gtv, edge], name="config4")
    f.validate()
    return f


def arith_dag(n_nodes: int = 60, seed: int = 0, n_channels: int = 2,
              n_images: int = 1, p_const: float = 0.3) -> Formula:
    """A random formula with number terms (the tool's basic arithmetic,
    Sec. 3): channel values combined by + - * / (with each other or with
    constants), compared by percentile thresholds (the values of products
    and quotients have no fixed range) and by sign tests against 0, and the
    masks combined by not / and / N / rho.  Roots: the unconsumed masks."""
    rng = np.random.default_rng(seed)
    nodes: List[Node] = []
    nums: List[int] = []
    masks: List[int] = []
    for im in range(n_images):
        for c in range(n_channels):
            nodes.append(Node("VALUE", image=im, channel=c))
            nums.append(len(nodes) - 1)
    consumed = set()
    while len(nodes) < n_nodes:
        r = rng.random()
        if r < 0.35 or len(masks) < 2:
            # arithmetic on recent terms (deep expressions), or a new channel
            a = nums[-1 - int(rng.integers(0, min(4, len(nums))))]
            op = ("ADD", "SUB", "MUL", "DIV")[int(rng.integers(0, 4))]
            if rng.random() < p_const:
                c = f32(rng.uniform(-2.0, 2.0))
                if op == "DIV" and c == 0.0:
                    c = 1.0
                nodes.append(Node(op, a=a, t=c))
            else:
                b = nums[int(rng.integers(0, len(nums)))]
                nodes.append(Node(op, a=a, b=b))
            nums.append(len(nodes) - 1)
            consumed.add(a)
            # compare it
            x = len(nodes) - 1
            if rng.random() < 0.7:
                op = "PCT_GT" if rng.random() < 0.5 else "PCT_LT"
                nodes.append(Node(op, a=x, q=float(rng.choice([0.1, 0.25, 0.5, 0.75, 0.9]))))
            else:
                op = "THR_GT" if rng.random() < 0.5 else "THR_LT"
                nodes.append(Node(op, a=x, t=0.0))
            masks.append(len(nodes) - 1)
        else:
            kind = ("NOT", "AND", "NEAR", "REACH")[int(rng.choice(4, p=(0.2, 0.35, 0.25, 0.2)))]
            a = masks[-1 - int(rng.integers(0, min(4, len(masks))))]
            if kind in ("NOT", "NEAR"):
                nodes.append(Node(kind, a=a))
            else:
                b = masks[int(rng.integers(0, len(masks)))]
                nodes.append(Node(kind, a=a, b=b))
                consumed.add(b)
            consumed.add(a)
            masks.append(len(nodes) - 1)
    roots = [m for m in masks if m not in consumed] or [masks[-1]]
    f = Formula(nodes, roots, name=f"arith{n_nodes}_s{seed}", meta={"seed": seed})
    f.validate()
    return f


def grow_spec_u16_formula() -> Formula:
    """The segmentation spec of Fig. "specification" as the paper runs it: on
    16-bit pixels, intensity > 62258 (0.95 of 65535) and > 56360 (0.86),
    gtv = grow(hI, vI)."""
    n = [Node("THR_GT", t=62258.0), Node("THR_GT", t=56360.0), Node("GROW", a=0, b=1)]
    f = Formula(n, [2], name="grow_spec_u16")
    f.validate()
    return f


def formula_to_records(f: Formula):
    """Plain tuples (op, a, b, image, channel, t, q) for marshalling."""
    return [tuple(nd) for nd in f.nodes]

