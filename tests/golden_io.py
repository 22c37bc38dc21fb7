"""Reader for the hand-worked fixtures in tests/golden/*.txt."""
from __future__ import annotations

import glob
import os
from typing import Dict, List

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _grid(lines: List[str]) -> np.ndarray:
    return np.array([[1 if c == "#" else 0 for c in ln] for ln in lines], dtype=np.uint8)


def _ints(lines: List[str]) -> np.ndarray:
    return np.array([[int(v) for v in ln.split()] for ln in lines], dtype=np.int64)


def load(path: str) -> Dict:
    """Parse a fixture: "//" comments, 'op NAME', named grids ('phi',
    'phi1', 'phi2'), an integer 'image' grid, 'expect conn=K' grids, or
    key/value lines."""
    out: Dict = {"path": path, "expect": {}, "kv": []}
    cur = None
    buf: List[str] = []

    def flush():
        nonlocal cur, buf
        if cur is None:
            return
        if cur.startswith("expect"):
            conn = int(cur.split("conn=")[1])
            out["expect"][conn] = _ints(buf) if out["op"] == "ccl" else _grid(buf)
        elif cur == "image":
            out[cur] = _ints(buf)
        else:
            out[cur] = _grid(buf)
        cur, buf = None, []

    with open(path) as fh:
        for raw in fh:
            ln = raw.rstrip("\n")
            if not ln.strip() or ln.startswith("//"):
                continue
            head = ln.split()[0]
            if head == "op":
                out["op"] = ln.split()[1]
            elif head in ("phi", "phi1", "phi2", "image") or head == "expect":
                flush()
                cur = ln.strip()
            elif head in ("values", "q", "scale", "const"):
                flush()
                out["kv"].append(ln.split())
            else:
                buf.append(ln.strip())
    flush()
    return out


def all_fixtures() -> List[Dict]:
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))]
