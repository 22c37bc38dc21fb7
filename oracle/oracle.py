"""ctypes front-end of the C oracle -- test infrastructure only.

The shared object is built from ``vl_oracle.c`` with gcc into
``oracle/_build/`` on first use (or by ``build()``).  Masks are numpy uint8
arrays of 0/1 shaped (H, W); images are float32 arrays shaped (C, H, W).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, NamedTuple, Optional, Sequence

import numpy as np

from .expand import expand

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB: Optional[C.CDLL] = None

_OPCODE = {"TRUE": 0, "FALSE": 1, "THR_GT": 2, "THR_LT": 3, "PCT_GT": 4,
           "PCT_LT": 5, "MASK": 6, "NOT": 7, "AND": 8, "NEAR": 9, "REACH": 10,
           "VALUE": 16, "ADD": 17, "SUB": 18, "MUL": 19, "DIV": 20}
_ARITH = {"ADD": 0, "SUB": 1, "MUL": 2, "DIV": 3}


class _Node(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32),
                ("image", C.c_int32), ("channel", C.c_int32), ("t", C.c_float),
                ("q", C.c_double)]


def lib_path() -> str:
    import platform
    return os.path.join(_BUILD, f"libvl_oracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only)."""
    out = lib_path()
    with _LOCK:
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = out + f".tmp{os.getpid()}"
            # no contraction of a*b+c into one rounding: every arithmetic
            # result is rounded on its own
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-fPIC",
                                   "-ffp-contract=off", "-shared", "-o", tmp, _SRC])
            os.replace(tmp, out)
    return out


def _lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.vlo_threshold.argtypes = [P, C.c_int64, C.c_float, C.c_int, P]
        lib.vlo_not.argtypes = [P, C.c_int64, P]
        lib.vlo_and.argtypes = [P, P, C.c_int64, P]
        lib.vlo_near.argtypes = [P, C.c_int, C.c_int, C.c_int, P]
        lib.vlo_reach.argtypes = [P, P, C.c_int, C.c_int, C.c_int, P]
        lib.vlo_reach.restype = C.c_int
        lib.vlo_ccl.argtypes = [P, C.c_int, C.c_int, C.c_int, P]
        lib.vlo_ccl.restype = C.c_int64
        lib.vlo_arith.argtypes = [C.c_int, P, P, C.c_float, C.c_int64, P]
        lib.vlo_near3.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P]
        lib.vlo_reach3.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P]
        lib.vlo_reach3.restype = C.c_int
        lib.vlo_ccl3.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P]
        lib.vlo_ccl3.restype = C.c_int64
        lib.vlo_percentile.argtypes = [P, C.c_int64, C.c_double]
        lib.vlo_percentile.restype = C.c_float
        lib.vlo_eval.argtypes = [P, C.c_int, P, C.c_int, P, C.c_int, C.c_int,
                                 P, C.c_int, C.c_int, C.c_int, C.c_int, P]
        lib.vlo_eval.restype = C.c_int
        _LIB = lib
    return _LIB


def _mask(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a) != 0, dtype=np.uint8)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ------------------------------------------------------------ primitives ---

def threshold(channel: np.ndarray, t: float, gt: bool = True) -> np.ndarray:
    ch = np.ascontiguousarray(channel, dtype=np.float32)
    out = np.empty(ch.shape, dtype=np.uint8)
    _lib().vlo_threshold(_ptr(ch), ch.size, float(np.float32(t)), int(gt), _ptr(out))
    return out


def op_not(a) -> np.ndarray:
    a = _mask(a)
    out = np.empty_like(a)
    _lib().vlo_not(_ptr(a), a.size, _ptr(out))
    return out


def op_and(a, b) -> np.ndarray:
    a, b = _mask(a), _mask(b)
    out = np.empty_like(a)
    _lib().vlo_and(_ptr(a), _ptr(b), a.size, _ptr(out))
    return out


def near(a, conn: int = 8) -> np.ndarray:
    a = _mask(a)
    out = np.empty_like(a)
    _lib().vlo_near(_ptr(a), a.shape[0], a.shape[1], conn, _ptr(out))
    return out


def reach(phi1, phi2, conn: int = 8) -> np.ndarray:
    a, b = _mask(phi1), _mask(phi2)
    out = np.empty_like(a)
    if _lib().vlo_reach(_ptr(a), _ptr(b), a.shape[0], a.shape[1], conn, _ptr(out)) != 0:
        raise MemoryError("oracle reach: out of memory")
    return out


def ccl(m, conn: int = 8):
    """(labels int32 (H, W), number of components); label = minimum linear
    index of the component, background -1."""
    m = _mask(m)
    lab = np.empty(m.shape, dtype=np.int32)
    n = _lib().vlo_ccl(_ptr(m), m.shape[0], m.shape[1], conn, _ptr(lab))
    if n < 0:
        raise MemoryError("oracle ccl: out of memory")
    return lab, int(n)


def arith(op: str, a: np.ndarray, b) -> np.ndarray:
    """a (op) b pixel by pixel in float32, op one of ADD, SUB, MUL, DIV; b is
    an array of a's shape or a float32 constant."""
    x = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.float32)
    if np.isscalar(b):
        _lib().vlo_arith(_ARITH[op], _ptr(x), None, float(np.float32(b)), x.size, _ptr(out))
    else:
        y = np.ascontiguousarray(b, dtype=np.float32)
        if y.shape != x.shape:
            raise ValueError("arith operands differ in shape")
        _lib().vlo_arith(_ARITH[op], _ptr(x), _ptr(y), 0.0, x.size, _ptr(out))
    return out


def percentile(channel: np.ndarray, q: float) -> float:
    ch = np.ascontiguousarray(channel, dtype=np.float32)
    return float(_lib().vlo_percentile(_ptr(ch), ch.size, float(q)))


# --------------------------------------------------------------- formulas ---

class OracleResult(NamedTuple):
    masks: List[np.ndarray]      # one (H, W) uint8 mask per root
    n_primitive: int             # primitive nodes after expansion + sharing
    prim_nodes: list             # the expanded primitive DAG
    prim_roots: list


def evaluate(nodes: Sequence, roots: Sequence[int],
             images: Sequence[np.ndarray] = (), masks: Sequence[np.ndarray] = (),
             conn: int = 8, shape=None) -> OracleResult:
    """Evaluate a formula (records (op, a, b, image, channel, t, q)) on a list
    of (C, H, W) float32 or uint16 images and (H, W) masks; all share H, W.
    A uint16 pixel is its integer value, which float32 holds exactly."""
    prim, proots = expand(nodes, roots)
    imgs = [np.ascontiguousarray(im, dtype=np.float32) for im in images]
    msks = [_mask(m) for m in masks]
    if imgs:
        Cn, H, W = imgs[0].shape
    elif msks:
        Cn, (H, W) = 1, msks[0].shape
    elif shape is not None:
        Cn, (H, W) = 1, shape
    else:
        raise ValueError("need at least one image, a mask or a shape")
    for im in imgs:
        if im.shape != (Cn, H, W):
            raise ValueError("all images must share (C, H, W)")
    for m in msks:
        if m.shape != (H, W):
            raise ValueError("all masks must share (H, W)")
    arr = (_Node * max(1, len(prim)))()
    for i, (op, a, b, img, ch, t, q) in enumerate(prim):
        arr[i] = _Node(_OPCODE[op], a, b, img, ch, float(np.float32(t)), float(q))
    rts = (C.c_int32 * max(1, len(proots)))(*proots)
    img_ptrs = (C.c_void_p * max(1, len(imgs)))(*[_ptr(x) for x in imgs])
    msk_ptrs = (C.c_void_p * max(1, len(msks)))(*[_ptr(x) for x in msks])
    outs = [np.empty((H, W), dtype=np.uint8) for _ in proots]
    out_ptrs = (C.c_void_p * max(1, len(outs)))(*[_ptr(x) for x in outs])
    rc = _lib().vlo_eval(C.addressof(arr), len(prim), C.addressof(rts), len(proots),
                         C.addressof(img_ptrs), len(imgs), Cn,
                         C.addressof(msk_ptrs), len(msks), H, W, conn,
                         C.addressof(out_ptrs))
    if rc == -1:
        raise ValueError("oracle: malformed formula or inputs")
    if rc != 0:
        raise MemoryError("oracle: out of memory")
    return OracleResult(outs, len(prim), prim, proots)


# ------------------------------------------------------------- 3D volumes ---
# Volumes are (D, H, W) arrays (masks) or (C, D, H, W) arrays (number
# images); adjacency 26 (3x3x3 cube) or 6 (faces).  The derived connectives,
# thresholds, percentiles and number terms are those of the 2D evaluator,
# applied voxel by voxel; only N and rho see the third axis.

def near3(a, conn: int = 26) -> np.ndarray:
    a = _mask(a)
    out = np.empty_like(a)
    _lib().vlo_near3(_ptr(a), a.shape[0], a.shape[1], a.shape[2], conn, _ptr(out))
    return out


def reach3(phi1, phi2, conn: int = 26) -> np.ndarray:
    a, b = _mask(phi1), _mask(phi2)
    out = np.empty_like(a)
    if _lib().vlo_reach3(_ptr(a), _ptr(b), a.shape[0], a.shape[1], a.shape[2], conn,
                         _ptr(out)) != 0:
        raise MemoryError("oracle reach3: out of memory")
    return out


def ccl3(m, conn: int = 26):
    """(labels int32 (D, H, W), number of components); label = minimum
    linear index z*H*W + y*W + x of the component, background -1."""
    m = _mask(m)
    lab = np.empty(m.shape, dtype=np.int32)
    n = _lib().vlo_ccl3(_ptr(m), m.shape[0], m.shape[1], m.shape[2], conn, _ptr(lab))
    if n < 0:
        raise MemoryError("oracle ccl3: out of memory")
    return lab, int(n)


def evaluate3(nodes: Sequence, roots: Sequence[int], volumes: Sequence[np.ndarray] = (),
              masks: Sequence[np.ndarray] = (), conn: int = 26) -> OracleResult:
    """Evaluate a formula on (C, D, H, W) number volumes (float32 or uint16)
    and (D, H, W) mask volumes, node by node in the expanded DAG's order."""
    if conn not in (6, 26):
        raise ValueError("volume adjacency is 6 or 26")
    prim, proots = expand(nodes, roots)
    vols = [np.ascontiguousarray(v, dtype=np.float32) for v in volumes]
    msks = [_mask(m) for m in masks]
    shape = vols[0].shape[1:] if vols else msks[0].shape
    val: List[Optional[np.ndarray]] = [None] * len(prim)
    for i, (op, a, b, img, ch, t, q) in enumerate(prim):
        if op == "TRUE":
            v = np.ones(shape, np.uint8)
        elif op == "FALSE":
            v = np.zeros(shape, np.uint8)
        elif op == "MASK":
            v = msks[img]
        elif op == "VALUE":
            v = np.ascontiguousarray(vols[img][ch])
        elif op in ("ADD", "SUB", "MUL", "DIV"):
            v = arith(op, val[a], np.float32(t) if b < 0 else val[b])
        elif op in ("THR_GT", "THR_LT", "PCT_GT", "PCT_LT"):
            x = val[a] if a >= 0 else vols[img][ch]
            thr = percentile(x, q) if op.startswith("PCT") else t
            v = threshold(x, thr, gt=op.endswith("GT"))
        elif op == "NOT":
            v = op_not(val[a])
        elif op == "AND":
            v = op_and(val[a], val[b])
        elif op == "NEAR":
            v = near3(val[a], conn)
        elif op == "REACH":
            v = reach3(val[a], val[b], conn)
        else:
            raise ValueError(f"unknown primitive {op}")
        val[i] = v
    return OracleResult([np.ascontiguousarray(val[r], dtype=np.uint8) for r in proots],
                        len(prim), prim, proots)

