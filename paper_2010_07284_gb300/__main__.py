"""Run a specification file, like the paper's command-line tool (Sec. 3: its
one parameter is a text file of commands).

    python -m paper_2010_07284_gb300 SPEC [--conn 8] [--device 0]

Each `load x = "s"` reads the NumPy file s (relative to SPEC's folder): a
bool array is a binary image (H, W), a uint16 array stays 16-bit, anything
else becomes float32; (H, W) is one channel, (C, H, W) several.  Each
`save "s" e` writes the mask e to the NumPy file s as a bool (H, W) array.
Evaluation runs on the GPU through the library (no CPU fallback)."""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np


def run(spec_path: str, conn: int = 8, device: int = 0, out=sys.stdout) -> list:
    import paper_2010_07284_gb300 as vg
    with open(spec_path) as fh:
        src = fh.read()
    base = os.path.dirname(os.path.abspath(spec_path))
    ctx = vg.Context(device=device)
    F = ctx.compile_text(src, conn)
    images = []
    for name, path in zip(F.loads, F.sources):
        a = np.load(os.path.join(base, path))
        if a.dtype == np.bool_:
            if a.ndim != 2:
                raise SystemExit(f"{path}: a binary image is (H, W), not {a.shape}")
            images.append(ctx.mask(a.astype(np.uint8)))
        else:
            if a.ndim == 2:
                a = a[None]
            if a.ndim != 3:
                raise SystemExit(f"{path}: an image is (H, W) or (C, H, W), not {a.shape}")
            images.append(ctx.image(a))
    t0 = time.perf_counter()
    res = ctx.eval(F, images)
    st = res.sync()
    if st != 0:
        raise SystemExit(f"evaluation failed (device status {st}): {ctx.last_error()}")
    ms = (time.perf_counter() - t0) * 1e3
    written = []
    for k, name in enumerate(F.saves):
        m = res.mask(k).astype(bool)
        path = os.path.join(base, name)
        np.save(path, m)
        written.append(path if path.endswith(".npy") else path + ".npy")
        print(f"{name}: {int(m.sum())} of {m.size} pixels", file=out)
    print(f"evaluated in {ms:.3f} ms (compile excluded)", file=out)
    return written


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_2010_07284_gb300",
                                 description="Run a specification file on the GPU.")
    ap.add_argument("spec")
    ap.add_argument("--conn", type=int, default=8, choices=[4, 8])
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    run(a.spec, a.conn, a.device)


if __name__ == "__main__":
    main()
