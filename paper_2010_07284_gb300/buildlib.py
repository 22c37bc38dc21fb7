"""Build the CUDA library in-tree: sm_103a kernels (nvcc) + host runtime
(g++), linked into paper_2010_07284_gb300/_build/libvlgb_<machine>.so with a
static CUDA runtime.  Translation units compile in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels.cu", "executor.cu", "noalloc.cu", "pointer_jump.cu", "volume.cu"]
CPP_SOURCES = ["api.cpp", "autotune.cpp", "compiler.cpp", "schedule.cpp", "server.cpp", "spec.cpp"]


def lib_path() -> str:
    return os.path.join(BUILD, f"libvlgb_{platform.machine()}.so")


def _sources():
    cu = [s for s in CU_SOURCES if os.path.exists(os.path.join(CSRC, s))]
    return cu, CPP_SOURCES


def _deps():
    names = os.listdir(CSRC)
    files = [os.path.join(CSRC, n) for n in names if n.endswith((".cu", ".cuh", ".h", ".cpp"))]
    files.append(os.path.join(ROOT, "include", "vl.h"))
    files.append(os.path.abspath(__file__))
    return files


def source_hash(names=None) -> str:
    """Hash of the library sources, or of the named ones (file names, e.g.
    the files a kernel is built from): identifies which kernels a profile
    saw."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(_deps()):
        if f.endswith("buildlib.py"):
            continue
        if names is not None and os.path.basename(f) not in names:
            continue
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in _deps())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    out = lib_path()
    if not force and not _stale(out):
        return out
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    tag = platform.machine()
    cu, cpp = _sources()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    objs = []
    for s in cu:
        o = os.path.join(BUILD, f"{s}.{tag}.o")
        objs.append(o)
        jobs.append([NVCC, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xptxas", "-v",
                     "-Xcompiler", "-fPIC,-fvisibility=hidden", *inc, "-c",
                     os.path.join(CSRC, s), "-o", o])
    for s in cpp:
        o = os.path.join(BUILD, f"{s}.{tag}.o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-Wall",
                     "-I", os.path.join(CUDA_HOME, "include"), *inc, "-c",
                     os.path.join(CSRC, s), "-o", o])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        for log in ex.map(_run, jobs):
            logs.append(log)
    tmp = out + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs,
          "-Xlinker", "--no-undefined", "-lpthread", "-ldl", "-lrt"])
    os.replace(tmp, out)
    with open(os.path.join(BUILD, f"ptxas_{tag}.log"), "w") as fh:
        fh.write("\n".join(logs))
    if verbose:
        print("\n".join(logs))
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
