"""GB300-native spatial model checking of SLCS formulas on 2D images.

The library (``include/vl.h``) evaluates formula DAGs made of threshold
atoms, not/and, the near operator N and reachability rho (plus derived
connectives) with hand-written sm_103a CUDA kernels; this package is its
ctypes front-end.
"""
from ._native import (VlError, OPCODES, EXEC_FUSED, EXEC_PLAIN, load, lib_path)
from .api import Context, Image, Formula, Result, Batch, Server, compile_formula
from .buildlib import build, source_hash

__all__ = ["VlError", "OPCODES", "EXEC_FUSED", "EXEC_PLAIN", "load", "lib_path", "Context",
           "Image", "Formula", "Result", "Batch", "Server", "build", "source_hash", "compile_formula"]
