"""GB300-native spatial model checking of SLCS formulas on 2D images.

The library (``include/vl.h``) evaluates formula DAGs made of threshold
atoms, not/and, the near operator N and reachability rho (plus derived
connectives) with hand-written sm_103a CUDA kernels; this package is its
ctypes front-end.

  ctx = Context()                         # one GPU, a memory pool, caches
  img = ctx.image(array)                  # (C, H, W) float32, or uint16 kept
                                          #   as uint16 on the device
  F = ctx.compile(nodes, roots, conn=8)   # records (op, a, b, image, channel,
                                          #   t, q): atoms, connectives, number
                                          #   terms (VALUE, ADD, SUB, MUL, DIV)
  res = ctx.eval(F, [img]); res.sync(); res.mask(0)
  ctx.eval_batch / ctx.batch / ctx.autotune   # many jobs in one launch
  Server(ctx, ...)                        # continuous batching of queries
  ctx.ccl(mask, labels)                   # component labels (union-find)
  ctx.ccl_pointer_jumping(mask, labels)   # the paper's Alg. 1, for comparison
"""
from ._native import (VlError, OPCODES, EXEC_FUSED, EXEC_PLAIN, load, lib_path)
from .api import Context, Image, Formula, Result, Batch, Server, compile_formula, compile_text
from .buildlib import build, source_hash

__all__ = ["VlError", "OPCODES", "EXEC_FUSED", "EXEC_PLAIN", "load", "lib_path", "Context",
           "Image", "Formula", "Result", "Batch", "Server", "build", "source_hash", "compile_formula",
           "compile_text"]
