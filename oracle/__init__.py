"""CPU oracle for SLCS formula evaluation -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the C evaluator lives in ``vl_oracle.c`` and the derived-operator
expansion in ``expand.py``.
"""
from .oracle import (build, lib_path, expand, threshold, op_not, op_and,
                     near, reach, ccl, arith, percentile, evaluate, OracleResult,
                     near3, reach3, ccl3, evaluate3)

__all__ = ["build", "lib_path", "expand", "threshold", "op_not", "op_and",
           "near", "reach", "ccl", "arith", "percentile", "evaluate", "OracleResult",
           "near3", "reach3", "ccl3", "evaluate3"]
