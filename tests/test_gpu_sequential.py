"""Sequential formulas f(g(...(x))) of Sec. 4.1 at 2000 nodes, in three
operator mixes: the paper's mixed chain, deep N chains cut by complements
(every fused group runs at the largest halo) and reachability chains (every
rho waits for the one before it).  Every 25th node is an output besides the
last, so the states along the chain are compared with the oracle, in the
fused and in the plain form, under both adjacencies."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl
from gpu_util import check_formula, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mix,conn", [("mixed", 8), ("near", 8), ("near", 4), ("reach", 8),
                                      ("reach", 4)])
def test_chain_2000(mix, conn):
    torch_cuda()
    f = wl.sequential_dag(2000, seed=3, mix=mix, taps=25)
    # a smooth field keeps dilations and erosions from filling the image at
    # once; 900 x 1300 leaves ragged tiles in both directions
    img = wl.gaussian_field_image(900, 1300, sigma=16.0, seed=3)
    exp = check_formula(wl.formula_to_records(f), f.roots, [img], conn=conn)
    # the chain is not trivial: many taps are neither empty nor full
    nontrivial = sum(1 for m in exp if 0 < m.sum() < m.size)
    assert nontrivial >= len(exp) // 3, f"{nontrivial} of {len(exp)} taps non-trivial"


def test_near_chain_depth_beyond_group_halo():
    """600 dilations in a row (no complement): one group per halo limit, the
    mask grows by 600 px and is clipped at the border on every side."""
    torch_cuda()
    from workloads.formulas import Formula, Node
    nodes = [Node("THR_GT", t=np.float32(0.9995).item())]
    for _ in range(600):
        nodes.append(Node("NEAR", a=len(nodes) - 1))
    f = Formula(nodes, [1, 7, 8, 9, 100, 333, 600])
    img = wl.uniform_image(700, 1300, seed=9)
    for conn in (8, 4):
        check_formula(wl.formula_to_records(f), f.roots, [img], conn=conn)
