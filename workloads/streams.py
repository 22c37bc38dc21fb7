"""Query streams for the serving workload: Poisson arrivals of model-checking
queries, each a (resident image, random formula) pair."""
from __future__ import annotations

from typing import List, NamedTuple

import numpy as np


class Query(NamedTuple):
    arrival_s: float     # arrival time, seconds from stream start
    image_id: int        # index into the resident image pool
    n_nodes: int         # formula size
    dag_seed: int        # seed for ``random_dag(n_nodes, dag_seed, min(500, n))``


def pool_sides(n_images: int = 512, lo: int = 128, hi: int = 4096,
               seed: int = 0) -> np.ndarray:
    """Square image sides, log-uniform over [lo, hi]."""
    rng = np.random.default_rng(seed)
    u = rng.random(n_images)
    return np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def poisson_queries(n_queries: int, rate_per_s: float, n_images: int = 512,
                    n_lo: int = 10, n_hi: int = 2000, seed: int = 0) -> List[Query]:
    """``n_queries`` arrivals of a Poisson process with the given rate; image
    uniform over the pool; formula size log-uniform over [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_queries)
    t = np.cumsum(gaps) - gaps[0]
    img = rng.integers(0, n_images, size=n_queries)
    u = rng.random(n_queries)
    sizes = np.rint(np.exp(np.log(n_lo) + u * (np.log(n_hi) - np.log(n_lo)))).astype(np.int64)
    seeds = rng.integers(0, 2**31 - 1, size=n_queries)
    return [Query(float(t[i]), int(img[i]), int(sizes[i]), int(seeds[i]))
            for i in range(n_queries)]
