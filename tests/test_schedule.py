"""The executor's work-list order (`order_work_items`, csrc/schedule.cpp),
host only: the persistent executor's CTAs pop items in list order and an
item waits for every step its own step depends on, so the list must hold
every item once, after all items of the steps it waits for -- for any
dependency lists, grid sizes and numbers of jobs.  Also that one job's list
starts a critical step as soon as it is ready, and that several jobs
interleave by progress (a short job is not held behind a long one)."""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_07284_gb300", "csrc")


@pytest.fixture(scope="module")
def sched(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("sched") / "libsched.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(ROOT, "tests", "sched_shim.cpp"),
                    os.path.join(CSRC, "schedule.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.sched_order.restype = C.c_int
    return lib


def order(lib, jobs, grid):
    """jobs: list of (steps, deps) with steps = [(n items, us per item)] and
    deps[s] = the earlier steps step s waits for.  Returns (job, step, first)
    triples in list order."""
    n_steps = [len(st) for st, _ in jobs]
    step_n = [n for st, _ in jobs for n, _ in st]
    step_us = [u for st, _ in jobs for _, u in st]
    dep_off, deps = [], []
    for st, dp in jobs:
        off = [0]
        for s in range(len(st)):
            deps += list(dp[s])
            off.append(off[-1] + len(dp[s]))
        dep_off += off
    total = sum(step_n)
    arr = lambda t, v: (t * max(1, len(v)))(*v)
    oj, os_, of = (C.c_int * max(1, total))(), (C.c_int * max(1, total))(), (C.c_int * max(1, total))()
    n = lib.sched_order(len(jobs), arr(C.c_int, n_steps), arr(C.c_int, step_n),
                        arr(C.c_double, step_us), arr(C.c_int, dep_off), arr(C.c_int, deps),
                        grid, oj, os_, of)
    assert n == total
    return [(oj[i], os_[i], of[i]) for i in range(total)]


def check_valid(jobs, items):
    assert len(set(items)) == len(items)
    want = {(j, s, k) for j, (st, _) in enumerate(jobs) for s, (n, _) in enumerate(st) for k in range(n)}
    assert set(items) == want
    last = {}
    for p, (j, s, _) in enumerate(items):
        last[(j, s)] = p
    for p, (j, s, _) in enumerate(items):
        for d in jobs[j][1][s]:
            assert last[(j, d)] < p, f"item {p} of job {j} step {s} before the end of step {d}"


def random_job(rng, max_steps=60):
    S = int(rng.integers(1, max_steps))
    steps = [(int(rng.integers(1, 50)), float(rng.uniform(1, 500))) for _ in range(S)]
    deps = []
    for s in range(S):
        k = int(rng.integers(0, min(s, 5) + 1)) if s else 0
        deps.append(sorted(set(int(x) for x in rng.choice(s, size=k, replace=False))) if k else [])
    return steps, deps


@pytest.mark.parametrize("seed", range(12))
def test_one_job_lists_every_item_after_what_it_waits_for(sched, seed):
    rng = np.random.default_rng(seed)
    job = random_job(rng)
    for grid in (1, 7, 304):
        check_valid([job], order(sched, [job], grid))


@pytest.mark.parametrize("seed", range(8))
def test_several_jobs_list_every_item_after_what_it_waits_for(sched, seed):
    rng = np.random.default_rng(100 + seed)
    jobs = [random_job(rng, 20) for _ in range(int(rng.integers(2, 9)))]
    for grid in (3, 304):
        check_valid(jobs, order(sched, jobs, grid))


def test_a_critical_step_starts_as_soon_as_it_is_ready(sched):
    # step 0 (one short item) -> step 1 (one long item); step 2: 100 short
    # independent items.  On 4 CTAs step 1 is ready after 10 us, when about
    # 30 of step 2's items have started: it must not wait for the other 70.
    job = ([(1, 10.0), (1, 1000.0), (100, 1.0)], [[], [0], []])
    items = order(sched, [job], 4)
    check_valid([job], items)
    assert items[0] == (0, 0, 0)
    assert items.index((0, 1, 0)) < 50


def test_several_jobs_interleave_by_progress(sched):
    # job 0: a chain of 20 long steps; job 1: one short step.  The short job
    # is not listed behind the long job's later steps.
    long_job = ([(10, 100.0)] * 20, [[]] + [[s] for s in range(19)])
    short_job = ([(10, 5.0)], [[]])
    items = order(sched, [long_job, short_job], 304)
    check_valid([long_job, short_job], items)
    first_short = min(p for p, (j, _, _) in enumerate(items) if j == 1)
    first_late = min(p for p, (j, s, _) in enumerate(items) if j == 0 and s >= 1)
    assert first_short < first_late


def test_dependencies_on_later_steps_are_refused(sched):
    with pytest.raises(AssertionError):
        order(sched, [([(1, 1.0), (1, 1.0)], [[1], []])], 4)
