"""Benchmark: SLCS formula evaluation on GB300.

Workload (one step): the large random formula -- a 2000-node DAG (35 %
thresholds, 35 % not/and, 20 % N, 10 % rho, depth <= 500, seed 0) over one
2048 x 2048 float32 U[0,1) image, 8-adjacency, every root mask produced.
Inputs are resident in HBM; L2 (129 MB) is flushed between timed steps by
writing a 512 MiB buffer.  `value` is Gpixel-ops/s: primitive nodes after
expansion and sharing x pixels / step time, summed over ranks.

Also reported: the plain per-operator form on the same workload, full
connected-component labelling of an 8192 x 8192 Bernoulli(0.5) mask (CCL
Gpix/s), end-to-end throughput through the public API with host buffers,
per-step p50/p99, the roofline of the persistent executor, SM clocks during
the timed region, and the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 2048
N_NODES = 2000
DAG_SEED = 0
CONN = 8
METRIC = "Gpixel-ops/s and CCL Gpix/s, batched vs plain on 1 GB300, bit-exact; p99 ms"
UNIT = "Gpixel-ops/s"
FLUSH_BYTES = 512 << 20
CPU_ROWS_REF = 64     # rows of the image per reference-arm step
CPU_ROWS_BASE = 512   # rows for the cpu_baseline sample


def workload_config(n_gpus: int) -> dict:
    return {"workload": "random-formula-2048x2048",
            "image": [H, W], "formula_nodes": N_NODES, "dag_seed": DAG_SEED,
            "connectivity": CONN, "l2": "flushed between steps (512 MiB write)",
            "parallelism": f"replicas{n_gpus}"}


def aggregate_throughput(total_ms: float, units_per_rank: float, world: int, device) -> tuple:
    """Whole-job throughput of `world` replicas: every rank processed
    `units_per_rank` units in its own `total_ms`; the job took the slowest
    rank's time (max over ranks), so value = world * units / max time (s).
    Returns (value, max_ms); needs an initialised process group if world > 1."""
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_max = float(t.item())
    return world * units_per_rank / (total_max / 1e3), total_max


def profiled_traffic(kernel: str, key: str):
    """DRAM bytes that an ncu capture of the current kernel sources measured
    (profiles/traffic.json: each entry lists the source files its kernels are
    built from and their hash when it was taken), or None when one of those
    files changed since."""
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        entry = json.load(open(tfile)).get(kernel, {})
        from paper_2010_07284_gb300 import buildlib
        if entry.get("source_hash") == buildlib.source_hash(entry.get("sources")):
            return entry.get(key)
    except Exception:
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def formula_alg_bytes(info: dict, P: float) -> float:
    """Algorithmic bytes of one evaluation of a formula over P pixels: each
    image channel read once (4 B/px), each materialised mask written once and
    read back once per consumer (1/8 B/px each), and 8.25 B/px per rho select
    (int32 labels written and read once, plus its flag mask)."""
    return (4.0 * P * info["n_channels_read"]
            + P / 8.0 * (info["mask_writes"] + info["mask_reads"])
            + P * (8.0 + 2.0 / 8.0) * info["n_selects"])


def sig(x, digits: int = 4):
    """Floats rounded to `digits` significant digits, recursively (keeps the
    printed line short)."""
    if isinstance(x, float):
        if x != x or x in (float("inf"), float("-inf")) or x == 0.0:
            return x
        return float(f"{x:.{digits}g}")
    if isinstance(x, dict):
        return {k: sig(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig(v, digits) for v in x]
    return x


def emit_leg(name: str, obj: dict) -> None:
    """A leg's full figures on a line of its own, before the result line
    (prefixed, so that it is not taken for the result line)."""
    print(f"# leg {name} " + json.dumps(sig(obj)), flush=True)


class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(rows: int):
    """CPU oracle on the same formula over the top `rows` rows of the image."""
    import oracle
    import workloads as wl
    f = wl.random_dag(N_NODES, seed=DAG_SEED)
    img = wl.uniform_image(H, W, seed=0)[:, :rows, :].copy()
    rec = wl.formula_to_records(f)
    t0 = time.perf_counter()
    r = oracle.evaluate(rec, f.roots, [img], conn=CONN)
    dt = time.perf_counter() - t0
    return r.n_primitive * rows * W / dt / 1e9, dt, r.n_primitive


def _oracle_warm(_):
    import oracle
    oracle.build()
    return os.getpid()


def _oracle_task(task):
    rec, roots, img = task
    import oracle
    t0 = time.perf_counter()
    r = oracle.evaluate(rec, roots, [img], conn=8)
    return time.perf_counter() - t0, float(r.n_primitive) * img.shape[-2] * img.shape[-1]


def oracle_all_cores(tasks) -> dict:
    """The CPU oracle, as it stands, over (records, roots, image) tasks on
    every host core: a spawn pool (workers start without the parent's CUDA
    context), warmed up before the clock starts.  Wall time of all tasks,
    summed task seconds, pixel-ops, cores."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_warm, range(cores)))
        t0 = time.perf_counter()
        res = list(ex.map(_oracle_task, tasks))
        wall = time.perf_counter() - t0
    return {"wall_s": wall, "task_s": float(sum(r[0] for r in res)),
            "pixel_ops": float(sum(r[1] for r in res)), "cores": cores, "tasks": len(tasks)}


def leg_grow_7680(ctx, stream, flush, peak: float, runs: int = 5) -> dict:
    """The case-study spec (two thresholds and grow, Sec. 4.2) on a 7680 x
    7680 upscaled MRI-shaped slice, the scale of the paper's only published
    timings: device time with the image resident, and end to end through the
    public API (pinned host image in, result mask out)."""
    import torch
    import workloads as wl
    from workloads.images import upscaled_slice
    f = wl.grow_spec_formula()
    img = upscaled_slice(7680)
    F = ctx.compile(wl.formula_to_records(f), f.roots, 8)
    finfo = F.info()
    n_prim = finfo["n_primitive"]
    P = img.shape[1] * img.shape[2]
    pin = torch.from_numpy(img).pin_memory()
    out = np.empty((img.shape[1], ((img.shape[2] + 127) // 128) * 4), dtype=np.uint32)
    out_t = torch.from_numpy(out).pin_memory()
    with torch.cuda.stream(stream):
        im = ctx.image(pin.numpy(), stream)
        b = ctx.batch([(F, [im])], stream)
        for _ in range(2):
            b.run(stream)
        ev = []
        for _ in range(runs):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.run(stream)
            z.record(stream)
            ev.append((a, z))
        stream.synchronize()
        if b.result(0).status_word() != 0:
            raise SystemExit("grow 7680 failed")
        dev_ms = float(np.mean([a.elapsed_time(z) for a, z in ev]))
        e2e = []
        for k in range(runs + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            im2 = ctx.image(pin.numpy(), stream)
            r = ctx.eval(F, [im2], stream=stream)
            r.mask_into(0, out_t.numpy(), on_device=False, stream=stream)
            t1 = time.perf_counter()
            if r.sync() != 0:
                raise SystemExit("grow 7680 e2e failed")
            if k:
                e2e.append(1e3 * (t1 - t0))
            r.close()
            im2.close()
        b.close()
        im.close()
        # the same spec as the paper runs it: 16-bit pixels, thresholds 62258
        # and 56360 (2 bytes per pixel read instead of 4)
        fu = wl.grow_spec_u16_formula()
        Fu = ctx.compile(wl.formula_to_records(fu), fu.roots, 8)
        img16 = wl.to_u16(img)
        im16 = ctx.image(img16, stream)
        bu = ctx.batch([(Fu, [im16])], stream)
        for _ in range(2):
            bu.run(stream)
        ev16 = []
        for _ in range(runs):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bu.run(stream)
            z.record(stream)
            ev16.append((a, z))
        stream.synchronize()
        if bu.result(0).status_word() != 0:
            raise SystemExit("grow 7680 uint16 failed")
        u16_ms = float(np.mean([a.elapsed_time(z) for a, z in ev16]))
        bu.close()
        im16.close()
    alg = formula_alg_bytes(finfo, P)
    ach = alg / (dev_ms / 1e3) / 1e9
    return {"workload": "grow(I > 0.95, I > 0.86) on a 7680x7680 upscaled MRI-shaped slice (59 Mpx)",
            "device_ms": dev_ms, "e2e_ms": float(np.mean(e2e)),
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "algorithmic_bytes": alg, "kernel": "k_exec"},
            "uint16": {"device_ms": u16_ms, "thresholds": [62258, 56360],
                       "value": n_prim * P / (u16_ms / 1e3) / 1e9},
            "value": n_prim * P / (dev_ms / 1e3) / 1e9, "unit": "Gpixel-ops/s",
            "e2e_bytes": {"h2d": int(img.nbytes), "d2h": int(out.nbytes)},
            "paper_context_ms": {"TITAN Xp (OpenCL, D2H included)": 600,
                                 "Intel HD 630 (OpenCL)": 3000, "i7-7700 CPU tool": 1100}}


def leg_volume(ctx, stream, flush, peak: float, shape=(155, 240, 240), runs: int = 5) -> dict:
    """The 40-primitive segmentation formula on an MRI-volume-shaped
    4-channel float32 phantom of 155 x 240 x 240 voxels (the size of the
    paper's brain scans before it takes one slice, Sec. 4.2), 26-adjacency:
    device time with the volume resident (volumes evaluate in the
    per-operator form), Gvoxel-ops/s and the roofline of the step, and the
    oracle on a bounded sub-volume on one core."""
    import torch
    import oracle
    import workloads as wl
    f = wl.config4_formula()
    rec = wl.formula_to_records(f)
    vol = wl.mri_phantom_volume(*shape, seed=0)
    F = ctx.compile(rec, f.roots, 26)
    finfo = F.info()
    n_prim = finfo["n_primitive"]
    P = float(np.prod(shape))
    with torch.cuda.stream(stream):
        im = ctx.volume(vol, stream)
        for _ in range(2):
            r = ctx.eval(F, [im], stream=stream)
            if r.sync() != 0:
                raise SystemExit("volume leg failed: " + ctx.last_error())
            r.close()
        ev = []
        for _ in range(runs):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = ctx.eval(F, [im], stream=stream)
            z.record(stream)
            ev.append((a, z, r))
        stream.synchronize()
        for a, z, r in ev:
            if r.sync() != 0:
                raise SystemExit("volume leg failed")
            r.close()
        ms = float(np.mean([a.elapsed_time(z) for a, z, _ in ev]))
        im.close()
    alg = formula_alg_bytes(finfo, P)
    ach = alg / (ms / 1e3) / 1e9
    # the oracle on the first 8 slices, one core
    sub = np.ascontiguousarray(vol[:, :8])
    t0 = time.perf_counter()
    oracle.evaluate3(rec, f.roots, volumes=[sub], conn=26)
    cpu_s = time.perf_counter() - t0
    return {"workload": f"segmentation formula on a {shape[0]}x{shape[1]}x{shape[2]} MRI-shaped "
                        "4-channel volume, 26-adjacency",
            "form": "per-operator kernels", "ms": ms,
            "value": n_prim * P / (ms / 1e3) / 1e9, "unit": "Gvoxel-ops/s",
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "algorithmic_bytes": alg},
            "cpu_oracle": {"kind": "oracle", "cores": 1, "sample": "first 8 slices",
                           "value": n_prim * sub[0].size / cpu_s / 1e9, "unit": "Gvoxel-ops/s"}}


def leg_formula_scaling(ctx, stream, flush, image, sizes=(10, 100, 500, 1000, 2000),
                        runs: int = 3) -> dict:
    """Time against formula size (Sec. 4.1): sequential formulas f(g(...(x)))
    and random DAGs of growing size on the same resident 2048 x 2048 image,
    the batched form (tuned per formula: the persistent executor, or the
    per-operator kernels captured in a graph) beside the plain per-operator
    form launched one kernel at a time; at 2000 nodes also the deep-N and
    the reachability chains."""
    import torch
    import workloads as wl
    P = H * W

    def timed(F, mode, n):
        ms = []
        with torch.cuda.stream(stream):
            b = ctx.batch([(F, [image])], stream) if mode == "batched" else None
            if b is not None:  # (a per-operator batch captures its graph on run 2)
                for _ in range(2):
                    b.run(stream)
            for k in range(n + 1):
                flush.zero_()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                if b is not None:
                    b.run(stream)
                else:
                    r = ctx.eval(F, [image], stream=stream, mode="plain")
                z.record(stream)
                stream.synchronize()
                st = b.result(0).status_word() if b is not None else r.sync()
                if st != 0:
                    raise SystemExit(f"formula scaling ({mode}) failed: {ctx.last_error()}")
                if b is None:
                    r.close()
                if k:
                    ms.append(a.elapsed_time(z))
            if b is not None:
                b.close()
        return float(np.mean(ms))

    rows = []
    cases = [("sequential", n, lambda n: wl.sequential_dag(n, seed=0)) for n in sizes]
    cases += [("random", n, lambda n: wl.random_dag(n, seed=0, max_depth=min(500, n)))
              for n in sizes]
    cases += [(f"sequential-{m}", 2000, lambda n, m=m: wl.sequential_dag(n, seed=0, mix=m))
              for m in ("near", "reach")]
    for kind, n, make in cases:
        f = make(n)
        F = ctx.compile(wl.formula_to_records(f), f.roots, CONN)
        info = F.info()
        # the batched form as the autotuner leaves it for this job: a tile
        # shape of the persistent executor, or the per-operator kernels in
        # a graph (0 x 0)
        with torch.cuda.stream(stream):
            best = ctx.autotune([(F, [image])], stream=stream, reps=2)["best"]
        form = ("per-operator graph" if best["tile_rows"] == 0 else
                f"executor {best['tile_rows']}x{best['tile_words']}")
        fused = timed(F, "batched", runs)
        plain = timed(F, "plain", max(2, runs - 1))
        rows.append({"kind": kind, "nodes": n, "n_primitive": info["n_primitive"],
                     "n_reach": info["n_reach"], "form": form, "fused_ms": fused, "plain_ms": plain,
                     "fused_gpixel_ops_s": info["n_primitive"] * P / (fused / 1e3) / 1e9,
                     "fused_over_plain": plain / fused})
        F.close()
    return {"image": [H, W], "connectivity": CONN, "l2": "flushed before every run",
            "rows": rows}


def leg_ccl(ctx, stream, flush, peak: float, S: int = 8192, runs: int = 6) -> dict:
    """Full connected-component labelling (int32 labels, 8-adjacency) of an
    S x S Bernoulli(0.5) mask: 2 untimed runs, then CUDA events per run."""
    import torch
    m = torch.rand((S, S), device="cuda", generator=torch.Generator("cuda").manual_seed(3)) < 0.5
    with torch.cuda.stream(stream):
        mimg = ctx.mask(m.to(torch.uint8), stream)
        labels = torch.empty(S * S, dtype=torch.int32, device="cuda")
        ce = []
        for k in range(runs):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.ccl(mimg, labels, 8, stream)
            b.record(stream)
            if k >= 2:
                ce.append((a, b))
        stream.synchronize()
        if ctx.ccl_status(stream) != 0:
            raise SystemExit("ccl failed: " + ctx.last_error())
    cms = float(np.mean([a.elapsed_time(b) for a, b in ce]))
    mimg.close()
    ach = 4.125 * S * S / (cms / 1e3) / 1e9
    return {"value": S * S / (cms / 1e3) / 1e9, "unit": "Gpix/s", "ms": cms,
            "mask": f"{S}x{S} Bernoulli(0.5), 8-adjacency",
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "algorithmic_bytes": 4.125 * S * S,
                         "kernel": "k_ccl_local + k_ccl_merge + k_ccl_final_labels",
                         "traffic": profiled_traffic("ccl", "dram_bytes_per_labelling")
                         if S == 8192 else None}}


def leg_pointer_jumping(ctx, stream, union_find_ms: float, S: int = 8192, runs: int = 3) -> dict:
    """The paper's pointer-jumping labelling (Alg. 1, reconnect every 16
    main iterations, host-checked termination each round) on the CCL leg's
    mask, timed on the host clock around the synchronous call: the in-library
    comparison for the union-find labelling (context, not a target)."""
    import torch
    m = torch.rand((S, S), device="cuda", generator=torch.Generator("cuda").manual_seed(3)) < 0.5
    with torch.cuda.stream(stream):
        mimg = ctx.mask(m.to(torch.uint8), stream)
        labels = torch.empty(S * S, dtype=torch.int32, device="cuda")
        stream.synchronize()
        ms, iters = [], 0
        for k in range(runs + 1):
            t0 = time.perf_counter()
            iters = ctx.ccl_pointer_jumping(mimg, labels, 8, period=16, stream=stream)
            if k:
                ms.append(1e3 * (time.perf_counter() - t0))
    mimg.close()
    pj = float(np.mean(ms))
    return {"algorithm": "pointer jumping (Alg. 1), reconnect period 16", "ms": pj,
            "main_iterations": iters, "value": S * S / (pj / 1e3) / 1e9, "unit": "Gpix/s",
            "mask": f"{S}x{S} Bernoulli(0.5), 8-adjacency",
            "union_find_speedup": pj / union_find_ms}


def leg_mri_batch(ctx, stream, flush, peak: float, n_images: int = 4096, reps: int = 5) -> dict:
    """4096 MRI-shaped 4-channel images of uneven sizes, the fixed 40-primitive
    segmentation formula with percentile thresholds, one persistent launch
    (autotuned tiles, CUDA graph) per step; beside it the plain per-operator
    form, one image at a time, on a sample of the same images."""
    import torch
    import workloads as wl
    f = wl.config4_formula()
    rec = wl.formula_to_records(f)
    sides = wl.mri_side_lengths(n_images, seed=0)
    imgs = wl.mri_phantom_batch_parallel(sides, seed=0)
    F = ctx.compile(rec, f.roots, 8)
    finfo = F.info()
    n_prim = finfo["n_primitive"]
    px = float(sum(int(im.shape[1]) * int(im.shape[2]) for im in imgs))
    with torch.cuda.stream(stream):
        handles = [ctx.image(im, stream) for im in imgs]
        jobs = [(F, [h]) for h in handles]
        tune = ctx.autotune(jobs, stream=stream, reps=1)
        batch = ctx.batch(jobs, stream)
        for _ in range(2):
            batch.run(stream)
        ev = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.run(stream)
            b.record(stream)
            ev.append((a, b))
        stream.synchronize()
        bad = sum(1 for k in range(0, n_images, 97) if batch.result(k).status_word() != 0)
        if bad:
            raise SystemExit("MRI batch: device status set")
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        # plain per-operator form, one image at a time (a sample)
        sample = list(range(0, n_images, n_images // 64))
        spx = float(sum(int(imgs[k].shape[1]) * int(imgs[k].shape[2]) for k in sample))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in sample:
            r = ctx.eval(F, [handles[k]], stream=stream, mode="plain")
            if r.sync() != 0:
                raise SystemExit("MRI plain form failed")
            r.close()
        plain_s = time.perf_counter() - t0
    batch.close()
    for h in handles:
        h.close()
    val = n_prim * px / (float(np.mean(ms)) / 1e3) / 1e9
    plain = n_prim * spx / plain_s / 1e9
    alg = formula_alg_bytes(finfo, px)
    ach = alg / (float(np.mean(ms)) / 1e3) / 1e9
    # the oracle on every host core over every 16th image
    cpu = oracle_all_cores([(rec, f.roots, imgs[k]) for k in range(0, n_images, 16)])
    return {"workload": f"{n_images} MRI-shaped images 160-512 px (median 240), 4 channels, "
                        "40-primitive formula with percentile thresholds, 8-adjacency",
            "value": val, "unit": "Gpixel-ops/s", "images_per_s": n_images / (float(np.mean(ms)) / 1e3),
            "ms_per_launch": float(np.mean(ms)), "p99_ms": float(np.percentile(ms, 99)),
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "algorithmic_bytes": alg, "kernel": "k_exec",
                         "note": "each image's working set fits in L2"},
            "tiles": {k: tune["best"][k] for k in ("tile_rows", "tile_words", "ctas_per_sm")},
            "plain_one_at_a_time": {"value": plain, "unit": "Gpixel-ops/s",
                                    "images": len(sample), "wall_s": plain_s},
            "batched_over_plain": val / plain,
            "cpu_oracle_all_cores": {"kind": "oracle", "cores": cpu["cores"],
                                     "sample": f"every 16th image ({cpu['tasks']} images)",
                                     "images_per_s": cpu["tasks"] / cpu["wall_s"],
                                     "value": cpu["pixel_ops"] / cpu["wall_s"] / 1e9,
                                     "unit": "Gpixel-ops/s"}}


def device_uniform(side: int, seed: int):
    """A side x side U[0,1) float32 image drawn on the GPU from a seeded
    generator (the serving pool is too large to draw on the host); the same
    call gives the same image again (for the oracle's sample)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.rand((1, side, side), generator=g, device="cuda", dtype=torch.float32)


def leg_serving(ctx, stream, n_queries: int = 20000, n_images: int = 512, n_formulas: int = 96,
                load: float = 0.8, n_other: int = 3000) -> dict:
    """Query stream: a pool of 512 square U[0,1) images with sides
    log-uniform over [128, 4096] resident in HBM, a pool of formulas of
    10-2000 nodes drawn like the random formula (depth cap min(500, n));
    20000 queries (image and formula drawn uniformly from the pools): first
    all at once (saturated throughput), then Poisson arrivals at `load` x
    that rate (p50 / p99 latency); the other arrival rates (0.5 and 0.95 x)
    on the first `n_other` queries; the plain form one query at a time on a
    sample; the oracle on every host core on a bounded sample."""
    import torch
    import paper_2010_07284_gb300 as vg
    import workloads as wl
    from workloads.streams import pool_sides
    rng = np.random.default_rng(5)
    sides = pool_sides(n_images, seed=1)
    with torch.cuda.stream(stream):
        pool = []
        for k, sd in enumerate(sides):
            t = device_uniform(int(sd), 100 + k)
            pool.append(ctx.image(t, stream))
            stream.synchronize()
            del t
    sizes = np.rint(np.exp(np.log(10) + rng.random(n_formulas) * (np.log(2000) - np.log(10)))).astype(int)
    forms = []
    for k, n in enumerate(sizes):
        fd = wl.random_dag(int(n), seed=1000 + k, max_depth=min(500, int(n)))
        forms.append(ctx.compile(wl.formula_to_records(fd), fd.roots, 8))
    prims = [F.info()["n_primitive"] for F in forms]
    qi = rng.integers(0, n_images, size=n_queries)
    qf = rng.integers(0, n_formulas, size=n_queries)
    work = float(sum(prims[f] * int(sides[i]) ** 2 for i, f in zip(qi, qf)))

    def run(arrivals, nq):
        """Submit nq queries (at the arrival times, or all at once) while a
        client thread takes the results in submission order and frees them
        (a result holds its root masks on the device until it is freed)."""
        import queue
        srv = vg.Server(ctx, max_inflight_batches=3, max_batch_jobs=64, batch_window_us=200)
        tickets = queue.Queue()
        failure = []

        def drain():
            for k in range(nq):
                t = tickets.get()
                st, res = srv.wait(t, timeout_us=300_000_000)
                if st != 0:
                    failure.append(f"serving: query {k} (side {int(sides[qi[k]])}, "
                                   f"{int(sizes[qf[k]])} nodes) status {st}: {ctx.last_error()}; "
                                   f"server {json.dumps(srv.stats())}")
                    return
                res.close()

        client = threading.Thread(target=drain)
        t0 = time.perf_counter()
        client.start()
        for k in range(nq):
            if arrivals is not None:
                dt = arrivals[k] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            tickets.put(srv.submit(forms[qf[k]], [pool[qi[k]]]))
        client.join()
        wall = time.perf_counter() - t0
        if failure:
            raise SystemExit(failure[0])
        stats = srv.stats()
        srv.close()
        return wall, stats

    wall_sat, st_sat = run(None, n_queries)
    rate = n_queries / wall_sat

    def poisson(ld, nq):
        gaps = rng.exponential(1.0 / (ld * rate), size=nq)
        arrivals = np.cumsum(gaps) - gaps[0]
        return run(arrivals, nq)

    wall_p, st_p = poisson(load, n_queries)
    others = []
    for ld in (0.5, 0.95):
        w, st = poisson(ld, n_other)
        others.append({"load": ld, "queries": n_other, "rate_per_s": ld * rate,
                       "queries_per_s": n_other / w, "p50_ms": st["p50_ms"],
                       "p99_ms": st["p99_ms"], "batches": st["batches"]})
    # plain form, one query at a time, on a sample
    sample = range(0, n_queries, max(1, n_queries // 100))
    swork = float(sum(prims[qf[k]] * int(sides[qi[k]]) ** 2 for k in sample))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in sample:
        r = ctx.eval(forms[qf[k]], [pool[qi[k]]], mode="plain")
        if r.sync() != 0:
            raise SystemExit("serving plain form failed")
        r.close()
    plain_s = time.perf_counter() - t0
    for im in pool:
        im.close()
    # the oracle on every host core over a seeded draw of at most 64 of the
    # queries whose images are at most 1024^2 (a 4096^2 query with a
    # 2000-node formula takes the oracle minutes; the whole stream would take
    # core-days)
    order = np.random.default_rng(9).permutation(n_queries)
    pick = [int(k) for k in order if int(sides[qi[k]]) <= 1024][:64]
    tasks = []
    for k in pick:
        fd = wl.random_dag(int(sizes[qf[k]]), seed=1000 + int(qf[k]), max_depth=min(500, int(sizes[qf[k]])))
        img = device_uniform(int(sides[qi[k]]), 100 + int(qi[k])).cpu().numpy()
        tasks.append((wl.formula_to_records(fd), fd.roots, img))
    cpu = oracle_all_cores(tasks)
    return {"queries": n_queries, "pool_images": n_images, "pool_formulas": n_formulas,
            "workload": f"{n_queries} queries over {n_images} resident images (sides log-uniform "
                        f"128-4096) and {n_formulas} formulas of 10-2000 nodes, 8-adjacency",
            "saturated": {"queries_per_s": rate, "value": work / wall_sat / 1e9,
                          "unit": "Gpixel-ops/s", "p50_ms": st_sat["p50_ms"], "p99_ms": st_sat["p99_ms"],
                          "batches": st_sat["batches"]},
            "poisson": {"load": load, "rate_per_s": load * rate, "queries_per_s": n_queries / wall_p,
                        "value": work / wall_p / 1e9, "unit": "Gpixel-ops/s",
                        "p50_ms": st_p["p50_ms"], "p99_ms": st_p["p99_ms"], "batches": st_p["batches"]},
            "poisson_other_loads": others,
            "plain_one_at_a_time": {"queries": len(sample), "queries_per_s": len(sample) / plain_s,
                                    "value": swork / plain_s / 1e9, "unit": "Gpixel-ops/s"},
            "cpu_oracle_all_cores": {"kind": "oracle", "cores": cpu["cores"],
                                     "sample": f"{cpu['tasks']} queries (seeded draw, sides <= 1024)",
                                     "cpu_s_per_query": cpu["task_s"] / max(1, cpu["tasks"]),
                                     "queries_per_s": cpu["tasks"] / cpu["wall_s"],
                                     "value": cpu["pixel_ops"] / cpu["wall_s"] / 1e9,
                                     "unit": "Gpixel-ops/s"}}


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_sample(CPU_ROWS_REF)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt, _ = oracle_sample(CPU_ROWS_REF)
        vals.append(v)
        times.append(dt)
    total = sum(times)
    n_prim = oracle_sample(1)[2]
    value = n_prim * CPU_ROWS_REF * W * args.steps / total / 1e9
    sample = f"full {N_NODES}-node formula on the top {CPU_ROWS_REF} rows of the 2048x2048 image per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip plain/ccl/e2e/cpu legs")
    ap.add_argument("--leg", default="", choices=["", "ccl", "scaling", "volume", "serving", "kexec"],
                    help="run only this leg and print its figures (for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    import paper_2010_07284_gb300 as vg
    import workloads as wl

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    ctx = vg.Context(device=local)
    if args.leg == "ccl":
        stream = torch.cuda.Stream()
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        print(json.dumps({"leg": "ccl", **leg_ccl(ctx, stream, flush, measured_peaks()[0])}), flush=True)
        return
    if args.leg == "kexec":
        # the bench's step as the bench runs it (default context, the
        # autotuner's tile shape), launched three times; the third launch
        # sits in an NVTX range "kexec" for a profiler to pick
        fk = wl.random_dag(N_NODES, seed=DAG_SEED)
        Fk = ctx.compile(wl.formula_to_records(fk), fk.roots, CONN)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            im = ctx.image(wl.uniform_image(H, W, seed=0), stream)
            best = ctx.autotune([(Fk, [im])], stream=stream, reps=1)["best"]
            b = ctx.batch([(Fk, [im])], stream)
            for k in range(3):
                if k == 2:
                    stream.synchronize()
                    torch.cuda.nvtx.range_push("kexec")
                b.run(stream)
                if k == 2:
                    stream.synchronize()
                    torch.cuda.nvtx.range_pop()
            stream.synchronize()
            if b.result(0).sync() != 0:
                raise SystemExit("kexec leg failed: " + ctx.last_error())
        print(json.dumps({"leg": "kexec", "launches": 3,
                          "tiles": [best["tile_rows"], best["tile_words"]]}), flush=True)
        return
    if args.leg == "serving":
        stream = torch.cuda.Stream()
        print(json.dumps({"leg": "serving", **leg_serving(ctx, stream)}), flush=True)
        return
    if args.leg == "volume":
        stream = torch.cuda.Stream()
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        print(json.dumps({"leg": "volume", **leg_volume(ctx, stream, flush, measured_peaks()[0])}),
              flush=True)
        return
    if args.leg == "scaling":
        stream = torch.cuda.Stream()
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(stream):
            image = ctx.image(wl.uniform_image(H, W, seed=0), stream)
        print(json.dumps({"leg": "formula_scaling",
                          **leg_formula_scaling(ctx, stream, flush, image)}), flush=True)
        return
    f = wl.random_dag(N_NODES, seed=DAG_SEED)
    rec = wl.formula_to_records(f)
    F = ctx.compile(rec, f.roots, CONN)
    info = F.info()
    n_prim = info["n_primitive"]
    P = H * W
    stream = torch.cuda.Stream()
    host_img = wl.uniform_image(H, W, seed=rank)
    dev_img = torch.from_numpy(host_img).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        image = ctx.image(dev_img, stream)
        # the autotuner times every tile shape on this job and keeps the best
        tune = ctx.autotune([(F, [image])], stream=stream, reps=3)
        batch = ctx.batch([(F, [image])], stream)
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            flush.zero_()
            batch.run(stream)
        stream.synchronize()
        st = batch.result(0).sync()
        if st != 0:
            raise SystemExit(f"device status {st}: {ctx.last_error()}")
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            pass
        clocks = ClockSampler(uuid)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks.start()
        time.sleep(0.25)
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            batch.run(stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        step_ms = np.array([a.elapsed_time(b) for a, b in ev])
        st = batch.result(0).sync()
        if st != 0:
            raise SystemExit(f"device status {st}: {ctx.last_error()}")
    value, total_max = aggregate_throughput(float(step_ms.sum()), args.steps * n_prim * P / 1e9,
                                            world, "cuda")
    ms_per_step = total_max / args.steps

    # roofline of the persistent executor (the only kernel of a step):
    # algorithmic bytes of the whole DAG per launch (formula_alg_bytes)
    alg_bytes = formula_alg_bytes(info, P)
    peak, peak_src = measured_peaks()
    achieved = alg_bytes / (float(np.mean(step_ms)) / 1e3) / 1e9
    traffic = profiled_traffic("k_exec", "dram_bytes_per_launch")
    tiles = {k: tune["best"][k] for k in ("tile_rows", "tile_words", "ctas_per_sm")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": dict(workload_config(world), tiles=tiles),
            "gpu_launches": args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_src} hbm_gbs", "kernel": "k_exec",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "clocks": clk,
            "formula": {"n_primitive": n_prim, "n_reach": info["n_reach"],
                        "n_steps": info["n_steps"], "n_roots": info["n_roots"]}}
    if rank == 0:
        emit_leg("autotune", {"best": tiles, "trials": [
            (t["tile_rows"], t["tile_words"], t["ctas_per_sm"], t["ms"]) for t in tune["trials"]]})

    if not args.no_extras:
        # ---- plain per-operator form, same workload and image
        with torch.cuda.stream(stream):
            pe = []
            for k in range(4):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = ctx.eval(F, [image], stream=stream, mode="plain")
                b.record(stream)
                stream.synchronize()
                if r.sync() != 0:
                    raise SystemExit("plain form failed")
                if k:
                    pe.append(a.elapsed_time(b))
                r.close()
        line["plain"] = {"value": n_prim * P / (np.mean(pe) / 1e3) / 1e9, "unit": UNIT,
                         "ms_per_step": float(np.mean(pe))}
        line["batched_over_plain"] = line["value"] / world / line["plain"]["value"]
        # ---- full CCL on an 8192 x 8192 Bernoulli(0.5) mask
        ccl = leg_ccl(ctx, stream, flush, peak)
        ccl["pointer_jumping"] = leg_pointer_jumping(ctx, stream, ccl["ms"])
        # ---- end to end through the public API with host buffers
        import torch as _t
        pin_in = _t.from_numpy(host_img).pin_memory()
        res_words = info["n_roots"] * H * (((W + 127) // 128) * 4)
        pin_out = _t.empty(res_words, dtype=_t.int32).pin_memory()
        e2e = []
        with torch.cuda.stream(stream):
            for k in range(4):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                im = ctx.image(pin_in.numpy(), stream)
                r = ctx.eval(F, [im], stream=stream)
                r.masks_into(pin_out.numpy(), on_device=False, stream=stream)
                t1 = time.perf_counter()
                if r.sync() != 0:
                    raise SystemExit("e2e failed")
                if k:
                    e2e.append(t1 - t0)
                r.close()
                im.close()
        line["e2e"] = {"value": world * n_prim * P / float(np.mean(e2e)) / 1e9, "unit": UNIT,
                       "h2d_bytes_per_step": int(host_img.nbytes),
                       "d2h_bytes_per_step": int(res_words * 4),
                       "ms_per_step": 1e3 * float(np.mean(e2e))}
        # ---- MRI-shaped batch, the serving stream, the case study, formula size
        mri = leg_mri_batch(ctx, stream, flush, peak)
        serving = leg_serving(ctx, stream)
        grow = leg_grow_7680(ctx, stream, flush, peak)
        volume = leg_volume(ctx, stream, flush, peak)
        scaling = leg_formula_scaling(ctx, stream, flush, image)
        if rank == 0:
            for name, obj in (("ccl", ccl), ("mri_batch", mri), ("serving", serving),
                              ("grow_7680", grow), ("volume", volume),
                              ("formula_scaling", scaling)):
                emit_leg(name, obj)
        # the headline figures of every leg, short enough that the whole
        # result line survives a truncated log
        line["ccl"] = {"value": ccl["value"], "unit": "Gpix/s", "ms": ccl["ms"],
                       "frac": ccl["roofline"]["frac"], "mask": ccl["mask"],
                       "pointer_jumping_ms": ccl["pointer_jumping"]["ms"]}
        line["mri_batch"] = {"value": mri["value"], "images_per_s": mri["images_per_s"],
                             "ms": mri["ms_per_launch"], "frac": mri["roofline"]["frac"],
                             "batched_over_plain": mri["batched_over_plain"]}
        sv = serving
        line["serving"] = {"queries": sv["queries"], "sat_qps": sv["saturated"]["queries_per_s"],
                           "load": sv["poisson"]["load"], "qps": sv["poisson"]["queries_per_s"],
                           "p50_ms": sv["poisson"]["p50_ms"], "p99_ms": sv["poisson"]["p99_ms"],
                           "plain_qps": sv["plain_one_at_a_time"]["queries_per_s"]}
        line["grow_7680"] = {"ms": grow["device_ms"], "e2e_ms": grow["e2e_ms"],
                             "u16_ms": grow["uint16"]["device_ms"],
                             "frac": grow["roofline"]["frac"]}
        line["volume"] = {"value": volume["value"], "unit": volume["unit"], "ms": volume["ms"],
                          "frac": volume["roofline"]["frac"], "shape": "155x240x240x4"}
        rows = scaling["rows"]
        line["formula_scaling"] = {
            "min_fused_over_plain": min(r["fused_over_plain"] for r in rows),
            "fused_plain_ms": [[r["kind"][:12], r["nodes"], r["fused_ms"], r["plain_ms"],
                                "g" if r["form"].startswith("per") else "x"] for r in rows]}
        # ---- CPU oracle on a bounded sample (rank 0 only)
        if rank == 0:
            v, dt, _ = oracle_sample(CPU_ROWS_BASE)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"full formula on the top {CPU_ROWS_BASE} rows "
                                              f"(of 2048) of the image, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(sig(line)), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
