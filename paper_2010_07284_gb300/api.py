"""Python front-end of the C ABI (include/vl.h): thin handle classes that
marshal arguments to the CUDA library.  Host arrays are numpy; device arrays
are torch CUDA tensors (PyTorch supplies device memory and streams only)."""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import _native as N

NodeRec = Tuple[str, int, int, int, int, float, float]


def _stream_handle(stream) -> int:
    """cudaStream_t of a torch stream / int / None (= torch's current stream)."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class _Handle:
    _ptr: Optional[int] = None

    def _check(self, rc: int, ctx=None):
        if rc != N.OK:
            c = ctx if ctx is not None else getattr(self, "ctx", None)
            msg = N.load().vl_last_error(c._ptr).decode() if c is not None and c._ptr else ""
            raise N.VlError(rc, msg)

    def close(self):
        if self._ptr:
            N.load().vl_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context(_Handle):
    def __init__(self, device: int = 0, exec_mode: str = "fused", use_graphs: bool = True,
                 spin_limit: int = 0, tile_rows: int = 0, tile_words: int = 0,
                 trace: bool = False):
        lib = N.load()
        cfg = N.VlConfig()
        lib.vl_config_default(C.byref(cfg))
        cfg.device = device
        cfg.exec_mode = N.EXEC_PLAIN if exec_mode == "plain" else N.EXEC_FUSED
        cfg.use_graphs = 1 if use_graphs else 0
        cfg.trace = 1 if trace else 0
        cfg.spin_limit = spin_limit
        cfg.tile_rows = tile_rows
        cfg.tile_words = tile_words
        out = C.c_void_p()
        rc = lib.vl_context_create(C.byref(cfg), C.byref(out))
        if rc != N.OK:
            raise N.VlError(rc, "context creation failed")
        self._ptr = out.value
        self.ctx = self

    # ------------------------------------------------------------ images
    def image(self, data, stream=None) -> "Image":
        """Number image (C, H, W) from a numpy array (host) or a CUDA tensor:
        uint16 data stays uint16 on the device, anything else becomes
        float32."""
        lib = N.load()
        out = C.c_void_p()
        if _is_torch_cuda(data):
            import torch
            u16 = getattr(torch, "uint16", None)
            t = data.contiguous()
            if u16 is None or t.dtype != u16:
                t = t.float()
            if t.dim() == 2:
                t = t[None]
            c, h, w = t.shape
            fn = lib.vl_image_create_u16 if t.dtype != torch.float32 else lib.vl_image_create
            rc = fn(self._ptr, h, w, c, t.data_ptr(), 1, _stream_handle(stream), C.byref(out))
            keep = t
        else:
            a = np.asarray(data)
            a = np.ascontiguousarray(a, dtype=np.uint16 if a.dtype == np.uint16 else np.float32)
            if a.ndim == 2:
                a = a[None]
            c, h, w = a.shape
            fn = lib.vl_image_create_u16 if a.dtype == np.uint16 else lib.vl_image_create
            rc = fn(self._ptr, h, w, c, a.ctypes.data, 0, _stream_handle(stream), C.byref(out))
            keep = a
        self._check(rc)
        return Image(self, out.value, keep)

    def mask(self, data, stream=None) -> "Image":
        """Binary image (H, W) from bytes/bools (numpy host or CUDA uint8 tensor)."""
        lib = N.load()
        out = C.c_void_p()
        if _is_torch_cuda(data):
            import torch
            t = data.contiguous().to(torch.uint8)
            h, w = t.shape
            rc = lib.vl_mask_create(self._ptr, h, w, t.data_ptr(), 1, _stream_handle(stream), C.byref(out))
            keep = t
        else:
            a = np.ascontiguousarray(np.asarray(data) != 0, dtype=np.uint8)
            h, w = a.shape
            rc = lib.vl_mask_create(self._ptr, h, w, a.ctypes.data, 0, _stream_handle(stream), C.byref(out))
            keep = a
        self._check(rc)
        return Image(self, out.value, keep)

    def volume(self, data, stream=None) -> "Image":
        """Number volume (C, D, H, W) from a host numpy array: uint16 stays
        uint16, anything else becomes float32.  Stored as D slices stacked."""
        lib = N.load()
        out = C.c_void_p()
        a = np.asarray(data)
        a = np.ascontiguousarray(a, dtype=np.uint16 if a.dtype == np.uint16 else np.float32)
        if a.ndim == 3:
            a = a[None]
        c, d, h, w = a.shape
        fn = lib.vl_volume_create_u16 if a.dtype == np.uint16 else lib.vl_volume_create
        self._check(fn(self._ptr, d, h, w, c, a.ctypes.data, 0, _stream_handle(stream),
                       C.byref(out)))
        return Image(self, out.value, a)

    def mask_volume(self, data, stream=None) -> "Image":
        """Binary volume (D, H, W) from a host array (nonzero = true)."""
        lib = N.load()
        out = C.c_void_p()
        a = np.ascontiguousarray(np.asarray(data) != 0, dtype=np.uint8)
        d, h, w = a.shape
        self._check(lib.vl_mask_volume_create(self._ptr, d, h, w, a.ctypes.data, 0,
                                              _stream_handle(stream), C.byref(out)))
        return Image(self, out.value, a)

    def mask_packed(self, words, h: int, w: int, stream=None) -> "Image":
        lib = N.load()
        out = C.c_void_p()
        if _is_torch_cuda(words):
            t = words.contiguous()
            rc = lib.vl_mask_create_packed(self._ptr, h, w, t.data_ptr(), 1, _stream_handle(stream), C.byref(out))
            keep = t
        else:
            a = np.ascontiguousarray(words, dtype=np.uint32)
            rc = lib.vl_mask_create_packed(self._ptr, h, w, a.ctypes.data, 0, _stream_handle(stream), C.byref(out))
            keep = a
        self._check(rc)
        return Image(self, out.value, keep)

    # ---------------------------------------------------------- formulas
    def compile(self, nodes: Sequence, roots: Sequence[int], conn: int = 8) -> "Formula":
        lib = N.load()
        arr = (N.VlNode * max(1, len(nodes)))()
        for i, nd in enumerate(nodes):
            op, a, b, img, ch, t, q = tuple(nd)
            arr[i] = N.VlNode(N.OPCODES[op] if isinstance(op, str) else int(op), int(a), int(b),
                              int(img), int(ch), float(np.float32(t)), float(q))
        rts = (C.c_int32 * max(1, len(roots)))(*[int(r) for r in roots])
        out = C.c_void_p()
        rc = lib.vl_formula_compile(self._ptr, arr, len(nodes), rts, len(roots), conn, C.byref(out))
        self._check(rc)
        return Formula(self, out.value)

    def compile_text(self, src: str, conn: int = 8) -> "Formula":
        """A specification text (vl_formula_compile_text) planned for this
        context; images go in the order of its loads."""
        return Formula(self, _compile_text(self._ptr, src, conn))

    # -------------------------------------------------------- evaluation
    def eval(self, formula: "Formula", images: Sequence["Image"], stream=None,
             mode: Optional[str] = None) -> "Result":
        lib = N.load()
        arr = (C.c_void_p * len(images))(*[im._ptr for im in images])
        out = C.c_void_p()
        if mode is None:
            rc = lib.vl_eval(self._ptr, formula._ptr, arr, len(images), _stream_handle(stream), C.byref(out))
        else:
            m = N.EXEC_PLAIN if mode == "plain" else N.EXEC_FUSED
            rc = lib.vl_eval_mode(self._ptr, formula._ptr, arr, len(images), m,
                                  _stream_handle(stream), C.byref(out))
        self._check(rc)
        return Result(self, out.value, keep=(formula, list(images)))

    def _jobs(self, jobs):
        arrs = []
        cj = (N.VlJob * len(jobs))()
        for k, (f, ims) in enumerate(jobs):
            a = (C.c_void_p * len(ims))(*[im._ptr for im in ims])
            arrs.append(a)
            cj[k] = N.VlJob(f._ptr, C.cast(a, C.POINTER(C.c_void_p)), len(ims), 0)
        return cj, arrs

    def eval_batch(self, jobs: Sequence[Tuple["Formula", Sequence["Image"]]], stream=None) -> List["Result"]:
        lib = N.load()
        cj, arrs = self._jobs(jobs)
        outs = (C.c_void_p * len(jobs))()
        rc = lib.vl_eval_batch(self._ptr, cj, len(jobs), _stream_handle(stream), outs)
        self._check(rc)
        return [Result(self, outs[k], keep=jobs[k]) for k in range(len(jobs))]

    def batch(self, jobs: Sequence[Tuple["Formula", Sequence["Image"]]], stream=None) -> "Batch":
        lib = N.load()
        cj, arrs = self._jobs(jobs)
        out = C.c_void_p()
        rc = lib.vl_batch_prepare(self._ptr, cj, len(jobs), _stream_handle(stream), C.byref(out))
        self._check(rc)
        return Batch(self, out.value, len(jobs), keep=list(jobs))

    # ---------------------------------------------------------- autotune
    @staticmethod
    def _choice(c) -> dict:
        return {"tile_rows": c.tile_rows, "tile_words": c.tile_words,
                "ctas_per_sm": c.ctas_per_sm, "status": c.status, "ms": c.ms}

    def autotune(self, jobs: Sequence[Tuple["Formula", Sequence["Image"]]], stream=None,
                 reps: int = 3) -> dict:
        """Time every candidate tile shape on these jobs; the fastest becomes
        the shape of later batches with the same signature."""
        lib = N.load()
        cj, arrs = self._jobs(jobs)
        trials = (N.VlTileChoice * 32)()
        n = C.c_int32()
        best = N.VlTileChoice()
        rc = lib.vl_autotune(self._ptr, cj, len(jobs), _stream_handle(stream), reps, trials, 32,
                             C.byref(n), C.byref(best))
        self._check(rc)
        return {"best": self._choice(best),
                "trials": [self._choice(trials[k]) for k in range(min(32, n.value))]}

    def tile_shape(self, jobs: Sequence[Tuple["Formula", Sequence["Image"]]]) -> dict:
        """The shape a batch of these jobs would use now (and whether it was measured)."""
        cj, arrs = self._jobs(jobs)
        out = N.VlTileChoice()
        tuned = C.c_int32()
        self._check(N.load().vl_tile_shape(self._ptr, cj, len(jobs), C.byref(out), C.byref(tuned)))
        d = self._choice(out)
        d["tuned"] = bool(tuned.value)
        return d

    def save_tuning(self, path: str) -> None:
        self._check(N.load().vl_tune_save(self._ptr, str(path).encode()))

    def load_tuning(self, path: str) -> None:
        self._check(N.load().vl_tune_load(self._ptr, str(path).encode()))

    # --------------------------------------------------------------- ccl
    def ccl(self, mask: "Image", labels, conn: int = 8, stream=None) -> None:
        """Labels into a caller-owned int32 CUDA tensor of H*W elements."""
        rc = N.load().vl_ccl(self._ptr, mask._ptr, conn, labels.data_ptr(), _stream_handle(stream))
        self._check(rc)

    def ccl_pointer_jumping(self, mask: "Image", labels, conn: int = 8, period: int = 16,
                            max_rounds: int = 0, stream=None) -> int:
        """The paper's pointer-jumping labelling (comparison only) into a
        caller-owned int32 CUDA tensor of H*W elements; synchronous.  Labels
        are one pixel index per component (not the minimum).  Returns the
        number of main iterations."""
        it = C.c_int32()
        rc = N.load().vl_ccl_pointer_jumping(self._ptr, mask._ptr, conn, period, max_rounds,
                                             labels.data_ptr(), _stream_handle(stream), C.byref(it))
        self._check(rc)
        return it.value

    def ccl_status(self, stream=None) -> int:
        return N.load().vl_ccl_status(self._ptr, _stream_handle(stream))

    def last_error(self) -> str:
        return N.load().vl_last_error(self._ptr).decode()

    def close(self):
        super().close()


class Image(_Handle):
    def __init__(self, ctx: Context, ptr: int, keep=None):
        self.ctx, self._ptr, self._keep = ctx, ptr, keep
        h, w, c, m = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        N.load().vl_image_info(ptr, C.byref(h), C.byref(w), C.byref(c), C.byref(m))
        self.h, self.w, self.channels, self.is_mask = h.value, w.value, c.value, bool(m.value)
        self.format = None  # masks
        if not self.is_mask:
            f = C.c_int32()
            N.load().vl_image_format(ptr, C.byref(f))
            self.format = "u16" if f.value == N.PX_U16 else "f32"

    def release_source(self):
        """Drop the reference to the source array once the stream has copied it."""
        self._keep = None


def compile_formula(nodes: Sequence, roots: Sequence[int], conn: int = 8) -> "Formula":
    """Compile without a context (host only): the plan targets the default
    tile configuration."""
    lib = N.load()
    arr = (N.VlNode * max(1, len(nodes)))()
    for i, nd in enumerate(nodes):
        op, a, b, img, ch, t, q = tuple(nd)
        arr[i] = N.VlNode(N.OPCODES[op] if isinstance(op, str) else int(op), int(a), int(b),
                          int(img), int(ch), float(np.float32(t)), float(q))
    rts = (C.c_int32 * max(1, len(roots)))(*[int(r) for r in roots])
    out = C.c_void_p()
    rc = lib.vl_formula_compile(None, arr, len(nodes), rts, len(roots), conn, C.byref(out))
    if rc != N.OK:
        raise N.VlError(rc, "formula compilation failed")
    return Formula(None, out.value)


def _compile_text(ctx_ptr, src: str, conn: int) -> int:
    lib = N.load()
    out = C.c_void_p()
    err = C.create_string_buffer(512)
    rc = lib.vl_formula_compile_text(ctx_ptr, src.encode(), conn, C.byref(out), err, len(err))
    if rc != N.OK:
        raise N.VlError(rc, err.value.decode() or "specification rejected")
    return out.value


def compile_text(src: str, conn: int = 8) -> "Formula":
    """Compile a specification text (vl_formula_compile_text) without a
    context (host only); images go in the order of its loads, roots are its
    saves (Formula.loads, Formula.saves)."""
    return Formula(None, _compile_text(None, src, conn))


class Formula(_Handle):
    def __init__(self, ctx: Optional[Context], ptr: int):
        self.ctx, self._ptr = ctx, ptr

    def _names(self, which: int) -> list:
        lib = N.load()
        n = C.c_int32()
        self._check(lib.vl_formula_spec_names(self._ptr, which, C.byref(n), 0, None, 0))
        buf = C.create_string_buffer(256)
        out = []
        for k in range(n.value):
            self._check(lib.vl_formula_spec_names(self._ptr, which, None, k, buf, len(buf)))
            out.append(buf.value.decode())
        return out

    @property
    def loads(self) -> list:
        """Image names of a formula compiled from text, in image order."""
        return self._names(0)

    @property
    def saves(self) -> list:
        """Output names of a formula compiled from text, in root order."""
        return self._names(1)

    @property
    def sources(self) -> list:
        """What each load of a formula compiled from text names, in image order."""
        return self._names(2)

    def plan(self) -> dict:
        """The compiled execution plan (steps, instructions, selects, slots)."""
        lib = N.load()
        sz = N.VlPlanSizes()
        self._check(lib.vl_formula_plan(self._ptr, C.byref(sz), None, None, None, None, None, None))
        steps = (N.VlPlanStep * max(1, sz.n_steps))()
        insns = (N.VlPlanInsn * max(1, sz.n_insns))()
        sels = (N.VlPlanSelect * max(1, sz.n_selects))()
        pct = (N.VlPlanPct * max(1, sz.n_pct))()
        roots = (C.c_int32 * max(1, sz.n_roots))()
        masks = (C.c_int32 * max(1, sz.n_mask_slots))()
        self._check(lib.vl_formula_plan(self._ptr, C.byref(sz), steps, insns, sels, pct, roots, masks))
        rec = lambda x: {f: getattr(x, f) for f, _ in x._fields_}
        rt = (N.VlPlanRank * max(1, sz.n_rank_tables))()
        rv = (C.c_float * max(1, sz.n_rank_values))()
        self._check(lib.vl_formula_rank_tables(self._ptr, rt, rv))
        doff = (C.c_int32 * (sz.n_steps + 1))()
        deps = (C.c_int32 * max(1, sz.n_deps))()
        self._check(lib.vl_formula_step_deps(self._ptr, doff, deps))
        na, nn, first = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(lib.vl_formula_arith(self._ptr, None, C.byref(na), C.byref(nn), C.byref(first)))
        ar = (N.VlPlanArith * max(1, na.value))()
        self._check(lib.vl_formula_arith(self._ptr, ar, None, None, None))
        return {
            "arith": [rec(ar[i]) for i in range(na.value)],
            "n_number_images": nn.value,
            "first_number_image": first.value,
            "deps": [list(deps[doff[i]:doff[i + 1]]) for i in range(sz.n_steps)],
            "rank_tables": [rec(rt[i]) for i in range(sz.n_rank_tables)],
            "rank_values": np.array(rv[:sz.n_rank_values], dtype=np.float32),
            "sizes": rec(sz),
            "steps": [rec(steps[i]) for i in range(sz.n_steps)],
            # opcode bit 7: a block barrier precedes the instruction
            "insns": [dict(rec(insns[i]), op=insns[i].op & 0x7F, sync=bool(insns[i].op & 0x80))
                      for i in range(sz.n_insns)],
            "selects": [rec(sels[i]) for i in range(sz.n_selects)],
            "pct": [rec(pct[i]) for i in range(sz.n_pct)],
            "root_slots": [roots[i] for i in range(sz.n_roots)],
            "mask_slot_images": [masks[i] for i in range(sz.n_mask_slots)],
        }

    def info(self) -> dict:
        s = N.VlFormulaStats()
        self._check(N.load().vl_formula_stats_get(self._ptr, C.byref(s)))
        return {f: getattr(s, f) for f, _ in N.VlFormulaStats._fields_}

    @property
    def n_primitive(self) -> int:
        return self.info()["n_primitive"]


class Result(_Handle):
    def __init__(self, ctx: Context, ptr: int, keep=None, borrowed: bool = False):
        self.ctx, self._ptr, self._keep, self._borrowed = ctx, ptr, keep, borrowed
        h, w, wp, nr = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        N.load().vl_result_info(ptr, C.byref(h), C.byref(w), C.byref(wp), C.byref(nr))
        self.h, self.w, self.wp, self.n_roots = h.value, w.value, wp.value, nr.value

    def sync(self) -> int:
        """Wait; returns the device status (0 ok) without raising."""
        return N.load().vl_result_sync(self._ptr)

    def check(self) -> None:
        self._check(self.sync())

    def status_word(self) -> int:
        w = C.c_int32()
        self._check(N.load().vl_result_status_word(self._ptr, C.byref(w)))
        return w.value

    def mask(self, root: int = 0, stream=None) -> np.ndarray:
        """Root mask as (H, W) uint8 on the host (unpacked by a device kernel);
        (D, H, W) for a volume."""
        out = np.empty((self.h, self.w), dtype=np.uint8)
        self._check(N.load().vl_result_mask_u8(self._ptr, root, out.ctypes.data, 0, _stream_handle(stream)))
        d = self.depth()
        return out.reshape(d, self.h // d, self.w) if d > 1 else out

    def depth(self) -> int:
        d = C.c_int32()
        self._check(N.load().vl_result_depth(self._ptr, C.byref(d)))
        return d.value

    def mask_packed(self, root: int = 0, stream=None) -> np.ndarray:
        out = np.empty((self.h, self.wp), dtype=np.uint32)
        self._check(N.load().vl_result_mask(self._ptr, root, out.ctypes.data, 0, _stream_handle(stream)))
        return out

    def mask_into(self, root: int, dst, on_device: bool, stream=None) -> None:
        ptr = dst.data_ptr() if on_device else dst.ctypes.data
        self._check(N.load().vl_result_mask(self._ptr, root, ptr, 1 if on_device else 0,
                                            _stream_handle(stream)))

    def masks_into(self, dst, on_device: bool, stream=None) -> None:
        """All roots, packed, back to back (n_roots x H x Wp uint32)."""
        ptr = dst.data_ptr() if on_device else dst.ctypes.data
        self._check(N.load().vl_result_masks(self._ptr, ptr, 1 if on_device else 0,
                                             _stream_handle(stream)))

    def device_ptr(self, root: int = 0) -> int:
        p = C.c_void_p()
        self._check(N.load().vl_result_device_ptr(self._ptr, root, C.byref(p)))
        return p.value

    def close(self):
        if not self._borrowed:
            super().close()
        self._ptr = None


class Batch(_Handle):
    def __init__(self, ctx: Context, ptr: int, n_jobs: int, keep=None):
        self.ctx, self._ptr, self.n_jobs, self._keep = ctx, ptr, n_jobs, keep

    def run(self, stream=None) -> None:
        self._check(N.load().vl_batch_run(self._ptr, _stream_handle(stream)))

    def result(self, job: int) -> Result:
        p = C.c_void_p()
        self._check(N.load().vl_batch_result(self._ptr, job, C.byref(p)))
        return Result(self.ctx, p.value, borrowed=True)

    def trace(self) -> np.ndarray:
        """Step timeline of the last run: rows {job, step, kind, start_ns,
        end_ns, busy_ns, wait_ns}."""
        lib = N.load()
        n = C.c_int64()
        self._check(lib.vl_batch_trace(self._ptr, None, 0, C.byref(n)))
        out = np.zeros((n.value, 7), dtype=np.int64)
        self._check(lib.vl_batch_trace(self._ptr, out.ctypes.data_as(C.POINTER(C.c_int64)),
                                       n.value, C.byref(n)))
        return out

    def info(self) -> dict:
        n, g, s = C.c_int64(), C.c_int32(), C.c_int64()
        self._check(N.load().vl_batch_info(self._ptr, C.byref(n), C.byref(g), C.byref(s)))
        return {"n_items": n.value, "grid": g.value, "smem_bytes": s.value}


class Server(_Handle):
    """Continuous-batching serving loop running on its own host thread."""

    def __init__(self, ctx: Context, max_inflight_batches: int = 2, max_batch_jobs: int = 256,
                 memory_budget: int = 0, batch_window_us: int = 200):
        cfg = N.VlServerConfig()
        cfg.max_inflight_batches = max_inflight_batches
        cfg.max_batch_jobs = max_batch_jobs
        cfg.memory_budget = memory_budget
        cfg.batch_window_us = batch_window_us
        out = C.c_void_p()
        self.ctx = ctx
        self._check(N.load().vl_server_create(ctx._ptr, C.byref(cfg), C.byref(out)))
        self._ptr = out.value
        self._keep = {}

    def submit(self, formula: Formula, images: Sequence[Image]) -> int:
        arr = (C.c_void_p * len(images))(*[im._ptr for im in images])
        t = C.c_int64()
        self._check(N.load().vl_server_submit(self._ptr, formula._ptr, arr, len(images), C.byref(t)))
        self._keep[t.value] = (formula, list(images))
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1):
        """(status, Result or None); status 0 = done, ERR_BUSY = still running."""
        out = C.c_void_p()
        rc = N.load().vl_server_wait(self._ptr, ticket, timeout_us, C.byref(out))
        if rc == N.ERR_BUSY:
            return rc, None
        keep = self._keep.pop(ticket, None)
        res = Result(self.ctx, out.value, keep=keep) if out.value else None
        return rc, res

    def cancel(self, ticket: int) -> int:
        return N.load().vl_server_cancel(self._ptr, ticket)

    def stats(self) -> dict:
        st = N.VlServerStats()
        self._check(N.load().vl_server_stats_get(self._ptr, C.byref(st)))
        return {f: getattr(st, f) for f, _ in N.VlServerStats._fields_}
