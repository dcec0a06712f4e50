"""Python binding of libigs (include/igs.h): argument marshalling only.

Every lowering step and every box copy runs in the library's CUDA kernels;
this module converts Python / numpy arguments to the C structs and back. It
raises if the compiled library is missing — there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libigs.so")

IGS_OK = 0
IGS_ERR_INVALID_ARG, IGS_ERR_OVERLAPPING_WRITE, IGS_ERR_CAPACITY, IGS_ERR_TRUNCATED = -1, -2, -3, -4
IGS_ERR_TIMEOUT, IGS_ERR_CUDA, IGS_ERR_BUDGET, IGS_ERR_STATE = -5, -6, -7, -8
IGS_ERR_OUT_OF_BOUNDS = -9
ERRORS = {-1: "INVALID_ARG", -2: "OVERLAPPING_WRITE", -3: "CAPACITY", -4: "TRUNCATED", -5: "TIMEOUT",
          -6: "CUDA", -7: "BUDGET", -8: "STATE", -9: "OUT_OF_BOUNDS"}
MODE_PLAIN, MODE_BATCHED = 0, 1
TASK_WORDS = W.TASK_HDR + W.ACC_W * W.MAX_ACC  # igs_task as uint32 words
LOOKAHEAD_INFINITE = 0xFFFFFFFF
LOOKAHEAD_HORIZONS = 0xFFFFFFFE  # the horizon-count heuristic (IGS_LOOKAHEAD_HORIZONS)

EXPORTS = ("igs_create", "igs_destroy", "igs_create_buffer", "igs_destroy_buffer", "igs_submit_task",
           "igs_set_lookahead", "igs_flush", "igs_sync", "igs_fetch_instructions", "igs_rejected_tasks",
           "igs_execute", "igs_read_buffer", "igs_lower_batch", "igs_counters", "igs_last_error", "igs_box_copy",
           "igs_set_timing", "igs_stats", "igs_profile", "igs_lower_static", "igs_submit_epoch",
           "igs_serve_create", "igs_serve_destroy", "igs_serve_attach", "igs_serve_start", "igs_serve_progress",
           "igs_serve_detach", "igs_serve_stop", "igs_run", "igs_lower_batch_shaped", "igs_set_executor",
           "igs_exec_stats", "igs_selftest_flow_wait", "igs_bounds_errors", "igs_serve_replay",
           "igs_horizon_plan", "igs_serve_enqueue", "igs_serve_stats", "igs_serve_replay_ex",
           "igs_replay_plain", "igs_set_item_times", "igs_item_times")
EXEC_LEVELS, EXEC_DATAFLOW = 0, 1  # IGS_EXEC_*
ORDER_SUBMISSION, ORDER_LONGEST_FIRST = 0, 1  # IGS_ORDER_*


class IgsError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"igs error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_uint32), ("devices_per_node", ctypes.c_uint32),
                ("horizon_step", ctypes.c_uint32), ("lookahead", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("max_instructions", ctypes.c_uint32), ("max_edges", ctypes.c_uint32),
                ("max_boxes", ctypes.c_uint32), ("map_heap", ctypes.c_uint32),
                ("scratch_capacity", ctypes.c_uint32), ("max_buffers", ctypes.c_uint32),
                ("max_live_allocs", ctypes.c_uint32),
                ("max_allocations", ctypes.c_uint32), ("max_queue", ctypes.c_uint32),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("flags", ctypes.c_uint32)]
FLAG_STAGE_D2D = 1  # IGS_FLAG_STAGE_D2D
FLAG_HORIZON_CP = 2  # IGS_FLAG_HORIZON_CP


class GraphView(ctypes.Structure):
    _fields_ = [("node", ctypes.c_uint32),
                ("instrs", ctypes.c_void_p), ("instr_cap", ctypes.c_uint32), ("num_instrs", ctypes.c_uint32),
                ("edges", ctypes.c_void_p), ("edge_cap", ctypes.c_uint32), ("num_edges", ctypes.c_uint32),
                ("boxes", ctypes.c_void_p), ("box_cap", ctypes.c_uint32), ("num_boxes", ctypes.c_uint32),
                ("binds", ctypes.c_void_p), ("bind_cap", ctypes.c_uint32), ("num_binds", ctypes.c_uint32),
                ("diags", ctypes.c_void_p), ("diag_cap", ctypes.c_uint32), ("num_diags", ctypes.c_uint32)]


class Box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint32 * 3), ("hi", ctypes.c_uint32 * 3)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_uint32), ("idle_timeout_ms", ctypes.c_uint32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("device", ctypes.c_int)]


class StaticBuffer(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_uint32), ("extent", ctypes.c_uint32 * 3), ("elem_size", ctypes.c_uint32),
                ("has_init", ctypes.c_uint32)]


class StaticOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("arg", ctypes.c_uint32)]


class StaticOutput(ctypes.Structure):
    _fields_ = [("instrs", ctypes.c_void_p), ("instr_cap", ctypes.c_uint32),
                ("edges", ctypes.c_void_p), ("edge_cap", ctypes.c_uint32),
                ("boxes", ctypes.c_void_p), ("box_cap", ctypes.c_uint32),
                ("binds", ctypes.c_void_p), ("bind_cap", ctypes.c_uint32),
                ("diags", ctypes.c_void_p), ("diag_cap", ctypes.c_uint32),
                ("counts", ctypes.c_void_p)]


class CopyJob(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("src_box", Box), ("dst_box", Box),
                ("box", Box), ("elem_size", ctypes.c_uint32)]


class BatchShape(ctypes.Structure):
    _fields_ = [("persistent_blocks", ctypes.c_uint32), ("order", ctypes.c_uint32), ("warps", ctypes.c_uint32),
                ("helped", ctypes.c_uint32)]


_lib = None


def lib():
    """Loads libigs.so; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libigs.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, P32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)
        L.igs_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
        L.igs_destroy.argtypes = [vp]
        L.igs_destroy.restype = None
        L.igs_create_buffer.argtypes = [vp, u32, P32, u32, vp, P32]
        L.igs_destroy_buffer.argtypes = [vp, u32]
        L.igs_submit_task.argtypes = [vp, P32, ctypes.POINTER(ctypes.c_uint64)]
        L.igs_set_lookahead.argtypes = [vp, u32]
        L.igs_flush.argtypes = [vp]
        L.igs_run.argtypes = [vp, u32]
        L.igs_set_executor.argtypes = [vp, u32]
        L.igs_exec_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.igs_selftest_flow_wait.argtypes = [u32]
        L.igs_bounds_errors.argtypes = [vp, vp, u32, P32]
        L.igs_serve_replay.argtypes = [vp, ctypes.POINTER(vp), u32, vp, u32, u32, vp, vp]
        L.igs_serve_replay_ex.argtypes = [vp, ctypes.POINTER(vp), u32, vp, u32, u32, u32, vp, vp]
        L.igs_serve_enqueue.argtypes = [vp, vp, u32, P32]
        L.igs_replay_plain.argtypes = [ctypes.POINTER(vp), u32, vp, u32, u32, vp, vp]
        L.igs_set_item_times.argtypes = [vp, ctypes.c_int]
        L.igs_item_times.argtypes = [vp, vp, u32, P32]
        L.igs_serve_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.igs_horizon_plan.argtypes = [vp, u32, vp, u32, u32, u32, vp]
        L.igs_sync.argtypes = [vp]
        L.igs_submit_epoch.argtypes = [vp]
        L.igs_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(vp)]
        L.igs_serve_destroy.argtypes = [vp]
        L.igs_serve_destroy.restype = None
        L.igs_serve_attach.argtypes = [vp, vp, u32]
        L.igs_serve_start.argtypes = [vp]
        L.igs_serve_progress.argtypes = [vp, P32, P32]
        L.igs_serve_detach.argtypes = [vp, vp, u32]
        L.igs_serve_stop.argtypes = [vp]
        L.igs_fetch_instructions.argtypes = [vp, ctypes.POINTER(GraphView)]
        L.igs_rejected_tasks.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), u32, P32]
        L.igs_execute.argtypes = [vp, u32]
        L.igs_read_buffer.argtypes = [vp, u32, P32, P32, vp]
        L.igs_lower_batch.argtypes = [ctypes.POINTER(vp), u32]
        L.igs_lower_batch_shaped.argtypes = [ctypes.POINTER(vp), u32, ctypes.POINTER(BatchShape)]
        L.igs_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.igs_last_error.argtypes = [vp]
        L.igs_last_error.restype = ctypes.c_char_p
        L.igs_box_copy.argtypes = [ctypes.POINTER(CopyJob), u32, vp]
        L.igs_set_timing.argtypes = [vp, ctypes.c_int]
        L.igs_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.igs_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.igs_lower_static.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(StaticBuffer), u32, P32, u32,
                                       ctypes.POINTER(StaticOp), u32, ctypes.POINTER(StaticOutput), vp]
        _lib = L
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class Context:
    """One lowering context (virtual nodes x devices) on one GPU."""

    def __init__(self, nodes: int, devices: int, horizon_step: int = 4, lookahead: int = 0,
                 mode: int = MODE_PLAIN, device: int = 0, stream: Optional[int] = None,
                 max_instructions: int = 0, map_heap: int = 0, scratch_capacity: int = 0,
                 max_buffers: int = 0, max_live_allocs: int = 0,
                 max_allocations: int = 0, max_queue: int = 0, max_edges: int = 0, max_boxes: int = 0,
                 flags: int = 0):
        self.nodes = nodes
        cfg = Config(nodes, devices, horizon_step, lookahead, mode, max_instructions, max_edges, max_boxes, map_heap,
                     scratch_capacity, max_buffers, max_live_allocs, max_allocations,
                     max_queue, device, stream, flags)
        h = ctypes.c_void_p()
        r = lib().igs_create(ctypes.byref(cfg), ctypes.byref(h))
        if r != IGS_OK:
            raise IgsError(r, "igs_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def _check(self, r: int, what: str):
        if r != IGS_OK:
            raise IgsError(r, f"{what}: {lib().igs_last_error(self._h).decode()}")
        return r

    def close(self):
        if getattr(self, "_h", None):
            lib().igs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def create_buffer(self, dims: int, extent: Sequence[int], elem_size: int, init: Optional[np.ndarray]) -> int:
        ext = np.ones(3, dtype=np.uint32)
        ext[:len(extent)] = extent
        out = np.zeros(1, dtype=np.uint32)
        ptr = None
        if init is not None:
            init = np.ascontiguousarray(init)
            ptr = init.ctypes.data_as(ctypes.c_void_p)
        self._check(lib().igs_create_buffer(self._h, dims, _p32(ext), elem_size, ptr, _p32(out)), "create_buffer")
        return int(out[0])

    def destroy_buffer(self, b: int):
        self._check(lib().igs_destroy_buffer(self._h, b), "destroy_buffer")

    def submit(self, task: W.Task) -> int:
        w = np.ascontiguousarray(task.flat(), dtype=np.uint32)
        seq = ctypes.c_uint64()
        self._check(lib().igs_submit_task(self._h, _p32(w), ctypes.byref(seq)), "submit_task")
        return 0

    def set_lookahead(self, L: int):
        self._check(lib().igs_set_lookahead(self._h, L), "set_lookahead")

    def flush(self, allow_rejected: bool = True) -> int:
        r = lib().igs_flush(self._h)
        if r == -2 and allow_rejected:
            return r
        return self._check(r, "flush")

    def sync(self, allow_rejected: bool = True) -> int:
        r = lib().igs_sync(self._h)
        if r == -2 and allow_rejected:
            return r
        return self._check(r, "sync")

    def submit_epoch(self):
        self._check(lib().igs_submit_epoch(self._h), "submit_epoch")

    def graph(self, node: int) -> dict:
        v = GraphView()
        v.node = node
        r = lib().igs_fetch_instructions(self._h, ctypes.byref(v))
        if r not in (IGS_OK, -4):
            self._check(r, "fetch_instructions")
        out = {"instrs": np.zeros((v.num_instrs, 11), np.uint32), "edges": np.zeros((v.num_edges, 3), np.uint32),
               "boxes": np.zeros((v.num_boxes, 6), np.uint32), "binds": np.zeros((v.num_binds, 7), np.uint32),
               "diags": np.zeros((v.num_diags, 3), np.uint32)}
        v.instrs, v.instr_cap = out["instrs"].ctypes.data, v.num_instrs
        v.edges, v.edge_cap = out["edges"].ctypes.data, v.num_edges
        v.boxes, v.box_cap = out["boxes"].ctypes.data, v.num_boxes
        v.binds, v.bind_cap = out["binds"].ctypes.data, v.num_binds
        v.diags, v.diag_cap = out["diags"].ctypes.data, v.num_diags
        self._check(lib().igs_fetch_instructions(self._h, ctypes.byref(v)), "fetch_instructions")
        return out

    def rejected(self) -> list:
        cnt = np.zeros(1, np.uint32)
        buf = (ctypes.c_uint64 * 1024)()
        self._check(lib().igs_rejected_tasks(self._h, buf, 1024, _p32(cnt)), "rejected_tasks")
        return [int(buf[i]) for i in range(min(int(cnt[0]), 1024))]

    def execute(self, sync: bool = True):
        self._check(lib().igs_execute(self._h, 1 if sync else 0), "execute")

    def set_executor(self, executor: int):
        """EXEC_LEVELS (by topological level) or EXEC_DATAFLOW (one
        persistent out-of-order launch per call)."""
        self._check(lib().igs_set_executor(self._h, executor), "set_executor")

    def exec_stats(self) -> dict:
        out = (ctypes.c_double * 8)()
        self._check(lib().igs_exec_stats(self._h, out), "exec_stats")
        keys = ("launches", "nodes", "tiles", "edges", "span_ms", "copy_busy_ms", "kernel_busy_ms", "overlap_ms")
        return dict(zip(keys, list(out)))

    def bounds_errors(self) -> list:
        """Accessor bounds violations recorded so far: dicts with seq, node,
        chunk, accessor and the bounding box (lo, hi) of the indices outside
        the accessor's permitted box."""
        cnt = np.zeros(1, np.uint32)
        self._check(lib().igs_bounds_errors(self._h, None, 0, _p32(cnt)), "bounds_errors")
        rec = np.zeros((max(1, int(cnt[0])), 10), np.uint32)
        self._check(lib().igs_bounds_errors(self._h, rec.ctypes.data, int(cnt[0]), _p32(cnt)), "bounds_errors")
        return [{"seq": int(r[0]), "node": int(r[1]), "chunk": int(r[2]), "accessor": int(r[3]),
                 "lo": tuple(int(v) for v in r[4:7]), "hi": tuple(int(v) for v in r[7:10])}
                for r in rec[:int(cnt[0])]]

    def run(self, window: int = 64):
        """Lowers the pending submissions in windows of `window` items while the
        previous window's instructions execute (igs_run)."""
        r = lib().igs_run(self._h, window)
        if r not in (IGS_OK, IGS_ERR_OVERLAPPING_WRITE):
            self._check(r, "run")
        return r

    def read_buffer(self, b: int, lo, hi, elem_size: int) -> np.ndarray:
        lo3 = np.zeros(3, np.uint32)
        hi3 = np.ones(3, np.uint32)
        lo3[:len(lo)] = lo
        hi3[:len(hi)] = hi
        shape = tuple(int(hi3[d] - lo3[d]) for d in range(3)) + (elem_size,)
        out = np.zeros(shape, np.uint8)
        self._check(lib().igs_read_buffer(self._h, b, _p32(lo3), _p32(hi3), out.ctypes.data_as(ctypes.c_void_p)),
                    "read_buffer")
        return out

    def counters(self) -> dict:
        c = (ctypes.c_uint64 * 8)()
        self._check(lib().igs_counters(self._h, c), "counters")
        return {"instructions": c[0], "edges": c[1], "boxes": c[2], "map_reads": c[3], "map_writes": c[4],
                "launches": c[5]}


def _stats(self) -> dict:
    c = (ctypes.c_double * 8)()
    self._check(lib().igs_stats(self._h, c), "stats")
    return {"lower_ms": c[0], "copy_ms": c[1], "workload_ms": c[2], "copy_bytes": c[3], "lower_launches": int(c[4]),
            "copy_launches": int(c[5]), "workload_launches": int(c[6]), "last_lower_ms": c[7]}


def _set_timing(self, on: bool = True):
    self._check(lib().igs_set_timing(self._h, 1 if on else 0), "set_timing")


def _set_item_times(self, on: bool = True):
    self._check(lib().igs_set_item_times(self._h, 1 if on else 0), "set_item_times")


def _item_times(self):
    """(kinds, times): per submitted item, its kind (0 create, 1 task, 2
    horizon, 3 epoch, 4 destroy, 5 lookahead) and the device time (ns) its
    last node finished lowering it (0 if not yet)."""
    cnt = np.zeros(1, np.uint32)
    self._check(lib().igs_item_times(self._h, None, 0, _p32(cnt)), "item_times")
    n = int(cnt[0])
    out = np.zeros(max(1, 2 * n), np.uint64)
    self._check(lib().igs_item_times(self._h, out.ctypes.data, n, _p32(cnt)), "item_times")
    out = out[:2 * n].reshape(-1, 2)
    return out[:, 0].astype(np.uint32), out[:, 1]


PHASES = ("split", "overlap", "push_await", "allocating", "alloc", "push", "receive", "coherence", "kernel",
          "remote", "sync_emit", "sync_apply", "total", "in_emit", "in_canonical", "in_find_alloc",
          "in_merge", "in_subtract", "in_query", "in_compact", "emit_probe", "emit_dedup", "emit_record",
          "emit_apply", "n_merge", "n_merge_probe", "n_subtract", "n_emit", "n_probe_entries", "n_tidy",
          "n_grow", "n_shared_phases")


def _profile(self) -> dict:
    c = (ctypes.c_uint64 * 32)()
    self._check(lib().igs_profile(self._h, c), "profile")
    return {name: int(c[i]) for i, name in enumerate(PHASES)}


Context.profile = _profile
Context.stats = _stats
Context.set_timing = _set_timing
Context.set_item_times = _set_item_times
Context.item_times = _item_times


def _pack_trace(trace):
    """igs_replay_item records (and the task words they point to) for a trace
    of (context index, Task or None for an epoch, arrival ns)."""
    n = len(trace)
    words = np.zeros((max(1, n), TASK_WORDS), np.uint32)
    items = np.zeros(max(1, n), dtype=np.dtype([("ctx", np.uint32), ("epoch", np.uint32), ("task", np.uint64),
                                                 ("arrival", np.uint64)]))
    base = words.ctypes.data
    for k, (ci, task, t_ns) in enumerate(trace):
        items[k]["ctx"] = ci
        items[k]["arrival"] = int(t_ns)
        if task is None:
            items[k]["epoch"] = 1
        else:
            words[k] = task.flat()
            items[k]["task"] = base + k * TASK_WORDS * 4
    return words, items


def replay_plain(ctxs: Sequence["Context"], trace, timeout_ms: int = 60000):
    """igs_replay_plain: the served loop's comparator, one lowering launch per
    item at its arrival on the item's (plain-mode) context. Returns (per-item
    latency in ns, ns until the last launch completed)."""
    n = len(trace)
    words, items = _pack_trace(trace)
    arr = (ctypes.c_void_p * len(ctxs))(*[c.handle.value for c in ctxs])
    lat = np.zeros(max(1, n), np.uint64)
    wall = np.zeros(1, np.uint64)
    r = lib().igs_replay_plain(arr, len(ctxs), items.ctypes.data, n, timeout_ms, lat.ctypes.data, wall.ctypes.data)
    if r != IGS_OK:
        raise IgsError(r, "replay_plain")
    return lat[:n], int(wall[0])


class Server:
    """Device-resident serving loop over attached contexts."""

    def __init__(self, max_slots: int = 256, hbm_budget_bytes: int = 0, idle_timeout_ms: int = 10000, device: int = 0):
        cfg = ServeConfig(max_slots, idle_timeout_ms, hbm_budget_bytes, device)
        h = ctypes.c_void_p()
        r = lib().igs_serve_create(ctypes.byref(cfg), ctypes.byref(h))
        if r != IGS_OK:
            raise IgsError(r, "serve_create")
        self._h = h

    def attach(self, ctx: Context, max_items: int) -> int:
        """IGS_OK, or the error code (e.g. -7 BUDGET) without raising."""
        return lib().igs_serve_attach(self._h, ctx.handle, max_items)

    def enqueue(self, ctx: Context, max_items: int) -> bool:
        """igs_serve_enqueue: attaches ctx now if it fits (True), else queues it
        for admission after a detach (False). Raises on a context that could
        never fit."""
        adm = np.zeros(1, np.uint32)
        r = lib().igs_serve_enqueue(self._h, ctx.handle, max_items, _p32(adm))
        if r != IGS_OK:
            raise IgsError(r, "serve_enqueue: " + lib().igs_last_error(ctx.handle).decode())
        return bool(adm[0])

    def stats(self) -> dict:
        c = (ctypes.c_uint64 * 8)()
        r = lib().igs_serve_stats(self._h, c)
        if r != IGS_OK:
            raise IgsError(r, "serve_stats")
        return {"admitted": int(c[0]), "admitted_from_queue": int(c[1]), "waiting": int(c[2]),
                "peak_waiting": int(c[3]), "slots_in_use": int(c[4]), "budget_bytes_in_use": int(c[5])}

    def start(self):
        r = lib().igs_serve_start(self._h)
        if r != IGS_OK:
            raise IgsError(r, "serve_start")

    @staticmethod
    def progress(ctx: Context):
        sub = np.zeros(1, np.uint32)
        tk = np.zeros(1, np.uint32)
        r = lib().igs_serve_progress(ctx.handle, _p32(sub), _p32(tk))
        return int(sub[0]), int(tk[0]), r

    def detach(self, ctx: Context, timeout_ms: int = 60000):
        r = lib().igs_serve_detach(self._h, ctx.handle, timeout_ms)
        if r != IGS_OK:
            raise IgsError(r, "serve_detach: " + lib().igs_last_error(ctx.handle).decode())

    def stop(self):
        lib().igs_serve_stop(self._h)

    def replay(self, ctxs: Sequence[Context], trace, timeout_ms: int = 60000, detach: bool = False):
        """igs_serve_replay: trace = [(context index, Task or None for an
        epoch, arrival in ns since the call)] in arrival order. Returns
        (per-item latency in ns as a numpy array, ns until the last item was
        taken). detach: each context is detached once its last item is taken
        (admitting contexts that wait for admission; igs_serve_replay_ex)."""
        n = len(trace)
        words, items = _pack_trace(trace)
        arr = (ctypes.c_void_p * len(ctxs))(*[c.handle.value for c in ctxs])
        lat = np.zeros(max(1, n), np.uint64)
        wall = np.zeros(1, np.uint64)
        r = lib().igs_serve_replay_ex(self._h, arr, len(ctxs), items.ctypes.data, n, timeout_ms,
                                      1 if detach else 0, lat.ctypes.data, wall.ctypes.data)
        if r != IGS_OK:
            raise IgsError(r, "serve_replay")
        return lat[:n], int(wall[0])

    def close(self):
        if getattr(self, "_h", None):
            lib().igs_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def horizon_plan(prog: W.Program) -> List[int]:
    """igs_horizon_plan over the program's tasks: indices of the tasks a
    horizon follows (host computation, no device)."""
    bufs = prog.buffers
    sb = (StaticBuffer * max(1, len(bufs)))()
    for i, b in enumerate(bufs):
        sb[i].dims, sb[i].elem_size, sb[i].has_init = b.dims, b.elem_size, int(b.init is not None)
        for d in range(3):
            sb[i].extent[d] = b.extent[d]
    tasks = prog.tasks
    words = np.concatenate([t.flat() for t in tasks]) if tasks else np.zeros(TASK_WORDS, np.uint32)
    out = np.zeros(max(1, len(tasks)), np.uint8)
    flags = FLAG_HORIZON_CP if prog.horizon_cp else 0
    r = lib().igs_horizon_plan(ctypes.cast(sb, ctypes.c_void_p), len(bufs), words.ctypes.data, len(tasks),
                               prog.horizon_step, flags, out.ctypes.data)
    if r != IGS_OK:
        raise IgsError(r, "horizon_plan")
    return [i for i in range(len(tasks)) if out[i]]


def selftest_flow_wait(wait_ms: int) -> int:
    """Runs the dataflow executor's bounded-wait self-test (a graph in which
    nothing ever becomes ready); returns the status code (IGS_ERR_TIMEOUT
    when the wait gave up as designed)."""
    return lib().igs_selftest_flow_wait(wait_ms)


def lower_batch(ctxs: Sequence[Context], shape: Optional[Tuple[int, ...]] = None):
    """One launch over the pending submissions of every context. shape =
    (persistent_blocks, order[, warps[, helped]]) takes the device work queue
    (igs_batch_shape); None or blocks 0: one block per (program, node)."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.handle.value for c in ctxs])
    if shape is None:
        r = lib().igs_lower_batch(arr, len(ctxs))
    else:
        f = list(shape) + [0] * (4 - len(shape))
        s = BatchShape(*[int(v) for v in f])
        r = lib().igs_lower_batch_shaped(arr, len(ctxs), ctypes.byref(s))
    if r not in (IGS_OK, -2):
        raise IgsError(r, "lower_batch: " + lib().igs_last_error(ctxs[0].handle).decode())


def batch_shape_candidates(n_units: int, sms: int) -> List[Optional[Tuple[int, int, int, int]]]:
    """Shapes worth timing for a batch of n_units (program, node) units on a
    GPU with `sms` SMs: one block per unit; work queues of 1-8 one-warp
    blocks per SM in longest-first order, and 1 and 4 per SM in submission
    order; 1-4 blocks per SM of 4 and 8 warps whose helpers serve the 8 to
    128 heaviest multi-device programs. Never more blocks than units."""
    out: List[Optional[Tuple[int, int, int, int]]] = [None]

    def add(per_sm, order, warps, helped):
        g = min(n_units, per_sm * sms)
        if (g, order, warps, helped) not in out:
            out.append((g, order, warps, helped))

    for per_sm in (1, 2, 4, 8):
        add(per_sm, ORDER_LONGEST_FIRST, 1, 0)
    for per_sm in (1, 4):
        add(per_sm, ORDER_SUBMISSION, 1, 0)
    for per_sm, warps, helped in ((1, 4, 8), (2, 4, 32), (2, 8, 32), (2, 4, 128), (4, 4, 64), (4, 2, 128)):
        add(per_sm, ORDER_LONGEST_FIRST, warps, helped)
    return out


def tune_lower_batch(make_batch: Callable[[], Sequence[Context]], candidates: Sequence[Optional[Tuple[int, int]]],
                     timer: Callable[[], float], repeats: int = 1):
    """Picks a batch shape by timing: for every candidate, make_batch() stages
    a fresh copy of the batch (identical pending submissions) and one
    lower_batch launch over it is timed with timer() (which must synchronise
    the device). Returns (best shape, [(shape, seconds), ...]); each
    candidate's time is its fastest of `repeats` copies."""
    times = []
    for shape in candidates:
        best = float("inf")
        for _ in range(repeats):
            ctxs = make_batch()
            t0 = timer()
            lower_batch(ctxs, shape)
            best = min(best, timer() - t0)
            for c in ctxs:
                c.close()
        times.append((shape, best))
    return min(times, key=lambda t: t[1])[0], times


def lower_static(prog: W.Program, outs: Sequence[dict], stream: Optional[int] = None) -> int:
    """Lowers a whole program through igs_lower_static (no allocation inside
    the library). outs[n]: device pointers and capacities of node n's output
    arrays: keys instrs, edges, boxes, binds, diags (pointer, capacity) and
    counts (pointer to 6 device uint32 words)."""
    bufs = prog.buffers
    sb = (StaticBuffer * max(1, len(bufs)))()
    for i, b in enumerate(bufs):
        sb[i].dims, sb[i].elem_size, sb[i].has_init = b.dims, b.elem_size, int(b.init is not None)
        for d in range(3):
            sb[i].extent[d] = b.extent[d]
    tasks = prog.tasks
    words = np.concatenate([t.flat() for t in tasks]) if tasks else np.zeros(123, np.uint32)
    words = np.ascontiguousarray(words, dtype=np.uint32)
    ops, nb, nt = [], 0, 0
    for op in prog.ops:
        if op[0] == "buffer":
            ops.append((0, nb)); nb += 1
        elif op[0] == "task":
            ops.append((1, nt)); nt += 1
        elif op[0] == "flush":
            ops.append((2, 0))
        elif op[0] == "destroy":
            ops.append((3, op[1]))
        elif op[0] == "lookahead":
            ops.append((4, op[1]))
    so = (StaticOp * max(1, len(ops)))(*[StaticOp(k, a) for k, a in ops])
    out = (StaticOutput * prog.nodes)()
    for n, o in enumerate(outs):
        out[n].instrs, out[n].instr_cap = o["instrs"]
        out[n].edges, out[n].edge_cap = o["edges"]
        out[n].boxes, out[n].box_cap = o["boxes"]
        out[n].binds, out[n].bind_cap = o["binds"]
        out[n].diags, out[n].diag_cap = o["diags"]
        out[n].counts = o["counts"]
    cfg = Config(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, None,
                 (FLAG_STAGE_D2D if prog.stage_d2d else 0) | (FLAG_HORIZON_CP if prog.horizon_cp else 0))
    return lib().igs_lower_static(ctypes.byref(cfg), sb, len(bufs), _p32(words), len(tasks), so, len(ops), out, stream)


def box_copy(jobs: Sequence[tuple], stream: Optional[int] = None):
    """jobs: (src_ptr, src_box, dst_ptr, dst_box, box, elem_size); boxes as 6-tuples (lo3 + hi3)."""
    arr = (CopyJob * len(jobs))()
    for i, (sp, sb, dp, db, bx, es) in enumerate(jobs):
        arr[i].src, arr[i].dst, arr[i].elem_size = sp, dp, es
        for name, b in (("src_box", sb), ("dst_box", db), ("box", bx)):
            B = getattr(arr[i], name)
            for d in range(3):
                B.lo[d], B.hi[d] = b[d], b[3 + d]
    r = lib().igs_box_copy(arr, len(jobs), stream)
    if r != IGS_OK:
        raise IgsError(r, "box_copy")


def small_caps(prog: W.Program, counts: Optional[dict] = None) -> dict:
    """Context capacities sized for one program (so that many contexts fit at
    once). counts: exact per-node maxima {"instrs", "edges", "boxes"} when
    known; otherwise generous estimates from the program's shape."""
    tasks = prog.tasks
    chunks = max((t.chunks for t in tasks), default=1)
    nacc = max((len(t.accessors) for t in tasks), default=1)
    look = min(prog.lookahead, len(tasks)) if prog.lookahead != LOOKAHEAD_INFINITE else len(tasks)
    if counts:
        ni, ne, nb = (int(counts[k] * 1.25) + 256 for k in ("instrs", "edges", "boxes"))
    else:
        ni = len(tasks) * (chunks * (nacc + 3) + 16) + 256
        ne, nb = ni * (chunks + 8), ni * 8
    return {"max_instructions": ni, "max_edges": ne, "max_boxes": nb, "map_heap": 1 << 17,
            "scratch_capacity": max(4096, (look + 2) * chunks * nacc * 2),
            "max_buffers": max(1, len(prog.buffers)), "max_live_allocs": 1024,
            "max_allocations": 16384,
            "max_queue": max(256, 2 * len(prog.ops) + 16)}


class GpuImpl:
    """Adapter with the same methods as the test harness implementations."""

    def __init__(self, prog: W.Program, mode: int = MODE_PLAIN, **kw):
        if prog.stage_d2d:
            kw["flags"] = kw.get("flags", 0) | FLAG_STAGE_D2D
        if prog.horizon_cp:
            kw["flags"] = kw.get("flags", 0) | FLAG_HORIZON_CP
        self.ctx = Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=mode, **kw)
        self.nodes = prog.nodes
        self.prog = prog
        self._buffers = []

    def create_buffer(self, dims, extent, elem, init):
        b = self.prog.buffers[len(self._buffers)]
        self._buffers.append(b)
        return self.ctx.create_buffer(dims, extent, elem, b.init if init else None)

    def submit(self, task):
        self.ctx.submit(task)
        return 0

    def flush(self):
        self.ctx.flush()

    def destroy_buffer(self, b):
        self.ctx.destroy_buffer(b)

    def set_lookahead(self, L):
        self.ctx.set_lookahead(L)

    def graph(self, n):
        return self.ctx.graph(n)

    def rejected(self):
        return self.ctx.rejected()
