"""CPU oracle for the instruction-graph lowering — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never does.

``igs_oracle.cpp`` restates the lowering rules of the paper (Sec. 3, Sec. 4.3,
Sec. 4.4) on plain box lists; this module compiles it with g++ on first use
and exposes it through ctypes, returning numpy record arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "igs_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

INSTR_W, EDGE_W, BOX_W, BIND_W, DIAG_W = 11, 3, 6, 7, 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain g++, -O2, no vector ISA flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32, vp = ctypes.c_uint32, ctypes.c_void_p
            P = ctypes.POINTER(ctypes.c_uint32)
            L.orc_create.restype = vp
            L.orc_create.argtypes = [u32, u32, u32, u32]
            L.orc_destroy.argtypes = [vp]
            L.orc_create_buffer.argtypes = [vp, u32, P, u32, ctypes.c_int]
            L.orc_create_buffer.restype = ctypes.c_int
            L.orc_destroy_buffer.argtypes = [vp, u32]
            L.orc_submit_task.argtypes = [vp, P]
            L.orc_submit_task.restype = ctypes.c_int
            L.orc_set_lookahead.argtypes = [vp, u32]
            L.orc_set_stage_d2d.argtypes = [vp, ctypes.c_int]
            L.orc_set_horizon_cp.argtypes = [vp, ctypes.c_int]
            L.orc_flush.argtypes = [vp]
            L.orc_count.argtypes = [vp, u32, ctypes.c_int]
            L.orc_count.restype = u32
            L.orc_copy_out.argtypes = [vp, u32, ctypes.c_int, P]
            L.orc_canonical.argtypes = [P, u32, P]
            L.orc_canonical.restype = u32
            L.orc_minus.argtypes = [P, u32, P, u32, P, u32]
            L.orc_minus.restype = u32
            _lib = L
        return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def canonical(boxes) -> np.ndarray:
    """Canonical (row-major maximal) form of a disjoint box list, shape (n, 6)."""
    a = np.ascontiguousarray(np.asarray(boxes, dtype=np.uint32).reshape(-1, 6))
    out = np.zeros((max(1, len(a) * 64), 6), dtype=np.uint32)
    n = lib().orc_canonical(_ptr(a), len(a), _ptr(out))
    return out[:n].copy()


def minus(a, b) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32).reshape(-1, 6))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint32).reshape(-1, 6))
    cap = max(16, 6 ** min(len(b), 6) * max(1, len(a)))
    out = np.zeros((cap, 6), dtype=np.uint32)
    n = lib().orc_minus(_ptr(a), len(a), _ptr(b), len(b), _ptr(out), cap)
    assert n != 0xFFFFFFFF
    return out[:n].copy()


class Oracle:
    """One lowering context: virtual nodes x devices, horizon cadence, lookahead."""

    def __init__(self, nodes: int, devices: int, horizon_step: int = 4, lookahead: int = 0):
        self.nodes = nodes
        self._h = lib().orc_create(nodes, devices, horizon_step, lookahead)
        if not self._h:
            raise ValueError("invalid oracle configuration")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def create_buffer(self, dims: int, extent, elem_size: int, has_init: bool) -> int:
        ext = np.zeros(3, dtype=np.uint32)
        ext[: len(extent)] = extent
        r = lib().orc_create_buffer(self._h, dims, _ptr(ext), elem_size, int(bool(has_init)))
        if r < 0:
            raise ValueError("invalid buffer")
        return r

    def destroy_buffer(self, b: int) -> None:
        lib().orc_destroy_buffer(self._h, b)

    def submit(self, flat_task: np.ndarray) -> int:
        w = np.ascontiguousarray(flat_task, dtype=np.uint32)
        return lib().orc_submit_task(self._h, _ptr(w))

    def set_stage_d2d(self, on: bool) -> None:
        """Device-to-device copies staged in host memory (R27)."""
        lib().orc_set_stage_d2d(self._h, 1 if on else 0)

    def set_horizon_cp(self, on: bool) -> None:
        """Horizons by the task graph's critical path (R29)."""
        lib().orc_set_horizon_cp(self._h, 1 if on else 0)

    def set_lookahead(self, L: int) -> None:
        lib().orc_set_lookahead(self._h, L)

    def flush(self) -> None:
        lib().orc_flush(self._h)

    def _get(self, node: int, what: int, width: int) -> np.ndarray:
        n = lib().orc_count(self._h, node, what)
        out = np.zeros((n, width), dtype=np.uint32)
        if n:
            lib().orc_copy_out(self._h, node, what, _ptr(out))
        return out

    def graph(self, node: int) -> dict:
        """All output of one node: instructions, edges, boxes, bindings, diagnostics."""
        return {
            "instrs": self._get(node, 0, INSTR_W),
            "edges": self._get(node, 1, EDGE_W),
            "boxes": self._get(node, 2, BOX_W),
            "binds": self._get(node, 3, BIND_W),
            "diags": self._get(node, 4, DIAG_W),
        }

    def rejected(self) -> list:
        return [int(x) for x in self._get(0, 5, 1).reshape(-1)]
