"""Shared test helpers: feed a program to an implementation, compare graphs."""
from __future__ import annotations

import numpy as np

from paper_2503_10516_gb300 import workloads as W

INSTR_FIELDS = ("id", "type", "seq", "a", "b", "c", "d", "box_off", "box_cnt", "bind_off", "bind_cnt")
TYPE_NAMES = ("epoch", "horizon", "alloc", "free", "copy", "send", "receive", "split_receive",
              "await_receive", "kernel")


def feed(impl, prog: W.Program, stop_before_flush: bool = False):
    """Run every op of ``prog`` through an implementation exposing
    create_buffer / submit / flush / destroy_buffer / set_lookahead."""
    results = []
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            impl.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init is not None)
        elif op[0] == "task":
            results.append(impl.submit(op[1]))
        elif op[0] == "flush":
            if stop_before_flush and op is prog.ops[-1]:
                continue
            impl.flush()
        elif op[0] == "destroy":
            impl.destroy_buffer(op[1])
        elif op[0] == "lookahead":
            impl.set_lookahead(op[1])
    return results


class OracleImpl:
    """Adapter: the oracle takes flat task words."""

    def __init__(self, prog: W.Program):
        import oracle
        self.o = oracle.Oracle(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead)
        if prog.stage_d2d:
            self.o.set_stage_d2d(True)
        if prog.horizon_cp:
            self.o.set_horizon_cp(True)
        self.nodes = prog.nodes

    def create_buffer(self, dims, extent, elem, init):
        return self.o.create_buffer(dims, extent, elem, init)

    def submit(self, task):
        return self.o.submit(task.flat())

    def flush(self):
        self.o.flush()

    def destroy_buffer(self, b):
        self.o.destroy_buffer(b)

    def set_lookahead(self, L):
        self.o.set_lookahead(L)

    def graph(self, n):
        return self.o.graph(n)

    def rejected(self):
        return self.o.rejected()


class BruteImpl:
    def __init__(self, prog: W.Program):
        from tests.brute_idag import Brute
        self.b = Brute(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead)
        self.b.stage_d2d = prog.stage_d2d
        self.b.horizon_cp = prog.horizon_cp
        self.nodes = prog.nodes

    def create_buffer(self, dims, extent, elem, init):
        return self.b.create_buffer(dims, extent, elem, init)

    def submit(self, task):
        return self.b.submit(task)

    def flush(self):
        self.b.flush()

    def destroy_buffer(self, b):
        self.b.destroy_buffer(b)

    def set_lookahead(self, L):
        self.b.set_lookahead(L)

    def graph(self, n):
        return self.b.graph(n)

    def rejected(self):
        return list(self.b.rejected)


def oracle_graphs(prog: W.Program):
    impl = OracleImpl(prog)
    feed(impl, prog)
    return [impl.graph(n) for n in range(prog.nodes)], impl.rejected()


def assert_same_graph(g1: dict, g2: dict, label: str = ""):
    for key in ("instrs", "edges", "boxes", "binds", "diags"):
        a, b = g1[key], g2[key]
        if a.shape != b.shape or not np.array_equal(a, b):
            # find first differing row for a readable message
            n = min(len(a), len(b))
            first = next((i for i in range(n) if not np.array_equal(a[i], b[i])), n)
            raise AssertionError(f"{label} {key} differ: shapes {a.shape} vs {b.shape}; first diff row {first}: "
                                 f"{a[first].tolist() if first < len(a) else None} vs "
                                 f"{b[first].tolist() if first < len(b) else None}")


def counts_by_type(g: dict, seq=None) -> dict:
    out = {}
    for r in g["instrs"]:
        if seq is not None and r[2] != seq:
            continue
        name = TYPE_NAMES[r[1]]
        out[name] = out.get(name, 0) + 1
    return out
