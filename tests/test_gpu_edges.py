"""Edge and degenerate cases of the CUDA lowering and executor, each against
the oracle's graphs and the sequential contents: no tasks at all, one-element
buffers, more chunks than rows, the most virtual nodes (32) and devices per
node (29, memory ids up to 30), every accessor slot used, empty mapped boxes,
and a program lowered twice in one context (flush in between)."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs
from tests.replay import sequential_run

pytestmark = pytest.mark.gpu


def _u32(n, seed):
    return np.random.default_rng(seed).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)


def _check(prog, mode=0):
    from paper_2503_10516_gb300 import igs
    ref, rej = oracle_graphs(prog)
    g = igs.GpuImpl(prog, mode=mode)
    feed(g, prog)
    assert g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(g.graph(n), ref[n], f"{prog.name} node {n}")
    g.ctx.execute()
    want, known = sequential_run(prog, set(rej))
    gone = {op[1] for op in prog.ops if op[0] == "destroy"}
    for b, buf in enumerate(prog.buffers):
        if b in gone:
            continue
        got = g.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        k = known[b]
        assert np.array_equal(got[k], want[b][k]), f"{prog.name}: buffer {b} differs"
    g.ctx.close()


class _Staged:
    """Batched adapter whose flush only submits the epoch (igs_run lowers)."""

    def __init__(self, prog):
        from paper_2503_10516_gb300 import igs
        self.g = igs.GpuImpl(prog, mode=igs.MODE_BATCHED)
        self.ctx = self.g.ctx

    def __getattr__(self, name):
        return getattr(self.g, name)

    def flush(self):
        self.ctx.submit_epoch()


def _check_run(prog, window=3):
    """The same through igs_run (lowering overlapped with execution)."""
    ref, rej = oracle_graphs(prog)
    s = _Staged(prog)
    feed(s, prog)
    s.ctx.run(window)
    assert s.g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(s.g.graph(n), ref[n], f"{prog.name} node {n} (run)")
    want, known = sequential_run(prog, set(rej))
    gone = {op[1] for op in prog.ops if op[0] == "destroy"}
    for b, buf in enumerate(prog.buffers):
        if b in gone:
            continue
        got = s.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        k = known[b]
        assert np.array_equal(got[k], want[b][k]), f"{prog.name}: buffer {b} differs (run)"
    s.ctx.close()


def _task(dims, rng, chunks, accs):
    return W.Task(dims, rng, chunks, W.K_GENERIC, accs)


def test_no_tasks():
    b = W.Buffer(2, (8, 8, 1), 4, _u32(64, 1), "u32")
    p = W.Program("empty", 2, 2, 4, 0, [("buffer", b), ("flush",)])
    _check(p)
    _check(p, mode=1)
    _check_run(p)


def test_one_element_buffers():
    a = W.Buffer(1, (1, 1, 1), 4, _u32(1, 2), "u32")
    o = W.Buffer(3, (1, 1, 1), 4, None, "u32")
    ops = [("buffer", a), ("buffer", o)]
    for _ in range(5):
        ops.append(("task", _task(3, (1, 1, 1), 4, [W.Accessor(1, W.WRITE, W.one_to_one()),
                                                    W.Accessor(0, W.READ, W.all_mapper())])))
        ops.append(("task", _task(1, (1, 1, 1), 3, [W.Accessor(0, W.READ_WRITE, W.one_to_one())])))
    ops.append(("flush",))
    _check(W.Program("one-element", 2, 2, 2, 1, ops))
    _check_run(W.Program("one-element", 2, 2, 2, 1, ops))


def test_more_chunks_than_rows():
    a = W.Buffer(2, (3, 17, 1), 4, _u32(51, 3), "u32")
    o = W.Buffer(2, (3, 17, 1), 4, None, "u32")
    ops = [("buffer", a), ("buffer", o)]
    for _ in range(4):
        ops.append(("task", _task(2, (3, 17, 1), 128, [W.Accessor(1, W.WRITE, W.one_to_one()),
                                                       W.Accessor(0, W.READ, W.neighborhood(1, 1))])))
        ops.append(("task", _task(2, (3, 17, 1), 64, [W.Accessor(0, W.WRITE, W.one_to_one()),
                                                      W.Accessor(1, W.READ, W.neighborhood(1, 1))])))
    ops.append(("flush",))
    _check(W.Program("chunks>rows", 4, 2, 4, 2, ops))
    _check_run(W.Program("chunks>rows", 4, 2, 4, 2, ops))


def test_thirty_two_nodes():
    _check(W.wave_program(n=64, steps=6, nodes=32, devices=1, chunks=64, lookahead=2))
    _check_run(W.wave_program(n=64, steps=6, nodes=32, devices=1, chunks=64, lookahead=2))


def test_twenty_nine_devices():
    """Memory ids run to 30 (M0, M1 and 29 devices): every bit of the
    up-to-date masks is used."""
    _check(W.wave_program(n=58, steps=5, nodes=1, devices=29, chunks=29, lookahead=0))
    _check(W.wave_program(n=58, steps=5, nodes=2, devices=29, chunks=58, lookahead=3), mode=1)
    _check_run(W.wave_program(n=58, steps=5, nodes=2, devices=29, chunks=58, lookahead=3))


def test_eight_accessors():
    bufs = [W.Buffer(2, (12, 10, 1), 4, _u32(120, 10 + i), "u32") for i in range(7)]
    out = W.Buffer(2, (12, 10, 1), 4, None, "u32")
    ops = [("buffer", b) for b in bufs] + [("buffer", out)]
    mappers = [W.one_to_one(), W.neighborhood(1, 2), W.all_mapper(), W.row_slice(), W.col_slice(),
               W.neighborhood(2, 1), W.one_to_one()]
    for step in range(3):
        accs = [W.Accessor(7, W.WRITE, W.one_to_one())] + [W.Accessor(i, W.READ, mappers[i]) for i in range(7)]
        ops.append(("task", _task(2, (12, 10, 1), 5, accs)))
        ops.append(("task", _task(2, (12, 10, 1), 3, [W.Accessor(step % 7, W.READ_WRITE, W.one_to_one()),
                                                      W.Accessor(7, W.READ, W.neighborhood(1, 1))])))
    ops.append(("flush",))
    _check(W.Program("eight-accessors", 3, 2, 3, 4, ops))
    _check_run(W.Program("eight-accessors", 3, 2, 3, 4, ops))


def test_empty_mapped_boxes():
    """Fixed mappers outside the buffer clamp to nothing: no access, no copy."""
    a = W.Buffer(2, (8, 8, 1), 4, _u32(64, 20), "u32")
    o = W.Buffer(2, (8, 8, 1), 4, None, "u32")
    far = [W.fixed(100, 120), W.fixed(0, 8), W.fixed(0, 1)]
    ops = [("buffer", a), ("buffer", o),
           ("task", _task(2, (8, 8, 1), 4, [W.Accessor(1, W.WRITE, W.one_to_one()), W.Accessor(0, W.READ, far)])),
           ("task", _task(2, (8, 8, 1), 4, [W.Accessor(0, W.READ_WRITE, W.one_to_one()),
                                            W.Accessor(1, W.READ, W.all_mapper())])),
           ("flush",)]
    _check(W.Program("empty-boxes", 2, 2, 4, 0, ops))
    _check_run(W.Program("empty-boxes", 2, 2, 4, 0, ops))


def test_flush_between_phases():
    """Lowering resumes after a flush in the same context (epochs in between)."""
    p = W.wave_program(n=32, steps=9, nodes=2, devices=2, chunks=8, lookahead=4)
    ops = []
    for i, op in enumerate(p.ops):
        ops.append(op)
        if op[0] == "task" and i % 3 == 0:
            ops.append(("flush",))
    p.ops = ops
    _check(p)
    _check(p, mode=1)
    _check_run(p, window=1)
