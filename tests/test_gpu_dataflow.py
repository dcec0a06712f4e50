"""The dataflow executor (one persistent out-of-order launch per execute call:
instructions become ready when their predecessors finish, blocks take tiles
of ready instructions) gives the sequential result byte for byte, in plain
execute calls, in several calls over one program, and in igs_run windows;
and its statistics describe the graph it ran."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs
from tests.replay import sequential_run

pytestmark = pytest.mark.gpu


def _contents(ctx, prog, rej, tag):
    want, known = sequential_run(prog, set(rej))
    gone = {op[1] for op in prog.ops if op[0] == "destroy"}
    for b, buf in enumerate(prog.buffers):
        if b in gone:
            continue
        got = ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        k = known[b]
        assert np.array_equal(got[k], want[b][k]), f"{prog.name}: buffer {b} differs ({tag})"


def _run(prog, mode=0, timing=False):
    from paper_2503_10516_gb300 import igs
    _, rej = oracle_graphs(prog)
    g = igs.GpuImpl(prog, mode=mode)
    g.ctx.set_executor(igs.EXEC_DATAFLOW)
    if timing:
        g.ctx.set_timing(True)
    feed(g, prog)
    g.ctx.execute()
    _contents(g.ctx, prog, rej, "dataflow")
    st = g.ctx.exec_stats()
    g.ctx.close()
    return st


class _Staged:
    def __init__(self, prog):
        from paper_2503_10516_gb300 import igs
        self.g = igs.GpuImpl(prog, mode=igs.MODE_BATCHED)
        self.ctx = self.g.ctx

    def __getattr__(self, name):
        return getattr(self.g, name)

    def flush(self):
        self.ctx.submit_epoch()


def _run_pipelined(prog, window):
    from paper_2503_10516_gb300 import igs
    ref, rej = oracle_graphs(prog)
    s = _Staged(prog)
    s.ctx.set_executor(igs.EXEC_DATAFLOW)
    feed(s, prog)
    s.ctx.run(window)
    assert s.g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(s.g.graph(n), ref[n], f"{prog.name} node {n}")
    _contents(s.ctx, prog, rej, f"dataflow run, window {window}")
    s.ctx.close()


@pytest.mark.parametrize("seed", range(60))
def test_random(seed):
    _run(W.random_program(seed, max_extent=10, max_tasks=12))


PAPER = [
    W.jacobi_program(),
    W.wave_program(n=64, steps=10, nodes=4, devices=4, chunks=64, lookahead=8),
    W.wave_program(n=48, steps=9, nodes=2, devices=2, chunks=8, lookahead=0),
    W.nbody_program(n=512, steps=3, nodes=8, devices=4, chunks=128, lookahead=4),
    W.nbody_program(n=700, steps=2, nodes=2, devices=2, chunks=6, lookahead=0),
    W.nbody_program(n=1300, steps=2, nodes=1, devices=2, chunks=2, lookahead=0),
    W.nbody_example_program(n=64, iterations=4),
    W.growing_program(rows_max=128, cols=32, grow=(1, 16), devices=2, chunks=2),
    W.growing_program(rows_max=128, cols=32, grow=(1, 16), devices=2, chunks=2, lookahead=0xFFFFFFFF),
    W.growing_program(rows_max=200, cols=1, grow=(1, 9), nodes=2, devices=2, chunks=4, lookahead=3),
    W.growing_program(rows_max=96, cols=1024, grow=(8, 40), devices=2, chunks=2, lookahead=0),
]


@pytest.mark.parametrize("prog", PAPER, ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped(prog):
    _run(prog)


def test_large_stencil_tiles():
    """Chunks of several stencil tiles with a ragged last tile (rows of 1000
    columns: 250 groups per row, 4096 groups per tile)."""
    p = W.wave_program(n=1000, steps=4, nodes=2, devices=2, chunks=4, lookahead=2)
    _run(p)


@pytest.mark.parametrize("seed", range(24))
def test_pipelined_random(seed):
    _run_pipelined(W.random_program(70_000 + seed, max_extent=10, max_tasks=12), window=1 + seed % 4)


@pytest.mark.parametrize("window", [1, 16])
@pytest.mark.parametrize("prog", [PAPER[1], PAPER[3], PAPER[9], PAPER[8]],
                         ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_pipelined_paper_shaped(prog, window):
    _run_pipelined(prog, window)


def test_calls_resume_after_flushes():
    """Several execute calls over one program (a flush after every third
    task): sends and receives of one task can fall into different calls."""
    from paper_2503_10516_gb300 import igs
    p = W.nbody_program(n=256, steps=4, nodes=4, devices=2, chunks=16, lookahead=2)
    _, rej = oracle_graphs(p)
    g = igs.GpuImpl(p, mode=igs.MODE_PLAIN)
    g.ctx.set_executor(igs.EXEC_DATAFLOW)
    k = 0
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            g.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init is not None)
        elif op[0] == "task":
            g.submit(op[1])
            k += 1
            if k % 3 == 0:
                g.ctx.execute()
        elif op[0] == "flush":
            g.flush()
    g.ctx.execute()
    _contents(g.ctx, p, rej, "dataflow, several calls")
    assert g.ctx.exec_stats()["launches"] >= 2
    g.ctx.close()


def test_executors_agree_and_stats():
    """Levels and dataflow give the same bytes; the dataflow statistics
    count the graph's nodes and tiles, and with timing on the span and busy
    times are consistent (overlap <= each busy time <= span)."""
    from paper_2503_10516_gb300 import igs
    p = W.wave_program(n=256, steps=8, nodes=2, devices=4, chunks=32, lookahead=4)
    st = _run(p, timing=True)
    assert st["launches"] == 1 and st["nodes"] > 0 and st["tiles"] >= st["nodes"] and st["edges"] > 0
    assert st["span_ms"] > 0
    assert 0 <= st["overlap_ms"] <= min(st["copy_busy_ms"], st["kernel_busy_ms"]) + 1e-9
    assert max(st["copy_busy_ms"], st["kernel_busy_ms"]) <= st["span_ms"] + 1e-9
    g = igs.GpuImpl(p)
    feed(g, p)
    g.ctx.execute()
    levels = [g.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size) for b, buf in enumerate(p.buffers)]
    g.ctx.close()
    h = igs.GpuImpl(p)
    h.ctx.set_executor(igs.EXEC_DATAFLOW)
    feed(h, p)
    h.ctx.execute()
    _, known = sequential_run(p, set())
    for b, buf in enumerate(p.buffers):
        got = h.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        assert np.array_equal(got[known[b]], levels[b][known[b]])
    h.ctx.close()


def test_bad_executor_is_rejected():
    from paper_2503_10516_gb300 import igs
    p = W.jacobi_program()
    g = igs.GpuImpl(p)
    with pytest.raises(igs.IgsError):
        g.ctx.set_executor(7)
    g.ctx.close()


def test_bounded_wait_gives_up_and_device_stays_usable():
    """A graph in which nothing ever becomes ready: every block waits, gives
    up after the limit, and the launch ends with the timeout status; the
    device then runs a normal dataflow execute."""
    import time

    from paper_2503_10516_gb300 import igs
    t0 = time.perf_counter()
    r = igs.selftest_flow_wait(200)
    dt = time.perf_counter() - t0
    assert r == igs.IGS_ERR_TIMEOUT
    assert 0.15 < dt < 10.0
    _run(W.jacobi_program())


def _split_receive_seeds(count=16, start=5000):
    """Seeds of small random programs whose graphs hold split receives (the
    oracle decides), for the receive-arbitration path."""
    out, seed = [], start
    while len(out) < count and seed < start + 4000:
        p = W.random_program(seed, max_extent=10, max_tasks=12)
        ref, _ = oracle_graphs(p)
        if sum(int((g["instrs"][:, 1] == 7).sum()) for g in ref):
            out.append(seed)
        seed += 1
    return out


_SPLIT = _split_receive_seeds()


@pytest.mark.parametrize("seed", _SPLIT)
def test_split_receives_arbitrated(seed):
    """Programs with split receives: each send's data lands through a copy of
    its own and an await receive completes once the sends meeting its region
    have landed; contents equal the sequential run (plain execute and
    pipelined run)."""
    p = W.random_program(seed, max_extent=10, max_tasks=12)
    _run(p)
    _run_pipelined(p, window=1 + seed % 3)
