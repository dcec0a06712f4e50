"""Executing the GPU-lowered graphs on one GPU (virtual memories as HBM
partitions, box-copy kernels, workload kernels) gives the sequential result,
byte for byte."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs
from tests.replay import sequential_run

pytestmark = pytest.mark.gpu


def _destroyed(prog):
    return {op[1] for op in prog.ops if op[0] == "destroy"}


def _run(prog, mode=0):
    from paper_2503_10516_gb300 import igs
    _, rej = oracle_graphs(prog)
    g = igs.GpuImpl(prog, mode=mode)
    feed(g, prog)
    g.ctx.execute()
    want, known = sequential_run(prog, set(rej))
    gone = _destroyed(prog)
    for b, buf in enumerate(prog.buffers):
        if b in gone:
            continue
        got = g.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        k = known[b]
        assert np.array_equal(got[k], want[b][k]), f"{prog.name}: buffer {b} differs"
    g.ctx.close()


@pytest.mark.parametrize("seed", range(60))
def test_random(seed):
    _run(W.random_program(seed, max_extent=10, max_tasks=12))


@pytest.mark.parametrize("prog", [
    W.jacobi_program(),
    W.wave_program(n=64, steps=10, nodes=4, devices=4, chunks=64, lookahead=8),
    W.wave_program(n=48, steps=9, nodes=2, devices=2, chunks=8, lookahead=0),
    W.nbody_program(n=512, steps=3, nodes=8, devices=4, chunks=128, lookahead=4),
    W.nbody_example_program(n=64, iterations=4),
    W.growing_program(rows_max=128, cols=32, grow=(1, 16), devices=2, chunks=2),
    W.growing_program(rows_max=128, cols=32, grow=(1, 16), devices=2, chunks=2, lookahead=0xFFFFFFFF),
    W.growing_program(rows_max=200, cols=1, grow=(1, 9), nodes=2, devices=2, chunks=4, lookahead=3),
], ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped(prog):
    _run(prog)


def test_batched_mode_contents():
    _run(W.wave_program(n=64, steps=10, nodes=4, devices=4, chunks=64, lookahead=8), mode=1)


def test_read_destroyed_buffer_is_an_error():
    from paper_2503_10516_gb300 import igs
    p = W.random_program(2, max_extent=10, max_tasks=12)
    g = igs.GpuImpl(p)
    feed(g, p)
    g.ctx.execute()
    with pytest.raises(igs.IgsError):
        g.ctx.read_buffer(1, (0, 0, 0), p.buffers[1].extent, 4)
    g.ctx.close()


class _Staged:
    """Batched-mode adapter whose flush only submits the epoch: everything is
    lowered later by igs_run."""

    def __init__(self, prog):
        from paper_2503_10516_gb300 import igs
        self.g = igs.GpuImpl(prog, mode=igs.MODE_BATCHED)
        self.ctx = self.g.ctx

    def __getattr__(self, name):
        return getattr(self.g, name)

    def flush(self):
        self.ctx.submit_epoch()


def _run_pipelined(prog, window):
    """igs_run: lowering of window k+1 overlaps execution of window k; the
    graphs equal the oracle's and the contents the sequential run's."""
    ref, rej = oracle_graphs(prog)
    s = _Staged(prog)
    feed(s, prog)
    s.ctx.run(window)
    assert s.g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(s.g.graph(n), ref[n], f"{prog.name} node {n}")
    want, known = sequential_run(prog, set(rej))
    gone = _destroyed(prog)
    for b, buf in enumerate(prog.buffers):
        if b in gone:
            continue
        got = s.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        k = known[b]
        assert np.array_equal(got[k], want[b][k]), f"{prog.name}: buffer {b} differs"
    s.ctx.close()


@pytest.mark.parametrize("seed", range(40))
def test_pipelined_random(seed):
    _run_pipelined(W.random_program(70_000 + seed, max_extent=10, max_tasks=12), window=1 + seed % 4)


@pytest.mark.parametrize("window", [1, 3, 16])
@pytest.mark.parametrize("prog", [
    W.wave_program(n=64, steps=10, nodes=4, devices=4, chunks=64, lookahead=8),
    W.nbody_program(n=512, steps=3, nodes=8, devices=4, chunks=128, lookahead=4),
    W.growing_program(rows_max=200, cols=1, grow=(1, 9), nodes=2, devices=2, chunks=4, lookahead=3),
    W.growing_program(rows_max=128, cols=32, grow=(1, 16), devices=2, chunks=2, lookahead=0xFFFFFFFF),
], ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_pipelined_paper_shaped(prog, window):
    _run_pipelined(prog, window)


@pytest.mark.parametrize("prog", [
    W.growing_program(rows_max=128, cols=32, grow=(1, 16), devices=2, chunks=2, lookahead=W.LOOKAHEAD_HORIZONS),
    W.wave_program(n=64, steps=20, nodes=4, devices=4, chunks=64, lookahead=W.LOOKAHEAD_HORIZONS),
], ids=lambda p: p.name)
def test_pipelined_horizon_lookahead(prog):
    _run_pipelined(prog, window=4)
    _run(prog)
