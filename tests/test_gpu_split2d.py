"""Splits along dims 0 and 1 (Sec. 3.1, hierarchical): the CUDA lowering
emits the oracle's graphs in one-task-per-launch, batched and pipelined
modes, and executing them (both executors, stencil fast paths on 2D chunk
boxes) gives the sequential contents."""
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


def _check(prog, mode, executor=0):
    from paper_2503_10516_gb300 import igs
    ref, rej = oracle_graphs(prog)
    g = igs.GpuImpl(prog, mode=mode)
    g.ctx.set_executor(executor)
    feed(g, prog)
    assert g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(g.graph(n), ref[n], f"{prog.name} node {n} mode {mode}")
    g.ctx.execute()
    _contents(g.ctx, prog, rej, f"mode {mode} executor {executor}")
    g.ctx.close()


@pytest.mark.parametrize("seed", range(48))
def test_random_programs(seed):
    p = W.random_program(400_000 + seed, max_extent=10, max_tasks=10, split2d=True, max_devices=3)
    _check(p, mode=seed % 2, executor=(seed // 2) % 2)


PAPER = [
    W.wave_program(n=64, steps=8, nodes=2, devices=4, chunks=4 | (4 << 16), lookahead=4),
    W.wave_program(n=48, steps=6, nodes=3, devices=2, chunks=6 | (3 << 16), lookahead=0),
    W.jacobi_program(n=64, steps=6, nodes=2, devices=2, chunks=2 | (2 << 16)),
]


@pytest.mark.parametrize("executor", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prog", PAPER, ids=lambda p: p.name)
def test_paper_shaped(prog, mode, executor):
    _check(prog, mode, executor)


class _Staged:
    def __init__(self, prog):
        from paper_2503_10516_gb300 import igs
        self.g = igs.GpuImpl(prog, mode=igs.MODE_BATCHED)
        self.ctx = self.g.ctx

    def __getattr__(self, name):
        return getattr(self.g, name)

    def flush(self):
        self.ctx.submit_epoch()


def test_pipelined():
    p = W.wave_program(n=64, steps=10, nodes=4, devices=2, chunks=8 | (2 << 16), lookahead=8)
    ref, rej = oracle_graphs(p)
    s = _Staged(p)
    feed(s, p)
    s.ctx.run(4)
    for n in range(p.nodes):
        assert_same_graph(s.g.graph(n), ref[n], f"{p.name} node {n} (run)")
    _contents(s.ctx, p, rej, "run")
    s.ctx.close()


def test_bad_2d_splits_are_rejected():
    from paper_2503_10516_gb300 import igs
    c = igs.Context(2, 2)
    c.create_buffer(1, (16,), 4, None)
    c.create_buffer(2, (8, 8), 4, None)
    for dims, rng, chunks, buf in ((1, (16, 1, 1), 2 | (2 << 16), 0), (2, (8, 8, 1), 0 | (2 << 16), 1)):
        t = W.Task(dims, rng, chunks, W.K_GENERIC, [W.Accessor(buf, W.WRITE, W.one_to_one())])
        with pytest.raises(igs.IgsError):
            c.submit(t)
    c.close()
