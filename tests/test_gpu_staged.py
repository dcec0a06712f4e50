"""Device-to-device copies staged in host memory (IGS_FLAG_STAGE_D2D, Sec.
3.3): the CUDA lowering emits the oracle's graphs (a host allocation, a copy
in, a copy out and a free per staged copy) in one-task-per-launch, batched
and pipelined modes, and executing them gives the sequential contents."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs
from tests.replay import sequential_run

pytestmark = pytest.mark.gpu


def _staged(p):
    p.stage_d2d = True
    return p


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


class _Staged:
    def __init__(self, prog):
        from paper_2503_10516_gb300 import igs
        self.g = igs.GpuImpl(prog, mode=igs.MODE_BATCHED)
        self.ctx = self.g.ctx

    def __getattr__(self, name):
        return getattr(self.g, name)

    def flush(self):
        self.ctx.submit_epoch()


@pytest.mark.parametrize("seed", range(40))
def test_random_programs(seed):
    p = _staged(W.random_program(300_000 + seed, max_extent=10, max_tasks=12))
    _check(p, mode=seed % 2, executor=(seed // 2) % 2)


PAPER = [
    W.wave_program(n=64, steps=10, nodes=4, devices=4, chunks=64, lookahead=8),
    W.wave_program(n=48, steps=9, nodes=1, devices=4, chunks=8, lookahead=0),
    W.nbody_program(n=512, steps=3, nodes=2, devices=4, chunks=32, lookahead=4),
    W.growing_program(rows_max=128, cols=32, grow=(1, 16), devices=3, chunks=3, lookahead=2),
]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prog", PAPER, ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped(prog, mode):
    _check(_staged(prog), mode)


@pytest.mark.parametrize("window", [1, 8])
def test_pipelined(window):
    p = _staged(W.wave_program(n=64, steps=10, nodes=2, devices=4, chunks=32, lookahead=8))
    ref, rej = oracle_graphs(p)
    s = _Staged(p)
    feed(s, p)
    s.ctx.run(window)
    for n in range(p.nodes):
        assert_same_graph(s.g.graph(n), ref[n], f"{p.name} node {n} (run)")
    _contents(s.ctx, p, rej, "run")
    s.ctx.close()


def test_unknown_flag_is_rejected():
    from paper_2503_10516_gb300 import igs
    with pytest.raises(igs.IgsError):
        igs.Context(1, 2, flags=4)
