"""Horizons by the task graph's critical path (IGS_FLAG_HORIZON_CP, Sec.
3.5): the library places them where the oracle does, so the CUDA lowering
emits the oracle's graphs (plain, batched, pipelined) and execution gives
the sequential contents."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs
from tests.replay import sequential_run

pytestmark = pytest.mark.gpu


def _check(prog, mode):
    from paper_2503_10516_gb300 import igs
    prog.horizon_cp = True
    ref, rej = oracle_graphs(prog)
    g = igs.GpuImpl(prog, mode=mode)
    feed(g, prog)
    assert g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(g.graph(n), ref[n], f"{prog.name} node {n} mode {mode}")
    g.ctx.execute()
    want, known = sequential_run(prog, set(rej))
    gone = {op[1] for op in prog.ops if op[0] == "destroy"}
    for b, buf in enumerate(prog.buffers):
        if b in gone:
            continue
        got = g.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        assert np.array_equal(got[known[b]], want[b][known[b]]), f"{prog.name}: buffer {b}"
    g.ctx.close()


@pytest.mark.parametrize("seed", range(32))
def test_random_programs(seed):
    _check(W.random_program(500_000 + seed, max_extent=10, max_tasks=12), mode=seed % 2)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prog", [
    W.wave_program(n=64, steps=10, nodes=4, devices=4, chunks=64, lookahead=8, horizon_step=3),
    W.nbody_program(n=256, steps=4, nodes=4, devices=2, chunks=16, lookahead=4, horizon_step=2),
], ids=lambda p: p.name)
def test_paper_shaped(prog, mode):
    _check(prog, mode)
