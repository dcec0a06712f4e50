"""The pipelined lowering launch (a front warp running push / await push
ahead of warp 0) under failures: a capacity that runs out on warp 0's side
while the front warp is ahead, and one that runs out on the front warp's side
first, both end the launch with IGS_ERR_CAPACITY (no hang, no partial graph
trusted), and the device then lowers the next program exactly."""
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, oracle_graphs

pytestmark = pytest.mark.gpu


def _stage(prog, **caps):
    from paper_2503_10516_gb300 import igs
    base = igs.small_caps(prog)
    base.update(caps)
    c = igs.Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=igs.MODE_BATCHED, **base)
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
        elif op[0] == "task":
            c.submit(op[1])
    return c


def _healthy_after():
    p = W.wave_program(n=32, steps=12, nodes=2, devices=2, chunks=8, lookahead=2)
    c = _stage(p)
    c.flush()
    ref, _ = oracle_graphs(p)
    for n in range(p.nodes):
        assert_same_graph(c.graph(n), ref[n], f"after a failed launch, node {n}")
    c.close()


@pytest.mark.parametrize("what", ["back_outputs", "front_scratch"])
def test_pipelined_launch_failure_reports_capacity(what):
    from paper_2503_10516_gb300 import igs
    p = W.wave_program(n=32, steps=24, nodes=2, devices=2, chunks=8, lookahead=2)
    if what == "back_outputs":
        # warp 0 runs out of instruction records a few tasks in, the front warp ahead of it
        c = _stage(p, max_instructions=40)
    else:
        # scratch tables too small for a task's 48 mapped boxes (16 chunks x 3 accessors): the front warp,
        # ahead, fails on the first task before warp 0 reaches it
        c = _stage(W.wave_program(n=32, steps=24, nodes=2, devices=2, chunks=16, lookahead=2), scratch_capacity=32)
    with pytest.raises(igs.IgsError) as ei:
        c.flush()
    assert ei.value.code == igs.IGS_ERR_CAPACITY
    c.close()
    _healthy_after()
