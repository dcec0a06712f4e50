"""Per-item lowering times (igs_set_item_times / igs_item_times): every
submitted item gets the device time its last node finished it, in submission
order, with its kind; the graphs are the oracle's with the timing on, in one
pipelined launch and one task per launch."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, oracle_graphs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1])
def test_item_times_in_order(mode):
    from paper_2503_10516_gb300 import igs
    p = W.wave_program(n=64, steps=24, nodes=2, devices=2, chunks=8, lookahead=2)
    c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=mode, **igs.small_caps(p))
    c.set_item_times(True)
    kinds = []
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
            kinds.append(0)
        elif op[0] == "task":
            c.submit(op[1])
            kinds.append(1)
            if sum(1 for k in kinds if k == 1) % p.horizon_step == 0:
                kinds.append(2)
        elif op[0] == "flush":
            c.flush()
            kinds.append(3)
    k, t = c.item_times()
    assert list(k) == kinds
    assert np.all(t > 0) and np.all(np.diff(t.astype(np.int64)) >= 0)
    ref, _ = oracle_graphs(p)
    for n in range(p.nodes):
        assert_same_graph(c.graph(n), ref[n], f"item times, mode {mode}, node {n}")
    c.close()
