"""Many uneven programs lowered in ONE launch (igs_lower_batch) give exactly
the oracle's graphs, and exactly the graphs of one-task-per-launch lowering."""
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, oracle_graphs

pytestmark = pytest.mark.gpu


def _counts(prog):
    ref, _ = oracle_graphs(prog)
    return {k: max(len(g[k]) for g in ref) for k in ("instrs", "edges", "boxes")}


def _stage(prog, mode, stream=None):
    from paper_2503_10516_gb300 import igs
    c = igs.Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=mode, stream=stream,
                    **igs.small_caps(prog, _counts(prog)))
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
        elif op[0] == "task":
            c.submit(op[1])
        elif op[0] == "flush":
            c.submit_epoch()
    return c


def test_batch_of_uneven_programs_one_launch():
    from paper_2503_10516_gb300 import igs
    progs = W.batch_programs(count=24, scale=0.01)
    ctxs = [_stage(p, igs.MODE_BATCHED) for p in progs]
    igs.lower_batch(ctxs)
    for p, c in zip(progs, ctxs):
        ref, rej = oracle_graphs(p)
        assert c.rejected() == rej
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n}")
        c.close()


def test_batch_equals_plain():
    from paper_2503_10516_gb300 import igs
    progs = W.batch_programs(count=8, scale=0.01, seed=777)
    ctxs = [_stage(p, igs.MODE_BATCHED) for p in progs]
    igs.lower_batch(ctxs)
    for p, c in zip(progs, ctxs):
        plain = _stage(p, igs.MODE_PLAIN)
        plain.sync()
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), plain.graph(n), f"{p.name} node {n}")
        plain.close()
        c.close()


def test_fragmented_maps_grow_in_heap():
    """Transposed column-strip reads on many nodes fragment the region maps
    into hundreds of boxes; the tables grow inside the node heap and the
    graphs still equal the oracle's, in plain and batched mode."""
    from paper_2503_10516_gb300 import igs
    progs = W.batch_programs(count=24, scale=0.01)
    frag = max(progs, key=lambda p: p.nodes * len(p.tasks))
    for mode in (igs.MODE_PLAIN, igs.MODE_BATCHED):
        c = _stage(frag, mode)
        if mode == igs.MODE_BATCHED:
            igs.lower_batch([c])
        else:
            c.sync()
        ref, rej = oracle_graphs(frag)
        assert c.rejected() == rej
        for n in range(frag.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{frag.name} node {n} mode {mode}")
        c.close()


def test_heap_exhaustion_reports_capacity():
    """A node heap too small for the program's tables ends the lowering with
    IGS_ERR_CAPACITY (no partial graph is trusted)."""
    from paper_2503_10516_gb300 import igs
    p = W.jacobi_program(n=32, steps=4)
    caps = igs.small_caps(p, _counts(p))
    caps["map_heap"] = 64
    c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED, **caps)
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
        elif op[0] == "task":
            c.submit(op[1])
    with pytest.raises(igs.IgsError) as ei:
        c.flush()
    assert ei.value.code == igs.IGS_ERR_CAPACITY
    c.close()


def test_timed_batch_workload_parity():
    """The 512 uneven programs the batched-lowering measurement times (task
    counts scaled to 1 %), all in one launch, in the configuration the
    measurement uses (capacities estimated from the program shapes)."""
    from paper_2503_10516_gb300 import igs
    progs = W.batch_programs(count=512, scale=0.01, seed=0x5EED + 3)
    ctxs = []
    for p in progs:
        c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED, **igs.small_caps(p))
        for op in p.ops:
            if op[0] == "buffer":
                b = op[1]
                c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
            elif op[0] == "task":
                c.submit(op[1])
            elif op[0] == "flush":
                c.submit_epoch()
        ctxs.append(c)
    igs.lower_batch(ctxs)
    for p, c in zip(progs, ctxs):
        ref, rej = oracle_graphs(p)
        assert c.rejected() == rej
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n}")
        c.close()
