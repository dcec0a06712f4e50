"""Many uneven programs lowered in ONE launch (igs_lower_batch) give exactly
the oracle's graphs, and exactly the graphs of one-task-per-launch lowering."""
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, oracle_graphs

pytestmark = pytest.mark.gpu


def _counts(prog):
    ref, _ = oracle_graphs(prog)
    return {k: max(len(g[k]) for g in ref) for k in ("instrs", "edges", "boxes")}


def _stage(prog, mode, stream=None, caps_from=None):
    from paper_2503_10516_gb300 import igs
    big = caps_from or prog
    c = igs.Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=mode, stream=stream,
                    **igs.small_caps(big, _counts(big)))
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


@pytest.mark.parametrize("shape", [(1, 1), (3, 0), (7, 1), (152, 1), (4096, 0), (2, 1, 4, 4), (5, 1, 8, 100),
                                   (3, 0, 2, 1), (1, 1, 8, 0)])
def test_work_queue_shapes_match_oracle(shape):
    """The device work queue (persistent blocks taking units in submission
    or longest-first order) gives the oracle's graphs for every shape: fewer
    blocks than units, one block, more blocks than units, multi-warp blocks
    whose helpers serve some, all or none of the multi-device programs."""
    from paper_2503_10516_gb300 import igs
    progs = W.batch_programs(count=16, scale=0.01, seed=31 + shape[0])
    ctxs = [_stage(p, igs.MODE_BATCHED) for p in progs]
    igs.lower_batch(ctxs, shape)
    for p, c in zip(progs, ctxs):
        ref, rej = oracle_graphs(p)
        assert c.rejected() == rej
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n} shape {shape}")
        c.close()


def test_work_queue_twice_in_one_context():
    """A second batched launch over the same contexts resumes where the first
    stopped (the queue head starts at zero again)."""
    from paper_2503_10516_gb300 import igs
    progs = W.batch_programs(count=6, scale=0.01, seed=91)
    longer = [W.Program(p.name, p.nodes, p.devices, p.horizon_step, p.lookahead,
                        list(p.ops) + [("task", t) for t in p.tasks[:3]] + [("flush",)]) for p in progs]
    ctxs = [_stage(p, igs.MODE_BATCHED, caps_from=q) for p, q in zip(progs, longer)]
    igs.lower_batch(ctxs, (2, igs.ORDER_LONGEST_FIRST))
    for p, c in zip(progs, ctxs):
        for t in p.tasks[:3]:
            c.submit(t)
        c.submit_epoch()
    igs.lower_batch(ctxs, (5, igs.ORDER_SUBMISSION, 4, 3))
    for p, q, c in zip(progs, longer, ctxs):
        ref, rej = oracle_graphs(q)
        assert c.rejected() == rej
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n} (second launch)")
        c.close()


def test_tuner_picks_a_timed_candidate():
    import time

    import torch
    from paper_2503_10516_gb300 import igs
    progs = W.batch_programs(count=12, scale=0.01, seed=5)
    units = sum(p.nodes for p in progs)
    cands = igs.batch_shape_candidates(units, torch.cuda.get_device_properties(0).multi_processor_count)
    assert cands[0] is None and all(1 <= c[0] <= units and 1 <= c[2] <= 8 for c in cands[1:])

    def timer():
        torch.cuda.synchronize()
        return time.perf_counter()

    best, times = igs.tune_lower_batch(lambda: [_stage(p, igs.MODE_BATCHED) for p in progs], cands, timer)
    assert [s for s, _ in times] == list(cands) and best in cands
    assert all(t > 0 for _, t in times)


def test_bad_shape_is_rejected():
    from paper_2503_10516_gb300 import igs
    p = W.batch_programs(count=1, scale=0.01, seed=3)[0]
    c = _stage(p, igs.MODE_BATCHED)
    for shape in ((4, 2), (4, 1, 9, 0)):
        with pytest.raises(igs.IgsError):
            igs.lower_batch([c], shape)
    igs.lower_batch([c], (4, 1, 2, 1))
    ref, _ = oracle_graphs(p)
    for n in range(p.nodes):
        assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n}")
    c.close()


def test_batch_full_task_counts_seeded_subset():
    """The benchmark's batch at full task counts (10-2000 tasks per program):
    four programs picked by a seeded permutation among those the oracle
    lowers in seconds (nodes x tasks x chunks < 2e6) are lowered in one
    launch; every node's graph equals the oracle's."""
    import numpy as np
    from paper_2503_10516_gb300 import igs
    full = W.batch_programs(count=512, scale=1.0)
    perm = np.random.default_rng(0x5EED + 31).permutation(len(full))
    cost = [p.nodes * len(p.tasks) * max(t.chunks for t in p.tasks) for p in full]
    picked = [int(i) for i in perm if cost[i] < 2e6][:4]
    progs = [full[i] for i in picked]
    assert min(len(p.tasks) for p in progs) >= 100
    refs = [oracle_graphs(p) for p in progs]
    ctxs = []
    for p, (ref, _) in zip(progs, refs):
        counts = {k: max(len(g[k]) for g in ref) for k in ("instrs", "edges", "boxes")}
        c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED,
                        **igs.small_caps(p, counts))
        for op in p.ops:
            if op[0] == "buffer":
                b = op[1]
                c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
            elif op[0] == "task":
                c.submit(op[1])
            elif op[0] == "flush":
                c.submit_epoch()
        ctxs.append(c)
    igs.lower_batch(ctxs, (152, igs.ORDER_LONGEST_FIRST, 4, 2))
    for p, c, (ref, rej) in zip(progs, ctxs, refs):
        assert c.rejected() == rej
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n} (full task counts)")
        c.close()
