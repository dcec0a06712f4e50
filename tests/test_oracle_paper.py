"""Pins of the oracle to what the paper states about concrete programs."""
import os

import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import OracleImpl, counts_by_type, feed, oracle_graphs
from tests.replay import (ALLOC, AWAIT_RECEIVE, COPY, FREE, HORIZON, K_FRONT, KERNEL, RECEIVE, SEND,
                          SPLIT_RECEIVE, _ancestors, task_seqs)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("="))
            out[k] = v
    return out


def _mem_of_alloc(g):
    mem = {}
    for r in g["instrs"]:
        if r[1] == ALLOC:
            mem[int(r[3])] = int(r[4])
    return mem


def _iteration_counts(g, seqs):
    mem = _mem_of_alloc(g)
    c = {"kernel": 0, "send": 0, "receive": 0, "split_receive": 0, "horizon": 0, "alloc": 0,
         "copy.d2h": 0, "copy.h2d": 0, "copy.d2d": 0}
    for r in g["instrs"]:
        if int(r[2]) not in seqs:
            continue
        t = r[1]
        if t == KERNEL:
            c["kernel"] += 1
        elif t == SEND:
            c["send"] += 1
        elif t == RECEIVE:
            c["receive"] += 1
        elif t == SPLIT_RECEIVE:
            c["split_receive"] += 1
        elif t == HORIZON:
            c["horizon"] += 1
        elif t == ALLOC:
            c["alloc"] += 1
        elif t == COPY:
            src, dst = mem.get(int(r[3]), 0), mem[int(r[4])]
            if src >= 2 and dst == 1:
                c["copy.d2h"] += 1
            elif src == 1 and dst >= 2:
                c["copy.h2d"] += 1
            elif src >= 2 and dst >= 2:
                c["copy.d2d"] += 1
    return c


def test_nbody_worked_example_node0():
    """Sec. 3.6: the instruction graph of node N0 for Listing 1 on 2 nodes x 2 devices."""
    gold = _golden("nbody_2x2_node0.txt")
    n = 64
    p = W.nbody_example_program(n=n, iterations=5)
    gs, rej = oracle_graphs(p)
    g = gs[0]
    assert not rej
    # first iteration allocations: P whole on M2 and M3, V quarters
    allocs = [(int(r[5]), int(r[4]), tuple(int(v) for v in g["boxes"][r[7]])) for r in g["instrs"] if r[1] == ALLOC]
    whole = (0, 0, 0, n, 1, 1)
    assert (0, 2, whole) in allocs and (0, 3, whole) in allocs
    assert gold["first.alloc.P.M2"] == "whole" and gold["first.alloc.P.M3"] == "whole"
    assert (1, 2, (0, 0, 0, n // 4, 1, 1)) in allocs
    assert (1, 3, (n // 4, 0, 0, n // 2, 1, 1)) in allocs
    # every later iteration has the steady topology
    seqs = task_seqs(p)
    hseq = lambda k: seqs[2 * k + 1] + 1  # horizon after each iteration (horizon step 2)
    for k in range(2, 5):
        it = {seqs[2 * k], seqs[2 * k + 1], hseq(k)}
        c = _iteration_counts(g, it)
        for key, v in gold.items():
            if key.startswith("steady."):
                assert c[key[len("steady."):]] == int(v), (k, key, c)
        assert c["alloc"] == 0
    # sends and the receive of one iteration are mutually concurrent (Fig. 5 caption)
    anc, _ = _ancestors(g["instrs"], g["edges"])
    for k in range(1, 5):
        ids = [i for i, r in enumerate(g["instrs"]) if int(r[2]) == seqs[2 * k] and r[1] in (SEND, RECEIVE)]
        assert len(ids) == 3
        for a in ids:
            for b in ids:
                if a < b:
                    assert not (anc[b] >> a) & 1, "send/receive ordered"
    # a horizon depends exactly on the execution front (instructions without successors)
    succ = set(int(e[0]) for e in g["edges"])
    for i, r in enumerate(g["instrs"]):
        if r[1] == HORIZON:
            preds = [int(e[0]) for e in g["edges"] if int(e[1]) == i]
            assert all(int(e[2]) == K_FRONT for e in g["edges"] if int(e[1]) == i)
            for q in preds:
                later = [int(e[1]) for e in g["edges"] if int(e[0]) == q and int(e[1]) < i]
                assert not later, "horizon predecessor already had a successor"


@pytest.mark.parametrize("lookahead,resizes", [(0, 1), (1, 0), (4, 0)])
def test_listing2_resize(lookahead, resizes):
    """Listing 2: one_to_one write, then neighborhood read -> one resize per
    device without lookahead (Sec. 4.3), none with lookahead."""
    p = W.listing2_program(16, lookahead, nodes=1, devices=2, chunks=2)
    g = oracle_graphs(p)[0][0]
    frees = [r for r in g["instrs"] if r[1] == FREE]
    resize_copies = [r for r in g["instrs"] if r[1] == COPY and r[6] == 1]
    assert len(frees) == 2 * resizes
    assert len(resize_copies) == 2 * resizes


def test_rsim_growing_resizes_every_step_without_lookahead():
    """Sec. 5 (RSim): a buffer growing by rows resizes on every time step."""
    p = W.growing_program(rows_max=96, cols=4, grow=(1, 6), devices=2, chunks=2, lookahead=0)
    g = oracle_graphs(p)[0][0]
    seqs = task_seqs(p)
    free_seqs = {int(r[2]) for r in g["instrs"] if r[1] == FREE}
    assert all(s in free_seqs for s in seqs[1:]), "a step without a resize"


def test_rsim_growing_no_resize_with_unbounded_lookahead():
    """Sec. 4.3: with the queue never flushed before the end, the first
    instructions already hold allocations covering the whole program."""
    p = W.growing_program(rows_max=96, cols=4, grow=(1, 6), devices=2, chunks=2, lookahead=0xFFFFFFFF)
    g = oracle_graphs(p)[0][0]
    assert not any(r[1] == FREE for r in g["instrs"])
    assert not any(r[1] == COPY and r[6] == 1 for r in g["instrs"])


def test_overlapping_write_rejected():
    """Sec. 4.4: an all-mapper write split over two devices is an error."""
    rng = np.random.default_rng(3)
    buf = W.Buffer(1, (16, 1, 1), 4, rng.integers(0, 2**32, 16, dtype=np.uint64).astype(np.uint32), "u32")
    ops = [("buffer", buf),
           ("task", W.Task(1, (16, 1, 1), 2, W.K_GENERIC, [W.Accessor(0, W.WRITE, W.all_mapper())])),
           ("task", W.Task(1, (16, 1, 1), 2, W.K_GENERIC, [W.Accessor(0, W.READ_WRITE, W.one_to_one())])),
           ("flush",)]
    p = W.Program("overlap", 1, 2, 4, 0, ops)
    impl = OracleImpl(p)
    res = feed(impl, p)
    assert res == [-2, 0]
    bad = task_seqs(p)[0]
    assert impl.rejected() == [bad]
    g = impl.graph(0)
    assert not any(int(r[2]) == bad for r in g["instrs"])
    # the accepted task still reads the host data: copies from the user allocation on M0
    alloced = {int(r[3]) for r in g["instrs"] if r[1] == ALLOC}
    srcs = {int(r[3]) for r in g["instrs"] if r[1] == COPY}
    assert srcs and all(s not in alloced for s in srcs)


def test_uninitialized_read_warning():
    """Sec. 4.4: reading a never-written region of a buffer is reported."""
    ops = [("buffer", W.Buffer(2, (8, 8, 1), 4, None, "u32")),
           ("buffer", W.Buffer(2, (8, 8, 1), 4, None, "u32")),
           ("task", W.Task(2, (8, 8, 1), 2, W.K_GENERIC,
                           [W.Accessor(1, W.WRITE, W.one_to_one()), W.Accessor(0, W.READ, W.one_to_one())])),
           ("flush",)]
    p = W.Program("uninit", 1, 2, 4, 0, ops)
    g = oracle_graphs(p)[0][0]
    seq = task_seqs(p)[0]
    assert sorted(map(tuple, g["diags"].tolist())) == [(seq, 0, 1), (seq, 1, 1)]
    assert not any(r[1] == COPY for r in g["instrs"])


def test_single_device_one_to_one_needs_no_copies_after_first_use():
    """With one node and one device, one_to_one-only programs copy host data once."""
    rng = np.random.default_rng(5)
    ops = [("buffer", W.Buffer(2, (8, 8, 1), 4, rng.integers(0, 2**32, 64, dtype=np.uint64).astype(np.uint32), "u32"))]
    for _ in range(6):
        ops.append(("task", W.Task(2, (8, 8, 1), 3, W.K_GENERIC, [W.Accessor(0, W.READ_WRITE, W.one_to_one())])))
    ops.append(("flush",))
    p = W.Program("o2o", 1, 1, 2, 0, ops)
    g = oracle_graphs(p)[0][0]
    seqs = task_seqs(p)
    copy_seqs = [int(r[2]) for r in g["instrs"] if r[1] == COPY]
    assert copy_seqs and set(copy_seqs) == {seqs[0]}


def test_split_receive_when_consumers_differ():
    """Sec. 3.4: consumers reading different parts of an awaited region get a
    split receive and one await receive each."""
    n = 16
    rng = np.random.default_rng(9)
    init = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    ops = [("buffer", W.Buffer(1, (n, 1, 1), 4, init, "u32")), ("buffer", W.Buffer(1, (n, 1, 1), 4, None, "u32")),
           # node 1 (chunks 2,3) overwrites the upper half
           ("task", W.Task(1, (n, 1, 1), 4, W.K_GENERIC, [W.Accessor(0, W.READ_WRITE, W.one_to_one())])),
           # node 0's two devices read the upper half shifted differently
           ("task", W.Task(1, (n, 1, 1), 4, W.K_GENERIC,
                           [W.Accessor(1, W.WRITE, W.one_to_one()),
                            W.Accessor(0, W.READ, [W.affine(0, n // 2, 0), W.all_dim(), W.all_dim()])])),
           ("flush",)]
    p = W.Program("split", 2, 2, 8, 0, ops)
    g = oracle_graphs(p)[0][0]
    kinds = [int(r[1]) for r in g["instrs"]]
    assert kinds.count(SPLIT_RECEIVE) == 1
    assert kinds.count(AWAIT_RECEIVE) == 2


def _emitted_after_each_task(p):
    """Node 0's instruction count after every submitted task (lowering as it
    happens, not only at the end)."""
    import oracle
    o = oracle.Oracle(p.nodes, p.devices, p.horizon_step, p.lookahead)
    seen = []
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            o.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init is not None)
        elif op[0] == "task":
            o.submit(op[1].flat())
            seen.append(len(o.graph(0)["instrs"]))
        elif op[0] == "flush":
            o.flush()
    g = o.graph(0)
    o.close()
    return seen, g


def test_horizon_heuristic_never_flushes_growing_rows():
    """Sec. 4.3: with requirements growing every step the horizon-count
    heuristic never flushes the queue before the end, so no allocation is
    ever resized (the RSim case, Sec. 5)."""
    p = W.growing_program(rows_max=96, cols=4, grow=(1, 6), devices=2, chunks=2, lookahead=W.LOOKAHEAD_HORIZONS)
    seen, g = _emitted_after_each_task(p)
    assert all(x == 1 for x in seen), "instructions were generated before the end"
    assert not any(r[1] == FREE for r in g["instrs"])
    assert not any(r[1] == COPY and r[6] == 1 for r in g["instrs"])


def test_horizon_heuristic_flushes_stable_patterns():
    """Sec. 4.3: once the access pattern is steady, two horizons after the
    last allocating task compile the queue (concurrency is kept), and the
    allocations made then cover what the queue saw: no resize."""
    p = W.wave_program(n=32, steps=24, nodes=2, devices=2, chunks=8, lookahead=W.LOOKAHEAD_HORIZONS, horizon_step=4)
    seen, g = _emitted_after_each_task(p)
    first = next(i for i, x in enumerate(seen) if x > 1)
    # the rotating buffers' halos make tasks 1-3 allocating; horizons follow
    # tasks 4 and 8, so the queue is compiled with the horizon after task 8
    # (index 7): one horizon too few would compile after task 4, one too many
    # after task 12
    assert first == 7
    assert all(x > 1 for x in seen[first:])
    assert not any(r[1] == FREE for r in g["instrs"])
    _, ref = _emitted_after_each_task(W.wave_program(n=32, steps=24, nodes=2, devices=2, chunks=8,
                                                     lookahead=W.LOOKAHEAD_INFINITE, horizon_step=4))
    assert sum(1 for r in g["instrs"] if r[1] == ALLOC) == sum(1 for r in ref["instrs"] if r[1] == ALLOC)


def _copy_memories(g):
    """(source memory, destination memory) of every copy, from the allocations."""
    mem = {}
    for r in g["instrs"]:
        if int(r[1]) == 2:  # ALLOC
            mem[int(r[3])] = int(r[4])
    out = []
    for r in g["instrs"]:
        if int(r[1]) == 4:  # COPY
            out.append((mem.get(int(r[3]), 0), mem.get(int(r[4]), 0)))
    return out


@pytest.mark.parametrize("prog", [
    W.wave_program(n=32, steps=6, nodes=1, devices=4, chunks=16, lookahead=2),
    W.wave_program(n=16, steps=5, nodes=2, devices=2, chunks=8, lookahead=0),
    W.nbody_program(n=64, steps=2, nodes=2, devices=2, chunks=8, lookahead=4),
], ids=lambda p: p.name)
def test_staged_d2d_replaces_every_device_to_device_copy(prog):
    """Sec. 3.3: with device-to-device copies staged in host memory, no copy
    goes from one device memory to another (resize copies stay within one
    memory); each one that did becomes a host
    allocation, a copy into it, a copy out of it and its free (3 more
    instructions each), and nothing else changes."""
    plain, _ = oracle_graphs(prog)
    prog.stage_d2d = True
    staged, _ = oracle_graphs(prog)
    for g0, g1 in zip(plain, staged):
        d2d = sum(1 for s, d in _copy_memories(g0) if s >= 2 and d >= 2 and s != d)
        assert d2d > 0 or prog.nodes > 1
        assert all(not (s >= 2 and d >= 2 and s != d) for s, d in _copy_memories(g1))
        assert len(g1["instrs"]) == len(g0["instrs"]) + 3 * d2d
        c0, c1 = counts_by_type(g0), counts_by_type(g1)
        assert c1.get("copy", 0) == c0.get("copy", 0) + d2d
        assert c1.get("alloc", 0) == c0.get("alloc", 0) + d2d
        assert c1.get("free", 0) == c0.get("free", 0) + d2d
        assert c1.get("kernel", 0) == c0.get("kernel", 0)
        to_host = sum(1 for s, d in _copy_memories(g1) if s >= 2 and d == 1)
        from_host = sum(1 for s, d in _copy_memories(g1) if s == 1 and d >= 2)
        assert to_host >= d2d and from_host >= d2d


def _kernel_boxes(g):
    out = []
    for r in g["instrs"]:
        if int(r[1]) == 9:  # KERNEL
            b = g["boxes"][int(r[7])]
            out.append((int(r[2]), int(r[3]), int(r[4]), tuple(int(v) for v in b)))
    return out


def test_split_2d_one_column_equals_the_1d_split():
    """A 2D split with one chunk column and a row count that is a multiple of
    the node count assigns exactly as the 1D split: the graphs are equal."""
    for N, D, C in ((2, 2, 4), (2, 3, 6), (3, 2, 6), (4, 4, 16)):
        p1 = W.wave_program(n=24, steps=4, nodes=N, devices=D, chunks=C, lookahead=2)
        p2 = W.wave_program(n=24, steps=4, nodes=N, devices=D, chunks=C | (1 << 16), lookahead=2)
        g1, _ = oracle_graphs(p1)
        g2, _ = oracle_graphs(p2)
        for n in range(N):
            for k in ("instrs", "edges", "boxes", "binds"):
                assert np.array_equal(g1[n][k], g2[n][k]), (N, D, C, n, k)


def test_split_2d_tiles_the_range_and_nodes_own_row_bands():
    """Per task the kernels' chunk boxes tile the range; each node's chunks
    cover a band of whole rows (one box); each device gets chunks; indices
    are iy * Cx + ix."""
    N, D, Cy, Cx, n_ = 2, 3, 4, 3, 24
    p = W.wave_program(n=n_, steps=2, nodes=N, devices=D, chunks=Cy | (Cx << 16), lookahead=0)
    gs, _ = oracle_graphs(p)
    by_seq = {}
    for node, g in enumerate(gs):
        for seq, idx, mem, b in _kernel_boxes(g):
            by_seq.setdefault(seq, []).append((node, idx, mem, b))
    for seq, ks in by_seq.items():
        cover = np.zeros((n_, n_), np.int32)
        for node, idx, mem, b in ks:
            cover[b[0]:b[3], b[1]:b[4]] += 1
            iy, ix = divmod(idx, Cx)
            assert (b[0], b[3]) == (iy * n_ // Cy, (iy + 1) * n_ // Cy)
            assert (b[1], b[4]) == (ix * n_ // Cx, (ix + 1) * n_ // Cx)
        assert (cover == 1).all()
        for node in range(N):
            mine = [b for nd, _, _, b in ks if nd == node]
            lo, hi = min(b[0] for b in mine), max(b[3] for b in mine)
            assert sum((b[3] - b[0]) * (b[4] - b[1]) for b in mine) == (hi - lo) * n_
            assert len({mem for nd, _, mem, _ in ks if nd == node}) == D


def _horizon_seqs(g):
    return [int(r[2]) for r in g["instrs"] if int(r[1]) == 1]  # HORIZON


def test_horizon_cp_on_a_chain_equals_the_count_cadence():
    """Every wave task depends on the one before (a chain): the critical path
    grows by one per task, so horizons come every horizon_step tasks, as with
    the count cadence — the graphs are identical."""
    for step in (1, 2, 4):
        p = W.wave_program(n=16, steps=12, nodes=2, devices=2, chunks=4, lookahead=2, horizon_step=step)
        g0, _ = oracle_graphs(p)
        p.horizon_cp = True
        g1, _ = oracle_graphs(p)
        for a, b in zip(g0, g1):
            for k in ("instrs", "edges", "boxes", "binds"):
                assert np.array_equal(a[k], b[k]), (step, k)


def _independent(k, step, chains=1):
    """k tasks writing `chains` separate buffers in turn, each task reading the
    buffer it writes (one chain per buffer)."""
    bufs = [W.Buffer(1, (8, 1, 1), 4, np.arange(8, dtype=np.uint32), "u32") for _ in range(chains)]
    ops = [("buffer", b) for b in bufs]
    for i in range(k):
        ops.append(("task", W.Task(1, (8, 1, 1), 2, W.K_GENERIC, [W.Accessor(i % chains, W.READ_WRITE, W.one_to_one())])))
    ops.append(("flush",))
    p = W.Program(f"chains{chains}", 1, 2, step, 0, ops)
    p.horizon_cp = True
    return p


def test_horizon_cp_counts_the_critical_path_not_the_tasks():
    """c interleaved independent chains of k tasks: the critical path grows by
    one every c tasks, so a horizon comes every c * horizon_step tasks; with
    tasks that share nothing (one task per chain) none ever comes after the
    first horizon_step levels."""
    for chains, k, step in ((1, 12, 3), (2, 12, 3), (3, 18, 2), (4, 16, 2)):
        g, _ = oracle_graphs(_independent(k, step, chains))
        seqs = _horizon_seqs(g[0])
        # task i (0-based) has depth i // chains + 1; a horizon follows the first
        # task of each depth that is a multiple of step
        tasks_with_horizon = [i for i in range(k) if i % chains == 0 and (i // chains + 1) % step == 0]
        assert len(seqs) == len(tasks_with_horizon), (chains, k, step, seqs)
    g, _ = oracle_graphs(_independent(10, 2, chains=10))
    assert _horizon_seqs(g[0]) == []
