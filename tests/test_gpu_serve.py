"""Served lowering: a persistent device loop lowers the submissions of many
concurrent program streams as they arrive. Every stream's graph is the same
in the mix as alone (the oracle's, and plain per-task lowering's)."""
import time

import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, oracle_graphs

pytestmark = pytest.mark.gpu


def _ctx(prog, mode=0):
    from paper_2503_10516_gb300 import igs
    c = igs.Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=mode, **igs.small_caps(prog))
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
    return c


def _streams():
    progs = [W.growing_program(rows_max=200, cols=16, grow=(1, 12), devices=2, chunks=2, lookahead=L, seed=100 + i)
             for i, L in enumerate([0, 4, 0xFFFFFFFF, 0, 8])]
    progs += [W.wave_program(n=32, steps=12, nodes=2, devices=2, chunks=8, lookahead=2),
              W.growing_program(rows_max=96, cols=1, grow=(1, 9), nodes=2, devices=2, chunks=4, lookahead=3, seed=7)]
    return progs


def _interleaved(progs, rng):
    """(stream, op) in a random interleaving that keeps each stream's order."""
    pos = [0] * len(progs)
    bodies = [[op for op in p.ops if op[0] != "buffer"] for p in progs]
    out = []
    while any(pos[i] < len(bodies[i]) for i in range(len(progs))):
        i = int(rng.choice([k for k in range(len(progs)) if pos[k] < len(bodies[k])]))
        out.append((i, bodies[i][pos[i]]))
        pos[i] += 1
    return out


def test_served_streams_match_alone():
    from paper_2503_10516_gb300 import igs
    progs = _streams()
    srv = igs.Server(max_slots=64)
    ctxs = [_ctx(p) for p in progs]
    for c, p in zip(ctxs, progs):
        assert srv.attach(c, 4 * len(p.ops) + 16) == 0
    srv.start()
    for i, op in _interleaved(progs, np.random.default_rng(1)):
        if op[0] == "task":
            ctxs[i].submit(op[1])
        elif op[0] == "flush":
            ctxs[i].submit_epoch()
    for c in ctxs:
        srv.detach(c)
    srv.stop()
    for c, p in zip(ctxs, progs):
        ref, rej = oracle_graphs(p)
        alone = _ctx(p)
        for op in p.ops:
            if op[0] == "task":
                alone.submit(op[1])
            elif op[0] == "flush":
                alone.flush()
        for n in range(p.nodes):
            g = c.graph(n)
            assert_same_graph(g, ref[n], f"{p.name} node {n} (served vs oracle)")
            assert_same_graph(g, alone.graph(n), f"{p.name} node {n} (served vs alone)")
        alone.close()
        c.close()
    srv.close()


def test_admission_by_hbm_budget():
    from paper_2503_10516_gb300 import igs
    p = W.growing_program(rows_max=64, cols=16, grow=(1, 8), devices=2, chunks=2)
    a, b = _ctx(p), _ctx(p)
    probe = igs.Server(max_slots=8)
    assert probe.attach(a, 1024) == 0
    probe.detach(a)
    probe.close()
    # a budget that fits one of them only
    from paper_2503_10516_gb300.igs import lib
    srv = igs.Server(max_slots=8, hbm_budget_bytes=1)
    assert srv.attach(b, 1024) == -7
    srv.close()
    a.close()
    b.close()


def test_served_after_idle_exit():
    """The loop leaves after its idle timeout; detach restarts it for the
    submissions that arrived meanwhile, and the graph is still exact."""
    from paper_2503_10516_gb300 import igs
    p = W.growing_program(rows_max=80, cols=8, grow=(1, 6), devices=2, chunks=2, lookahead=0, seed=3)
    c = _ctx(p)
    srv = igs.Server(max_slots=8, idle_timeout_ms=20)
    assert srv.attach(c, 4 * len(p.ops) + 16) == 0
    srv.start()
    time.sleep(0.3)  # the loop has left by now
    for op in p.ops:
        if op[0] == "task":
            c.submit(op[1])
        elif op[0] == "flush":
            c.submit_epoch()
    srv.detach(c)
    ref, _ = oracle_graphs(p)
    assert_same_graph(c.graph(0), ref[0], "served after idle exit")
    c.close()
    srv.close()


@pytest.mark.parametrize("rate", [2e4, 1e6])
def test_replayed_trace_matches_alone(rate):
    """A timed trace replayed by the library's own submission loop
    (igs_serve_replay) at 2e4 and 1e6 arrivals/s: every item completes with
    a latency, and every stream's graph equals the oracle's."""
    from paper_2503_10516_gb300 import igs
    progs = _streams()
    srv = igs.Server(max_slots=64)
    ctxs = [_ctx(p) for p in progs]
    for c, p in zip(ctxs, progs):
        assert srv.attach(c, 4 * len(p.ops) + 16) == 0
    srv.start()
    rng = np.random.default_rng(3)
    order = _interleaved(progs, rng)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(order))) * 1e9
    trace = [(i, op[1] if op[0] == "task" else None, int(t[k])) for k, (i, op) in enumerate(order)]
    lat, wall = srv.replay(ctxs, trace, timeout_ms=60000)
    assert len(lat) == len(trace) and wall > 0
    assert int(lat.max()) <= wall
    for c in ctxs:
        srv.detach(c)
    srv.stop()
    for p, c in zip(progs, ctxs):
        ref, rej = oracle_graphs(p)
        assert c.rejected() == rej
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n} (replayed at {rate:g}/s)")
        c.close()
    srv.close()


def _queue_streams():
    """Ten one-node growing-row streams (one slot each) with mixed lookahead,
    and two two-node wave streams (two slots each)."""
    progs = [W.growing_program(rows_max=120, cols=16, grow=(1, 12), devices=2, chunks=2, lookahead=L, seed=300 + i)
             for i, L in enumerate([0, 4, 0, 8, 0xFFFFFFFF, 0, 2, 0, 4, 0])]
    progs += [W.wave_program(n=32, steps=10, nodes=2, devices=2, chunks=8, lookahead=2),
              W.wave_program(n=24, steps=8, nodes=2, devices=2, chunks=4, lookahead=0)]
    return progs


def _check_against_oracle_and_alone(progs, ctxs, what):
    for c, p in zip(ctxs, progs):
        ref, rej = oracle_graphs(p)
        assert c.rejected() == rej
        alone = _ctx(p)
        for op in p.ops:
            if op[0] == "task":
                alone.submit(op[1])
            elif op[0] == "flush":
                alone.flush()
        for n in range(p.nodes):
            g = c.graph(n)
            assert_same_graph(g, ref[n], f"{p.name} node {n} ({what} vs oracle)")
            assert_same_graph(g, alone.graph(n), f"{p.name} node {n} ({what} vs alone)")
        alone.close()


@pytest.mark.parametrize("rate", [5e4, 1e6])
def test_admission_queue_more_streams_than_slots(rate):
    """Continuous batching: 12 streams needing 14 slots on a loop of 4 slots.
    The first streams are admitted at once, the rest wait in the admission
    queue (FIFO) and are admitted as detaches free their slots (the replay
    detaches a stream once its last item is taken). Every stream's graph
    equals the oracle's and its graph lowered alone."""
    from paper_2503_10516_gb300 import igs
    progs = _queue_streams()
    srv = igs.Server(max_slots=4)
    ctxs = [_ctx(p) for p in progs]
    admitted = [srv.enqueue(c, 4 * len(p.ops) + 16) for c, p in zip(ctxs, progs)]
    assert admitted == [True] * 4 + [False] * (len(progs) - 4)
    st = srv.stats()
    assert st["waiting"] == len(progs) - 4 and st["slots_in_use"] == 4 and st["admitted"] == 4
    srv.start()
    rng = np.random.default_rng(11)
    order = _interleaved(progs, rng)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(order))) * 1e9
    trace = [(i, op[1] if op[0] == "task" else None, int(t[k])) for k, (i, op) in enumerate(order)]
    lat, wall = srv.replay(ctxs, trace, timeout_ms=60000, detach=True)
    assert len(lat) == len(trace) and int(lat.max()) <= wall
    st = srv.stats()
    # every queued stream was admitted after a detach freed its slots
    assert st["admitted"] == len(progs) and st["admitted_from_queue"] == len(progs) - 4
    assert st["waiting"] == 0 and st["peak_waiting"] == len(progs) - 4 and st["slots_in_use"] == 0
    srv.stop()
    _check_against_oracle_and_alone(progs, ctxs, f"admitted from the queue at {rate:g}/s")
    for c in ctxs:
        c.close()
    srv.close()


def test_admission_queue_by_budget():
    """Admission by HBM footprint: a budget for two streams at a time; the
    others wait and are admitted in arrival order as streams detach."""
    from paper_2503_10516_gb300 import igs
    progs = [W.growing_program(rows_max=64, cols=16, grow=(1, 8), devices=2, chunks=2, lookahead=L, seed=40 + i)
             for i, L in enumerate([0, 3, 0, 0xFFFFFFFF, 1])]
    ctxs = [_ctx(p) for p in progs]
    foot = []
    for c, p in zip(ctxs, progs):  # each stream's footprint, as the server charges it
        probe = igs.Server(max_slots=8)
        assert probe.enqueue(c, 4 * len(p.ops) + 16)
        foot.append(probe.stats()["budget_bytes_in_use"])
        probe.detach(c)
        probe.close()
    assert max(foot) < 2 * min(foot)
    srv = igs.Server(max_slots=16, hbm_budget_bytes=foot[0] + foot[1] + min(foot) // 2)
    admitted = [srv.enqueue(c, 4 * len(p.ops) + 16) for c, p in zip(ctxs, progs)]
    assert admitted == [True, True, False, False, False]
    srv.start()
    trace = [(i, op[1] if op[0] == "task" else None, 1000 * k)
             for k, (i, op) in enumerate(_interleaved(progs, np.random.default_rng(5)))]
    srv.replay(ctxs, trace, timeout_ms=60000, detach=True)
    st = srv.stats()
    assert st["admitted_from_queue"] == 3 and st["waiting"] == 0 and st["peak_waiting"] == 3
    srv.stop()
    _check_against_oracle_and_alone(progs, ctxs, "admitted by budget")
    # a stream larger than the whole budget is refused, not queued
    big = _ctx(W.growing_program(rows_max=4096, cols=1024, grow=(1, 8), devices=2, chunks=2, seed=9))
    with pytest.raises(igs.IgsError):
        srv.enqueue(big, 1024)
    big.close()
    for c in ctxs:
        c.close()
    srv.close()


@pytest.mark.parametrize("rate", [2e4, 1e6])
def test_plain_replay_comparator(rate):
    """The served loop's comparator (igs_replay_plain): one lowering launch
    per submission at its arrival, contexts on their own streams. Every
    stream's graph equals the oracle's, every item has a latency."""
    from paper_2503_10516_gb300 import igs
    progs = _streams()
    ctxs = [_ctx(p) for p in progs]
    rng = np.random.default_rng(4)
    order = _interleaved(progs, rng)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(order))) * 1e9
    trace = [(i, op[1] if op[0] == "task" else None, int(t[k])) for k, (i, op) in enumerate(order)]
    lat, wall = igs.replay_plain(ctxs, trace, timeout_ms=60000)
    assert len(lat) == len(trace) and wall > 0 and int(lat.max()) <= wall
    for p, c in zip(progs, ctxs):
        ref, rej = oracle_graphs(p)
        assert c.rejected() == rej
        for n in range(p.nodes):
            assert_same_graph(c.graph(n), ref[n], f"{p.name} node {n} (plain replay at {rate:g}/s)")
        c.close()
