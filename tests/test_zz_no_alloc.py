"""igs_lower_static: the entry point for callers that cannot allocate device
memory (their device memory all comes from their own pool, or they must not
enter the driver's allocator on a latency-critical path). It lowers a whole
program with a file-scope device array as its only scratch. Its graphs must be
identical to those of the regular entry points (igs_create / igs_submit_task /
igs_flush / igs_fetch_instructions), on two calls in a row — the second call
reuses the array the first one left behind.

This file is collected last on purpose (pytest orders files by name)."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs

pytestmark = pytest.mark.gpu

CAP = 1 << 14


def _outputs(torch, nodes):
    outs, keep = [], []
    for _ in range(nodes):
        t = {"instrs": torch.zeros(CAP * 11, dtype=torch.int32, device="cuda"),
             "edges": torch.zeros(CAP * 4 * 3, dtype=torch.int32, device="cuda"),
             "boxes": torch.zeros(CAP * 4 * 6, dtype=torch.int32, device="cuda"),
             "binds": torch.zeros(CAP * 2 * 7, dtype=torch.int32, device="cuda"),
             "diags": torch.zeros(CAP * 3, dtype=torch.int32, device="cuda"),
             "counts": torch.full((6,), 7, dtype=torch.int32, device="cuda")}
        keep.append(t)
        outs.append({"instrs": (t["instrs"].data_ptr(), CAP), "edges": (t["edges"].data_ptr(), 4 * CAP),
                     "boxes": (t["boxes"].data_ptr(), 4 * CAP), "binds": (t["binds"].data_ptr(), 2 * CAP),
                     "diags": (t["diags"].data_ptr(), CAP), "counts": t["counts"].data_ptr()})
    return outs, keep


def _static_graphs(prog, expect=0):
    import torch
    from paper_2503_10516_gb300 import igs
    outs, keep = _outputs(torch, prog.nodes)
    stream = torch.cuda.current_stream().cuda_stream
    assert igs.lower_static(prog, outs, stream) == expect
    graphs = []
    for t in keep:
        cnt = t["counts"].cpu().numpy().view(np.uint32)
        assert cnt[5] == 0, f"node status {cnt[5]}"
        widths = {"instrs": 11, "edges": 3, "boxes": 6, "binds": 7, "diags": 3}
        g = {}
        for k, key in enumerate(("instrs", "edges", "boxes", "binds", "diags")):
            arr = t[key].cpu().numpy().view(np.uint32).reshape(-1, widths[key])
            g[key] = arr[:cnt[k]].copy()
        graphs.append(g)
    return graphs


def _regular_graphs(prog):
    from paper_2503_10516_gb300 import igs
    g = igs.GpuImpl(prog)
    feed(g, prog)
    out = [g.graph(n) for n in range(prog.nodes)]
    g.ctx.close()
    return out


@pytest.mark.parametrize("seed", [3, 11])
def test_static_entry_point_matches_regular_twice(seed):
    progs = [W.wave_program(n=32, steps=10, nodes=2, devices=2, chunks=8, lookahead=2),
             W.random_program(seed, max_extent=10, max_tasks=12)]
    for p in progs:  # two calls in a row on the same array
        ref = _regular_graphs(p)
        orc, rej = oracle_graphs(p)
        got = _static_graphs(p, expect=-2 if rej else 0)
        for n in range(p.nodes):
            assert_same_graph(got[n], ref[n], f"{p.name} node {n}")
            assert_same_graph(got[n], orc[n], f"{p.name} node {n} (oracle)")


def test_static_entry_point_rejects_oversized_programs():
    import torch
    from paper_2503_10516_gb300 import igs
    p = W.wave_program(n=8, steps=2, nodes=32, devices=1, chunks=32)
    outs, keep = _outputs(torch, p.nodes)
    assert igs.lower_static(p, outs, torch.cuda.current_stream().cuda_stream) == -3


def _prog(ops, nodes=1, devices=2):
    return W.Program("static-checks", nodes, devices, 4, 0, ops)


def _buf(extent=(16, 8, 1), dims=2, elem=4):
    return W.Buffer(dims, extent, elem, None)


def _task(accs, rng=(16, 8, 1), dims=2, chunks=2):
    return W.Task(dims, rng, chunks, W.K_GENERIC, accs)


def test_static_entry_point_checks_like_the_context_api():
    """The inputs the context API rejects are rejected here too, before any
    lowering: a task on a destroyed buffer, a second destruction, an unused
    range dimension other than 1, a zero extent or element size, unknown
    configuration flags."""
    import torch
    from paper_2503_10516_gb300 import igs
    w = W.Accessor(0, W.WRITE, W.one_to_one())
    r = W.Accessor(0, W.READ, W.one_to_one())
    cases = {
        "read after destroy": _prog([("buffer", _buf()), ("task", _task([w])), ("destroy", 0), ("task", _task([r]))]),
        "destroy twice": _prog([("buffer", _buf()), ("task", _task([w])), ("destroy", 0), ("destroy", 0)]),
        "unused range dim": _prog([("buffer", _buf()), ("task", _task([w], rng=(16, 8, 2)))]),
        "zero extent": _prog([("buffer", _buf(extent=(16, 0, 1))), ("task", _task([w]))]),
        "zero element size": _prog([("buffer", _buf(elem=0)), ("task", _task([w]))]),
    }
    for what, p in cases.items():
        outs, keep = _outputs(torch, p.nodes)
        assert igs.lower_static(p, outs, torch.cuda.current_stream().cuda_stream) == -1, what
    p = _prog([("buffer", _buf()), ("task", _task([w]))])
    p.horizon_cp = True
    outs, keep = _outputs(torch, p.nodes)
    from paper_2503_10516_gb300.igs import Config, lib
    import ctypes
    cfg = Config(1, 2, 4, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, None, 1 << 7)  # an undefined flag bit
    sb = (igs.StaticBuffer * 1)()
    sb[0].dims, sb[0].elem_size = 2, 4
    sb[0].extent[0], sb[0].extent[1], sb[0].extent[2] = 16, 8, 1
    out = (igs.StaticOutput * 1)()
    o = outs[0]
    out[0].instrs, out[0].instr_cap = o["instrs"]
    out[0].edges, out[0].edge_cap = o["edges"]
    out[0].boxes, out[0].box_cap = o["boxes"]
    out[0].binds, out[0].bind_cap = o["binds"]
    out[0].diags, out[0].diag_cap = o["diags"]
    out[0].counts = o["counts"]
    so = (igs.StaticOp * 1)(igs.StaticOp(0, 0))
    words = np.zeros(123, np.uint32)
    assert lib().igs_lower_static(ctypes.byref(cfg), sb, 1, igs._p32(words), 0, so, 1, out,
                                  torch.cuda.current_stream().cuda_stream) == -1


def test_static_entry_point_reports_overlapping_writes():
    """A task whose chunks write overlapping regions (Sec. 4.4) is left out of
    the graph and the call returns IGS_ERR_OVERLAPPING_WRITE; the graph of the
    other tasks equals the oracle's."""
    w = W.Accessor(0, W.WRITE, W.one_to_one())
    bad = W.Accessor(1, W.WRITE, W.neighborhood(1, 0))
    p = _prog([("buffer", _buf()), ("buffer", _buf()), ("task", _task([w])), ("task", _task([bad])),
               ("task", _task([w, W.Accessor(1, W.WRITE, W.one_to_one())])), ("flush",)])
    orc, rej = oracle_graphs(p)
    assert len(rej) == 1
    got = _static_graphs(p, expect=-2)
    for n in range(p.nodes):
        assert_same_graph(got[n], orc[n], f"overlapping writes node {n}")
