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
from tests.harness import assert_same_graph, feed

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


def _static_graphs(prog):
    import torch
    from paper_2503_10516_gb300 import igs
    outs, keep = _outputs(torch, prog.nodes)
    stream = torch.cuda.current_stream().cuda_stream
    assert igs.lower_static(prog, outs, stream) == 0
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
        got = _static_graphs(p)
        for n in range(p.nodes):
            assert_same_graph(got[n], ref[n], f"{p.name} node {n}")


def test_static_entry_point_rejects_oversized_programs():
    import torch
    from paper_2503_10516_gb300 import igs
    p = W.wave_program(n=8, steps=2, nodes=32, devices=1, chunks=32)
    outs, keep = _outputs(torch, p.nodes)
    assert igs.lower_static(p, outs, torch.cuda.current_stream().cuda_stream) == -3
