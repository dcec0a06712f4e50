"""Accessor bounds checking (Sec. 4.4): a kernel that reads one row past its
accessor's one_to_one range reports, per kernel instruction, exactly the row
after its chunk as the bounding box of its out-of-range indices, on both
executors; the accesses inside the range give the expected values; a kernel
whose reads stay inside what its mappers grant reports nothing."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W

pytestmark = pytest.mark.gpu

H, WID = 33, 16


def _shift_program(dy, dx, mapper, nodes=2, devices=2, chunks=4, lookahead=0):
    rng = np.random.default_rng(12)
    src = rng.random((H, WID), dtype=np.float32)
    ops = [("buffer", W.Buffer(2, (H, WID, 1), 4, src, "f32")), ("buffer", W.Buffer(2, (H, WID, 1), 4, None, "f32"))]
    ops.append(("task", W.Task(2, (H - 1, WID, 1), chunks, W.K_SHIFT,
                               [W.Accessor(0, W.READ, mapper), W.Accessor(1, W.WRITE, W.one_to_one())],
                               params=(dy & 0xFFFFFFFF, dx & 0xFFFFFFFF, 0, 0))))
    ops.append(("flush",))
    return W.Program(f"shift{dy}{dx}", nodes, devices, 4, lookahead, ops), src


def _kernels(ctx, nodes):
    """(seq, node, chunk, chunk box) of every kernel instruction."""
    out = []
    for n in range(nodes):
        g = ctx.graph(n)
        for ins in g["instrs"]:
            if int(ins[1]) == 9:  # IGS_KERNEL
                b = g["boxes"][int(ins[7])]
                out.append((int(ins[2]), n, int(ins[3]), tuple(int(v) for v in b[:3]), tuple(int(v) for v in b[3:])))
    return out


@pytest.mark.parametrize("executor", [0, 1])
def test_row_past_the_chunk_is_reported(executor):
    from paper_2503_10516_gb300 import igs
    p, src = _shift_program(1, 0, W.one_to_one())
    g = igs.GpuImpl(p)
    g.ctx.set_executor(executor)
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            g.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, True if b.init is not None else False)
        elif op[0] == "task":
            g.submit(op[1])
        elif op[0] == "flush":
            g.flush()
    with pytest.raises(igs.IgsError) as e:
        g.ctx.execute()
    assert e.value.code == igs.IGS_ERR_OUT_OF_BOUNDS
    kernels = _kernels(g.ctx, p.nodes)
    assert len(kernels) == 4
    want = sorted((seq, n, ch, 0, (hi[0], 0, 0), (hi[0] + 1, WID, 1)) for seq, n, ch, lo, hi in kernels)
    got = sorted((r["seq"], r["node"], r["chunk"], r["accessor"], r["lo"], r["hi"]) for r in g.ctx.bounds_errors())
    assert got == want
    # rows whose shifted read stayed inside the chunk's range hold the source row below
    out = g.ctx.read_buffer(1, (0, 0, 0), (H, WID, 1), 4).view(np.float32).reshape(H, WID)
    for seq, n, ch, lo, hi in kernels:
        for y in range(lo[0], hi[0] - 1):
            assert np.array_equal(out[y], src[y + 1]), f"row {y}"
    # a second execute with nothing new reports nothing new
    g.ctx.execute()
    assert len(g.ctx.bounds_errors()) == 4
    g.ctx.close()


@pytest.mark.parametrize("executor", [0, 1])
def test_reads_inside_the_permitted_box_report_nothing(executor):
    """The same kernel reading row y+1 and column x-1 through an `all`
    accessor: every index is permitted, and the output is the shifted input."""
    from paper_2503_10516_gb300 import igs
    p, src = _shift_program(1, -1, W.all_mapper())
    g = igs.GpuImpl(p)
    g.ctx.set_executor(executor)
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            g.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, True if b.init is not None else False)
        elif op[0] == "task":
            g.submit(op[1])
        elif op[0] == "flush":
            g.flush()
    g.ctx.execute()
    assert g.ctx.bounds_errors() == []
    out = g.ctx.read_buffer(1, (0, 0, 0), (H, WID, 1), 4).view(np.float32).reshape(H, WID)
    assert np.array_equal(out[:H - 1, 1:], src[1:, :WID - 1])
    assert np.array_equal(out[:H - 1, 0], np.zeros(H - 1, np.float32))
    g.ctx.close()


def test_pipelined_run_reports_too():
    from paper_2503_10516_gb300 import igs
    p, _ = _shift_program(2, 0, W.one_to_one(), nodes=1, devices=2, chunks=2)
    c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED)
    c.set_executor(igs.EXEC_DATAFLOW)
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
        elif op[0] == "task":
            c.submit(op[1])
    c.submit_epoch()
    with pytest.raises(igs.IgsError) as e:
        c.run(1)
    assert e.value.code == igs.IGS_ERR_OUT_OF_BOUNDS
    errs = c.bounds_errors()
    kernels = _kernels(c, p.nodes)
    assert sorted((r["chunk"], r["lo"][0], r["hi"][0]) for r in errs) == \
        sorted((ch, hi[0], min(hi[0] + 2, H)) for _, _, ch, _, hi in kernels)
    c.close()
