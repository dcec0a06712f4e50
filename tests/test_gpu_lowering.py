"""CUDA lowering engine vs the CPU oracle: identical graphs (instructions,
edges, box lists, bindings, diagnostics), through the C ABI."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs

pytestmark = pytest.mark.gpu


def _gpu(prog, mode=0, **kw):
    from paper_2503_10516_gb300 import igs
    g = igs.GpuImpl(prog, mode=mode, **kw)
    res = feed(g, prog)
    return g, res


def _check(prog, mode=0):
    ref, rej = oracle_graphs(prog)
    g, _ = _gpu(prog, mode)
    assert g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(g.graph(n), ref[n], f"{prog.name} node {n}")
    g.ctx.close()


@pytest.mark.parametrize("seed", range(120))
def test_random_programs_plain(seed):
    _check(W.random_program(seed, max_extent=10, max_tasks=12))


@pytest.mark.parametrize("seed", range(40))
def test_random_programs_batched(seed):
    _check(W.random_program(10_000 + seed, max_extent=10, max_tasks=12), mode=1)


@pytest.mark.parametrize("seed", range(20))
def test_random_uninitialized_reads(seed):
    _check(W.random_program(50_000 + seed, max_extent=8, max_tasks=8, uninit_reads=True))


@pytest.mark.parametrize("prog", [
    W.jacobi_program(n=16, steps=6),
    W.listing2_program(8, 0, devices=2, chunks=2),
    W.listing2_program(8, 1, devices=2, chunks=2),
    W.nbody_example_program(n=16, iterations=3),
    W.growing_program(rows_max=24, cols=4, grow=(1, 4)),
    W.growing_program(rows_max=24, cols=4, grow=(1, 4), lookahead=0xFFFFFFFF),
    W.growing_program(rows_max=30, cols=1, grow=(1, 5), devices=3, chunks=3, lookahead=2),
    W.wave_program(n=16, steps=6, nodes=2, devices=2, chunks=8, lookahead=2),
    W.wave_program(n=12, steps=5, nodes=3, devices=1, chunks=5, lookahead=0),
    W.wave_program(n=64, steps=12, nodes=4, devices=4, chunks=64, lookahead=8),
    W.nbody_program(n=256, steps=4, nodes=8, devices=4, chunks=128, lookahead=4),
], ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped(prog):
    _check(prog)
    _check(prog, mode=1)


def test_jacobi_256_full_config():
    """The 256x256 Jacobi configuration: 2 nodes x 2 devices, 4 chunks, 8 steps."""
    _check(W.jacobi_program())


def _shape_only(prog, extents, task_range):
    """The same program with tiny data: lowering depends on shapes only."""
    for op in prog.ops:
        if op[0] == "buffer":
            op[1].extent = extents
        elif op[0] == "task":
            op[1].range = task_range
    return prog


def _check_full(prog, big_inits):
    """Graph parity at full size; GPU buffers get zero-filled host data of the
    full shape (lowering never looks at values)."""
    from paper_2503_10516_gb300 import igs
    ref, rej = oracle_graphs(prog)
    g = igs.GpuImpl(prog)
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            init = big_inits(b) if b.init is not None else None
            g.ctx.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, init)
            g._buffers.append(b)
        elif op[0] == "task":
            g.ctx.submit(op[1])
        elif op[0] == "flush":
            g.ctx.flush()
    assert g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(g.graph(n), ref[n], f"{prog.name} node {n}")
    g.ctx.close()


def test_wave_8192_full_config():
    """3 x 8192^2 fp32, 4 nodes x 4 devices, 64 chunks, 1000 steps, lookahead 8."""
    p = W.wave_program(n=8, steps=1000, nodes=4, devices=4, chunks=64, lookahead=8)
    _shape_only(p, (8192, 8192, 1), (8192, 8192, 1))
    _check_full(p, lambda b: np.zeros((8192, 8192), np.float32))


def test_nbody_1m_full_config():
    """2^20 float4 positions and velocities, 8 nodes x 4 devices, 128 chunks,
    200 steps of two tasks, lookahead 4."""
    n = 1 << 20
    p = W.nbody_program(n=8, steps=200, nodes=8, devices=4, chunks=128, lookahead=4)
    _shape_only(p, (n, 1, 1), (n, 1, 1))
    _check_full(p, lambda b: np.zeros((n, 4), np.float32))


@pytest.mark.parametrize("seed", range(60))
def test_random_programs_horizon_lookahead(seed):
    """The horizon-count lookahead heuristic (Sec. 4.3) on the GPU."""
    p = W.random_program(200_000 + seed, max_extent=10, max_tasks=12, horizon_lookahead=True)
    _check(p, mode=seed % 2)


@pytest.mark.parametrize("prog", [
    W.growing_program(rows_max=64, cols=8, grow=(1, 6), devices=2, chunks=2, lookahead=W.LOOKAHEAD_HORIZONS),
    W.wave_program(n=64, steps=24, nodes=4, devices=4, chunks=64, lookahead=W.LOOKAHEAD_HORIZONS),
    W.nbody_program(n=256, steps=6, nodes=8, devices=4, chunks=128, lookahead=W.LOOKAHEAD_HORIZONS),
], ids=lambda p: p.name)
def test_paper_shaped_horizon_lookahead(prog):
    _check(prog)
    _check(prog, mode=1)
