"""The oracle emits exactly the graph of the per-element brute-force generator."""
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import BruteImpl, OracleImpl, assert_same_graph, feed


def _check(p):
    o, b = OracleImpl(p), BruteImpl(p)
    r1, r2 = feed(o, p), feed(b, p)
    assert r1 == r2
    assert o.rejected() == b.rejected()
    for n in range(p.nodes):
        assert_same_graph(o.graph(n), b.graph(n), f"{p.name} node {n}")


@pytest.mark.parametrize("seed", range(400))
def test_random_programs(seed):
    _check(W.random_program(seed, max_extent=10, max_tasks=12))


@pytest.mark.parametrize("seed", range(40))
def test_random_programs_uninitialized_reads(seed):
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
], ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped_programs(prog):
    _check(prog)


@pytest.mark.parametrize("seed", range(150))
def test_random_programs_horizon_lookahead(seed):
    """The horizon-count lookahead heuristic (Sec. 4.3), switched on and off
    within programs, in both generators."""
    _check(W.random_program(200_000 + seed, max_extent=10, max_tasks=12, horizon_lookahead=True))


@pytest.mark.parametrize("prog", [
    W.growing_program(rows_max=40, cols=4, grow=(1, 5), lookahead=W.LOOKAHEAD_HORIZONS),
    W.wave_program(n=16, steps=14, nodes=2, devices=2, chunks=8, lookahead=W.LOOKAHEAD_HORIZONS),
    W.listing2_program(8, W.LOOKAHEAD_HORIZONS, devices=2, chunks=2),
], ids=lambda p: p.name)
def test_paper_shaped_programs_horizon_lookahead(prog):
    _check(prog)


def _staged(p):
    p.stage_d2d = True
    p.name += "-staged"
    return p


@pytest.mark.parametrize("seed", range(150))
def test_random_programs_staged_d2d(seed):
    """Device-to-device copies staged in host memory (Sec. 3.3): both
    generators emit the same allocation, two copies and free per staged copy."""
    _check(_staged(W.random_program(300_000 + seed, max_extent=10, max_tasks=12)))


@pytest.mark.parametrize("prog", [
    W.wave_program(n=16, steps=6, nodes=2, devices=2, chunks=8, lookahead=2),
    W.wave_program(n=12, steps=5, nodes=1, devices=3, chunks=6, lookahead=0),
    W.growing_program(rows_max=30, cols=1, grow=(1, 5), devices=3, chunks=3, lookahead=2),
    W.nbody_example_program(n=16, iterations=3),
], ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped_programs_staged_d2d(prog):
    _check(_staged(prog))


@pytest.mark.parametrize("seed", range(150))
def test_random_programs_split_2d(seed):
    """Splits along dims 0 and 1 (Sec. 3.1, hierarchical): both generators
    emit the same graph."""
    _check(W.random_program(400_000 + seed, max_extent=10, max_tasks=10, split2d=True, max_devices=3))


@pytest.mark.parametrize("prog", [
    W.wave_program(n=16, steps=5, nodes=2, devices=2, chunks=2 | (2 << 16), lookahead=2),
    W.wave_program(n=12, steps=4, nodes=3, devices=2, chunks=4 | (3 << 16), lookahead=0),
    W.jacobi_program(n=16, steps=4, nodes=2, devices=3, chunks=3 | (2 << 16)),
], ids=lambda p: p.name)
def test_paper_shaped_programs_split_2d(prog):
    _check(prog)


@pytest.mark.parametrize("seed", range(150))
def test_random_programs_horizon_cp(seed):
    """Horizons by the task graph's critical path (Sec. 3.5): both generators
    build the same task-level dependencies and emit the same graph."""
    p = W.random_program(500_000 + seed, max_extent=10, max_tasks=12)
    p.horizon_cp = True
    _check(p)


@pytest.mark.parametrize("seed", range(100))
def test_random_programs_all_variants_together(seed):
    """2D splits, staged device-to-device copies, critical-path horizons and
    the horizon-count lookahead in one program: both generators agree."""
    p = W.random_program(600_000 + seed, max_extent=9, max_tasks=12, split2d=True, max_devices=3,
                         horizon_lookahead=True)
    p.stage_d2d = True
    p.horizon_cp = True
    _check(p)
