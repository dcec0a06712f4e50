"""Oracle graphs satisfy the structural invariants, and executing them on
virtual memories gives the sequential result with every read coherent."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import oracle_graphs
from tests.replay import check_invariants, replay, sequential_run


def _run(p):
    gs, rej = oracle_graphs(p)
    for n, g in enumerate(gs):
        check_invariants(p, g, n)
    seq_data, seq_known = sequential_run(p, set(rej))
    data, known, stats = replay(p, gs, set(rej))
    for b in range(len(p.buffers)):
        assert np.array_equal(known[b], seq_known[b])
        k = known[b]
        assert np.array_equal(data[b][k], seq_data[b][k]), f"buffer {b} differs from sequential execution"
    return stats


@pytest.mark.parametrize("seed", range(150))
def test_random(seed):
    _run(W.random_program(seed, max_extent=10, max_tasks=12))


@pytest.mark.parametrize("prog", [
    W.jacobi_program(n=32, steps=8),
    W.wave_program(n=32, steps=10, nodes=2, devices=2, chunks=8, lookahead=8),
    W.wave_program(n=24, steps=7, nodes=4, devices=4, chunks=16, lookahead=0),
    W.nbody_program(n=64, steps=3, nodes=2, devices=2, chunks=8, lookahead=4),
    W.nbody_example_program(n=32, iterations=4),
    W.growing_program(rows_max=40, cols=8, grow=(1, 6), devices=2, chunks=2),
    W.growing_program(rows_max=40, cols=8, grow=(1, 6), devices=2, chunks=2, lookahead=0xFFFFFFFF),
    W.growing_program(rows_max=64, cols=1, grow=(1, 9), nodes=2, devices=2, chunks=4, lookahead=3),
], ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped(prog):
    stats = _run(prog)
    assert stats["kernels"] > 0 and stats["reads_checked"] > 0


def test_replay_detects_dropped_copy():
    # a graph with its coherence copies emptied must fail the stale-read check
    p = W.wave_program(n=16, steps=4, nodes=2, devices=2, chunks=8, lookahead=2)
    gs, rej = oracle_graphs(p)
    for g in gs:
        for r in g["instrs"]:
            if r[1] == 4 and r[6] == 0:
                r[8] = 0
    with pytest.raises(AssertionError, match="stale read"):
        replay(p, gs, set(rej))


def _staged(p):
    p.stage_d2d = True
    return p


@pytest.mark.parametrize("seed", range(60))
def test_random_staged_d2d(seed):
    """Host-staged device-to-device copies keep every read coherent and the
    result sequential."""
    _run(_staged(W.random_program(300_000 + seed, max_extent=10, max_tasks=12)))


@pytest.mark.parametrize("prog", [
    W.wave_program(n=32, steps=10, nodes=2, devices=2, chunks=8, lookahead=8),
    W.wave_program(n=24, steps=7, nodes=1, devices=4, chunks=16, lookahead=0),
    W.nbody_program(n=64, steps=3, nodes=2, devices=2, chunks=8, lookahead=4),
    W.growing_program(rows_max=64, cols=1, grow=(1, 9), nodes=2, devices=2, chunks=4, lookahead=3),
], ids=lambda p: f"{p.name}-L{p.lookahead}")
def test_paper_shaped_staged_d2d(prog):
    stats = _run(_staged(prog))
    assert stats["kernels"] > 0 and stats["reads_checked"] > 0


@pytest.mark.parametrize("seed", range(60))
def test_random_split_2d(seed):
    """Splits along dims 0 and 1 keep every read coherent and the result
    sequential."""
    _run(W.random_program(400_000 + seed, max_extent=10, max_tasks=10, split2d=True, max_devices=3))


@pytest.mark.parametrize("prog", [
    W.wave_program(n=32, steps=8, nodes=2, devices=2, chunks=4 | (4 << 16), lookahead=4),
    W.jacobi_program(n=32, steps=6, nodes=2, devices=2, chunks=2 | (3 << 16)),
], ids=lambda p: p.name)
def test_paper_shaped_split_2d(prog):
    stats = _run(prog)
    assert stats["kernels"] > 0 and stats["reads_checked"] > 0


@pytest.mark.parametrize("seed", range(40))
def test_random_horizon_cp(seed):
    """Horizons by the critical path keep every read coherent and the result
    sequential."""
    p = W.random_program(500_000 + seed, max_extent=10, max_tasks=12)
    p.horizon_cp = True
    _run(p)


@pytest.mark.parametrize("seed", range(40))
def test_random_all_variants_together(seed):
    p = W.random_program(600_000 + seed, max_extent=9, max_tasks=12, split2d=True, max_devices=3,
                         horizon_lookahead=True)
    p.stage_d2d = True
    p.horizon_cp = True
    _run(p)
