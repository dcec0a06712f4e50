"""Host logic of the library, without a device: where igs_horizon_plan (the
library's own task-graph tracker, which igs_submit_task and igs_lower_static
consult) puts horizons equals where the oracle's graphs have them, for the
critical-path cadence and for the count cadence."""
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import oracle_graphs


def _oracle_plan(p):
    """Indices of the tasks a horizon follows in the oracle's graph: walking
    the operations, a task is followed by a horizon when the next sequence
    number is one of the graph's horizons."""
    g, _ = oracle_graphs(p)
    horizons = {int(r[2]) for r in g[0]["instrs"] if int(r[1]) == 1}
    seq, k, after = 0, 0, []
    for op in p.ops:
        if op[0] == "task":
            seq += 1
            if seq in horizons:
                after.append(k)
                seq += 1
            k += 1
        elif op[0] in ("buffer", "flush", "destroy"):
            seq += 1
    return after


@pytest.mark.parametrize("cp", [False, True])
@pytest.mark.parametrize("seed", range(60))
def test_plan_matches_the_oracle(seed, cp):
    from paper_2503_10516_gb300 import igs
    p = W.random_program(500_000 + seed, max_extent=10, max_tasks=14)
    p.horizon_cp = cp
    assert igs.horizon_plan(p) == _oracle_plan(p)


@pytest.mark.parametrize("prog", [
    W.wave_program(n=32, steps=13, nodes=2, devices=2, chunks=8, lookahead=2, horizon_step=3),
    W.nbody_program(n=64, steps=5, nodes=2, devices=2, chunks=8, lookahead=0, horizon_step=2),
    W.growing_program(rows_max=60, cols=4, grow=(1, 7), devices=2, chunks=2, lookahead=0, horizon_step=2),
], ids=lambda p: p.name)
def test_plan_matches_the_oracle_paper_shaped(prog):
    from paper_2503_10516_gb300 import igs
    prog.horizon_cp = True
    assert igs.horizon_plan(prog) == _oracle_plan(prog)
