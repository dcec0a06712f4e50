"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
and exports every entry point declared in include/igs.h; the binding's batch
shape candidates and the host-only horizon plan behave."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "igs.h")).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(igs_\w+)\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2503_10516_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("igs_create", "igs_submit_task", "igs_set_lookahead", "igs_flush", "igs_fetch_instructions",
              "igs_execute", "igs_create_buffer", "igs_box_copy", "igs_lower_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    from paper_2503_10516_gb300 import igs
    L = igs.lib()
    for n in igs.EXPORTS:
        assert hasattr(L, n)


def test_binding_exports_match_header():
    from paper_2503_10516_gb300 import igs
    assert set(igs.EXPORTS) == set(_declared())


def test_batch_shape_candidates():
    """The tuner's candidate shapes: one block per unit first, then work
    queues of 1-8 blocks per SM (never more blocks than units, no repeats),
    both orders, and multi-warp blocks with helped programs."""
    from paper_2503_10516_gb300 import igs
    for units, sms in ((4073, 152), (100, 152), (1, 152), (700, 16)):
        c = igs.batch_shape_candidates(units, sms)
        assert c[0] is None
        rest = c[1:]
        assert len(rest) == len(set(rest))
        assert all(1 <= g <= units and order in (0, 1) and 1 <= warps <= 8 and helped >= 0
                   for g, order, warps, helped in rest)
        assert any(order == igs.ORDER_LONGEST_FIRST for _, order, _, _ in rest)
        assert any(warps > 1 and helped > 0 for _, _, warps, helped in rest)


def test_horizon_plan_rejects_unknown_buffers():
    from paper_2503_10516_gb300 import igs
    from paper_2503_10516_gb300 import workloads as W
    b = W.Buffer(1, (8, 1, 1), 4, None)
    p = W.Program("bad", 1, 1, 2, 0, [("buffer", b),
                                      ("task", W.Task(1, (8, 1, 1), 1, W.K_GENERIC,
                                                      [W.Accessor(3, W.WRITE, W.one_to_one())]))])
    with pytest.raises(igs.IgsError):
        igs.horizon_plan(p)
