"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
and exports every entry point declared in include/igs.h."""
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
