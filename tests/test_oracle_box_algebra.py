"""Box algebra of the oracle, pinned against dense per-element masks."""
import numpy as np
import pytest

import oracle
from tests.brute_idag import boxes_of, box_mask


def _random_disjoint(rng, shape, n):
    """n random boxes made disjoint by subtracting earlier ones (via masks)."""
    m = np.zeros(shape, dtype=bool)
    out = []
    for _ in range(n):
        lo = [int(rng.integers(0, shape[d])) for d in range(3)]
        hi = [int(rng.integers(lo[d] + 1, shape[d] + 1)) for d in range(3)]
        b = box_mask(shape, tuple(lo + hi)) & ~m
        m |= b
        out.extend(boxes_of(b))
    rng.shuffle(out)
    return out, m


@pytest.mark.parametrize("seed", range(200))
def test_canonical_matches_dense(seed):
    rng = np.random.default_rng(seed)
    dims = [1, 2, 3][seed % 3]
    shape = tuple(int(rng.integers(1, 9)) if d < dims else 1 for d in range(3))
    boxes, mask = _random_disjoint(rng, shape, int(rng.integers(1, 7)))
    got = [tuple(int(v) for v in b) for b in oracle.canonical(boxes)]
    assert got == boxes_of(mask)


def test_canonical_unique_under_fragmentation():
    # the same point set split in different ways has one canonical form
    a = [(0, 0, 0, 4, 4, 1)]
    b = [(0, 0, 0, 2, 4, 1), (2, 0, 0, 4, 2, 1), (2, 2, 0, 4, 4, 1)]
    c = [(0, 0, 0, 1, 1, 1)] + [tuple(x) for x in oracle.minus([(0, 0, 0, 4, 4, 1)], [(0, 0, 0, 1, 1, 1)])]
    ref = oracle.canonical(a).tolist()
    assert oracle.canonical(b).tolist() == ref
    assert oracle.canonical(c).tolist() == ref


def test_canonical_row_major_form():
    # an L-shape: row 0 spans [0,4), row 1 spans [0,2) -> two boxes, row-major maximal
    got = oracle.canonical([(0, 0, 0, 2, 2, 1), (0, 2, 0, 1, 4, 1)]).tolist()
    assert got == [[0, 0, 0, 1, 4, 1], [1, 0, 0, 2, 2, 1]]


@pytest.mark.parametrize("seed", range(100))
def test_minus_volume_identity(seed):
    # |A \ B| + |A n B| = |A|, and A \ B is disjoint from B
    rng = np.random.default_rng(1000 + seed)
    shape = (7, 6, 5)
    A, ma = _random_disjoint(rng, shape, 3)
    B, mb = _random_disjoint(rng, shape, 3)
    diff = oracle.minus(A, B)
    md = np.zeros(shape, dtype=bool)
    vol = 0
    for b in diff:
        bm = box_mask(shape, tuple(int(v) for v in b))
        assert not (md & bm).any(), "pieces overlap"
        md |= bm
        vol += int(bm.sum())
    assert vol == int(ma.sum()) - int((ma & mb).sum())
    assert np.array_equal(md, ma & ~mb)
