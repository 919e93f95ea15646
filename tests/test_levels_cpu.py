"""Algorithm 2's mask functions (host code of the library; no GPU)."""
import os
from itertools import combinations
from math import comb

import pytest

from paper_2009_01177_gb300 import tor


@pytest.fixture(scope="module", autouse=True)
def lib():
    tor.load_library()


def golden_next_masks():
    path = os.path.join(os.path.dirname(__file__), "golden", "alg2_next_mask.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    return [(int(n), int(a, 2), int(b, 2)) for n, a, b in rows]


def test_paper_worked_example():
    cases = golden_next_masks()
    assert cases
    for n, mask, nxt in cases:
        assert tor.level_next_mask(mask) == nxt
        # the same two masks are consecutive ranks of their level
        m = bin(mask).count("1")
        r = next(r for r in range(comb(n, m)) if tor.level_kth_mask(n, m, r) == mask)
        assert tor.level_kth_mask(n, m, r + 1) == nxt


@pytest.mark.parametrize("k", [1, 5, 8, 10])
def test_unranking_enumerates_each_level_in_decreasing_order(k):
    for m in range(k + 1):
        want = sorted((sum(1 << b for b in c) for c in combinations(range(k), m)), reverse=True)
        got = [tor.level_kth_mask(k, m, r) for r in range(comb(k, m))]
        assert got == want, (k, m)
        for a, b in zip(got, got[1:]):
            assert tor.level_next_mask(a) == b
        assert tor.level_next_mask(got[-1]) == 0          # the smallest mask of the level


def test_large_ranks_and_limits():
    k, m = 48, 24
    top = tor.level_kth_mask(k, m, 0)
    assert top == ((1 << 24) - 1) << 24
    last = tor.level_kth_mask(k, m, comb(k, m) - 1)
    assert last == (1 << 24) - 1
    r = 123456789012
    assert tor.level_next_mask(tor.level_kth_mask(k, m, r)) == tor.level_kth_mask(k, m, r + 1)
    with pytest.raises(tor.TorError):
        tor.level_kth_mask(k, m, comb(k, m))
    with pytest.raises(tor.TorError):
        tor.level_kth_mask(49, 3, 0)
