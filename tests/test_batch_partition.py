"""laps_batch_partition (host arithmetic, no GPU): the split of a batch's
problems over ranks by longest processing time first.

Checked against brute force on small instances: Graham's bound for LPT
(makespan at most (4/3 - 1/(3m)) times the optimum over all m^n
assignments), the header's bound (total / m plus the largest cost), the
stated tie rules, and rejections."""
import itertools
import types

import numpy as np
import pytest

from paper_2601_16696_gb300 import build


@pytest.fixture(scope="module")
def L():
    build.build()
    from paper_2601_16696_gb300 import laps
    laps.lib()
    return laps


def _probs(shapes):
    return [types.SimpleNamespace(d=d, M=M) for d, M in shapes]


def _cost(d, M):
    return (d + 3) // 4 * 4 * M


def _loads(shares, shapes, m):
    return [sum(_cost(*shapes[k]) for k in shares[r]) for r in range(m)]


def test_graham_bound_against_brute_force(L):
    rng = np.random.default_rng(5)
    for _ in range(60):
        n = int(rng.integers(1, 8))
        m = int(rng.integers(1, 4))
        shapes = [(int(rng.integers(2, 300)), int(rng.integers(2, 40))) for _ in range(n)]
        shares = L.partition_problems(_probs(shapes), m)
        assert sorted(sum(shares, [])) == list(range(n))
        got = max(_loads(shares, shapes, m))
        costs = [_cost(*s) for s in shapes]
        opt = min(max(sum(c for c, r in zip(costs, a) if r == q) for q in range(m))
                  for a in itertools.product(range(m), repeat=n))
        assert got <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-9
        assert got <= sum(costs) / m + max(costs)


def test_ties_and_order(L):
    # equal costs: problems in index order, each to the least-loaded, lower rank first
    assert L.partition_problems(_probs([(8, 4)] * 4), 2) == [[0, 2], [1, 3]]
    # the largest problem first; d is padded to a multiple of 4 (d = 5 costs as 8)
    assert L.partition_problems(_probs([(4, 10), (5, 10), (8, 9)]), 2) == [[1], [0, 2]]
    # more ranks than problems: the spare ranks get none
    assert L.partition_problems(_probs([(4, 2), (4, 3)]), 4) == [[1], [0], [], []]


def test_rejections(L):
    with pytest.raises(L.LapsError):
        L.partition_problems(_probs([(4, 2)]), 0)
    with pytest.raises(L.LapsError):
        L.partition_problems(_probs([(0, 2)]), 2)
    with pytest.raises(L.LapsError):
        L.partition_problems([], 2)
