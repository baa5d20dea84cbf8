"""cudisc_partition (host logic of the multi-GPU split): contiguous ranges
whose largest cost is the smallest any contiguous split reaches, checked
against every split of small inputs, and the argument errors."""
import itertools

import numpy as np
import pytest

from paper_2402_18471_b300 import coag


def brute_best(cost, parts):
    """Smallest largest-range cost over all contiguous splits into <= parts ranges."""
    n = len(cost)
    pre = np.concatenate([[0.0], np.cumsum(cost)])
    best = np.inf
    for k in range(1, min(parts, max(n, 1)) + 1):
        for cuts in itertools.combinations(range(1, n), k - 1):
            b = (0,) + cuts + (n,)
            best = min(best, max(pre[b[i + 1]] - pre[b[i]] for i in range(k)))
    return best if n else 0.0


@pytest.mark.parametrize("seed", range(40))
def test_optimal_against_every_split(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 11))
    parts = int(rng.integers(1, 5))
    cost = rng.exponential(1.0, n) * (rng.random(n) < 0.8)      # some zero costs
    b = coag.cudisc_partition(cost, parts, n_items=n) if n else coag.cudisc_partition(None, parts, n_items=0)
    assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0) and len(b) == parts + 1
    pre = np.concatenate([[0.0], np.cumsum(cost)])
    worst = max(pre[b[i + 1]] - pre[b[i]] for i in range(parts))
    assert worst <= brute_best(cost, parts) * (1 + 1e-12) + 1e-300


def test_equal_items_split_evenly():
    b = coag.cudisc_partition(None, 8, n_items=8192)
    assert np.array_equal(b, np.arange(0, 8193, 1024))
    # whole discs of equal cost: one each
    b = coag.cudisc_partition(np.full(4, 8192.0 * 100 ** 2), 4)
    assert np.array_equal(b, np.arange(5))
    # more parts than items: trailing ranges empty, every item once
    b = coag.cudisc_partition(np.ones(3), 5)
    assert np.array_equal(b, [0, 1, 2, 3, 3, 3])


def test_errors():
    with pytest.raises(coag.CoagError):
        coag.cudisc_partition(np.array([1.0, -1.0]), 2)
    with pytest.raises(coag.CoagError):
        coag.cudisc_partition(np.array([1.0, np.nan]), 2)
    with pytest.raises(coag.CoagError):
        coag.cudisc_partition(np.ones(3), 0)
