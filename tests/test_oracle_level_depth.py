"""The depth bound the device-driven sorts use to launch fewer level passes, checked on the oracle's
powersort trees (Definition "Node Power", Corollary "Cartesian tree").

A node of power p (the boundary between two runs, merging the runs between its nearest
boundaries of smaller power) spans fewer than 4 n / 2^p elements: every boundary inside its
range has power >= p, so all its runs' midpoints lie in one dyadic interval of length 2^(1-p)
of the normalised array, and a first or last run's half length is below the distance from its
midpoint to its neighbour's.  With depth < power, a node larger than sub_lim (one that a level
pass merges) has depth at most pmax - 2 for the smallest pmax with sub_lim * 2^pmax >= 4 n.  Checked on random, skewed
(halving and doubling run lengths), Pareto and alternating long/short run partitions."""
import numpy as np
import pytest

import oracle


def _nodes(lengths: np.ndarray):
    """Per boundary j = 1..r-1: (power, size of its merge range, depth) from the oracle's tree."""
    _, _, power = oracle.powersort_cost(lengths)
    r = lengths.size
    S = np.concatenate([[0], np.cumsum(lengths)])
    parent, rc = oracle.cartesian_parent(power)
    assert rc == 0
    out = []
    for j in range(1, r):
        L = j - 1
        while L > 0 and power[L] >= power[j]:
            L -= 1
        R = j + 1
        while R < r and power[R] >= power[j]:
            R += 1
        d, x = 0, parent[j]
        while x > 0:  # ancestors among the boundaries 1..r-1
            d += 1
            x = parent[x]
        out.append((int(power[j]), int(S[R] - S[L]), d))
    return out


def _pmax(n: int, sub_lim: int) -> int:
    p = 0
    while (sub_lim << p) < 4 * n:
        p += 1
    return p


def _cases():
    rng = np.random.default_rng(5)
    yield np.array([1 << k for k in range(16, 0, -1)] + [1], np.int64)       # halving lengths
    yield np.array([1] + [1 << k for k in range(1, 17)], np.int64)           # doubling lengths
    yield np.array([2] * 300 + [1 << 18] + [2] * 300, np.int64)
    yield np.tile(np.array([5000, 2], np.int64), 200)
    for _ in range(6):
        yield rng.integers(1, 3000, size=int(rng.integers(50, 400))).astype(np.int64)
    for _ in range(4):
        yield np.minimum(np.floor(rng.pareto(1.2, size=500) + 1) * 3, 1 << 17).astype(np.int64)


@pytest.mark.parametrize("case", list(range(len(list(_cases())))))
def test_node_size_below_four_n_over_two_to_power(case):
    lengths = list(_cases())[case]
    n = int(lengths.sum())
    for p, size, depth in _nodes(lengths):
        assert depth < p
        assert size * (1 << p) < 4 * n
        for sub_lim in (2048, 4096, 64, 300):
            if size > sub_lim:
                assert depth <= _pmax(n, sub_lim) - 2
