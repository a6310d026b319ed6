"""Pins for the oracle's minimal run length (Sec. 5.1: runs shorter than w are extended to w
elements by insertion sort, capped at the end of the array; the next run starts after the
extended run).  The hand-worked partitions below follow that rule step by step; the closed
forms and special cases do not depend on the oracle's code."""
import numpy as np
import pytest

import oracle
import workloads


# Each case: keys, w, expected run starts (with n), expected "first pair strictly descending".
# Worked by hand, e.g. the first: from 0 the greedy run is 5 > 4 > 3 (3 <= 9 ends it), length
# 3 < 4, so the run is [0, 4); from 4 the greedy run is 9 > 1 (1 <= 2 ends it), length 2, so
# [4, 8); from 8 the run 7 8 8 9 10 is weakly ascending (10 > 3 ends it), length 5 >= 4, so
# [8, 13); position 13 is the last element: [13, min(14, 17)) = [13, 14).
@pytest.mark.parametrize("keys,w,starts,desc", [
    ([5, 4, 3, 9, 9, 1, 2, 0, 7, 8, 8, 9, 10, 3], 4, [0, 4, 8, 13, 14], [1, 1, 0, 0]),
    # [1 2 2] has length 3 = w; [1 0] is extended to min(5, 3 + 3) = 5: nothing changes
    ([1, 2, 2, 1, 0], 3, [0, 3, 5], [0, 1]),
    # [3 1] -> [0, 3); [0 5] -> [3, min(6, 6))
    ([3, 1, 2, 0, 5, 4], 3, [0, 3, 6], [1, 0]),
    # w = 2: greedy runs already have length >= 2 except a last single element
    ([3, 1, 2, 0, 5, 4], 2, [0, 2, 4, 6], [1, 1, 1]),
    ([3, 1, 2, 0, 5, 4], 1, [0, 2, 4, 6], [1, 1, 1]),
    # one ascending run longer than w
    ([0, 1, 2, 3, 4, 5, 6], 5, [0, 7], [0]),
    # the array is shorter than w: one run, extended only up to n
    ([2, 1, 0], 5, [0, 3], [1]),
    # [1 0] -> [0, 3); [0 1] -> [3, 6); the last element alone
    ([1, 0, 1, 0, 1, 0, 1], 3, [0, 3, 6, 7], [1, 0, 0]),
    # ties: [4 4 4] is one ascending run of length 3 < 4 -> [0, 4); [3 3] -> [4, min(8, 6))
    ([4, 4, 4, 3, 3, 3], 4, [0, 4, 6], [0, 0]),
])
def test_minrun_worked_examples(keys, w, starts, desc):
    a = np.array(keys, dtype=np.int32)
    res = oracle.powersort(a, np.arange(a.size, dtype=np.uint32), min_run=w)
    assert list(res.starts) == starts
    assert list(res.desc) == desc
    # the output is the stable sort whatever the partition
    order = np.argsort(a, kind="stable")
    assert np.array_equal(res.keys, a[order]) and np.array_equal(res.vals, order.astype(np.uint32))


@pytest.mark.parametrize("w", [16, 24, 32])
def test_random_permutation_partition_closed_form(w):
    """Distinct random keys: a greedy run of length >= w has probability 2 / w! per start, so
    every run is extended to exactly w elements and the partition is 0, w, 2w, ..., n."""
    n = 1000 * w + 7
    keys, _ = workloads.perm_i32(n, seed=11)
    res = oracle.powersort(keys, None, min_run=w)
    assert np.array_equal(res.starts, np.append(np.arange(0, n, w), n))
    lengths = np.diff(res.starts)
    assert res.cost == oracle.powersort_cost(lengths)[0]


@pytest.mark.parametrize("w", [2, 7, 24, 32])
def test_monotone_inputs_are_one_run(w):
    n = 5000
    up = np.sort(np.random.default_rng(w).integers(-50, 50, n).astype(np.int32))
    down = np.arange(n, 0, -1, dtype=np.int32)
    for a in (up, down):
        res = oracle.powersort(a, None, min_run=w)
        assert list(res.starts) == [0, n] and res.cost == 0


def test_long_runs_are_not_changed():
    """Every greedy run at least w long: the partition is the greedy one."""
    rng = np.random.default_rng(4)
    parts = []
    for _ in range(400):
        m = int(rng.integers(40, 400))
        blk = np.sort(rng.integers(0, 1 << 20, m)).astype(np.int32)
        parts.append(blk if rng.random() < 0.7 else np.unique(blk)[::-1].copy())
    keys = np.concatenate(parts)
    plain = oracle.powersort(keys, None)
    assert np.diff(plain.starts)[:-1].min() >= 32
    ext = oracle.powersort(keys, None, min_run=32)
    assert np.array_equal(ext.starts, plain.starts) and ext.cost == plain.cost


@pytest.mark.parametrize("seed,w", [(1, 24), (2, 5), (3, 32)])
def test_minrun_partition_invariants(seed, w):
    """Random runs with ties and descents: every run but the last is at least w long; a run
    longer than w is monotone (weakly ascending or strictly descending) and cannot be extended
    by the next element; the merge cost is the powersort cost of the run lengths (Alg. 2), and
    the output is the stable sort."""
    keys, vals = workloads.pareto_u64(60000, seed=seed, alpha=1.2, distinct=50, max_len=2000)
    res = oracle.powersort(keys, vals, kt="u64", min_run=w)
    s = res.starts
    n = keys.size
    L = np.diff(s)
    assert s[0] == 0 and s[-1] == n and L.min() >= 1
    assert L[:-1].min() >= w
    for i in np.nonzero(L > w)[0]:
        a = keys[s[i]:s[i + 1]]
        asc = bool(np.all(a[:-1] <= a[1:]))
        dsc = bool(np.all(a[:-1] > a[1:]))
        assert asc or dsc
        if s[i + 1] < n:
            nxt = keys[s[i + 1]]
            assert (asc and a[-1] > nxt) or (dsc and a[-1] <= nxt)
    assert res.cost == oracle.powersort_cost(L)[0]
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(res.keys, keys[order]) and np.array_equal(res.vals, vals[order])
