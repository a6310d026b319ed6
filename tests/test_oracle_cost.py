"""Pins for the oracle's merge costs: the bounds of the Powersort and Peeksort theorems, the
entropy lower bound (Sec. 2.3), brute-force optimal trees, and the paper's printed average
merge cost on random-runs inputs (Sec. 5.3)."""
import functools
import math

import numpy as np
import pytest

import oracle
import workloads


def _compositions(n):
    """All sequences of positive integers summing to n."""
    for mask in range(1 << (n - 1)):
        out, cur = [], 1
        for b in range(n - 1):
            if mask >> b & 1:
                out.append(cur)
                cur = 1
            else:
                cur += 1
        out.append(cur)
        yield out


def _brute_opt(L):
    """Minimum of sum d_i L_i over every binary tree with leaves L in order (enumeration)."""
    @functools.lru_cache(maxsize=None)
    def best(i, j):  # leaves i..j-1
        if j - i == 1:
            return 0
        w = sum(L[i:j])
        return w + min(best(i, k) + best(k, j) for k in range(i + 1, j))
    return best(0, len(L))


def test_opt_dp_equals_enumeration():
    rng = np.random.default_rng(2)
    for _ in range(200):
        r = int(rng.integers(1, 8))
        L = [int(x) for x in rng.integers(1, 30, size=r)]
        assert oracle.opt_cost(L) == _brute_opt(tuple(L))


@pytest.mark.parametrize("n", range(1, 13))
def test_bounds_all_compositions(n):
    for L in _compositions(n):
        r = len(L)
        H = oracle.entropy_bits(L)
        opt = oracle.opt_cost(L)
        mp, dp, pw = oracle.powersort_cost(L)
        mk, dk = oracle.peeksort_cost(L)
        eps = 1e-9 * n
        assert H * n - eps <= opt <= mp <= H * n + 2 * n + eps       # Sec. 2.3, Powersort thm
        assert opt <= mk <= H * n + 2 * n - (r + 2) + eps or r == 1  # Peeksort theorem
        assert mp == sum(d * l for d, l in zip(dp, L))
        assert mk == sum(d * l for d, l in zip(dk, L))
        if r >= 2:
            assert max(pw[1:-1]) <= math.floor(math.log2(n)) + 1


def test_trace_consistency_on_data():
    keys, vals = workloads.runs_i32(50000, seed=9)
    res = oracle.powersort(keys, vals)
    L = np.diff(res.starts)
    assert len(res.merges) == res.r - 1                 # exactly r-1 merges
    assert res.cost == int((res.merges[:, 2] - res.merges[:, 0]).sum())
    assert res.cost == int((L * res.leaf_depth).sum())  # M = sum d_i L_i
    m, d, p = oracle.powersort_cost(L)
    assert m == res.cost and np.array_equal(d, res.leaf_depth) and np.array_equal(p, res.power)
    # every merge joins two adjacent sorted ranges
    for lo, mid, hi in res.merges:
        assert lo < mid < hi
    n = keys.size
    H = oracle.entropy_bits(L)
    assert H * n <= res.cost <= H * n + 2 * n


@pytest.mark.slow
def test_paper_random_runs_average_cost():
    """Sec. 5.3: random-runs inputs, n = 10^7, geometric run lengths with mean 3000, methods with
    minimal run length w = 24: powersort's average merge cost is 1.14e8 < n lg r ~ 1.17e8.
    Soft pin: within 3% on two seeds."""
    n = 10 ** 7
    for seed in (1, 2):
        keys, _ = workloads.random_runs_i32(n, seed=seed, mean_len=3000)
        res = oracle.powersort(keys, None, min_run=24)
        assert abs(res.cost / 1.14e8 - 1) < 0.03, res.cost
        assert res.cost < n * math.log2(res.r)
        assert np.all(np.diff(res.keys) >= 0)


def test_random_permutation_costs_close():
    """Sec. 5.2: on random permutations the merge costs of all methods lie within 1.5%."""
    keys, _ = workloads.perm_i32(200000, seed=3)
    L = np.diff(oracle.detect_runs(keys)[0])
    mp, _, _ = oracle.powersort_cost(L)
    mk, _ = oracle.peeksort_cost(L)
    assert abs(mp / mk - 1) < 0.015
