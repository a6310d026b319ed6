"""Pins for the oracle's node powers and merge trees (Definition "Node Power", Fig. 1,
Corollary "Cartesian tree", Lemma "Path power monotonicity")."""
import itertools
import math

import numpy as np
import pytest

import oracle
from conftest import golden


def _starts(lengths):
    return np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)


def test_fig1_printed_powers():
    g = golden("fig1_node_powers.txt")
    L = g["run_lengths"]
    st = _starts(L)
    n = int(st[-1])
    exact = [oracle.node_power(st[j - 1], st[j], st[j + 1], n) for j in range(1, len(L))]
    bits = [oracle.node_power_bits(st[j - 1], st[j], st[j + 1], n) for j in range(1, len(L))]
    assert exact == g["powers"]
    assert bits == g["powers"]
    _, _, p = oracle.powersort_cost(L)
    assert list(p[1:-1]) == g["powers"]


def test_fig1_drawn_trees_and_costs():
    g = golden("fig1_node_powers.txt")
    L = g["run_lengths"]
    m_power, d_power, _ = oracle.powersort_cost(L)
    m_peek, d_peek = oracle.peeksort_cost(L)
    assert list(d_power) == g["leaf_depths_method2"]
    assert list(d_peek) == g["leaf_depths_method1"]
    # Sec. 2.3: M = sum_i d_i L_i
    assert m_power == sum(d * l for d, l in zip(g["leaf_depths_method2"], L)) == 67
    assert m_peek == sum(d * l for d, l in zip(g["leaf_depths_method1"], L)) == 65
    # footnote of Sec. 2.3: the left tree is the better one here; it is also optimal
    assert oracle.opt_cost(L) == 65


@pytest.mark.parametrize("q,m", [(1, 0), (2, 3), (3, 1), (4, 2), (5, 0), (6, 4)])
def test_equal_runs_complete_tree(q, m):
    """2^q runs of equal length 2^m: the bisection tree is the complete binary tree, so the
    power of boundary j is q - (number of trailing zero bits of j) and M = n*q."""
    r, ln = 1 << q, 1 << m
    L = [ln] * r
    cost, depth, p = oracle.powersort_cost(L)
    for j in range(1, r):
        tz = (j & -j).bit_length() - 1
        assert p[j] == q - tz
    assert cost == r * ln * q
    assert all(d == q for d in depth)


def test_powers_range_and_uniqueness():
    rng = np.random.default_rng(5)
    for _ in range(300):
        r = int(rng.integers(2, 60))
        L = rng.integers(1, 1000, size=r)
        n = int(L.sum())
        _, _, p = oracle.powersort_cost(L)
        inner = p[1:-1]
        assert inner.min() >= 1 and inner.max() <= math.floor(math.log2(n)) + 1
        assert np.all(inner[1:] != inner[:-1])  # adjacent boundaries never tie
        assert np.count_nonzero(inner == 1) == 1  # a unique root
        # equal powers are always separated by a smaller one
        for a, b in itertools.combinations(range(len(inner)), 2):
            if inner[a] == inner[b]:
                assert inner[a + 1:b].min() < inner[a]


def test_exact_power_equals_31bit_form_large_n():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        n = int(rng.integers(3, (1 << 31) - 1))
        s1 = int(rng.integers(0, n - 2))
        e1 = int(rng.integers(s1 + 1, n - 1))
        e2 = int(rng.integers(e1 + 1, n + 1))
        assert oracle.node_power(s1, e1, e2, n) == oracle.node_power_bits(s1, e1, e2, n)


def test_31bit_form_exact_for_greedy_boundaries_below_2p32():
    """For 2^31 <= n < 2^32 the 31-bit form still equals the exact power on every boundary a
    greedy run partition can produce: two runs of total length >= 4 (b - a >= 2^-31), or the
    array's last boundary with lengths (>= 2, 1) -- the only place a run of one element occurs.
    So powers stay <= 31 although the general bound floor(lg n) + 1 is 32."""
    rng = np.random.default_rng(8)
    top = []
    for _ in range(4000):
        n = int(rng.integers(1 << 31, 1 << 32))
        l1 = int(rng.integers(2, 8))
        l2 = int(rng.integers(max(2, 4 - l1), 8))
        s1 = int(rng.integers(0, n - l1 - l2 + 1))
        p = oracle.node_power(s1, s1 + l1, s1 + l1 + l2, n)
        assert p == oracle.node_power_bits(s1, s1 + l1, s1 + l1 + l2, n) <= 31
        top.append(p)
        for l1 in (2, 3, 5):  # the last boundary: a run of one element at the end
            p = oracle.node_power(n - 1 - l1, n - 1, n, n)
            assert p == oracle.node_power_bits(n - 1 - l1, n - 1, n, n) <= 31
    assert max(top) == 31  # the largest power of these sizes does occur
    # the general bound is reached only by two adjacent runs of one element, which greedy runs
    # never produce
    assert oracle.node_power((1 << 31) + 1, (1 << 31) + 2, (1 << 31) + 3, (1 << 32) - 1) == 32


def test_cartesian_tree_equals_stack_tree_and_monotone_paths():
    rng = np.random.default_rng(11)
    for _ in range(200):
        r = int(rng.integers(2, 80))
        L = rng.integers(2, 50, size=r)
        # build data whose greedy runs are exactly L: ascending runs, each starting below the
        # previous run's end
        keys = []
        base = 10 ** 6
        for ln in L:
            keys.extend(range(base, base + ln))
            base -= 1000
        keys = np.array(keys, dtype=np.int32)
        res = oracle.powersort(keys)
        assert res.r == r
        parent, rc = oracle.cartesian_parent(res.power)
        assert rc == 0
        assert np.array_equal(parent[1:r], res.node_parent[1:r])
        for j in range(1, r):
            if parent[j] >= 0:
                assert res.power[parent[j]] < res.power[j]
        # leaf parents are the adjacent boundary with the larger power
        for i in range(r):
            cand = [b for b in (i, i + 1) if 1 <= b <= r - 1]
            want = max(cand, key=lambda b: res.power[b]) if cand else -1
            assert res.leaf_parent[i] == want
