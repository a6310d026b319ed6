"""Pins for the oracle's run detection (Sec. 2 run convention) and its sorted output."""
import itertools

import numpy as np
import pytest

import oracle
import workloads


@pytest.mark.parametrize("seq,starts,desc", [
    ([], [0], []),
    ([5], [0, 1], [0]),
    ([1, 2, 2, 1, 0], [0, 3, 5], [0, 1]),      # turn element belongs to the earlier run
    ([3, 2, 1], [0, 3], [1]),
    ([1, 1, 1], [0, 3], [0]),
    ([2, 1, 1], [0, 2, 3], [1, 0]),            # descending runs are strict
    ([1, 0, 1, 0, 1], [0, 2, 4, 5], [1, 1, 0]),
    ([0, 1, 0, 1, 0, 1], [0, 2, 4, 6], [0, 0, 0]),
    ([3, 3, 2, 2, 1], [0, 2, 4, 5], [0, 0, 0]),
    ([3, 3, 2, 1, 1], [0, 2, 4, 5], [0, 1, 0]),
])
def test_runs_worked_examples(seq, starts, desc):
    s, d = oracle.detect_runs(np.array(seq, dtype=np.int32))
    assert list(s) == starts
    assert list(d) == desc


def _check_partition(a, starts, desc):
    """The greedy partition is the unique one in which every run is weakly ascending or strictly
    descending with its direction set by its own first pair, every run but the last has length
    >= 2, and the element after a run breaks that run's direction."""
    n = len(a)
    assert starts[0] == 0 and starts[-1] == n
    r = len(starts) - 1
    for k in range(r):
        s, e = starts[k], starts[k + 1]
        assert e > s
        if k < r - 1:
            assert e - s >= 2
        if e - s >= 2:
            assert desc[k] == (1 if a[s] > a[s + 1] else 0)
        for i in range(s, e - 1):
            if desc[k]:
                assert a[i] > a[i + 1]
            else:
                assert a[i] <= a[i + 1]
        if k < r - 1:
            if desc[k]:
                assert not (a[e - 1] > a[e])
            else:
                assert not (a[e - 1] <= a[e])


def test_runs_exhaustive_small():
    for n in range(0, 8):
        for seq in itertools.product(range(3), repeat=n):
            a = np.array(seq, dtype=np.int32)
            s, d = oracle.detect_runs(a)
            _check_partition(list(seq), list(s), list(d))


def _total_order_key(bits):
    # IEEE totalOrder on binary32 patterns as an unsigned integer key (independent statement:
    # flip all bits of negatives, set the top bit of non-negatives)
    b = bits.astype(np.uint64)
    neg = (b >> 31) == 1
    return np.where(neg, (~b) & 0xFFFFFFFF, b | 0x80000000)


@pytest.mark.parametrize("kt", ["i32", "u32", "u64", "f32"])
def test_powersort_equals_stable_sort(kt):
    rng = np.random.default_rng(3)
    for trial in range(6):
        n = int(rng.integers(0, 3000))
        if kt == "i32":
            keys, vals = workloads.runs_i32(n, seed=trial + 1, max_len=40)
        elif kt == "u32":
            keys, vals = workloads.runs_i32(n, seed=trial + 1, max_len=40, signed=False)
        elif kt == "u64":
            keys, vals = workloads.pareto_u64(n, seed=trial + 1, distinct=7)
        else:
            keys, vals = workloads.pareto_f32(n, seed=trial + 1, special_frac=0.1)
        res = oracle.powersort(keys, vals, kt=kt)
        order = np.argsort(_total_order_key(keys) if kt == "f32" else keys, kind="stable")
        assert np.array_equal(res.keys, keys[order])
        assert np.array_equal(res.vals, vals[order])
        sk, sv = oracle.stable_sort(keys, vals, kt=kt)
        assert np.array_equal(sk, keys[order]) and np.array_equal(sv, vals[order])
        pk, pv, _, _ = oracle.peeksort(keys, vals, kt=kt)
        assert np.array_equal(pk, keys[order]) and np.array_equal(pv, vals[order])


def test_f32_total_order_agrees_with_float_order():
    vals = np.array([-np.inf, -3.5, -1e-30, -0.0, 0.0, 1e-30, 2.0, np.inf], dtype=np.float32)
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(vals))
    k, _ = oracle.stable_sort(vals[perm].view(np.uint32), kt="f32")
    got = k.view(np.float32)
    assert np.array_equal(got, vals)
    assert np.signbit(got[3]) and not np.signbit(got[4])  # -0 before +0
    nan_neg = np.array([0xFFC00001], np.uint32)
    nan_pos = np.array([0x7FC00001], np.uint32)
    mixed = np.concatenate([nan_pos, vals.view(np.uint32), nan_neg])
    k, _ = oracle.stable_sort(mixed, kt="f32")
    assert k[0] == nan_neg[0] and k[-1] == nan_pos[0]


def test_segmented_equals_per_segment():
    keys, vals, off = workloads.segmented_i32(40, seed=4, lo_exp=0, hi_exp=10)
    off[5] = off[4]  # an empty segment
    k, v, st, d, p, ld, cost = oracle.sort_segmented(keys, vals, off)
    total = 0
    run_pos = 0
    for s in range(len(off) - 1):
        a, b = int(off[s]), int(off[s + 1])
        res = oracle.powersort(keys[a:b], vals[a:b])
        assert np.array_equal(k[a:b], res.keys) and np.array_equal(v[a:b], res.vals)
        if b > a:
            assert np.array_equal(st[run_pos:run_pos + res.r], res.starts[:-1] + a)
            assert np.array_equal(ld[run_pos:run_pos + res.r], res.leaf_depth)
            assert p[run_pos] == 0
            assert np.array_equal(p[run_pos + 1:run_pos + res.r], res.power[1:res.r])
            run_pos += res.r
        total += res.cost
    assert cost == total and run_pos == len(st) - 1
