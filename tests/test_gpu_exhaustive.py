"""Exhaustive small cases on the GPU, all in one segmented call each, against the CPU oracle:
every pattern of adjacent relations (<, =, >) for 2 <= n <= 8 (3^(n-1) arrays per n) and every
composition of 12 into run lengths (2^11 arrays, ascending runs separated by drops, plain and
with descending runs) -- output and payload bit-exact, run starts, directions, node powers, leaf
depths and merge cost equal.  Plus structural properties of the device tree: powers in
[1, floor(lg n_seg) + 1], adjacent powers differ, a node's parent has the smaller power, and on
random permutations powersort's and peeksort's merge costs are within 1.5% of each other.  The
same relation patterns and compositions with runs extended to a minimal length w (Sec. 5.1)
match the oracle's minimal-run-length powersort array by array."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_1805_04154_gb300 as ps
    from paper_1805_04154_gb300 import _build
    _build.build()
    ps.load()
    return ps


def _relation_arrays():
    rng = np.random.default_rng(5)
    arrays = []
    for n in range(2, 9):
        for pat in itertools.product((-1, 0, 1), repeat=n - 1):
            steps = np.array(pat, np.int64) * rng.integers(1, 4, size=n - 1)
            arrays.append(np.concatenate([[0], np.cumsum(steps)]).astype(np.int32))
    return arrays


def _composition_arrays():
    arrays = []
    for cuts in itertools.product((0, 1), repeat=11):
        lens, cur = [], 1
        for c in cuts:
            if c:
                lens.append(cur)
                cur = 1
            else:
                cur += 1
        lens.append(cur)
        for desc in (False, True):
            parts, base = [], 1000
            for k, L in enumerate(lens):
                run = np.arange(base, base + L, dtype=np.int32)
                if desc and k % 2:
                    run = run[::-1].copy()
                parts.append(run)
                base -= 50  # every run starts below the previous one
            arrays.append(np.concatenate(parts))
    return arrays


def _check_batch(ps, arrays):
    off = np.zeros(len(arrays) + 1, np.int64)
    off[1:] = np.cumsum([a.size for a in arrays])
    keys = np.concatenate(arrays).astype(np.int32)
    vals = np.arange(keys.size, dtype=np.uint32)
    ref = oracle.sort_segmented(keys, vals, off)
    dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
    doff = torch.from_numpy(off).cuda()
    an = ps.ps_analyze(dk, offsets=doff, key_type=0)
    np.testing.assert_array_equal(an["starts"], ref[2])
    np.testing.assert_array_equal(an["desc"], ref[3])
    np.testing.assert_array_equal(an["power"].astype(np.int32), ref[4])
    np.testing.assert_array_equal(an["leaf_depth"].astype(np.int32), ref[5])
    assert an["cost"] == ref[6]
    ps.ps_sort_segmented(dk, dv, doff, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref[1])
    return an, off


def test_all_relation_patterns(ps):
    _check_batch(ps, _relation_arrays())


def test_all_compositions_of_12(ps):
    _check_batch(ps, _composition_arrays())


def test_tree_structure_properties(ps):
    keys, vals, off = workloads.segmented_i32(200, seed=17, lo_exp=1, hi_exp=16)
    an, _ = _check_batch(ps, [keys[a:b] for a, b in zip(off[:-1], off[1:])])
    S, P, L, R = an["starts"], an["power"].astype(np.int64), an["node_left"], an["node_right"]
    seg_of_run = np.searchsorted(off, S[:-1], side="right") - 1
    for j in range(1, an["runs"]):
        if seg_of_run[j] != seg_of_run[j - 1]:
            assert P[j] == 0  # segment border
            continue
        s = seg_of_run[j]
        n_seg = int(off[s + 1] - off[s])
        assert 1 <= P[j] <= int(np.floor(np.log2(n_seg))) + 1
        assert P[j] != P[j - 1] or P[j - 1] == 0
        par = L[j] if P[L[j]] > P[R[j]] else R[j]
        assert P[par] < P[j]


def test_permutation_costs_of_both_trees_agree(ps):
    keys, _ = workloads.perm_i32(1 << 20, seed=23)
    dk = torch.from_numpy(keys).cuda()
    c_pow = ps.ps_analyze(dk, key_type=0)["cost"]
    c_peek = ps.ps_analyze(dk, key_type=0, tree=ps.PS_TREE_PEEKSORT)["cost"]
    assert abs(c_pow - c_peek) / c_pow < 0.015


def test_bounded_wait_timeout_reported_and_device_usable(ps):
    ps.ps_selftest_wait_timeout(1 << 12)
    assert ps.ps_stream_status() == 5  # PS_ERR_TIMEOUT, then cleared
    assert ps.ps_stream_status() == 0
    keys, vals = workloads.runs_i32(50001, seed=3)
    ref = oracle.powersort(keys, vals)
    dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
    ps.ps_sort(dk, dv, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)


def test_level_pass_timeout_reported_and_device_usable(ps):
    """The production merge kernel's own bounded waits: in the deepest level pass one CTA never
    issues the copies of its first tile (a stage that never fills), so its consumers' wait runs
    out after the given number of polls.  The timeout is reported, nothing faults or hangs, and
    the next sort on the device equals the oracle's."""
    keys, vals = workloads.runs_i32(1 << 20, seed=8, max_len=40000)
    ref = oracle.powersort(keys, vals)
    dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
    ws = torch.empty(ps.ps_workspace_size(0, True, keys.size), dtype=torch.uint8, device="cuda")
    ps.ps_selftest_level_pass_timeout(dk, dv, ws, polls=1 << 10, key_type=0)
    assert ps.ps_stream_status() == 5  # PS_ERR_TIMEOUT, then cleared
    assert ps.ps_stream_status() == 0
    dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
    ps.ps_sort_ws(dk, dv, ws, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
    # an array without any merge large enough for a level pass has no stage to withhold
    small, _ = workloads.runs_i32(3000, seed=9)
    with pytest.raises(ps.PowersortError) as e:
        ps.ps_selftest_level_pass_timeout(torch.from_numpy(small).cuda(), None, ws, key_type=0)
    assert e.value.status == 2


def _check_batch_minrun(ps, arrays, w):
    """All arrays as segments of one minimal-run-length call, against the oracle per array."""
    off = np.zeros(len(arrays) + 1, np.int64)
    off[1:] = np.cumsum([a.size for a in arrays])
    keys = np.concatenate(arrays).astype(np.int32)
    vals = np.arange(keys.size, dtype=np.uint32)
    exp_s, exp_d, exp_ld, exp_k, exp_v, cost = [], [], [], [], [], 0
    for i, a in enumerate(arrays):
        ref = oracle.powersort(a, vals[off[i]:off[i + 1]], min_run=w)
        exp_s.append(ref.starts[:-1] + off[i])
        exp_d.append(ref.desc)
        exp_ld.append(ref.leaf_depth)
        exp_k.append(ref.keys)
        exp_v.append(ref.vals)
        cost += ref.cost
    dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
    doff = torch.from_numpy(off).cuda()
    an = ps.ps_analyze(dk, offsets=doff, key_type=0, min_run=w)
    np.testing.assert_array_equal(an["starts"], np.concatenate(exp_s + [np.array([keys.size])]))
    np.testing.assert_array_equal(an["desc"] & 1, np.concatenate(exp_d))
    np.testing.assert_array_equal(an["leaf_depth"].astype(np.int32), np.concatenate(exp_ld))
    assert an["cost"] == cost
    ws = torch.empty(ps.ps_workspace_size(0, True, keys.size, True), dtype=torch.uint8, device="cuda")
    ps.ps_sort_minrun_ws(dk, dv, ws, w, offsets=doff, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), np.concatenate(exp_k))
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), np.concatenate(exp_v))


@pytest.mark.parametrize("w", [2, 3, 4, 5, 8])
def test_all_relation_patterns_minrun(ps, w):
    """Every relation pattern of 2 <= n <= 8 with runs extended to w (Sec. 5.1): partition,
    directions, tree, cost and output equal to the oracle's for each array."""
    _check_batch_minrun(ps, _relation_arrays(), w)


@pytest.mark.parametrize("w", [3, 5, 12])
def test_all_compositions_of_12_minrun(ps, w):
    _check_batch_minrun(ps, _composition_arrays(), w)
