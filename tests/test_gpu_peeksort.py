"""GPU parity of the peeksort merge tree (Alg. 1, Mehlhorn's Method 1 on the greedy runs;
PS_TREE_PEEKSORT) against the CPU oracle's peeksort: bit-exact output, identical runs, and the
tree itself -- every leaf depth (which fixes a binary tree over ordered leaves) and the merge cost.
Node records are checked for consistency: depth = power - 1 and each node's parent is the deeper
end of its range."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

KT = {"i32": 0, "u32": 1, "u64": 2, "f32": 3}


@pytest.fixture(scope="module")
def ps():
    import paper_1805_04154_gb300 as ps
    from paper_1805_04154_gb300 import _build
    _build.build()
    ps.load()
    return ps


def _dev(a: np.ndarray) -> torch.Tensor:
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def _check_tree(an):
    r = an["runs"]
    P, L, R, D = an["power"], an["node_left"], an["node_right"], an["node_depth"]
    for j in range(1, r):
        if P[j] == 0:
            continue
        assert D[j] == P[j] - 1
        assert L[j] < j < R[j]
        pl, pr = int(P[L[j]]), int(P[R[j]])
        if D[j] == 0:
            assert pl == 0 and pr == 0
        else:
            assert max(pl, pr) == P[j] - 1


def _compare(ps, keys, vals, kt):
    k_ref, v_ref, cost_ref, _ = oracle.peeksort(keys, vals, kt=kt)
    an = ps.ps_analyze(_dev(keys), key_type=KT[kt], tree=ps.PS_TREE_PEEKSORT)
    ref_runs = oracle.detect_runs(keys, kt)
    starts = np.asarray(ref_runs[0])
    np.testing.assert_array_equal(an["starts"], starts)
    c, depth = oracle.peeksort_cost(np.diff(starts))
    assert c == cost_ref
    np.testing.assert_array_equal(an["leaf_depth"].astype(np.int32), depth)
    assert an["cost"] == cost_ref
    _check_tree(an)
    dk, dv = _dev(keys), _dev(vals)
    ps.ps_sort_tree(dk, dv, ps.PS_TREE_PEEKSORT, key_type=KT[kt])
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy().view(keys.dtype), k_ref)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), v_ref)


@pytest.mark.parametrize("n", [2, 3, 17, 4097, 65537, 1 << 17, 300001])
def test_peeksort_sizes(ps, n):
    keys, vals = workloads.runs_i32(n, seed=n, max_len=max(2, int(2 * np.sqrt(n))))
    _compare(ps, keys, vals, "i32")


@pytest.mark.parametrize("max_len", [1, 3, 64, 5000, 70000])
def test_peeksort_run_regimes(ps, max_len):
    keys, vals = workloads.runs_i32(200000, seed=3, max_len=max_len)
    _compare(ps, keys, vals, "i32")


def test_peeksort_key_types_and_permutation(ps):
    keys, vals = workloads.perm_i32(1 << 18, seed=2)
    _compare(ps, keys, vals, "i32")
    keys, vals = workloads.runs_i32(1 << 17, seed=5, signed=False)
    _compare(ps, keys, vals, "u32")
    keys, vals = workloads.pareto_u64(1 << 19, seed=6)
    _compare(ps, keys, vals, "u64")
    keys, vals = workloads.pareto_f32(1 << 18, seed=7)
    _compare(ps, keys, vals, "f32")
    keys, vals = workloads.random_runs_i32(10 ** 6, seed=8, mean_len=3000)
    _compare(ps, keys, vals, "i32")


def test_peeksort_degenerate(ps):
    n = 50001
    for keys in (np.arange(n, dtype=np.int32), np.arange(n, 0, -1, dtype=np.int32), np.full(n, 3, np.int32),
                 np.tile(np.array([0, 5], np.int32), n // 2 + 1)[:n], (np.arange(n) % 977).astype(np.int32)):
        _compare(ps, keys, np.arange(n, dtype=np.uint32), "i32")


def test_peeksort_segmented(ps):
    keys, vals, off = workloads.segmented_i32(200, seed=9, lo_exp=0, hi_exp=14)
    off = off.copy()
    off[7] = off[6]  # an empty segment
    an = ps.ps_analyze(_dev(keys), offsets=torch.from_numpy(off).cuda(), key_type=0, tree=ps.PS_TREE_PEEKSORT)
    _check_tree(an)
    starts = an["starts"]
    depth_all = an["leaf_depth"].astype(np.int32)
    total = 0
    for s in range(off.size - 1):
        a, b = int(off[s]), int(off[s + 1])
        if a == b:
            continue
        i0, i1 = np.searchsorted(starts, a), np.searchsorted(starts, b)
        c, depth = oracle.peeksort_cost(np.diff(starts[i0:i1 + 1]))
        np.testing.assert_array_equal(depth_all[i0:i1], depth)
        total += c
    assert an["cost"] == total
    dk, dv = _dev(keys), _dev(vals)
    ps.ps_sort_tree(dk, dv, ps.PS_TREE_PEEKSORT, offsets=torch.from_numpy(off).cuda(), key_type=0)
    assert ps.ps_stream_status() == 0
    ref = oracle.sort_segmented(keys, vals, off)
    np.testing.assert_array_equal(dk.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref[1])


def test_peeksort_cost_not_above_bound(ps):
    """Peeksort theorem: M <= H n + 2n - (r + 2) for the greedy runs (checked on the GPU plan)."""
    keys, _ = workloads.runs_i32(1 << 20, seed=11, max_len=3000)
    an = ps.ps_analyze(_dev(keys), key_type=0, tree=ps.PS_TREE_PEEKSORT)
    L = np.diff(an["starts"]).astype(np.float64)
    n, r = L.sum(), L.size
    H = float(-(L / n * np.log2(L / n)).sum())
    assert an["cost"] <= H * n + 2 * n - (r + 2)
