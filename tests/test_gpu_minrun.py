"""GPU parity of the minimal-run-length variant (Sec. 5.1: runs shorter than w extended to w
elements, capped at the end of the array or segment) against the CPU oracle's powersort with
the same w: identical run starts, directions, leaf depths and merge cost, and bit-exact output.
Sizes span several detection tiles and tile groups (256 tiles of 8192 positions) with ragged
tails; segments include empty, one-element and shorter-than-w ones."""
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


def _extended_ok(keys, starts, flags, w, ends):
    """Bit 1 marks exactly the runs whose greedy run was shorter than their extension: such a
    run has length min(w, end - start); a run without it is monotone."""
    for i in range(starts.size - 1):
        s, e = int(starts[i]), int(starts[i + 1])
        if flags[i] & 2:
            assert e - s == min(w, int(ends[i]) - s)
        else:
            a = keys[s:e]
            assert bool(np.all(a[:-1] <= a[1:])) or bool(np.all(a[:-1] > a[1:]))


def _order_keys(keys, kt):
    """Keys as integers in the sort order (float32 patterns by IEEE totalOrder)."""
    if kt != "f32":
        return keys
    u = keys.view(np.uint32).astype(np.uint64)
    return np.where(u >> 31, u ^ 0xFFFFFFFF, u ^ 0x80000000)


def _check(ps, keys, vals, kt, w):
    n = keys.size
    ref = oracle.powersort(keys, vals, kt=kt, min_run=w)
    dk = _dev(keys)
    an = ps.ps_analyze(dk, key_type=KT[kt], min_run=w)
    assert an["runs"] == ref.r and an["cost"] == ref.cost
    np.testing.assert_array_equal(an["starts"], ref.starts)
    np.testing.assert_array_equal(an["desc"] & 1, ref.desc)
    np.testing.assert_array_equal(an["leaf_depth"].astype(np.int32), ref.leaf_depth)
    if n <= 300000:
        _extended_ok(_order_keys(keys, kt), an["starts"], an["desc"], w, np.full(max(ref.r, 1), n))
    dv = _dev(vals)
    ws = torch.empty(ps.ps_workspace_size(KT[kt], True, n), dtype=torch.uint8, device="cuda")
    ps.ps_sort_minrun_ws(dk, dv, ws, w, key_type=KT[kt])
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)


def _case(name, n, seed):
    if name == "short_runs":
        return workloads.runs_i32(n, seed=seed, max_len=40), "i32"
    if name == "perm":
        return workloads.perm_i32(n, seed=seed), "i32"
    if name == "random_runs":
        return workloads.random_runs_i32(n, seed=seed, mean_len=30), "i32"
    if name == "pareto_u64":
        return workloads.pareto_u64(n, seed=seed, alpha=1.2, distinct=30, max_len=5000), "u64"
    if name == "f32":
        return workloads.pareto_f32(n, seed=seed), "f32"
    if name == "few_values_u32":
        rng = np.random.default_rng(seed)
        return (rng.integers(0, 4, n).astype(np.uint32), np.arange(n, dtype=np.uint32)), "u32"
    raise ValueError(name)


@pytest.mark.parametrize("w", [2, 3, 7, 24, 32])
@pytest.mark.parametrize("name", ["short_runs", "perm", "random_runs", "pareto_u64", "f32", "few_values_u32"])
def test_minrun_parity(ps, name, w):
    (keys, vals), kt = _case(name, 100003 + 7 * w, seed=w)
    _check(ps, keys, vals, kt, w)


@pytest.mark.parametrize("n", [1, 2, 3, 23, 24, 25, 31, 32, 33, 63, 64, 65, 8191, 8192, 8193, 8192 * 3 + 17])
def test_minrun_small_and_tile_edges(ps, n):
    rng = np.random.default_rng(n)
    for w in (3, 24, 32):
        keys = rng.integers(-3, 3, n).astype(np.int32)
        _check(ps, keys, np.arange(n, dtype=np.uint32), "i32", w)


@pytest.mark.parametrize("n,name", [(2 ** 21 + 5, "perm"), (3 * 2 ** 21 + 12345, "random_runs"),
                                    (2 ** 22, "short_runs")])
def test_minrun_several_tile_groups(ps, n, name):
    """More than 256 detection tiles: the group tables and the walk over groups are exercised."""
    (keys, vals), kt = _case(name, n, seed=5)
    _check(ps, keys, vals, kt, 24)


def test_minrun_one_is_the_greedy_partition(ps):
    keys, vals = workloads.runs_i32(200001, seed=9, max_len=60)
    dk = _dev(keys)
    a = ps.ps_analyze(dk, key_type=0)
    b = ps.ps_analyze(dk, key_type=0, min_run=1)
    for k in ("starts", "desc", "power", "leaf_depth"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["cost"] == b["cost"]


def test_minrun_argument_errors(ps):
    keys, vals = workloads.runs_i32(1000, seed=1)
    dk, dv = _dev(keys), _dev(vals)
    ws = torch.empty(ps.ps_workspace_size(0, True, 1000), dtype=torch.uint8, device="cuda")
    for w in (0, 33, -1):
        with pytest.raises(ps.PowersortError) as e:
            ps.ps_sort_minrun_ws(dk, dv, ws, w, key_type=0)
        assert e.value.status == 1
    np.testing.assert_array_equal(dk.cpu().numpy(), keys)


@pytest.mark.parametrize("w", [3, 24, 32])
def test_minrun_segmented(ps, w):
    """Segments sorted on their own: every segment's runs are the oracle's for that segment
    (extensions stop at the segment's end)."""
    rng = np.random.default_rng(w)
    sizes = [0, 1, 2, 3, w - 1, w, w + 1, 0, 31, 32, 33, 64, 65, 0, 8193]
    sizes += [int(x) for x in rng.integers(0, 6000, 120)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    keys = np.concatenate([workloads.runs_i32(max(s, 1), seed=i, max_len=int(rng.integers(2, 80)))[0][:s]
                           for i, s in enumerate(sizes)]).astype(np.int32)
    vals = np.arange(n, dtype=np.uint32)
    exp_k, exp_v, exp_s, exp_d, exp_ld, cost, ends = [], [], [], [], [], 0, []
    for i in range(len(sizes)):
        a, b = int(off[i]), int(off[i + 1])
        if a == b:
            continue
        ref = oracle.powersort(keys[a:b], vals[a:b], min_run=w)
        exp_k.append(ref.keys)
        exp_v.append(ref.vals)
        exp_s.append(ref.starts[:-1] + a)
        exp_d.append(ref.desc)
        exp_ld.append(ref.leaf_depth)
        ends.append(np.full(ref.r, b))
        cost += ref.cost
    exp_s = np.concatenate(exp_s + [np.array([n])])
    doff = torch.from_numpy(off).cuda()
    dk, dv = _dev(keys), _dev(vals)
    an = ps.ps_analyze(dk, offsets=doff, key_type=0, min_run=w)
    np.testing.assert_array_equal(an["starts"], exp_s)
    np.testing.assert_array_equal(an["desc"] & 1, np.concatenate(exp_d))
    np.testing.assert_array_equal(an["leaf_depth"].astype(np.int32), np.concatenate(exp_ld))
    assert an["cost"] == cost
    _extended_ok(keys, an["starts"], an["desc"], w, np.concatenate(ends))
    ws = torch.empty(ps.ps_workspace_size(0, True, n, True), dtype=torch.uint8, device="cuda")
    ps.ps_sort_minrun_ws(dk, dv, ws, w, offsets=doff, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), np.concatenate(exp_k))
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), np.concatenate(exp_v))


def test_paper_random_runs_minrun_24(ps):
    """Sec. 5.1's random-runs input (n = 10^7, geometric run lengths with mean 3000) with the
    paper's w = 24: GPU = oracle bit for bit, and the merge cost is the paper's printed average
    1.14e8 within 3%."""
    keys, vals = workloads.random_runs_i32(10 ** 7, seed=1, mean_len=3000)
    ref = oracle.powersort(keys, vals, min_run=24)
    dk, dv = _dev(keys), _dev(vals)
    an = ps.ps_analyze(dk, key_type=0, min_run=24)
    assert an["cost"] == ref.cost and abs(an["cost"] / 1.14e8 - 1) < 0.03
    np.testing.assert_array_equal(an["starts"], ref.starts)
    ws = torch.empty(ps.ps_workspace_size(0, True, keys.size), dtype=torch.uint8, device="cuda")
    ps.ps_sort_minrun_ws(dk, dv, ws, 24, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)


def test_full_random_permutation_minrun_24(ps):
    """n = 1e8 random permutation (the non-adaptive benchmark input) with w = 24."""
    keys, vals = workloads.perm_i32(10 ** 8, seed=7)
    _check(ps, keys, vals, "i32", 24)
