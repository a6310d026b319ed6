"""GPU parity of the device-driven entry point (ps_sort_async_ws: no host round trip, every
launch sized from the plan on the device) against the CPU oracle, its device-side error path,
and CUDA-graph capture: one captured sort replayed on new inputs in the same buffers gives the
oracle's result every time (one array and many segments)."""
import os

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


def _dev(a):
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def _ws(ps, kt, n, seg=False, tree=0):
    return torch.empty(ps.ps_workspace_size(kt, True, n, seg, tree), dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("case", ["runs", "perm", "u64", "f32", "tiny", "peek"])
def test_async_matches_oracle(ps, case):
    tree, kt, ktn = 0, 0, "i32"
    if case == "runs":
        keys, vals = workloads.runs_i32(400001, seed=1, max_len=3000)
    elif case == "perm":
        keys, vals = workloads.perm_i32(1 << 18, seed=2)
    elif case == "u64":
        keys, vals = workloads.pareto_u64(1 << 19, seed=3)
        kt, ktn = 2, "u64"
    elif case == "f32":
        keys, vals = workloads.pareto_f32(1 << 18, seed=4)
        kt, ktn = 3, "f32"
    elif case == "tiny":
        keys, vals = workloads.runs_i32(5, seed=5, max_len=3)
    else:
        keys, vals = workloads.runs_i32(300001, seed=6, max_len=900)
        tree = 1
    ref = oracle.powersort(keys, vals, kt=ktn)
    dk, dv = _dev(keys), _dev(vals)
    ps.ps_sort_async_ws(dk, dv, _ws(ps, kt, keys.size, False, tree), tree=tree, key_type=kt)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)


def test_async_segmented_and_bad_offsets(ps):
    keys, vals, off = workloads.segmented_i32(300, seed=7, lo_exp=0, hi_exp=15)
    ref = oracle.sort_segmented(keys, vals, off)
    dk, dv, doff = _dev(keys), _dev(vals), torch.from_numpy(off).cuda()
    ps.ps_sort_async_ws(dk, dv, _ws(ps, 0, keys.size, True), offsets=doff, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref[1])
    # offsets that decrease: found on the device, reported by ps_stream_status, nothing moves
    k2, v2 = workloads.runs_i32(1000, seed=8)
    dk, dv = _dev(k2), _dev(v2)
    before = dk.clone()
    bad = torch.tensor([0, 600, 400, 1000], dtype=torch.int64, device="cuda")
    ps.ps_sort_async_ws(dk, dv, _ws(ps, 0, 1000, True), offsets=bad, key_type=0)
    assert ps.ps_stream_status() == 1
    assert torch.equal(dk, before)
    assert ps.ps_stream_status() == 0  # the status word was read and cleared


def test_cuda_graph_capture_and_replay(ps):
    n = 250003
    dk = torch.empty(n, dtype=torch.int32, device="cuda")
    dv = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = _ws(ps, 0, n)
    keys0, vals0 = workloads.runs_i32(n, seed=10, max_len=1000)
    dk.copy_(_dev(keys0))
    dv.copy_(_dev(vals0))
    ps.ps_sort_async_ws(dk, dv, ws, key_type=0)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ps.ps_sort_async_ws(dk, dv, ws, key_type=0)
    for seed in (11, 12, 13):
        keys, vals = workloads.runs_i32(n, seed=seed, max_len=int(2 * np.sqrt(n)))
        dk.copy_(_dev(keys))
        dv.copy_(_dev(vals))
        g.replay()
        torch.cuda.synchronize()
        assert ps.ps_stream_status() == 0
        ref = oracle.powersort(keys, vals)
        np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
        np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)


def test_cuda_graph_segmented_replay(ps):
    keys, vals, off = workloads.segmented_i32(500, seed=14, lo_exp=4, hi_exp=14)
    n = keys.size
    dk, dv, doff = _dev(keys), _dev(vals), torch.from_numpy(off).cuda()
    ws = _ws(ps, 0, n, True)
    ps.ps_sort_async_ws(dk, dv, ws, offsets=doff, key_type=0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ps.ps_sort_async_ws(dk, dv, ws, offsets=doff, key_type=0)
    rng = np.random.default_rng(15)
    for _ in range(2):
        # new keys with the same segment layout
        k2 = rng.integers(-1000, 1000, size=n, dtype=np.int32)
        v2 = np.arange(n, dtype=np.uint32)
        dk.copy_(_dev(k2))
        dv.copy_(_dev(v2))
        g.replay()
        torch.cuda.synchronize()
        assert ps.ps_stream_status() == 0
        ref = oracle.sort_segmented(k2, v2, off)
        np.testing.assert_array_equal(dk.cpu().numpy(), ref[0])
        np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref[1])


CHILD_OVERFLOW = r"""
import sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle, workloads
import paper_1805_04154_gb300 as ps
ps.load()
keys, vals = workloads.perm_i32(300001, seed=5)
ref = oracle.powersort(keys, vals)
dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals.view(np.int32)).cuda()
ws = torch.empty(ps.ps_workspace_size(0, True, keys.size), dtype=torch.uint8, device="cuda")
ps.ps_sort_async_ws(dk, dv, ws, key_type=0)
assert ps.ps_stream_status() == 0
assert np.array_equal(dk.cpu().numpy(), ref.keys) and np.array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
k2, v2, off = workloads.segmented_i32(400, seed=6, lo_exp=0, hi_exp=14)
ref2 = oracle.sort_segmented(k2, v2, off)
dk, dv = torch.from_numpy(k2).cuda(), torch.from_numpy(v2.view(np.int32)).cuda()
ws = torch.empty(ps.ps_workspace_size(0, True, k2.size, True), dtype=torch.uint8, device="cuda")
ps.ps_sort_async_ws(dk, dv, ws, offsets=torch.from_numpy(off).cuda(), key_type=0)
assert ps.ps_stream_status() == 0
assert np.array_equal(dk.cpu().numpy(), ref2[0]) and np.array_equal(dv.cpu().numpy().view(np.uint32), ref2[1])
print("overflow path ok")
"""


def test_device_driven_tasks_beyond_the_one_task_grid():
    """The device-driven call launches one CTA per subtree task up to a bound the host computes
    without the plan; tasks beyond it go to a persistent kernel.  A child process caps the
    one-task grid at 7 CTAs (PS_SUBTREE_GRID, a test setting) so that the persistent kernel
    takes almost all tasks of a permutation and of a batch of segments; both equal the oracle."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PS_SUBTREE_GRID="7")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % root + CHILD_OVERFLOW], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "overflow path ok" in r.stdout


def _comb(lengths, seed):
    """int32 keys made of ascending runs of the given lengths (random values), uint32 index payload."""
    rng = np.random.default_rng(seed)
    parts = [np.sort(rng.integers(-(1 << 31), 1 << 31, size=int(m), dtype=np.int64)).astype(np.int32) for m in lengths]
    keys = np.concatenate(parts)
    return keys, np.arange(keys.size, dtype=np.uint32)


@pytest.mark.parametrize("order", ["halving", "doubling", "nested"])
def test_async_deep_trees_of_large_nodes(ps, order):
    """Merge trees whose nodes larger than the subtree limit reach the greatest depth the
    device-driven entry launches level passes for (a node of power p spans fewer than 4n/2^p
    elements): halving and doubling run lengths, and a large run between two such combs.  A bound
    that stopped too shallow would leave the deepest merges undone."""
    halving = [1 << k for k in range(21, 11, -1)] + [4096] * 8
    if order == "halving":
        lengths = halving
    elif order == "doubling":
        lengths = halving[::-1]
    else:
        lengths = halving[::-1] + [1 << 22] + halving
    keys, vals = _comb(lengths, seed=len(lengths))
    n = keys.size
    ref = oracle.powersort(keys, vals)
    _, depth, power = oracle.powersort_cost(np.array(lengths, np.int64))
    dk, dv = _dev(keys), _dev(vals)
    ps.ps_sort_async_ws(dk, dv, _ws(ps, 0, n), key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
    # the input does reach deep: a leaf larger than the subtree limit at depth >= 8
    big = np.array(lengths) > 4096
    assert depth[big].max() >= 8


def test_bounded_entry_matches_oracle_and_checks_its_bound(ps):
    """ps_sort_async_bounded_ws: the caller's bound on the longest segment trims the level-pass
    launches and gives the oracle's result; a segment longer than the bound is rejected on the
    device (nothing moves); a single array longer than the bound is an argument error; a CUDA
    graph of the bounded call replays to the oracle's result."""
    keys, vals, off = workloads.segmented_i32(400, seed=21, lo_exp=6, hi_exp=17)
    longest = int(np.diff(off).max())
    ref = oracle.sort_segmented(keys, vals, off)
    n = keys.size
    ws = _ws(ps, 0, n, True)
    dk, dv, doff = _dev(keys), _dev(vals), torch.from_numpy(off).cuda()
    before = ps.ps_launch_count()
    ps.ps_sort_async_bounded_ws(dk, dv, ws, longest, offsets=doff, key_type=0)
    bounded_launches = ps.ps_launch_count() - before
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref[1])
    dk, dv = _dev(keys), _dev(vals)
    before = ps.ps_launch_count()
    ps.ps_sort_async_ws(dk, dv, ws, offsets=doff, key_type=0)
    assert ps.ps_launch_count() - before > bounded_launches  # fewer level passes queued
    assert ps.ps_stream_status() == 0
    # a bound one element short of the longest segment: rejected on the device, nothing moves
    dk, dv = _dev(keys), _dev(vals)
    orig = dk.clone()
    ps.ps_sort_async_bounded_ws(dk, dv, ws, longest - 1, offsets=doff, key_type=0)
    assert ps.ps_stream_status() == 1
    assert torch.equal(dk, orig)
    assert ps.ps_stream_status() == 0
    # one array: the bound is checked on the host
    k1, v1 = workloads.runs_i32(5000, seed=22, max_len=200)
    with pytest.raises(ps.PowersortError):
        ps.ps_sort_async_bounded_ws(_dev(k1), _dev(v1), _ws(ps, 0, 5000), 4999, key_type=0)
    # captured and replayed on new keys in the same segment layout
    dk, dv = _dev(keys), _dev(vals)
    ps.ps_sort_async_bounded_ws(dk, dv, ws, longest, offsets=doff, key_type=0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ps.ps_sort_async_bounded_ws(dk, dv, ws, longest, offsets=doff, key_type=0)
    rng = np.random.default_rng(23)
    k2 = rng.integers(-5000, 5000, size=n, dtype=np.int32)
    v2 = np.arange(n, dtype=np.uint32)
    dk.copy_(_dev(k2))
    dv.copy_(_dev(v2))
    g.replay()
    torch.cuda.synchronize()
    assert ps.ps_stream_status() == 0
    ref2 = oracle.sort_segmented(k2, v2, off)
    np.testing.assert_array_equal(dk.cpu().numpy(), ref2[0])
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref2[1])
