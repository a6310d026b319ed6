"""GPU parity at the benchmark's full sizes, in the same launch configuration bench.py times
(ps_sort_ws with a workspace from PyTorch's allocator).

n = 1e8 single arrays are compared with the CPU oracle element by element (the oracle sorts
them in seconds).  The 10,000-segment batched input (about 1.23e9 keys) is checked on the
device by properties that together determine the stable sort uniquely -- every segment is
sorted, every output element is the input element its payload names, each payload index appears
once and stays in its segment, and equal keys keep payload order -- and then compared with the
oracle's segmented sort element by element, together with its whole segmented plan."""
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


def _dev(a: np.ndarray) -> torch.Tensor:
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def _sort_and_compare(ps, keys, vals, kt_name, kt):
    ref = oracle.powersort(keys, vals, kt=kt_name)
    dk, dv = _dev(keys), _dev(vals)
    an = ps.ps_analyze(dk, key_type=kt)
    ws = torch.empty(ps.ps_workspace_size(kt, True, keys.size), dtype=torch.uint8, device="cuda")
    ps.ps_sort_ws(dk, dv, ws, key_type=kt)
    assert ps.ps_stream_status() == 0
    assert an["runs"] == ref.r and an["cost"] == ref.cost
    assert np.array_equal(an["starts"], ref.starts)
    assert np.array_equal(an["leaf_depth"].astype(np.int32), ref.leaf_depth)
    assert np.array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys)
    assert np.array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)


def test_full_runs_i32_1e8(ps):
    """n = 1e8 int32 + uint32, runs uniform in [1, 20000], 25% descending (the benchmark)."""
    keys, vals = workloads.runs_i32(10 ** 8, seed=42, max_len=20000)
    _sort_and_compare(ps, keys, vals, "i32", 0)


def test_full_random_permutation_1e8(ps):
    """The non-adaptive limit: a random permutation of 1e8 int32 keys (runs of about 2.4)."""
    keys, vals = workloads.perm_i32(10 ** 8, seed=7)
    _sort_and_compare(ps, keys, vals, "i32", 0)


def test_full_pareto_u64_1e8(ps):
    """Stability stress: 1e8 uint64 keys from 1000 distinct values, Pareto(1.2) runs."""
    keys, vals = workloads.pareto_u64(10 ** 8, seed=3, alpha=1.2, distinct=1000, max_len=10 ** 7)
    _sort_and_compare(ps, keys, vals, "u64", 2)


def test_full_segmented_10k(ps):
    """10,000 int32 arrays, sizes floor(2^U(8,20)), runs uniform in [1, 2 sqrt(size)]."""
    keys, vals, off = workloads.segmented_i32(10000, seed=5)
    n = keys.size
    dk, dv = _dev(keys), _dev(vals)
    doff = torch.from_numpy(off).cuda()
    ws = torch.empty(ps.ps_workspace_size(0, True, n, True), dtype=torch.uint8, device="cuda")
    ps.ps_sort_segmented_ws(dk, dv, doff, ws, key_type=0)
    assert ps.ps_stream_status() == 0
    orig = _dev(keys)
    del ws
    # segment of every position
    pos = torch.arange(n, device="cuda", dtype=torch.int64)
    seg = torch.searchsorted(doff[1:], pos, right=True)
    idx = dv.to(torch.int64) & 0xFFFFFFFF
    # payload names an input element of the same segment, and each appears exactly once
    assert torch.equal(seg, torch.searchsorted(doff[1:], idx, right=True))
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    counts.index_add_(0, idx, torch.ones(n, dtype=torch.int32, device="cuda"))
    assert bool((counts == 1).all())
    del counts
    # every output element is the input element its payload names
    assert torch.equal(dk, orig[idx])
    # sorted within segments, and stable: equal neighbours keep payload order
    same = seg[1:] == seg[:-1]
    assert bool(((dk[1:] >= dk[:-1]) | ~same).all())
    eq = same & (dk[1:] == dk[:-1])
    assert bool(((idx[1:] > idx[:-1]) | ~eq).all())
    hk = dk.cpu().numpy()
    hv = dv.cpu().numpy().view(np.uint32)
    del dk, dv, orig, pos, seg, idx, same, eq
    # the whole batch against the oracle: every segment sorted by Alg. 2 on its own, element by
    # element, and the segmented plan (runs, directions, powers with 0 between segments, leaf
    # depths, merge cost) from ps_analyze with the same offsets
    ref = oracle.sort_segmented(keys, vals, off)
    assert np.array_equal(hk, ref[0]) and np.array_equal(hv, ref[1])
    del hk, hv
    an = ps.ps_analyze(_dev(keys), offsets=doff, key_type=0)
    assert an["runs"] == ref[2].size - 1
    assert np.array_equal(an["starts"], ref[2])
    assert np.array_equal(an["desc"], ref[3])
    assert np.array_equal(an["power"].astype(np.int32), ref[4])
    assert np.array_equal(an["leaf_depth"].astype(np.int32), ref[5])
    assert an["cost"] == ref[6]


@pytest.mark.parametrize("mean_len", [3000, 100000])
def test_paper_random_runs_1e7(ps, mean_len):
    """The paper's random-runs inputs (Sec. 5.1): n = 10^7, a random permutation whose segments
    of geometric length with mean 3000 (and 10^5) are sorted.  GPU = oracle bit for bit, and the
    merge cost is the oracle's (no minimal run length; the paper's printed 1.14e8 uses w = 24 and
    is pinned on the oracle side)."""
    keys, vals = workloads.random_runs_i32(10 ** 7, seed=1, mean_len=mean_len)
    _sort_and_compare(ps, keys, vals, "i32", 0)
