"""Every level-pass configuration the library carries (items per thread x ring stages) gives the
oracle's result bit for bit, and the autotuner times them all and keeps one."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

VARIANTS = [(12, 2), (12, 3), (12, 4), (8, 2), (8, 3), (16, 2), (6, 2), (10, 2)]


@pytest.fixture(scope="module")
def ps():
    import paper_1805_04154_gb300 as ps
    from paper_1805_04154_gb300 import _build
    _build.build()
    ps.load()
    yield ps
    for kt in range(4):
        for v in (False, True):
            ps.ps_tune_set(kt, v, 0, 0)


@pytest.mark.parametrize("ipt,stages", VARIANTS)
def test_each_configuration_matches_oracle(ps, ipt, stages):
    for kt, ktn, gen in ((0, "i32", lambda: workloads.runs_i32(600001, seed=ipt * 10 + stages, max_len=9000)),
                         (2, "u64", lambda: workloads.pareto_u64(1 << 19, seed=stages, distinct=300))):
        keys, vals = gen()
        ps.ps_tune_set(kt, True, ipt, stages)
        ps.ps_tune_set(kt, False, ipt, stages)
        ref = oracle.powersort(keys, vals, kt=ktn)
        dk = torch.from_numpy(keys.view(np.int64) if kt == 2 else keys).cuda()
        dv = torch.from_numpy(vals.view(np.int32)).cuda()
        ps.ps_sort(dk, dv, key_type=kt)
        assert ps.ps_stream_status() == 0
        np.testing.assert_array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys)
        np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
        dk = torch.from_numpy(keys.view(np.int64) if kt == 2 else keys).cuda()
        ps.ps_sort(dk, None, key_type=kt)
        np.testing.assert_array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys)
        ps.ps_tune_set(kt, True, 0, 0)
        ps.ps_tune_set(kt, False, 0, 0)


def test_autotune_picks_a_configuration(ps):
    keys, vals = workloads.runs_i32(1 << 21, seed=3, max_len=3000)
    dk = torch.from_numpy(keys).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    before_k, before_v = dk.clone(), dv.clone()
    res = ps.ps_autotune(dk, dv, key_type=0)
    assert [(v["items_per_thread"], v["stages"]) for v in res["variants"]] == VARIANTS
    assert all(v["ms"] > 0 for v in res["variants"])
    best = min(res["variants"], key=lambda v: v["ms"])
    assert (res["items_per_thread"], res["stages"]) == (best["items_per_thread"], best["stages"])
    # the tuned entry belongs to plain sorts of this size bucket (2^20 <= n < 2^24)
    assert ps.ps_tune_get_for(0, True, keys.size) == (res["items_per_thread"], res["stages"])
    assert torch.equal(dk, before_k) and torch.equal(dv, before_v)  # the input is left alone
    ps.ps_sort(dk, dv, key_type=0)
    ref = oracle.powersort(keys, vals)
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)


def test_tuned_entries_by_kind_and_size_bucket(ps):
    """ps_autotune_segmented times the segmented sort of a batch and keeps its choice for segmented
    sorts of that size bucket only; ps_tune_set sets the default and clears the tuned entries."""
    ps.ps_tune_set(0, True, 12, 3)  # a default that differs from the tuned entries below
    keys, vals, off = workloads.segmented_i32(300, seed=12, lo_exp=8, hi_exp=15)
    dk = torch.from_numpy(keys).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    doff = torch.from_numpy(off).cuda()
    res = ps.ps_autotune_segmented(dk, dv, doff, key_type=0)
    assert len(res["variants"]) == len(VARIANTS)
    best = min(res["variants"], key=lambda v: v["ms"])
    choice = (res["items_per_thread"], res["stages"])
    assert choice == (best["items_per_thread"], best["stages"])
    assert ps.ps_tune_get_for(0, True, keys.size, segmented=True) == choice
    assert ps.ps_tune_get_for(0, True, keys.size, segmented=False) == (12, 3)  # plain: the default
    assert ps.ps_tune_get_for(0, True, 1 << 26, segmented=True) == (12, 3)    # another bucket
    ref = oracle.sort_segmented(keys, vals, off)
    ps.ps_sort_segmented(dk, dv, doff, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref[1])
    ps.ps_tune_set(0, True, 0, 0)
    assert ps.ps_tune_get_for(0, True, keys.size, segmented=True) == (8, 2)


def test_autotune_u64_times_every_configuration(ps):
    """The autotuner times all eight configurations on 8-byte keys too, and the tuned sort equals
    the oracle."""
    keys, vals = workloads.pareto_u64(1 << 20, seed=5, distinct=1000)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    res = ps.ps_autotune(dk, dv, key_type=2)
    assert [(v["items_per_thread"], v["stages"]) for v in res["variants"]] == VARIANTS
    assert ps.ps_tune_get_for(2, True, keys.size) == (res["items_per_thread"], res["stages"])
    ps.ps_sort(dk, dv, key_type=2)
    ref = oracle.powersort(keys, vals, kt="u64")
    np.testing.assert_array_equal(dk.cpu().numpy().view(np.uint64), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
    ps.ps_tune_set(2, True, 0, 0)
