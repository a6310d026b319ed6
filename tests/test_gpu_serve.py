"""Continuous-batching server: each result equals the oracle's and is the same alone and in the
mix (bit-exact), with requests of mixed sizes arriving while earlier batches are on the GPU,
float32 keys with NaN/+-0 specials (IEEE totalOrder) and Pareto(1.5) runs, and a tight
device-memory budget."""
import threading
import time

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


def _requests(count, seed, lo_exp=10, hi_exp=18):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(2 ** rng.uniform(lo_exp, hi_exp))
        k, v = workloads.pareto_f32(n, seed=seed * 1000 + i, alpha=1.5, special_frac=0.01)
        out.append((k, v))
    return out


def _pinned(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(a.view(np.int32)).pin_memory()


def _alone(ps, k, v):
    dk = torch.from_numpy(k.view(np.int32)).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    ps.ps_sort(dk, dv, key_type=ps.PS_KEY_F32)
    torch.cuda.synchronize()
    return dk.cpu().numpy().view(np.uint32), dv.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("budget,slots", [(64 << 30, 3), (2 << 30, 1)])
def test_results_same_alone_and_in_mix(ps, budget, slots):
    from paper_1805_04154_gb300.serve import SortServer, latency_stats
    reqs = _requests(60, seed=slots)
    srv = SortServer(ps.PS_KEY_F32, budget_bytes=budget, max_batch_keys=1 << 20, slots=slots)
    handles = []
    try:
        # arrivals spread in time so that later requests join while earlier batches run; the
        # first half sorts in place, the second half into separate output tensors
        for i, (k, v) in enumerate(reqs):
            tk, tv = _pinned(k), _pinned(v)
            if i % 2:
                handles.append(srv.submit(tk, tv, torch.empty_like(tk).pin_memory(),
                                          torch.empty_like(tv).pin_memory()))
            else:
                handles.append(srv.submit(tk, tv))
            if i % 7 == 0:
                time.sleep(0.002)
        srv.drain(timeout=120)
    finally:
        srv.close()
    assert srv.batches >= 2
    # every request: the served result equals the oracle's powersort of that request alone, bit
    # for bit, and equals the same request sorted alone on the GPU
    for (k, v), h in zip(reqs, handles):
        assert h.error is None
        ref = oracle.powersort(k, v, kt="f32")
        assert np.array_equal(h.out_keys.numpy().view(np.uint32), ref.keys)
        assert np.array_equal(h.out_vals.numpy().view(np.uint32), ref.vals)
        ak, av = _alone(ps, k, v)
        assert np.array_equal(ak, ref.keys) and np.array_equal(av, ref.vals)
    st = latency_stats(handles)
    assert st["requests"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0


def test_budget_and_oversized_request(ps):
    from paper_1805_04154_gb300.serve import SortServer
    with pytest.raises(ValueError):
        SortServer(ps.PS_KEY_F32, budget_bytes=1 << 20, max_batch_keys=1 << 20)
    srv = SortServer(ps.PS_KEY_F32, budget_bytes=1 << 30, max_batch_keys=1 << 16, slots=2)
    try:
        k, v = workloads.pareto_f32((1 << 16) + 1, seed=3)
        with pytest.raises(ValueError):
            srv.submit(_pinned(k), _pinned(v))
    finally:
        srv.close()
