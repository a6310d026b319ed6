"""The host-array pipeline (copy-in, device-driven sort, copy-out with several arrays in flight):
every array comes back as its stable sort, for arrays of different sizes (including empty and
one-element ones) and more arrays than buffer sets."""
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


def test_pipeline_many_arrays(ps):
    from paper_1805_04154_gb300.pipeline import HostSortPipeline
    sizes = [100003, 0, 1, 2, 77777, 100003, 5, 65536, 99999, 3]
    pipe = HostSortPipeline(max(sizes), torch.int32, True, depth=3)
    ins, outs = [], []
    for i, n in enumerate(sizes):
        k, v = workloads.runs_i32(max(n, 1), seed=100 + i, max_len=300)
        k, v = k[:n], v[:n]
        hk = torch.from_numpy(k.copy()).pin_memory()
        hv = torch.from_numpy(v.view(np.int32).copy()).pin_memory()
        ok = torch.empty_like(hk).pin_memory()
        ov = torch.empty_like(hv).pin_memory()
        pipe.submit(hk, hv, ok, ov)
        ins.append((k, v))
        outs.append((ok, ov))
    pipe.synchronize()
    torch.cuda.synchronize()
    for (k, v), (ok, ov) in zip(ins, outs):
        ref = oracle.powersort(k, v)
        np.testing.assert_array_equal(ok.numpy(), ref.keys)
        np.testing.assert_array_equal(ov.numpy().view(np.uint32), ref.vals)


def test_pipeline_in_place_keys_only(ps):
    from paper_1805_04154_gb300.pipeline import HostSortPipeline
    pipe = HostSortPipeline(50000, torch.int32, False, depth=2)
    arrays = [torch.from_numpy(workloads.perm_i32(50000 - 7 * i, seed=i)[0]).pin_memory() for i in range(5)]
    refs = [np.sort(a.numpy(), kind="stable") for a in arrays]
    for a in arrays:
        pipe.submit(a, None, a, None)  # output aliases the input
    pipe.synchronize()
    torch.cuda.synchronize()
    for a, r in zip(arrays, refs):
        np.testing.assert_array_equal(a.numpy(), r)
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros(60000, dtype=torch.int32), None, torch.zeros(60000, dtype=torch.int32), None)
