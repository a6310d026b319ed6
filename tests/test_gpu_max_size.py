"""The largest array one call accepts: n = 2^31 - 1 int32 keys with uint32 payloads (runs
uniform in [1, 2 sqrt(n)], 25% descending).  Index arithmetic near 2^31 (the last detection
thread, the last leaf tiles, the last level-pass tile and its 16-byte widened copies) is
exercised; the result is checked by properties that together fix the stable sort uniquely:
sorted keys, each output key is the input key its payload names, every payload appears once,
and equal keys keep payload order.  n = 2^31 is rejected with PS_ERR_UNSUPPORTED."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_1805_04154_gb300 as ps
    from paper_1805_04154_gb300 import _build
    _build.build()
    ps.load()
    return ps


def test_max_size_2p31_minus_1(ps):
    n = (1 << 31) - 1
    free, _ = torch.cuda.mem_get_info()
    if free < (120 << 30):
        pytest.skip("needs about 120 GB of free device memory")
    keys, vals = workloads.runs_i32(n, seed=31, max_len=2 * int(n ** 0.5))
    dk = torch.from_numpy(keys).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    del keys, vals
    orig = dk.clone()
    ws = torch.empty(ps.ps_workspace_size(0, True, n), dtype=torch.uint8, device="cuda")
    ps.ps_sort_ws(dk, dv, ws, key_type=0)
    assert ps.ps_stream_status() == 0
    del ws
    torch.cuda.empty_cache()
    assert bool((dk[1:] >= dk[:-1]).all())
    idx = dv.to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(dk, orig[idx])
    del orig
    seen = torch.zeros(n, dtype=torch.bool, device="cuda")
    seen[idx] = True
    assert bool(seen.all())
    del seen
    eq = dk[1:] == dk[:-1]
    assert bool(((idx[1:] > idx[:-1]) | ~eq).all())


def test_size_limit_rejected(ps):
    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    lib = ps.load()
    # the element count alone decides: nothing is read or written
    st = lib.ps_sort_ws(0, t.data_ptr(), None, 1 << 31, ws.data_ptr(), ws.numel(), None)
    assert st == 2  # PS_ERR_UNSUPPORTED
