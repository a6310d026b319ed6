"""Arrays of 2^31 elements and more: unsigned 32-bit element positions with 64-bit addresses, and
node powers formed from 64-bit products (Definition "Node Power"; Appendix B's implementation
note: its int form of the power overflows for large n).

n = 2^31 + 3 * 2^20 + 17 int32 keys with uint32 payloads, made of runs uniform in
[1, 2 sqrt(n)] (25% descending) with a 2^20-element random permutation embedded, whose runs of
two or three elements give boundaries of the largest powers (30 and 31 here: powers above 31
would need two adjacent runs shorter than n / 2^30 in total).  The plan -- run starts,
directions, node powers, leaf depths, merge cost -- equals the oracle's (its run detection and
its powersort tree on the run lengths, exact 128-bit powers), and the sorted
output is checked by properties that together fix the stable sort uniquely: sorted keys, each
output key is the input key its payload names, every payload appears once, and equal keys keep
payload order.  n = 2^32 is rejected with PS_ERR_UNSUPPORTED before anything is read."""
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


def _input(n: int, seed: int):
    keys, vals = workloads.runs_i32(n, seed=seed, max_len=2 * int(n ** 0.5))
    perm, _ = workloads.perm_i32(1 << 20, seed=seed + 1)
    at = (1 << 30) + 12345
    keys[at:at + perm.size] = perm * 2047  # spread over the int32 range; distinct
    return keys, vals


def test_beyond_2p31_elements(ps):
    n = (1 << 31) + 3 * (1 << 20) + 17
    free, _ = torch.cuda.mem_get_info()
    if free < (110 << 30):
        pytest.skip("needs about 110 GB of free device memory")
    keys, vals = _input(n, seed=31)
    starts, desc = oracle.detect_runs(keys, "i32")
    lengths = np.diff(starts)
    cost, depth, power = oracle.powersort_cost(lengths)
    assert power.max() >= 31, "the input must reach the largest node powers of its size"

    dk = torch.from_numpy(keys).cuda()
    an = ps.ps_analyze(dk, key_type=0)
    assert an["runs"] == lengths.size and an["cost"] == cost
    assert np.array_equal(an["starts"], starts)
    assert np.array_equal(an["desc"], desc)
    assert np.array_equal(an["power"].astype(np.int32), power)
    assert np.array_equal(an["leaf_depth"].astype(np.int32), depth)
    del an, starts, desc, lengths, depth, power
    torch.cuda.empty_cache()

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
    del dv
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
    st = lib.ps_sort_ws(0, t.data_ptr(), None, 1 << 32, ws.data_ptr(), ws.numel(), None)
    assert st == 2  # PS_ERR_UNSUPPORTED
