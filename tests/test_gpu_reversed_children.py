"""Large strictly descending runs that are leaves of even depth >= 2 are not reversed by leaf
placement: their parent (a merge of odd depth, done by a level pass) reads them backwards
(Sec. 2 run convention: a descending run is a reversed ascending one).

Checked on inputs made mostly of long descending runs: the output equals the oracle's bit for bit
(keys and payloads), such leaves really occur, and the placement stage's algorithmic bytes equal
exactly the leaves it still has to move -- large leaves of odd depth (copied to the scratch
buffer) and descending leaves that are a whole array (reversed in place) -- and nothing for the
leaves that are read backwards."""
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


def _desc_runs(values: np.ndarray, seed: int, max_len: int) -> np.ndarray:
    """values cut into runs of length uniform in [1, max_len], each sorted descending."""
    rng = np.random.default_rng(seed)
    out = values.copy()
    pos = 0
    while pos < out.size:
        m = min(int(rng.integers(1, max_len + 1)), out.size - pos)
        out[pos:pos + m] = np.sort(out[pos:pos + m])[::-1]
        pos += m
    return out


def _input(kt: str, n: int, seed: int):
    vals = np.arange(n, dtype=np.uint32)
    if kt == "i32":
        keys, _ = workloads.runs_i32(n, seed, max_len=60000, desc_frac=1.0)
        return keys, vals
    rng = np.random.default_rng(seed)
    if kt == "u64":  # distinct with overwhelming probability: no run splits at ties
        return _desc_runs(rng.integers(0, np.iinfo(np.uint64).max, n, dtype=np.uint64, endpoint=True), seed,
                          60000), vals
    # float32 of both signs, no zeros or NaNs: value order is IEEE totalOrder here
    f = rng.standard_normal(n).astype(np.float32)
    f[f == 0] = 1.0
    return _desc_runs(f, seed, 60000).view(np.uint32), vals


@pytest.mark.parametrize("kt,seed,with_vals", [("i32", 1, True), ("i32", 2, False), ("u64", 3, True),
                                               ("f32", 4, True)])
def test_descending_leaves_read_backwards(ps, kt, seed, with_vals):
    n = 3_000_001
    keys, vals = _input(kt, n, seed)
    if not with_vals:
        vals = None
    ref = oracle.powersort(keys, vals, kt=kt)
    kb = keys.dtype.itemsize
    sub_lim = 4096 if kb == 4 else 2048
    eb = kb + (4 if with_vals else 0)
    lengths = np.diff(ref.starts)
    depth = ref.leaf_depth
    large = lengths > sub_lim
    backwards = large & (ref.desc == 1) & (depth >= 2) & (depth % 2 == 0)
    assert backwards.sum() >= 3, "the input must have large descending leaves of even depth"
    moved = lengths[large & (depth % 2 == 1)].sum() + 2 * (lengths[large & (ref.desc == 1) & (depth == 0)] // 2).sum()

    dk = _dev(keys)
    dv = None if vals is None else _dev(vals)
    ws = torch.empty(ps.ps_workspace_size(KT[kt], with_vals, n), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    ps.ps_profile_enable(True)
    ps.ps_sort_ws(dk, dv, ws, key_type=KT[kt])
    torch.cuda.synchronize()
    prof = ps.ps_profile_read()
    ps.ps_profile_enable(False)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy().view(keys.dtype), ref.keys)
    if vals is not None:
        np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
    assert prof["leaf_place"]["bytes"] == 2 * eb * int(moved)


def test_descending_whole_array_and_device_driven(ps):
    """A single descending run (depth 0, no merge above it) is still reversed in place, and the
    device-driven entry (no host round trip) reads descending leaves backwards as well."""
    n = 1_000_003
    keys = np.arange(n, 0, -1, dtype=np.int32)
    vals = np.arange(n, dtype=np.uint32)
    ref = oracle.powersort(keys, vals)
    dk, dv = _dev(keys), _dev(vals)
    ps.ps_sort(dk, dv, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)

    keys, vals = workloads.runs_i32(n, 9, max_len=40000, desc_frac=1.0)
    ref = oracle.powersort(keys, vals)
    dk, dv = _dev(keys), _dev(vals)
    ws = torch.empty(ps.ps_workspace_size(0, True, n), dtype=torch.uint8, device="cuda")
    ps.ps_sort_async_ws(dk, dv, ws, key_type=0)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)
