"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Sorting is exact, so every comparison is bit-exact: keys, payloads (hence the order of equal
keys), and the plan (run starts, directions, node powers, leaf depths, merge cost)."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

KT_NAME = {"i32": 0, "u32": 1, "u64": 2, "f32": 3}


@pytest.fixture(scope="module")
def ps():
    import paper_1805_04154_gb300 as ps
    from paper_1805_04154_gb300 import _build
    _build.build()
    ps.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return ps


def _to_dev(a: np.ndarray) -> torch.Tensor:
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def _gpu_sort(ps, keys: np.ndarray, vals: np.ndarray | None, kt: str, offsets=None):
    dk = _to_dev(keys)
    dv = None if vals is None else _to_dev(vals)
    if offsets is None:
        ps.ps_sort(dk, dv, key_type=KT_NAME[kt])
    else:
        ps.ps_sort_segmented(dk, dv, torch.from_numpy(np.asarray(offsets, np.int64)).cuda(),
                             key_type=KT_NAME[kt])
    assert ps.ps_stream_status() == 0
    k = dk.cpu().numpy().view(keys.dtype)
    v = None if dv is None else dv.cpu().numpy().view(np.uint32)
    return k, v


def _check_against_oracle(ps, keys, vals, kt):
    ref = oracle.powersort(keys, vals, kt=kt)
    k, v = _gpu_sort(ps, keys, vals, kt)
    np.testing.assert_array_equal(k, ref.keys)
    if vals is not None:
        np.testing.assert_array_equal(v, ref.vals)
    return ref


def _check_plan(ps, keys, kt, ref):
    an = ps.ps_analyze(_to_dev(keys), key_type=KT_NAME[kt])
    r = ref.r
    assert an["runs"] == r
    np.testing.assert_array_equal(an["starts"], ref.starts)
    np.testing.assert_array_equal(an["desc"], ref.desc)
    np.testing.assert_array_equal(an["power"].astype(np.int32), ref.power)
    np.testing.assert_array_equal(an["leaf_depth"].astype(np.int32), ref.leaf_depth)
    assert an["cost"] == ref.cost
    # node ranges: node j merges [S[L], S[j]) and [S[j], S[R]); its parent (Cartesian tree) is the
    # nearer of L and R, i.e. the one with the larger power
    for j in range(1, r):
        L, R = an["node_left"][j], an["node_right"][j]
        pl, pr = ref.power[L], ref.power[R]
        par = -1 if (pl == 0 and pr == 0) else (L if pl > pr else R)
        assert par == ref.node_parent[j]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_config_small_runs_i32(ps, seed):
    """n = 2^17 int32 + uint32 payload, runs uniform in [1, 2 sqrt(n)], 25% descending."""
    keys, vals = workloads.runs_i32(1 << 17, seed)
    ref = _check_against_oracle(ps, keys, vals, "i32")
    _check_plan(ps, keys, "i32", ref)


@pytest.mark.parametrize("n", [2, 3, 5, 17, 255, 4095, 4096, 4097, 8191, 12289, 65537, 300001])
def test_sizes_and_ragged_tails(ps, n):
    keys, vals = workloads.runs_i32(n, seed=n, max_len=max(2, int(2 * np.sqrt(n))))
    ref = _check_against_oracle(ps, keys, vals, "i32")
    _check_plan(ps, keys, "i32", ref)


@pytest.mark.parametrize("max_len", [1, 3, 64, 5000, 70000])
def test_run_length_regimes(ps, max_len):
    keys, vals = workloads.runs_i32(200000, seed=7, max_len=max_len)
    ref = _check_against_oracle(ps, keys, vals, "i32")
    _check_plan(ps, keys, "i32", ref)


def test_degenerate_inputs(ps):
    n = 100003
    cases = {
        "ascending": np.arange(n, dtype=np.int32),
        "descending": np.arange(n, 0, -1, dtype=np.int32),
        "all_equal": np.full(n, 7, dtype=np.int32),
        "zigzag": np.tile(np.array([0, 5], np.int32), n // 2 + 1)[:n],
        "down_zigzag": np.tile(np.array([5, 0], np.int32), n // 2 + 1)[:n],
        "two_values": (np.random.default_rng(0).integers(0, 2, n)).astype(np.int32),
        "sawtooth": (np.arange(n) % 4099).astype(np.int32),
        "desc_blocks": (-(np.arange(n) % 6007)).astype(np.int32),
    }
    for name, keys in cases.items():
        vals = np.arange(n, dtype=np.uint32)
        ref = _check_against_oracle(ps, keys, vals, "i32")
        _check_plan(ps, keys, "i32", ref)


def test_tiny_and_empty(ps):
    for n in (0, 1):
        keys = np.arange(n, dtype=np.int32)[::-1].copy()
        vals = np.arange(n, dtype=np.uint32)
        k, v = _gpu_sort(ps, keys, vals, "i32")
        np.testing.assert_array_equal(k, np.sort(keys))


def test_keys_only(ps):
    keys, _ = workloads.runs_i32(150001, seed=5)
    ref = oracle.powersort(keys, None)
    k, _ = _gpu_sort(ps, keys, None, "i32")
    np.testing.assert_array_equal(k, ref.keys)


def test_random_permutation(ps):
    keys, vals = workloads.perm_i32(1 << 18, seed=3)
    ref = _check_against_oracle(ps, keys, vals, "i32")
    _check_plan(ps, keys, "i32", ref)


def test_u32_keys(ps):
    keys, vals = workloads.runs_i32(1 << 17, seed=11, signed=False)
    ref = _check_against_oracle(ps, keys, vals, "u32")
    _check_plan(ps, keys, "u32", ref)


@pytest.mark.parametrize("seed", [1, 2])
def test_pareto_u64_dense_duplicates(ps, seed):
    """Stability stress: uint64 keys from 1000 distinct values, Pareto(1.2) run lengths."""
    keys, vals = workloads.pareto_u64(1 << 20, seed)
    ref = _check_against_oracle(ps, keys, vals, "u64")
    _check_plan(ps, keys, "u64", ref)


def test_u64_keys_only_and_sizes(ps):
    for n in (3, 2047, 2048, 2049, 40001):
        keys, vals = workloads.pareto_u64(n, seed=n, distinct=5)
        _check_against_oracle(ps, keys, vals, "u64")
        ref = oracle.powersort(keys, None, kt="u64")
        k, _ = _gpu_sort(ps, keys, None, "u64")
        np.testing.assert_array_equal(k, ref.keys)


def test_f32_total_order_with_specials(ps):
    keys, vals = workloads.pareto_f32(1 << 18, seed=4, special_frac=0.01)
    ref = _check_against_oracle(ps, keys, vals, "f32")
    _check_plan(ps, keys, "f32", ref)


def test_segmented_small(ps):
    keys, vals, off = workloads.segmented_i32(300, seed=6, lo_exp=0, hi_exp=15)
    off = off.copy()
    off[10] = off[9]  # empty segments
    off[11] = off[9]
    ref = oracle.sort_segmented(keys, vals, off)
    k, v = _gpu_sort(ps, keys, vals, "i32", offsets=off)
    np.testing.assert_array_equal(k, ref[0])
    np.testing.assert_array_equal(v, ref[1])
    an = ps.ps_analyze(_to_dev(keys), offsets=torch.from_numpy(off).cuda(), key_type=0)
    np.testing.assert_array_equal(an["starts"], ref[2])
    np.testing.assert_array_equal(an["desc"], ref[3])
    np.testing.assert_array_equal(an["power"].astype(np.int32), ref[4])
    np.testing.assert_array_equal(an["leaf_depth"].astype(np.int32), ref[5])
    assert an["cost"] == ref[6]


def test_segmented_bad_offsets_rejected(ps):
    keys, vals = workloads.runs_i32(1000, seed=1)
    dk, dv = _to_dev(keys), _to_dev(vals)
    before = dk.clone()
    off = torch.tensor([0, 600, 400, 1000], dtype=torch.int64, device="cuda")
    with pytest.raises(ps.PowersortError) as e:
        ps.ps_sort_segmented(dk, dv, off, key_type=0)
    assert e.value.status == 1
    assert torch.equal(dk, before)


def test_pool_entry_point_and_stats(ps):
    keys, vals = workloads.runs_i32(1 << 16, seed=21)
    ref = oracle.powersort(keys, vals)
    dk, dv = _to_dev(keys), _to_dev(vals)
    st = ps.ps_sort_stats(dk, key_type=0)
    assert st["runs"] == ref.r and st["merge_cost"] == ref.cost
    H = oracle.entropy_bits(np.diff(ref.starts))
    assert abs(st["entropy_bits"] - H) < 1e-3
    ps.ps_sort(dk, dv, key_type=0, pool=True)
    assert ps.ps_stream_status() == 0
    np.testing.assert_array_equal(dk.cpu().numpy(), ref.keys)
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), ref.vals)


@pytest.mark.parametrize("kt,off", [("i32", 1), ("i32", 3), ("u64", 1), ("f32", 2)])
def test_unaligned_subarray_views(ps, kt, off):
    """Sub-arrays at element offsets that are not 16-byte aligned: sorted bit-exactly, and the
    elements around the view are left untouched."""
    n = 70001
    if kt == "u64":
        keys, vals = workloads.pareto_u64(n, seed=off, distinct=50)
    elif kt == "f32":
        keys, vals = workloads.pareto_f32(n, seed=off)
    else:
        keys, vals = workloads.runs_i32(n, seed=off, max_len=900)
    ref = oracle.powersort(keys, vals, kt=kt)
    pad = np.zeros(off, dtype=keys.dtype)
    big_k = _to_dev(np.concatenate([pad, keys, pad]))
    big_v = _to_dev(np.concatenate([np.full(off, 7, np.uint32), vals, np.full(off, 9, np.uint32)]))
    dk, dv = big_k[off:off + n], big_v[off:off + n]
    ps.ps_sort(dk, dv, key_type=KT_NAME[kt])
    assert ps.ps_stream_status() == 0
    hk = big_k.cpu().numpy().view(keys.dtype)
    hv = big_v.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(hk[off:off + n], ref.keys)
    np.testing.assert_array_equal(hv[off:off + n], ref.vals)
    assert (hk[:off] == 0).all() and (hk[off + n:] == 0).all()
    assert (hv[:off] == 7).all() and (hv[off + n:] == 9).all()


def test_host_ws_entry_on_streams(ps):
    """ps_sort_host_ws: host arrays through caller-owned device buffers, three calls in flight on
    three streams (copy-in, sort and copy-out of different arrays overlap); each result equals the
    oracle's."""
    inputs = [workloads.runs_i32(150001 + 7 * i, seed=40 + i) for i in range(3)]
    refs = [oracle.powersort(k, v) for k, v in inputs]
    streams = [torch.cuda.Stream() for _ in range(3)]
    jobs = []
    for (k, v), s in zip(inputs, streams):
        n = k.size
        hk, hv = torch.from_numpy(k).pin_memory(), torch.from_numpy(v.view(np.int32)).pin_memory()
        ok_, ov = torch.empty_like(hk).pin_memory(), torch.empty_like(hv).pin_memory()
        dk = torch.empty(n, dtype=torch.int32, device="cuda")
        dv = torch.empty(n, dtype=torch.int32, device="cuda")
        ws = torch.empty(ps.ps_workspace_size(0, True, n), dtype=torch.uint8, device="cuda")
        ps.ps_sort_host_ws(0, hk.data_ptr(), hv.data_ptr(), ok_.data_ptr(), ov.data_ptr(), n, dk, dv, ws, stream=s)
        jobs.append((hk, hv, ok_, ov, dk, dv, ws))
    torch.cuda.synchronize()
    assert ps.ps_stream_status() == 0
    for (hk, hv, ok_, ov, *_), ref in zip(jobs, refs):
        np.testing.assert_array_equal(ok_.numpy(), ref.keys)
        np.testing.assert_array_equal(ov.numpy().view(np.uint32), ref.vals)
