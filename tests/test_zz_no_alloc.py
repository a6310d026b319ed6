"""ps_sort_noalloc: the allocation-free entry point for callers that must not allocate device
memory while they run (its scratch is one fixed array in the library's device image).

Every result is compared with the CPU oracle's powersort element by element (keys and
payloads, so the order of equal keys too), and with the regular entry point (ps_sort with a
workspace from the library's pool) beside it, on two calls in a row.  A warm call must leave the
device's free memory unchanged, and a size beyond the fixed maximum must be refused without
touching the data.  This file is collected last on purpose, and it must pass both alone in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

PS_NOALLOC_MAX_N = 262144


@pytest.fixture(scope="module")
def lib():
    import paper_1805_04154_gb300 as ps
    from paper_1805_04154_gb300 import _build
    _build.build()
    lib = ps.load()
    lib.ps_sort_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_void_p]
    lib.ps_sort_noalloc.restype = ctypes.c_int
    assert torch.cuda.is_available()
    return lib


def _reference_sort(keys: torch.Tensor, vals: torch.Tensor | None, kt: int):
    import paper_1805_04154_gb300 as ps
    k, v = keys.clone(), None if vals is None else vals.clone()
    ps.ps_sort(k, v, key_type=kt)
    torch.cuda.synchronize()
    return k, v


def _noalloc_sort(lib, keys: torch.Tensor, vals: torch.Tensor | None, kt: int) -> int:
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.ps_sort_noalloc(kt, ctypes.c_void_p(keys.data_ptr()),
                             None if vals is None else ctypes.c_void_p(vals.data_ptr()), keys.numel(), stream)
    torch.cuda.synchronize()
    return st


def _host(t: torch.Tensor, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def test_noalloc_matches_oracle_two_calls_in_a_row(lib):
    # call 1: int32 runs with payload; call 2: uint64 keys with dense duplicates at the maximum size
    k1, v1 = workloads.runs_i32(200003, seed=31)
    k2, v2 = workloads.pareto_u64(PS_NOALLOC_MAX_N, seed=32, distinct=1000)
    inputs = [(k1, v1, "i32", 0, torch.from_numpy(k1).cuda(), torch.from_numpy(v1.view(np.int32)).cuda()),
              (k2, v2, "u64", 2, torch.from_numpy(k2.view(np.int64)).cuda(),
               torch.from_numpy(v2.view(np.int32)).cuda())]
    for hk, hv, name, kt, dk, dv in inputs:
        ref = oracle.powersort(hk, hv, kt=name)
        want_k, want_v = _reference_sort(dk, dv, kt)
        assert _noalloc_sort(lib, dk, dv, kt) == 0
        np.testing.assert_array_equal(_host(dk, hk.dtype), ref.keys)
        np.testing.assert_array_equal(_host(dv, np.uint32), ref.vals)
        assert torch.equal(dk, want_k)
        assert torch.equal(dv, want_v)


def test_noalloc_keys_only_and_repeat(lib):
    k, _ = workloads.perm_i32(100000, seed=33)
    ref = oracle.powersort(k, None, kt="i32")
    for _ in range(2):
        dk = torch.from_numpy(k).cuda()
        want_k, _ = _reference_sort(dk, None, 0)
        assert _noalloc_sort(lib, dk, None, 0) == 0
        np.testing.assert_array_equal(_host(dk, np.int32), ref.keys)
        assert torch.equal(dk, want_k)


def test_noalloc_allocates_nothing(lib):
    """After a first call of the same key type and payload choice (kernel modules loaded), a call
    leaves the device's free memory exactly as it was."""
    k, v = workloads.runs_i32(150001, seed=35)
    ref = oracle.powersort(k, v, kt="i32")
    dk = torch.from_numpy(k).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    warm_k, warm_v = dk.clone(), dv.clone()
    assert _noalloc_sort(lib, warm_k, warm_v, 0) == 0
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    assert _noalloc_sort(lib, dk, dv, 0) == 0
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    np.testing.assert_array_equal(_host(dk, np.int32), ref.keys)
    np.testing.assert_array_equal(_host(dv, np.uint32), ref.vals)


def test_noalloc_refuses_sizes_beyond_its_scratch(lib):
    k, v = workloads.runs_i32(PS_NOALLOC_MAX_N + 1, seed=34)
    dk = torch.from_numpy(k).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    before = dk.clone()
    assert _noalloc_sort(lib, dk, dv, 0) == 1  # PS_ERR_INVALID_ARG
    assert torch.equal(dk, before)
