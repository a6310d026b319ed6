"""ps_sort_noalloc: the allocation-free entry point for callers that must not allocate device
memory while they run (its scratch is one fixed array in the library's device image).

Checked through the C ABI against the regular entry point (ps_sort_ws with a workspace from
PyTorch's allocator): the results must be identical, bit for bit, on two calls in a row, and a
size beyond the fixed maximum must be refused without touching the data.  This file is
collected last on purpose, and it must pass both alone in a fresh process and after the other
tests."""
import ctypes

import numpy as np
import pytest
import torch

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


def test_noalloc_matches_regular_entry_two_calls_in_a_row(lib):
    # call 1: int32 runs with payload; call 2: uint64 keys with dense duplicates at the maximum size
    k1, v1 = workloads.runs_i32(200003, seed=31)
    k2, v2 = workloads.pareto_u64(PS_NOALLOC_MAX_N, seed=32, distinct=1000)
    inputs = [(torch.from_numpy(k1).cuda(), torch.from_numpy(v1.view(np.int32)).cuda(), 0),
              (torch.from_numpy(k2.view(np.int64)).cuda(), torch.from_numpy(v2.view(np.int32)).cuda(), 2)]
    for dk, dv, kt in inputs:
        want_k, want_v = _reference_sort(dk, dv, kt)
        assert _noalloc_sort(lib, dk, dv, kt) == 0
        assert torch.equal(dk, want_k)
        assert torch.equal(dv, want_v)


def test_noalloc_keys_only_and_repeat(lib):
    k, _ = workloads.perm_i32(100000, seed=33)
    for _ in range(2):
        dk = torch.from_numpy(k).cuda()
        want_k, _ = _reference_sort(dk, None, 0)
        assert _noalloc_sort(lib, dk, None, 0) == 0
        assert torch.equal(dk, want_k)


def test_noalloc_refuses_sizes_beyond_its_scratch(lib):
    k, v = workloads.runs_i32(PS_NOALLOC_MAX_N + 1, seed=34)
    dk = torch.from_numpy(k).cuda()
    dv = torch.from_numpy(v.view(np.int32)).cuda()
    before = dk.clone()
    assert _noalloc_sort(lib, dk, dv, 0) == 1  # PS_ERR_INVALID_ARG
    assert torch.equal(dk, before)
