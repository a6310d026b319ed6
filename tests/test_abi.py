"""CPU checks of the C ABI: the library loads, exports every function include/*.h declares,
rejects bad arguments before touching a GPU, and its host-only merge cost agrees with the
oracle."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    import paper_1805_04154_gb300 as ps
    from paper_1805_04154_gb300 import _build
    _build.build()
    return ps.load()


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ps_[a-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("ps_sort", "ps_sort_segmented", "ps_merge_cost", "ps_sort_stats", "ps_stream_status",
                 "ps_status_string", "ps_analyze", "ps_sort_ws", "ps_workspace_size"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    import paper_1805_04154_gb300 as ps
    for s in range(7):
        assert len(ps.ps_status_string(s)) > 0
    assert ps.ps_version() >= 100


def test_argument_errors_without_gpu(lib):
    ws = ctypes.c_void_p(256)
    # unknown key type, negative n, misaligned pointer, too large n: rejected before any CUDA call
    assert lib.ps_sort_ws(9, ctypes.c_void_p(4096), None, 10, ws, 1 << 20, None) == 1
    assert lib.ps_sort_ws(0, ctypes.c_void_p(4096), None, -1, ws, 1 << 20, None) == 1
    assert lib.ps_sort_ws(0, ctypes.c_void_p(4098), None, 10, ws, 1 << 20, None) == 1  # int32 needs 4 B
    assert lib.ps_sort_ws(2, ctypes.c_void_p(4100), None, 10, ws, 1 << 20, None) == 1  # uint64 needs 8 B
    assert lib.ps_sort_ws(0, ctypes.c_void_p(4096), ctypes.c_void_p(4106), 10, ws, 1 << 20, None) == 1
    assert lib.ps_sort_ws(0, ctypes.c_void_p(4096), None, 1 << 32, ws, 1 << 20, None) == 2
    # n = 2^31 is accepted (64-bit positions); a workspace of 1 MiB is refused as too small
    assert lib.ps_sort_ws(0, ctypes.c_void_p(4096), None, 1 << 31, ws, 1 << 20, None) == 3
    # a single array needs run arrays for n/2 + 3 runs, a segmented one for n + 2
    assert lib.ps_workspace_size(0, 1, 1 << 31, 0) < lib.ps_workspace_size(0, 1, 1 << 31, 1)
    assert lib.ps_workspace_size(0, 1, 1000, 0) > 1000 * 8
    assert lib.ps_workspace_size(7, 1, 1000, 0) == 0
    # n = 0 and n = 1 are no-ops
    assert lib.ps_sort_ws(0, ctypes.c_void_p(4096), None, 0, None, 0, None) == 0
    assert lib.ps_sort_ws(0, ctypes.c_void_p(4096), None, 1, None, 0, None) == 0


def test_merge_cost_host_matches_oracle(lib):
    import paper_1805_04154_gb300 as ps
    rng = np.random.default_rng(1)
    assert ps.ps_merge_cost([5, 3, 3, 14, 1, 2]) == 67  # Fig. 1, Method 2 tree
    for _ in range(300):
        r = int(rng.integers(1, 300))
        L = rng.integers(1, int(rng.choice([3, 100, 10 ** 6])), size=r)
        assert ps.ps_merge_cost(L) == oracle.powersort_cost(L)[0]
    # large n beyond 2^31 still exact (62-bit formulation)
    L = rng.integers(1, 1 << 40, size=50)
    assert ps.ps_merge_cost(L) == oracle.powersort_cost(L)[0]
    out = ctypes.c_uint64()
    bad = np.array([3, 0, 2], np.int64)
    assert lib.ps_merge_cost(ctypes.c_void_p(bad.ctypes.data), 3, ctypes.byref(out)) == 1
    assert lib.ps_merge_cost(None, 3, ctypes.byref(out)) == 1


def test_tree_argument_errors_without_gpu(lib):
    ws = ctypes.c_void_p(256)
    # unknown merge tree: rejected before any CUDA call
    assert lib.ps_sort_tree_ws(0, ctypes.c_void_p(4096), None, 10, None, 1, 7, ws, 1 << 20, None) == 1
    assert lib.ps_workspace_size_tree(0, 1, 1000, 0, 7) == 0
    assert lib.ps_workspace_size_tree(0, 1, 1000, 0, 1) > lib.ps_workspace_size_tree(0, 1, 1000, 0, 0)


def test_bounded_async_argument_errors_without_gpu(lib):
    ws = ctypes.c_void_p(256)
    keys = ctypes.c_void_p(4096)
    # a bound below one element, or one array longer than its bound: rejected before any CUDA call
    for bound in (0, -5, 9):
        assert lib.ps_sort_async_bounded_ws(0, keys, None, 10, None, 1, bound, ws, 1 << 20, None) == 1


def test_minrun_argument_errors_without_gpu(lib):
    ws = ctypes.c_void_p(256)
    keys = ctypes.c_void_p(4096)
    # minimal run length outside [1, 32]: rejected before any CUDA call
    for w in (0, -3, 33, 1000):
        assert lib.ps_sort_minrun_ws(0, keys, None, 10, None, 1, w, ws, 1 << 20, None) == 1
        assert lib.ps_analyze_minrun(0, keys, 10, None, 1, w, ws, 1 << 20, None, None, None, None, None,
                                     None, None, None, None, None) == 1


def test_release_build_has_no_bounds_checks(lib):
    import paper_1805_04154_gb300 as ps
    if ps.lib_path.endswith("libpowersort.so"):
        assert ps.ps_debug_bounds() is None  # PS_ERR_UNSUPPORTED without -DPS_DEBUG


def test_tuning_table_without_gpu(lib):
    import paper_1805_04154_gb300 as ps
    assert ps.ps_tune_get(0, True) == (8, 2)
    ps.ps_tune_set(0, True, 16, 2)
    assert ps.ps_tune_get(0, True) == (16, 2)
    assert ps.ps_tune_get(0, False) == (8, 2)
    with pytest.raises(ps.PowersortError):
        ps.ps_tune_set(0, True, 10, 3)  # not a configuration the library carries
    ps.ps_tune_set(0, True, 0, 0)
    assert ps.ps_tune_get(0, True) == (8, 2)
    assert ps.ps_tune_get(2, True) == (6, 2)  # 8-byte keys: 6 items per thread by default
    assert ps.ps_tune_get(2, False) == (6, 2)


def test_binding_rejects_mismatched_buffers_without_gpu(lib):
    """The Python binding checks what the C ABI cannot see behind its pointers (key width against
    the key type, payload and offsets sizes, dtypes and devices) before anything is launched."""
    import torch

    import paper_1805_04154_gb300 as ps
    k32 = torch.zeros(8, dtype=torch.int32)
    ws = torch.zeros(256, dtype=torch.uint8)
    with pytest.raises(ValueError, match="8-byte keys"):
        ps.ps_sort_ws(k32, None, ws, key_type=ps.PS_KEY_U64)
    with pytest.raises(ValueError, match="unknown key type"):
        ps.ps_sort_ws(k32, None, ws, key_type=7)
    with pytest.raises(ValueError, match="32-bit payloads"):
        ps.ps_sort_ws(k32, torch.zeros(7, dtype=torch.int32), ws)
    with pytest.raises(ValueError, match="32-bit payloads"):
        ps.ps_sort_async_ws(k32, torch.zeros(8, dtype=torch.int64), ws)
    with pytest.raises(TypeError, match="int64"):
        ps.ps_sort_tree_ws(k32, None, ws, offsets=torch.tensor([0, 8], dtype=torch.int32))
    with pytest.raises(TypeError, match="int64"):
        ps.ps_sort_segmented_ws(k32, None, torch.tensor([0, 8], dtype=torch.int32), ws)
    with pytest.raises(ValueError, match="offsets are required"):
        ps.ps_sort_segmented(k32, None, None)
    with pytest.raises(ValueError, match="32-bit payloads"):
        ps.ps_sort_segmented(k32, torch.zeros(9, dtype=torch.int32), torch.tensor([0, 8]))
    # host arrays: sizes and widths against n and the key type
    a = np.zeros(8, np.int32)
    with pytest.raises(ValueError, match="8 elements of 4 bytes"):
        ps.ps_sort_host(a, None, np.zeros(7, np.int32), None, ps.PS_KEY_I32)
    with pytest.raises(ValueError, match="of 8 bytes"):
        ps.ps_sort_host(a, None, np.zeros(8, np.int32), None, ps.PS_KEY_U64)
    with pytest.raises(ValueError, match="neither"):
        ps.ps_sort_host(a, np.zeros(8, np.uint32), np.zeros(8, np.int32), None, ps.PS_KEY_I32)
    with pytest.raises(ValueError, match="dev_keys"):
        ps.ps_sort_host_ws(ps.PS_KEY_I32, 1, None, 1, None, 16, k32, None, ws)
