"""GB300 powersort: stable natural mergesort in powersort's merge order (Munro & Wild,
arXiv 1805.04154), as hand-written CUDA kernels for sm_103a behind a C ABI.

This module is the thin Python binding of ``libpowersort.so`` (``include/powersort.h``): it
marshals PyTorch CUDA tensors (pointers, sizes, the current stream, a workspace tensor from
PyTorch's caching allocator) into the C entry points of the same names.  Every step of the sort
runs in the library's kernels; there is no CPU or PyTorch fallback, and importing this module
fails loudly when the library has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

__all__ = [
    "PowersortError", "PS_KEY_I32", "PS_KEY_U32", "PS_KEY_U64", "PS_KEY_F32", "lib_path", "load",
    "ps_sort", "ps_sort_ws", "ps_sort_segmented", "ps_sort_segmented_ws", "ps_workspace_size",
    "ps_sort_minrun", "ps_sort_minrun_ws",
    "ps_merge_cost", "ps_analyze", "ps_sort_stats", "ps_stream_status", "ps_status_string",
    "ps_version", "key_type_of", "ps_sort_host", "ps_profile_enable", "ps_profile_read",
    "ps_launch_count", "STAGES", "PS_TREE_POWERSORT", "PS_TREE_PEEKSORT", "ps_sort_tree_ws",
    "ps_sort_tree", "ps_sort_host_ws", "ps_sort_async_ws", "ps_sort_async_bounded_ws", "ps_autotune", "ps_tune_set", "ps_tune_get",
]

STAGES = ["detect", "meta", "subtree_smem", "leaf_place", "unused", "level_pass"]

PS_KEY_I32, PS_KEY_U32, PS_KEY_U64, PS_KEY_F32 = 0, 1, 2, 3
PS_TREE_POWERSORT, PS_TREE_PEEKSORT = 0, 1
_STATUS = {0: "PS_OK", 1: "PS_ERR_INVALID_ARG", 2: "PS_ERR_UNSUPPORTED", 3: "PS_ERR_OUT_OF_MEMORY",
           4: "PS_ERR_CUDA", 5: "PS_ERR_TIMEOUT", 6: "PS_ERR_INTERNAL"}

_HERE = os.path.dirname(os.path.abspath(__file__))
# PS_DEBUG=1 selects the bounds-checked build (libpowersort_debug.so, see _build.build(debug=True))
lib_path = os.path.join(_HERE, "libpowersort_debug.so" if os.environ.get("PS_DEBUG") == "1" else "libpowersort.so")
_lib = None
_lock = threading.Lock()


class _Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_uint64 * 8),
                ("bytes", ctypes.c_uint64 * 8)]


class PowersortError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)} ({ps_status_string(status)})")


class _Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("runs", ctypes.c_int64), ("merge_cost", ctypes.c_uint64),
                ("entropy_bits", ctypes.c_double), ("max_depth", ctypes.c_int32),
                ("merge_passes", ctypes.c_int32), ("small_tasks", ctypes.c_int64)]


def load():
    """Load libpowersort.so (built in-tree); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(lib_path):
                raise ImportError(f"{lib_path} is missing: build it with __graft_entry__.build()")
            lib = ctypes.CDLL(lib_path)
            vp, i32, i64, u64, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                     ctypes.c_size_t)
            sigs = {
                "ps_workspace_size": ([i32, i32, i64, i32], sz),
                "ps_sort_ws": ([i32, vp, vp, i64, vp, sz, vp], i32),
                "ps_sort": ([i32, vp, vp, i64, vp], i32),
                "ps_sort_i32": ([vp, vp, i64, vp], i32),
                "ps_sort_u32": ([vp, vp, i64, vp], i32),
                "ps_sort_u64": ([vp, vp, i64, vp], i32),
                "ps_sort_f32": ([vp, vp, i64, vp], i32),
                "ps_sort_segmented_ws": ([i32, vp, vp, i64, vp, i64, vp, sz, vp], i32),
                "ps_sort_segmented": ([i32, vp, vp, vp, i64, vp], i32),
                "ps_merge_cost": ([vp, i64, vp], i32),
                "ps_analyze": ([i32, vp, i64, vp, i64, vp, sz, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
                "ps_sort_stats": ([i32, vp, i64, vp, vp], i32),
                "ps_stream_status": ([vp], i32),
                "ps_status_string": ([i32], ctypes.c_char_p),
                "ps_version": ([], i32),
                "ps_sort_host": ([i32, vp, vp, vp, vp, i64, vp], i32),
                "ps_profile_enable": ([i32], i32),
                "ps_profile_read": ([vp], i32),
                "ps_launch_count": ([], u64),
                "ps_workspace_size_tree": ([i32, i32, i64, i32, i32], sz),
                "ps_sort_host_ws": ([i32, vp, vp, vp, vp, i64, vp, vp, vp, sz, vp], i32),
                "ps_sort_async_ws": ([i32, vp, vp, i64, vp, i64, i32, vp, sz, vp], i32),
                "ps_sort_async_bounded_ws": ([i32, vp, vp, i64, vp, i64, i64, vp, sz, vp], i32),
                "ps_autotune": ([i32, vp, vp, i64, vp, vp], i32),
                "ps_tune_set": ([i32, i32, i32, i32], i32),
                "ps_tune_get": ([i32, i32, vp, vp], i32),
                "ps_tune_get_for": ([i32, i32, i64, i32, vp, vp], i32),
                "ps_autotune_segmented": ([i32, vp, vp, i64, vp, i64, vp, vp], i32),
                "ps_selftest_wait_timeout": ([ctypes.c_uint32, vp], i32),
                "ps_selftest_level_pass_timeout": ([i32, vp, vp, i64, ctypes.c_uint32, vp, sz, vp], i32),
                "ps_sort_tree_ws": ([i32, vp, vp, i64, vp, i64, i32, vp, sz, vp], i32),
                "ps_analyze_tree": ([i32, vp, i64, vp, i64, i32, vp, sz, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                     vp], i32),
                "ps_sort_minrun_ws": ([i32, vp, vp, i64, vp, i64, i32, vp, sz, vp], i32),
                "ps_debug_bounds": ([vp], i32),
                "ps_analyze_minrun": ([i32, vp, i64, vp, i64, i32, vp, sz, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                       vp], i32),
            }
            for name, (args, res) in sigs.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def ps_status_string(status: int) -> str:
    return load().ps_status_string(int(status)).decode()


def ps_version() -> int:
    return int(load().ps_version())


def _check(status: int, where: str):
    if status != 0:
        raise PowersortError(status, where)


def key_type_of(t: torch.Tensor) -> int:
    dt = t.dtype
    if dt == torch.int32:
        return PS_KEY_I32
    if dt == torch.float32:
        return PS_KEY_F32
    if dt == torch.int64 or dt == getattr(torch, "uint64", None):
        return PS_KEY_U64
    if dt == getattr(torch, "uint32", None):
        return PS_KEY_U32
    raise TypeError(f"unsupported key dtype {dt}")


def _stream_ptr(stream, device) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t: torch.Tensor | None, name: str):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


_KEY_BYTES = {PS_KEY_I32: 4, PS_KEY_U32: 4, PS_KEY_U64: 8, PS_KEY_F32: 4}


def _key_type(keys: torch.Tensor, key_type: int | None) -> int:
    """The key type passed to the library: the dtype's, or the caller's choice when its key width
    matches the tensor's elements (the library reads n keys of that width from the pointer)."""
    kt = key_type_of(keys) if key_type is None else int(key_type)
    if kt not in _KEY_BYTES:
        raise ValueError(f"unknown key type {kt}")
    if keys.element_size() != _KEY_BYTES[kt]:
        raise ValueError(f"key type {kt} reads {_KEY_BYTES[kt]}-byte keys but keys are {keys.dtype}")
    return kt


def _check_vals(vals: torch.Tensor | None, keys: torch.Tensor) -> None:
    if vals is None:
        return
    if vals.numel() != keys.numel() or vals.element_size() != 4:
        raise ValueError("vals must hold n 32-bit payloads")
    if vals.device != keys.device:
        raise ValueError("vals must be on the keys' device")


def _segments(offsets: torch.Tensor | None, keys: torch.Tensor) -> int:
    """Segment count of ``offsets`` (int64, count + 1 entries, on the keys' device); 1 without."""
    if offsets is None:
        return 1
    if offsets.dtype != torch.int64:
        raise TypeError("offsets must be int64")
    if offsets.device != keys.device:
        raise ValueError("offsets must be on the keys' device")
    return offsets.numel() - 1


def _ws_bytes(workspace: torch.Tensor, keys: torch.Tensor) -> int:
    if workspace.device != keys.device:
        raise ValueError("workspace must be on the keys' device")
    return workspace.numel() * workspace.element_size()


def ps_workspace_size(key_type: int, has_vals: bool, n: int, segmented: bool = False,
                      tree: int = PS_TREE_POWERSORT) -> int:
    if tree == PS_TREE_POWERSORT:
        return int(load().ps_workspace_size(key_type, 1 if has_vals else 0, n, 1 if segmented else 0))
    return int(load().ps_workspace_size_tree(key_type, 1 if has_vals else 0, n, 1 if segmented else 0, tree))


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def ps_sort_ws(keys: torch.Tensor, vals: torch.Tensor | None, workspace: torch.Tensor,
               key_type: int | None = None, stream=None) -> None:
    """Stable in-place sort of ``keys`` (and ``vals``) with a caller-provided workspace tensor."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    _check_vals(vals, keys)
    _check(load().ps_sort_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n,
                             _dev_ptr(workspace, "workspace"), _ws_bytes(workspace, keys),
                             _stream_ptr(stream, keys.device)), "ps_sort_ws")


def ps_sort(keys: torch.Tensor, vals: torch.Tensor | None = None, key_type: int | None = None,
            stream=None, pool: bool = False) -> torch.Tensor:
    """Stable in-place powersort of a CUDA tensor of keys (int32 / uint32 / uint64 / float32 in
    IEEE totalOrder), carrying an optional 32-bit payload.  The workspace comes from PyTorch's
    caching allocator, or from the library's own stream-ordered pool when ``pool``."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    _check_vals(vals, keys)
    sp = _stream_ptr(stream, keys.device)
    if pool:
        _check(load().ps_sort(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n, sp), "ps_sort")
        return keys
    ws = _workspace(ps_workspace_size(kt, vals is not None, n), keys.device)
    _check(load().ps_sort_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n,
                             _dev_ptr(ws, "workspace"), ws.numel(), sp), "ps_sort")
    return keys


def ps_sort_tree_ws(keys: torch.Tensor, vals: torch.Tensor | None, workspace: torch.Tensor,
                    tree: int = PS_TREE_PEEKSORT, offsets: torch.Tensor | None = None,
                    key_type: int | None = None, stream=None) -> None:
    """ps_sort_ws / ps_sort_segmented_ws with the merge tree chosen by ``tree``."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    _check_vals(vals, keys)
    count = _segments(offsets, keys)
    _check(load().ps_sort_tree_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n,
                                  _dev_ptr(offsets, "offsets"), count, int(tree), _dev_ptr(workspace, "workspace"),
                                  _ws_bytes(workspace, keys), _stream_ptr(stream, keys.device)), "ps_sort_tree_ws")


def ps_sort_tree(keys: torch.Tensor, vals: torch.Tensor | None = None, tree: int = PS_TREE_PEEKSORT,
                 offsets: torch.Tensor | None = None, key_type: int | None = None, stream=None) -> torch.Tensor:
    """In-place stable sort with the merge tree chosen by ``tree`` (workspace from PyTorch)."""
    kt = _key_type(keys, key_type)
    ws = _workspace(ps_workspace_size(kt, vals is not None, keys.numel(), offsets is not None, tree), keys.device)
    ps_sort_tree_ws(keys, vals, ws, tree, offsets, kt, stream)
    return keys


def ps_sort_minrun_ws(keys: torch.Tensor, vals: torch.Tensor | None, workspace: torch.Tensor, min_run: int,
                      offsets: torch.Tensor | None = None, key_type: int | None = None, stream=None) -> None:
    """ps_sort_ws / ps_sort_segmented_ws with runs extended to ``min_run`` elements (Sec. 5.1)."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    _check_vals(vals, keys)
    count = _segments(offsets, keys)
    _check(load().ps_sort_minrun_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n,
                                    _dev_ptr(offsets, "offsets"), count, int(min_run),
                                    _dev_ptr(workspace, "workspace"), _ws_bytes(workspace, keys),
                                    _stream_ptr(stream, keys.device)), "ps_sort_minrun_ws")


def ps_sort_minrun(keys: torch.Tensor, vals: torch.Tensor | None = None, min_run: int = 24,
                   offsets: torch.Tensor | None = None, key_type: int | None = None, stream=None) -> torch.Tensor:
    """In-place stable sort with runs extended to ``min_run`` elements (workspace from PyTorch)."""
    kt = _key_type(keys, key_type)
    ws = _workspace(ps_workspace_size(kt, vals is not None, keys.numel(), offsets is not None), keys.device)
    ps_sort_minrun_ws(keys, vals, ws, min_run, offsets, kt, stream)
    return keys


def ps_sort_segmented(keys: torch.Tensor, vals: torch.Tensor | None, offsets: torch.Tensor,
                      key_type: int | None = None, stream=None) -> torch.Tensor:
    """Sort every segment [offsets[k], offsets[k+1]) on its own (offsets: CUDA int64, count+1)."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    _check_vals(vals, keys)
    if offsets is None:
        raise ValueError("offsets are required")
    count = _segments(offsets, keys)
    ws = _workspace(ps_workspace_size(kt, vals is not None, n, True), keys.device)
    _check(load().ps_sort_segmented_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n,
                                       _dev_ptr(offsets, "offsets"), count, _dev_ptr(ws, "workspace"),
                                       ws.numel(), _stream_ptr(stream, keys.device)),
           "ps_sort_segmented")
    return keys


def ps_sort_segmented_ws(keys, vals, offsets, workspace, key_type=None, stream=None) -> None:
    """ps_sort_segmented with a caller-provided workspace tensor."""
    kt = _key_type(keys, key_type)
    _check_vals(vals, keys)
    if offsets is None:
        raise ValueError("offsets are required")
    count = _segments(offsets, keys)
    _check(load().ps_sort_segmented_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), keys.numel(),
                                       _dev_ptr(offsets, "offsets"), count,
                                       _dev_ptr(workspace, "workspace"), _ws_bytes(workspace, keys),
                                       _stream_ptr(stream, keys.device)), "ps_sort_segmented_ws")


def ps_merge_cost(run_lengths) -> int:
    """Powersort merge cost M of runs with the given lengths (host computation)."""
    L = np.ascontiguousarray(run_lengths, dtype=np.int64)
    out = ctypes.c_uint64(0)
    _check(load().ps_merge_cost(ctypes.c_void_p(L.ctypes.data), L.size, ctypes.byref(out)),
           "ps_merge_cost")
    return int(out.value)


def ps_analyze(keys: torch.Tensor, offsets: torch.Tensor | None = None, key_type: int | None = None,
               stream=None, tree: int = PS_TREE_POWERSORT, min_run: int = 1) -> dict:
    """Run detection, node powers (or peeksort's tree) and merge tree on the device (keys
    untouched); returns numpy arrays: starts, desc, power, leaf_depth, node_left, node_right,
    node_depth, and runs, cost.  With ``min_run`` > 1 the runs are extended to that length
    (powersort tree only) and desc carries bit 1 for extended runs."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    seg = offsets is not None
    count = _segments(offsets, keys)
    ws = _workspace(ps_workspace_size(kt, False, n, seg, tree), keys.device)
    cap = n + 2
    out = {"starts": np.empty(cap, np.int64), "desc": np.empty(cap, np.uint8), "power": np.empty(cap, np.uint8),
           "leaf_depth": np.empty(cap, np.uint8), "node_left": np.empty(cap, np.int32),
           "node_right": np.empty(cap, np.int32), "node_depth": np.empty(cap, np.uint8)}
    runs = ctypes.c_int64(0)
    cost = ctypes.c_uint64(0)
    p = {k: ctypes.c_void_p(v.ctypes.data) for k, v in out.items()}
    if min_run != 1:
        if tree != PS_TREE_POWERSORT:
            raise ValueError("min_run > 1 builds the powersort tree only")
        fn, sel = load().ps_analyze_minrun, int(min_run)
    else:
        fn, sel = load().ps_analyze_tree, int(tree)
    _check(fn(kt, _dev_ptr(keys, "keys"), n, _dev_ptr(offsets, "offsets"), count, sel, _dev_ptr(ws, "workspace"),
              ws.numel(), ctypes.byref(runs), ctypes.byref(cost), p["starts"], p["desc"],
              p["power"], p["leaf_depth"], p["node_left"], p["node_right"], p["node_depth"],
              _stream_ptr(stream, keys.device)), "ps_analyze")
    r = int(runs.value)
    res = {"runs": r, "cost": int(cost.value), "starts": out["starts"][: r + 1].copy(),
           "desc": out["desc"][:r].copy(), "power": out["power"][: r + 1].copy(),
           "leaf_depth": out["leaf_depth"][:r].copy(), "node_left": out["node_left"][: r + 1].copy(),
           "node_right": out["node_right"][: r + 1].copy(), "node_depth": out["node_depth"][: r + 1].copy()}
    return res


def ps_sort_stats(keys: torch.Tensor, key_type: int | None = None, stream=None) -> dict:
    kt = _key_type(keys, key_type)
    st = _Stats()
    _check(load().ps_sort_stats(kt, _dev_ptr(keys, "keys"), keys.numel(), ctypes.byref(st),
                                _stream_ptr(stream, keys.device)), "ps_sort_stats")
    return {f: getattr(st, f) for f, _ in _Stats._fields_}


def ps_debug_bounds() -> int | None:
    """Out-of-range accesses counted by a bounds-checked library (None for a library built
    without the checks)."""
    v = ctypes.c_ulonglong(0)
    st = load().ps_debug_bounds(ctypes.byref(v))
    if st == 2:
        return None
    _check(st, "ps_debug_bounds")
    return int(v.value)


def ps_stream_status(stream=None, device=None) -> int:
    """Synchronize the stream and return (and clear) device-posted status (0 = ok)."""
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(load().ps_stream_status(ctypes.c_void_p(stream.cuda_stream)))


def ps_sort_host(keys_in: np.ndarray, vals_in: np.ndarray | None, keys_out: np.ndarray,
                 vals_out: np.ndarray | None, key_type: int, stream=None) -> None:
    """Sort host arrays through the GPU (copies in, sorts, copies out; synchronizes)."""
    n = keys_in.size
    if key_type not in _KEY_BYTES:
        raise ValueError(f"unknown key type {key_type}")
    if (vals_in is None) != (vals_out is None):
        raise ValueError("give both vals_in and vals_out, or neither")
    for a, width in ((keys_in, _KEY_BYTES[key_type]), (keys_out, _KEY_BYTES[key_type]), (vals_in, 4), (vals_out, 4)):
        if a is None:
            continue
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous")
        if a.size != n or a.itemsize != width:
            raise ValueError(f"host arrays must hold n = {n} elements of {width} bytes (got {a.size} of {a.itemsize})")
    if not keys_out.flags["WRITEABLE"] or (vals_out is not None and not vals_out.flags["WRITEABLE"]):
        raise ValueError("output arrays must be writeable")
    sp = _stream_ptr(stream, torch.device("cuda", torch.cuda.current_device()))
    ptr = (lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data))
    _check(load().ps_sort_host(key_type, ptr(keys_in), ptr(vals_in), ptr(keys_out), ptr(vals_out), n, sp),
           "ps_sort_host")


def ps_sort_host_ptr(key_type: int, keys_in: int, vals_in: int | None, keys_out: int, vals_out: int | None,
                     n: int, stream=None) -> None:
    """ps_sort_host on raw host addresses (e.g. pinned torch tensors' data_ptr())."""
    sp = _stream_ptr(stream, torch.device("cuda", torch.cuda.current_device()))
    vp = (lambda a: None if a is None else ctypes.c_void_p(a))
    _check(load().ps_sort_host(key_type, vp(keys_in), vp(vals_in), vp(keys_out), vp(vals_out), n, sp),
           "ps_sort_host")


def ps_profile_enable(on: bool = True) -> None:
    _check(load().ps_profile_enable(1 if on else 0), "ps_profile_enable")


def ps_profile_read() -> dict:
    """Per stage: device ms, kernel launches, algorithmic HBM bytes since the last enable."""
    p = _Profile()
    _check(load().ps_profile_read(ctypes.byref(p)), "ps_profile_read")
    return {name: {"ms": p.ms[i], "launches": int(p.launches[i]), "bytes": int(p.bytes[i])}
            for i, name in enumerate(STAGES)}


def ps_launch_count() -> int:
    return int(load().ps_launch_count())


def ps_sort_host_ws(key_type: int, keys_in: int, vals_in: int | None, keys_out: int, vals_out: int | None, n: int,
                    dev_keys: torch.Tensor, dev_vals: torch.Tensor | None, workspace: torch.Tensor,
                    stream=None) -> None:
    """Queue copy-in, sort and copy-out of host arrays (raw host pointers, pinned for asynchrony)
    through caller-owned device buffers on ``stream``; synchronize the stream before reading the
    output."""
    if key_type not in _KEY_BYTES:
        raise ValueError(f"unknown key type {key_type}")
    if dev_keys.numel() < n or dev_keys.element_size() != _KEY_BYTES[key_type]:
        raise ValueError(f"dev_keys must hold at least n = {n} keys of {_KEY_BYTES[key_type]} bytes")
    if (not vals_in) != (dev_vals is None) or (not vals_out) != (dev_vals is None):
        raise ValueError("vals_in, vals_out and dev_vals go together")
    if dev_vals is not None and (dev_vals.numel() < n or dev_vals.element_size() != 4
                                 or dev_vals.device != dev_keys.device):
        raise ValueError(f"dev_vals must hold at least n = {n} 32-bit payloads on the keys' device")
    _check(load().ps_sort_host_ws(key_type, ctypes.c_void_p(keys_in), ctypes.c_void_p(vals_in) if vals_in else None,
                                  ctypes.c_void_p(keys_out), ctypes.c_void_p(vals_out) if vals_out else None, n,
                                  _dev_ptr(dev_keys, "dev_keys"), _dev_ptr(dev_vals, "dev_vals"),
                                  _dev_ptr(workspace, "workspace"), _ws_bytes(workspace, dev_keys),
                                  _stream_ptr(stream, dev_keys.device)), "ps_sort_host_ws")


def ps_sort_async_ws(keys: torch.Tensor, vals: torch.Tensor | None, workspace: torch.Tensor,
                     offsets: torch.Tensor | None = None, tree: int = PS_TREE_POWERSORT,
                     key_type: int | None = None, stream=None) -> None:
    """Device-driven sort (no host round trip; capturable into a CUDA graph).  Device-side
    errors are reported by ``ps_stream_status``."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    _check_vals(vals, keys)
    count = _segments(offsets, keys)
    _check(load().ps_sort_async_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n,
                                   _dev_ptr(offsets, "offsets"), count, int(tree), _dev_ptr(workspace, "workspace"),
                                   _ws_bytes(workspace, keys), _stream_ptr(stream, keys.device)), "ps_sort_async_ws")


def ps_sort_async_bounded_ws(keys: torch.Tensor, vals: torch.Tensor | None, workspace: torch.Tensor,
                             max_segment: int, offsets: torch.Tensor | None = None, key_type: int | None = None,
                             stream=None) -> None:
    """ps_sort_async_ws (powersort's tree) for a caller that knows every segment holds at most
    ``max_segment`` elements (checked on the device): fewer level-pass launches are queued."""
    kt = _key_type(keys, key_type)
    n = keys.numel()
    _check_vals(vals, keys)
    count = _segments(offsets, keys)
    _check(load().ps_sort_async_bounded_ws(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), n,
                                           _dev_ptr(offsets, "offsets"), count, int(max_segment),
                                           _dev_ptr(workspace, "workspace"), _ws_bytes(workspace, keys),
                                           _stream_ptr(stream, keys.device)), "ps_sort_async_bounded_ws")


class _Tune(ctypes.Structure):
    _fields_ = [("items_per_thread", ctypes.c_int), ("stages", ctypes.c_int), ("n_variants", ctypes.c_int),
                ("variant_items", ctypes.c_int * 8), ("variant_stages", ctypes.c_int * 8),
                ("variant_ms", ctypes.c_double * 8)]


def ps_autotune(keys: torch.Tensor, vals: torch.Tensor | None = None, key_type: int | None = None,
                stream=None) -> dict:
    """Time every level-pass configuration on copies of ``keys``/``vals`` (unchanged) and keep the
    fastest for this key type and payload choice; returns the choice and all timings."""
    kt = _key_type(keys, key_type)
    out = _Tune()
    _check(load().ps_autotune(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), keys.numel(), ctypes.byref(out),
                              _stream_ptr(stream, keys.device)), "ps_autotune")
    return {"items_per_thread": out.items_per_thread, "stages": out.stages,
            "variants": [{"items_per_thread": out.variant_items[i], "stages": out.variant_stages[i],
                          "ms": out.variant_ms[i]} for i in range(out.n_variants)]}


def ps_autotune_segmented(keys: torch.Tensor, vals: torch.Tensor | None, offsets: torch.Tensor,
                          key_type: int | None = None, stream=None) -> dict:
    """ps_autotune for segmented batches: times the segmented sort of ``keys``/``vals`` (unchanged)
    with ``offsets`` and keeps the fastest configuration for segmented sorts of this size."""
    kt = _key_type(keys, key_type)
    _check_vals(vals, keys)
    count = _segments(offsets, keys)
    out = _Tune()
    _check(load().ps_autotune_segmented(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), keys.numel(),
                                        _dev_ptr(offsets, "offsets"), count, ctypes.byref(out),
                                        _stream_ptr(stream, keys.device)), "ps_autotune_segmented")
    return {"items_per_thread": out.items_per_thread, "stages": out.stages,
            "variants": [{"items_per_thread": out.variant_items[i], "stages": out.variant_stages[i],
                          "ms": out.variant_ms[i]} for i in range(out.n_variants)]}


def ps_tune_get_for(key_type: int, has_vals: bool, n: int, segmented: bool = False) -> tuple[int, int]:
    """The level-pass configuration a sort of n elements uses (tuned entry of its size bucket, else
    the default)."""
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().ps_tune_get_for(key_type, 1 if has_vals else 0, int(n), 1 if segmented else 0, ctypes.byref(a),
                                  ctypes.byref(b)), "ps_tune_get_for")
    return a.value, b.value


def ps_tune_set(key_type: int, has_vals: bool, items_per_thread: int, stages: int) -> None:
    _check(load().ps_tune_set(key_type, 1 if has_vals else 0, items_per_thread, stages), "ps_tune_set")


def ps_tune_get(key_type: int, has_vals: bool) -> tuple[int, int]:
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().ps_tune_get(key_type, 1 if has_vals else 0, ctypes.byref(a), ctypes.byref(b)), "ps_tune_get")
    return a.value, b.value


def ps_selftest_level_pass_timeout(keys: torch.Tensor, vals: torch.Tensor | None, workspace: torch.Tensor,
                                   polls: int = 1 << 12, key_type: int | None = None, stream=None) -> None:
    """Queue the level-pass timeout self-test on ``keys`` (see include/powersort.h); then
    ps_stream_status() reports PS_ERR_TIMEOUT and the contents of ``keys`` are unspecified."""
    kt = _key_type(keys, key_type)
    _check_vals(vals, keys)
    _check(load().ps_selftest_level_pass_timeout(kt, _dev_ptr(keys, "keys"), _dev_ptr(vals, "vals"), keys.numel(),
                                                 int(polls), _dev_ptr(workspace, "workspace"),
                                                 _ws_bytes(workspace, keys), _stream_ptr(stream, keys.device)),
           "ps_selftest_level_pass_timeout")


def ps_selftest_wait_timeout(polls: int = 1 << 14, stream=None) -> None:
    """Queue the bounded-wait self-test (see include/powersort.h); then ps_stream_status()
    reports PS_ERR_TIMEOUT."""
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().ps_selftest_wait_timeout(int(polls), ctypes.c_void_p(stream.cuda_stream)), "ps_selftest_wait_timeout")
