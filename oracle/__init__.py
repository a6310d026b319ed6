"""CPU oracle for powersort / peeksort (Munro & Wild, arXiv 1805.04154).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``; the GPU library never imports, links or calls it, and the
two share no code.  The arithmetic lives in ``powersort_oracle.cpp`` (plain sequential C++);
this module only marshals numpy arrays through ctypes.

Parity status of each function (what pins it; see tests/test_oracle_*.py):

* ``detect_runs``        hand-worked examples of the run convention (Sec. 2), exhaustive
                         property checks on all short sequences over a 3-letter alphabet.
* ``node_power``         Fig. 1's printed powers, closed form for 2^q equal runs, the
                         31-bit formulation (Appendix B), range bound 1..floor(lg n)+1.
* ``powersort``          std::stable_sort (output), Powersort theorem bound, OPT (interval DP)
                         as a lower bound, Cartesian-tree corollary, the paper's printed
                         average merge cost on random-runs inputs (Sec. 5.3).
* ``peeksort``           Fig. 1 left tree cost, Peeksort theorem bound, OPT lower bound.
* ``opt_cost``           brute force over all binary trees for tiny r.
* ``stable_sort``        numpy's stable argsort on the same keys.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "powersort_oracle.cpp")
_LIB = os.path.join(_HERE, "libpsoracle.so")
_lock = threading.Lock()
_lib = None

KT = {"i32": 0, "u32": 1, "u64": 2, "f32": 3}
_DT = {"i32": np.int32, "u32": np.uint32, "u64": np.uint64, "f32": np.uint32}


def build(force: bool = False) -> str:
    """Compile the oracle (portable host C++17)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, i32, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
            lib.ps_oracle_detect_runs.argtypes = [i32, vp, i64, vp, vp]
            lib.ps_oracle_detect_runs.restype = i64
            lib.ps_oracle_node_power.argtypes = [i64, i64, i64, i64]
            lib.ps_oracle_node_power.restype = i32
            lib.ps_oracle_node_power_bits.argtypes = [i64, i64, i64, i64]
            lib.ps_oracle_node_power_bits.restype = i32
            lib.ps_oracle_powersort.argtypes = [i32, vp, vp, i64, i64] + [vp] * 8
            lib.ps_oracle_powersort.restype = i64
            lib.ps_oracle_sort_segmented.argtypes = [i32, vp, vp, vp, i64, vp, vp, vp, vp, vp]
            lib.ps_oracle_sort_segmented.restype = i64
            lib.ps_oracle_cartesian_parent.argtypes = [vp, i64, vp]
            lib.ps_oracle_cartesian_parent.restype = i32
            lib.ps_oracle_powersort_cost.argtypes = [vp, i64, vp, vp]
            lib.ps_oracle_powersort_cost.restype = u64
            lib.ps_oracle_peeksort.argtypes = [i32, vp, vp, i64, vp]
            lib.ps_oracle_peeksort.restype = u64
            lib.ps_oracle_peeksort_cost.argtypes = [vp, i64, vp]
            lib.ps_oracle_peeksort_cost.restype = u64
            lib.ps_oracle_opt_cost.argtypes = [vp, i64]
            lib.ps_oracle_opt_cost.restype = u64
            lib.ps_oracle_stable_sort.argtypes = [i32, vp, vp, i64]
            lib.ps_oracle_stable_sort.restype = None
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _keys(keys: np.ndarray, kt: str) -> np.ndarray:
    k = np.ascontiguousarray(keys)
    if kt == "f32" and k.dtype == np.float32:
        k = k.view(np.uint32)
    if k.dtype != _DT[kt]:
        raise TypeError(f"keys dtype {k.dtype} does not match key type {kt}")
    return k


def detect_runs(keys: np.ndarray, kt: str = "i32"):
    """Greedy runs (Sec. 2; ExtendRunRight of Alg. 2).  Returns (starts[r+1], desc[r])."""
    k = _keys(keys, kt)
    n = k.size
    starts = np.empty(n + 1, dtype=np.int64)
    desc = np.empty(max(n, 1), dtype=np.uint8)
    r = _load().ps_oracle_detect_runs(KT[kt], _p(k), n, _p(starts), _p(desc))
    return starts[: r + 1].copy(), desc[:r].copy()


def node_power(s1: int, e1: int, e2: int, n: int) -> int:
    """Definition "Node Power" for runs [s1, e1), [e1, e2) of an array of length n."""
    return int(_load().ps_oracle_node_power(s1, e1, e2, n))


def node_power_bits(s1: int, e1: int, e2: int, n: int) -> int:
    return int(_load().ps_oracle_node_power_bits(s1, e1, e2, n))


class PowersortResult:
    __slots__ = ("keys", "vals", "starts", "desc", "power", "node_parent", "leaf_parent",
                 "leaf_depth", "merges", "cost", "r")


def powersort(keys: np.ndarray, vals: np.ndarray | None = None, kt: str = "i32",
              min_run: int = 1) -> PowersortResult:
    """Alg. 2 on copies of (keys, vals); returns the sorted arrays and the full trace."""
    k = _keys(keys, kt).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    n = k.size
    cap = n + 2
    # the C code writes every entry it defines (r+1 or r of them); np.empty keeps untouched
    # capacity unallocated
    starts = np.empty(cap, np.int64)
    desc = np.empty(cap, np.uint8)
    power = np.empty(cap, np.int32)
    npar = np.empty(cap, np.int64)
    lpar = np.empty(cap, np.int64)
    ldep = np.empty(cap, np.int32)
    merges = np.empty(3 * cap, np.int64)
    cost = ctypes.c_uint64(0)
    r = _load().ps_oracle_powersort(KT[kt], _p(k), _p(v), n, min_run, _p(starts), _p(desc),
                                    _p(power), _p(npar), _p(lpar), _p(ldep), _p(merges),
                                    ctypes.byref(cost))
    res = PowersortResult()
    res.keys, res.vals, res.r = k, v, int(r)
    res.starts = starts[: r + 1].copy()
    res.desc = desc[:r].copy()
    res.power = power[: r + 1].copy()
    res.node_parent = npar[: r + 1].copy()
    res.leaf_parent = lpar[:r].copy()
    res.leaf_depth = ldep[:r].copy()
    res.merges = merges[: 3 * max(r - 1, 0)].reshape(-1, 3).copy()
    res.cost = int(cost.value)
    return res


def sort_segmented(keys: np.ndarray, vals: np.ndarray | None, offsets: np.ndarray,
                   kt: str = "i32"):
    """Every segment sorted by Alg. 2 on its own.  Returns (keys, vals, starts, desc, power,
    leaf_depth, cost) with the per-run arrays concatenated over segments (power 0 on the
    boundary between two segments)."""
    k = _keys(keys, kt).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    count = off.size - 1
    n = int(off[-1] - off[0])
    cap = n + 2
    starts = np.zeros(cap, np.int64)
    desc = np.zeros(cap, np.uint8)
    power = np.zeros(cap, np.int32)
    ldep = np.zeros(cap, np.int32)
    cost = ctypes.c_uint64(0)
    R = _load().ps_oracle_sort_segmented(KT[kt], _p(k), _p(v), _p(off), count, _p(starts),
                                         _p(desc), _p(power), _p(ldep), ctypes.byref(cost))
    return (k, v, starts[: R + 1].copy(), desc[:R].copy(), power[: R + 1].copy(),
            ldep[:R].copy(), int(cost.value))


def cartesian_parent(power: np.ndarray):
    """Parent of every boundary in the min-Cartesian tree of the powers (Corollary)."""
    p = np.ascontiguousarray(power, dtype=np.int32)
    r = p.size - 1
    parent = np.full(r + 1, -1, np.int64)
    rc = _load().ps_oracle_cartesian_parent(_p(p), r, _p(parent))
    return parent, rc


def powersort_cost(lengths) -> tuple[int, np.ndarray, np.ndarray]:
    """Alg. 2 on run lengths alone: (M, leaf depths, powers)."""
    L = np.ascontiguousarray(lengths, dtype=np.int64)
    r = L.size
    depth = np.zeros(max(r, 1), np.int32)
    power = np.zeros(r + 1, np.int32)
    c = _load().ps_oracle_powersort_cost(_p(L), r, _p(depth), _p(power))
    return int(c), depth[:r].copy(), power


def peeksort(keys: np.ndarray, vals: np.ndarray | None = None, kt: str = "i32"):
    """Alg. 1 on copies; returns (keys, vals, cost, merges)."""
    k = _keys(keys, kt).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    m = ctypes.c_int64(0)
    c = _load().ps_oracle_peeksort(KT[kt], _p(k), _p(v), k.size, ctypes.byref(m))
    return k, v, int(c), int(m.value)


def peeksort_cost(lengths) -> tuple[int, np.ndarray]:
    L = np.ascontiguousarray(lengths, dtype=np.int64)
    depth = np.zeros(max(L.size, 1), np.int32)
    c = _load().ps_oracle_peeksort_cost(_p(L), L.size, _p(depth))
    return int(c), depth[: L.size].copy()


def opt_cost(lengths) -> int:
    L = np.ascontiguousarray(lengths, dtype=np.int64)
    return int(_load().ps_oracle_opt_cost(_p(L), L.size))


def stable_sort(keys: np.ndarray, vals: np.ndarray | None = None, kt: str = "i32"):
    k = _keys(keys, kt).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    _load().ps_oracle_stable_sort(KT[kt], _p(k), _p(v), k.size)
    return k, v


def entropy_bits(lengths) -> float:
    """H(L_1/n, ..., L_r/n) in bits (Sec. 2), in float64."""
    L = np.asarray(lengths, dtype=np.float64)
    n = L.sum()
    p = L / n
    return float(-(p * np.log2(p)).sum())
