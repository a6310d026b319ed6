"""Seeded synthetic inputs shared by the GPU tests, the benchmark and the CPU oracle.

The generators only draw random data (run lengths, run contents, orientation); none of the
sorting method's arithmetic lives here.  The C++ source is ``gen.cpp``; it is compiled into
``libpsgen.so`` next to this file on first use (or by ``__graft_entry__.build()``).

Workload shapes (sizes are parameters so tests can scale them down):

* ``runs_i32``      run lengths uniform in [1, max_len] (default 2*sqrt(n)), sorted uniform
                    int32 contents, 25% of runs descending.
* ``perm_i32``      a uniformly random permutation (runs of length about 2).
* ``pareto_u64``    uint64 keys from 1000 distinct values, Pareto(1.2) run lengths clipped
                    to n/10, 25% descending.
* ``segmented_i32`` segment sizes log-uniform in [2^8, 2^20], each segment like ``runs_i32``.
* ``pareto_f32``    float32 bit patterns with ~1% NaN/+-0, Pareto(1.5) run lengths.
* ``random_runs_i32`` the paper's random-runs inputs: a random permutation whose segments of
                    geometric length (mean ``mean_len``) are sorted.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cpp")
_LIB = os.path.join(_HERE, "libpsgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.cpp into libpsgen.so (host code; portable C++17, no arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, dbl, i32, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_void_p)
            lib.psgen_runs32.argtypes = [u64, i64, i64, dbl, i32, vp, vp]
            lib.psgen_perm32.argtypes = [u64, i64, vp, vp]
            lib.psgen_random_runs32.argtypes = [u64, i64, dbl, vp, vp]
            lib.psgen_pareto64.argtypes = [u64, i64, dbl, i64, i64, dbl, vp, vp]
            lib.psgen_pareto_f32.argtypes = [u64, i64, dbl, dbl, dbl, vp, vp]
            lib.psgen_segment_sizes.argtypes = [u64, i64, dbl, dbl, vp]
            lib.psgen_segmented_runs32.argtypes = [u64, i64, vp, dbl, i32, vp, vp]
            for f in (lib.psgen_runs32, lib.psgen_perm32, lib.psgen_random_runs32,
                      lib.psgen_pareto64, lib.psgen_pareto_f32, lib.psgen_segment_sizes,
                      lib.psgen_segmented_runs32):
                f.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def runs_i32(n: int, seed: int, max_len: int | None = None, desc_frac: float = 0.25,
             signed: bool = True):
    """Runs of length uniform in [1, max_len] (default floor(2*sqrt(n))), sorted contents."""
    if max_len is None:
        max_len = max(1, int(2 * np.sqrt(n)))
    keys = np.empty(n, dtype=np.int32 if signed else np.uint32)
    vals = np.empty(n, dtype=np.uint32)
    _load().psgen_runs32(seed, n, max_len, desc_frac, 1 if signed else 0, _ptr(keys), _ptr(vals))
    return keys, vals


def perm_i32(n: int, seed: int):
    keys = np.empty(n, dtype=np.int32)
    vals = np.empty(n, dtype=np.uint32)
    _load().psgen_perm32(seed, n, _ptr(keys), _ptr(vals))
    return keys, vals


def random_runs_i32(n: int, seed: int, mean_len: float):
    keys = np.empty(n, dtype=np.int32)
    vals = np.empty(n, dtype=np.uint32)
    _load().psgen_random_runs32(seed, n, float(mean_len), _ptr(keys), _ptr(vals))
    return keys, vals


def pareto_u64(n: int, seed: int, alpha: float = 1.2, distinct: int = 1000,
               max_len: int | None = None, desc_frac: float = 0.25):
    if max_len is None:
        max_len = max(1, n // 10)
    keys = np.empty(n, dtype=np.uint64)
    vals = np.empty(n, dtype=np.uint32)
    _load().psgen_pareto64(seed, n, alpha, distinct, max_len, desc_frac, _ptr(keys), _ptr(vals))
    return keys, vals


def pareto_f32(n: int, seed: int, alpha: float = 1.5, special_frac: float = 0.01,
               desc_frac: float = 0.25):
    """float32 keys returned as their uint32 bit patterns."""
    keys = np.empty(n, dtype=np.uint32)
    vals = np.empty(n, dtype=np.uint32)
    _load().psgen_pareto_f32(seed, n, alpha, special_frac, desc_frac, _ptr(keys), _ptr(vals))
    return keys, vals


def segment_offsets(count: int, seed: int, lo_exp: float = 8.0, hi_exp: float = 20.0):
    sizes = np.empty(count, dtype=np.int64)
    _load().psgen_segment_sizes(seed, count, lo_exp, hi_exp, _ptr(sizes))
    offsets = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    return offsets


def segmented_i32(count: int, seed: int, lo_exp: float = 8.0, hi_exp: float = 20.0,
                  desc_frac: float = 0.25, offsets: np.ndarray | None = None):
    """Returns (keys, vals, offsets[count+1])."""
    if offsets is None:
        offsets = segment_offsets(count, seed, lo_exp, hi_exp)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = int(offsets[-1])
    keys = np.empty(n, dtype=np.int32)
    vals = np.empty(n, dtype=np.uint32)
    _load().psgen_segmented_runs32(seed, count, _ptr(offsets), desc_frac, 1, _ptr(keys), _ptr(vals))
    return keys, vals, offsets


def config_small(seed: int = 1):
    """n = 2^17 int32 keys with uint32 payload, runs uniform in [1, 2*sqrt(n)], 25% descending."""
    return runs_i32(1 << 17, seed)
