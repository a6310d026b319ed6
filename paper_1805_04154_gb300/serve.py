"""Continuous-batching sort service on one GPU.

Requests (host tensors of keys, optional 32-bit payload) are packed back to back into one of a
few fixed device arena slots and sorted by a single device-driven segmented call
(``ps_sort_async_bounded_ws``, no host round trip) per slot (each request is one segment, so each result
is exactly what ``ps_sort`` gives for that request alone).  The slots rotate through three CUDA streams, so the host-to-device copies of one batch,
the sort of another and the device-to-host copies of a third overlap on the GPU; a request that
arrives while earlier batches are on the GPU joins the next batch as soon as a slot frees up.

Admission is by device memory: the slots (keys, payloads and the segmented workspace for
``max_batch_keys`` keys each) are allocated once and their total stays within
``budget_bytes``; a request larger than a slot is refused at submission.

A request's latency is measured from ``submit`` to the moment its result is back in host
memory.  Every sorting step runs in the library's kernels through the C ABI; this module only
moves bytes, keeps the schedule and records latencies.
"""
from __future__ import annotations

import collections
import ctypes
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import PS_KEY_F32, PS_KEY_I32, PS_KEY_U32, PS_KEY_U64, _check, load, ps_workspace_size

_KEY_BYTES = {PS_KEY_I32: 4, PS_KEY_U32: 4, PS_KEY_U64: 8, PS_KEY_F32: 4}


@dataclass
class Request:
    rid: int
    keys: torch.Tensor          # host keys (contiguous; pinned memory gives asynchronous copies)
    vals: torch.Tensor | None   # host 32-bit payload or None
    out_keys: torch.Tensor      # where the sorted keys go (the input tensors unless given)
    out_vals: torch.Tensor | None
    t_submit: float = 0.0
    t_done: float = 0.0
    done: threading.Event = field(default_factory=threading.Event)
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class _Slot:
    def __init__(self, idx: int, cap: int, kdt, with_vals: bool, ws_bytes: int, dev):
        self.idx = idx
        self.dk = torch.empty(cap, dtype=kdt, device=dev)
        self.dv = torch.empty(cap, dtype=torch.int32, device=dev) if with_vals else None
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        self.hoff = torch.empty(cap + 1, dtype=torch.int64, pin_memory=True)
        self.doff = torch.empty(cap + 1, dtype=torch.int64, device=dev)
        self.reqs: list = []
        self.done_event = None


class SortServer:
    """Continuous-batching powersort service.

    key_type: one of PS_KEY_*; all requests of a server share it.
    budget_bytes: device memory the server may hold (all arena slots together).
    max_batch_keys: keys one slot (one batch, one launch sequence) holds; also the largest request.
    slots: arena slots (2-4; three let copy-in, sort and copy-out of different batches overlap).
    """

    def __init__(self, key_type: int, budget_bytes: int = 64 << 30, max_batch_keys: int = 1 << 25,
                 slots: int = 3, device: int | None = None, with_vals: bool = True):
        load()
        if key_type not in _KEY_BYTES:
            raise ValueError(f"unknown key type {key_type}")
        self.kt = key_type
        self.kb = _KEY_BYTES[key_type]
        self.kdt = {4: torch.int32, 8: torch.int64}[self.kb]
        self.with_vals = with_vals
        self.dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        ws_bytes = ps_workspace_size(key_type, with_vals, max_batch_keys, True)
        slot_bytes = max_batch_keys * (self.kb + (4 if with_vals else 0) + 8) + ws_bytes
        nslots = int(min(slots, budget_bytes // slot_bytes))
        if nslots < 1:
            raise ValueError("budget_bytes cannot hold one arena slot of max_batch_keys keys")
        self.cap = int(max_batch_keys)
        self.budget = int(budget_bytes)
        self.held_bytes = nslots * slot_bytes
        self.h2d = torch.cuda.Stream(self.dev)
        self.compute = torch.cuda.Stream(self.dev)
        self.d2h = torch.cuda.Stream(self.dev)
        with torch.cuda.device(self.dev):
            self._free = collections.deque(_Slot(i, self.cap, self.kdt, with_vals, ws_bytes, self.dev)
                                           for i in range(nslots))
        torch.cuda.synchronize(self.dev)
        self._pending = collections.deque()
        self._busy = collections.deque()
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._stop = False
        self._next_id = 0
        self._outstanding = 0
        self.batches = 0
        self.completed: list[Request] = []
        self._launcher = threading.Thread(target=self._launch_loop, name="powersort-launch", daemon=True)
        self._completer = threading.Thread(target=self._complete_loop, name="powersort-complete", daemon=True)
        self._launcher.start()
        self._completer.start()

    # ---------------------------------------------------------------- public API
    def submit(self, keys: torch.Tensor, vals: torch.Tensor | None = None,
               out_keys: torch.Tensor | None = None, out_vals: torch.Tensor | None = None) -> Request:
        """Queue one sort of host tensors (pinned memory gives asynchronous copies).  The result
        goes to out_keys/out_vals, or back into keys/vals when those are not given.  Returns a
        Request whose ``done`` event is set when the result is in host memory."""
        t_submit = time.perf_counter()
        if keys.device.type != "cpu" or not keys.is_contiguous() or keys.element_size() != self.kb:
            raise TypeError("keys must be a contiguous CPU tensor of the server's key width")
        if self.with_vals and (vals is None or vals.numel() != keys.numel() or vals.element_size() != 4):
            raise ValueError("this server carries a 32-bit payload per key")
        if keys.numel() > self.cap:
            raise ValueError(f"request of {keys.numel()} keys exceeds the arena slot ({self.cap} keys)")
        for buf, width, name in ((out_keys, self.kb, "out_keys"), (out_vals if self.with_vals else None, 4, "out_vals")):
            if buf is not None and (buf.device.type != "cpu" or not buf.is_contiguous()
                                    or buf.numel() != keys.numel() or buf.element_size() != width):
                raise ValueError(f"{name} must be a contiguous CPU tensor shaped like the request")
        r = Request(0, keys, vals if self.with_vals else None,
                    keys if out_keys is None else out_keys,
                    (vals if out_vals is None else out_vals) if self.with_vals else None, t_submit)
        with self._cv:
            r.rid = self._next_id
            self._next_id += 1
            self._outstanding += 1
            self._pending.append(r)
            self._cv.notify_all()
        return r

    def drain(self, timeout: float | None = None) -> None:
        """Wait until every submitted request is done; raise if the device reported an error for
        any batch since the last drain (the sorts run without host round trips, so device-side
        errors are collected here)."""
        with self._cv:
            ok = self._cv.wait_for(lambda: self._outstanding == 0, timeout)
        if not ok:
            raise TimeoutError("server did not drain")
        _check(load().ps_stream_status(ctypes.c_void_p(self.compute.cuda_stream)), "SortServer batch")

    def close(self) -> None:
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._launcher.join()
        self._completer.join()

    # ---------------------------------------------------------------- internals
    def _launch_loop(self) -> None:
        torch.cuda.set_device(self.dev)
        while True:
            with self._cv:
                self._cv.wait_for(lambda: self._stop or (self._pending and self._free))
                if self._stop and not self._pending:
                    return
                slot = self._free.popleft()
                reqs, n = [], 0
                while self._pending and n + self._pending[0].keys.numel() <= self.cap:
                    r = self._pending.popleft()
                    reqs.append(r)
                    n += r.keys.numel()
            try:
                self._launch(slot, reqs, n)
            except Exception as e:  # report on every request of the batch
                for r in reqs:
                    r.error = str(e)
                    r.t_done = time.perf_counter()
                    r.done.set()
                with self._cv:
                    self._free.append(slot)
                    self._outstanding -= len(reqs)
                    self._cv.notify_all()
                continue
            with self._cv:
                self._busy.append(slot)
                self._cv.notify_all()

    def _launch(self, slot: _Slot, reqs: list, n: int) -> None:
        off = slot.hoff.numpy()
        count = len(reqs)
        off[0] = 0
        np.cumsum([r.keys.numel() for r in reqs], out=off[1:count + 1])
        with torch.cuda.stream(self.h2d):
            slot.doff[:count + 1].copy_(slot.hoff[:count + 1], non_blocking=True)
            for r, a, e in zip(reqs, off[:count], off[1:count + 1]):
                slot.dk[a:e].copy_(r.keys.view(self.kdt), non_blocking=True)
                if slot.dv is not None:
                    slot.dv[a:e].copy_(r.vals.view(torch.int32), non_blocking=True)
            h2d_done = torch.cuda.Event()
            h2d_done.record(self.h2d)
        self.compute.wait_event(h2d_done)
        # device-driven segmented sort: queued without a host round trip, so this thread goes on
        # to the next batch while the GPU copies and sorts this one; the batch's longest request
        # bounds the level passes it needs
        longest = max(r.keys.numel() for r in reqs)
        st = load().ps_sort_async_bounded_ws(self.kt, ctypes.c_void_p(slot.dk.data_ptr()),
                                             None if slot.dv is None else ctypes.c_void_p(slot.dv.data_ptr()), n,
                                             ctypes.c_void_p(slot.doff.data_ptr()), count, max(longest, 1),
                                             ctypes.c_void_p(slot.ws.data_ptr()), slot.ws.numel(),
                                             ctypes.c_void_p(self.compute.cuda_stream))
        _check(st, "ps_sort_async_bounded_ws")
        sort_done = torch.cuda.Event()
        sort_done.record(self.compute)
        self.d2h.wait_event(sort_done)
        with torch.cuda.stream(self.d2h):
            for r, a, e in zip(reqs, off[:count], off[1:count + 1]):
                r.out_keys.view(self.kdt).copy_(slot.dk[a:e], non_blocking=True)
                if slot.dv is not None:
                    r.out_vals.view(torch.int32).copy_(slot.dv[a:e], non_blocking=True)
            slot.done_event = torch.cuda.Event()
            slot.done_event.record(self.d2h)
        slot.reqs = reqs
        self.batches += 1

    def _complete_loop(self) -> None:
        torch.cuda.set_device(self.dev)
        while True:
            with self._cv:
                self._cv.wait_for(lambda: self._busy or (self._stop and self._outstanding == 0))
                if not self._busy:
                    return
                slot = self._busy[0]
            err = None
            try:
                slot.done_event.synchronize()
            except Exception as e:  # a CUDA error: report it on the batch's requests, keep serving
                err = str(e)
            t = time.perf_counter()
            for r in slot.reqs:
                r.error = err
                r.t_done = t
                r.done.set()
            with self._cv:
                self._busy.popleft()
                self.completed.extend(slot.reqs)
                self._outstanding -= len(slot.reqs)
                slot.reqs = []
                self._free.append(slot)
                self._cv.notify_all()


def latency_stats(reqs) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1000.0
    keys = sum(r.keys.numel() for r in reqs)
    t0 = min(r.t_submit for r in reqs)
    t1 = max(r.t_done for r in reqs)
    return {"requests": len(reqs), "keys": int(keys), "wall_s": t1 - t0,
            "keys_per_s": keys / (t1 - t0), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}
