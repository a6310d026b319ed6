"""Streaming host arrays through the GPU sort.

`HostSortPipeline` sorts a sequence of host arrays (pinned memory) with the device-driven
pipeline (`ps_sort_async_ws`): the copy-in of one array, the sort of another and the copy-out of
a third overlap.  The host link is the shared resource, so copies in each direction run in
submission order (every copy-in waits for the previous copy-in, every copy-out for the previous
copy-out); sorts run on per-slot streams.  `submit` only queues work; the returned event or
`synchronize()` waits for it.  All sorting runs in the library's kernels; this class only orders
copies and launches.
"""
from __future__ import annotations

import torch

from . import PS_TREE_POWERSORT, key_type_of, ps_sort_async_ws, ps_stream_status, ps_workspace_size


class HostSortPipeline:
    """Sort host arrays of up to ``n_max`` elements (keys of one key type, optional uint32
    payloads) with ``depth`` device buffer sets in flight."""

    def __init__(self, n_max: int, key_dtype: torch.dtype = torch.int32, with_vals: bool = True,
                 depth: int = 4, device=None, key_type: int | None = None, ordered_copies: bool = True):
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        probe = torch.empty(0, dtype=key_dtype)
        self.key_type = key_type_of(probe) if key_type is None else key_type
        self.n_max = int(n_max)
        self.with_vals = with_vals
        wsz = ps_workspace_size(self.key_type, with_vals, self.n_max)
        self._sets = []
        for _ in range(depth):
            k = torch.empty(self.n_max, dtype=key_dtype, device=self.device)
            v = torch.empty(self.n_max, dtype=torch.int32, device=self.device) if with_vals else None
            w = torch.empty(wsz, dtype=torch.uint8, device=self.device)
            self._sets.append((k, v, w, torch.cuda.Stream(self.device)))
        self.ordered_copies = ordered_copies
        self._next = 0
        self._last_in = None
        self._last_out = None

    def submit(self, keys_in: torch.Tensor, vals_in: torch.Tensor | None, keys_out: torch.Tensor,
               vals_out: torch.Tensor | None) -> torch.cuda.Event:
        """Queue copy-in, sort and copy-out of one host array (1-D CPU tensors, pinned for
        overlap; keys_out/vals_out may alias the inputs).  Returns the event that completes with
        the copy-out."""
        n = keys_in.numel()
        if n > self.n_max:
            raise ValueError(f"array of {n} elements exceeds the pipeline's n_max={self.n_max}")
        if (vals_in is None) != (not self.with_vals) or (vals_out is None) != (vals_in is None):
            raise ValueError("payloads must be given exactly when the pipeline was built with_vals")
        kb = self._sets[0][0].element_size()
        for buf, width, name in ((keys_in, kb, "keys_in"), (keys_out, kb, "keys_out"), (vals_in, 4, "vals_in"),
                                 (vals_out, 4, "vals_out")):
            if buf is None:
                continue
            if buf.is_cuda or not buf.is_contiguous() or buf.numel() != n or buf.element_size() != width:
                raise ValueError(f"{name} must be a contiguous host tensor of n = {n} elements of {width} bytes")
        k, v, w, st = self._sets[self._next]
        self._next = (self._next + 1) % len(self._sets)
        dk = k[:n]
        dv = v[:n] if v is not None else None
        with torch.cuda.stream(st):
            if self.ordered_copies and self._last_in is not None:
                st.wait_event(self._last_in)
            dk.copy_(keys_in, non_blocking=True)
            if dv is not None:
                dv.copy_(vals_in.view(torch.int32), non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(st)
            self._last_in = ev_in
            if n > 0:
                ps_sort_async_ws(dk, dv, w, tree=PS_TREE_POWERSORT, key_type=self.key_type, stream=st)
            if self.ordered_copies and self._last_out is not None:
                st.wait_event(self._last_out)
            keys_out.copy_(dk, non_blocking=True)
            if dv is not None:
                vals_out.view(torch.int32).copy_(dv, non_blocking=True)
            ev_out = torch.cuda.Event()
            ev_out.record(st)
            self._last_out = ev_out
        return ev_out

    def synchronize(self) -> None:
        """Wait for every queued array and raise if a sort reported a device-side error."""
        for _, _, _, st in self._sets:
            status = ps_stream_status(st)
            if status != 0:
                raise RuntimeError(f"device-side sort error {status}")
