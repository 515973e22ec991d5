"""Many lattices advanced together through the C ABI batch calls.

All lattices of a batch share the storage type (FP32 or 16-bit); their
shapes and parameters may differ.  One kernel launch per step covers every
tile of every lattice, replayed from a CUDA graph.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _abi
from .solver import Solver, diag_dict


class Batch:
    def __init__(self, solvers: list[Solver], stream: torch.cuda.Stream | None = None,
                 seg_rows: int = 0, warps_per_block: int = 0, graph_steps: int = 8, row_fetch: int = 0):
        if not solvers:
            raise ValueError("empty batch")
        self.L = _abi.load()
        self.solvers = list(solvers)
        self.stream = stream or solvers[0].stream
        n = len(self.solvers)
        nb = C.c_size_t()
        _abi.check(self.L.lb_batch_required_bytes(n, C.byref(nb)))
        self.buffer = torch.empty(int(nb.value), dtype=torch.uint8, device=self.solvers[0].device)
        arr = (C.c_void_p * n)(*[s.ctx.value for s in self.solvers])
        h = C.c_void_p()
        _abi.check(self.L.lb_batch_create(arr, n, C.c_void_p(self.buffer.data_ptr()), self.buffer.numel(),
                                          C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.set_launch(seg_rows, warps_per_block, graph_steps, row_fetch)

    def set_launch(self, seg_rows: int = 0, warps_per_block: int = 0, graph_steps: int = 8,
                   row_fetch: int = 0) -> None:
        """row_fetch: 0 keep, 1 plain loads, 3 TMA ring read in place, 4 the
        same with three ring stages (FP32), 5 one persistent launch per
        step() call with every work item resident (neighbour progress flags
        instead of launch boundaries)."""
        _abi.check(self.L.lb_batch_set_launch(self.h, int(seg_rows), int(warps_per_block), int(graph_steps),
                                              int(row_fetch)))

    def set_segments(self, seg_rows: list | None) -> None:
        """Rows per z-segment of each lattice (0: the common value; None:
        every lattice back to the common value)."""
        if seg_rows is None:
            _abi.check(self.L.lb_batch_set_segments(self.h, None))
            return
        if len(seg_rows) != len(self.solvers):
            raise ValueError("one value per lattice")
        arr = (C.c_int32 * len(seg_rows))(*[int(v) for v in seg_rows])
        _abi.check(self.L.lb_batch_set_segments(self.h, arr))

    def occupancy(self) -> tuple:
        """(resident warps of the batched step, work items of one step)."""
        r, n = C.c_int32(), C.c_int32()
        _abi.check(self.L.lb_batch_get_occupancy(self.h, C.byref(r), C.byref(n)))
        return r.value, n.value

    def step(self, n: int = 1) -> None:
        _abi.check(self.L.lb_batch_step(self.h, int(n)))

    def diag(self) -> list:
        """Diagnostics of every lattice (one download for the whole batch)."""
        out = (_abi.lb_diag * len(self.solvers))()
        _abi.check(self.L.lb_batch_diagnostics(self.h, C.cast(out, C.c_void_p)))
        return [diag_dict(d) for d in out]

    def close(self) -> None:
        if getattr(self, "h", None):
            self.L.lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nodes(self) -> int:
        return sum(s.n for s in self.solvers)
