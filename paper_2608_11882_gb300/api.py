"""Convenience classes over the C ABI: Heat (a resident field), Operator and
CG.  They take numpy arrays (host) or torch tensors (host or device) and pass
raw pointers and the current torch CUDA stream to libheatcg.so.  Torch is used
for device memory and streams only; no arithmetic of the method runs here."""
from __future__ import annotations

import numpy as np

from . import _native as native
from ._native import (HS_ALLOW_UNSTABLE, HS_EXACT_ROUNDING, HS_F32, HS_F64, HS_FIXED64, HS_FP64_PIPE,
                      HS_OP_CSR, HS_OP_STENCIL7, HS_SCHED_FULL, HS_VARKAPPA, HeatCGError)

__all__ = ["Heat", "HeatBatch", "Operator", "CG", "CGBatch", "native", "HeatCGError", "HS_F64", "HS_F32",
           "HS_ALLOW_UNSTABLE", "HS_EXACT_ROUNDING", "HS_SCHED_FULL", "HS_FIXED64", "HS_VARKAPPA",
           "HS_FP64_PIPE", "HS_OP_STENCIL7", "HS_OP_CSR"]

_DTYPES = {"f64": (HS_F64, np.float64), "f32": (HS_F32, np.float32)}


def _torch():
    import torch
    return torch


def _stream_handle(stream) -> int:
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _buffer(arr, np_dtype, count: int):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor of count elements."""
    if isinstance(arr, np.ndarray):
        if arr.dtype != np_dtype or not arr.flags["C_CONTIGUOUS"] or arr.size != count:
            raise ValueError(f"expected a C-contiguous {np.dtype(np_dtype).name} array of {count} elements")
        return arr.ctypes.data, False, arr
    torch = _torch()
    if isinstance(arr, torch.Tensor):
        want = torch.float64 if np_dtype == np.float64 else torch.float32
        if arr.dtype != want or not arr.is_contiguous() or arr.numel() != count:
            raise ValueError(f"expected a contiguous {want} tensor of {count} elements")
        return arr.data_ptr(), bool(arr.is_cuda), arr
    raise TypeError("expected a numpy array or a torch tensor")


class Heat:
    """A resident heat field (heat_create / heat_upload / heat_step / heat_read)."""

    def __init__(self, nx: int, ny: int, nz: int, r: float, dtype: str = "f64", flags: int = 0,
                 stream=None, tdepth=0, buffers=None):
        """tdepth: steps per pass (0 = the library's default: 2 for FP32, 1
        otherwise; 1..4), or "auto" for
        the autotuner's cached or freshly measured choice for this shape (the
        depth, and the Interior kernel's planes per block).
        buffers: optional pair of caller-owned CUDA tensors for the two padded
        time levels (each at least ``Heat.buffer_bytes(...)`` bytes); the
        handle keeps references to them while it lives."""
        self.shape = (nz, ny, nx)
        self.dtype_code, self.np_dtype = _DTYPES[dtype]
        self.dtype = dtype
        tuned = None
        if tdepth == "auto":
            from .autotune import Tuner
            arith = ("fixed64" if flags & HS_FIXED64 else "f64exact" if flags & HS_EXACT_ROUNDING
                     else "f64pipe" if flags & HS_FP64_PIPE else dtype)
            tuned = ({"depth": 1, "kc_factor": 1.0} if flags & (HS_VARKAPPA | HS_SCHED_FULL)
                     else Tuner().best(arith, self.shape))
            tdepth = tuned["depth"]
        self.stream = _stream_handle(stream)
        desc = native.hs_heat_desc(nx=nx, ny=ny, nz=nz, r=r, flags=flags, dtype=self.dtype_code,
                                   tdepth=tdepth, stream=self.stream)
        self._buffers = None
        if buffers is not None:
            b0, b1 = buffers
            if not (b0.is_cuda and b1.is_cuda):
                raise ValueError("caller-owned heat buffers must be CUDA tensors")
            desc.dev_buf0, desc.dev_buf1 = b0.data_ptr(), b1.data_ptr()
            self._buffers = (b0, b1)
        self.handle = native.heat_create(desc)
        if tuned is not None and tuned["kc_factor"] != 1.0 and tuned["depth"] == 1:
            lib_kc = native.heat_get_kchunk(self.handle)
            native.heat_set_kchunk(self.handle, max(4, int(round(lib_kc * tuned["kc_factor"]))))

    @property
    def kchunk(self) -> int:
        """Planes per block of the one-step Interior kernel (heat_get_kchunk)."""
        return native.heat_get_kchunk(self.handle)

    @kchunk.setter
    def kchunk(self, planes: int) -> None:
        native.heat_set_kchunk(self.handle, planes)

    @staticmethod
    def buffer_bytes(nx: int, ny: int, nz: int, dtype: str = "f64") -> int:
        """Bytes of one padded time-level buffer (heat_buffer_bytes)."""
        desc = native.hs_heat_desc(nx=nx, ny=ny, nz=nz, r=0.0, flags=0, dtype=_DTYPES[dtype][0])
        return native.heat_buffer_bytes(desc)

    @property
    def count(self) -> int:
        return self.shape[0] * self.shape[1] * self.shape[2]

    def upload(self, u) -> "Heat":
        ptr, dev, keep = _buffer(u, self.np_dtype, self.count)
        native.heat_upload(self.handle, ptr, dev)
        self._keep = keep   # the copy may still be in flight on the stream
        return self

    def step(self, n_steps: int) -> "Heat":
        native.heat_step(self.handle, n_steps)
        return self

    def interior(self):
        native.heat_interior(self.handle)

    def boundary(self):
        native.heat_boundary(self.handle)

    def swap(self):
        native.heat_swap(self.handle)

    def read(self, out=None):
        """Interior field as a new numpy array (nz, ny, nx), or into ``out``
        (numpy array or torch tensor, host or device)."""
        if out is None:
            out = np.empty(self.shape, dtype=self.np_dtype)
        ptr, dev, _ = _buffer(out, self.np_dtype, self.count)
        native.heat_read(self.handle, ptr, dev)
        return out

    @property
    def tdepth(self) -> int:
        """Steps per pass the handle runs with (1: Interior + Boundary every step)."""
        return native.heat_get_tdepth(self.handle)

    @property
    def steps_done(self) -> int:
        return native.heat_steps_done(self.handle)

    def time_interior(self, enable: bool = True):
        """Bracket every Interior launch of ``step`` with timing events."""
        native.heat_time_interior(self.handle, enable)
        return self

    def interior_time(self):
        """(mean milliseconds, launches) of the Interior launches timed since
        the last call; waits for the last one."""
        return native.heat_interior_time(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            native.heat_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HeatBatch:
    """Several Heat handles advanced together by one persistent launch
    (heat_batch_create / heat_batch_run / heat_batch_wait)."""

    def __init__(self, heats, steps, stream=None, kz=None, tile_w=None):
        """kz: planes per work item and tile_w: column-tile width (64 or 32),
        each a list with one value per grid (0 = the library's choice) or None;
        kz="auto" takes both from the autotuner, per grid size class."""
        self.heats = list(heats)
        self.steps = [int(s) for s in steps]
        self.stream = _stream_handle(stream)
        if kz == "auto":
            from .autotune import Tuner
            t = Tuner()
            picks = [t.best_batch(h.dtype, h.shape) for h in self.heats]
            kz = [p["kz"] for p in picks]
            tile_w = [p["tile_w"] for p in picks]
        self.kz, self.tile_w = kz, tile_w
        self.handle = native.heat_batch_create([h.handle for h in self.heats], self.steps, self.stream,
                                               kz=kz, tile_w=tile_w)

    def run(self, use_graph: bool = True) -> "HeatBatch":
        native.heat_batch_run(self.handle, use_graph)
        return self

    def wait(self) -> None:
        native.heat_batch_wait(self.handle)

    @property
    def lups(self) -> int:
        return native.heat_batch_info(self.handle)[0]

    @property
    def blocks(self) -> int:
        return native.heat_batch_info(self.handle)[1]

    def close(self):
        if getattr(self, "handle", None):
            native.heat_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """The CG operator: matrix-free 7-point stencil or CSR arrays (torch CUDA
    tensors, or numpy arrays that cg_create copies to the device)."""

    def __init__(self, op: native.hs_op, keep=()):
        self.op = op
        self._keep = keep

    @classmethod
    def stencil(cls, nx: int, ny: int, nz: int) -> "Operator":
        return cls(native.hs_op(kind=HS_OP_STENCIL7, nx=nx, ny=ny, nz=nz, n=nx * ny * nz, nnz=0,
                                dtype=HS_F64, host=0))

    @classmethod
    def csr(cls, rowptr, col, val) -> "Operator":
        n = len(rowptr) - 1
        nnz = len(col)
        if isinstance(rowptr, np.ndarray):
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
            ptrs, host = (rowptr.ctypes.data, col.ctypes.data, val.ctypes.data), 1
        else:
            torch = _torch()
            if rowptr.dtype != torch.int32 or col.dtype != torch.int32 or val.dtype != torch.float64:
                raise ValueError("CSR tensors must be int32, int32, float64")
            ptrs, host = (rowptr.data_ptr(), col.data_ptr(), val.data_ptr()), 0 if rowptr.is_cuda else 1
        op = native.hs_op(kind=HS_OP_CSR, nx=0, ny=0, nz=0, n=n, nnz=nnz, rowptr=ptrs[0], col=ptrs[1],
                          val=ptrs[2], dtype=HS_F64, host=host)
        return cls(op, (rowptr, col, val))

    @property
    def n(self) -> int:
        return int(self.op.n)

    def apply(self, p, y, stream=None):
        """y = A p for torch CUDA tensors of n float64 values."""
        pp, pd, _ = _buffer(p, np.float64, self.n)
        yp, yd, _ = _buffer(y, np.float64, self.n)
        if not (pd and yd):
            raise ValueError("op_apply takes device tensors")
        native.op_apply(self.op, pp, yp, _stream_handle(stream))
        return y

    _SPMV_KERNELS = {"auto": native.HS_SPMV_AUTO, "rows": native.HS_SPMV_ROWS,
                     "staged": native.HS_SPMV_STAGED, "tma": native.HS_SPMV_TMA}

    def spmv(self, p, q, kernel: str = "auto", stream=None) -> float:
        """q = A p through one launch of the SpMV kernel a CG iteration runs
        ("auto": the one cg_run picks; "rows", "staged", "tma"); returns p.q."""
        pp, pd, _ = _buffer(p, np.float64, self.n)
        qp, qd, _ = _buffer(q, np.float64, self.n)
        if not (pd and qd):
            raise ValueError("cg_spmv takes device tensors")
        return native.cg_spmv(self.op, pp, qp, self._SPMV_KERNELS[kernel], _stream_handle(stream))


class CG:
    """A CG context with resident workspace (cg_create / cg_run / cg_destroy)."""

    def __init__(self, op: Operator, stream=None, mixed: bool = False, inner_rtol: float = 0.0,
                 max_inner: int = 0):
        """mixed=True: FP64 iterative refinement around FP32 CG (cg_create_mixed)."""
        self.op = op
        self.stream = _stream_handle(stream)
        if mixed:
            self.handle = native.cg_create_mixed(op.op, inner_rtol, max_inner, self.stream)
        else:
            self.handle = native.cg_create(op.op, self.stream)

    def run(self, b, x=None, rtol: float = 1e-8, max_iter: int = 10000):
        """Solve A x = b.  b and x are numpy arrays (host path: the library
        copies them) or torch CUDA tensors.  x (if given) is the start vector
        and receives the solution.  Returns (x, info dict)."""
        n = self.op.n
        if x is None:
            if isinstance(b, np.ndarray):
                x = np.zeros(n)
            else:
                x = _torch().zeros(n, dtype=_torch().float64, device=b.device)
        bp, bd, _ = _buffer(b, np.float64, n)
        xp, xd, _ = _buffer(x, np.float64, n)
        if bd != xd:
            raise ValueError("b and x must both be host or both be device buffers")
        rc, info = native.cg_run(self.handle, bp, xp, not bd, rtol, max_iter)
        return x, {"iters": info.iters, "status": info.status, "relres_recur": info.relres_recur,
                   "relres_true": info.relres_true, "refinements": info.refinements,
                   "converged": rc == native.HS_OK}

    def close(self):
        if getattr(self, "handle", None):
            native.cg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CGBatch:
    """Several CG systems solved together (cg_batch_create / cg_batch_run)."""

    def __init__(self, ops, stream=None):
        self.ops = list(ops)
        self.stream = _stream_handle(stream)
        self.handle = native.cg_batch_create([o.op for o in self.ops], self.stream)

    def run(self, bs, xs=None, rtol: float = 1e-8, max_iter: int = 10000):
        """bs, xs: lists of torch CUDA float64 tensors (xs are start vectors and
        receive the solutions; zeros when omitted).  Returns (xs, infos)."""
        torch = _torch()
        if xs is None:
            xs = [torch.zeros_like(b) for b in bs]
        for o, b, x in zip(self.ops, bs, xs):
            if b.numel() != o.n or x.numel() != o.n or not (b.is_cuda and x.is_cuda):
                raise ValueError("each b and x must be a CUDA tensor of its system's size")
        rc, infos = native.cg_batch_run(self.handle, [b.data_ptr() for b in bs],
                                        [x.data_ptr() for x in xs], rtol, max_iter)
        return xs, [{"iters": i.iters, "status": i.status, "relres_recur": i.relres_recur,
                     "relres_true": i.relres_true, "converged": i.status == native.HS_OK}
                    for i in infos]

    def close(self):
        if getattr(self, "handle", None):
            native.cg_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
