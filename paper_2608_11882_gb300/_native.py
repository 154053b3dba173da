"""ctypes binding of libheatcg.so: the C ABI of include/heatcg.h under the same
names.  Argument marshalling only -- every step of the heat and CG paths runs in
the library's CUDA kernels.  Importing this module fails loudly when the
library has not been built; there is no fallback."""
from __future__ import annotations

import ctypes
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libheatcg.so"

HS_OK, HS_EINVAL, HS_ENOMEM, HS_ECUDA = 0, -1, -2, -3
HS_EUNSTABLE, HS_ENOCONV, HS_ETIMEOUT, HS_EBUSY, HS_ERANGE = -4, -5, -6, -7, -8
HS_F64, HS_F32 = 0, 1
HS_ALLOW_UNSTABLE, HS_EXACT_ROUNDING, HS_SCHED_FULL, HS_FIXED64, HS_VARKAPPA = 0x1, 0x2, 0x4, 0x8, 0x10
HS_FP64_PIPE = 0x20
HS_OP_STENCIL7, HS_OP_CSR = 0, 1
HS_SPMV_AUTO, HS_SPMV_ROWS, HS_SPMV_STAGED, HS_SPMV_TMA = 0, 1, 2, 3

_CODE_NAMES = {HS_EINVAL: "HS_EINVAL", HS_ENOMEM: "HS_ENOMEM", HS_ECUDA: "HS_ECUDA",
               HS_EUNSTABLE: "HS_EUNSTABLE", HS_ENOCONV: "HS_ENOCONV", HS_ETIMEOUT: "HS_ETIMEOUT",
               HS_EBUSY: "HS_EBUSY", HS_ERANGE: "HS_ERANGE"}


class HeatCGError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func}: {_CODE_NAMES.get(code, code)}: {msg}")
        self.code = code


class hs_heat_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("r", ctypes.c_double), ("flags", ctypes.c_uint32), ("dtype", ctypes.c_int32),
                ("tdepth", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("dev_buf0", ctypes.c_void_p), ("dev_buf1", ctypes.c_void_p)]


class hs_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("host", ctypes.c_int32)]


class hs_cg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("relres_recur", ctypes.c_double), ("relres_true", ctypes.c_double),
                ("refinements", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class hs_cg_mixed_opts(ctypes.Structure):
    _fields_ = [("inner_rtol", ctypes.c_double), ("max_inner", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"libheatcg.so is not built ({_LIB_PATH}); run "
                          "paper_2608_11882_gb300.build.build() on a machine with nvcc")
    lib = ctypes.CDLL(str(_LIB_PATH))
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "heat_create": [ctypes.POINTER(vp), ctypes.POINTER(hs_heat_desc)],
        "heat_device_bytes": [ctypes.POINTER(hs_heat_desc), ctypes.POINTER(ctypes.c_size_t)],
        "heat_buffer_bytes": [ctypes.POINTER(hs_heat_desc), ctypes.POINTER(ctypes.c_size_t)],
        "heat_upload": [vp, vp, ctypes.c_int],
        "heat_step": [vp, i64],
        "heat_interior": [vp],
        "heat_boundary": [vp],
        "heat_swap": [vp],
        "heat_read": [vp, vp, ctypes.c_int],
        "heat_steps_done": [vp, ctypes.POINTER(i64)],
        "heat_time_interior": [vp, ctypes.c_int],
        "heat_interior_time": [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)],
        "heat_get_tdepth": [vp, ctypes.POINTER(i32)],
        "heat_set_kchunk": [vp, i32],
        "heat_get_kchunk": [vp, ctypes.POINTER(i32)],
        "heat_batch_create_tiled": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                    ctypes.POINTER(i32), ctypes.POINTER(i32), i32, vp],
        "heat_destroy": [vp],
        "op_apply": [ctypes.POINTER(hs_op), vp, vp, vp],
        "cg_spmv": [ctypes.POINTER(hs_op), vp, vp, ctypes.c_int, ctypes.POINTER(dbl), vp],
        "heat_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64), i32, vp],
        "heat_batch_run": [vp, ctypes.c_int],
        "heat_batch_wait": [vp],
        "heat_batch_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "heat_batch_destroy": [vp],
        "heat_batch_set_wait_limit": [i64],
        "cg_create": [ctypes.POINTER(vp), ctypes.POINTER(hs_op), vp],
        "cg_create_mixed": [ctypes.POINTER(vp), ctypes.POINTER(hs_op), ctypes.POINTER(hs_cg_mixed_opts), vp],
        "cg_run": [vp, vp, vp, ctypes.c_int, dbl, i32, ctypes.POINTER(hs_cg_info)],
        "cg_destroy": [vp],
        "cg_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(hs_op), i32, vp],
        "cg_batch_run": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dbl, i32, ctypes.POINTER(hs_cg_info)],
        "cg_batch_destroy": [vp],
        "cg_solve": [ctypes.POINTER(hs_op), vp, vp, dbl, i32, ctypes.POINTER(hs_cg_info), vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.hs_last_error.restype = ctypes.c_char_p
    lib.hs_last_error.argtypes = []
    lib.hs_version.restype = ctypes.c_int
    lib.hs_launch_count.restype = ctypes.c_int64
    return lib


lib = _load()
LIB_PATH = _LIB_PATH


def last_error() -> str:
    return lib.hs_last_error().decode(errors="replace")


def check(rc: int, func: str, ok=(HS_OK,)) -> int:
    if rc not in ok:
        raise HeatCGError(rc, func, last_error())
    return rc


def launch_count() -> int:
    return int(lib.hs_launch_count())


# ---- same-name wrappers (pointers are ints: tensor.data_ptr() or ndarray.ctypes.data) ----

def heat_create(desc: hs_heat_desc) -> int:
    h = ctypes.c_void_p()
    check(lib.heat_create(ctypes.byref(h), ctypes.byref(desc)), "heat_create")
    return h.value


def heat_device_bytes(desc: hs_heat_desc) -> int:
    b = ctypes.c_size_t()
    check(lib.heat_device_bytes(ctypes.byref(desc), ctypes.byref(b)), "heat_device_bytes")
    return b.value


def heat_buffer_bytes(desc: hs_heat_desc) -> int:
    b = ctypes.c_size_t()
    check(lib.heat_buffer_bytes(ctypes.byref(desc), ctypes.byref(b)), "heat_buffer_bytes")
    return b.value


def heat_upload(h: int, ptr: int, src_is_device: bool) -> None:
    check(lib.heat_upload(h, ptr, int(bool(src_is_device))), "heat_upload")


def heat_step(h: int, n_steps: int) -> None:
    check(lib.heat_step(h, int(n_steps)), "heat_step")


def heat_interior(h: int) -> None:
    check(lib.heat_interior(h), "heat_interior")


def heat_boundary(h: int) -> None:
    check(lib.heat_boundary(h), "heat_boundary")


def heat_swap(h: int) -> None:
    check(lib.heat_swap(h), "heat_swap")


def heat_read(h: int, ptr: int, dst_is_device: bool) -> None:
    check(lib.heat_read(h, ptr, int(bool(dst_is_device))), "heat_read")


def heat_steps_done(h: int) -> int:
    s = ctypes.c_int64()
    check(lib.heat_steps_done(h, ctypes.byref(s)), "heat_steps_done")
    return s.value


def heat_time_interior(h: int, enable: bool) -> None:
    check(lib.heat_time_interior(h, int(bool(enable))), "heat_time_interior")


def heat_interior_time(h: int):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    check(lib.heat_interior_time(h, ctypes.byref(ms), ctypes.byref(n)), "heat_interior_time")
    return ms.value, n.value


def heat_get_tdepth(h: int) -> int:
    t = ctypes.c_int32()
    check(lib.heat_get_tdepth(h, ctypes.byref(t)), "heat_get_tdepth")
    return t.value


def heat_set_kchunk(h: int, planes: int) -> None:
    check(lib.heat_set_kchunk(h, int(planes)), "heat_set_kchunk")


def heat_get_kchunk(h: int) -> int:
    t = ctypes.c_int32()
    check(lib.heat_get_kchunk(h, ctypes.byref(t)), "heat_get_kchunk")
    return t.value


def heat_destroy(h: int) -> None:
    check(lib.heat_destroy(h), "heat_destroy")


def heat_batch_create(handles, steps, stream: int = 0, kz=None, tile_w=None) -> int:
    """kz: planes per work item for each grid, tile_w: column-tile width (64 or
    32) for each grid (0 or None: the library's choice)."""
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*handles)
    st = (ctypes.c_int64 * n)(*[int(s) for s in steps])
    b = ctypes.c_void_p()
    if kz is None and tile_w is None:
        check(lib.heat_batch_create(ctypes.byref(b), arr, st, n, stream), "heat_batch_create")
    else:
        kza = None if kz is None else (ctypes.c_int32 * n)(*[int(k) for k in kz])
        twa = None if tile_w is None else (ctypes.c_int32 * n)(*[int(w) for w in tile_w])
        check(lib.heat_batch_create_tiled(ctypes.byref(b), arr, st, kza, twa, n, stream),
              "heat_batch_create_tiled")
    return b.value


def heat_batch_run(b: int, use_graph: bool = True) -> None:
    check(lib.heat_batch_run(b, int(bool(use_graph))), "heat_batch_run")


def heat_batch_wait(b: int) -> None:
    check(lib.heat_batch_wait(b), "heat_batch_wait")


def heat_batch_info(b: int):
    lups, blocks = ctypes.c_int64(), ctypes.c_int32()
    check(lib.heat_batch_info(b, ctypes.byref(lups), ctypes.byref(blocks)), "heat_batch_info")
    return lups.value, blocks.value


def heat_batch_set_wait_limit(cycles: int) -> None:
    check(lib.heat_batch_set_wait_limit(int(cycles)), "heat_batch_set_wait_limit")


def heat_batch_destroy(b: int) -> None:
    check(lib.heat_batch_destroy(b), "heat_batch_destroy")


def op_apply(op: hs_op, p_ptr: int, y_ptr: int, stream: int = 0) -> None:
    check(lib.op_apply(ctypes.byref(op), p_ptr, y_ptr, stream), "op_apply")


def cg_spmv(op: hs_op, p_ptr: int, q_ptr: int, kernel: int = HS_SPMV_AUTO, stream: int = 0) -> float:
    """q = A p through one SpMV launch of the named kernel; returns p.q."""
    pq = ctypes.c_double()
    check(lib.cg_spmv(ctypes.byref(op), p_ptr, q_ptr, int(kernel), ctypes.byref(pq), stream), "cg_spmv")
    return pq.value


def cg_create(op: hs_op, stream: int = 0) -> int:
    c = ctypes.c_void_p()
    check(lib.cg_create(ctypes.byref(c), ctypes.byref(op), stream), "cg_create")
    return c.value


def cg_create_mixed(op: hs_op, inner_rtol: float = 0.0, max_inner: int = 0, stream: int = 0) -> int:
    c = ctypes.c_void_p()
    opts = hs_cg_mixed_opts(inner_rtol=inner_rtol, max_inner=max_inner, reserved=0)
    check(lib.cg_create_mixed(ctypes.byref(c), ctypes.byref(op), ctypes.byref(opts), stream),
          "cg_create_mixed")
    return c.value


def cg_run(c: int, b_ptr: int, x_ptr: int, host_buffers: bool, rtol: float, max_iter: int):
    info = hs_cg_info()
    rc = lib.cg_run(c, b_ptr, x_ptr, int(bool(host_buffers)), float(rtol), int(max_iter),
                    ctypes.byref(info))
    check(rc, "cg_run", ok=(HS_OK, HS_ENOCONV))
    return rc, info


def cg_batch_create(ops, stream: int = 0) -> int:
    n = len(ops)
    arr = (hs_op * n)(*ops)
    b = ctypes.c_void_p()
    check(lib.cg_batch_create(ctypes.byref(b), arr, n, stream), "cg_batch_create")
    return b.value


def cg_batch_run(b: int, b_ptrs, x_ptrs, rtol: float, max_iter: int):
    n = len(b_ptrs)
    bs = (ctypes.c_void_p * n)(*b_ptrs)
    xs = (ctypes.c_void_p * n)(*x_ptrs)
    infos = (hs_cg_info * n)()
    rc = lib.cg_batch_run(b, bs, xs, float(rtol), int(max_iter), infos)
    check(rc, "cg_batch_run", ok=(HS_OK, HS_ENOCONV))
    return rc, list(infos)


def cg_batch_destroy(b: int) -> None:
    check(lib.cg_batch_destroy(b), "cg_batch_destroy")


def cg_destroy(c: int) -> None:
    check(lib.cg_destroy(c), "cg_destroy")


def cg_solve(op: hs_op, b_ptr: int, x_ptr: int, rtol: float, max_iter: int, stream: int = 0):
    info = hs_cg_info()
    rc = lib.cg_solve(ctypes.byref(op), b_ptr, x_ptr, float(rtol), int(max_iter),
                      ctypes.byref(info), stream)
    check(rc, "cg_solve", ok=(HS_OK, HS_ENOCONV))
    return rc, info


# ---- allocation-free CG (cg_solve_noalloc) ----------------------------------------
HS_NOALLOC_MAX_N = 2097152
lib.cg_solve_noalloc.argtypes = [ctypes.POINTER(hs_op), ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_double, ctypes.c_int32, ctypes.POINTER(hs_cg_info),
                                 ctypes.c_void_p]
lib.cg_solve_noalloc.restype = ctypes.c_int


def cg_solve_noalloc(op: hs_op, b_ptr: int, x_ptr: int, rtol: float, max_iter: int,
                     stream: int = 0):
    """cg_solve without allocating: for callers that cannot allocate device
    memory while they solve (scratch comes from a fixed array in the library;
    at most HS_NOALLOC_MAX_N unknowns; overlapping calls race)."""
    info = hs_cg_info()
    rc = lib.cg_solve_noalloc(ctypes.byref(op), b_ptr, x_ptr, float(rtol), int(max_iter),
                              ctypes.byref(info), stream)
    check(rc, "cg_solve_noalloc", ok=(HS_OK, HS_ENOCONV))
    return rc, info
