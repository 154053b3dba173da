"""FP64 CPU oracle for the heat stencil and the CG solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2608_11882_gb300``) never imports, links or calls it, and the oracle
never imports the product library: the two share nothing but the seeded input
generators in ``workloads``.

The arithmetic lives in plain C (``heat_oracle.c``, ``cg_oracle.c``), compiled
with ``-O2 -ffp-contract=off`` so that every operation rounds once in the
written order.  This module only marshals numpy arrays.  Every function cites
the passage of the paper it follows; the C files hold the full statement.

Pins (tests that do not compare against any implementation): the exact
per-step decay of discrete sine modes, the 1x1x1 closed form, the maximum
principle and the instability above the stability bound, a dense Kronecker-sum
matrix power on tiny grids, a dense direct solve for CG, one-iteration
convergence on an eigenvector, the distinct-eigenvalue bound on 3x3x3, and
bitwise agreement of the CSR and matrix-free operators.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle.so"
_SOURCES = [_HERE / "heat_oracle.c", _HERE / "cg_oracle.c"]

OP_STENCIL7 = 0
OP_CSR = 1


def build(force: bool = False) -> Path:
    """Compile the oracle's C sources into ``oracle/_build/liboracle.so``."""
    _BUILD.mkdir(exist_ok=True)
    newest = max(s.stat().st_mtime for s in _SOURCES)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < newest:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
               "-fPIC", "-o", str(tmp)] + [str(s) for s in _SOURCES] + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("relres_recur", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("status", ctypes.c_int32),
                ("loop_seconds", ctypes.c_double)]


class _Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("n", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        # ORACLE_LIB names another build of these sources: the mutation tests
        # point it at copies with a planted mistake to show the pins catch it
        override = os.environ.get("ORACLE_LIB")
        lib = ctypes.CDLL(override if override else str(build()))
        dp = ctypes.c_void_p
        lib.oracle_heat_run.argtypes = [ctypes.c_int32] * 3 + [ctypes.c_double, ctypes.c_int64,
                                                                dp, dp, ctypes.c_int32]
        lib.oracle_heat_run.restype = ctypes.c_int
        lib.oracle_heat_run_timed.argtypes = lib.oracle_heat_run.argtypes + [dp]
        lib.oracle_heat_run_timed.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_heat_vk_run.argtypes = [ctypes.c_int32] * 3 + [ctypes.c_double, ctypes.c_int64,
                                                                   dp, dp, ctypes.c_int32,
                                                                   ctypes.c_double, ctypes.c_int32]
        lib.oracle_heat_vk_run.restype = ctypes.c_int
        lib.oracle_lap7_apply.argtypes = [ctypes.c_int32] * 3 + [dp, dp, ctypes.c_int32]
        lib.oracle_csr_spmv.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_int32]
        lib.oracle_dot.argtypes = [ctypes.c_int64, dp, dp]
        lib.oracle_dot.restype = ctypes.c_double
        lib.oracle_cg.argtypes = [ctypes.POINTER(_Op), dp, dp, ctypes.c_double, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.POINTER(_CgInfo)]
        lib.oracle_cg.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def heat_run(u0: np.ndarray, r: float, n_steps: int, threads: int = 1,
             return_seconds: bool = False):
    """Advance the interior field ``u0`` (shape (nz, ny, nx), x fastest) by
    ``n_steps`` explicit FTCS steps with zero Dirichlet boundary.

    Section 4, Eq. 4 in its constant-coefficient form u' = u + r (sum of six
    neighbours - 6u); boundary fixed at zero; the double buffer and pointer
    swap of Algorithm "1-GPU Baseline"; loop order of COMPUTE_SINGLE_GPU.
    With ``return_seconds`` also returns the wall time of the step loop alone.
    """
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    if u0.ndim != 3:
        raise ValueError("u0 must have shape (nz, ny, nx)")
    nz, ny, nx = u0.shape
    out = np.empty_like(u0)
    secs = ctypes.c_double(0.0)
    rc = _load().oracle_heat_run_timed(nx, ny, nz, float(r), int(n_steps), _ptr(u0), _ptr(out),
                                       int(threads), ctypes.addressof(secs))
    if rc != 0:
        raise ValueError(f"oracle_heat_run failed with {rc}")
    return (out, secs.value) if return_seconds else out


def heat_vk_run(u0: np.ndarray, r: float, n_steps: int, threads: int = 1,
                kappa_const: float = 0.0, with_source: bool = True) -> np.ndarray:
    """The paper's variable-coefficient update (Section 4, Eqs. 1-4):
    kappa = 0.5 + 0.45 sin sin sin, f = 1 + cos cos cos, dt = r h_min^2,
    u' = u + dt f + sum_d dt/(2 h_d^2) D_d with face-averaged D_d
    (D_x = (k[i+1]+k[i])(u[i+1]-u[i]) - (k[i]+k[i-1])(u[i]-u[i-1])).
    kappa_const > 0 makes kappa that constant; with_source=False drops f."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    nz, ny, nx = u0.shape
    out = np.empty_like(u0)
    rc = _load().oracle_heat_vk_run(nx, ny, nz, float(r), int(n_steps), _ptr(u0), _ptr(out),
                                    int(threads), float(kappa_const), int(bool(with_source)))
    if rc != 0:
        raise ValueError(f"oracle_heat_vk_run failed with {rc}")
    return out


def lap7_apply(p: np.ndarray, threads: int = 1) -> np.ndarray:
    """y = A p for the 7-point Dirichlet Laplacian (6 on the diagonal, -1 to
    each interior face neighbour) on the grid of ``p``'s shape (nz, ny, nx).
    Section 7.5: the CG operator; terms added in ascending column order."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    nz, ny, nx = p.shape
    y = np.empty_like(p)
    _load().oracle_lap7_apply(nx, ny, nz, _ptr(p), _ptr(y), int(threads))
    return y


def csr_spmv(rowptr: np.ndarray, col: np.ndarray, val: np.ndarray, p: np.ndarray,
             threads: int = 1) -> np.ndarray:
    """y = A p for a CSR matrix, row by row (Section 7.5, Algorithm "spmv" (a))."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
    n = rowptr.size - 1
    y = np.empty(n, dtype=np.float64)
    _load().oracle_csr_spmv(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(p), _ptr(y), int(threads))
    return y


def dot(a: np.ndarray, b: np.ndarray) -> float:
    """Sequential FP64 dot product in index order."""
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    return float(_load().oracle_dot(a.size, _ptr(a), _ptr(b)))


def cg_solve(b: np.ndarray, rtol: float, max_iter: int, *, shape=None, csr=None,
             x0: np.ndarray | None = None, threads: int = 1):
    """Unpreconditioned FP64 CG (Section 7.5; tolerance on ||r_k|| / ||b||).

    Give either ``shape=(nz, ny, nx)`` for the matrix-free 7-point operator or
    ``csr=(rowptr, col, val)``.  Returns (x, info) with info a dict of
    iters, relres_recur, relres_true and status (0 converged, 1 max_iter
    reached, -1 breakdown).
    """
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1).copy()
    op = _Op()
    keep = []
    if csr is not None:
        rowptr, col, val = (np.ascontiguousarray(csr[0], dtype=np.int32),
                            np.ascontiguousarray(csr[1], dtype=np.int32),
                            np.ascontiguousarray(csr[2], dtype=np.float64))
        keep += [rowptr, col, val]
        op.kind, op.n = OP_CSR, n
        op.rowptr, op.col, op.val = _ptr(rowptr), _ptr(col), _ptr(val)
    else:
        nz, ny, nx = shape
        if nx * ny * nz != n:
            raise ValueError("shape does not match b")
        op.kind, op.nx, op.ny, op.nz, op.n = OP_STENCIL7, nx, ny, nz, n
    info = _CgInfo()
    rc = _load().oracle_cg(ctypes.byref(op), _ptr(b), _ptr(x), float(rtol), int(max_iter),
                           int(threads), ctypes.byref(info))
    if rc != 0:
        raise ValueError(f"oracle_cg failed with {rc}")
    return x, {"iters": info.iters, "relres_recur": info.relres_recur,
               "relres_true": info.relres_true, "status": info.status,
               "loop_seconds": info.loop_seconds}


def sine_mode_factor(k: tuple, n: tuple, r: float) -> float:
    """Per-step amplification of the discrete sine mode prod_d sin(k_d pi x_d)
    under the constant-coefficient update of Section 4, Eq. 4, on an interior
    grid of n_d points per axis (h_d = 1/(n_d+1)):
        g = 1 - 4 r sum_d sin^2(k_d pi h_d / 2).
    It follows from the update being linear with a translation-invariant
    stencil whose eigenvectors, under zero Dirichlet data, are these modes.
    Used to compute full-size heat results point by point when the initial
    field is a sum of modes without noise."""
    return 1.0 - 4.0 * r * sum(np.sin(kd * np.pi / (nd + 1) / 2.0) ** 2 for kd, nd in zip(k, n))


def sine_modes_exact(modes, amps, shape, r: float, n_steps: int, points) -> np.ndarray:
    """Values after ``n_steps`` at the given interior points (array of (k, j, i)
    indices) of the field sum_m amps[m] prod_d sin(modes[m][d] pi x_d), where
    modes[m] = (kx, ky, kz) and shape = (nz, ny, nx).  Exact in real
    arithmetic; evaluated here in FP64."""
    nz, ny, nx = shape
    pts = np.asarray(points, dtype=np.int64).reshape(-1, 3)
    out = np.zeros(pts.shape[0])
    for (kx, ky, kz), a in zip(modes, amps):
        g = sine_mode_factor((kx, ky, kz), (nx, ny, nz), r)
        val = (a * g ** n_steps
               * np.sin(kx * np.pi * (pts[:, 2] + 1) / (nx + 1))
               * np.sin(ky * np.pi * (pts[:, 1] + 1) / (ny + 1))
               * np.sin(kz * np.pi * (pts[:, 0] + 1) / (nz + 1)))
        out += val
    return out
