"""Helpers for the GPU tests: skip when no CUDA device, build-on-demand of the
library, and the tolerances the parity tests use."""
import numpy as np
import pytest


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib():
    require_cuda()
    from paper_2608_11882_gb300.build import build
    build()
    import paper_2608_11882_gb300 as pkg
    return pkg


# FP64 gate: max |u_gpu - u_ref| / max |u_ref| <= 1e-12 (the FMA-contracted
# GPU update and the oracle's separately rounded one differ by about one ulp
# per step; over 1000 steps that stays below 1e-13).
F64_REL = 1e-12


def rel_max_err(a, ref):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - ref)) / np.max(np.abs(ref)))


def paper_criterion(a, ref):
    """Section 6.1.7: every |u_gpu - u_cpu| <= 1e-6 + 1e-5 |u_cpu|, no NaN/Inf."""
    a = np.asarray(a, dtype=np.float64)
    return bool(np.all(np.isfinite(a)) and np.all(np.abs(a - ref) <= 1e-6 + 1e-5 * np.abs(ref)))


def f32_bound(n_steps, max_u0):
    """Derived FP32 error bound against the FP64 oracle: for r <= 1/6 the update
    is a convex combination, so errors never grow; each step adds at most the
    rounding of ~9 float operations on values <= max|u0| (about 9 * 2^-24 *
    max|u0|), and the initial rounding adds 2^-24 max|u0|."""
    return (9 * n_steps + 1) * 2.0 ** -24 * max_u0
