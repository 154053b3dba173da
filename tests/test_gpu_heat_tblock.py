"""Temporal blocking (tdepth L >= 2: L steps of Section 4's update per pass
over HBM) against stepping one step at a time, and against the oracle."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, f32_bound, lib, rel_max_err
from workloads import heat_u0_single_mode

pytestmark = pytest.mark.gpu

DEPTHS = [2, 3, 4]
# (70, 90, 300), (43, 67, 263) and (40, 70, 384) hold blocks whose every
# computed point lies inside the interior (the unmasked form) beside edge
# blocks, several z-chunks and ragged tails; FP32 grids 384, 256 and 250 wide
# take the 34-thread rows (128-column tiles), the others 32-thread rows; (4, 2,
# 256) has fewer rows than one tile
SHAPES = [(1, 1, 1), (2, 3, 5), (33, 9, 17), (70, 3, 40), (40, 65, 31), (5, 100, 90),
          (70, 90, 300), (43, 67, 263), (40, 70, 384), (9, 30, 250), (4, 2, 256)]


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def run(pkg, u0, r, steps, dtype="f64", flags=0, tdepth=0):
    nz, ny, nx = u0.shape
    with pkg.Heat(nx, ny, nz, r, dtype=dtype, flags=flags, tdepth=tdepth) as h:
        h.upload(np.ascontiguousarray(u0, dtype=h.np_dtype))
        h.step(steps)
        assert h.steps_done == steps
        return h.read()


@pytest.mark.parametrize("tdepth", DEPTHS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_blocked_equals_stepwise_bitwise(pkg, tdepth, shape, dtype):
    """Same per-point arithmetic, so the blocked pass reproduces one-step
    stepping bit for bit (FP64 blocking computes on the FP64 pipe, so its
    one-step twin is an HS_FP64_PIPE handle); 19 steps leaves a remainder for
    every depth."""
    rng = np.random.default_rng(sum(shape) + tdepth)
    u0 = rng.uniform(-1, 1, size=shape)
    flags = pkg.HS_FP64_PIPE if dtype == "f64" else 0
    a = run(pkg, u0, 0.16, 19, dtype=dtype, flags=flags, tdepth=1)
    b = run(pkg, u0, 0.16, 19, dtype=dtype, tdepth=tdepth)
    assert np.array_equal(a, b)
    if dtype == "f64":   # and the default one-step (exact-sum) arithmetic agrees within the gate
        c = run(pkg, u0, 0.16, 19, dtype=dtype, tdepth=1)
        assert rel_max_err(c, b) <= F64_REL


@pytest.mark.parametrize("tdepth", DEPTHS)
@pytest.mark.parametrize("shape", [(45, 38, 29), (150, 50, 40)])
def test_blocked_exact_rounding_equals_oracle_bitwise(pkg, tdepth, shape):
    """One rounding per operation in the written order: the oracle bit for
    bit (the 150-wide grid holds unmasked interior blocks)."""
    u0 = heat_u0_single_mode(*shape, seed=12)
    ref = oracle.heat_run(u0, 0.1, 25)
    assert np.array_equal(run(pkg, u0, 0.1, 25, flags=pkg.HS_EXACT_ROUNDING, tdepth=tdepth), ref)


def test_small_workload_blocked(pkg):
    u0 = heat_u0_single_mode(64, 64, 64)
    ref = oracle.heat_run(u0, 0.1, 100, threads=oracle.max_threads())
    assert rel_max_err(run(pkg, u0, 0.1, 100, tdepth=4), ref) <= F64_REL
    got32 = run(pkg, u0.astype(np.float32), 0.1, 100, dtype="f32", tdepth=3)
    assert float(np.max(np.abs(got32 - ref))) <= f32_bound(100, float(np.max(np.abs(u0))))


def test_bad_tdepth(pkg):
    for bad in (5, 6, 8, -1):
        with pytest.raises(pkg.HeatCGError):
            pkg.Heat(8, 8, 8, 0.1, tdepth=bad)
    with pytest.raises(pkg.HeatCGError):
        pkg.Heat(8, 8, 8, 0.1, flags=pkg.HS_SCHED_FULL, tdepth=2)


def test_default_depth(pkg):
    """The library's choice: two steps per pass for FP32 (HBM-bound), one step
    per pass for FP64, for the one-step schedule and for the
    variable-coefficient problem."""
    with pkg.Heat(8, 8, 8, 0.1, dtype="f32") as h:
        assert h.tdepth == 2
    with pkg.Heat(8, 8, 8, 0.1) as h:
        assert h.tdepth == 1
    with pkg.Heat(8, 8, 8, 0.1, dtype="f32", flags=pkg.HS_SCHED_FULL) as h:
        assert h.tdepth == 1
    with pkg.Heat(8, 8, 8, 0.01, dtype="f32", flags=pkg.HS_VARKAPPA) as h:
        assert h.tdepth == 1
