"""The default FP64 arithmetic (FP64 fields, exact fixed-point neighbour sum,
one FP64 fused multiply-add per point) against the FP64 oracle of Section 4's
update, over the field ranges where it converts and where it falls back to
the FP64 pipe, and against the all-FP64-pipe form of the same handle."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, lib, rel_max_err
from workloads import heat_u0_modes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def run(pkg, u0, r, steps, flags=0, sched_full=False):
    nz, ny, nx = u0.shape
    if sched_full:
        flags |= pkg.HS_SCHED_FULL
    with pkg.Heat(nx, ny, nz, r, flags=flags) as h:
        h.upload(np.ascontiguousarray(u0, dtype=np.float64))
        h.step(steps)
        return h.read()


@pytest.mark.parametrize("scale", [1.0, 1e-280, 1e-300, 1e-305, 1e300, 1e307])
def test_scales_against_oracle(pkg, scale):
    """1e-280 and 1e300 convert (largest exponent field inside [70, 2040]);
    1e-300, 1e-305 and 1e307 take the FP64 pipe."""
    rng = np.random.default_rng(7)
    u0 = rng.uniform(-1, 1, size=(19, 23, 37)) * scale
    ref = oracle.heat_run(u0, 0.15, 30)
    got = run(pkg, u0, 0.15, 30)
    assert rel_max_err(got, ref) <= F64_REL


def test_wide_dynamic_range(pkg):
    """Magnitudes log-uniform over 40 decades with random signs: values far below
    the maximum drop out of the neighbour sum, within the stated error bound."""
    rng = np.random.default_rng(11)
    shape = (21, 34, 47)
    u0 = rng.choice([-1.0, 1.0], size=shape) * 10.0 ** rng.uniform(-40, 0, size=shape)
    ref = oracle.heat_run(u0, 0.1, 40)
    got = run(pkg, u0, 0.1, 40)
    assert rel_max_err(got, ref) <= F64_REL
    # per step at most r * 24 * 2^-57 max|u| from the sum plus two roundings of each result
    bound = 40 * (0.1 * 24 * 2.0**-57 + 4 * 2.0**-53) * float(np.max(np.abs(u0)))
    assert float(np.max(np.abs(got - ref))) <= bound


@pytest.mark.parametrize("shape,steps", [((1, 1, 1), 50), ((1, 1, 1), 210), ((1, 1, 1), 400),
                                         ((3, 3, 3), 1500), ((3, 3, 3), 2100)])
def test_decay_across_the_conversion_threshold(pkg, shape, steps):
    """Small grids decay geometrically (a 1x1x1 grid by 1 - 6r per step, a 3^3
    grid by about 0.72) from 1 to below 1e-300 and on to 0, so a run switches
    from the conversion to the FP64 pipe part way."""
    u0 = np.full(shape, 0.75)
    ref = oracle.heat_run(u0, 0.16, steps)
    got = run(pkg, u0, 0.16, steps)
    if np.max(np.abs(ref)) == 0:
        assert np.max(np.abs(got)) == 0
    else:
        assert rel_max_err(got, ref) <= F64_REL


def test_non_finite_values_propagate_like_fp64(pkg):
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1, 1, size=(9, 10, 11))
    u0[4, 5, 6] = np.nan
    u0[1, 2, 3] = np.inf
    ref = oracle.heat_run(u0, 0.1, 5)
    got = run(pkg, u0, 0.1, 5)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(np.isinf(got), np.isinf(ref))
    fin = np.isfinite(ref)
    assert rel_max_err(got[fin], ref[fin]) <= F64_REL


def test_unstable_growth(pkg):
    """r > 1/6 grows the highest mode; the tracked maximum follows it up."""
    n = 12
    s = np.sin(n * np.pi * (np.arange(n) + 1) / (n + 1))
    mode = s[:, None, None] * s[None, :, None] * s[None, None, :]
    ref = oracle.heat_run(mode, 0.2, 300)
    got = run(pkg, mode, 0.2, 300, flags=pkg.HS_ALLOW_UNSTABLE)
    assert np.max(np.abs(ref)) > 1e10
    assert rel_max_err(got, ref) <= F64_REL


def test_long_run_at_benchmark_distribution(pkg):
    """1000 steps at r = 0.15 on the benchmark's field recipe, 128^3."""
    u0, _, _ = heat_u0_modes(128, 128, 128)
    ref = oracle.heat_run(u0, 0.15, 1000, threads=oracle.max_threads())
    got = run(pkg, u0, 0.15, 1000)
    err = rel_max_err(got, ref)
    assert err <= F64_REL
    assert rel_max_err(run(pkg, u0, 0.15, 1000, flags=pkg.HS_FP64_PIPE), ref) <= F64_REL


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 5), (3, 37, 65), (40, 65, 31), (17, 130, 129)])
def test_split_full_and_pipe_agree(pkg, shape):
    """Interior + Boundary equals the full-step kernel bit for bit (same
    arithmetic, same per-step maxima); the FP64-pipe form agrees within the gate."""
    rng = np.random.default_rng(sum(shape))
    u0 = rng.uniform(-1, 1, size=shape)
    a = run(pkg, u0, 0.14, 21)
    b = run(pkg, u0, 0.14, 21, sched_full=True)
    assert np.array_equal(a, b)
    c = run(pkg, u0, 0.14, 21, flags=pkg.HS_FP64_PIPE)
    assert rel_max_err(a, c) <= F64_REL
    assert rel_max_err(a, oracle.heat_run(u0, 0.14, 21)) <= F64_REL


def test_flag_errors(pkg):
    for kw in (dict(dtype="f32", flags=pkg.HS_FP64_PIPE), dict(flags=pkg.HS_FP64_PIPE | pkg.HS_FIXED64)):
        with pytest.raises(pkg.HeatCGError):
            pkg.Heat(4, 4, 4, 0.1, **kw)


@pytest.mark.parametrize("dtype,flags", [("f64", 0), ("f64", "HS_FIXED64"), ("f32", 0)])
def test_side_stream_boundary_equals_full_step(pkg, dtype, flags):
    """A grid of 2^22 points or more runs each step's Boundary kernel on a side
    stream beside the Interior kernel; the result equals the one-kernel full
    step bit for bit (disjoint planes, the same per-step maxima)."""
    flags = getattr(pkg, flags) if flags else 0
    nz, ny, nx = 163, 161, 166   # 4,356,478 points, ragged against every tile
    rng = np.random.default_rng(23)
    u0 = rng.uniform(-1, 1, size=(nz, ny, nx))
    out = []
    for extra in (0, pkg.HS_SCHED_FULL):
        with pkg.Heat(nx, ny, nz, 0.13, dtype=dtype, flags=flags | extra) as h:
            h.upload(u0.astype(np.float64 if dtype == "f64" else np.float32))
            h.step(7)
            out.append(h.read())
    assert np.array_equal(out[0], out[1])
    if dtype == "f64":
        assert rel_max_err(out[0], oracle.heat_run(u0, 0.13, 7, threads=oracle.max_threads())) <= F64_REL


def test_split_entry_points_and_interior_timing(pkg):
    """heat_boundary + heat_interior + heat_swap per step equal heat_step bit
    for bit (on a grid where heat_step runs the two kernels side by side); with
    timing on, heat_step records one Interior duration per step, and reading
    the record clears it."""
    nz, ny, nx = 161, 163, 166
    u0 = np.random.default_rng(29).uniform(-1, 1, size=(nz, ny, nx))
    with pkg.Heat(nx, ny, nz, 0.12) as a:
        a.upload(u0)
        a.time_interior(True)
        a.step(5)
        ms, n = a.interior_time()
        assert n == 5 and ms > 0.0
        assert a.interior_time() == (0.0, 0)
        a.time_interior(False)
        a.step(1)
        assert a.interior_time() == (0.0, 0)
        ra = a.read()
    with pkg.Heat(nx, ny, nz, 0.12) as b:
        b.upload(u0)
        for _ in range(6):
            b.boundary()
            b.interior()
            b.swap()
        rb = b.read()
    assert np.array_equal(ra, rb)
