"""Parity of the FIXED64 heat path (FP64 interface, 64-bit fixed-point state,
exact integer steps with one rounding per point) against the FP64 oracle and
the exact modal decay of Section 4's update, through the C ABI."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, lib, rel_max_err
from workloads import heat_u0_modes, heat_u0_single_mode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def run_fx(pkg, u0, r, steps, extra=0, tdepth=0):
    nz, ny, nx = u0.shape
    with pkg.Heat(nx, ny, nz, r, flags=pkg.HS_FIXED64 | extra, tdepth=tdepth) as h:
        h.upload(np.ascontiguousarray(u0, dtype=np.float64))
        h.step(steps)
        return h.read()


def test_small_workload_parity(pkg):
    u0 = heat_u0_single_mode(64, 64, 64)
    ref = oracle.heat_run(u0, 0.1, 100, threads=oracle.max_threads())
    assert rel_max_err(run_fx(pkg, u0, 0.1, 100), ref) <= F64_REL


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 2), (33, 9, 17), (1, 40, 1), (70, 1, 3),
                                   (2, 2, 2), (3, 37, 65), (11, 130, 33)])
def test_odd_shapes(pkg, shape):
    rng = np.random.default_rng(sum(shape) + 1)
    u0 = rng.uniform(-1, 1, size=shape)
    ref = oracle.heat_run(u0, 0.15, 23)
    assert rel_max_err(run_fx(pkg, u0, 0.15, 23), ref) <= F64_REL


def test_interior_plus_boundary_equals_full_step_kernel(pkg):
    u0 = heat_u0_single_mode(45, 38, 29, seed=9)
    assert np.array_equal(run_fx(pkg, u0, 0.12, 17, tdepth=1),
                          run_fx(pkg, u0, 0.12, 17, pkg.HS_SCHED_FULL))


def test_sine_mode_closer_to_exact_decay_than_fp64(pkg):
    """Exact integer steps with one rounding per point: the decayed mode is
    within a few units of 2^-E of g^N times the encoded mode."""
    nz, ny, nx = 21, 19, 23
    k = (3, 2, 5)
    xs, ys, zs = [(np.arange(m) + 1) / (m + 1) for m in (nx, ny, nz)]
    mode = (np.sin(k[2] * np.pi * zs)[:, None, None] * np.sin(k[1] * np.pi * ys)[None, :, None]
            * np.sin(k[0] * np.pi * xs)[None, None, :])
    r, steps = 0.15, 300
    g = oracle.sine_mode_factor(k, (nx, ny, nz), r)
    out = run_fx(pkg, mode, r, steps)
    assert np.max(np.abs(out - g ** steps * mode)) <= 2e-14


def test_full_size_against_oracle_few_steps(pkg):
    u0, _, _ = heat_u0_modes(512, 512, 512)
    ref = oracle.heat_run(u0, 0.15, 4, threads=oracle.max_threads())
    assert rel_max_err(run_fx(pkg, u0, 0.15, 4), ref) <= F64_REL


def test_full_size_1000_steps_closed_form(pkg):
    u0, modes, amps = heat_u0_modes(512, 512, 512, noise=0.0)
    got = run_fx(pkg, u0, 0.15, 1000)
    pts = np.random.default_rng(1).integers(0, 512, size=(4000, 3))
    expect = oracle.sine_modes_exact(modes, amps, u0.shape, 0.15, 1000, pts)
    vals = got[pts[:, 0], pts[:, 1], pts[:, 2]]
    assert np.max(np.abs(vals - expect)) <= F64_REL * np.max(np.abs(u0))


@pytest.mark.parametrize("scale", [1e-12, 1e12, 3.0e-300, 1e300])
def test_magnitudes(pkg, scale):
    u0 = heat_u0_single_mode(20, 16, 12, seed=3) * scale
    ref = oracle.heat_run(u0, 0.1, 40)
    assert rel_max_err(run_fx(pkg, u0, 0.1, 40), ref) <= F64_REL


def test_zero_field_and_reupload(pkg):
    z = np.zeros((6, 7, 8))
    assert not run_fx(pkg, z, 0.1, 5).any()
    u0 = heat_u0_single_mode(8, 7, 6, seed=4)
    straight = oracle.heat_run(u0, 0.1, 50)
    with pkg.Heat(8, 7, 6, 0.1, flags=pkg.HS_FIXED64) as h:
        mid = h.upload(u0).step(20).read()
        out = h.upload(mid).step(30).read()
    assert rel_max_err(out, straight) <= F64_REL


def test_errors(pkg):
    from paper_2608_11882_gb300._native import HS_EINVAL, HS_ERANGE
    for kw in [dict(dtype="f32", flags=pkg.HS_FIXED64),
               dict(flags=pkg.HS_FIXED64 | pkg.HS_ALLOW_UNSTABLE),
               dict(flags=pkg.HS_FIXED64 | pkg.HS_EXACT_ROUNDING)]:
        with pytest.raises(pkg.HeatCGError) as e:
            pkg.Heat(4, 4, 4, 0.1, **kw)
        assert e.value.code == HS_EINVAL
    bad = np.ones((4, 4, 4))
    bad[1, 2, 3] = np.nan
    with pkg.Heat(4, 4, 4, 0.1, flags=pkg.HS_FIXED64) as h:
        h.upload(bad).step(1)
        with pytest.raises(pkg.HeatCGError) as e:
            h.read()
        assert e.value.code == HS_ERANGE


@pytest.mark.parametrize("tdepth", [1, 2, 3, 4])
def test_temporal_depths_against_oracle(pkg, tdepth):
    for shape in [(37, 29, 41), (150, 50, 40)]:   # (nx, ny, nz); the second holds unmasked interior blocks
        u0 = heat_u0_single_mode(*shape, seed=6)
        ref = oracle.heat_run(u0, 0.13, 29)
        assert rel_max_err(run_fx(pkg, u0, 0.13, 29, tdepth=tdepth), ref) <= F64_REL
