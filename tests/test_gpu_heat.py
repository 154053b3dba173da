"""Parity of the CUDA heat path (Interior + Boundary kernels, Section 6.1
Algorithms INTERIOR/BOUNDARY; update of Section 4, Eq. 4) against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, f32_bound, lib, paper_criterion, rel_max_err, require_cuda
from workloads import heat_u0_modes, heat_u0_single_mode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def run_gpu(pkg, u0, r, steps, dtype="f64", flags=0):
    nz, ny, nx = u0.shape
    with pkg.Heat(nx, ny, nz, r, dtype=dtype, flags=flags) as h:
        h.upload(np.ascontiguousarray(u0, dtype=h.np_dtype))
        h.step(steps)
        return h.read()


def test_small_workload_parity(pkg):
    """64^3 interior, h = 1/65, r = 0.1, 100 steps, u0 = sin sin sin + 0.01 noise."""
    u0 = heat_u0_single_mode(64, 64, 64)
    ref = oracle.heat_run(u0, 0.1, 100, threads=oracle.max_threads())
    got = run_gpu(pkg, u0, 0.1, 100)
    assert rel_max_err(got, ref) <= F64_REL
    assert paper_criterion(got, ref)


def test_small_workload_exact_rounding_is_bitwise(pkg):
    u0 = heat_u0_single_mode(64, 64, 64)
    ref = oracle.heat_run(u0, 0.1, 100, threads=oracle.max_threads())
    got = run_gpu(pkg, u0, 0.1, 100, flags=pkg.HS_EXACT_ROUNDING)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 2), (33, 9, 17), (1, 40, 1), (70, 1, 3),
                                   (2, 2, 2), (3, 37, 65), (11, 130, 33)])
def test_odd_shapes(pkg, shape):
    rng = np.random.default_rng(sum(shape))
    u0 = rng.uniform(-1, 1, size=shape)
    ref = oracle.heat_run(u0, 0.15, 23)
    assert np.array_equal(run_gpu(pkg, u0, 0.15, 23, flags=pkg.HS_EXACT_ROUNDING), ref)
    assert rel_max_err(run_gpu(pkg, u0, 0.15, 23), ref) <= F64_REL


@pytest.mark.parametrize("exact", [False, True])
def test_interior_plus_boundary_equals_full_step_kernel(pkg, exact):
    u0 = heat_u0_single_mode(45, 38, 29, seed=9)
    base = pkg.HS_EXACT_ROUNDING if exact else 0
    split = run_gpu(pkg, u0, 0.12, 17, flags=base)
    full = run_gpu(pkg, u0, 0.12, 17, flags=base | pkg.HS_SCHED_FULL)
    assert np.array_equal(split, full)


def test_step_parts_equal_step(pkg):
    u0 = heat_u0_single_mode(20, 21, 22, seed=4)
    with pkg.Heat(20, 21, 22, 0.1) as a, pkg.Heat(20, 21, 22, 0.1) as b:
        a.upload(u0).step(3)
        b.upload(u0)
        for _ in range(3):
            b.boundary()
            b.interior()
            b.swap()
        assert b.steps_done == 3
        assert np.array_equal(a.read(), b.read())


def test_zero_steps_and_device_upload(pkg):
    torch = require_cuda()
    u0 = heat_u0_single_mode(16, 8, 4, seed=2)
    with pkg.Heat(16, 8, 4, 0.1) as h:
        h.upload(torch.from_numpy(u0).cuda())
        assert np.array_equal(h.read(), u0)
        h.step(0)
        out = torch.empty(4 * 8 * 16, dtype=torch.float64, device="cuda")
        h.read(out)
        assert np.array_equal(out.cpu().numpy().reshape(u0.shape), u0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(9, 7, 13), (12, 10, 64), (3, 5, 1)])
def test_pinned_host_buffers(pkg, dtype, shape):
    """Pinned host tensors are read and written by the re-layout kernel
    through their mapped device address (pageable arrays by a strided copy):
    the same field either way, rows whose bytes are or are not a multiple of
    16 alike, and after steps the same result as the pageable path."""
    torch = require_cuda()
    nz, ny, nx = shape
    u0 = heat_u0_single_mode(nx, ny, nz, seed=17)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    pinned = torch.from_numpy(u0).to(tdt).pin_memory()
    back = torch.empty_like(pinned).pin_memory()
    with pkg.Heat(nx, ny, nz, 0.12, dtype=dtype) as h:
        h.upload(pinned)
        h.read(back)
        assert np.array_equal(back.numpy(), pinned.numpy())
        h.step(7)
        h.read(back)
        pageable = h.read()
    assert np.array_equal(back.numpy(), pageable)
    with pkg.Heat(nx, ny, nz, 0.12, dtype=dtype) as h:
        assert np.array_equal(h.upload(pinned.numpy().copy()).step(7).read(), pageable)


def test_resume_from_snapshot_is_bitwise(pkg):
    u0 = heat_u0_single_mode(30, 20, 25, seed=8)
    straight = run_gpu(pkg, u0, 0.1, 50)
    with pkg.Heat(30, 20, 25, 0.1) as h:
        snap = h.upload(u0).step(30).read()
        h.upload(snap).step(20)
        assert np.array_equal(h.read(), straight)


def test_argument_errors(pkg):
    from paper_2608_11882_gb300._native import HS_EINVAL, HS_EUNSTABLE
    with pytest.raises(pkg.HeatCGError) as e:
        pkg.Heat(8, 8, 8, 0.17)
    assert e.value.code == HS_EUNSTABLE
    for bad in [dict(nx=0, ny=4, nz=4, r=0.1), dict(nx=4, ny=4, nz=4, r=-0.1),
                dict(nx=4, ny=4, nz=4, r=float("nan"))]:
        with pytest.raises(pkg.HeatCGError) as e:
            pkg.Heat(**bad)
        assert e.value.code == HS_EINVAL
    with pytest.raises(pkg.HeatCGError) as e:
        pkg.Heat(4, 4, 4, 0.1, flags=0x800)
    assert e.value.code == HS_EINVAL
    with pytest.raises(pkg.HeatCGError):
        pkg.Heat(4, 4, 4, 0.1, dtype="f32", flags=pkg.HS_EXACT_ROUNDING)
    with pkg.Heat(4, 4, 4, 0.1) as h:
        with pytest.raises(pkg.HeatCGError):
            h.step(-1)


def test_unstable_r_grows_when_allowed(pkg):
    n = 16
    s = np.sin(n * np.pi * (np.arange(n) + 1) / (n + 1))
    mode = s[:, None, None] * s[None, :, None] * s[None, None, :]
    out = run_gpu(pkg, mode, 0.17, 200, flags=pkg.HS_ALLOW_UNSTABLE)
    assert np.max(np.abs(out)) > np.max(np.abs(mode))
    assert rel_max_err(out, oracle.heat_run(mode, 0.17, 200)) <= F64_REL


def test_f32_error_within_derived_bound(pkg):
    u0 = heat_u0_single_mode(64, 64, 64)
    ref = oracle.heat_run(u0, 0.1, 100, threads=oracle.max_threads())
    got = run_gpu(pkg, u0.astype(np.float32), 0.1, 100, dtype="f32")
    err = float(np.max(np.abs(got.astype(np.float64) - ref)))
    assert err <= f32_bound(100, float(np.max(np.abs(u0))))


def test_full_size_f64_against_oracle_few_steps(pkg):
    """512^3 interior, r = 0.15, the benchmark's launch configuration, 4 steps
    against the oracle element by element."""
    u0, _, _ = heat_u0_modes(512, 512, 512)
    ref = oracle.heat_run(u0, 0.15, 4, threads=oracle.max_threads())
    got = run_gpu(pkg, u0, 0.15, 4)
    assert rel_max_err(got, ref) <= F64_REL


def test_full_size_f64_1000_steps_closed_form(pkg):
    """512^3, r = 0.15, 1000 steps of the noise-free 8-mode field against the
    exact modal decay evaluated point by point at sampled interior points."""
    u0, modes, amps = heat_u0_modes(512, 512, 512, noise=0.0)
    got = run_gpu(pkg, u0, 0.15, 1000)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 512, size=(4000, 3))
    expect = oracle.sine_modes_exact(modes, amps, u0.shape, 0.15, 1000, pts)
    vals = got[pts[:, 0], pts[:, 1], pts[:, 2]]
    assert np.max(np.abs(vals - expect)) <= F64_REL * np.max(np.abs(u0))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_caller_owned_buffers(pkg, dtype):
    """Torch-allocated time-level buffers passed through hs_heat_desc.dev_buf0/1:
    the library zeroes them, steps in them (the small workload, against the
    oracle), and leaves them allocated and usable after the handle is gone."""
    torch = require_cuda()
    u0 = heat_u0_single_mode(64, 64, 64)
    nbytes = pkg.Heat.buffer_bytes(64, 64, 64, dtype)
    bufs = [torch.full((nbytes,), 7, dtype=torch.uint8, device="cuda") for _ in range(2)]
    h = pkg.Heat(64, 64, 64, 0.1, dtype=dtype, buffers=bufs)
    h.upload(np.ascontiguousarray(u0, dtype=h.np_dtype))
    torch.cuda.synchronize()
    # the field sits in the caller's buffer 0: padded layout, interior at plane,
    # row and column 1 (column offset lead = 32 bytes), boundary layer zero
    elem = 8 if dtype == "f64" else 4
    tdt = torch.float64 if dtype == "f64" else torch.float32
    lead = 32 // elem
    pitch = nbytes // elem // (66 * 66)
    f0 = bufs[0].view(tdt).reshape(66, 66, pitch)
    assert np.array_equal(f0[1:65, 1:65, lead:lead + 64].cpu().numpy(), u0.astype(h.np_dtype))
    assert not f0[0].any() and not f0[:, 0].any() and not f0[:, :, lead - 1].any()
    h.step(100)
    got = h.read()
    h.close()
    ref = oracle.heat_run(u0, 0.1, 100, threads=oracle.max_threads())
    if dtype == "f64":
        assert rel_max_err(got, ref) <= F64_REL
    else:
        assert np.max(np.abs(got - ref)) <= f32_bound(100, np.max(np.abs(u0)))
    # after 100 steps (an even count) the current level is buffer 0 again
    assert np.array_equal(f0[1:65, 1:65, lead:lead + 64].cpu().numpy(), got)
    bufs[1].zero_()                       # still the caller's, still allocated
    torch.cuda.synchronize()
