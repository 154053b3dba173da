"""The paper's variable-coefficient problem (HS_VARKAPPA; Section 4, Eqs.
1-4, face-averaged D) on the GPU against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, lib, rel_max_err
from workloads import heat_u0_single_mode

pytestmark = pytest.mark.gpu

R_PAPER = 1.0 / (12 * 0.95)   # dt = h^2/(12 kappa_max)


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def run_vk(pkg, u0, r, steps, dtype="f64"):
    nz, ny, nx = u0.shape
    with pkg.Heat(nx, ny, nz, r, dtype=dtype, flags=pkg.HS_VARKAPPA) as h:
        h.upload(np.ascontiguousarray(u0, dtype=h.np_dtype))
        h.step(steps)
        return h.read()


@pytest.mark.parametrize("shape", [(64, 64, 64), (1, 1, 1), (2, 3, 5), (33, 9, 17), (40, 65, 31)])
def test_vk_parity(pkg, shape):
    nz, ny, nx = shape
    u0 = heat_u0_single_mode(nx, ny, nz, seed=13)
    ref = oracle.heat_vk_run(u0, R_PAPER, 60, threads=oracle.max_threads())
    assert rel_max_err(run_vk(pkg, u0, R_PAPER, 60), ref) <= F64_REL


def test_vk_without_initial_field_grows_from_the_source(pkg):
    u = run_vk(pkg, np.zeros((20, 18, 22)), R_PAPER, 40)
    ref = oracle.heat_vk_run(np.zeros((20, 18, 22)), R_PAPER, 40)
    assert np.all(u >= 0) and rel_max_err(u, ref) <= F64_REL


@pytest.mark.parametrize("shape", [(48, 48, 48), (9, 13, 37), (30, 7, 22), (5, 3, 1)])
def test_vk_f32_within_bound(pkg, shape):
    """FP32 (four x points per thread; 37, 22 and 1 wide leave ragged vectors)
    against the FP64 oracle within the FP32 rounding bound."""
    nz, ny, nx = shape
    u0 = heat_u0_single_mode(nx, ny, nz, seed=14)
    ref = oracle.heat_vk_run(u0, R_PAPER, 100, threads=oracle.max_threads())
    got = run_vk(pkg, u0.astype(np.float32), R_PAPER, 100, dtype="f32")
    # each step adds at most ~24 float roundings of values <= max|u| + dt f
    bound = (24 * 100 + 1) * 2.0 ** -24 * float(np.max(np.abs(ref)) + 1.0)
    assert float(np.max(np.abs(got - ref))) <= bound


@pytest.mark.parametrize("shape", [(33, 33, 33), (21, 34, 27)])
@pytest.mark.parametrize("scale", [1.0, 1e-250, 1e250, 1e-300])
def test_vk_f64_exact_sum_against_oracle(pkg, scale, shape):
    """FP64 grids take the exact-sum form (the operator sums exact in 128 bits
    on the field's fixed-point scale, rounded once: the whole sum on a cubic
    grid, each axis's sum on the non-cubic one) while the field's exponent
    allows; 1e-300 starts on the FP64 form and the source lifts the field into
    range within a step, 1e-250 and 1e250 run exact throughout."""
    nz, ny, nx = shape
    u0 = heat_u0_single_mode(nx, ny, nz, seed=16) * scale
    ref = oracle.heat_vk_run(u0, R_PAPER, 40, threads=oracle.max_threads())
    assert rel_max_err(run_vk(pkg, u0, R_PAPER, 40), ref) <= F64_REL


def test_vk_f64_cubic_from_zero_field(pkg):
    u = run_vk(pkg, np.zeros((24, 24, 24)), R_PAPER, 30)
    ref = oracle.heat_vk_run(np.zeros((24, 24, 24)), R_PAPER, 30)
    assert np.all(u >= 0) and rel_max_err(u, ref) <= F64_REL


def test_vk_f64_cubic_tight_against_oracle(pkg):
    """The exact-sum form rounds the operator sums once per point, so after 50
    steps at 40^3 (and on a non-cubic grid) it stays within 1e-13 of the
    oracle (relative to max|u|), ten times inside the FP64 gate."""
    for nz, ny, nx in [(40, 40, 40), (36, 44, 41)]:
        u0 = heat_u0_single_mode(nx, ny, nz, seed=18)
        ref = oracle.heat_vk_run(u0, R_PAPER, 50, threads=oracle.max_threads())
        got = run_vk(pkg, u0, R_PAPER, 50)
        assert rel_max_err(got, ref) <= 1e-13, (nz, ny, nx)


def test_vk_f64_one_step_close_to_oracle(pkg):
    """One step of the exact-sum form differs from the oracle's written-order
    FP64 step only by roundings (each operator sum is exact before its one
    rounding): within 2e-15 of max|u| on a cubic and a non-cubic grid."""
    for nz, ny, nx in [(30, 30, 30), (26, 31, 35)]:
        u0 = heat_u0_single_mode(nx, ny, nz, seed=19)
        ref = oracle.heat_vk_run(u0, R_PAPER, 1)
        assert rel_max_err(run_vk(pkg, u0, R_PAPER, 1), ref) <= 2e-15, (nz, ny, nx)


def test_vk_errors(pkg):
    from paper_2608_11882_gb300._native import HS_EINVAL, HS_EUNSTABLE
    with pytest.raises(pkg.HeatCGError) as e:
        pkg.Heat(8, 8, 8, 1.0 / (6 * 0.95) * 1.01, flags=pkg.HS_VARKAPPA)
    assert e.value.code == HS_EUNSTABLE
    for flags, td in ((pkg.HS_VARKAPPA | pkg.HS_FIXED64, 0), (pkg.HS_VARKAPPA, 2)):
        with pytest.raises(pkg.HeatCGError) as e:
            pkg.Heat(8, 8, 8, 0.05, flags=flags, tdepth=td)
        assert e.value.code == HS_EINVAL
    h = pkg.Heat(8, 8, 8, 0.05, flags=pkg.HS_VARKAPPA)
    with pytest.raises(pkg.HeatCGError):
        pkg.HeatBatch([h], [3])
    h.close()


def test_vk_paper_size_against_oracle(pkg):
    """The paper's N = 512 (510^3 interior nodes), dt = h^2/(12 kappa_max), a
    few steps against the oracle element by element."""
    n = 510
    u0 = heat_u0_single_mode(n, n, n, seed=15)
    ref = oracle.heat_vk_run(u0, R_PAPER, 3, threads=oracle.max_threads())
    assert rel_max_err(run_vk(pkg, u0, R_PAPER, 3), ref) <= F64_REL
