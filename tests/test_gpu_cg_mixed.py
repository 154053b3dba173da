"""Mixed-precision CG (FP32 Krylov vectors inside FP64 iterative refinement)
against the FP64 oracle: the returned x must meet rtol in FP64 terms, which
the oracle's operator checks independently."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import lib, require_cuda
from workloads import cg_rhs, lap7_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def dev(a):
    torch = require_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def kappa(nx, ny, nz):
    lo = 4 * sum(np.sin(np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    hi = 4 * sum(np.sin(m * np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    return hi / lo


def make_op(pkg, kind, nx, ny, nz):
    if kind == "stencil":
        return pkg.Operator.stencil(nx, ny, nz)
    return pkg.Operator.csr(*[dev(a) for a in lap7_csr(nx, ny, nz)])


def true_relres(x, b, shape):
    r = b - oracle.lap7_apply(x.reshape(shape), threads=oracle.max_threads()).reshape(-1)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("kind", ["stencil", "csr"])
@pytest.mark.parametrize("shape,rtol", [((24, 24, 24), 1e-10), ((9, 17, 33), 1e-12),
                                        ((40, 31, 22), 1e-8), ((2, 2, 2), 1e-10),
                                        ((37, 21, 132), 1e-10), ((5, 3, 4), 1e-10)])
def test_mixed_meets_rtol_in_fp64(pkg, kind, shape, rtol):
    nz, ny, nx = shape
    b = cg_rhs(nx * ny * nz, seed=31)
    with pkg.CG(make_op(pkg, kind, nx, ny, nz), mixed=True) as cg:
        x, info = cg.run(dev(b), rtol=rtol, max_iter=50000)
    x = x.cpu().numpy()
    assert info["converged"] and info["status"] == 0
    assert info["relres_true"] <= rtol
    assert true_relres(x, b, shape) <= 1.5 * rtol
    x_ref, info_ref = oracle.cg_solve(b, rtol, 50000, shape=shape)
    assert np.linalg.norm(x - x_ref) <= 2 * kappa(nx, ny, nz) * rtol * np.linalg.norm(x_ref)
    if rtol < 1e-7:
        assert info["refinements"] >= 1   # beyond FP32 accuracy takes refinement


def test_mixed_inner_tolerance_and_limits(pkg):
    from paper_2608_11882_gb300._native import HS_ENOCONV
    n = 20
    b = cg_rhs(n ** 3, seed=32)
    op = pkg.Operator.stencil(n, n, n)
    with pkg.CG(op, mixed=True, inner_rtol=1e-2) as cg:
        x, info = cg.run(dev(b), rtol=1e-10, max_iter=50000)
    assert info["converged"] and info["refinements"] >= 3
    assert true_relres(x.cpu().numpy(), b, (n, n, n)) <= 1.5e-10
    with pkg.CG(op, mixed=True) as cg:
        _, info = cg.run(dev(b), rtol=1e-12, max_iter=5)
        assert not info["converged"] and info["status"] == HS_ENOCONV and info["iters"] <= 5
        x0, info0 = cg.run(dev(np.zeros(n ** 3)), rtol=1e-8, max_iter=10)
        assert info0["iters"] == 0 and info0["converged"] and not x0.cpu().numpy().any()
        xh, infoh = cg.run(b.copy(), rtol=1e-9, max_iter=50000)   # host buffers
    assert infoh["converged"] and true_relres(xh, b, (n, n, n)) <= 1.5e-9
    for bad in (1.0, -1e-3):
        with pytest.raises(pkg.HeatCGError):
            pkg.CG(op, mixed=True, inner_rtol=bad)


@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_mixed_full_size_256(pkg, kind):
    n = 256
    b = cg_rhs(n ** 3)
    with pkg.CG(make_op(pkg, kind, n, n, n), mixed=True) as cg:
        x, info = cg.run(dev(b), rtol=1e-8, max_iter=100000)
    assert info["converged"]
    assert true_relres(x.cpu().numpy(), b, (n, n, n)) <= 1.5e-8


def test_mixed_precision_workload_512_rtol_1e10(pkg):
    """The precision workload: CG on the 512^3 Laplacian to rtol 1e-10 with FP32
    Krylov vectors and FP64 residual/refinement."""
    n = 512
    b = cg_rhs(n ** 3)
    with pkg.CG(pkg.Operator.stencil(n, n, n), mixed=True) as cg:
        x, info = cg.run(dev(b), rtol=1e-10, max_iter=200000)
    assert info["converged"] and info["refinements"] >= 1
    assert true_relres(x.cpu().numpy(), b, (n, n, n)) <= 1.5e-10


def test_mixed_repeat_runs_agree_bitwise(pkg):
    """The matrix-free FP32 SpMV forms each new direction into the other of two
    p buffers, so a second solve on the same context may start from either
    buffer: its x, iteration and refinement counts must equal the first solve's
    and a fresh context's bit for bit (ragged x and y tiles: nx = 136 is one
    128-point tile and 8 points, ny = 21 is two 8-row tiles and 5 rows)."""
    nz, ny, nx = 40, 21, 136
    b = cg_rhs(nx * ny * nz, seed=35)
    op = pkg.Operator.stencil(nx, ny, nz)
    with pkg.CG(op, mixed=True) as cg:
        x1, i1 = cg.run(dev(b), rtol=1e-10, max_iter=50000)
        x2, i2 = cg.run(dev(b), rtol=1e-10, max_iter=50000)
    with pkg.CG(op, mixed=True) as cg:
        x3, i3 = cg.run(dev(b), rtol=1e-10, max_iter=50000)
    assert i1["converged"]
    for x, i in ((x2, i2), (x3, i3)):
        assert (i["iters"], i["refinements"]) == (i1["iters"], i1["refinements"])
        assert np.array_equal(x.cpu().numpy(), x1.cpu().numpy())
    assert true_relres(x1.cpu().numpy(), b, (nz, ny, nx)) <= 1.5e-10
