"""Parity of the CUDA CG path (Section 7.5) against the FP64 oracle, through
the C ABI."""
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


def csr_op(pkg, nx, ny, nz):
    rowptr, col, val = lap7_csr(nx, ny, nz)
    return pkg.Operator.csr(dev(rowptr), dev(col), dev(val))


@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_operator_apply_matches_oracle(pkg, kind):
    torch = require_cuda()
    nz, ny, nx = 13, 7, 11
    p = np.random.default_rng(1).standard_normal((nz, ny, nx))
    op = pkg.Operator.stencil(nx, ny, nz) if kind == "stencil" else csr_op(pkg, nx, ny, nz)
    y = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    op.apply(dev(p.reshape(-1)), y)
    ref = oracle.lap7_apply(p).reshape(-1)
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 4 * np.finfo(float).eps * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(24, 24, 24), (9, 17, 33), (1, 1, 5), (2, 2, 2)])
@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_cg_matches_oracle(pkg, shape, kind):
    nz, ny, nx = shape
    n = nx * ny * nz
    b = cg_rhs(n, seed=11)
    op = pkg.Operator.stencil(nx, ny, nz) if kind == "stencil" else csr_op(pkg, nx, ny, nz)
    rtol = 1e-8
    x_ref, info_ref = oracle.cg_solve(b, rtol, 5000, shape=shape)
    with pkg.CG(op) as cg:
        x, info = cg.run(dev(b), rtol=rtol, max_iter=5000)
    x = x.cpu().numpy()
    assert info["converged"] and info["status"] == 0
    assert abs(info["iters"] - info_ref["iters"]) <= 2
    assert info["relres_true"] <= 1.5 * rtol
    # both are solutions to rtol; they differ by at most ~2 kappa rtol
    lam_min = 4 * sum(np.sin(np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    lam_max = 4 * sum(np.sin(m * np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    kappa = lam_max / lam_min
    assert np.linalg.norm(x - x_ref) <= 2 * kappa * rtol * np.linalg.norm(x_ref) + 1e-300
    # true residual recomputed by the oracle's operator
    r = b - oracle.lap7_apply(x.reshape(shape)).reshape(-1)
    assert np.linalg.norm(r) <= 1.5 * rtol * np.linalg.norm(b)


def test_cg_is_deterministic_and_host_path_matches(pkg):
    nz, ny, nx = 20, 18, 16
    b = cg_rhs(nx * ny * nz, seed=12)
    op = pkg.Operator.stencil(nx, ny, nz)
    with pkg.CG(op) as cg:
        x1, i1 = cg.run(dev(b), rtol=1e-10, max_iter=3000)
        x2, i2 = cg.run(dev(b), rtol=1e-10, max_iter=3000)
        x3, i3 = cg.run(b.copy(), rtol=1e-10, max_iter=3000)   # host buffers
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    assert np.array_equal(x1.cpu().numpy(), x3)
    assert i1 == i2 and i1["iters"] == i3["iters"]


@pytest.mark.parametrize("mixed", [False, True])
def test_pinned_host_vectors(pkg, mixed):
    """Pinned host tensors for b and x (copied by a kernel through their
    mapped address) give the solve of device vectors bit for bit, in FP64 and
    in mixed precision; a start vector in x is read too."""
    torch = require_cuda()
    nz, ny, nx = 21, 17, 14
    n = nx * ny * nz
    b = cg_rhs(n, seed=13)
    op = pkg.Operator.stencil(nx, ny, nz)
    x0 = np.random.default_rng(14).uniform(-1, 1, n)
    with pkg.CG(op, mixed=mixed) as cg:
        xd, idev = cg.run(dev(b), dev(x0), rtol=1e-10, max_iter=3000)
        bp = torch.from_numpy(b.copy()).pin_memory()
        xp = torch.from_numpy(x0.copy()).pin_memory()
        _, ipin = cg.run(bp, xp, rtol=1e-10, max_iter=3000)
    assert np.array_equal(xp.numpy(), xd.cpu().numpy())
    assert idev["iters"] == ipin["iters"] and idev["relres_true"] == ipin["relres_true"]


def test_cg_eigenvector_one_iteration(pkg):
    nz, ny, nx = 7, 5, 6
    xs, ys, zs = [(np.arange(m) + 1) / (m + 1) for m in (nx, ny, nz)]
    b = (np.sin(1 * np.pi * zs)[:, None, None] * np.sin(3 * np.pi * ys)[None, :, None]
         * np.sin(2 * np.pi * xs)[None, None, :]).reshape(-1)
    lam = 4 * (np.sin(2 * np.pi / 14) ** 2 + np.sin(3 * np.pi / 12) ** 2 + np.sin(np.pi / 16) ** 2)
    with pkg.CG(pkg.Operator.stencil(nx, ny, nz)) as cg:
        x, info = cg.run(dev(b), rtol=1e-10, max_iter=50)
    assert info["iters"] == 1
    assert np.max(np.abs(x.cpu().numpy() - b / lam)) <= 1e-13 * np.max(np.abs(b / lam))


def test_cg_max_iter_and_zero_rhs_and_x0(pkg):
    from paper_2608_11882_gb300._native import HS_ENOCONV
    nz = ny = nx = 10
    b = cg_rhs(1000, seed=13)
    with pkg.CG(pkg.Operator.stencil(nx, ny, nz)) as cg:
        x, info = cg.run(dev(b), rtol=1e-12, max_iter=3)
        assert not info["converged"] and info["status"] == HS_ENOCONV and info["iters"] == 3
        x0, info0 = cg.run(dev(np.zeros(1000)), rtol=1e-8, max_iter=10)
        assert info0["iters"] == 0 and not x0.cpu().numpy().any()
        # start from a nonzero x0: same answer as the oracle started there
        start = np.random.default_rng(3).standard_normal(1000)
        xs, infos = cg.run(dev(b), x=dev(start.copy()), rtol=1e-9, max_iter=1000)
    x_ref, info_ref = oracle.cg_solve(b, 1e-9, 1000, shape=(nz, ny, nx), x0=start)
    assert abs(infos["iters"] - info_ref["iters"]) <= 2
    assert infos["relres_true"] <= 1.5e-9


def test_cg_argument_errors(pkg):
    from paper_2608_11882_gb300._native import HS_EINVAL, hs_op, cg_create
    with pytest.raises(pkg.HeatCGError) as e:
        cg_create(hs_op(kind=7, n=4, dtype=0))
    assert e.value.code == HS_EINVAL
    with pytest.raises(pkg.HeatCGError):
        cg_create(hs_op(kind=1, n=4, nnz=4, dtype=0))   # CSR without arrays


@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_full_size_cg_256(pkg, kind):
    """256^3 Laplacian, b ~ N(0,1), rtol 1e-8: the benchmark's configuration.
    The oracle recomputes the true residual of the GPU solution."""
    nz = ny = nx = 256
    b = cg_rhs(nx * ny * nz)
    op = pkg.Operator.stencil(nx, ny, nz) if kind == "stencil" else csr_op(pkg, nx, ny, nz)
    with pkg.CG(op) as cg:
        x, info = cg.run(dev(b), rtol=1e-8, max_iter=20000)
    assert info["converged"]
    x = x.cpu().numpy()
    r = b - oracle.lap7_apply(x.reshape(nz, ny, nx), threads=oracle.max_threads()).reshape(-1)
    assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_unaligned_solution_buffer_same_result(pkg, kind):
    """x one element into an allocation (8-byte, not 16-byte aligned) on a grid
    with an odd number of unknowns: the same iterates bit for bit."""
    torch = require_cuda()
    nx, ny, nz = 13, 11, 9
    n = nx * ny * nz
    op = pkg.Operator.stencil(nx, ny, nz) if kind == "stencil" else csr_op(pkg, nx, ny, nz)
    b = dev(cg_rhs(n, seed=17))
    with pkg.CG(op) as cg:
        x1, i1 = cg.run(b, rtol=1e-10)
        store = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        x2, i2 = cg.run(b, x=store[1:], rtol=1e-10)
    assert i1["iters"] == i2["iters"]
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())


@pytest.mark.parametrize("shape,kind", [((176, 176, 176), "stencil"), ((176, 176, 175), "stencil"),
                                        ((20, 18, 16), "stencil"), ((12, 10, 14), "csr")])
def test_launch_count_of_a_solve(pkg, shape, kind):
    """hs_launch_count counts every kernel a solve launches, once: q = A x0, the
    start kernel, three kernels per enqueued iteration (iterations go out in
    chunks of 4, 8, 16, then 32 between reads of the stop flag), the final
    A x and the residual norm -- whichever SpMV kernel the grid takes (TMA-staged
    for 176^3, load-staged for nx = 175, row kernel for the small grid, CSR)."""
    from paper_2608_11882_gb300 import _native
    nz, ny, nx = shape
    n = nx * ny * nz
    op = pkg.Operator.stencil(nx, ny, nz) if kind == "stencil" else csr_op(pkg, nx, ny, nz)
    b = dev(cg_rhs(n, seed=31))
    with pkg.CG(op) as cg:
        c0 = _native.launch_count()
        _, info = cg.run(b, rtol=1e-8, max_iter=5000)
        launched = _native.launch_count() - c0
    assert info["converged"]
    enq, chunk = 0, 4
    while enq < info["iters"]:
        enq += chunk
        chunk = min(2 * chunk, 32)
    assert launched == 4 + 3 * enq
