"""Batched CG: every system equals solving it alone with cg_run, bit for bit,
and meets rtol by the oracle's operator."""
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


def systems(pkg, n, seed, edge=(32, 128)):
    rng = np.random.default_rng(seed)
    out, keep = [], []
    for i in range(n):
        nz, ny, nx = (int(v) for v in np.round(np.exp(rng.uniform(np.log(edge[0]), np.log(edge[1]), 3))))
        if i % 3 == 2:
            arrs = [dev(a) for a in lap7_csr(nx, ny, nz)]
            keep.append(arrs)
            op = pkg.Operator.csr(*arrs)
        else:
            op = pkg.Operator.stencil(nx, ny, nz)
        out.append(((nz, ny, nx), op, cg_rhs(nx * ny * nz, seed=seed * 100 + i)))
    return out, keep


def test_batch_equals_single_bitwise(pkg):
    sy, keep = systems(pkg, 9, seed=3, edge=(6, 40))
    sy[4] = (sy[4][0], sy[4][1], np.zeros_like(sy[4][2]))   # zero right-hand side
    with pkg.CGBatch([s[1] for s in sy]) as cb:
        xs, infos = cb.run([dev(s[2]) for s in sy], rtol=1e-9, max_iter=5000)
    for (shape, op, b), x, info in zip(sy, xs, infos):
        with pkg.CG(op) as cg:
            x1, i1 = cg.run(dev(b), rtol=1e-9, max_iter=5000)
        assert np.array_equal(x.cpu().numpy(), x1.cpu().numpy())
        assert info["iters"] == i1["iters"] and info["converged"]
        if b.any():
            r = b - oracle.lap7_apply(x.cpu().numpy().reshape(shape)).reshape(-1)
            assert np.linalg.norm(r) <= 1.5e-9 * np.linalg.norm(b)


def test_batch_max_iter_per_system(pkg):
    from paper_2608_11882_gb300._native import HS_ENOCONV
    sy, keep = systems(pkg, 4, seed=4, edge=(10, 30))
    with pkg.CGBatch([s[1] for s in sy]) as cb:
        xs, infos = cb.run([dev(s[2]) for s in sy], rtol=1e-12, max_iter=7)
    assert all(i["iters"] == 7 and i["status"] == HS_ENOCONV for i in infos)


def test_batch_workload_64_solves(pkg):
    """The batching workload's CG half: 64 solves with edges in [32, 128]."""
    sy, keep = systems(pkg, 64, seed=20261202)
    with pkg.CGBatch([s[1] for s in sy]) as cb:
        xs, infos = cb.run([dev(s[2]) for s in sy], rtol=1e-8, max_iter=20000)
    assert all(i["converged"] and i["relres_true"] <= 1.5e-8 for i in infos)
    for k in (0, 21, 63):
        shape, op, b = sy[k]
        r = b - oracle.lap7_apply(xs[k].cpu().numpy().reshape(shape)).reshape(-1)
        assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(b)


def test_batch_with_staged_system_equals_single_bitwise(pkg):
    """A batch that holds a grid large enough for the staged exact-sum SpMV
    (176^3, one item of 4+ planes per block), a small matrix-free grid (row
    kernel) and a CSR system: each equals its own cg_run bit for bit."""
    big = (176, 176, 176)
    ops = [(big, pkg.Operator.stencil(*big[::-1]), cg_rhs(176 ** 3, seed=91)),
           ((20, 24, 28), pkg.Operator.stencil(28, 24, 20), cg_rhs(20 * 24 * 28, seed=92))]
    arrs = [dev(a) for a in lap7_csr(30, 22, 18)]
    ops.append(((18, 22, 30), pkg.Operator.csr(*arrs), cg_rhs(18 * 22 * 30, seed=93)))
    with pkg.CGBatch([o[1] for o in ops]) as cb:
        xs, infos = cb.run([dev(o[2]) for o in ops], rtol=1e-8, max_iter=5000)
    for (shape, op, b), x, info in zip(ops, xs, infos):
        with pkg.CG(op) as cg:
            x1, i1 = cg.run(dev(b), rtol=1e-8, max_iter=5000)
        assert info["iters"] == i1["iters"] and info["converged"]
        assert np.array_equal(x.cpu().numpy(), x1.cpu().numpy())
    shape, _, b = ops[0]
    r = b - oracle.lap7_apply(xs[0].cpu().numpy().reshape(shape), threads=oracle.max_threads()).reshape(-1)
    assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("shape", [(200, 101, 190), (160, 120, 177)])
def test_ragged_staged_grid_single_equals_batch(pkg, shape):
    """Ragged grids large enough for the staged SpMV.  With nx even (190) a
    single solve stages p by TMA, whose boxes reach past the grid's last
    column, row and plane and read zeros there; with nx odd (177) it stages p
    with loads.  A batch of one takes the load-staged kernel either way: the
    two agree bit for bit, and the solution meets rtol by the oracle."""
    nz, ny, nx = shape
    b = cg_rhs(nx * ny * nz, seed=94)
    op = pkg.Operator.stencil(nx, ny, nz)
    with pkg.CG(op) as cg:
        x1, i1 = cg.run(dev(b), rtol=1e-8, max_iter=5000)
    with pkg.CGBatch([op]) as cb:
        xs, infos = cb.run([dev(b)], rtol=1e-8, max_iter=5000)
    assert i1["converged"] and infos[0]["iters"] == i1["iters"]
    assert np.array_equal(xs[0].cpu().numpy(), x1.cpu().numpy())
    r = b - oracle.lap7_apply(x1.cpu().numpy().reshape(shape), threads=oracle.max_threads()).reshape(-1)
    assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(b)
