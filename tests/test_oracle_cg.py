"""Pins for the CG oracle (Section 7.5): dense direct solves, eigenvector and
distinct-eigenvalue facts of CG in exact arithmetic, and the operator built
two independent ways."""
import numpy as np
import pytest

from tests.dense_ref import laplacian_kron
from workloads import cg_rhs, lap7_csr


def test_matrix_free_operator_equals_kronecker_sum(oracle_mod):
    nz, ny, nx = 4, 5, 6
    p = np.random.default_rng(1).standard_normal((nz, ny, nx))
    expect = laplacian_kron(nx, ny, nz) @ p.reshape(-1)
    got = oracle_mod.lap7_apply(p).reshape(-1)
    assert np.max(np.abs(got - expect)) <= 1e-14 * np.max(np.abs(expect))


def test_csr_operator_equals_matrix_free_bitwise(oracle_mod):
    nz, ny, nx = 5, 6, 7
    p = np.random.default_rng(2).standard_normal((nz, ny, nx))
    rowptr, col, val = lap7_csr(nx, ny, nz)
    a = oracle_mod.csr_spmv(rowptr, col, val, p)
    b = oracle_mod.lap7_apply(p).reshape(-1)
    assert np.array_equal(a, b)


def test_csr_structure_counts():
    for nx, ny, nz in ((1, 1, 1), (3, 4, 5), (16, 16, 16)):
        rowptr, col, val = lap7_csr(nx, ny, nz)
        n = nx * ny * nz
        assert rowptr[-1] == 7 * n - 2 * (nx * ny + ny * nz + nx * nz)
        assert np.all(np.diff(rowptr) >= 1)
        for r in range(0, n, max(1, n // 50)):
            cs = col[rowptr[r]:rowptr[r + 1]]
            assert np.all(np.diff(cs) > 0)


@pytest.mark.parametrize("shape", [(2, 2, 2), (5, 4, 3), (8, 8, 8)])
@pytest.mark.parametrize("use_csr", [False, True])
def test_cg_matches_dense_direct_solve(oracle_mod, shape, use_csr):
    nz, ny, nx = shape
    b = cg_rhs(nx * ny * nz, seed=3)
    a = laplacian_kron(nx, ny, nz)
    x_star = np.linalg.solve(a, b)
    rtol = 1e-12
    kwargs = {"csr": lap7_csr(nx, ny, nz)} if use_csr else {"shape": shape}
    x, info = oracle_mod.cg_solve(b, rtol, 1000, **kwargs)
    assert info["status"] == 0
    cond = np.linalg.cond(a)
    assert np.linalg.norm(x - x_star) <= 2 * cond * rtol * np.linalg.norm(x_star)
    assert info["relres_true"] <= 10 * rtol


def test_cg_eigenvector_rhs_converges_in_one_iteration(oracle_mod):
    nz, ny, nx = 7, 5, 6
    kx, ky, kz = 2, 3, 1
    xs, ys, zs = [(np.arange(n) + 1) / (n + 1) for n in (nx, ny, nz)]
    b = (np.sin(kz * np.pi * zs)[:, None, None] * np.sin(ky * np.pi * ys)[None, :, None]
         * np.sin(kx * np.pi * xs)[None, None, :]).reshape(-1)
    lam = 4 * (np.sin(kx * np.pi / (2 * (nx + 1))) ** 2 + np.sin(ky * np.pi / (2 * (ny + 1))) ** 2
               + np.sin(kz * np.pi / (2 * (nz + 1))) ** 2)
    x, info = oracle_mod.cg_solve(b, 1e-10, 50, shape=(nz, ny, nx))
    assert info["status"] == 0 and info["iters"] == 1
    assert np.max(np.abs(x - b / lam)) <= 1e-13 * np.max(np.abs(b / lam))


def test_cg_iterations_bounded_by_distinct_eigenvalues(oracle_mod):
    # 3x3x3: eigenvalues are sums of three of {4 sin^2(k pi / 8), k = 1, 2, 3}:
    # C(5, 3) = 10 distinct values, so exact CG ends within 10 iterations.
    b = cg_rhs(27, seed=4)
    x, info = oracle_mod.cg_solve(b, 1e-12, 100, shape=(3, 3, 3))
    assert info["status"] == 0
    assert info["iters"] <= 10
    assert info["relres_true"] <= 1e-12


def test_cg_status_when_max_iter_reached(oracle_mod):
    b = cg_rhs(10 * 10 * 10, seed=5)
    x, info = oracle_mod.cg_solve(b, 1e-12, 3, shape=(10, 10, 10))
    assert info["status"] == 1 and info["iters"] == 3


def test_cg_zero_rhs_gives_zero(oracle_mod):
    x, info = oracle_mod.cg_solve(np.zeros(8), 1e-8, 10, shape=(2, 2, 2))
    assert info["iters"] == 0 and info["status"] == 0 and not np.any(x)


def test_cg_threads_do_not_change_results(oracle_mod):
    b = cg_rhs(9 * 8 * 7, seed=6)
    x1, i1 = oracle_mod.cg_solve(b, 1e-10, 500, shape=(9, 8, 7), threads=1)
    x4, i4 = oracle_mod.cg_solve(b, 1e-10, 500, shape=(9, 8, 7), threads=4)
    i1.pop("loop_seconds")
    i4.pop("loop_seconds")
    assert np.array_equal(x1, x4) and i1 == i4
