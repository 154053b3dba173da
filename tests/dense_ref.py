"""Dense reference operators for tiny grids, built as Kronecker sums of 1-D
second-difference matrices -- a construction independent of the stencil loops
of the oracle and of the CUDA kernels (test helper only)."""
import numpy as np


def second_difference(n: int) -> np.ndarray:
    """tridiag(-1, 2, -1) of size n: the 1-D Dirichlet second difference times -h^2."""
    return 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def laplacian_kron(nx: int, ny: int, nz: int) -> np.ndarray:
    """6I - adjacency of the 7-point grid, rows/columns in (z, y, x) order with x fastest."""
    ix, iy, iz = np.eye(nx), np.eye(ny), np.eye(nz)
    return (np.kron(iz, np.kron(iy, second_difference(nx)))
            + np.kron(iz, np.kron(second_difference(ny), ix))
            + np.kron(second_difference(nz), np.kron(iy, ix)))
