"""Pins for the variable-coefficient oracle (Section 4, Eqs. 1-4 with the
face-averaged reading of D): it reduces to the pinned constant-coefficient
update, it matches a dense operator assembled face by face on tiny grids,
and without the source it obeys the maximum principle."""
import numpy as np
import pytest

KMAX = 0.95


def dense_vk_step(shape, r, with_source=True):
    """(M, c) with u' = M u + c, assembled by visiting every face once."""
    nz, ny, nx = shape
    n = nx * ny * nz
    hs = [1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1)]
    h = min(hs)
    dt = r * h * h

    def kap(i, j, k):   # padded node indices
        return 0.5 + 0.45 * np.sin(np.pi * i * hs[0]) * np.sin(np.pi * j * hs[1]) * np.sin(np.pi * k * hs[2])

    def idx(i, j, k):
        if 1 <= i <= nx and 1 <= j <= ny and 1 <= k <= nz:
            return ((k - 1) * ny + (j - 1)) * nx + (i - 1)
        return None

    L = np.zeros((n, n))
    c = np.zeros(n)
    for k in range(1, nz + 1):
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                row = idx(i, j, k)
                for d, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    beta = dt / (2 * hs[d] ** 2)
                    for s in (1, -1):
                        w = beta * (kap(i, j, k) + kap(i + s * di, j + s * dj, k + s * dk))
                        L[row, row] -= w
                        nb = idx(i + s * di, j + s * dj, k + s * dk)
                        if nb is not None:
                            L[row, nb] += w
                if with_source:
                    x, y, z = i * hs[0], j * hs[1], k * hs[2]
                    c[row] = dt * (1 + np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z))
    return np.eye(n) + L, c


def test_constant_kappa_reduces_to_constant_coefficient_update(oracle_mod):
    rng = np.random.default_rng(2)
    u0 = rng.uniform(-1, 1, size=(9, 9, 9))
    r, k0 = 0.12, 0.6
    a = oracle_mod.heat_vk_run(u0, r, 30, kappa_const=k0, with_source=False)
    # cubic grid: dt/(2h^2) * 2 k0 = r k0 is the constant-coefficient r
    b = oracle_mod.heat_run(u0, r * k0, 30)
    assert np.max(np.abs(a - b)) <= 1e-13


@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 4, 4), (2, 6, 3)])
@pytest.mark.parametrize("with_source", [True, False])
def test_matches_dense_face_assembly(oracle_mod, shape, with_source):
    r = 1.0 / (12 * KMAX)
    rng = np.random.default_rng(sum(shape))
    u0 = rng.uniform(-1, 1, size=shape)
    m, c = dense_vk_step(shape, r, with_source)
    u = u0.reshape(-1).copy()
    for _ in range(17):
        u = m @ u + c
    got = oracle_mod.heat_vk_run(u0, r, 17, with_source=with_source).reshape(-1)
    assert np.max(np.abs(got - u)) <= 1e-13 * max(1.0, np.max(np.abs(u)))


def test_max_principle_without_source(oracle_mod):
    rng = np.random.default_rng(3)
    cur = rng.uniform(-1, 1, size=(11, 10, 12))
    for _ in range(15):
        nxt = oracle_mod.heat_vk_run(cur, 1.0 / (12 * KMAX), 1, with_source=False)
        assert np.max(np.abs(nxt)) <= np.max(np.abs(cur)) * (1 + 1e-15)
        cur = nxt


def test_source_drives_a_zero_field_positive(oracle_mod):
    # f = 1 + cos cos cos >= 0 everywhere, so from u0 = 0 the field stays >= 0 and grows
    u = oracle_mod.heat_vk_run(np.zeros((8, 8, 8)), 1.0 / (12 * KMAX), 20)
    assert np.all(u >= 0) and np.max(u) > 0
