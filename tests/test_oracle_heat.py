"""Pins for the heat oracle: facts fixed by the mathematics of the explicit
update (Section 4, Eq. 4 with kappa = 1, f = 0; Eq. 6 stability), not by any
implementation."""
import numpy as np
import pytest

from tests.dense_ref import laplacian_kron
from workloads import heat_u0_modes, heat_u0_single_mode


def test_single_interior_point_closed_form(oracle_mod):
    # A 1x1x1 interior has six zero neighbours: u_{m+1} = (1 - 6r) u_m.
    for r in (0.05, 0.1, 1.0 / 6.0):
        u0 = np.full((1, 1, 1), 0.75)
        out = oracle_mod.heat_run(u0, r, 40)
        assert out[0, 0, 0] == pytest.approx(0.75 * (1 - 6 * r) ** 40, rel=1e-13, abs=1e-300)


def test_zero_steps_is_identity(oracle_mod):
    u0 = heat_u0_single_mode(5, 4, 3, seed=1)
    assert np.array_equal(oracle_mod.heat_run(u0, 0.1, 0), u0)


@pytest.mark.parametrize("shape,k,r,steps", [
    ((11, 7, 9), (2, 3, 5), 0.1, 60),      # (nz, ny, nx), modes (kx, ky, kz)
    ((6, 13, 5), (5, 1, 4), 0.15, 40),
    ((16, 16, 16), (1, 1, 1), 1.0 / 6.0, 100),
])
def test_sine_mode_decays_by_exact_factor(oracle_mod, shape, k, r, steps):
    """prod sin(k_d pi x_d) is an eigenvector of the update with factor
    g = 1 - 4 r sum_d sin^2(k_d pi h_d / 2); distinct k and n per axis catch a
    transposed stride or a dropped axis."""
    nz, ny, nx = shape
    kx, ky, kz = k
    xs = (np.arange(nx) + 1) / (nx + 1)
    ys = (np.arange(ny) + 1) / (ny + 1)
    zs = (np.arange(nz) + 1) / (nz + 1)
    mode = (np.sin(kz * np.pi * zs)[:, None, None] * np.sin(ky * np.pi * ys)[None, :, None]
            * np.sin(kx * np.pi * xs)[None, None, :])
    g = 1 - 4 * r * (np.sin(kx * np.pi / (2 * (nx + 1))) ** 2
                     + np.sin(ky * np.pi / (2 * (ny + 1))) ** 2
                     + np.sin(kz * np.pi / (2 * (nz + 1))) ** 2)
    out = oracle_mod.heat_run(mode, r, steps)
    expect = g ** steps * mode
    assert np.max(np.abs(out - expect)) <= 1e-13 * np.max(np.abs(mode))


def test_matches_dense_kronecker_matrix_power(oracle_mod):
    """u_N = (I - r L)^N u_0 with L = 6I - adjacency built from Kronecker sums."""
    nz, ny, nx = 5, 4, 3
    rng = np.random.default_rng(7)
    u0 = rng.uniform(-1, 1, size=(nz, ny, nx))
    r, steps = 0.13, 25
    m = np.eye(nx * ny * nz) - r * laplacian_kron(nx, ny, nz)
    expect = np.linalg.matrix_power(m, steps) @ u0.reshape(-1)
    out = oracle_mod.heat_run(u0, r, steps).reshape(-1)
    assert np.max(np.abs(out - expect)) <= 1e-13


def test_max_principle_for_stable_r(oracle_mod):
    rng = np.random.default_rng(11)
    u = rng.uniform(-1, 1, size=(9, 8, 7))
    for r in (0.1, 1.0 / 6.0):
        cur = u
        for _ in range(20):
            nxt = oracle_mod.heat_run(cur, r, 1)
            assert np.max(np.abs(nxt)) <= np.max(np.abs(cur)) * (1 + 1e-15)
            cur = nxt


def test_highest_mode_grows_above_stability_bound(oracle_mod):
    """For the checkerboard mode k = n on every axis, |g| = |1 - 12 r sin^2(n pi h/2)|
    exceeds 1 once r > 1/(6 sin^2(n pi h / 2)): the 3-D bound r <= 1/6, not the
    1-D bound printed as Eq. 6."""
    n = 16
    xs = (np.arange(n) + 1) / (n + 1)
    s = np.sin(n * np.pi * xs)
    mode = s[:, None, None] * s[None, :, None] * s[None, None, :]
    s2 = np.sin(n * np.pi / (2 * (n + 1))) ** 2
    for r, grows in ((0.17, True), (1.0 / 6.0, False), (0.1, False)):
        out = oracle_mod.heat_run(mode, r, 200)
        ratio = np.max(np.abs(out)) / np.max(np.abs(mode))
        g = 1 - 12 * r * s2
        assert ratio == pytest.approx(abs(g) ** 200, rel=1e-9)
        assert (ratio > 1.0) == grows


def test_modes_without_noise_match_closed_form(oracle_mod):
    u0, modes, amps = heat_u0_modes(20, 18, 22, seed=5, noise=0.0)
    out = oracle_mod.heat_run(u0, 0.15, 30)
    pts = np.array([(k, j, i) for k in (0, 7, 21) for j in (0, 9, 17) for i in (0, 11, 19)])
    expect = oracle_mod.sine_modes_exact(modes, amps, u0.shape, 0.15, 30, pts)
    got = out[pts[:, 0], pts[:, 1], pts[:, 2]]
    assert np.max(np.abs(got - expect)) <= 1e-13 * np.max(np.abs(u0))


def test_threads_do_not_change_results(oracle_mod):
    u0 = heat_u0_single_mode(17, 9, 33, seed=3)
    a = oracle_mod.heat_run(u0, 0.1, 10, threads=1)
    b = oracle_mod.heat_run(u0, 0.1, 10, threads=4)
    assert np.array_equal(a, b)
