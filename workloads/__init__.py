"""Seeded synthetic inputs shared by the CUDA path's tests and benchmark and by
the CPU oracle.

This module holds none of the method's arithmetic: it only draws initial
fields, right-hand sides and the CSR structure of the 7-point operator, so that
both sides consume the very same arrays.  It imports neither the oracle nor the
product library.

Recipes (all grids are interior counts, x fastest, h_d = 1/(n_d + 1)):

* ``heat_u0_single_mode``: sin(pi x) sin(pi y) sin(pi z) plus uniform noise of
  amplitude 0.01 -- the initial condition of Section 4, Eq. 5, with the noise
  the small parity workload (64^3, r = 0.1, 100 steps) adds.
* ``heat_u0_modes``: a sum of 8 sine modes with wave numbers k in [1, 16] per
  axis and amplitudes in [0.5, 1], plus uniform noise of amplitude 1e-3 -- the
  512^3 benchmark workload.  ``noise=0`` gives a field whose exact evolution is
  known in closed form.
* ``cg_rhs``: b ~ N(0, 1).
* ``lap7_csr``: the CSR structure of the 7-point Dirichlet Laplacian, int32
  indices, columns ascending within each row (natural ordering, Section 7.5).
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20261202


def grid_coords(n: int) -> np.ndarray:
    """Interior node coordinates (i+1)/(n+1), i = 0..n-1, on the unit interval."""
    return (np.arange(n, dtype=np.float64) + 1.0) / (n + 1)


def heat_u0_single_mode(nx: int, ny: int, nz: int, seed: int = DEFAULT_SEED,
                        noise: float = 0.01) -> np.ndarray:
    rng = np.random.default_rng(seed)
    sx = np.sin(np.pi * grid_coords(nx))
    sy = np.sin(np.pi * grid_coords(ny))
    sz = np.sin(np.pi * grid_coords(nz))
    u = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    if noise:
        u = u + noise * rng.uniform(-1.0, 1.0, size=u.shape)
    return np.ascontiguousarray(u)


def draw_modes(seed: int = DEFAULT_SEED, n_modes: int = 8, kmax: int = 16):
    """Wave numbers (kx, ky, kz) in [1, kmax] and amplitudes in [0.5, 1]."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(1, kmax + 1, size=(n_modes, 3))
    amps = rng.uniform(0.5, 1.0, size=n_modes)
    return [tuple(int(v) for v in k) for k in ks], [float(a) for a in amps]


def heat_u0_modes(nx: int, ny: int, nz: int, seed: int = DEFAULT_SEED, n_modes: int = 8,
                  kmax: int = 16, noise: float = 1e-3, dtype=np.float64):
    """Returns (u0, modes, amps).  Noise is drawn after the modes from the same
    generator, so ``noise=0`` leaves the modes unchanged."""
    modes, amps = draw_modes(seed, n_modes, kmax)
    u = np.zeros((nz, ny, nx), dtype=np.float64)
    xs, ys, zs = grid_coords(nx), grid_coords(ny), grid_coords(nz)
    for (kx, ky, kz), a in zip(modes, amps):
        sx = np.sin(kx * np.pi * xs)
        sy = np.sin(ky * np.pi * ys)
        sz = a * np.sin(kz * np.pi * zs)
        for k in range(nz):                       # plane by plane: bounded temporaries
            u[k] += sz[k] * np.outer(sy, sx)
    if noise:
        rng = np.random.default_rng([seed, 1])
        for k in range(nz):
            u[k] += noise * rng.uniform(-1.0, 1.0, size=(ny, nx))
    return np.ascontiguousarray(u.astype(dtype, copy=False)), modes, amps


def heat_u0_modes_device(nx: int, ny: int, nz: int, device, seed: int = DEFAULT_SEED, n_modes: int = 8,
                         kmax: int = 16, noise: float = 1e-3):
    """The sum of sine modes of heat_u0_modes (the same wave numbers and
    amplitudes) formed directly on a torch device, for grids too large to
    generate on the host in seconds (1024^3: 8.6 GB).  The noise, of the same
    distribution, comes from torch's seeded generator on that device, so it
    is a different draw than heat_u0_modes's."""
    import torch
    modes, amps = draw_modes(seed, n_modes, kmax)
    f64 = torch.float64
    xs = torch.from_numpy(grid_coords(nx)).to(device)
    ys = torch.from_numpy(grid_coords(ny)).to(device)
    zs = torch.from_numpy(grid_coords(nz)).to(device)
    u = torch.zeros((nz, ny, nx), dtype=f64, device=device)
    for (kx, ky, kz), a in zip(modes, amps):
        sx = torch.sin(kx * np.pi * xs)
        sy = torch.sin(ky * np.pi * ys)
        sz = a * torch.sin(kz * np.pi * zs)
        u += sz[:, None, None] * (sy[:, None] * sx[None, :])[None, :, :]
    if noise:
        gen = torch.Generator(device=device).manual_seed(seed * 7919 + 1)
        u += noise * (2.0 * torch.rand((nz, ny, nx), dtype=f64, device=device, generator=gen) - 1.0)
    return u


def cg_rhs(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    return np.random.default_rng([seed, 2]).standard_normal(n)


def lap7_csr(nx: int, ny: int, nz: int):
    """(rowptr int32, col int32, val float64) of the 7-point Dirichlet
    Laplacian: diagonal 6, -1 towards each interior face neighbour, rows and
    columns in natural order, columns ascending within a row."""
    n = nx * ny * nz
    if n >= 2**31 or 7 * n >= 2**31:
        raise ValueError("grid too large for int32 CSR indices")
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k, j, i = k.reshape(-1), j.reshape(-1), i.reshape(-1)
    row = np.arange(n, dtype=np.int64)
    # neighbour slots in ascending column order: z-1, y-1, x-1, self, x+1, y+1, z+1
    offs = [-(nx * ny), -nx, -1, 0, 1, nx, nx * ny]
    present = [k > 0, j > 0, i > 0, np.ones(n, dtype=bool), i < nx - 1, j < ny - 1, k < nz - 1]
    del k, j, i
    pres = np.stack(present, axis=1)
    counts = pres.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    cols = np.empty((n, 7), dtype=np.int32)
    vals = np.empty((n, 7), dtype=np.float64)
    for s, o in enumerate(offs):
        cols[:, s] = (row + o).astype(np.int32)
        vals[:, s] = 6.0 if o == 0 else -1.0
    mask = pres.reshape(-1)
    col = cols.reshape(-1)[mask]
    val = vals.reshape(-1)[mask]
    return rowptr.astype(np.int32), np.ascontiguousarray(col), np.ascontiguousarray(val)


def heat_batch_specs(n: int = 256, seed: int = DEFAULT_SEED, edge=(16, 128), steps=(50, 500)):
    """The batching workload's heat grids: edges log-uniform in [16, 128]
    (independently per axis, so non-cubic), r ~ U[0.05, 0.16], steps ~ U{50..500},
    FP64 and FP32 alternating; u0 ~ U[-1, 1].  Returns a list of dicts."""
    rng = np.random.default_rng([seed, 3])
    out = []
    for g in range(n):
        nz, ny, nx = (int(v) for v in np.round(np.exp(rng.uniform(np.log(edge[0]), np.log(edge[1]), 3))))
        out.append(dict(shape=(nz, ny, nx), r=float(rng.uniform(0.05, 0.16)),
                        steps=int(rng.integers(steps[0], steps[1] + 1)),
                        dtype="f32" if g % 2 else "f64",
                        u0=rng.uniform(-1.0, 1.0, size=(nz, ny, nx))))
    return out


def cg_batch_specs(n: int = 64, seed: int = DEFAULT_SEED, edge=(32, 128)):
    """The batching workload's CG systems: 7-point Laplacians with edges
    log-uniform in [32, 128] per axis, b ~ N(0, 1).  Returns (shape, b) pairs."""
    rng = np.random.default_rng([seed, 4])
    out = []
    for i in range(n):
        nz, ny, nx = (int(v) for v in np.round(np.exp(rng.uniform(np.log(edge[0]), np.log(edge[1]), 3))))
        out.append(((nz, ny, nx), rng.standard_normal(nx * ny * nz)))
    return out
