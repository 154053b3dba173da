"""Writes tests/golden/heat_small_oracle.json and cg_small_oracle.json.

Calls only ``oracle`` and the seeded generators in ``workloads``; run it from
the repository root with ``python tests/golden/make_golden.py``.  The stored
values are regression anchors for the oracle itself (for example across the
x86 and Arm builds); the pins in tests/test_oracle_*.py are what tie it to the
mathematics.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import cg_rhs, heat_u0_single_mode, lap7_csr  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLE = [(0, 0, 0), (31, 32, 33), (63, 63, 63), (10, 50, 3), (5, 0, 62)]


def main():
    u0 = heat_u0_single_mode(64, 64, 64, seed=20261202)
    u = oracle.heat_run(u0, 0.1, 100, threads=oracle.max_threads())
    heat = {
        "workload": "heat 64^3 interior, h=1/65, r=0.1, 100 steps, u0 = sin sin sin + 0.01 U[-1,1], seed 20261202",
        "sum": float(u.sum()), "max_abs": float(np.abs(u).max()),
        "samples": [{"kji": list(p), "value": float(u[p])} for p in SAMPLE],
    }
    with open(os.path.join(HERE, "heat_small_oracle.json"), "w") as f:
        json.dump(heat, f, indent=1)

    nx = ny = nz = 24
    b = cg_rhs(nx * ny * nz, seed=20261202)
    x_mf, info_mf = oracle.cg_solve(b, 1e-8, 2000, shape=(nz, ny, nx))
    x_csr, info_csr = oracle.cg_solve(b, 1e-8, 2000, csr=lap7_csr(nx, ny, nz))
    cg = {
        "workload": "CG 24^3 7-point Dirichlet Laplacian, b ~ N(0,1) seed 20261202, rtol 1e-8, x0 = 0",
        "matrix_free": dict(info_mf, x_norm=float(np.linalg.norm(x_mf))),
        "csr": dict(info_csr, x_norm=float(np.linalg.norm(x_csr))),
    }
    with open(os.path.join(HERE, "cg_small_oracle.json"), "w") as f:
        json.dump(cg, f, indent=1)


if __name__ == "__main__":
    main()
