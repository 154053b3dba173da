"""The oracle against its stored regression anchors (written by
tests/golden/make_golden.py, which calls only the oracle) and against the
paper's printed acceptance rule."""
import json
import os

import numpy as np

from workloads import cg_rhs, heat_u0_single_mode

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_heat_small_matches_stored_anchor(oracle_mod):
    g = _load("heat_small_oracle.json")
    u = oracle_mod.heat_run(heat_u0_single_mode(64, 64, 64, seed=20261202), 0.1, 100, threads=4)
    # u0 comes from numpy's sin, which may differ by an ulp between machines.
    assert abs(float(u.sum()) - g["sum"]) <= 1e-10 * abs(g["sum"])
    assert abs(float(np.abs(u).max()) - g["max_abs"]) <= 1e-13
    for s in g["samples"]:
        assert abs(float(u[tuple(s["kji"])]) - s["value"]) <= 1e-13


def test_cg_small_matches_stored_anchor(oracle_mod):
    g = _load("cg_small_oracle.json")
    b = cg_rhs(24 ** 3, seed=20261202)
    x, info = oracle_mod.cg_solve(b, 1e-8, 2000, shape=(24, 24, 24))
    assert abs(info["iters"] - g["matrix_free"]["iters"]) <= 1
    assert info["relres_true"] <= 1e-8
    assert abs(np.linalg.norm(x) - g["matrix_free"]["x_norm"]) <= 1e-9 * g["matrix_free"]["x_norm"]


def test_paper_constants_are_consistent():
    c = _load("paper_constants.json")
    # Algorithm heat3d: dt = h^2/(12 kappa_max), beta = dt/(2h^2) = 1/(24 kappa_max).
    kmax = c["kappa_max"]["value"]
    beta = (1.0 / (12 * kmax)) / 2.0
    assert abs(beta - 1.0 / (24 * kmax)) < 1e-15
    # dt/h^2 = 1/(12*0.95) = 0.0877 lies inside both the printed 1-D bound and the 3-D bound 1/6.
    assert 1.0 / (12 * kmax) < c["stability_printed"]["value"] and 1.0 / (12 * kmax) < 1.0 / 6.0
    assert c["acceptance_atol"]["value"] == 1e-6 and c["acceptance_rtol"]["value"] == 1e-5
