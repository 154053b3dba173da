"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of the oracle's C sources (a dropped term, a wrong sign, index,
stride, coefficient or loop bound, a missing buffer swap, a wrong CG
coefficient), builds it with the oracle's own flags, and runs the pin tests
(test_oracle_heat, test_oracle_heat_vk, test_oracle_cg) against that build in
a separate process: at least one pin must fail.  The unmodified copy must
pass them all.  CPU only."""
import os
import shutil
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "oracle"
PINS = ["tests/test_oracle_heat.py", "tests/test_oracle_heat_vk.py", "tests/test_oracle_cg.py"]

# (name, file, text, replacement): each replacement hits exactly one place
MUTATIONS = [
    ("heat: dropped z neighbours", "heat_oracle.c",
     "const double s = (along_x + along_y) + along_z;", "const double s = (along_x + along_y);"),
    ("heat: wrong sign of the update", "heat_oracle.c",
     "dst[c] = u + r * (s - 6.0 * u);", "dst[c] = u - r * (s - 6.0 * u);"),
    ("heat: wrong centre coefficient", "heat_oracle.c",
     "dst[c] = u + r * (s - 6.0 * u);", "dst[c] = u + r * (s - 4.0 * u);"),
    ("heat: transposed stride", "heat_oracle.c",
     "const double along_y = src[c - sy] + src[c + sy];", "const double along_y = src[c - sz] + src[c + sy];"),
    ("heat: last x column skipped", "heat_oracle.c",
     "            for (int64_t i = 1; i <= nx; ++i) {\n                const size_t c = pad_index(i, j, k, nx, ny);\n                const double u = src[c];",
     "            for (int64_t i = 1; i < nx; ++i) {\n                const size_t c = pad_index(i, j, k, nx, ny);\n                const double u = src[c];"),
    ("heat: buffers not swapped", "heat_oracle.c",
     "        double* t = a; a = b; b = t;   /* pointer swap, no data movement */", ""),
    ("variable kappa: wrong beta", "heat_oracle.c",
     "const double bx = dt / (2.0 * hx * hx)", "const double bx = dt / (hx * hx)"),
    ("variable kappa: wrong face weight", "heat_oracle.c",
     "const double dx = (kap[c + 1] + kc) * (a[c + 1] - u)", "const double dx = (kap[c + 1] + kap[c + 1]) * (a[c + 1] - u)"),
    ("variable kappa: dropped source", "heat_oracle.c",
     "b[c] = (u + fdt[c]) + s;", "b[c] = u + s;"),
    ("variable kappa: dropped z axis", "heat_oracle.c",
     "const double s = (bx * dx + by * dy) + bz * dz;", "const double s = (bx * dx + by * dy);"),
    ("Laplacian: wrong diagonal", "cg_oracle.c",
     "s = s + 6.0 * p[row];", "s = s + 5.0 * p[row];"),
    ("Laplacian: dropped z+1 neighbour", "cg_oracle.c",
     "if (k < nz - 1) s = s + (-1.0) * p[row + sz];", ""),
    ("CG: inverted beta", "cg_oracle.c",
     "const double beta = rho_new / rho;", "const double beta = rho / rho_new;"),
    ("CG: wrong sign of the x update", "cg_oracle.c",
     "x[i] = x[i] + alpha * p[i];", "x[i] = x[i] - alpha * p[i];"),
    ("CG: steepest descent (p update dropped)", "cg_oracle.c",
     "p[i] = r[i] + beta * p[i];", "p[i] = r[i] + 0.0 * beta * p[i];"),
    ("CG: dot of a with itself", "cg_oracle.c",
     "s = s + a[i] * b[i];", "s = s + a[i] * a[i];"),
]


def build_copy(tmp: Path, mutation=None) -> Path:
    for f in ("heat_oracle.c", "cg_oracle.c"):
        text = (SRC / f).read_text()
        if mutation and mutation[1] == f:
            assert text.count(mutation[2]) == 1, mutation[0]
            text = text.replace(mutation[2], mutation[3])
        (tmp / f).write_text(text)
    lib = tmp / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
                    "-o", str(lib), str(tmp / "heat_oracle.c"), str(tmp / "cg_oracle.c"), "-lm"], check=True)
    return lib


def run_pins(lib: Path) -> subprocess.CompletedProcess:
    env = dict(os.environ, ORACLE_LIB=str(lib))
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"]
                          + PINS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def gcc():
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")


def test_unmodified_copy_passes_the_pins(gcc, tmp_path):
    res = run_pins(build_copy(tmp_path))
    assert res.returncode == 0, res.stdout[-2000:]


@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(gcc, tmp_path, mutation):
    res = run_pins(build_copy(tmp_path, mutation))
    assert res.returncode != 0 and " failed" in res.stdout, res.stdout[-2000:]
