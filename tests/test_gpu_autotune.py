"""The autotuner on the device: it times real handles and batches, caches its
choices, and the tuned launch shapes give the same results (bit for bit where
the arithmetic is the same, else within the FP64 gate of the oracle)."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, lib, rel_max_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def test_tuner_on_a_real_handle_caches_and_keeps_results(pkg, tmp_path, monkeypatch):
    from paper_2608_11882_gb300 import autotune
    cache = tmp_path / "tune.json"
    monkeypatch.setattr(autotune, "_DEFAULT_CACHE", cache)
    shape = (40, 48, 70)
    nz, ny, nx = shape
    u0 = np.random.default_rng(61).uniform(-1, 1, size=shape)
    t = autotune.Tuner()
    choice = t.best("f32", shape)
    assert choice["depth"] in autotune.DEPTHS and cache.exists()
    assert autotune.Tuner().best("f32", shape) == choice          # from the file
    pick = t.best_batch("f64", shape)
    assert 0 <= pick["kz"] <= nz and pick["tile_w"] in (0, 32, 64)
    with pkg.Heat(nx, ny, nz, 0.12, dtype="f32", tdepth="auto") as h:
        tuned = h.upload(u0.astype(np.float32)).step(30).read()
    with pkg.Heat(nx, ny, nz, 0.12, dtype="f32", tdepth=1) as h:
        plain = h.upload(u0.astype(np.float32)).step(30).read()
    assert np.array_equal(tuned, plain)      # FP32: every depth and chunking gives the same bits
    with pkg.Heat(nx, ny, nz, 0.12, tdepth="auto") as h:
        f64 = h.upload(u0).step(30).read()
    assert rel_max_err(f64, oracle.heat_run(u0, 0.12, 30)) <= F64_REL


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_kchunk_changes_speed_only(pkg, dtype):
    shape = (57, 33, 70)
    nz, ny, nx = shape
    u0 = np.random.default_rng(62).uniform(-1, 1, size=shape)
    outs = []
    for planes in (0, 1, 5, 8, 1000):
        with pkg.Heat(nx, ny, nz, 0.15, dtype=dtype, tdepth=1) as h:
            h.kchunk = planes
            assert h.kchunk == (min(planes, nz - 2) if planes else h.kchunk)
            outs.append(h.upload(u0.astype(h.np_dtype)).step(9).read())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
