"""Batched heat stepping (one persistent launch for many uneven grids,
FP32 and FP64, optionally a CUDA graph): every grid must equal the same grid
stepped alone through heat_step, bit for bit."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, lib, rel_max_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def draw_batch(n, seed, edge=(16, 128), steps=(50, 500)):
    """Edges log-uniform in [16, 128] (non-cubic), r ~ U[0.05, 0.16],
    steps ~ U{lo..hi}, dtype alternating FP32 / FP64."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(n):
        nz, ny, nx = np.round(np.exp(rng.uniform(np.log(edge[0]), np.log(edge[1]), 3))).astype(int)
        out.append(dict(shape=(int(nz), int(ny), int(nx)), r=float(rng.uniform(0.05, 0.16)),
                        steps=int(rng.integers(steps[0], steps[1] + 1)),
                        dtype="f32" if g % 2 else "f64",
                        u0=rng.uniform(-1, 1, size=(int(nz), int(ny), int(nx)))))
    return out


def alone(pkg, spec, steps):
    nz, ny, nx = spec["shape"]
    with pkg.Heat(nx, ny, nz, spec["r"], dtype=spec["dtype"], tdepth=1) as h:
        h.upload(spec["u0"].astype(h.np_dtype))
        h.step(steps)
        return h.read()


def make_heats(pkg, specs):
    hs = []
    for s in specs:
        nz, ny, nx = s["shape"]
        h = pkg.Heat(nx, ny, nz, s["r"], dtype=s["dtype"], tdepth=1)
        h.upload(s["u0"].astype(h.np_dtype))
        hs.append(h)
    return hs


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone_bitwise(pkg, use_graph):
    specs = draw_batch(14, seed=5, edge=(4, 70), steps=(0, 60))
    specs[3]["steps"] = 0
    heats = make_heats(pkg, specs)
    with pkg.HeatBatch(heats, [s["steps"] for s in specs]) as b:
        b.run(use_graph=use_graph)
        b.wait()
        assert b.lups == sum(np.prod(s["shape"]) * s["steps"] for s in specs)
    for s, h in zip(specs, heats):
        assert h.steps_done == s["steps"]
        assert np.array_equal(h.read(), alone(pkg, s, s["steps"]))
        h.close()


def test_graph_replay_keeps_stepping(pkg):
    specs = draw_batch(6, seed=6, edge=(5, 40), steps=(3, 17))
    heats = make_heats(pkg, specs)
    with pkg.HeatBatch(heats, [s["steps"] for s in specs]) as b:
        for _ in range(3):
            b.run(use_graph=True)
        b.wait()
    for s, h in zip(specs, heats):
        assert np.array_equal(h.read(), alone(pkg, s, 3 * s["steps"]))
        h.close()


def test_batch_against_oracle(pkg):
    specs = draw_batch(4, seed=7, edge=(8, 48), steps=(10, 40))
    for s in specs:
        s["dtype"] = "f64"
    heats = make_heats(pkg, specs)
    with pkg.HeatBatch(heats, [s["steps"] for s in specs]) as b:
        b.run().wait()
    for s, h in zip(specs, heats):
        assert rel_max_err(h.read(), oracle.heat_run(s["u0"], s["r"], s["steps"])) <= F64_REL
        h.close()


def test_batch_rejects_bad_input(pkg):
    a = pkg.Heat(8, 8, 8, 0.1)
    fx = pkg.Heat(8, 8, 8, 0.1, flags=pkg.HS_FIXED64)
    for handles, steps in (([a, a], [1, 1]), ([fx], [1]), ([a], [-1])):
        with pytest.raises(pkg.HeatCGError):
            pkg.HeatBatch(handles, steps)
    a.close()
    fx.close()


def test_batch_workload_256_grids_subset(pkg):
    """The batching workload's recipe (256 grids, edges log-uniform in [16, 128],
    r ~ U[0.05, 0.16], steps ~ U[50, 500], FP32 and FP64); every 16th grid is
    checked against a run alone."""
    specs = draw_batch(256, seed=20261202)
    heats = make_heats(pkg, specs)
    with pkg.HeatBatch(heats, [s["steps"] for s in specs]) as b:
        b.run(use_graph=True).wait()
    for i in range(0, 256, 16):
        assert np.array_equal(heats[i].read(), alone(pkg, specs[i], specs[i]["steps"]))
    for h in heats:
        h.close()


def test_bounded_step_wait_runs_out_then_recovers(pkg):
    """A step wait that runs out (its limit set to a few SM cycles, so a grid's
    step m+1 cannot wait for step m to finish): the run stops early and
    heat_batch_wait reports HS_ETIMEOUT; no fault, no endless wait.  With the
    default limit restored, the same handles re-uploaded give the oracle's
    result, stepped alone and batched."""
    from paper_2608_11882_gb300 import _native as nat
    specs = draw_batch(2, seed=8, edge=(40, 64), steps=(12, 12))
    for s in specs:
        s["dtype"] = "f64"
    heats = make_heats(pkg, specs)
    try:
        nat.heat_batch_set_wait_limit(4)
        b = pkg.HeatBatch(heats, [s["steps"] for s in specs])
    finally:
        nat.heat_batch_set_wait_limit(0)
    with b:
        b.run(use_graph=False)
        with pytest.raises(pkg.HeatCGError) as e:
            b.wait()
        assert e.value.code == nat.HS_ETIMEOUT
    # the handles and the context stay usable
    for s, h in zip(specs, heats):
        h.upload(s["u0"])
        h.step(s["steps"])
        assert rel_max_err(h.read(), oracle.heat_run(s["u0"], s["r"], s["steps"])) <= F64_REL
        h.upload(s["u0"])
    with pkg.HeatBatch(heats, [s["steps"] for s in specs]) as b2:
        b2.run(use_graph=True).wait()
    for s, h in zip(specs, heats):
        assert rel_max_err(h.read(), oracle.heat_run(s["u0"], s["r"], s["steps"])) <= F64_REL
        h.close()
    with pytest.raises(pkg.HeatCGError):
        nat.heat_batch_set_wait_limit(-1)


@pytest.mark.parametrize("kz,tw", [(1, 64), (3, 32), (16, 64), (16, 32), (0, 0), (0, 32)])
def test_z_chunked_items_equal_alone_bitwise(pkg, kz, tw):
    """Work items split into z-chunks of kz planes (1 = one plane per item;
    0 = the library's choice) over 64 x 8 or 32 x 16 column tiles (0: the
    library's choice per grid): the same bits as each grid stepped alone."""
    specs = draw_batch(8, seed=9, edge=(5, 70), steps=(2, 25))
    heats = make_heats(pkg, specs)
    with pkg.HeatBatch(heats, [s["steps"] for s in specs], kz=[kz] * len(specs),
                       tile_w=[tw] * len(specs)) as b:
        b.run(use_graph=True).wait()
    for s, h in zip(specs, heats):
        assert np.array_equal(h.read(), alone(pkg, s, s["steps"]))
        h.close()


def test_tuned_batch_equals_alone(pkg, tmp_path, monkeypatch):
    from paper_2608_11882_gb300 import autotune
    monkeypatch.setattr(autotune, "_DEFAULT_CACHE", tmp_path / "tune.json")
    specs = draw_batch(4, seed=10, edge=(16, 48), steps=(5, 20))
    heats = make_heats(pkg, specs)
    with pkg.HeatBatch(heats, [s["steps"] for s in specs], kz="auto") as b:
        assert len(b.kz) == 4
        b.run().wait()
    for s, h in zip(specs, heats):
        assert np.array_equal(h.read(), alone(pkg, s, s["steps"]))
        h.close()


def test_batch_with_blocked_handles_then_heat_step(pkg):
    """Handles at their default depth (FP32: two steps per pass) join a batch,
    which steps them one step per item; heat_step then continues them in
    blocked passes from the buffer the batch left current.  FP32 results equal
    one-step stepping bit for bit at every depth; the plain FP64 handle (exact
    sum at depth 1) equals itself stepped alone."""
    specs = draw_batch(4, seed=31, edge=(20, 90), steps=(5, 9))
    heats = []
    for s in specs:
        nz, ny, nx = s["shape"]
        h = pkg.Heat(nx, ny, nz, s["r"], dtype=s["dtype"])
        assert h.tdepth == (2 if s["dtype"] == "f32" else 1)
        h.upload(s["u0"].astype(h.np_dtype))
        heats.append(h)
    with pkg.HeatBatch(heats, [s["steps"] for s in specs]) as b:
        b.run(use_graph=False)
        b.wait()
    for s, h in zip(specs, heats):
        h.step(5)
        assert h.steps_done == s["steps"] + 5
        assert np.array_equal(h.read(), alone(pkg, s, s["steps"] + 5)), s["shape"]
        h.close()
