"""Host logic of bench.py that needs no GPU: the roofline objects it reports
and the reference arm (the oracle on the host cores) with its JSON line."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_hbm_roofline_object(bench):
    """FP64 exact-sum Interior at 512^3: algorithmic bytes are 16 B per point of
    planes 1..510, achieved = bytes / launch time, frac = achieved / peak, and
    the measured DRAM traffic per launch sits just above the algorithmic bytes."""
    ms = 0.408
    r = bench.interior_roofline("f64", 512, ms, 6758.5, "measured", 1)
    algo = 512 * 512 * 510 * 16
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6758.5
    assert r["achieved"] == pytest.approx(algo / (ms * 1e-3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6758.5)
    assert r["traffic"] == bench.KERNEL_TRAFFIC_BYTES[("f64", 512, 1)]
    assert 1.0 <= r["traffic_per_algorithmic"] < 1.05
    assert r["frac_of_nominal"] == pytest.approx(r["achieved"] / 7900.0)


def test_roofline_traffic_is_null_where_not_captured(bench):
    for mode, n, depth in (("f32", 512, 1), ("fixed64", 256, 1), ("f64", 256, 1), ("f32", 512, 3)):
        r = bench.interior_roofline(mode, n, 0.2, 6758.5, "measured", depth)
        assert r["traffic"] is None and r["traffic_per_algorithmic"] is None


def test_roofline_traffic_where_captured(bench):
    """Captured kernels report their DRAM bytes per launch, within a few
    percent above the algorithmic bytes (8 B per point per two-step FP32 pass
    over all 512^3 points; 16 B per FIXED64 point of planes 1..510)."""
    r = bench.interior_roofline("f32", 512, 0.27, 6758.5, "measured", 2)
    assert r["traffic"] == bench.KERNEL_TRAFFIC_BYTES[("f32", 512, 2)]
    assert 1.0 <= r["traffic_per_algorithmic"] < 1.06
    r = bench.interior_roofline("fixed64", 512, 0.364, 6758.5, "measured", 1)
    assert r["traffic"] == bench.KERNEL_TRAFFIC_BYTES[("fixed64", 512, 1)]
    assert 1.0 <= r["traffic_per_algorithmic"] < 1.05


def test_alu_roofline_object(bench):
    """The FP64-pipe form is bound by FP64 instruction issue: 7 instructions
    per point against the nominal 0.625 T instructions/s."""
    ms = 1.805
    r = bench.interior_roofline("f64pipe", 512, ms, 6758.5, "measured", 1)
    lup = 512 * 512 * 510
    assert r["bound"] == "alu" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(lup * 7 / (ms * 1e-3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 0.625)
    assert r["hbm_achieved_gbs"] == pytest.approx(lup * 16 / (ms * 1e-3) / 1e9)


def test_blocked_roofline_counts_all_planes_and_steps(bench):
    """A temporally blocked launch covers all n planes and L steps: algorithmic
    bytes are one read and one write of the field per launch."""
    r = bench.interior_roofline("f32", 512, 1.0, 6758.5, "measured", 4)
    assert r["achieved"] == pytest.approx(512 ** 3 * 8 / 1e-3 / 1e9)
    assert r["effective_gbs"] == pytest.approx(4 * r["achieved"])
    assert r["steps_per_launch"] == 4


def test_measured_peaks_file(bench):
    peak, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            assert peak == float(json.load(f)["hbm_gbs"]) and kind == "measured"
    else:
        assert kind == "fallback"


def run_reference(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--heat-n", "20", "--steps", "2", "--warmup", "3"],
                          capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_json_line():
    """--impl reference times the oracle on the host cores and prints one JSON
    line with the base contract's keys, a cpu_baseline describing the run and
    an e2e object with no transfers."""
    p = run_reference()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d
    assert d["impl"] == "reference" and d["unit"] == "GLUP/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["higher_is_better"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "GLUP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    p = run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0 and not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_side_selection(bench):
    import argparse
    ns = lambda **kw: argparse.Namespace(**{"no_side": False, "no_serving": False, "sides": "all", **kw})
    assert bench.sides_of(ns()) == set(bench.SIDES)
    assert bench.sides_of(ns(no_side=True)) == set()
    assert bench.sides_of(ns(sides="mixed,batching")) == {"mixed", "batching"}
    assert bench.sides_of(ns(no_serving=True)) == set(bench.SIDES) - {"serving"}
    with pytest.raises(SystemExit):
        bench.sides_of(ns(sides="bogus"))


def test_cg_byte_models(bench):
    """Bytes per unknown and iteration behind the CG roofline objects: FP64 CG
    moves 16 (SpMV) + 48 (x/r update) + 24 (p update) = 88 B per row; the
    mixed-precision inner iteration 40 B matrix-free (the p update folded into
    the FP32 SpMV: read r and p, write p and q = 16 B, update 24 B) and 44 B
    for CSR (SpMV 8 B + 24 B + p update 12 B), each FP32 value 4 B."""
    assert bench.CG_BYTES_PER_ROW == 16 + 48 + 24
    assert bench.MIXED_INNER_BYTES_PER_ROW == {"matrix_free": 4 * 4 + 6 * 4, "csr": 2 * 4 + 6 * 4 + 3 * 4}
    r = bench.hbm_roofline("CG", 851 * 88 * 256.0 ** 3, 228.5, 6794.8, "measured")
    assert r["frac"] == pytest.approx(851 * 88 * 256.0 ** 3 / 0.2285 / 1e9 / 6794.8)
