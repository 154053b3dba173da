"""The temporal-depth autotuner: picks the fastest measured depth, caches it
by GPU, arithmetic and size class, and reuses the cache (CPU, fake timer)."""
from paper_2608_11882_gb300.autotune import Tuner, key, size_class


def test_size_class_rounds_edges_up_to_powers_of_two():
    assert size_class((512, 500, 3)) == "512x512x4"
    assert key("GB300", "f32", (64, 64, 64)) == "GB300|f32|64x64x64"


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def timer(arith, shape, d):
        calls.append(d)
        return {1: 3.0, 2: 1.0, 3: 2.0, 4: 5.0}[d]

    t = Tuner(tmp_path / "c.json", timer=timer, gpu_name="fake")
    assert t.best_depth("f32", (100, 100, 100)) == 2
    assert sorted(calls) == [1, 2, 3, 4]
    t2 = Tuner(tmp_path / "c.json", timer=lambda *a: 1 / 0, gpu_name="fake")
    assert t2.best_depth("f32", (120, 90, 100)) == 2          # same size class, from the file
    assert t2.cache["fake|f32|128x128x128"]["seconds_per_step"]["4"] == 5.0
    calls.clear()
    assert t.best_depth("f32", (100, 100, 100), retune=True) == 2 and len(calls) == 4
