"""The autotuner: picks the fastest measured (depth, planes per block) for a
single grid and the fastest planes per batched work item, caches them by GPU,
arithmetic and size class, and reuses the cache (CPU, fake timers)."""
from paper_2608_11882_gb300.autotune import CANDIDATES, Tuner, batch_kz_for, key, size_class


def test_size_class_rounds_edges_up_to_powers_of_two():
    assert size_class((512, 500, 3)) == "512x512x4"
    assert key("GB300", "f32", (64, 64, 64)) == "GB300|f32|64x64x64"


def test_picks_fastest_and_caches(tmp_path):
    calls = []
    table = {(1, 1.0): 3.0, (1, 0.5): 2.5, (1, 2.0): 4.0, (2, 1.0): 1.0, (3, 1.0): 2.0, (4, 1.0): 5.0}

    def timer(arith, shape, d, f):
        calls.append((d, f))
        return table[(d, f)]

    t = Tuner(tmp_path / "c.json", timer=timer, gpu_name="fake")
    assert t.best("f32", (100, 100, 100)) == {"depth": 2, "kc_factor": 1.0}
    assert sorted(calls) == sorted(CANDIDATES)
    t2 = Tuner(tmp_path / "c.json", timer=lambda *a: 1 / 0, gpu_name="fake")
    assert t2.best_depth("f32", (120, 90, 100)) == 2          # same size class, from the file
    assert t2.cache["fake|f32|128x128x128"]["seconds_per_step"]["4x1.0"] == 5.0
    calls.clear()
    assert t.best_depth("f32", (100, 100, 100), retune=True) == 2 and len(calls) == len(CANDIDATES)
    table[(1, 0.5)] = 0.5
    assert t.best("f64", (100, 100, 100)) == {"depth": 1, "kc_factor": 0.5}


def test_batch_choice_picks_fastest_and_caches(tmp_path):
    seen = []

    def bt(arith, shape, kz, w):
        seen.append((kz, w))
        return {(0, 0): 3.0, (40, 64): 2.0, (32, 64): 1.5, (16, 64): 1.2,
                (40, 32): 2.5, (32, 32): 1.4, (16, 32): 1.0}[(kz, w)]

    t = Tuner(tmp_path / "c.json", batch_timer=bt, gpu_name="fake")
    # nz = 40: whole columns (40) and chunks of 32 or 16, each with both tile widths
    assert t.best_batch("f64", (40, 20, 30)) == {"kz": 16, "tile_w": 32}
    assert sorted(seen) == sorted([(0, 0), (32, 64), (16, 64), (40, 64), (32, 32), (16, 32), (40, 32)])
    t2 = Tuner(tmp_path / "c.json", batch_timer=lambda *a: 1 / 0, gpu_name="fake")
    assert t2.best_batch("f64", (60, 30, 17)) == {"kz": 16, "tile_w": 32}   # same class, cached
    assert batch_kz_for((40, 1, 1), -1) == 40 and batch_kz_for((40, 1, 1), 64) == 40
    assert batch_kz_for((40, 1, 1), 0) == 0
