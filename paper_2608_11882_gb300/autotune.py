"""Autotuner for the heat path's temporal depth (steps per pass over HBM).

For a grid shape and arithmetic it times ``heat_step`` with every built depth
(1 = Interior + Boundary kernels every step, 2..4 = the temporally blocked
kernel) on a short sample of steps on the actual device, keeps the fastest,
and caches the choice in a JSON file keyed by GPU name, arithmetic and size
class, so later handles of that kind start from the cached depth.  Results
depend on the choice only through rounding: FP32 and FP64-pipe results are
bitwise equal across depths, FIXED64 may rescale at other steps, and a plain
FP64 handle runs the exact-sum arithmetic at depth 1 and the FP64 pipe at
depths 2..4, both within the FP64 tolerance of the exact update.
"""
from __future__ import annotations

import json
import os
import threading
from pathlib import Path

DEPTHS = (1, 2, 3, 4)
_DEFAULT_CACHE = Path(os.environ.get("HEATCG_TUNE_CACHE", Path.home() / ".cache" / "heatcg_tune.json"))
_lock = threading.Lock()


def size_class(shape) -> str:
    """Grids in the same class share a tuning result: each edge rounded to the
    next power of two."""
    return "x".join(str(1 << max(0, (int(e) - 1).bit_length())) for e in shape)


def key(gpu: str, arith: str, shape) -> str:
    return f"{gpu}|{arith}|{size_class(shape)}"


class Tuner:
    def __init__(self, cache_path: Path | str | None = None, timer=None, gpu_name: str | None = None):
        self.path = Path(cache_path) if cache_path else _DEFAULT_CACHE
        self.timer = timer           # timer(arith, shape, depth) -> seconds per step
        self._gpu = gpu_name
        self.cache = self._load()

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def _save(self) -> None:
        with _lock:
            self.path.parent.mkdir(parents=True, exist_ok=True)
            tmp = self.path.with_suffix(f".{os.getpid()}.tmp")
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    @property
    def gpu(self) -> str:
        if self._gpu is None:
            import torch
            self._gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
        return self._gpu

    def best_depth(self, arith: str, shape, retune: bool = False) -> int:
        """The fastest depth for this arithmetic ("f64", "f32", "fixed64",
        "f64exact") and shape (nz, ny, nx), timing every depth if no cached
        result exists (or retune is set)."""
        k = key(self.gpu, arith, shape)
        if not retune and k in self.cache:
            return int(self.cache[k]["depth"])
        timer = self.timer or _gpu_timer
        times = {d: float(timer(arith, shape, d)) for d in DEPTHS}
        best = min(times, key=times.get)
        self.cache[k] = {"depth": best, "seconds_per_step": times}
        self._save()
        return best


def _gpu_timer(arith: str, shape, depth: int, steps: int = 24) -> float:
    """Seconds per step of heat_step on the current device (CUDA events)."""
    import numpy as np
    import torch

    import paper_2608_11882_gb300 as pkg
    nz, ny, nx = shape
    flags = {"fixed64": pkg.HS_FIXED64, "f64exact": pkg.HS_EXACT_ROUNDING,
             "f64pipe": pkg.HS_FP64_PIPE}.get(arith, 0)
    dtype = "f32" if arith == "f32" else "f64"
    u0 = np.random.default_rng(0).uniform(-1, 1, size=shape)
    with pkg.Heat(nx, ny, nz, 0.1, dtype=dtype, flags=flags, tdepth=depth) as h:
        h.upload(u0.astype(h.np_dtype))
        h.step(depth * 2)   # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        e0.record(s)
        h.step(steps)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3 / steps
