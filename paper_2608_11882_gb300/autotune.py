"""Autotuner for the heat path's launch shapes.

For a single grid it chooses the temporal depth (steps per pass over HBM: 1 =
the Interior + Boundary kernels every step, 2..4 = the temporally blocked
kernel) together with the Interior kernel's planes per block (the library's
choice, half of it or twice it); for a grid inside a batch it chooses the
planes per work item and the column tile width (64 or 32 columns) of the
persistent batched kernel (or the library's choice of both).  Each candidate is
timed on the actual device on a short sample of steps of a grid of the same
shape and arithmetic; the fastest is cached in a JSON file keyed by GPU name,
arithmetic and size class, so later grids of that kind start from the cached
choice.  The choices change speed, and results only through rounding: FP32
and FP64-pipe results are bitwise equal across depths, FIXED64 may rescale at
other steps, a plain FP64 handle runs the exact-sum arithmetic at depth 1 and
the FP64 pipe at depths 2..4 (both within the FP64 tolerance of the exact
update); planes per block and per batch item never change a result.
"""
from __future__ import annotations

import json
import os
import threading
from pathlib import Path

DEPTHS = (1, 2, 3, 4)
# (depth, factor on the library's planes per Interior block); depth >= 2 passes
# choose their own chunking
CANDIDATES = ((1, 1.0), (1, 0.5), (1, 2.0), (2, 1.0), (3, 1.0), (4, 1.0))
# (planes per batched work item, column-tile width): 0 = the library's choice,
# -1 = whole columns
BATCH_CANDIDATES = ((0, 0), (32, 64), (16, 64), (-1, 64), (32, 32), (16, 32), (-1, 32))
_DEFAULT_CACHE = Path(os.environ.get("HEATCG_TUNE_CACHE", Path.home() / ".cache" / "heatcg_tune.json"))
_lock = threading.Lock()


def size_class(shape) -> str:
    """Grids in the same class share a tuning result: each edge rounded to the
    next power of two."""
    return "x".join(str(1 << max(0, (int(e) - 1).bit_length())) for e in shape)


def key(gpu: str, arith: str, shape) -> str:
    return f"{gpu}|{arith}|{size_class(shape)}"


def batch_kz_for(shape, choice: int) -> int:
    """The kz argument of heat_batch_create_tiled for a cached batch choice."""
    return int(shape[0]) if choice == -1 else int(min(choice, shape[0])) if choice > 0 else 0


class Tuner:
    def __init__(self, cache_path: Path | str | None = None, timer=None, batch_timer=None,
                 gpu_name: str | None = None):
        """timer(arith, shape, depth, kc_factor) and batch_timer(arith, shape, kz,
        tile_w) return seconds per step (defaults: CUDA-event timings on the
        device)."""
        self.path = Path(cache_path) if cache_path else _DEFAULT_CACHE
        self.timer = timer
        self.batch_timer = batch_timer
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

    def best(self, arith: str, shape, retune: bool = False) -> dict:
        """{"depth": d, "kc_factor": f} for this arithmetic ("f64", "f32",
        "fixed64", "f64exact", "f64pipe") and shape (nz, ny, nx), timing every
        candidate if no cached result exists (or retune is set)."""
        k = key(self.gpu, arith, shape)
        hit = self.cache.get(k)
        if not retune and hit and "kc_factor" in hit:
            return {"depth": int(hit["depth"]), "kc_factor": float(hit["kc_factor"])}
        timer = self.timer or _gpu_timer
        times = {c: float(timer(arith, shape, c[0], c[1])) for c in CANDIDATES}
        d, f = min(times, key=times.get)
        self.cache[k] = {"depth": d, "kc_factor": f,
                         "seconds_per_step": {f"{a}x{b}": t for (a, b), t in times.items()}}
        self._save()
        return {"depth": d, "kc_factor": f}

    def best_depth(self, arith: str, shape, retune: bool = False) -> int:
        return self.best(arith, shape, retune)["depth"]

    def best_batch(self, arith: str, shape, retune: bool = False) -> dict:
        """{"kz": planes per work item, "tile_w": column-tile width} for a grid of
        this arithmetic ("f64" or "f32") and shape inside a batch (the
        arguments of heat_batch_create_tiled; 0 = the library's choice), timing
        every candidate if none is cached."""
        k = "batch|" + key(self.gpu, arith, shape)
        hit = self.cache.get(k)
        if not retune and hit and "tile_w" in hit:
            return {"kz": batch_kz_for(shape, int(hit["kz"])), "tile_w": int(hit["tile_w"])}
        timer = self.batch_timer or _gpu_batch_timer
        cands, seen = [], set()
        for c, w in BATCH_CANDIDATES:
            real = (batch_kz_for(shape, c), w)
            if (c, w) == (0, 0) or real not in seen:
                cands.append((c, w))
                seen.add(real)
        times = {cw: float(timer(arith, shape, batch_kz_for(shape, cw[0]), cw[1])) for cw in cands}
        c, w = min(times, key=times.get)
        self.cache[k] = {"kz": c, "tile_w": w,
                         "seconds_per_step": {f"{a}x{b}": t for (a, b), t in times.items()}}
        self._save()
        return {"kz": batch_kz_for(shape, c), "tile_w": w}


def _flags(pkg, arith):
    return {"fixed64": pkg.HS_FIXED64, "f64exact": pkg.HS_EXACT_ROUNDING,
            "f64pipe": pkg.HS_FP64_PIPE}.get(arith, 0)


def _gpu_timer(arith: str, shape, depth: int, kc_factor: float = 1.0, steps: int = 24) -> float:
    """Seconds per step of heat_step on the current device (CUDA events)."""
    import numpy as np
    import torch

    import paper_2608_11882_gb300 as pkg
    from paper_2608_11882_gb300 import _native as native
    nz, ny, nx = shape
    dtype = "f32" if arith == "f32" else "f64"
    u0 = np.random.default_rng(0).uniform(-1, 1, size=shape)
    with pkg.Heat(nx, ny, nz, 0.1, dtype=dtype, flags=_flags(pkg, arith), tdepth=depth) as h:
        if kc_factor != 1.0:
            lib_kc = native.heat_get_kchunk(h.handle)
            native.heat_set_kchunk(h.handle, max(4, int(round(lib_kc * kc_factor))))
        h.upload(u0.astype(h.np_dtype))
        h.step(depth * 2)   # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        e0.record(s)
        h.step(steps)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3 / steps


def _gpu_batch_timer(arith: str, shape, kz: int, tile_w: int, copies: int = 8, steps: int = 32) -> float:
    """Seconds per step of a batch of `copies` grids of this shape advanced
    together by heat_batch (planes per work item kz, column-tile width tile_w;
    0 = the library's choice)."""
    import numpy as np
    import torch

    import paper_2608_11882_gb300 as pkg
    nz, ny, nx = shape
    dtype = "f32" if arith == "f32" else "f64"
    u0 = np.random.default_rng(0).uniform(-1, 1, size=shape)
    heats = [pkg.Heat(nx, ny, nz, 0.1, dtype=dtype, tdepth=1) for _ in range(copies)]
    try:
        for h in heats:
            h.upload(u0.astype(h.np_dtype))
        s = torch.cuda.current_stream()
        with pkg.HeatBatch(heats, [steps] * copies, stream=s, kz=[kz] * copies, tile_w=[tile_w] * copies) as b:
            b.run(use_graph=False).wait()   # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            b.run(use_graph=False)
            e1.record(s)
            b.wait()
            return e0.elapsed_time(e1) * 1e-3 / steps
    finally:
        for h in heats:
            h.close()
