"""Continuous-batching solve server for heat and CG requests.

Requests (heat: a field, r and a step count; CG: a right-hand side and a
tolerance) arrive over time.  The scheduler admits a request as soon as it has
arrived, a slot is free and its device memory fits the free-HBM budget; the
admitted request's field stays resident on the device until it completes.
Every tick all admitted heat requests advance together by up to `quantum`
steps in ONE batched persistent launch (heat_batch_*), so requests that arrive
while others are running join the next tick's batch.  A tick's batch runs
while the host admits and uploads new requests and reads back those the
previous tick finished (on a stream of their own), so host work overlaps the
device work.  CG requests are solved on worker threads, each with its own CUDA
stream, so they overlap on the device with the heat batches and with each
other.  The per-point and
per-iteration arithmetic is the library's, and a request's result does not
depend on what it ran beside: heat equals heat_step alone and CG equals
cg_run alone, bit for bit.

The GPU work goes through a backend object so the scheduling logic can be
exercised without a GPU (``FakeBackend`` in the tests).  Latency is
completion minus arrival; throughput is heat lattice-point updates per
second of makespan.
"""
from __future__ import annotations

import math
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    kind: str                    # "heat" or "cg"
    shape: tuple                 # (nz, ny, nx)
    dtype: str = "f64"           # heat: "f64" or "f32"; CG is FP64
    r: float = 0.1               # heat
    steps: int = 0               # heat
    rtol: float = 1e-8           # CG
    max_iter: int = 100000       # CG
    arrival: float = 0.0         # seconds after the start of the run
    payload: object = None       # heat: u0 (nz, ny, nx); CG: b (n,)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))

    @property
    def lups(self) -> int:
        return self.points * self.steps if self.kind == "heat" else 0


@dataclass
class Result:
    rid: int
    kind: str
    arrival: float
    admitted: float
    completed: float
    output: object = None
    info: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


def device_bytes(req: Request) -> int:
    """Device memory a request holds while admitted (both padded field buffers
    and, for FP64, the 64-byte per-step state, for heat; r, p, q, b and x for
    CG), with row padding to 128 bytes."""
    nz, ny, nx = req.shape
    if req.kind == "heat":
        elem = 8 if req.dtype == "f64" else 4
        pitch = -(-(32 // elem + nx + 1) * elem // 128) * 128
        return 2 * pitch * (ny + 2) * (nz + 2) + (64 if req.dtype == "f64" else 0)
    return 5 * 8 * req.points


def kbar(samples) -> float:
    """The paper's per-point cost model (Section 5.6): one step costs
    t_step = k (N-2)^3 for (N-2)^3 computed points, so each grid size gives
    k = T_total / (n_steps (N-2)^3), and k-bar is the plain mean of k over the
    sizes measured.  samples: (points, steps, seconds) per grid size, points =
    the interior points (N-2)^3.  (The paper's printed rearrangement multiplies
    by (N-2)^3 where the division is meant.)"""
    ks = [t / (steps * pts) for pts, steps, t in samples]
    if not ks:
        raise ValueError("kbar needs at least one sample")
    return sum(ks) / len(ks)


def predict_seconds(req: Request, kbars: dict) -> float:
    """Standalone device time of a heat request by the k-bar model of its
    arithmetic: k-bar * points * steps (nan when no k-bar is known)."""
    k = kbars.get(req.dtype) if kbars else None
    return float(k) * req.points * req.steps if (k and req.kind == "heat") else float("nan")


def percentile(values, q: float) -> float:
    """Nearest-rank percentile (q in [0, 100])."""
    if not values:
        return float("nan")
    v = sorted(values)
    k = max(0, min(len(v) - 1, int(math.ceil(q / 100.0 * len(v))) - 1))
    return float(v[k])


class GpuBackend:
    """The library on the current CUDA device: heat handles (uploads and reads
    on an I/O stream) advanced by heat_batch on a batch stream, CG contexts on
    per-worker streams."""

    def __init__(self, workers: int = 4):
        import torch

        import paper_2608_11882_gb300 as pkg
        self.torch = torch
        self.pkg = pkg
        self.stream = torch.cuda.Stream()      # heat batches
        self.io_stream = torch.cuda.Stream()   # heat handles: create, upload, read, release
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self._local = threading.local()
        self._stage = None   # pinned staging for read-backs, grown on demand

    def free_bytes(self) -> int:
        return int(self.torch.cuda.mem_get_info()[0])

    def calibrate(self, edges=(96, 160, 256), steps=40) -> dict:
        """k-bar per arithmetic from heat_step alone on this device (CUDA events
        around `steps` steps of an edge^3 grid, one warm-up pass each)."""
        torch = self.torch
        out = {}
        for dt in ("f64", "f32"):
            samples = []
            for n in edges:
                with self.pkg.Heat(n, n, n, 0.1, dtype=dt, stream=self.stream, tdepth=1) as h:
                    h.upload(np.random.default_rng(n).uniform(-1, 1, (n, n, n)).astype(h.np_dtype))
                    h.step(4)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(self.stream)
                    h.step(steps)
                    e1.record(self.stream)
                    e1.synchronize()
                    samples.append((n ** 3, steps, e0.elapsed_time(e1) * 1e-3))
            out[dt] = kbar(samples)
        return out

    def heat_open(self, req: Request):
        nz, ny, nx = req.shape
        h = self.pkg.Heat(nx, ny, nz, req.r, dtype=req.dtype, stream=self.io_stream, tdepth=1)
        # pageable memory: pinning a buffer of every request's own size costs more than it saves
        h.upload(np.ascontiguousarray(req.payload, dtype=h.np_dtype))
        return h

    def heat_launch(self, handles, steps):
        """Start one tick's batch (returns at once; heat_wait ends it)."""
        b = self.pkg.HeatBatch(handles, steps, stream=self.stream)
        b.run(use_graph=False)
        return b

    def heat_wait(self, b) -> None:
        b.wait()
        b.close()

    def heat_advance(self, handles, steps) -> None:
        self.heat_wait(self.heat_launch(handles, steps))

    def heat_close(self, h):
        # the device-to-host copy into pinned staging is fast; the host copy
        # into the result array follows (a pageable destination is far slower)
        torch = self.torch
        tdt = torch.float64 if h.np_dtype == np.float64 else torch.float32
        nbytes = h.count * np.dtype(h.np_dtype).itemsize
        if self._stage is None or self._stage.numel() < nbytes:
            self._stage = torch.empty(max(nbytes, 1 << 26), dtype=torch.uint8, pin_memory=True)
        view = self._stage[:nbytes].view(tdt)
        h.read(view)
        h.close()
        return view.numpy().reshape(h.shape).copy()

    def _cg_job(self, req: Request):
        torch = self.torch
        s = getattr(self._local, "stream", None)
        if s is None:
            s = self._local.stream = torch.cuda.Stream()
        nz, ny, nx = req.shape
        with torch.cuda.stream(s):
            b = torch.from_numpy(np.ascontiguousarray(req.payload, dtype=np.float64)).pin_memory()
            b = b.cuda(non_blocking=True)
            with self.pkg.CG(self.pkg.Operator.stencil(nx, ny, nz), stream=s) as cg:
                x, info = cg.run(b, rtol=req.rtol, max_iter=req.max_iter)
            out = x.cpu().numpy()
        return out, info

    def cg_submit(self, req: Request):
        return self.pool.submit(self._cg_job, req)

    def close(self):
        self.pool.shutdown(wait=True)


class Server:
    """Continuous-batching scheduler (see the module docstring).

    hbm_budget: bytes the admitted requests may hold at once (default: the
    backend's free device memory minus `reserve` at start).  max_slots:
    requests admitted at once.  quantum: heat steps per tick.
    """

    def __init__(self, backend, hbm_budget: int | None = None, reserve: int = 2 << 30,
                 max_slots: int = 32, quantum: int = 64, clock=time.perf_counter,
                 sleep=time.sleep, kbars: dict | None = None):
        """kbars: k-bar per arithmetic (GpuBackend.calibrate); each heat result
        then carries its predicted standalone device time in info["predicted_s"]."""
        self.backend = backend
        self.kbars = kbars or {}
        self.budget = hbm_budget if hbm_budget is not None else max(0, backend.free_bytes() - reserve)
        self.max_slots = max_slots
        self.quantum = quantum
        self.clock = clock
        self.sleep = sleep
        self.peak_bytes = 0
        self.peak_slots = 0
        self.rejected = []

    def run(self, requests):
        """Serve requests (their arrival offsets relative to the start) and
        return the results in request-id order."""
        pending = sorted(requests, key=lambda q: (q.arrival, q.rid))
        for q in pending:
            if device_bytes(q) > self.budget:
                self.rejected.append(q.rid)
        pending = [q for q in pending if q.rid not in set(self.rejected)]
        launch = getattr(self.backend, "heat_launch", None)
        t0 = self.clock()
        used = 0
        heat = {}          # rid -> [req, handle, remaining, admitted]
        cg = {}            # rid -> [req, future, admitted]
        results = {}
        inflight = None    # (token, [(rid, steps)]) of the tick on the device
        i = 0
        while i < len(pending) or heat or cg or inflight is not None:
            worked = False
            # the tick in flight ends: its requests have advanced
            if inflight is not None:
                token, parts = inflight
                self.backend.heat_wait(token)
                for rid, st in parts:
                    heat[rid][2] -= st
                inflight = None
                worked = True
            # admit everything that has arrived and fits
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                q = pending[i]
                need = device_bytes(q)
                if len(heat) + len(cg) >= self.max_slots or used + need > self.budget:
                    break
                used += need
                if q.kind == "heat":
                    heat[q.rid] = [q, self.backend.heat_open(q), q.steps, now]
                else:
                    cg[q.rid] = [q, self.backend.cg_submit(q), now]
                i += 1
            self.peak_bytes = max(self.peak_bytes, used)
            self.peak_slots = max(self.peak_slots, len(heat) + len(cg))
            # start the next tick: every admitted heat request with steps left
            live = [(rid, v) for rid, v in heat.items() if v[2] > 0]
            if live:
                steps = [min(self.quantum, v[2]) for _, v in live]
                handles = [v[1] for _, v in live]
                if launch is not None:
                    inflight = (launch(handles, steps), [(rid, st) for (rid, _), st in zip(live, steps)])
                else:
                    self.backend.heat_advance(handles, steps)
                    for (_, v), st in zip(live, steps):
                        v[2] -= st
                worked = True
            # read back and release the finished heat requests (while the tick runs)
            busy = {rid for rid, _ in inflight[1]} if inflight is not None else set()
            for rid in [r for r, v in heat.items() if v[2] == 0 and r not in busy]:
                q, h, _, adm = heat.pop(rid)
                out = self.backend.heat_close(h)
                results[rid] = Result(rid, "heat", q.arrival, adm, self.clock() - t0, out,
                                      {"predicted_s": predict_seconds(q, self.kbars)})
                used -= device_bytes(q)
                worked = True
            for rid in [r for r, v in cg.items() if v[1].done()]:
                q, fut, adm = cg.pop(rid)
                out, info = fut.result()
                results[rid] = Result(rid, "cg", q.arrival, adm, self.clock() - t0, out, info)
                used -= device_bytes(q)
                worked = True
            if not worked:
                # idle: wait a little for the next arrival or a CG completion
                wait = 0.0005
                if i < len(pending) and not cg:
                    wait = min(max(pending[i].arrival - (self.clock() - t0), 0.0), 0.001)
                self.sleep(wait)
        self.makespan = self.clock() - t0
        return [results[r] for r in sorted(results)]


def summarize(results, requests, makespan: float) -> dict:
    """p50/p99 latency per kind and overall, heat GLUP/s over the makespan."""
    by = {"heat": [], "cg": []}
    for r in results:
        by[r.kind].append(r.latency)
    lups = sum(q.lups for q in requests if q.rid in {r.rid for r in results})
    out = {"requests": len(results), "makespan_s": makespan,
           "glups": lups / makespan / 1e9 if makespan > 0 else float("nan"),
           "latency_s": {"p50": percentile([r.latency for r in results], 50),
                         "p99": percentile([r.latency for r in results], 99)}}
    for k, v in by.items():
        out[f"latency_{k}_s"] = {"p50": percentile(v, 50), "p99": percentile(v, 99), "n": len(v)}
    return out


def poisson_trace(n: int, rate: float, seed: int, edge=(32, 384), steps=(10, 2000),
                  heat_frac: float = 0.75, f32_frac: float = 0.5, rtol: float = 1e-8):
    """Seeded requests: exponential inter-arrival times of mean 1/rate; heat
    with probability heat_frac; edges log-uniform per axis in `edge`; steps
    log-uniform in `steps`; FP32/FP64 by f32_frac; u0 ~ U[-1, 1]; b ~ N(0, 1).
    Payloads are windows, at seeded offsets, of two seeded pools (uniform and
    normal) a little longer than the largest request, so a trace of thousands
    of requests holds two pools instead of one array per request."""
    rng = np.random.default_rng([seed, 5])
    prng = np.random.default_rng([seed, 6])
    pool_n = edge[1] ** 3 + (1 << 22)
    upool = prng.uniform(-1.0, 1.0, size=pool_n)
    npool = prng.standard_normal(pool_n)

    def window(pool, shape):
        pts = int(np.prod(shape))
        off = int(rng.integers(0, pool_n - pts + 1))
        return pool[off:off + pts].reshape(shape)

    t = 0.0
    reqs = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        shape = tuple(int(v) for v in np.round(np.exp(rng.uniform(np.log(edge[0]), np.log(edge[1]), 3))))
        if rng.uniform() < heat_frac:
            st = int(round(math.exp(rng.uniform(math.log(steps[0]), math.log(steps[1])))))
            dt = "f32" if rng.uniform() < f32_frac else "f64"
            reqs.append(Request(rid, "heat", shape, dt, float(rng.uniform(0.05, 0.16)), st,
                                arrival=t, payload=window(upool, shape)))
        else:
            reqs.append(Request(rid, "cg", shape, "f64", rtol=rtol, arrival=t,
                                payload=window(npool, (int(np.prod(shape)),))))
    return reqs
