"""The serving scheduler's logic on the CPU, with a fake backend: admission by
an injected free-HBM budget and by slots, quanta of heat steps, continuous
joining of late arrivals, percentiles."""
from concurrent.futures import Future

import numpy as np

from paper_2608_11882_gb300.serve import (Request, Server, device_bytes, percentile, poisson_trace,
                                          summarize)


class FakeBackend:
    def __init__(self, free=1 << 40):
        self.free = free
        self.advances = []      # (rids, steps) per heat batch
        self.open = set()

    def free_bytes(self):
        return self.free

    def heat_open(self, req):
        self.open.add(req.rid)
        return {"rid": req.rid, "done": 0}

    def heat_advance(self, handles, steps):
        for h, s in zip(handles, steps):
            h["done"] += s
        self.advances.append(([h["rid"] for h in handles], list(steps)))

    def heat_close(self, h):
        self.open.discard(h["rid"])
        return h["done"]

    def cg_submit(self, req):
        f = Future()
        f.set_result((np.zeros(req.points), {"iters": 1}))
        return f


def heat(rid, shape=(8, 8, 8), steps=100, arrival=0.0):
    return Request(rid, "heat", shape, "f64", 0.1, steps, arrival=arrival)


def test_every_request_gets_exactly_its_steps():
    be = FakeBackend()
    reqs = [heat(i, steps=s) for i, s in enumerate([1, 64, 65, 200, 0, 7])]
    res = Server(be, quantum=64).run(reqs)
    assert [r.output for r in res] == [1, 64, 65, 200, 0, 7]
    assert all(max(st) <= 64 for _, st in be.advances)
    assert not be.open


def test_admission_respects_budget_and_slots():
    be = FakeBackend()
    reqs = [heat(i, shape=(16, 16, 16), steps=50) for i in range(10)]
    one = device_bytes(reqs[0])
    srv = Server(be, hbm_budget=3 * one, max_slots=8, quantum=10)
    res = srv.run(reqs)
    assert len(res) == 10 and srv.peak_bytes <= 3 * one and srv.peak_slots <= 3
    srv = Server(FakeBackend(), hbm_budget=100 * one, max_slots=2, quantum=10)
    srv.run(reqs)
    assert srv.peak_slots <= 2


def test_requests_that_can_never_fit_are_rejected():
    be = FakeBackend()
    small, big = heat(0, (8, 8, 8)), heat(1, (64, 64, 64))
    srv = Server(be, hbm_budget=device_bytes(small) * 2, quantum=64)
    res = srv.run([small, big])
    assert [r.rid for r in res] == [0] and srv.rejected == [1]


def test_default_budget_comes_from_free_memory():
    srv = Server(FakeBackend(free=10 << 30), reserve=2 << 30)
    assert srv.budget == 8 << 30


def test_late_arrivals_join_running_batches():
    be = FakeBackend()
    reqs = [heat(0, steps=2000, arrival=0.0), heat(1, steps=100, arrival=0.01)]
    t = {"now": 0.0}

    def clock():
        return t["now"]

    def sleep(dt):
        t["now"] += max(dt, 1e-4)

    class Stepping(FakeBackend):
        def heat_advance(self, handles, steps):
            super().heat_advance(handles, steps)
            t["now"] += 0.005          # each batch takes 5 ms of "device time"

    be = Stepping()
    res = Server(be, quantum=64, clock=clock, sleep=sleep).run(reqs)
    assert [r.output for r in res] == [2000, 100]
    joint = [rids for rids, _ in be.advances if rids == [0, 1]]
    assert joint, "request 1 should have joined request 0's batches"
    assert res[1].completed < res[0].completed


def test_percentiles_and_summary():
    assert percentile([3, 1, 2, 4], 50) == 2
    assert percentile(list(range(1, 101)), 99) == 99
    reqs = poisson_trace(20, rate=100.0, seed=1, edge=(8, 16), steps=(5, 20))
    assert len(reqs) == 20 and all(b.arrival >= a.arrival for a, b in zip(reqs, reqs[1:]))
    res = Server(FakeBackend(), quantum=8).run(reqs)
    s = summarize(res, reqs, 1.0)
    assert s["requests"] == 20 and s["latency_s"]["p99"] >= s["latency_s"]["p50"]


class PipelinedBackend(FakeBackend):
    """A tick starts at heat_launch and its steps land only at heat_wait, as on
    the device; reading a handle that a running tick still advances is an error."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.running = None
        self.launches = 0

    def heat_launch(self, handles, steps):
        assert self.running is None, "one tick at a time"
        self.running = (handles, list(steps))
        self.launches += 1
        self.advances.append(([h["rid"] for h in handles], list(steps)))
        return self.launches

    def heat_wait(self, token):
        assert self.running is not None and token == self.launches
        for h, s in zip(*self.running):
            h["done"] += s
        self.running = None

    def heat_close(self, h):
        assert self.running is None or all(h is not x for x in self.running[0]), "read while in flight"
        return super().heat_close(h)


def test_pipelined_ticks_give_exact_steps_and_never_read_in_flight():
    be = PipelinedBackend()
    reqs = [heat(i, steps=s, arrival=0.0) for i, s in enumerate([1, 64, 65, 200, 0, 7, 130])]
    res = Server(be, quantum=64).run(reqs)
    assert [r.output for r in res] == [1, 64, 65, 200, 0, 7, 130]
    assert be.running is None and not be.open
    assert all(max(st) <= 64 for _, st in be.advances)


def test_pipelined_late_arrivals_join():
    t = {"now": 0.0}

    def clock():
        return t["now"]

    def sleep(dt):
        t["now"] += max(dt, 1e-4)

    class Timed(PipelinedBackend):
        def heat_wait(self, token):
            super().heat_wait(token)
            t["now"] += 0.005

    be = Timed()
    reqs = [heat(0, steps=2000, arrival=0.0), heat(1, steps=100, arrival=0.01)]
    res = Server(be, quantum=64, clock=clock, sleep=sleep).run(reqs)
    assert [r.output for r in res] == [2000, 100]
    assert any(rids == [0, 1] for rids, _ in be.advances)
    assert res[1].completed < res[0].completed


def test_kbar_follows_the_papers_model():
    """t_step = k (N-2)^3: timings generated from known k per size give back
    their mean; the prediction scales with points and steps."""
    from paper_2608_11882_gb300.serve import kbar, predict_seconds
    ks = {64: 2e-12, 128: 3e-12, 256: 4e-12}
    samples = [(n ** 3, 50, 50 * k * n ** 3) for n, k in ks.items()]
    assert abs(kbar(samples) - 3e-12) < 1e-24
    q = heat(0, shape=(10, 20, 30), steps=7)
    assert abs(predict_seconds(q, {"f64": 3e-12}) - 3e-12 * 6000 * 7) < 1e-20
    assert predict_seconds(q, {}) != predict_seconds(q, {})   # nan without a model


def test_results_carry_predictions():
    reqs = [heat(0, steps=10), heat(1, steps=0)]
    res = Server(FakeBackend(), quantum=8, kbars={"f64": 1e-12}).run(reqs)
    assert abs(res[0].info["predicted_s"] - 1e-12 * 512 * 10) < 1e-20
