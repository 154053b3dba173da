"""Serving on the GPU: a mixed trace of heat (FP32/FP64) and CG requests
served with continuous batching; every result equals running that request
alone, bit for bit, and a sample of them matches the oracle."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import F64_REL, f32_bound, lib, rel_max_err, require_cuda

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    pkg = lib()
    torch = require_cuda()
    from paper_2608_11882_gb300.serve import GpuBackend, Server, poisson_trace, summarize
    reqs = poisson_trace(24, rate=400.0, seed=9, edge=(8, 40), steps=(5, 150), heat_frac=0.7)
    be = GpuBackend(workers=3)
    srv = Server(be, quantum=16, max_slots=8)
    res = srv.run(reqs)
    be.close()
    assert len(res) == len(reqs)
    stats = summarize(res, reqs, srv.makespan)
    assert stats["latency_s"]["p99"] >= stats["latency_s"]["p50"] > 0
    for q, r in zip(sorted(reqs, key=lambda q: q.rid), res):
        nz, ny, nx = q.shape
        if q.kind == "heat":
            with pkg.Heat(nx, ny, nz, q.r, dtype=q.dtype, tdepth=1) as h:
                alone = h.upload(q.payload.astype(h.np_dtype)).step(q.steps).read()
            assert np.array_equal(r.output, alone), q.rid
        else:
            with pkg.CG(pkg.Operator.stencil(nx, ny, nz)) as cg:
                x, info = cg.run(torch.from_numpy(q.payload).cuda(), rtol=q.rtol, max_iter=q.max_iter)
            assert np.array_equal(r.output, x.cpu().numpy()), q.rid
            assert r.info["converged"]
    # a sample of the mix against the oracle: FP64 heat to the 1e-12 gate, FP32
    # heat within its derived bound, CG to rtol with the iteration count of the
    # oracle's solve within 2
    oracle.build()
    byid = {r.rid: r for r in res}
    checked = {"f64": 0, "f32": 0, "cg": 0}
    for q in sorted(reqs, key=lambda q: q.rid):
        key = q.dtype if q.kind == "heat" else "cg"
        if checked[key] >= 3:
            continue
        checked[key] += 1
        out = byid[q.rid].output
        u0 = np.asarray(q.payload, dtype=np.float64)
        if q.kind == "heat" and q.dtype == "f64":
            assert rel_max_err(out, oracle.heat_run(u0, q.r, q.steps)) <= F64_REL, q.rid
        elif q.kind == "heat":
            ref = oracle.heat_run(u0.astype(np.float32).astype(np.float64), q.r, q.steps)
            assert np.max(np.abs(out - ref)) <= f32_bound(q.steps, np.max(np.abs(u0))), q.rid
        else:
            _, oinfo = oracle.cg_solve(u0, q.rtol, q.max_iter, shape=q.shape)
            assert abs(byid[q.rid].info["iters"] - oinfo["iters"]) <= 2, q.rid
            rr = u0 - oracle.lap7_apply(np.asarray(out).reshape(q.shape)).reshape(-1)
            assert np.linalg.norm(rr) <= 1.5 * q.rtol * np.linalg.norm(u0), q.rid
    assert min(checked.values()) >= 1
