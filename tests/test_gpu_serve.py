"""Serving on the GPU: a mixed trace of heat (FP32/FP64) and CG requests
served with continuous batching; every result equals running that request
alone, bit for bit."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import lib, require_cuda

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
