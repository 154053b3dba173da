"""cg_solve_noalloc: CG for callers that cannot allocate memory while they
solve (for example a serving loop that reserved its device memory up front,
or code under another framework's memory manager).  Its scratch lives in a
fixed array inside the library.  This file is collected last on purpose.

Checks, through the C ABI: two or more calls in a row (different systems and
sizes, so each runs on what the one before left in the shared scratch) give
the same x, iteration count and residuals as cg_solve bit for bit -- the same
kernels on the same data -- one of them also against the oracle; a thin grid
with even nx (16 x 256 x 256, within the 128^3 limit) takes the staged SpMV
with p loaded by TMA from the fixed array; sizes above the fixed maximum are
rejected before any work."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import lib, require_cuda
from workloads import cg_rhs, lap7_csr

pytestmark = pytest.mark.gpu


def _solve(nat, op, b, rtol, fn):
    torch = require_cuda()
    x = torch.zeros(b.numel(), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, info = fn(op, b.data_ptr(), x.data_ptr(), rtol, 5000, stream)
    return rc, info, x.cpu().numpy()


def test_noalloc_matches_cg_solve_on_consecutive_calls():
    lib()
    oracle.build()
    torch = require_cuda()
    from paper_2608_11882_gb300 import _native as nat
    rtol = 1e-8
    cases = [("stencil", (40, 33, 29), 21), ("csr", (17, 26, 12), 22), ("stencil", (256, 256, 16), 24),
             ("stencil", (9, 8, 7), 23)]
    keep = []
    for kind, (nz, ny, nx), seed in cases:
        n = nx * ny * nz
        if kind == "stencil":
            op = nat.hs_op(kind=nat.HS_OP_STENCIL7, nx=nx, ny=ny, nz=nz, n=n, nnz=0, dtype=0, host=0)
        else:
            arrs = [torch.from_numpy(a).cuda() for a in lap7_csr(nx, ny, nz)]
            keep.append(arrs)
            op = nat.hs_op(kind=nat.HS_OP_CSR, n=n, nnz=arrs[1].numel(), rowptr=arrs[0].data_ptr(),
                           col=arrs[1].data_ptr(), val=arrs[2].data_ptr(), dtype=0, host=0)
        b_np = cg_rhs(n, seed=seed)
        b = torch.from_numpy(b_np).cuda()
        rc_ref, info_ref, x_ref = _solve(nat, op, b, rtol, nat.cg_solve)
        rc, info, x = _solve(nat, op, b, rtol, nat.cg_solve_noalloc)
        assert rc == nat.HS_OK and rc_ref == nat.HS_OK
        assert np.array_equal(x, x_ref)
        assert (info.iters, info.relres_recur, info.relres_true) == \
            (info_ref.iters, info_ref.relres_recur, info_ref.relres_true)
        if (nz, ny, nx) == (256, 256, 16):
            # against the oracle: iterations within 2, true residual by its operator
            _, oinfo = oracle.cg_solve(b_np, rtol, 5000, shape=(nz, ny, nx), threads=oracle.max_threads())
            assert abs(info.iters - oinfo["iters"]) <= 2
            r = b_np - oracle.lap7_apply(x.reshape(nz, ny, nx), threads=oracle.max_threads()).reshape(-1)
            assert np.linalg.norm(r) <= 1.5 * rtol * np.linalg.norm(b_np)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib()
    torch = require_cuda()
    from paper_2608_11882_gb300 import _native as nat
    nx, ny, nz = 129, 128, 128          # 2,113,536 > 2,097,152 unknowns
    op = nat.hs_op(kind=nat.HS_OP_STENCIL7, nx=nx, ny=ny, nz=nz, n=nx * ny * nz, nnz=0, dtype=0,
                   host=0)
    b = torch.ones(nx * ny * nz, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(nat.HeatCGError) as e:
        nat.cg_solve_noalloc(op, b.data_ptr(), x.data_ptr(), 1e-8, 10,
                             torch.cuda.current_stream().cuda_stream)
    assert e.value.code == nat.HS_EINVAL
    assert not x.any()
