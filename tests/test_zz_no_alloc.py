"""cg_solve_noalloc: CG for callers that cannot allocate memory while they
solve (for example a serving loop that reserved its device memory up front,
or code under another framework's memory manager).  Its scratch lives in a
fixed array inside the library.  This file is collected last on purpose.

Checks, through the C ABI: two calls in a row (different systems and sizes,
so the second runs on what the first left in the shared scratch) give the
same result as cg_solve within the tolerances the other CG tests use; sizes
above the fixed maximum are rejected before any work."""
import numpy as np
import pytest

from tests.gpu_util import lib, require_cuda
from workloads import cg_rhs, lap7_csr

pytestmark = pytest.mark.gpu


def _solve(nat, op, b, rtol, fn):
    torch = require_cuda()
    x = torch.zeros(b.numel(), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, info = fn(op, b.data_ptr(), x.data_ptr(), rtol, 5000, stream)
    return rc, info, x.cpu().numpy()


def _kappa(nx, ny, nz):
    lo = 4 * sum(np.sin(np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    hi = 4 * sum(np.sin(m * np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    return hi / lo


def test_noalloc_matches_cg_solve_on_consecutive_calls():
    lib()
    torch = require_cuda()
    from paper_2608_11882_gb300 import _native as nat
    rtol = 1e-8
    cases = [("stencil", (40, 33, 29), 21), ("csr", (17, 26, 12), 22), ("stencil", (9, 8, 7), 23)]
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
        b = torch.from_numpy(cg_rhs(n, seed=seed)).cuda()
        rc_ref, info_ref, x_ref = _solve(nat, op, b, rtol, nat.cg_solve)
        rc, info, x = _solve(nat, op, b, rtol, nat.cg_solve_noalloc)
        assert rc == nat.HS_OK and rc_ref == nat.HS_OK
        assert abs(info.iters - info_ref.iters) <= 2
        assert info.relres_true <= 1.5 * rtol
        assert np.linalg.norm(x - x_ref) <= 2 * _kappa(nx, ny, nz) * rtol * np.linalg.norm(x_ref)


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
