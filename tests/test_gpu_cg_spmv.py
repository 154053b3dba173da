"""Parity of the CG SpMV kernels (Section 7.5) against the oracle's operator,
element by element, through cg_spmv: one launch of the very kernel a CG
iteration runs (the block count and work order of cg_run), so these are the
kernels behind every matrix-free CG number the benchmark reports.

Error bounds (u = 2^-53, M = max|p|, exact = 6p - (sum of the six face
neighbours) in exact arithmetic):

* exact-sum kernels (staged by loads or by TMA): every value is converted to
  a 64-bit integer within two units of p 2^(1080-e), e the largest exponent
  field of p (one unit <= 2^-57 M), the stencil sum of the integers is exact,
  and the sum is rounded once to a double:
      |q - exact| <= 24 * 2^-57 * M + ulp(q) / 2;
* FP64-pipe arithmetic (the row kernel, and the staged kernels when p's
  exponents fall outside the convertible range): five additions of partial
  sums bounded by 2M, 2M, 4M, 2M, 6M, then fma(6, p, -s) with |q| <= 12M:
      |q - exact| <= (16 + 12) u M;
* the oracle adds the seven terms left to right (partial sums bounded by
  M, 2M, 3M, 9M, 10M, 11M, 12M) after rounding 6p:
      |q_oracle - exact| <= (47 + 6) u M,
  so against the oracle every kernel is within (53 + 28) u M.

The exact value comes from an error-free two-sum cascade (4p and 2p are exact
scalings), accurate to far below these bounds.  p.q is checked against the
exactly summed products within (depth + 1) u sum|p_i q_i|, depth bounding the
additions on any path of the kernel's fixed-order reduction.
"""
import math

import numpy as np
import pytest

import oracle
from tests.gpu_util import lib, require_cuda
from workloads import cg_rhs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def pkg():
    oracle.build()
    return lib()


def dev(a):
    torch = require_cuda()
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def exact_lap7(p):
    """6p - (face neighbours) as hi + lo, Dirichlet zeros outside the box."""
    nb = []
    for ax in range(3):
        lo = np.zeros_like(p)
        hi = np.zeros_like(p)
        sl_dst = [slice(None)] * 3
        sl_src = [slice(None)] * 3
        sl_dst[ax], sl_src[ax] = slice(1, None), slice(None, -1)
        lo[tuple(sl_dst)] = p[tuple(sl_src)]
        sl_dst[ax], sl_src[ax] = slice(None, -1), slice(1, None)
        hi[tuple(sl_dst)] = p[tuple(sl_src)]
        nb += [lo, hi]
    s = 4.0 * p
    e = np.zeros_like(p)
    for t in [2.0 * p] + [-v for v in nb]:
        s, err = two_sum(s, t)
        e += err
    return s, e


def gpu_spmv(pkg, shape, p, kernel):
    torch = require_cuda()
    nz, ny, nx = shape
    op = pkg.Operator.stencil(nx, ny, nz)
    q = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    pq = op.spmv(dev(p), q, kernel=kernel)
    torch.cuda.synchronize()
    return q.cpu().numpy().reshape(shape), pq


def check_against_exact_and_oracle(p, q, pq, conv, depth):
    M = float(np.max(np.abs(p)))
    hi, lo = exact_lap7(p)
    d = np.abs((q - hi) - lo)
    if conv:
        bound = 24 * 2.0 ** -57 * M + 0.5 * np.spacing(np.abs(q))
    else:
        bound = np.full_like(q, 28 * U * M)
    bound = bound + 2.0 ** -100 * M          # the two-sum value's own error
    worst = int(np.argmax(d - bound))
    assert np.all(d <= bound), (d.flat[worst], bound.flat[worst])
    q_or = oracle.lap7_apply(p, threads=oracle.max_threads())
    assert np.max(np.abs(q - q_or)) <= (53 + 28) * U * M
    if M * M * 12 > np.finfo(np.float64).max:
        return   # p.q itself overflows at this scale (on the device too); q is what is checked
    prod = (p * q).reshape(-1)
    ref = math.fsum(prod.tolist())
    assert abs(pq - ref) <= (depth + 1) * U * float(np.sum(np.abs(prod))) + 1e-300


def reduction_depth(shape):
    """Longest chain of additions in the fused p.q of any SpMV kernel: a
    thread's own accumulation (four points per plane of its block's share of
    the (tile, plane) pairs in the staged kernels, plus one addition per run of
    planes; its rows in the row kernel), the block's shuffle tree (8 levels), a
    thread's share of the partials, and the final tree.  The staged kernels
    split the pairs into as many shares as blocks of theirs are resident at
    once, at most cg_run's block count and at least one block per SM: the
    bound takes the fewest shares, so the longest chain."""
    nz, ny, nx = shape
    n = nx * ny * nz
    grid = max(1, min(-(-n // 256), 152 * 8))
    tiles = -(-nx // 64) * -(-ny // 8)
    share = -(-(tiles * nz) // min(grid, 152))
    chain = max(4 * share + -(-share // nz) + 1, -(-n // (grid * 256)))
    return chain + 8 + -(-grid // 128) + 8


SHAPES = [(176, 176, 176), (200, 101, 190), (160, 120, 177), (256, 256, 256)]


@pytest.mark.parametrize("shape", SHAPES)
def test_spmv_kernels_match_oracle_normal(pkg, shape):
    """p ~ N(0,1): the staged (loads), TMA-staged (even nx) and row kernels, and
    the one cg_run picks; the staged kernels agree bit for bit."""
    nz, ny, nx = shape
    p = np.random.default_rng(41).standard_normal(shape)
    kernels = ["staged", "rows"] + (["tma"] if nx % 2 == 0 else [])
    res = {}
    for k in kernels + ["auto"]:
        res[k] = gpu_spmv(pkg, shape, p, k)
    depth = reduction_depth(shape)
    for k in kernels:
        q, pq = res[k]
        check_against_exact_and_oracle(p, q, pq, conv=(k != "rows"), depth=depth)
    if "tma" in res:
        assert np.array_equal(res["tma"][0], res["staged"][0]) and res["tma"][1] == res["staged"][1]
    # every grid here is large enough that a solve stages p (TMA when nx is even)
    auto = "tma" if nx % 2 == 0 else "staged"
    assert np.array_equal(res["auto"][0], res[auto][0]) and res["auto"][1] == res[auto][1]


@pytest.mark.parametrize("shape", [(176, 176, 176), (160, 120, 177)])
def test_spmv_wide_dynamic_range(pkg, shape):
    """Magnitudes spread over 40 decades: values far below max|p| are quantised
    to units of 2^-57 max|p|, and the absolute bound still holds."""
    rng = np.random.default_rng(42)
    p = rng.standard_normal(shape) * 10.0 ** rng.uniform(-20, 20, size=shape)
    nx = shape[2]
    for k in ["staged"] + (["tma"] if nx % 2 == 0 else []):
        q, pq = gpu_spmv(pkg, shape, p, k)
        check_against_exact_and_oracle(p, q, pq, conv=True, depth=reduction_depth(shape))


@pytest.mark.parametrize("scale", [1e-300, 1e306])
@pytest.mark.parametrize("shape", [(176, 176, 176), (160, 120, 177)])
def test_spmv_fp64_fallback_out_of_range(pkg, shape, scale):
    """p's largest exponent outside the convertible range (tiny fields; values
    whose sums of twelve would come near overflow): the staged kernels take
    the FP64-pipe arithmetic and meet its bound."""
    p = np.random.default_rng(43).standard_normal(shape) * scale
    nx = shape[2]
    for k in ["staged"] + (["tma"] if nx % 2 == 0 else []):
        q, pq = gpu_spmv(pkg, shape, p, k)
        check_against_exact_and_oracle(p, q, pq, conv=False, depth=reduction_depth(shape))


@pytest.mark.parametrize("shape", [(9, 17, 33), (1, 1, 5), (3, 8, 64), (20, 18, 130)])
def test_staged_kernels_on_small_and_ragged_grids(pkg, shape):
    """The staged kernels on grids cg_run would give the row kernel: partial
    tiles in x and y, a single plane, a chunk shorter than the ring."""
    p = np.random.default_rng(44).standard_normal(shape)
    nx = shape[2]
    for k in ["staged", "rows"] + (["tma"] if nx % 2 == 0 else []):
        q, pq = gpu_spmv(pkg, shape, p, k)
        check_against_exact_and_oracle(p, q, pq, conv=(k != "rows"), depth=reduction_depth(shape))


def test_spmv_csr_rows_kernel_matches_oracle(pkg):
    torch = require_cuda()
    from workloads import lap7_csr
    nz, ny, nx = 40, 33, 29
    rowptr, col, val = lap7_csr(nx, ny, nz)
    op = pkg.Operator.csr(*[torch.from_numpy(a).cuda() for a in (rowptr, col, val)])
    p = np.random.default_rng(45).standard_normal(nx * ny * nz)
    q = torch.empty_like(dev(p))
    op.spmv(dev(p), q, kernel="rows")
    ref = oracle.csr_spmv(rowptr, col, val, p)
    # FMA row loop against the oracle's row loop: (7 + 7) roundings of partial
    # sums bounded by 12 max|p|
    assert np.max(np.abs(q.cpu().numpy() - ref)) <= 14 * 12 * U * np.max(np.abs(p))
    with pytest.raises(pkg.HeatCGError):
        op.spmv(dev(p), q, kernel="staged")


def test_spmv_argument_errors(pkg):
    torch = require_cuda()
    from paper_2608_11882_gb300._native import HS_EINVAL
    op = pkg.Operator.stencil(7, 4, 5)          # odd nx: no TMA map
    p = torch.zeros(140, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(p)
    with pytest.raises(pkg.HeatCGError) as e:
        op.spmv(p, q, kernel="tma")
    assert e.value.code == HS_EINVAL
    with pytest.raises(pkg.HeatCGError):
        op.spmv(p, p, kernel="staged")           # p and q overlap


@pytest.mark.parametrize("shape", [(176, 176, 176), (176, 176, 175)])
def test_cg_at_staged_sizes_matches_oracle(pkg, shape):
    """A whole solve at a size where cg_run stages p (by TMA for even nx, by
    loads for odd nx): iterations within 2 of the oracle's, the true residual
    (recomputed by the oracle's operator) within 1.5 rtol, and the solution
    within 2 kappa rtol of the oracle's."""
    nz, ny, nx = shape
    n = nx * ny * nz
    b = cg_rhs(n, seed=46)
    rtol = 1e-8
    x_ref, info_ref = oracle.cg_solve(b, rtol, 5000, shape=shape, threads=oracle.max_threads())
    with pkg.CG(pkg.Operator.stencil(nx, ny, nz)) as cg:
        x, info = cg.run(dev(b), rtol=rtol, max_iter=5000)
    x = x.cpu().numpy()
    assert info["converged"] and info_ref["status"] == 0
    assert abs(info["iters"] - info_ref["iters"]) <= 2
    r = b - oracle.lap7_apply(x.reshape(shape), threads=oracle.max_threads()).reshape(-1)
    assert np.linalg.norm(r) <= 1.5 * rtol * np.linalg.norm(b)
    lam_min = 4 * sum(np.sin(np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    lam_max = 4 * sum(np.sin(m * np.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    assert np.linalg.norm(x - x_ref) <= 2 * (lam_max / lam_min) * rtol * np.linalg.norm(x_ref)
