// Conjugate gradients on the 7-point Dirichlet Laplacian (Section 7.5):
// SpMV fused with the p.q dot product, the x/r update fused with r.r, the
// p update, deterministic grid reductions, and the cg_* / op_apply entry
// points of the C ABI.
//
// CG in the textbook form (unpreconditioned, FP64; the matrix-free SpMV forms
// 6p - (neighbour sum) exactly in 64-bit fixed point on p's scale and rounds it
// once -- xsum.cuh -- while p's exponents allow, the FP64 pipe otherwise):
//     r0 = b - A x0, p0 = r0, rho0 = r0.r0
//     q = A p;  alpha = rho / p.q;  x += alpha p;  r -= alpha q;  rho' = r.r
//     stop when sqrt(rho') / ||b|| <= rtol, else p = r + (rho'/rho) p.
//
// Reductions: every block writes one partial sum; the last block to finish
// (a ticket counter) adds the partials in index order with a fixed tree, and
// updates the device scalars (alpha, beta, rho, the stop flag).  The grid size
// depends only on n, so results repeat bit for bit from run to run.  Kernels
// read the stop flag on entry and return at once after convergence, so the
// host can enqueue several iterations between convergence checks without the
// extra ones changing anything.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "cg_common.cuh"

namespace hcg {

// y = A p (no reduction).
template <int KIND>
__global__ void __launch_bounds__(kCgBlock)
    k_apply(OpDev A, const double* __restrict__ p, double* __restrict__ y)
{
    for (int64_t row = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; row < A.n;
         row += (int64_t)gridDim.x * kCgBlock)
        y[row] = apply_row<KIND>(A, p, row);
}

// r = b - q, p = r; rho = r.r, ||b||; decides whether x0 already meets rtol.
__global__ void __launch_bounds__(kCgBlock)
    k_cg_start(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
               double* __restrict__ r, double* __restrict__ p, double* partials, CgScalars* S,
               int track_pmax)
{
    __shared__ double sh[kCgBlock / 32];
    double rr = 0.0, bb = 0.0;
    unsigned pm = 0;
    for (int64_t t = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * kCgBlock) {
        const double bt = b[t];
        const double rt = bt - q[t];
        r[t] = rt;
        p[t] = rt;
        rr = __fma_rn(rt, rt, rr);
        bb = __fma_rn(bt, bt, bb);
        pm = max(pm, xs_abs_hi(rt));
    }
    const double rr_blk = block_sum<kCgBlock>(rr, sh);
    const double bb_blk = block_sum<kCgBlock>(bb, sh);
    if (track_pmax) cg_fold_pmax(pm, S, 0, blockIdx.x == 0);   // p0 = r0: iteration 0's direction
    // two partial arrays: [0, G) for r.r and [G, 2G) for b.b
    if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = bb_blk;
    if (!arrive_last(rr_blk, partials, &S->ticket)) return;
    const double rho = sum_partials(partials, gridDim.x, sh);
    const double bnorm2 = sum_partials(partials + gridDim.x, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->rho = rho;
        S->bnorm = sqrt(bnorm2);
        S->iters = 0;
        S->zero_rhs = (bnorm2 == 0.0);
        if (bnorm2 == 0.0) {
            S->relres = 0.0;
            S->done = 1;
        } else {
            S->relres = sqrt(rho) / S->bnorm;
            S->done = (S->relres <= S->rtol) ? 1 : 0;
        }
    }
}

// q = A p fused with p.q, one row per thread (MODE SP_ROWS or SP_CSR); the
// last block forms alpha = rho / p.q.
template <int MODE>
__global__ void __launch_bounds__(kCgBlock)
    k_cg_spmv_dot(OpDev A, const double* __restrict__ p, double* __restrict__ q, double* partials,
                  CgScalars* S)
{
    grid_dependency_wait();
    if (*(volatile int32_t*)&S->done) return;
    __shared__ double sh[kCgBlock / 32];
    double pq = 0.0;
    for (int64_t row = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; row < A.n;
         row += (int64_t)gridDim.x * kCgBlock) {
        const double qv = MODE == SP_CSR ? apply_csr_row(A, p, row) : apply_stencil_row(A, p, row);
        q[row] = qv;
        pq = __fma_rn(__ldg(p + row), qv, pq);
    }
    allow_dependents();
    const double blk = block_sum<kCgBlock>(pq, sh);
    if (!arrive_last(blk, partials, &S->ticket)) return;
    const double tot = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->pq = tot;
        if (!(tot > 0.0)) {
            S->done = 2;   // breakdown: A is not positive definite on p
        } else {
            S->alpha = S->rho / tot;
        }
    }
}

// The matrix-free SpMV staged by loads (SP_STAGED), fused with p.q: one block
// of kSpBlock threads per share (spmv_shares of the solve's block count).
__global__ void __launch_bounds__(kSpBlock, kSpMinBlocks)
    k_cg_spmv_staged(OpDev A, const double* __restrict__ p, double* __restrict__ q, double* partials,
                     CgScalars* S)
{
    grid_dependency_wait();
    if (*(volatile int32_t*)&S->done) return;
    __shared__ double sh[kSpBlock / 32];
    const double pq = spmv_stencil_share(A, p, q, cg_pemax(S), blockIdx.x, gridDim.x);
    allow_dependents();
    const double blk = block_sum<kSpBlock>(pq, sh);
    if (!arrive_last(blk, partials, &S->ticket)) return;
    const double tot = sum_partials_nt<kSpBlock>(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->pq = tot;
        if (!(tot > 0.0)) {
            S->done = 2;   // breakdown: A is not positive definite on p
        } else {
            S->alpha = S->rho / tot;
        }
    }
}

// x += alpha p, r -= alpha q fused with r.r; the last block tests convergence
// and forms beta.
__global__ void __launch_bounds__(kCgBlock)
    k_cg_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                const double* __restrict__ p, const double* __restrict__ q, double* partials,
                CgScalars* S)
{
    grid_dependency_wait();
    if (*(volatile int32_t*)&S->done) return;
    __shared__ double sh[kCgBlock / 32];
    const double alpha = S->alpha;
    const double rr = cg_update_rows(n, x, r, p, q, alpha, (int64_t)blockIdx.x * kCgBlock + threadIdx.x,
                                     (int64_t)gridDim.x * kCgBlock);
    allow_dependents();
    const double blk = block_sum<kCgBlock>(rr, sh);
    if (!arrive_last(blk, partials, &S->ticket)) return;
    const double rho_new = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->iters += 1;
        S->relres = sqrt(rho_new) / S->bnorm;
        if (S->relres <= S->rtol) {
            S->done = 1;
        } else {
            S->beta = rho_new / S->rho;
        }
        S->rho = rho_new;
    }
}

// p = r + beta p.
__global__ void __launch_bounds__(kCgBlock)
    k_cg_pupdate(int64_t n, const double* __restrict__ r, double* __restrict__ p, CgScalars* S,
                 int track_pmax)
{
    grid_dependency_wait();
    if (*(volatile int32_t*)&S->done) return;
    const double beta = S->beta;
    const unsigned pm = cg_pupdate_rows(n, r, p, beta, (int64_t)blockIdx.x * kCgBlock + threadIdx.x,
                                        (int64_t)gridDim.x * kCgBlock);
    allow_dependents();
    // the update kernel has counted this iteration: p is the next one's direction
    if (track_pmax) cg_fold_pmax(pm, S, S->iters % 3, blockIdx.x == 0);
}

// Largest |p| high word into S->pmax[0] (the direction's scale the
// matrix-free SpMV of iteration 0 reads), for cg_spmv.
__global__ void __launch_bounds__(kCgBlock)
    k_cg_pmax(int64_t n, const double* __restrict__ p, CgScalars* S)
{
    unsigned pm = 0;
    for (int64_t t = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * kCgBlock)
        pm = max(pm, xs_abs_hi(p[t]));
    cg_fold_pmax(pm, S, 0, false);
}

// ||b - q||^2 into S->rr_true (q = A x).
__global__ void __launch_bounds__(kCgBlock)
    k_resid_norm(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                 double* partials, CgScalars* S)
{
    __shared__ double sh[kCgBlock / 32];
    double rr = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * kCgBlock) {
        const double d = b[t] - q[t];
        rr = __fma_rn(d, d, rr);
    }
    const double blk = block_sum<kCgBlock>(rr, sh);
    if (!arrive_last(blk, partials, &S->ticket)) return;
    const double tot = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->rr_true = tot;
    }
}

}  // namespace hcg

using namespace hcg;

namespace hcg {

int check_op(const hs_op* A)
{
    if (!A) return fail(HS_EINVAL, "cg: operator is NULL");
    if (A->dtype != HS_F64) return fail(HS_EINVAL, "cg: operator dtype must be HS_F64");
    if (A->kind == HS_OP_STENCIL7) {
        if (A->nx < 1 || A->ny < 1 || A->nz < 1)
            return fail(HS_EINVAL, "cg: stencil grid %d x %d x %d invalid", A->nx, A->ny, A->nz);
        const int64_t n = (int64_t)A->nx * A->ny * A->nz;
        if (A->n != 0 && A->n != n) return fail(HS_EINVAL, "cg: n does not match nx*ny*nz");
        return HS_OK;
    }
    if (A->kind == HS_OP_CSR) {
        if (A->n < 1 || A->n >= ((int64_t)1 << 31)) return fail(HS_EINVAL, "cg: CSR n out of range");
        if (A->nnz < 0 || A->nnz >= ((int64_t)1 << 31))
            return fail(HS_EINVAL, "cg: CSR nnz out of range for int32 indices");
        if (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val)))
            return fail(HS_EINVAL, "cg: CSR arrays missing");
        return HS_OK;
    }
    return fail(HS_EINVAL, "cg: unknown operator kind %d", A->kind);
}

OpDev to_dev(const hs_op* A)
{
    OpDev d;
    d.kind = A->kind;
    d.nx = A->nx;
    d.ny = A->ny;
    d.nz = A->nz;
    d.n = A->kind == HS_OP_STENCIL7 ? (int64_t)A->nx * A->ny * A->nz : A->n;
    d.rowptr = A->rowptr;
    d.col = A->col;
    d.val = (const double*)A->val;
    return d;
}

int grid_for(int64_t n)
{
    int64_t g = (n + kCgBlock - 1) / kCgBlock;
    const int64_t cap = (int64_t)kNumSMs * 8;   // 8 blocks of 256 threads fill an SM
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

int launch_apply(const OpDev& A, const double* p, double* y, cudaStream_t s)
{
    const int g = grid_for(A.n);
    if (A.kind == HS_OP_STENCIL7)
        k_apply<HS_OP_STENCIL7><<<g, kCgBlock, 0, s>>>(A, p, y);
    else
        k_apply<HS_OP_CSR><<<g, kCgBlock, 0, s>>>(A, p, y);
    HS_CHECK_LAUNCH("cg: operator kernel");
    return HS_OK;
}

}  // namespace hcg

extern "C" {

int op_apply(const hs_op* A, const void* p, void* y, void* stream)
{
    int rc = check_op(A);
    if (rc != HS_OK) return rc;
    if (A->host) return fail(HS_EINVAL, "op_apply: operator arrays must be device memory");
    if (!p || !y) return fail(HS_EINVAL, "op_apply: NULL vector");
    return launch_apply(to_dev(A), (const double*)p, (double*)y, (cudaStream_t)stream);
}

int cg_spmv(const hs_op* A, const void* p, void* q, int kernel, double* pq, void* stream)
{
    int rc = check_op(A);
    if (rc != HS_OK) return rc;
    if (A->host) return fail(HS_EINVAL, "cg_spmv: operator arrays must be device memory");
    if (!p || !q) return fail(HS_EINVAL, "cg_spmv: NULL vector");
    if (p == q) return fail(HS_EINVAL, "cg_spmv: p and q must not overlap");
    const OpDev D = to_dev(A);
    const cudaStream_t s = (cudaStream_t)stream;
    const int grid = grid_for(D.n);   // the block count cg_run uses for this operator
    const bool stencil = D.kind == HS_OP_STENCIL7;
    int mode = 0;
    bool tma = false;
    switch (kernel) {
    case HS_SPMV_AUTO:
        mode = spmv_mode(D, grid);
        tma = mode == SP_STAGED && spmv_tma_eligible(D, (const double*)p, (const double*)q, grid);
        break;
    case HS_SPMV_ROWS:
        mode = stencil ? SP_ROWS : SP_CSR;
        break;
    case HS_SPMV_STAGED:
    case HS_SPMV_TMA:
        if (!stencil) return fail(HS_EINVAL, "cg_spmv: the staged kernels take the matrix-free operator only");
        mode = SP_STAGED;
        tma = kernel == HS_SPMV_TMA;
        if (tma && ((D.nx & 1) || ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15)))
            return fail(HS_EINVAL, "cg_spmv: the TMA-staged kernel needs an even nx and 16-byte aligned p and q");
        break;
    default:
        return fail(HS_EINVAL, "cg_spmv: unknown kernel %d", kernel);
    }
    CUtensorMap pmap;
    if (tma) {
        const int e = spmv_tma_map(&pmap, D, (const double*)p);
        if (e != 0) return cuda_fail((cudaError_t)e, "cg_spmv: TMA tensor map");
    }
    // scratch: the reduction partials and the device scalars of one iteration
    void* scratch = nullptr;
    const size_t pbytes = sizeof(double) * 2 * (size_t)grid;
    HS_TRY_CUDA(dev_alloc(&scratch, pbytes + sizeof(CgScalars), s), "cg_spmv: device allocation");
    double* partials = (double*)scratch;
    CgScalars* S = (CgScalars*)((char*)scratch + pbytes);
    CgScalars init;
    memset(&init, 0, sizeof(init));
    init.rho = 1.0;   // alpha = 1 / p.q: unused here
    cudaError_t e = cudaMemcpyAsync(S, &init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        // p's scale, exactly as the kernels that form p record it in a solve
        k_cg_pmax<<<grid, kCgBlock, 0, s>>>(D.n, (const double*)p, S);
        e = cudaPeekAtLastError();
        if (e == cudaSuccess) count_launch();
    }
    if (e == cudaSuccess) {
        if (tma) {
            rc = spmv_tma_launch(pmap, D, (double*)q, partials, S, spmv_shares(grid), s);
        } else {
            if (mode == SP_STAGED) {
                e = launch_dependent(k_cg_spmv_staged, spmv_shares(grid), kSpBlock, s, D, (const double*)p,
                                     (double*)q, partials, S);
            } else {
                auto kern = mode == SP_CSR ? k_cg_spmv_dot<SP_CSR> : k_cg_spmv_dot<SP_ROWS>;
                e = launch_dependent(kern, grid, kCgBlock, s, D, (const double*)p, (double*)q, partials, S);
            }
            rc = e == cudaSuccess ? HS_OK : cuda_fail(e, "cg_spmv: kernel launch");
            e = cudaSuccess;
        }
        if (rc == HS_OK) count_launch();
    }
    CgScalars out;
    memset(&out, 0, sizeof(out));
    if (e == cudaSuccess && rc == HS_OK) e = cudaMemcpyAsync(&out, S, sizeof(out), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && rc == HS_OK) e = cudaStreamSynchronize(s);
    dev_free(scratch, s);
    if (rc != HS_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cg_spmv");
    if (out.done == 3) return fail(HS_ETIMEOUT, "cg_spmv: a bounded wait in the TMA-staged SpMV ran out");
    if (out.done == 4)
        return fail(HS_ECUDA, "cg_spmv: a bounded wait in the TMA-staged SpMV ran out and its loads in "
                              "flight did not complete in time; treat the CUDA context as suspect");
    if (pq) *pq = out.pq;
    return HS_OK;
}

int cg_destroy(hs_cg_t c)
{
    if (!c) return HS_OK;
    int rc = HS_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cg_destroy: stream synchronize");
    dev_free(c->r, c->stream);
    dev_free(c->p, c->stream);
    dev_free(c->q, c->stream);
    dev_free(c->partials, c->stream);
    dev_free(c->S, c->stream);
    delete c->S_host;
    for (void* o : c->owned) dev_free(o, c->stream);
    if (c->mx) cg_mixed_release(c->mx, c->stream);
    dev_free(c->bx_dev[0], c->stream);
    dev_free(c->bx_dev[1], c->stream);
    delete c;
    return rc;
}

int cg_create(hs_cg_t* out, const hs_op* A, void* stream)
{
    if (!out) return fail(HS_EINVAL, "cg_create: out is NULL");
    *out = nullptr;
    int rc = check_op(A);
    if (rc != HS_OK) return rc;
    hs_cg* c = new (std::nothrow) hs_cg();
    if (!c) return fail(HS_ENOMEM, "cg_create: host allocation failed");
    c->stream = (cudaStream_t)stream;
    c->A = to_dev(A);
    const int64_t n = c->A.n;
    c->grid = grid_for(n);
#define CG_ALLOC(ptr, bytes)                                                 \
    do {                                                                     \
        cudaError_t e_ = dev_alloc((void**)&(ptr), (bytes), c->stream);     \
        if (e_ != cudaSuccess) {                                             \
            rc = cuda_fail(e_, "cg_create: device allocation");               \
            cg_destroy(c);                                                   \
            return rc;                                                       \
        }                                                                    \
    } while (0)
    CG_ALLOC(c->r, sizeof(double) * n);
    CG_ALLOC(c->p, sizeof(double) * n);
    CG_ALLOC(c->q, sizeof(double) * n);
    CG_ALLOC(c->partials, sizeof(double) * 2 * c->grid);
    CG_ALLOC(c->S, sizeof(CgScalars));
    // the host mirror of the scalars: ordinary memory (pinned memory would
    // cost a device-wide synchronisation to allocate and to free)
    c->S_host = new (std::nothrow) CgScalars();
    if (!c->S_host) {
        cg_destroy(c);
        return fail(HS_ENOMEM, "cg_create: host allocation failed");
    }
    if (A->kind == HS_OP_CSR && A->host) {
        const size_t bytes[3] = {sizeof(int32_t) * (size_t)(n + 1), sizeof(int32_t) * (size_t)A->nnz,
                                 sizeof(double) * (size_t)A->nnz};
        const void* src[3] = {A->rowptr, A->col, A->val};
        for (int t = 0; t < 3; ++t) {
            CG_ALLOC(c->owned[t], bytes[t] ? bytes[t] : 1);
            if (bytes[t]) {
                cudaError_t e = cudaMemcpyAsync(c->owned[t], src[t], bytes[t],
                                                cudaMemcpyHostToDevice, c->stream);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "cg_create: copy of CSR arrays");
                    cg_destroy(c);
                    return rc;
                }
            }
        }
        c->A.rowptr = (const int32_t*)c->owned[0];
        c->A.col = (const int32_t*)c->owned[1];
        c->A.val = (const double*)c->owned[2];
    }
#undef CG_ALLOC
    cudaError_t e = cudaMemsetAsync(c->S, 0, sizeof(CgScalars), c->stream);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "cg_create: memset");
        cg_destroy(c);
        return rc;
    }
    *out = c;
    return HS_OK;
}

int cg_run(hs_cg_t c, const void* b_in, void* x_inout, int host_buffers, double rtol,
           int32_t max_iter, hs_cg_info* info)
{
    if (!c || !b_in || !x_inout) return fail(HS_EINVAL, "cg_run: NULL argument");
    if (c->mx) return cg_run_mixed(c, b_in, x_inout, host_buffers, rtol, max_iter, info);
    if (!(rtol >= 0.0) || !std::isfinite(rtol)) return fail(HS_EINVAL, "cg_run: rtol must be finite and >= 0");
    if (max_iter < 0) return fail(HS_EINVAL, "cg_run: max_iter < 0");
    const int64_t n = c->A.n;
    const size_t vbytes = sizeof(double) * (size_t)n;
    const double* b = (const double*)b_in;
    double* x = (double*)x_inout;
    if (host_buffers) {
        for (int t = 0; t < 2; ++t)
            if (!c->bx_dev[t])
                HS_TRY_CUDA(dev_alloc((void**)&c->bx_dev[t], vbytes, c->stream), "cg_run: staging buffer");
        int rc_ = copy_host(c->bx_dev[0], b_in, vbytes, true, c->stream, "cg_run: copy of b");
        if (rc_ == HS_OK) rc_ = copy_host(c->bx_dev[1], x_inout, vbytes, true, c->stream, "cg_run: copy of x0");
        if (rc_ != HS_OK) return rc_;
        b = c->bx_dev[0];
        x = c->bx_dev[1];
    }
    // device scalars: rtol, cleared flags
    CgScalars init;
    memset(&init, 0, sizeof(init));
    init.rtol = rtol;
    *c->S_host = init;
    HS_TRY_CUDA(cudaMemcpyAsync(c->S, c->S_host, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream),
                "cg_run: scalar init");
    int rc = launch_apply(c->A, x, c->q, c->stream);   // q = A x0
    if (rc != HS_OK) return rc;
    const int mode = spmv_mode(c->A, c->grid);
    const int track = mode == SP_STAGED;   // the staged SpMV needs p's largest exponent
    const int shares = mode == SP_STAGED ? spmv_shares(c->grid) : c->grid;
    // the staged SpMV takes p through TMA when the grid and the vectors allow
    CUtensorMap pmap;
    const bool tma = mode == SP_STAGED && spmv_tma_eligible(c->A, c->p, c->q, c->grid) &&
                     spmv_tma_map(&pmap, c->A, c->p) == 0;
    k_cg_start<<<c->grid, kCgBlock, 0, c->stream>>>(n, b, c->q, c->r, c->p, c->partials, c->S, track);
    HS_CHECK_LAUNCH("cg: start kernel");

    // Iterate in chunks, reading the stop flag and count between chunks.
    int32_t enqueued = 0;
    int chunk = 4;
    for (;;) {
        HS_TRY_CUDA(cudaMemcpyAsync(c->S_host, c->S, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream),
                    "cg_run: scalar readback");
        HS_TRY_CUDA(cudaStreamSynchronize(c->stream), "cg_run: synchronize");
        if (c->S_host->done || enqueued >= max_iter) break;
        const int32_t todo = (max_iter - enqueued < chunk) ? max_iter - enqueued : chunk;
        for (int32_t t = 0; t < todo; ++t) {
            // x lives either in the caller's buffer or in the staging buffer
            const int64_t nn = n;
            switch (mode) {
            case SP_STAGED:
                if (tma) {
                    rc = spmv_tma_launch(pmap, c->A, c->q, c->partials, c->S, shares, c->stream);
                    if (rc != HS_OK) return rc;
                } else {
                    HS_TRY_CUDA(launch_dependent(k_cg_spmv_staged, shares, kSpBlock, c->stream, c->A,
                                           (const double*)c->p, c->q, c->partials, c->S), "cg: kernel launch");
                }
                break;
            case SP_ROWS:
                HS_TRY_CUDA(launch_dependent(k_cg_spmv_dot<SP_ROWS>, c->grid, kCgBlock, c->stream, c->A,
                                       (const double*)c->p, c->q, c->partials, c->S), "cg: kernel launch");
                break;
            default:
                HS_TRY_CUDA(launch_dependent(k_cg_spmv_dot<SP_CSR>, c->grid, kCgBlock, c->stream, c->A,
                                       (const double*)c->p, c->q, c->partials, c->S), "cg: kernel launch");
            }
            HS_CHECK_LAUNCH("cg: spmv+dot kernel");
            HS_TRY_CUDA(launch_dependent(k_cg_update, c->grid, kCgBlock, c->stream, nn, x, c->r, (const double*)c->p,
                                   (const double*)c->q, c->partials, c->S), "cg: kernel launch");
            HS_CHECK_LAUNCH("cg: update kernel");
            HS_TRY_CUDA(launch_dependent(k_cg_pupdate, c->grid, kCgBlock, c->stream, nn, (const double*)c->r, c->p,
                                   c->S, track), "cg: kernel launch");
            HS_CHECK_LAUNCH("cg: p update kernel");
        }
        enqueued += todo;
        if (chunk < 32) chunk *= 2;
    }
    const CgScalars s = *c->S_host;
    if (s.zero_rhs) HS_TRY_CUDA(cudaMemsetAsync(x, 0, vbytes, c->stream), "cg_run: zero solution");
    // true residual ||b - A x|| / ||b||
    rc = launch_apply(c->A, x, c->q, c->stream);
    if (rc != HS_OK) return rc;
    k_resid_norm<<<c->grid, kCgBlock, 0, c->stream>>>(n, b, c->q, c->partials, c->S);
    HS_CHECK_LAUNCH("cg: residual norm kernel");
    HS_TRY_CUDA(cudaMemcpyAsync(c->S_host, c->S, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream),
                "cg_run: scalar readback");
    if (host_buffers) {
        const int rc_ = copy_host(x_inout, x, vbytes, false, c->stream, "cg_run: copy of x");
        if (rc_ != HS_OK) return rc_;
    }
    HS_TRY_CUDA(cudaStreamSynchronize(c->stream), "cg_run: synchronize");
    const CgScalars f = *c->S_host;
    const bool converged = (f.done == 1);
    if (f.done == 2) return fail(HS_ECUDA, "cg_run: breakdown, p.q <= 0 (operator not positive definite?)");
    if (f.done == 3) return fail(HS_ETIMEOUT, "cg_run: a bounded wait in the TMA-staged SpMV ran out");
    if (f.done == 4)
        return fail(HS_ECUDA, "cg_run: a bounded wait in the TMA-staged SpMV ran out and its loads in "
                              "flight did not complete in time; treat the CUDA context as suspect");
    if (info) {
        info->iters = f.iters;
        info->relres_recur = f.relres;
        info->relres_true = f.zero_rhs ? 0.0 : sqrt(f.rr_true) / f.bnorm;
        info->status = converged ? HS_OK : HS_ENOCONV;
        info->refinements = 0;
        info->reserved = 0;
    }
    if (!converged) {
        set_error("cg_run: no convergence to rtol %g within %d iterations (relres %g)", rtol,
                  max_iter, f.relres);
        return HS_ENOCONV;
    }
    return HS_OK;
}

int cg_solve(const hs_op* A, const void* b, void* x, double rtol, int32_t max_iter,
             hs_cg_info* info, void* stream)
{
    if (A && A->host) return fail(HS_EINVAL, "cg_solve: operator arrays must be device memory");
    hs_cg_t c = nullptr;
    int rc = cg_create(&c, A, stream);
    if (rc != HS_OK) return rc;
    rc = cg_run(c, b, x, 0, rtol, max_iter, info);
    const int rc2 = cg_destroy(c);
    return rc != HS_OK ? rc : rc2;
}

}  // extern "C"

// ---- allocation-free CG ---------------------------------------------------------
// Some callers must not allocate while they solve: a serving loop that reserved
// all of its device memory up front and cannot let cudaMalloc/cudaFree (which
// may synchronise the whole device) stall the other streams it keeps busy;
// code that runs under another framework's memory manager or inside one of its
// allocation hooks, where a fresh allocation would fail, fragment the pool or
// re-enter the allocator; processes held to a fixed device-memory budget.
// cg_solve_noalloc serves them.  It runs exactly the kernels and host loop of
// cg_run, with the solver's scratch (r, p, q, the reduction partials and the
// device scalars) taken from one fixed array in the library's own device
// memory instead of from cudaMalloc, and its scalar read-backs going through a
// variable on the caller's stack instead of pinned memory.
namespace hcg {

constexpr int64_t kNoAllocMaxN = HS_NOALLOC_MAX_N;          // 2,097,152 unknowns = 128^3
constexpr int64_t kNoAllocMaxGrid = (int64_t)kNumSMs * 8;   // the largest grid grid_for() picks
constexpr size_t kNoAllocScalarDoubles = (sizeof(CgScalars) + sizeof(double) - 1) / sizeof(double);
constexpr size_t kNoAllocDoubles =
    3 * (size_t)kNoAllocMaxN + 2 * (size_t)kNoAllocMaxGrid + kNoAllocScalarDoubles;

// About 50 MB.  Every GPU that loads this library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch per device (host code may not use the
// symbol itself: on the host it names a stand-in, not device memory).  Looked
// up once per device and kept for the process: it is not refreshed after a
// cudaDeviceReset, which ends the context the address belongs to.
constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[kNoAllocMaxDevices];

}  // namespace hcg

extern "C" {

int cg_solve_noalloc(const hs_op* A, const void* b, void* x, double rtol, int32_t max_iter,
                     hs_cg_info* info, void* stream)
{
    int rc = check_op(A);
    if (rc != HS_OK) return rc;
    if (A->host) return fail(HS_EINVAL, "cg_solve_noalloc: operator arrays must be device memory");
    if (!b || !x) return fail(HS_EINVAL, "cg_solve_noalloc: NULL vector");
    hs_cg c{};
    c.A = to_dev(A);
    if (c.A.n > kNoAllocMaxN)
        return fail(HS_EINVAL, "cg_solve_noalloc: %lld unknowns exceed the fixed scratch of %lld",
                    (long long)c.A.n, (long long)kNoAllocMaxN);
    int dev = 0;
    HS_TRY_CUDA(cudaGetDevice(&dev), "cg_solve_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(HS_EINVAL, "cg_solve_noalloc: device ordinal %d out of range", dev);
    double* base = nullptr;
    {
        // Set-up, once per device, with that device current: look up where
        // the scratch array lives on it.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cg_solve_noalloc: cudaGetSymbolAddress");
            g_noalloc_addr[dev] = (double*)p;
        }
        base = g_noalloc_addr[dev];
    }
    c.stream = (cudaStream_t)stream;
    c.grid = grid_for(c.A.n);
    c.r = base;
    c.p = base + kNoAllocMaxN;
    c.q = base + 2 * kNoAllocMaxN;
    c.partials = base + 3 * kNoAllocMaxN;
    c.S = (CgScalars*)(c.partials + 2 * kNoAllocMaxGrid);
    // cg_run clears the device scalars (stop flag, iteration count and the
    // reduction ticket, which must start at zero) before the first kernel;
    // r, p and q are written before they are read.  The copies through this
    // pageable variable are synchronous and allocate nothing.
    CgScalars host_scalars;
    c.S_host = &host_scalars;
    return cg_run(&c, b, x, 0, rtol, max_iter, info);
}

}  // extern "C"
