// Batched CG: many independent systems A_s x_s = b_s (7-point Laplacians of
// different grids, matrix-free or CSR) solved together, three kernel launches
// per iteration for the whole batch instead of three per system.
//
// Each system gets the same number of blocks and the same grid-stride row
// partition as its own cg_run would use, its own reduction partials, ticket
// and device scalars, so its iterates -- and results -- equal a solve of it
// alone bit for bit.  Systems that have converged (or hit max_iter) stop at
// the top of each kernel; the host reads all stop flags once per chunk of
// iterations.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "cg_common.cuh"

namespace hcg {

struct SysDev {
    OpDev A;
    const double* b;
    double* x;
    double* r;
    double* p;
    double* q;
    double* partials;   // 2 * nblocks
    CgScalars* S;
    int32_t block0;     // first block of this system in the batch grid
    int32_t nblocks;
    int32_t max_iter;
    int32_t mode;       // SpmvMode of the operator with this block count
    int32_t nshares;    // SP_STAGED: shares of the SpMV (spmv_shares(nblocks)), else nblocks
};

// System of this block (binary search over block0) and the block's index in it.
__device__ __forceinline__ int sys_of_block(const SysDev* sys, int nsys, int* local)
{
    int lo = 0, hi = nsys - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sys[mid].block0 <= b) lo = mid; else hi = mid - 1;
    }
    *local = b - sys[lo].block0;
    return lo;
}

// arrive_last for a block range: partial at [local], ticket of the system.
__device__ __forceinline__ bool arrive_last_sys(double total, double* partials, uint32_t* ticket,
                                                int local, int nblocks)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[local] = total;
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        last = (t == (uint32_t)nblocks - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ double sum_partials_n(const double* partials, int m, double* sh)
{
    double v = 0.0;
    for (int t = threadIdx.x; t < m; t += kCgBlock) v += __ldcg(partials + t);
    return block_sum<kCgBlock>(v, sh);
}

__device__ __forceinline__ double apply_sys(const OpDev& A, const double* __restrict__ p, int64_t row)
{
    return A.kind == HS_OP_STENCIL7 ? apply_stencil_row(A, p, row) : apply_csr_row(A, p, row);
}

// q = A x0 (start), then r = b - q, p = r, rho, ||b||.
__global__ void __launch_bounds__(kCgBlock) k_cgb_apply_x(const SysDev* sys, int nsys)
{
    int local;
    const SysDev& s = sys[sys_of_block(sys, nsys, &local)];
    for (int64_t row = (int64_t)local * kCgBlock + threadIdx.x; row < s.A.n;
         row += (int64_t)s.nblocks * kCgBlock)
        s.q[row] = apply_sys(s.A, s.x, row);
}

__global__ void __launch_bounds__(kCgBlock) k_cgb_start(const SysDev* sys, int nsys)
{
    int local;
    const SysDev& s = sys[sys_of_block(sys, nsys, &local)];
    __shared__ double sh[kCgBlock / 32];
    double rr = 0.0, bb = 0.0;
    unsigned pm = 0;
    for (int64_t t = (int64_t)local * kCgBlock + threadIdx.x; t < s.A.n;
         t += (int64_t)s.nblocks * kCgBlock) {
        const double bt = s.b[t];
        const double rt = bt - s.q[t];
        s.r[t] = rt;
        s.p[t] = rt;
        rr = __fma_rn(rt, rt, rr);
        bb = __fma_rn(bt, bt, bb);
        pm = max(pm, xs_abs_hi(rt));
    }
    const double rr_blk = block_sum<kCgBlock>(rr, sh);
    const double bb_blk = block_sum<kCgBlock>(bb, sh);
    if (s.mode == SP_STAGED) cg_fold_pmax(pm, s.S, 0, local == 0);
    if (threadIdx.x == 0) s.partials[s.nblocks + local] = bb_blk;
    if (!arrive_last_sys(rr_blk, s.partials, &s.S->ticket, local, s.nblocks)) return;
    const double rho = sum_partials_n(s.partials, s.nblocks, sh);
    const double bnorm2 = sum_partials_n(s.partials + s.nblocks, s.nblocks, sh);
    if (threadIdx.x == 0) {
        CgScalars* S = s.S;
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

// One kernel per SpmvMode, so each has its own register budget (and, for the
// staged mode, block size); blocks of the other modes' systems return at once.
template <int MODE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_cgb_spmv_dot(const SysDev* sys, int nsys)
{
    grid_dependency_wait();
    int local;
    const SysDev& s = sys[sys_of_block(sys, nsys, &local)];
    if (s.mode != MODE || *(volatile int32_t*)&s.S->done || s.S->iters >= s.max_iter) return;
    __shared__ double sh[NT / 32];
    double pq = 0.0;
    // as k_cg_spmv_dot / k_cg_spmv_staged: the same points per thread and the
    // same arithmetic, so the same results
    const int64_t row0 = (int64_t)local * NT + threadIdx.x;
    const int64_t stride = (int64_t)s.nblocks * NT;
    if (MODE == SP_STAGED) {
        // share `local` of a single solve's launch; the blocks beyond the shares add 0
        if (local < s.nshares) pq = spmv_stencil_share(s.A, s.p, s.q, cg_pemax(s.S), local, s.nshares);
    } else for (int64_t row = row0; row < s.A.n; row += stride) {
        const double qv = MODE == SP_CSR ? apply_csr_row(s.A, s.p, row) : apply_stencil_row(s.A, s.p, row);
        s.q[row] = qv;
        pq = __fma_rn(__ldg(s.p + row), qv, pq);
    }
    allow_dependents();
    const double blk = block_sum<NT>(pq, sh);
    if (!arrive_last_sys(blk, s.partials, &s.S->ticket, local, s.nblocks)) return;
    const double tot = sum_partials_nt<NT>(s.partials, s.nshares, sh);
    if (threadIdx.x == 0) {
        CgScalars* S = s.S;
        S->ticket = 0;
        S->pq = tot;
        if (!(tot > 0.0))
            S->done = 2;
        else
            S->alpha = S->rho / tot;
    }
}

__global__ void __launch_bounds__(kCgBlock) k_cgb_update(const SysDev* sys, int nsys)
{
    grid_dependency_wait();
    int local;
    const SysDev& s = sys[sys_of_block(sys, nsys, &local)];
    if (*(volatile int32_t*)&s.S->done || s.S->iters >= s.max_iter) return;
    __shared__ double sh[kCgBlock / 32];
    const double alpha = s.S->alpha;
    const double rr = cg_update_rows(s.A.n, s.x, s.r, s.p, s.q, alpha, (int64_t)local * kCgBlock + threadIdx.x,
                                     (int64_t)s.nblocks * kCgBlock);
    allow_dependents();
    const double blk = block_sum<kCgBlock>(rr, sh);
    if (!arrive_last_sys(blk, s.partials, &s.S->ticket, local, s.nblocks)) return;
    const double rho_new = sum_partials_n(s.partials, s.nblocks, sh);
    if (threadIdx.x == 0) {
        CgScalars* S = s.S;
        S->ticket = 0;
        S->iters += 1;
        S->relres = sqrt(rho_new) / S->bnorm;
        if (S->relres <= S->rtol)
            S->done = 1;
        else
            S->beta = rho_new / S->rho;
        S->rho = rho_new;
    }
}

__global__ void __launch_bounds__(kCgBlock) k_cgb_pupdate(const SysDev* sys, int nsys)
{
    grid_dependency_wait();
    int local;
    const SysDev& s = sys[sys_of_block(sys, nsys, &local)];
    // the update kernel of this iteration has already counted it
    if (*(volatile int32_t*)&s.S->done) return;
    const double beta = s.S->beta;
    const unsigned pm = cg_pupdate_rows(s.A.n, s.r, s.p, beta, (int64_t)local * kCgBlock + threadIdx.x,
                                        (int64_t)s.nblocks * kCgBlock);
    allow_dependents();
    if (s.mode == SP_STAGED) cg_fold_pmax(pm, s.S, s.S->iters % 3, local == 0);
}

// ||b - A x||^2 into rr_true (q = A x from k_cgb_apply_x).
__global__ void __launch_bounds__(kCgBlock) k_cgb_resid(const SysDev* sys, int nsys)
{
    int local;
    const SysDev& s = sys[sys_of_block(sys, nsys, &local)];
    __shared__ double sh[kCgBlock / 32];
    double rr = 0.0;
    for (int64_t t = (int64_t)local * kCgBlock + threadIdx.x; t < s.A.n;
         t += (int64_t)s.nblocks * kCgBlock) {
        const double d = s.b[t] - s.q[t];
        rr = __fma_rn(d, d, rr);
    }
    const double blk = block_sum<kCgBlock>(rr, sh);
    if (!arrive_last_sys(blk, s.partials, &s.S->ticket, local, s.nblocks)) return;
    const double tot = sum_partials_n(s.partials, s.nblocks, sh);
    if (threadIdx.x == 0) {
        s.S->ticket = 0;
        s.S->rr_true = tot;
    }
}

}  // namespace hcg

using namespace hcg;

struct hs_cg_batch {
    cudaStream_t stream;
    int32_t n;
    int32_t total_blocks;
    bool has_mode[3];          // SpmvModes present (one SpMV kernel each)
    std::vector<SysDev> sys;   // host copy (b, x filled per run)
    std::vector<int64_t> rows;
    SysDev* d_sys;
    void* arena;               // r, p, q, partials, scalars of all systems
    CgScalars* d_S;
    CgScalars* h_S;            // host mirror of the scalars, n entries
};

extern "C" {

int cg_batch_destroy(hs_cg_batch_t b)
{
    if (!b) return HS_OK;
    int rc = HS_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cg_batch_destroy: synchronize");
    dev_free(b->d_sys, b->stream);
    dev_free(b->arena, b->stream);
    delete[] b->h_S;
    delete b;
    return rc;
}

int cg_batch_create(hs_cg_batch_t* out, const hs_op* ops, int32_t n, void* stream)
{
    if (!out) return fail(HS_EINVAL, "cg_batch_create: out is NULL");
    *out = nullptr;
    if (!ops || n < 1) return fail(HS_EINVAL, "cg_batch_create: no systems");
    for (int32_t i = 0; i < n; ++i) {
        const int rc = check_op(&ops[i]);
        if (rc != HS_OK) return rc;
        if (ops[i].host) return fail(HS_EINVAL, "cg_batch_create: operator %d must be device memory", i);
    }
    hs_cg_batch* b = new (std::nothrow) hs_cg_batch();
    if (!b) return fail(HS_ENOMEM, "cg_batch_create: host allocation failed");
    b->stream = (cudaStream_t)stream;
    b->n = n;
    b->sys.resize((size_t)n);
    b->rows.resize((size_t)n);
    int64_t vec_total = 0, part_total = 0;
    int64_t blocks = 0;
    for (int32_t i = 0; i < n; ++i) {
        SysDev& s = b->sys[(size_t)i];
        memset(&s, 0, sizeof(s));
        s.A = to_dev(&ops[i]);
        s.nblocks = grid_for(s.A.n);
        s.mode = spmv_mode(s.A, s.nblocks);
        s.nshares = s.mode == SP_STAGED ? spmv_shares(s.nblocks) : s.nblocks;
        b->has_mode[s.mode] = true;
        s.block0 = (int32_t)blocks;
        blocks += s.nblocks;
        b->rows[(size_t)i] = s.A.n;
        vec_total += (s.A.n + 1) & ~(int64_t)1;   // every vector starts 16-byte aligned
        part_total += 2 * (int64_t)s.nblocks;
    }
    if (blocks > INT32_MAX) {
        delete b;
        return fail(HS_EINVAL, "cg_batch_create: batch too large");
    }
    b->total_blocks = (int32_t)blocks;
    const size_t bytes = sizeof(double) * (size_t)(3 * vec_total + part_total) + sizeof(CgScalars) * (size_t)n;
    cudaError_t e = dev_alloc(&b->arena, bytes, b->stream);
    if (e == cudaSuccess) e = dev_alloc((void**)&b->d_sys, sizeof(SysDev) * (size_t)n, b->stream);
    if (e == cudaSuccess) {
        b->h_S = new (std::nothrow) CgScalars[(size_t)n]();
        if (!b->h_S) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "cg_batch_create: allocation");
        cg_batch_destroy(b);
        return rc;
    }
    double* base = (double*)b->arena;
    double* part = base + 3 * vec_total;
    b->d_S = (CgScalars*)(part + part_total);
    int64_t off = 0, poff = 0;
    for (int32_t i = 0; i < n; ++i) {
        SysDev& s = b->sys[(size_t)i];
        s.r = base + off;
        s.p = base + vec_total + off;
        s.q = base + 2 * vec_total + off;
        s.partials = part + poff;
        s.S = b->d_S + i;
        off += (s.A.n + 1) & ~(int64_t)1;
        poff += 2 * (int64_t)s.nblocks;
    }
    *out = b;
    return HS_OK;
}

int cg_batch_run(hs_cg_batch_t b, const void* const* bs, void* const* xs, double rtol, int32_t max_iter,
                 hs_cg_info* infos)
{
    if (!b || !bs || !xs) return fail(HS_EINVAL, "cg_batch_run: NULL argument");
    if (!(rtol >= 0.0) || !std::isfinite(rtol)) return fail(HS_EINVAL, "cg_batch_run: bad rtol");
    if (max_iter < 0) return fail(HS_EINVAL, "cg_batch_run: max_iter < 0");
    const int n = b->n;
    for (int i = 0; i < n; ++i) {
        if (!bs[i] || !xs[i]) return fail(HS_EINVAL, "cg_batch_run: NULL vector of system %d", i);
        b->sys[(size_t)i].b = (const double*)bs[i];
        b->sys[(size_t)i].x = (double*)xs[i];
        b->sys[(size_t)i].max_iter = max_iter;
    }
    HS_TRY_CUDA(cudaMemcpyAsync(b->d_sys, b->sys.data(), sizeof(SysDev) * (size_t)n, cudaMemcpyHostToDevice,
                                b->stream),
                "cg_batch_run: system table");
    for (int i = 0; i < n; ++i) {
        memset(&b->h_S[i], 0, sizeof(CgScalars));
        b->h_S[i].rtol = rtol;
    }
    HS_TRY_CUDA(cudaMemcpyAsync(b->d_S, b->h_S, sizeof(CgScalars) * (size_t)n, cudaMemcpyHostToDevice,
                                b->stream),
                "cg_batch_run: scalars");
    const int G = b->total_blocks;
#define CGB_LAUNCH(kern, what)                                                 \
    do {                                                                       \
        kern<<<G, kCgBlock, 0, b->stream>>>(b->d_sys, n);                      \
        HS_CHECK_LAUNCH(what);                                                 \
    } while (0)
    // the iteration kernels launch as dependent launches: each waits on entry
    // for the kernel before it, and its launch overlaps that kernel's tail
#define CGB_LAUNCH_DEP(kern, what)                                                             \
    do {                                                                                       \
        HS_TRY_CUDA(launch_dependent(kern, G, kCgBlock, b->stream, b->d_sys, n), "cg batch: kernel launch"); \
        HS_CHECK_LAUNCH(what);                                                                 \
    } while (0)
    CGB_LAUNCH(k_cgb_apply_x, "cg batch: A x0 kernel");
    CGB_LAUNCH(k_cgb_start, "cg batch: start kernel");
    int32_t enqueued = 0;
    int chunk = 4;
    for (;;) {
        HS_TRY_CUDA(cudaMemcpyAsync(b->h_S, b->d_S, sizeof(CgScalars) * (size_t)n, cudaMemcpyDeviceToHost,
                                    b->stream),
                    "cg_batch_run: scalar readback");
        HS_TRY_CUDA(cudaStreamSynchronize(b->stream), "cg_batch_run: synchronize");
        bool all = true;
        for (int i = 0; i < n; ++i)
            if (!b->h_S[i].done && b->h_S[i].iters < max_iter) all = false;
        if (all || enqueued >= max_iter) break;
        const int32_t todo = (max_iter - enqueued < chunk) ? max_iter - enqueued : chunk;
        for (int32_t t = 0; t < todo; ++t) {
            if (b->has_mode[SP_STAGED]) {
                HS_TRY_CUDA(launch_dependent(k_cgb_spmv_dot<SP_STAGED, kSpBlock, kSpMinBlocks>, G, kSpBlock, b->stream, b->d_sys,
                                             n),
                            "cg batch: kernel launch");
                HS_CHECK_LAUNCH("cg batch: spmv+dot kernel");
            }
            if (b->has_mode[SP_ROWS]) CGB_LAUNCH_DEP((k_cgb_spmv_dot<SP_ROWS, kCgBlock, 1>), "cg batch: spmv+dot kernel");
            if (b->has_mode[SP_CSR]) CGB_LAUNCH_DEP((k_cgb_spmv_dot<SP_CSR, kCgBlock, 1>), "cg batch: spmv+dot kernel");
            CGB_LAUNCH_DEP(k_cgb_update, "cg batch: update kernel");
            CGB_LAUNCH_DEP(k_cgb_pupdate, "cg batch: p update kernel");
        }
        enqueued += todo;
        if (chunk < 32) chunk *= 2;
    }
    // zero right-hand sides have the solution 0
    for (int i = 0; i < n; ++i)
        if (b->h_S[i].zero_rhs)
            HS_TRY_CUDA(cudaMemsetAsync(xs[i], 0, sizeof(double) * (size_t)b->rows[(size_t)i], b->stream),
                        "cg_batch_run: zero solution");
    CGB_LAUNCH(k_cgb_apply_x, "cg batch: A x kernel");
    CGB_LAUNCH(k_cgb_resid, "cg batch: residual kernel");
#undef CGB_LAUNCH
#undef CGB_LAUNCH_DEP
    HS_TRY_CUDA(cudaMemcpyAsync(b->h_S, b->d_S, sizeof(CgScalars) * (size_t)n, cudaMemcpyDeviceToHost,
                                b->stream),
                "cg_batch_run: scalar readback");
    HS_TRY_CUDA(cudaStreamSynchronize(b->stream), "cg_batch_run: synchronize");
    int rc = HS_OK;
    for (int i = 0; i < n; ++i) {
        const CgScalars& f = b->h_S[i];
        if (f.done == 2) return fail(HS_ECUDA, "cg_batch_run: breakdown in system %d", i);
        const bool conv = (f.done == 1);
        if (!conv) rc = HS_ENOCONV;
        if (infos) {
            infos[i].iters = f.iters;
            infos[i].status = conv ? HS_OK : HS_ENOCONV;
            infos[i].relres_recur = f.relres;
            infos[i].relres_true = f.zero_rhs ? 0.0 : sqrt(f.rr_true) / f.bnorm;
            infos[i].refinements = 0;
            infos[i].reserved = 0;
        }
    }
    if (rc == HS_ENOCONV) set_error("cg_batch_run: some systems did not reach rtol %g in %d iterations", rtol,
                                    max_iter);
    return rc;
}

}  // extern "C"
