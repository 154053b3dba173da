// Definitions shared by the CG solvers: device scalars, the operator as the
// kernels see it, the context behind hs_cg_t, and host helpers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace hcg {

struct CgScalars {
    double rho;        // r.r of the current residual
    double pq;         // p.q
    double alpha;
    double beta;
    double bnorm;      // ||b||
    double rtol;
    double relres;     // sqrt(rho)/||b|| at the last check
    double rr_true;    // ||b - A x||^2 at exit
    int32_t done;      // 1: converged (or nothing to do); 2: breakdown (p.q <= 0)
    int32_t iters;
    uint32_t ticket;   // blocks finished in the running reduction
    int32_t zero_rhs;  // ||b|| == 0
};

constexpr int kCgBlock = 256;

struct OpDev {
    int32_t kind;
    int32_t nx, ny, nz;
    int64_t n;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
};

// Writes this block's partial and returns true in every thread of the last
// block to finish, after which partials[0..gridDim.x) are all visible.
__device__ __forceinline__ bool arrive_last(double block_total, double* partials,
                                            uint32_t* ticket)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = block_total;
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Sum of partials[0..m) in a fixed order by the whole block; valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* partials, int m, double* sh)
{
    double v = 0.0;
    for (int t = threadIdx.x; t < m; t += kCgBlock) v += __ldcg(partials + t);
    return block_sum<kCgBlock>(v, sh);
}

// (A p)[row] for the matrix-free 7-point operator: 6 p - sum of the interior
// face neighbours; missing neighbours (outside the box) are Dirichlet zeros.
__device__ __forceinline__ double apply_stencil_row(const OpDev& A, const double* __restrict__ p,
                                                    int64_t row)
{
    const int nx = A.nx, ny = A.ny;
    const int64_t sxy = (int64_t)nx * ny;
    const int i = (int)(row % nx);
    const int64_t jk = row / nx;
    const int j = (int)(jk % ny);
    const int k = (int)(jk / ny);
    const double zm = k > 0 ? __ldg(p + row - sxy) : 0.0;
    const double ym = j > 0 ? __ldg(p + row - nx) : 0.0;
    const double xm = i > 0 ? __ldg(p + row - 1) : 0.0;
    const double xp = i < nx - 1 ? __ldg(p + row + 1) : 0.0;
    const double yp = j < ny - 1 ? __ldg(p + row + nx) : 0.0;
    const double zp = k < A.nz - 1 ? __ldg(p + row + sxy) : 0.0;
    const double s = ((zm + ym) + (xm + xp)) + (yp + zp);
    return __fma_rn(6.0, __ldg(p + row), -s);
}

// (A p)[row] for CSR: the row loop of Algorithm "spmv" (b), accumulated with FMA.
__device__ __forceinline__ double apply_csr_row(const OpDev& A, const double* __restrict__ p,
                                                int64_t row)
{
    double s = 0.0;
    const int e = __ldg(A.rowptr + row + 1);
    for (int t = __ldg(A.rowptr + row); t < e; ++t)
        s = __fma_rn(__ldg(A.val + t), __ldg(p + __ldg(A.col + t)), s);
    return s;
}

template <int KIND>
__device__ __forceinline__ double apply_row(const OpDev& A, const double* __restrict__ p,
                                            int64_t row)
{
    if (KIND == HS_OP_STENCIL7) return apply_stencil_row(A, p, row);
    return apply_csr_row(A, p, row);
}

struct CgMixed;   // mixed-precision state (cg_mixed.cu)

int check_op(const hs_op* A);
OpDev to_dev(const hs_op* A);
int grid_for(int64_t n);
int launch_apply(const OpDev& A, const double* p, double* y, cudaStream_t s);

}  // namespace hcg

struct hs_cg {
    hcg::OpDev A;
    cudaStream_t stream;
    int grid;
    double* r;
    double* p;
    double* q;
    double* partials;      // 2 * grid doubles
    hcg::CgScalars* S;     // device scalars
    hcg::CgScalars* S_host;  // pinned mirror
    void* owned[3];        // device copies of host CSR arrays
    double* bx_dev[2];     // device staging of host b and x (allocated on demand)
    int64_t staged_n;
    hcg::CgMixed* mx;      // mixed-precision state (cg_create_mixed), else NULL
};

namespace hcg {
int cg_run_mixed(hs_cg* c, const void* b_in, void* x_inout, int host_buffers, double rtol,
                 int32_t max_iter, hs_cg_info* info);
void cg_mixed_release(CgMixed* m);
}  // namespace hcg
