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
