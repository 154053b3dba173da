// Definitions shared by the CG solvers: device scalars, the operator as the
// kernels see it, the context behind hs_cg_t, and host helpers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "xsum.cuh"

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
    int32_t done;      // 1: converged (or nothing to do); 2: breakdown (p.q <= 0);
                       // 3: a bounded wait of the TMA-staged SpMV ran out; 4: that,
                       // and the block's loads in flight did not complete in time
    int32_t iters;
    uint32_t ticket;   // blocks finished in the running reduction
    int32_t zero_rhs;  // ||b|| == 0
    // Largest |p| bit pattern of the direction p_i in slot i % 3 (matrix-free
    // operator): the kernel that forms p_i folds its values in and clears slot
    // (i+1) % 3; the SpMV of iteration i reads slot i % 3.
    unsigned long long pmax[3];
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

// Largest exponent field of the direction p of the current iteration, and
// whether the matrix-free SpMV may use the exact-sum form for it.
__device__ __forceinline__ int cg_pemax(const CgScalars* S)
{
    return (int)(__ldcg(&S->pmax[S->iters % 3]) >> 52);
}

__device__ __forceinline__ bool cg_xs_ok(int emax) { return emax >= kXsEmaxLo && emax <= kXsEmaxHi; }

// ---- matrix-free SpMV staged through shared memory ---------------------------------
// A block of kSpBlock = 128 threads (4 warps) owns a tile of 64 x 8 points of
// the grid and a chunk of z-planes, and marches up the chunk: every thread two
// consecutive x points in each of two adjacent rows, so its per-plane work
// (barrier, addresses, loop) is shared by four points and the y neighbours
// between its own rows come from its registers.  Each z-plane of the tile,
// with a one-point halo, is loaded once with coalesced loads (two planes
// ahead of its use), converted once to fixed point (exact-sum form) and
// written to one of two shared plane buffers; a thread keeps its own values
// at k-1, k and k+1 in registers, reads the other neighbours from the buffer
// of plane k, and one block barrier per plane orders the buffers.  Points
// outside the grid are staged as zeros (the Dirichlet boundary).  The work is
// cut into `nshares` equal shares of the (tile, plane) pairs in tile-major
// order -- share b is one run of consecutive planes of one tile, or two at a
// tile boundary -- where nshares is the number of TMA-staged blocks resident
// on the device at once (spmv_shares), so one wave of blocks moves the same
// bytes each and none waits for a second wave on part of the GPU.  Each
// thread adds its p.q products in a fixed order (run by run, plane by plane,
// row by row, x ascending) and the reduction sums the shares' partials in
// share order, so p.q repeats bit for bit wherever the same operator runs
// with the same share count (a batch uses its systems' own).
constexpr int kSpTW = 64, kSpTY = 8, kSpBW = 68, kSpD = 2;   // tile width/rows, buffer row, x offset
constexpr int kSpPlane = (kSpTY + 2) * kSpBW;                // buffer elements per plane
constexpr int kSpBlock = 128, kSpRT = 2;                     // threads of a staged block, rows per thread
constexpr int kSpMinBlocks = 5;   // load-staged blocks per SM (102 registers): measured fastest
static_assert(kSpTY == (kSpBlock / 32) * kSpRT, "four warps of two rows each cover the tile");

// Sum of partials[0..m) in a fixed order by a whole block of NT threads;
// valid in thread 0.
template <int NT>
__device__ __forceinline__ double sum_partials_nt(const double* partials, int m, double* sh)
{
    double v = 0.0;
    for (int t = threadIdx.x; t < m; t += NT) v += __ldcg(partials + t);
    return block_sum<NT>(v, sh);
}

struct SpmvPlan {
    int64_t tiles;
    int tiles_x;   // tiles per row of tiles
};

__host__ __device__ inline SpmvPlan spmv_plan(const OpDev& A)
{
    SpmvPlan P;
    P.tiles_x = (A.nx + kSpTW - 1) / kSpTW;
    P.tiles = (int64_t)P.tiles_x * ((A.ny + kSpTY - 1) / kSpTY);
    return P;
}

// Share b of nshares: the pairs [next, last) of the tile-major order, taken
// as runs of planes [kb, ke) of one tile each by spmv_next_run.
struct SpmvShare {
    int64_t next, last;
};

__device__ __forceinline__ SpmvShare spmv_share(const OpDev& A, const SpmvPlan& P, int b, int nshares)
{
    const int64_t pairs = P.tiles * A.nz;
    return SpmvShare{pairs * b / nshares, pairs * (b + 1) / nshares};
}

__device__ __forceinline__ void spmv_next_run(const OpDev& A, SpmvShare& sh, int64_t& tile, int& kb, int& ke)
{
    tile = sh.next / A.nz;
    kb = (int)(sh.next % A.nz);
    ke = sh.last - sh.next < (int64_t)(A.nz - kb) ? kb + (int)(sh.last - sh.next) : A.nz;
    sh.next += ke - kb;
}

// The share count of the staged SpMV for a system of nblocks blocks: the
// TMA-staged blocks resident on the device at once, at most nblocks (host).
int spmv_shares(int nblocks);

// q for one thread's 2 x 2 points of a plane from their values B (below), C
// (at), A (above), the row below the first row and above the last, and the x
// neighbours beyond the pairs: the exact-sum form (fixed-point values; one of
// the four converted back on the FP64 pipe, the others with integers, the same
// double either way) or the FP64 pipe on raw bits.
template <bool CONV>
__device__ __forceinline__ void spmv_points(const long long (&B)[2][2], const long long (&C)[2][2],
                                            const long long (&A)[2][2], const long long (&ym)[2],
                                            const long long (&yp)[2], const long long (&left)[2],
                                            const long long (&right)[2], int emax, double (&qv)[2][2])
{
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const long long xm = i == 0 ? left[j] : C[j][0];
            const long long xp = i == 1 ? right[j] : C[j][1];
            const long long yl = j == 0 ? ym[i] : C[0][i];
            const long long yh = j == 1 ? yp[i] : C[1][i];
            if constexpr (CONV) {
                const long long L = 6 * C[j][i] - (((B[j][i] + yl) + (xm + xp)) + (yh + A[j][i]));
                qv[j][i] = (j == 0 && i == 0) ? xs_unfix_dp(L, emax) : xs_unfix(L, emax);
            } else {
                auto d = [](long long b) { return __longlong_as_double(b); };
                const double sv = ((d(B[j][i]) + d(yl)) + (d(xm) + d(xp))) + (d(yh) + d(A[j][i]));
                qv[j][i] = __fma_rn(6.0, d(C[j][i]), -sv);
            }
        }
}

// One run: q = A p on the tile's planes [kb, ke), returning this
// thread's share of p.q.  CONV: the exact-sum form (emax = p's largest
// exponent field); otherwise FP64 arithmetic on raw values.
template <bool CONV>
__device__ __forceinline__ double spmv_item(const OpDev& A, const double* __restrict__ p,
                                            double* __restrict__ q, int emax, const SpmvPlan& P,
                                            int64_t tile, int kb, int ke, long long* buf)
{
    constexpr int V = 2, RT = kSpRT, BW = kSpBW;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int64_t sxy = (int64_t)nx * ny;
    const int x0 = (int)(tile % P.tiles_x) * kSpTW, y0 = (int)(tile / P.tiles_x) * kSpTY;
    const int X = x0 + V * tx, Y0 = y0 + RT * ty;
    const int own = (RT * ty + 1) * BW + kSpD + V * tx;   // row j: + j BW
    bool ok[RT][V], vec[RT];
    int64_t rowoff[RT];
#pragma unroll
    for (int j = 0; j < RT; ++j) {
        ok[j][0] = Y0 + j < ny && X < nx;
        ok[j][1] = Y0 + j < ny && X + 1 < nx;
        // a 16-byte pair: X is even, so the pair is aligned when nx is even and
        // both vectors start 16-byte aligned
        vec[j] = ok[j][1] && (nx & 1) == 0 &&
                 (((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15) == 0);
        rowoff[j] = (int64_t)(Y0 + j) * nx + X;
    }
    // halo: every thread one value of halo row 0 (threads 0..63) or 9 (64..127),
    // threads 0..15 also one value of the halo columns
    const int hc = tid % kSpTW;
    const int hidx = (tid < kSpTW ? 0 : kSpTY + 1) * BW + kSpD + hc;
    const int hy = tid < kSpTW ? y0 - 1 : y0 + kSpTY;
    const bool hok = x0 + hc < nx && hy >= 0 && hy < ny;
    const int64_t hoff = (int64_t)hy * nx + x0 + hc;
    int hidx2 = -1;
    bool hok2 = false;
    int64_t hoff2 = 0;
    if (tid < 2 * kSpTY) {
        const int rr = 1 + tid % kSpTY;
        const bool rgt = tid >= kSpTY;
        const int hx2 = rgt ? x0 + kSpTW : x0 - 1, hy2 = y0 + rr - 1;
        hidx2 = rr * BW + (rgt ? kSpD + kSpTW : kSpD - 1);
        hok2 = hx2 >= 0 && hx2 < nx && hy2 < ny;
        hoff2 = (int64_t)hy2 * nx + hx2;
    }
    const long long* pb = reinterpret_cast<const long long*>(p);
    auto ld_own = [&](int k, long long (&o)[RT][V]) {
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            o[j][0] = 0;
            o[j][1] = 0;
            if (k < 0 || k >= nz) continue;
            const long long* src = pb + (int64_t)k * sxy + rowoff[j];
            if (vec[j]) {
                const longlong2 v = __ldg(reinterpret_cast<const longlong2*>(src));
                o[j][0] = v.x;
                o[j][1] = v.y;
            } else {
                if (ok[j][0]) o[j][0] = __ldg(src);
                if (ok[j][1]) o[j][1] = __ldg(src + 1);
            }
        }
    };
    auto ld_halo = [&](int k, bool okh, int64_t off) -> long long {
        return (okh && k >= 0 && k < nz) ? __ldg(pb + (int64_t)k * sxy + off) : 0;
    };
    auto fix = [&](long long b) -> long long { return CONV ? xs_fix(b, emax) : b; };
    auto put = [&](long long* bp, const long long (&v)[RT][V], long long h, long long h2) {
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            bp[own + j * BW] = v[j][0];
            bp[own + j * BW + 1] = v[j][1];
        }
        bp[hidx] = fix(h);
        if (hidx2 >= 0) bp[hidx2] = fix(h2);
    };

    long long below[RT][V], cur[RT][V], above[RT][V], nown[RT][V], t[RT][V];
    double craw[RT][V], araw[RT][V];
    ld_own(kb - 1, t);
#pragma unroll
    for (int j = 0; j < RT; ++j)
#pragma unroll
        for (int i = 0; i < V; ++i) below[j][i] = fix(t[j][i]);
    ld_own(kb, t);
#pragma unroll
    for (int j = 0; j < RT; ++j)
#pragma unroll
        for (int i = 0; i < V; ++i) {
            craw[j][i] = __longlong_as_double(t[j][i]);
            cur[j][i] = fix(t[j][i]);
        }
    put(buf + (kb & 1) * kSpPlane, cur, ld_halo(kb, hok, hoff), ld_halo(kb, hok2, hoff2));
    ld_own(kb + 1, t);
#pragma unroll
    for (int j = 0; j < RT; ++j)
#pragma unroll
        for (int i = 0; i < V; ++i) {
            araw[j][i] = __longlong_as_double(t[j][i]);
            above[j][i] = fix(t[j][i]);
        }
    long long h1 = ld_halo(kb + 1, hok, hoff), h1b = ld_halo(kb + 1, hok2, hoff2), nh = 0, nhb = 0;
    ld_own(kb + 2 <= ke ? kb + 2 : nz, nown);   // plane nz reads as zeros
    if (kb + 2 <= ke) {
        nh = ld_halo(kb + 2, hok, hoff);
        nhb = ld_halo(kb + 2, hok2, hoff2);
    }
    __syncthreads();

    double pq = 0.0;
    for (int k = kb; k < ke; ++k) {
        put(buf + ((k + 1) & 1) * kSpPlane, above, h1, h1b);   // plane k+1: read in the next iteration
        const long long* pc = buf + (k & 1) * kSpPlane + own;
        const long long ym[V] = {pc[-BW], pc[1 - BW]}, yp[V] = {pc[RT * BW], pc[RT * BW + 1]};
        const long long left[RT] = {pc[-1], pc[BW - 1]}, right[RT] = {pc[V], pc[BW + V]};
        double qv[RT][V];
        spmv_points<CONV>(below, cur, above, ym, yp, left, right, emax, qv);
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            double* dst = q + (int64_t)k * sxy + rowoff[j];
            if (vec[j]) {
                *reinterpret_cast<double2*>(dst) = make_double2(qv[j][0], qv[j][1]);
            } else {
                if (ok[j][0]) dst[0] = qv[j][0];
                if (ok[j][1]) dst[1] = qv[j][1];
            }
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (ok[j][i]) pq = __fma_rn(craw[j][i], qv[j][i], pq);
        }
#pragma unroll
        for (int j = 0; j < RT; ++j)
#pragma unroll
            for (int i = 0; i < V; ++i) {
                below[j][i] = cur[j][i];
                cur[j][i] = above[j][i];
                craw[j][i] = araw[j][i];
                araw[j][i] = __longlong_as_double(nown[j][i]);
                above[j][i] = fix(nown[j][i]);
            }
        h1 = nh;
        h1b = nhb;
        if (k + 3 <= ke) {
            ld_own(k + 3, nown);
            nh = ld_halo(k + 3, hok, hoff);
            nhb = ld_halo(k + 3, hok2, hoff2);
        }
        __syncthreads();
    }
    return pq;
}

// The matrix-free SpMV of share b of nshares; returns the thread's p.q.
__device__ __forceinline__ double spmv_stencil_share(const OpDev& A, const double* __restrict__ p,
                                                     double* __restrict__ q, int emax, int b, int nshares)
{
    __shared__ __align__(16) long long buf[2 * kSpPlane];
    const SpmvPlan P = spmv_plan(A);
    double pq = 0.0;
    const bool conv = cg_xs_ok(emax);
    for (SpmvShare sh = spmv_share(A, P, b, nshares); sh.next < sh.last;) {
        int64_t tile;
        int kb, ke;
        spmv_next_run(A, sh, tile, kb, ke);
        pq += conv ? spmv_item<true>(A, p, q, emax, P, tile, kb, ke, buf)
                   : spmv_item<false>(A, p, q, emax, P, tile, kb, ke, buf);
    }
    return pq;
}

// SpMV kernels, chosen per operator on the host: the matrix-free operator is
// staged (exact-sum form) when a system of nblocks blocks has at least 4
// (tile, plane) pairs per block, and runs row by row on the FP64 pipe
// otherwise -- a rule of the operator and the block count only, so a batch
// and a single solve pick the same kernel.  Separate kernels keep the staged
// kernel's registers from lowering the others' occupancy.
enum SpmvMode { SP_ROWS = 0, SP_CSR = 1, SP_STAGED = 2 };

__host__ __device__ inline int spmv_mode(const OpDev& A, int nblocks)
{
    if (A.kind == HS_OP_CSR) return SP_CSR;
    const SpmvPlan P = spmv_plan(A);
    return P.tiles * (A.nz / 4) >= nblocks ? SP_STAGED : SP_ROWS;
}


// ---- the vector updates of a CG iteration, shared by single and batched CG -----------
// A system's rows are taken as pairs of consecutive values by threads t0,
// t0 + stride, ...; the odd last value by thread t0 == 0.  The solver's own
// vectors start 16-byte aligned and move as 16-byte vectors; the caller's x
// does too when it is aligned, value by value otherwise (same pairs, same
// order).  The per-value arithmetic is the textbook one; single and batched CG
// use these with the same partition, so their dot products add in the same
// order.

// x += alpha p, r -= alpha q; returns this thread's share of r.r.
__device__ __forceinline__ double cg_update_rows(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                 const double* __restrict__ p, const double* __restrict__ q,
                                                 double alpha, int64_t t0, int64_t stride)
{
    double rr = 0.0;
    const int64_t npairs = n >> 1;
    const bool xvec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    for (int64_t t = t0; t < npairs; t += stride) {
        const double2 pv = reinterpret_cast<const double2*>(p)[t];
        const double2 qv = reinterpret_cast<const double2*>(q)[t];
        double2 xv = xvec ? reinterpret_cast<double2*>(x)[t] : make_double2(x[2 * t], x[2 * t + 1]);
        double2 rv = reinterpret_cast<double2*>(r)[t];
        xv.x = __fma_rn(alpha, pv.x, xv.x);
        xv.y = __fma_rn(alpha, pv.y, xv.y);
        rv.x = __fma_rn(-alpha, qv.x, rv.x);
        rv.y = __fma_rn(-alpha, qv.y, rv.y);
        if (xvec) {
            reinterpret_cast<double2*>(x)[t] = xv;
        } else {
            x[2 * t] = xv.x;
            x[2 * t + 1] = xv.y;
        }
        reinterpret_cast<double2*>(r)[t] = rv;
        rr = __fma_rn(rv.x, rv.x, rr);
        rr = __fma_rn(rv.y, rv.y, rr);
    }
    if ((n & 1) && t0 == 0) {
        x[n - 1] = __fma_rn(alpha, p[n - 1], x[n - 1]);
        const double rt = __fma_rn(-alpha, q[n - 1], r[n - 1]);
        r[n - 1] = rt;
        rr = __fma_rn(rt, rt, rr);
    }
    return rr;
}

// p = r + beta p; returns the largest |p| high word of this thread's values.
__device__ __forceinline__ unsigned cg_pupdate_rows(int64_t n, const double* __restrict__ r,
                                                    double* __restrict__ p, double beta, int64_t t0,
                                                    int64_t stride)
{
    unsigned pm = 0;
    const int64_t npairs = n >> 1;
    for (int64_t t = t0; t < npairs; t += stride) {
        const double2 a = reinterpret_cast<const double2*>(p)[t];
        const double2 b = reinterpret_cast<const double2*>(r)[t];
        const double2 v = make_double2(__fma_rn(beta, a.x, b.x), __fma_rn(beta, a.y, b.y));
        reinterpret_cast<double2*>(p)[t] = v;
        pm = max(pm, max(xs_abs_hi(v.x), xs_abs_hi(v.y)));
    }
    if ((n & 1) && t0 == 0) {
        const double v = __fma_rn(beta, p[n - 1], r[n - 1]);
        p[n - 1] = v;
        pm = max(pm, xs_abs_hi(v));
    }
    return pm;
}

// Folds a block's largest |p| high word (m, per thread) into S->pmax[slot] and,
// from the system's first block, clears the slot after it.  All threads call it.
__device__ __forceinline__ void cg_fold_pmax(unsigned m, CgScalars* S, int slot, bool first_block)
{
    __shared__ unsigned wmax[kCgBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned b = 0;
        for (int w = 0; w < kCgBlock / 32; ++w) b = max(b, wmax[w]);
        atomicMax(&S->pmax[slot], (unsigned long long)b << 32);
        if (first_block) S->pmax[(slot + 1) % 3] = 0;
    }
}

struct CgMixed;   // mixed-precision state (cg_mixed.cu)

// The TMA-staged form of the SP_STAGED SpMV (cg_spmv_tma.cu) for single
// solves: eligible when nx is even and p, q are 16-byte aligned; the tensor
// map spans p (spmv_tma_map returns 0 on success).  spmv_tma_launch runs
// nshares blocks (spmv_shares of the system's block count) and leaves the
// launch check and count to its caller.
bool spmv_tma_eligible(const OpDev& A, const double* p, const double* q, int nblocks);
int spmv_tma_map(CUtensorMap* map, const OpDev& A, const double* p);
int spmv_tma_launch(const CUtensorMap& map, const OpDev& A, double* q, double* partials, CgScalars* S,
                    int nshares, cudaStream_t stream);

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
    hcg::CgScalars* S_host;  // host mirror of the scalars
    void* owned[3];        // device copies of host CSR arrays
    double* bx_dev[2];     // device staging of host b and x (allocated on demand)
    int64_t staged_n;
    hcg::CgMixed* mx;      // mixed-precision state (cg_create_mixed), else NULL
};

namespace hcg {
int cg_run_mixed(hs_cg* c, const void* b_in, void* x_inout, int host_buffers, double rtol,
                 int32_t max_iter, hs_cg_info* info);
void cg_mixed_release(CgMixed* m, cudaStream_t s);
}  // namespace hcg
