// Matrix-free CG SpMV fused with p.q, with the planes of p staged in shared
// memory by TMA (Section 7.5; the operator of Eq. 4 without the time step:
// q = 6p - sum of the six face neighbours, Dirichlet zeros outside the box).
//
// The same work as the staged kernel of cg_common.cuh, in the same order and
// with the same arithmetic: a block of 128 threads owns a 64 x 8 tile for a
// run of z-planes at a time, every thread two consecutive x points in each of
// two adjacent rows, block b taking share b of the (tile, plane) pairs as
// spmv_share and spmv_next_run give them.  The grid is one resident wave: spmv_shares()
// blocks (760 at five per SM), every block the same bytes to within a plane
// (fixed 26-plane items for 1216 blocks left a second wave on part of the
// GPU: 71.4 us at 256^3).  q and every thread's share of p.q therefore come
// out bit for bit as in the staged kernel, so a single solve (this kernel)
// and a batched solve (the staged kernel) still agree.
//
// What differs is how p arrives: each plane of the tile with its one-point
// halo is one 3-D tiled TMA box, (8 + 2) rows of 68 doubles starting 16 bytes
// left of the tile, loaded into a ring of kSpNst = 4 stages up to 2 planes
// ahead of use (five blocks of 128 threads per SM, 94 registers: 3730 CG
// iterations/s at 256^3 against 3659 with six blocks, whose 80 registers
// spill, and fewer with eight blocks at 64 registers).  The tensor map spans the unpadded nx x ny x nz vector,
// so boxes that reach past the box of the grid (the planes -1 and nz, the rows
// -1 and ny, the columns -1 and nx) read zeros: the Dirichlet boundary with no
// bounds checks.  The box starts at x0 - 2 with x0 a multiple of 64, so its x
// coordinate times 8 bytes is a multiple of 16 as TMA requires; the map needs
// nx even (16-byte row stride) and p 16-byte aligned, which the host checks.
// Every thread converts its own four values of each new plane to fixed point in
// place (and warps 0-2 the halo), so each staged value is converted once.
//
// Each mbarrier wait is bounded (about a second); one that runs out marks the
// solve with done = 3 (HS_ETIMEOUT on the host), waits (bounded) for the
// block's loads in flight and ends the block.  If that wait runs out as well,
// loads may still land in shared memory a later block reuses: done = 4, which
// the host reports as HS_ECUDA with the context to be treated as suspect.
#include <cuda.h>

#include "cg_common.cuh"
#include "tma.cuh"

namespace hcg {

constexpr int kSpNst = 4;
constexpr uint32_t kSpBoxBytes = (uint32_t)kSpPlane * sizeof(double);     // 10 x 68 doubles
constexpr int kSpStage = (int)((kSpBoxBytes + 127) / 128 * 128 / sizeof(double));
static_assert(kSpBW * sizeof(double) % 16 == 0, "TMA box rows are a 16-byte multiple");
static_assert(kSpD * sizeof(double) == 16, "the box starts 16 bytes left of the tile");

template <bool CONV>
__device__ __forceinline__ double spmv_item_tma(const CUtensorMap* map, const OpDev& A,
                                                double* __restrict__ q, int emax, const SpmvPlan& P,
                                                int64_t tile, int kb, int ke, long long* stage,
                                                uint64_t* bars, uint32_t& seq, bool& aborted,
                                                bool& drained)
{
    constexpr int V = 2, RT = kSpRT, BW = kSpBW, NST = kSpNst;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int nx = A.nx, ny = A.ny;
    const int64_t sxy = (int64_t)nx * ny;
    const int x0 = (int)(tile % P.tiles_x) * kSpTW, y0 = (int)(tile / P.tiles_x) * kSpTY;
    const int X = x0 + V * tx, Y0 = y0 + RT * ty;
    const int own = (RT * ty + 1) * BW + kSpD + V * tx;   // row j: + j BW
    // nx is even and X is even: both points of a pair are inside or both outside
    bool ok[RT];
#pragma unroll
    for (int j = 0; j < RT; ++j) ok[j] = Y0 + j < ny && X < nx;
    // the values this thread converts besides its own: a pair of halo row 0
    // (warp 0) or 9 (warp 1), or one halo-column value (warp 2)
    int extra = -1;
    if (ty == 0) extra = kSpD + V * tx;
    else if (ty == 1) extra = (kSpTY + 1) * BW + kSpD + V * tx;
    else if (ty == 2 && tx < 2 * kSpTY)
        extra = tx < kSpTY ? (tx + 1) * BW + kSpD - 1 : (tx - kSpTY + 1) * BW + kSpD + kSpTW;
    const int np = ke - kb + 2;   // planes kb-1 .. ke
    const int s0 = (int)(seq % NST);
    const uint32_t ph0 = (seq / NST) & 1u;
    bool bad = false;   // a wait of this thread ran out
    auto wait = [&](int sl, uint32_t ph) {
        if (!mbar_wait_bounded(&bars[sl], ph)) bad = true;
    };
    auto fix = [&](long long b) -> long long { return CONV ? xs_fix(b, emax) : b; };
    auto convert = [&](long long* pl, long long (&fx)[RT][V], double (&raw)[RT][V]) {
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            const longlong2 b = *reinterpret_cast<const longlong2*>(pl + own + j * BW);
            raw[j][0] = __longlong_as_double(b.x);
            raw[j][1] = __longlong_as_double(b.y);
            fx[j][0] = fix(b.x);
            fx[j][1] = fix(b.y);
            if constexpr (CONV) *reinterpret_cast<longlong2*>(pl + own + j * BW) = make_longlong2(fx[j][0], fx[j][1]);
        }
        if constexpr (CONV) {
            if (ty < 2) {
                const longlong2 h = *reinterpret_cast<const longlong2*>(pl + extra);
                *reinterpret_cast<longlong2*>(pl + extra) = make_longlong2(fix(h.x), fix(h.y));
            } else if (extra >= 0) {
                pl[extra] = fix(pl[extra]);
            }
        }
    };

    int issued = 0;
    if (tid == 0) {
        fence_proxy_async_smem();
        for (int sl = s0; issued < NST && issued < np; ++issued, sl = sl + 1 == NST ? 0 : sl + 1) {
            mbar_arrive_expect_tx(&bars[sl], kSpBoxBytes);
            tma_load_3d(stage + sl * kSpStage, map, x0 - kSpD, y0 - 1, kb - 1 + issued, &bars[sl]);
        }
    }
    // the planes below, at and above k (fixed-point values, raw bits when
    // !CONV) and the raw values at and above k
    long long B[RT][V], C[RT][V], Ab[RT][V];
    double RC[RT][V], RA[RT][V];
    int s_cur = s0;
    uint32_t ph_cur = ph0;
    wait(s_cur, ph_cur);
#pragma unroll
    for (int j = 0; j < RT; ++j) {
        const longlong2 b = *reinterpret_cast<const longlong2*>(stage + s_cur * kSpStage + own + j * BW);
        B[j][0] = fix(b.x);
        B[j][1] = fix(b.y);
    }
    if (++s_cur == NST) {
        s_cur = 0;
        ph_cur ^= 1u;
    }
    wait(s_cur, ph_cur);
    convert(stage + s_cur * kSpStage, C, RC);
    if constexpr (CONV) fence_proxy_async_smem();
    // the barriers reduce the threads' wait results, so all agree on an abort
    aborted = __syncthreads_or(bad) != 0;

    double pq = 0.0;
    for (int k = kb; !aborted && k < ke; ++k) {
        const int s_nxt = s_cur + 1 == NST ? 0 : s_cur + 1;
        const uint32_t ph_nxt = s_nxt == 0 ? ph_cur ^ 1u : ph_cur;
        wait(s_nxt, ph_nxt);
        convert(stage + s_nxt * kSpStage, Ab, RA);
        const long long* pc = stage + s_cur * kSpStage + own;
        const long long ym[V] = {pc[-BW], pc[1 - BW]}, yp[V] = {pc[RT * BW], pc[RT * BW + 1]};
        const long long left[RT] = {pc[-1], pc[BW - 1]}, right[RT] = {pc[V], pc[BW + V]};
        double qv[RT][V];
        spmv_points<CONV>(B, C, Ab, ym, yp, left, right, emax, qv);
#pragma unroll
        for (int j = 0; j < RT; ++j)
            if (ok[j]) {
                double* dst = q + (int64_t)k * sxy + (int64_t)(Y0 + j) * nx + X;
                *reinterpret_cast<double2*>(dst) = make_double2(qv[j][0], qv[j][1]);
                pq = __fma_rn(RC[j][0], qv[j][0], pq);
                pq = __fma_rn(RC[j][1], qv[j][1], pq);
            }
#pragma unroll
        for (int j = 0; j < RT; ++j)
#pragma unroll
            for (int i = 0; i < V; ++i) {
                B[j][i] = C[j][i];
                C[j][i] = Ab[j][i];
                RC[j][i] = RA[j][i];
            }
        if constexpr (CONV) fence_proxy_async_smem();
        aborted = __syncthreads_or(bad) != 0;
        // the slot of the plane below is free: every thread is past its last use
        if (!aborted && tid == 0 && issued < np) {
            const int sl = s_cur == 0 ? NST - 1 : s_cur - 1;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[sl], kSpBoxBytes);
            tma_load_3d(stage + sl * kSpStage, map, x0 - kSpD, y0 - 1, kb - 1 + issued, &bars[sl]);
            ++issued;
        }
        s_cur = s_nxt;
        ph_cur = ph_nxt;
    }
    if (aborted && tid == 0) {
        // the last load issued into each slot, consumed or not, completes
        // before the block may end
        const long long t0 = clock64();   // one time budget for the whole drain
        for (int j = issued > NST ? issued - NST : 0; j < issued; ++j)
            if (!mbar_wait_until(&bars[(seq + j) % NST], ((seq + j) / NST) & 1u, t0, kWaitCycles)) {
                drained = false;   // loads may still be landing: the context is suspect
                break;
            }
    }
    seq += (uint32_t)np;
    return pq;
}

__global__ void __launch_bounds__(kSpBlock, 5)
    k_cg_spmv_tma(const __grid_constant__ CUtensorMap map, OpDev A, double* __restrict__ q,
                  double* partials, CgScalars* S)
{
    __shared__ __align__(128) long long stage[kSpNst * kSpStage];
    __shared__ __align__(8) uint64_t bars[kSpNst];
    __shared__ double sh[kSpBlock / 32];
    __shared__ int32_t s_done;
    const int tid = threadIdx.x;
    grid_dependency_wait();   // p, the scalars and the stop flag come from the kernels before
    if (tid == 0) {
        // one read for the block: another block's abort may change the flag
        s_done = *(volatile int32_t*)&S->done;
        for (int s = 0; s < kSpNst; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_done) return;
    const int emax = cg_pemax(S);
    const bool conv = cg_xs_ok(emax);
    const SpmvPlan P = spmv_plan(A);
    uint32_t seq = 0;
    bool aborted = false, drained = true;
    double pq = 0.0;
    for (SpmvShare sh = spmv_share(A, P, blockIdx.x, gridDim.x); sh.next < sh.last;) {
        int64_t tile;
        int kb, ke;
        spmv_next_run(A, sh, tile, kb, ke);
        pq += conv ? spmv_item_tma<true>(&map, A, q, emax, P, tile, kb, ke, stage, bars, seq, aborted, drained)
                   : spmv_item_tma<false>(&map, A, q, emax, P, tile, kb, ke, stage, bars, seq, aborted, drained);
        if (aborted) break;   // the same in every thread
    }
    if (aborted) {
        // 3: a wait ran out; 4: so did the wait for this block's loads in flight
        if (tid == 0) atomicMax(reinterpret_cast<int*>(&S->done), drained ? 3 : 4);
        return;
    }
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

bool spmv_tma_eligible(const OpDev& A, const double* p, const double* q, int nblocks)
{
    return A.kind == HS_OP_STENCIL7 && spmv_mode(A, nblocks) == SP_STAGED && (A.nx & 1) == 0 &&
           ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15) == 0;
}

int spmv_tma_map(CUtensorMap* map, const OpDev& A, const double* p)
{
    return encode_field_map(map, const_cast<double*>(p), CU_TENSOR_MAP_DATA_TYPE_INT64, sizeof(double),
                            (uint64_t)A.nx, (uint64_t)A.ny, (uint64_t)A.nz, kSpBW, kSpTY + 2);
}

// The caller checks and counts the launch, as for the other SpMV kernels.
int spmv_tma_launch(const CUtensorMap& map, const OpDev& A, double* q, double* partials, CgScalars* S,
                    int nshares, cudaStream_t stream)
{
    const cudaError_t e = launch_dependent(k_cg_spmv_tma, nshares, kSpBlock, stream, map, A, q, partials, S);
    return e == cudaSuccess ? HS_OK : cuda_fail(e, "cg: spmv+dot kernel (TMA-staged)");
}

// Resident TMA-staged blocks, asked once per process (a single GPU): blocks per
// SM at the kernel's registers and shared memory, times the SM count.
int spmv_shares(int nblocks)
{
    static const int slots = [] {
        int per_sm = 0, dev = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_spmv_tma, kSpBlock, 0) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return kNumSMs * kSpMinBlocks;
        }
        return per_sm > 0 && sms > 0 ? per_sm * sms : kNumSMs * kSpMinBlocks;
    }();
    return nblocks < slots ? nblocks : slots;
}

}  // namespace hcg
