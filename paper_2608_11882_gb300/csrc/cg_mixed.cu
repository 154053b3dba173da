// Mixed-precision CG: FP32 Krylov vectors inside FP64 iterative refinement.
//
//   x (FP64, the caller's)                     outer loop, until ||b - A x|| / ||b|| <= rtol:
//     r  = b - A x              in FP64          (true residual, FP64 operator)
//     solve A d = r approximately by CG with d, r', p, q stored in FP32 and
//        the FP32 operator (matrix-free, or the CSR values rounded to FP32),
//        stopping once ||r'|| <= max(inner_rtol, rtol ||b|| / (2 ||r||)) ||r'_0||
//     x += d                    in FP64
//
// The CG of each inner solve is the textbook one of Section 7.5.  Its dot
// products accumulate in FP64 across the grid: each thread adds at most 4
// FP32 products before promoting them to its FP64 sum (the SpMV kernels keep
// that sum as an exact FP32 two-sum pair instead and convert it once), so
// the long sums --
// the part whose stability needs FP64 -- stay FP64 while the FP64 pipe (about
// 1/64 of FP32 issue on this GPU) sees one add per 8 elements.  alpha, beta
// and the residual norms are FP64 device scalars.  Refinement converges while
// kappa(A) times FP32's unit roundoff is well below one (about 6e-3 for the
// 512^3 Laplacian).
#include <cmath>
#include <cstring>
#include <new>

#include "cg_common.cuh"
#include "tma.cuh"

namespace hcg {

struct MxScalars {
    double rho;       // r'.r' of the inner recurrence
    double rho0;      // r'.r' at the start of the inner solve
    double pq;
    double alpha, beta;
    double rr64;      // ||b - A x||^2 (FP64)
    double bnorm;     // ||b||
    double rtol, inner_rtol;
    double inner_stop;    // the inner solve ends once r'.r' <= inner_stop
    int32_t outer_done;   // 1: ||b - A x|| / ||b|| <= rtol (or b = 0)
    int32_t inner_done;   // 1: inner solve finished; 2: breakdown; 3: a bounded wait of the
                          // TMA-staged SpMV ran out; 4: that, and its loads in flight did not
                          // complete in time
    int32_t iters;        // inner iterations, all solves
    uint32_t ticket;
    int32_t zero_rhs;
    int32_t first;        // 1 until ||b|| has been computed
};

struct OpDev32 {
    int32_t kind;
    int32_t nx, ny, nz;
    int64_t n;
    const int32_t* rowptr;
    const int32_t* col;
    const float* val;
};

}  // namespace hcg

struct hcg::CgMixed {
    OpDev32 A32;
    float* d;
    float* r;
    float* p;
    float* q;
    double* r64;         // FP64 residual (the context's r)
    double* q64;         // A x in FP64 (the context's q)
    float* val32;        // CSR values in FP32 (owned), else NULL
    double* partials;    // 2 * grid
    MxScalars* S;
    MxScalars* S_host;   // host mirror
    double inner_rtol;
    int32_t max_inner;
    bool tma;            // the matrix-free SpMV stages r and p by TMA (nx a multiple of 4)
    int spmv_grid;       // its grid: the blocks resident at once, at most the context's grid
    float* p2;           // with tma: the second p buffer (p' goes to the other one)
    int pcur;            // with tma: which of p, p2 holds the current direction
    CUtensorMap rmap;    // TMA maps of r, p and p2 (unpadded nx x ny x nz floats)
    CUtensorMap pmaps[2];
};

namespace hcg {

// FP64 sum of FP32 products: add() promotes every 8 terms (one product at a
// time), add4() sums four products in FP32 and promotes them at once -- one
// conversion and one FP64 add per four products, with no per-product branch
// that the compiler could turn into a conversion per product.
struct Acc32 {
    double hi = 0.0;
    float lo = 0.0f;
    int n = 0;
    __device__ __forceinline__ void add(float a, float b)
    {
        lo = __fmaf_rn(a, b, lo);
        if (++n == 8) {
            hi += (double)lo;
            lo = 0.0f;
            n = 0;
        }
    }
    __device__ __forceinline__ void add4(float a0, float b0, float a1, float b1, float a2, float b2, float a3,
                                         float b3)
    {
        const float s = __fmaf_rn(a3, b3, __fmaf_rn(a2, b2, __fmaf_rn(a1, b1, __fmul_rn(a0, b0))));
        hi += (double)s;
    }
    __device__ __forceinline__ double total() const { return hi + (double)lo; }
};

// The same sums kept in two FP32 words (Knuth's two-sum: hi + lo holds the
// running sum to about 2^-48 of its size) and turned into FP64 once, at the
// end: groups of four products summed in FP32 as in Acc32::add4, then added
// without rounding error -- no FP64 instruction in the loop.
struct AccF2 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add4(float a0, float b0, float a1, float b1, float a2, float b2, float a3,
                                         float b3)
    {
        const float v = __fmaf_rn(a3, b3, __fmaf_rn(a2, b2, __fmaf_rn(a1, b1, __fmul_rn(a0, b0))));
        const float s = __fadd_rn(hi, v);
        const float bv = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    // one product, rounded to FP32, added without rounding error
    __device__ __forceinline__ void add(float a, float b)
    {
        const float v = __fmul_rn(a, b);
        const float s = __fadd_rn(hi, v);
        const float bv = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    __device__ __forceinline__ double total() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ float apply32_csr(const OpDev32& A, const float* __restrict__ p, int64_t row)
{
    float s = 0.0f;
    const int e = __ldg(A.rowptr + row + 1);
    for (int t = __ldg(A.rowptr + row); t < e; ++t)
        s = __fmaf_rn(__ldg(A.val + t), __ldg(p + __ldg(A.col + t)), s);
    return s;
}


__global__ void __launch_bounds__(kCgBlock)
    k_mx_to_f32(int64_t n, const double* __restrict__ src, float* __restrict__ dst)
{
    for (int64_t t = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * kCgBlock)
        dst[t] = __double2float_rn(src[t]);
}

// r64 = b - q64 (q64 = A x); ||r64||^2 (and ||b||^2 the first time) in FP64;
// the inner start r' = p = float(r64), d = 0, rho0 = r'.r'.  Decides the outer stop.
__global__ void __launch_bounds__(kCgBlock)
    k_mx_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ q64,
                  double* __restrict__ r64, float* __restrict__ r, float* __restrict__ p,
                  float* __restrict__ d, double* partials, MxScalars* S)
{
    __shared__ double sh[kCgBlock / 32];
    const bool first = S->first != 0;
    double rr = 0.0, bb = 0.0;
    Acc32 rho;
    for (int64_t t = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * kCgBlock) {
        const double bt = b[t];
        const double rt = bt - q64[t];
        r64[t] = rt;
        const float rf = __double2float_rn(rt);
        r[t] = rf;
        p[t] = rf;
        d[t] = 0.0f;
        rr = __fma_rn(rt, rt, rr);
        if (first) bb = __fma_rn(bt, bt, bb);
        rho.add(rf, rf);
    }
    const double rr_blk = block_sum<kCgBlock>(rr, sh);
    const double bb_blk = block_sum<kCgBlock>(bb, sh);
    const double rho_blk = block_sum<kCgBlock>(rho.total(), sh);
    if (threadIdx.x == 0) {
        partials[gridDim.x + blockIdx.x] = bb_blk;
        partials[2 * gridDim.x + blockIdx.x] = rho_blk;
    }
    if (!arrive_last(rr_blk, partials, &S->ticket)) return;
    const double rr_tot = sum_partials(partials, gridDim.x, sh);
    const double bb_tot = first ? sum_partials(partials + gridDim.x, gridDim.x, sh) : 0.0;
    const double rho_tot = sum_partials(partials + 2 * gridDim.x, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        if (first) {
            S->bnorm = sqrt(bb_tot);
            S->zero_rhs = (bb_tot == 0.0);
            S->first = 0;
        }
        S->rr64 = rr_tot;
        S->rho = rho_tot;
        S->rho0 = rho_tot;
        // reduce the residual by inner_rtol, or just by what reaching rtol (with a
        // factor-2 margin) needs, whichever is the smaller reduction
        double f2 = S->inner_rtol * S->inner_rtol;
        const double need = 0.5 * S->rtol * S->bnorm;
        if (rr_tot > 0.0 && need * need / rr_tot > f2) f2 = need * need / rr_tot;
        S->inner_stop = f2 * rho_tot;
        S->inner_done = 0;
        S->beta = 0.0;   // the first direction of the inner solve is r itself
        S->outer_done = (S->zero_rhs || sqrt(rr_tot) / S->bnorm <= S->rtol) ? 1 : 0;
        if (S->outer_done || rho_tot == 0.0) S->inner_done = 1;
    }
}

template <int KIND>
__global__ void __launch_bounds__(kCgBlock)
    k_mx_spmv_dot(OpDev32 A, const float* __restrict__ p, float* __restrict__ q, double* partials,
                  MxScalars* S)
{
    grid_dependency_wait();
    if (*(volatile int32_t*)&S->inner_done) return;
    __shared__ double sh[kCgBlock / 32];
    AccF2 pq;
    const int64_t row0 = (int64_t)blockIdx.x * kCgBlock + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * kCgBlock;
    if (KIND == HS_OP_STENCIL7) {
        // (tile of 32 x 8 columns, chunk of z-planes) items taken by the blocks
        // in a fixed order; a thread marches up its column with the values at
        // k-1, k, k+1 in registers, the in-plane neighbours through L1
        const int nx = A.nx, ny = A.ny, nz = A.nz;
        const int64_t sxy = (int64_t)nx * ny;
        const int tiles_x = (nx + 31) / 32;
        const int64_t tiles = (int64_t)tiles_x * ((ny + 7) / 8);
        int64_t chunks = (2 * (int64_t)gridDim.x + tiles - 1) / tiles;
        const int64_t maxc = nz / 4 > 1 ? nz / 4 : 1;
        if (chunks > maxc) chunks = maxc;
        const int kc = (int)((nz + chunks - 1) / chunks);
        chunks = (nz + kc - 1) / kc;
        const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
        for (int64_t item = blockIdx.x; item < tiles * chunks; item += gridDim.x) {
            const int64_t tile = item % tiles;
            const int i = (int)(tile % tiles_x) * 32 + tx, j = (int)(tile / tiles_x) * 8 + ty;
            const int kb = (int)(item / tiles) * kc, ke = min(kb + kc, nz);
            if (i >= nx || j >= ny) continue;
            int64_t c = (int64_t)kb * sxy + (int64_t)j * nx + i;
            float below = kb > 0 ? __ldg(p + c - sxy) : 0.0f;
            float cur = __ldg(p + c);
            for (int k = kb; k < ke; ++k) {
                const float above = k < nz - 1 ? __ldg(p + c + sxy) : 0.0f;
                const float ym = j > 0 ? __ldg(p + c - nx) : 0.0f;
                const float xm = i > 0 ? __ldg(p + c - 1) : 0.0f;
                const float xp = i < nx - 1 ? __ldg(p + c + 1) : 0.0f;
                const float yp = j < ny - 1 ? __ldg(p + c + nx) : 0.0f;
                const float sum = ((below + ym) + (xm + xp)) + (yp + above);
                const float qv = __fmaf_rn(6.0f, cur, -sum);
                q[c] = qv;
                pq.add(cur, qv);
                below = cur;
                cur = above;
                c += sxy;
            }
        }
    } else {
        for (int64_t row = row0; row < A.n; row += stride) {
            const float qv = apply32_csr(A, p, row);
            q[row] = qv;
            pq.add(__ldg(p + row), qv);
        }
    }
    allow_dependents();
    const double blk = block_sum<kCgBlock>(pq.total(), sh);
    if (!arrive_last(blk, partials, &S->ticket)) return;
    const double tot = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->pq = tot;
        if (!(tot > 0.0))
            S->inner_done = 2;
        else
            S->alpha = S->rho / tot;
    }
}

// The matrix-free FP32 SpMV with the direction update folded in, r and p staged
// by TMA: it forms p' = r + beta p (the p update of the iteration before) and
// q = A p' in one pass, so p is read once and written once per iteration
// instead of twice, and the iteration runs two kernels instead of three.
// Because blocks read the halo planes, rows and columns of their tiles, p' goes
// to the other of two p buffers (p_old stays intact for every block).  A block
// of 256 threads (8 warps) owns a tile of 128 x 8 points of the grid -- every
// lane four consecutive x points of one row, one 16-byte vector -- and a run of
// z-planes at a time: the grid is one resident wave of blocks, block b taking
// the b-th of gridDim.x equal shares of the (tile, plane) pairs in tile-major
// order (one run of planes, or two at a tile boundary).  Each
// plane of the tile with its one-point halo is two TMA boxes (r and p_old) of
// (8 + 2) rows of 136 floats starting 16 bytes left of the tile, over the
// unpadded vectors, so boxes that reach past the grid read zeros and give p' = 0
// there (the Dirichlet boundary).  Boxes land in a ring of kMxNst stages up to
// kMxNst - 2 planes ahead of use; once a plane lands, each thread forms p' in
// place for its own vector (warps 0-1 also the halo rows, warp 2 the halo
// columns) and keeps its own values at k-1, k and k+1 in registers; the other
// neighbours are read from the stage of plane k after the block barrier.  p' =
// fma(beta, p, r) and q = fma(6, p', -(((zm + ym) + (xm + xp)) + (yp + zp)))
// point by point, as in the p-update kernel and the column kernel, so p, q and
// every iterate are the same bit for bit as with the two separate passes.
// Every mbarrier wait is bounded; one that runs out stops the inner solve
// (inner_done 3) after the block's loads in flight have landed (4 if they do
// not in time).  Measured at 256^3 (solve to 1e-8): before the fold 30.0 us
// per SpMV and 141.8-142.9 ms per solve (one wave of equal shares was slower
// there: 144.1-144.5 ms); folded, with 1216 blocks of fixed 14-plane items (1.6
// waves), 52.8 us per launch and 132.6-132.7 ms; folded, one wave: 131.0 ms.
constexpr int kMxTW = 128, kMxTY = 8, kMxD = 4, kMxBW = 136, kMxNst = 4;
constexpr uint32_t kMxBoxBytes = (kMxTY + 2) * kMxBW * sizeof(float);
constexpr int kMxStage = (int)((kMxBoxBytes + 127) / 128 * 128 / sizeof(float));
static_assert(kMxBW * sizeof(float) % 16 == 0 && kMxD * sizeof(float) == 16, "TMA box geometry");
static_assert(kMxTY * 32 == kCgBlock, "one warp per tile row");
static_assert(2 * kMxTY <= 32, "one warp forms the halo columns");

__global__ void __launch_bounds__(kCgBlock)
    k_mx_spmv_tma(const __grid_constant__ CUtensorMap rmap, const __grid_constant__ CUtensorMap pmap,
                  OpDev32 A, float* __restrict__ pn, float* __restrict__ q, double* partials, MxScalars* S)
{
    // stage sl: the r box at 2 sl, the p box (p' once formed) at 2 sl + 1
    __shared__ __align__(128) float stage[kMxNst * 2 * kMxStage];
    __shared__ __align__(8) uint64_t bars[kMxNst];
    __shared__ double sh[kCgBlock / 32];
    __shared__ int32_t s_done;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    grid_dependency_wait();   // r, p, the scalars and the stop flag come from the kernels before
    if (tid == 0) {
        s_done = *(volatile int32_t*)&S->inner_done;
        for (int sl = 0; sl < kMxNst; ++sl) mbar_init(&bars[sl], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_done) return;
    const float beta = (float)S->beta;
    const int nx = A.nx, ny = A.ny;
    const int tiles_x = (nx + kMxTW - 1) / kMxTW;
    const int64_t sxy = (int64_t)nx * ny;
    // this thread's vector in a box, and the halo it forms besides
    const int own = (ty + 1) * kMxBW + kMxD + 4 * tx;
    int hvec = -1, hone = -1;
    if (ty < 2)
        hvec = (ty == 0 ? 0 : kMxTY + 1) * kMxBW + kMxD + 4 * tx;
    else if (ty == 2 && tx < 2 * kMxTY)
        hone = tx < kMxTY ? (tx + 1) * kMxBW + kMxD - 1 : (tx - kMxTY + 1) * kMxBW + kMxD + kMxTW;
    uint32_t seq = 0;   // planes staged so far: plane j of the block sits in slot j % NST
    bool bad = false, aborted = false, drained = true;
    int issued = 0, np = 0;
    AccF2 pq;
    // this block's share of the (tile, plane) pairs in tile-major order
    const int64_t pairs = (int64_t)tiles_x * ((ny + kMxTY - 1) / kMxTY) * A.nz;
    int64_t next = pairs * blockIdx.x / gridDim.x;
    const int64_t last = pairs * (blockIdx.x + 1) / gridDim.x;
    while (next < last && !aborted) {
        const int64_t tile = next / A.nz;
        const int kb = (int)(next % A.nz);
        const int ke = last - next < (int64_t)(A.nz - kb) ? kb + (int)(last - next) : A.nz;
        next += ke - kb;
        const int x0 = (int)(tile % tiles_x) * kMxTW, y0 = (int)(tile / tiles_x) * kMxTY;
        const int X = x0 + 4 * tx, Y = y0 + ty;
        const int nvalid = Y < ny ? min(4, nx - X) : 0;   // nx % 4 == 0: 4 or none
        np = ke - kb + 2;                                // planes kb-1 .. ke
        issued = 0;
        auto wait = [&](int j) {
            const uint32_t g = seq + (uint32_t)j;
            if (!mbar_wait_bounded(&bars[g % kMxNst], (g / kMxNst) & 1u)) bad = true;
        };
        auto issue = [&](int j) {   // plane kb - 1 + j into its slot (thread 0)
            const int sl = (int)((seq + j) % kMxNst);
            mbar_arrive_expect_tx(&bars[sl], 2 * kMxBoxBytes);
            tma_load_3d(stage + 2 * sl * kMxStage, &rmap, x0 - kMxD, y0 - 1, kb - 1 + j, &bars[sl]);
            tma_load_3d(stage + (2 * sl + 1) * kMxStage, &pmap, x0 - kMxD, y0 - 1, kb - 1 + j, &bars[sl]);
        };
        if (tid == 0) {
            fence_proxy_async_smem();   // the slots were last written by this block's threads
            for (; issued < kMxNst && issued < np; ++issued) issue(issued);
        }
        // p' = fma(beta, p, r) in place in the p box of plane j; o: this thread's vector
        auto form = [&](int j, float (&o)[4]) {
            const int sl = (int)((seq + j) % kMxNst);
            const float* rb = stage + 2 * sl * kMxStage;
            float* pb = stage + (2 * sl + 1) * kMxStage;
            auto vec = [&](int at) {
                const float4 rv = *reinterpret_cast<const float4*>(rb + at);
                float4 pv = *reinterpret_cast<const float4*>(pb + at);
                pv.x = __fmaf_rn(beta, pv.x, rv.x);
                pv.y = __fmaf_rn(beta, pv.y, rv.y);
                pv.z = __fmaf_rn(beta, pv.z, rv.z);
                pv.w = __fmaf_rn(beta, pv.w, rv.w);
                *reinterpret_cast<float4*>(pb + at) = pv;
                return pv;
            };
            const float4 v = vec(own);
            o[0] = v.x;
            o[1] = v.y;
            o[2] = v.z;
            o[3] = v.w;
            if (hvec >= 0) vec(hvec);
            if (hone >= 0) pb[hone] = __fmaf_rn(beta, pb[hone], rb[hone]);
            fence_proxy_async_smem();   // before the barrier after which TMA may refill the slot
        };
        float below[4], cur[4], above[4];
        wait(0);
        form(0, below);
        wait(1);
        form(1, cur);
        if (__syncthreads_or(bad)) {
            aborted = true;
            break;
        }
        const int64_t at = (int64_t)kb * sxy + (int64_t)(Y < ny ? Y : 0) * nx + (X < nx ? X : 0);
        float* dst = q + at;
        float* dstp = pn + at;
        for (int k = kb; k < ke; ++k) {
            const int j = k - kb + 1;   // plane k is plane j of the run
            wait(j + 1);
            form(j + 1, above);
            const float* pc = stage + (2 * ((seq + j) % kMxNst) + 1) * kMxStage + own;
            const float4 ymv = *reinterpret_cast<const float4*>(pc - kMxBW);
            const float4 ypv = *reinterpret_cast<const float4*>(pc + kMxBW);
            const float ym[4] = {ymv.x, ymv.y, ymv.z, ymv.w}, yp[4] = {ypv.x, ypv.y, ypv.z, ypv.w};
            const float left = pc[-1], right = pc[4];
            float qv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float xm = i == 0 ? left : cur[i - 1];
                const float xp = i == 3 ? right : cur[i + 1];
                const float sum = ((below[i] + ym[i]) + (xm + xp)) + (yp[i] + above[i]);
                qv[i] = __fmaf_rn(6.0f, cur[i], -sum);
            }
            if (nvalid == 4) {
                *reinterpret_cast<float4*>(dstp) = make_float4(cur[0], cur[1], cur[2], cur[3]);
                *reinterpret_cast<float4*>(dst) = make_float4(qv[0], qv[1], qv[2], qv[3]);
                pq.add4(cur[0], qv[0], cur[1], qv[1], cur[2], qv[2], cur[3], qv[3]);
            }
            dst += sxy;
            dstp += sxy;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                below[i] = cur[i];
                cur[i] = above[i];
            }
            if (__syncthreads_or(bad)) {
                aborted = true;
                break;
            }
            // the slot of plane k-1 is free: every thread is past its last use
            // (refilling plane k's slot, one plane earlier, measured no faster)
            if (tid == 0 && issued < np) {
                fence_proxy_async_smem();
                issue(issued);
                ++issued;
            }
        }
        if (!aborted) aborted = __syncthreads_or(bad) != 0;
        if (aborted) break;
        seq += (uint32_t)np;
    }
    if (aborted) {
        if (tid == 0) {
            // the last load issued into each slot, consumed or not, completes before the block ends
            const long long t0 = clock64();
            for (int j = issued > kMxNst ? issued - kMxNst : 0; j < issued; ++j) {
                const uint32_t g = seq + (uint32_t)j;
                if (!mbar_wait_until(&bars[g % kMxNst], (g / kMxNst) & 1u, t0, kWaitCycles)) {
                    drained = false;
                    break;
                }
            }
            atomicMax(reinterpret_cast<int*>(&S->inner_done), drained ? 3 : 4);
        }
        return;
    }
    allow_dependents();
    const double blk = block_sum<kCgBlock>(pq.total(), sh);
    if (!arrive_last(blk, partials, &S->ticket)) return;
    const double tot = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->pq = tot;
        if (!(tot > 0.0))
            S->inner_done = 2;
        else
            S->alpha = S->rho / tot;
    }
}

__global__ void __launch_bounds__(kCgBlock)
    k_mx_update(int64_t n, float* __restrict__ d, float* __restrict__ r, const float* __restrict__ p,
                const float* __restrict__ q, double* partials, MxScalars* S)
{
    grid_dependency_wait();
    if (*(volatile int32_t*)&S->inner_done) return;
    __shared__ double sh[kCgBlock / 32];
    const float alpha = (float)S->alpha;
    Acc32 rr;
    // groups of four values as 16-byte vectors (the FP32 vectors start aligned),
    // the last n % 4 values by thread 0
    const int64_t t0 = (int64_t)blockIdx.x * kCgBlock + threadIdx.x, stride = (int64_t)gridDim.x * kCgBlock;
    const int64_t n4 = n >> 2;
    for (int64_t t = t0; t < n4; t += stride) {
        const float4 pv = reinterpret_cast<const float4*>(p)[t];
        const float4 qv = reinterpret_cast<const float4*>(q)[t];
        float4 dv = reinterpret_cast<float4*>(d)[t];
        float4 rv = reinterpret_cast<float4*>(r)[t];
        dv.x = __fmaf_rn(alpha, pv.x, dv.x);
        dv.y = __fmaf_rn(alpha, pv.y, dv.y);
        dv.z = __fmaf_rn(alpha, pv.z, dv.z);
        dv.w = __fmaf_rn(alpha, pv.w, dv.w);
        rv.x = __fmaf_rn(-alpha, qv.x, rv.x);
        rv.y = __fmaf_rn(-alpha, qv.y, rv.y);
        rv.z = __fmaf_rn(-alpha, qv.z, rv.z);
        rv.w = __fmaf_rn(-alpha, qv.w, rv.w);
        reinterpret_cast<float4*>(d)[t] = dv;
        reinterpret_cast<float4*>(r)[t] = rv;
        rr.add4(rv.x, rv.x, rv.y, rv.y, rv.z, rv.z, rv.w, rv.w);
    }
    if (t0 == 0)
        for (int64_t t = n4 << 2; t < n; ++t) {
            d[t] = __fmaf_rn(alpha, p[t], d[t]);
            const float rt = __fmaf_rn(-alpha, q[t], r[t]);
            r[t] = rt;
            rr.add(rt, rt);
        }
    allow_dependents();
    const double blk = block_sum<kCgBlock>(rr.total(), sh);
    if (!arrive_last(blk, partials, &S->ticket)) return;
    const double rho_new = sum_partials(partials, gridDim.x, sh);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->iters += 1;
        if (rho_new <= S->inner_stop) {
            S->inner_done = 1;
        } else {
            S->beta = rho_new / S->rho;
        }
        S->rho = rho_new;
    }
}

__global__ void __launch_bounds__(kCgBlock)
    k_mx_pupdate(int64_t n, const float* __restrict__ r, float* __restrict__ p, MxScalars* S)
{
    grid_dependency_wait();
    if (*(volatile int32_t*)&S->inner_done) return;
    const float beta = (float)S->beta;
    const int64_t t0 = (int64_t)blockIdx.x * kCgBlock + threadIdx.x, stride = (int64_t)gridDim.x * kCgBlock;
    const int64_t n4 = n >> 2;
    for (int64_t t = t0; t < n4; t += stride) {
        const float4 rv = reinterpret_cast<const float4*>(r)[t];
        float4 pv = reinterpret_cast<float4*>(p)[t];
        pv.x = __fmaf_rn(beta, pv.x, rv.x);
        pv.y = __fmaf_rn(beta, pv.y, rv.y);
        pv.z = __fmaf_rn(beta, pv.z, rv.z);
        pv.w = __fmaf_rn(beta, pv.w, rv.w);
        reinterpret_cast<float4*>(p)[t] = pv;
    }
    if (t0 == 0)
        for (int64_t t = n4 << 2; t < n; ++t) p[t] = __fmaf_rn(beta, p[t], r[t]);
}

// x += d in FP64.
__global__ void __launch_bounds__(kCgBlock)
    k_mx_correct(int64_t n, double* __restrict__ x, const float* __restrict__ d)
{
    for (int64_t t = (int64_t)blockIdx.x * kCgBlock + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * kCgBlock)
        x[t] += (double)d[t];
}

void cg_mixed_release(CgMixed* m, cudaStream_t s)
{
    if (!m) return;
    dev_free(m->d, s);
    dev_free(m->r, s);
    dev_free(m->p, s);
    dev_free(m->p2, s);
    dev_free(m->q, s);
    dev_free(m->val32, s);
    dev_free(m->partials, s);
    dev_free(m->S, s);
    delete m->S_host;
    delete m;
}

// Outer/inner loop on the host: one synchronisation per outer step and one
// per chunk of inner iterations (kernels return at once after the inner stop).
int cg_run_mixed(hs_cg* c, const void* b_in, void* x_inout, int host_buffers, double rtol,
                 int32_t max_iter, hs_cg_info* info)
{
    CgMixed* m = c->mx;
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
    MxScalars init;
    memset(&init, 0, sizeof(init));
    init.rtol = rtol;
    init.inner_rtol = m->inner_rtol;
    init.first = 1;
    *m->S_host = init;
    HS_TRY_CUDA(cudaMemcpyAsync(m->S, m->S_host, sizeof(MxScalars), cudaMemcpyHostToDevice, c->stream),
                "cg_run: scalar init");
    const int G = c->grid;
    int32_t outer = 0;
    bool converged = false, breakdown = false;
    for (;;) {
        int rc = launch_apply(c->A, x, m->q64, c->stream);   // A x in FP64
        if (rc != HS_OK) return rc;
        k_mx_residual<<<G, kCgBlock, 0, c->stream>>>(n, b, m->q64, m->r64, m->r,
                                                    m->tma && m->pcur ? m->p2 : m->p, m->d,
                                                    m->partials, m->S);
        HS_CHECK_LAUNCH("cg mixed: residual kernel");
        HS_TRY_CUDA(cudaMemcpyAsync(m->S_host, m->S, sizeof(MxScalars), cudaMemcpyDeviceToHost, c->stream),
                    "cg_run: scalar readback");
        HS_TRY_CUDA(cudaStreamSynchronize(c->stream), "cg_run: synchronize");
        if (m->S_host->outer_done) {
            converged = true;
            break;
        }
        if (m->S_host->iters >= max_iter) break;
        // inner FP32 solve
        int32_t inner = 0;
        int chunk = 4;
        for (;;) {
            const int32_t budget_total = max_iter - m->S_host->iters - inner;
            const int32_t budget_inner = m->max_inner - inner;
            int32_t todo = chunk;
            if (todo > budget_total) todo = budget_total;
            if (todo > budget_inner) todo = budget_inner;
            if (todo <= 0) break;
            for (int32_t t = 0; t < todo; ++t) {
                // dependent launches: each kernel's launch overlaps the previous
                // kernel's final reduction (it waits for that kernel on entry)
                if (m->tma) {
                    // p' = r + beta p into the other buffer, q = A p', then the update
                    float* pn = m->pcur ? m->p : m->p2;
                    HS_TRY_CUDA(launch_dependent(k_mx_spmv_tma, m->spmv_grid, kCgBlock, c->stream, m->rmap,
                                                 m->pmaps[m->pcur], m->A32, pn, m->q, m->partials, m->S),
                                "cg mixed: kernel launch");
                    HS_CHECK_LAUNCH("cg mixed: p update + spmv + dot kernel");
                    HS_TRY_CUDA(launch_dependent(k_mx_update, G, kCgBlock, c->stream, n, m->d, m->r,
                                                 (const float*)pn, (const float*)m->q, m->partials, m->S),
                                "cg mixed: kernel launch");
                    HS_CHECK_LAUNCH("cg mixed: update kernel");
                    m->pcur ^= 1;
                    continue;
                }
                if (c->A.kind == HS_OP_STENCIL7)
                    HS_TRY_CUDA(launch_dependent(k_mx_spmv_dot<HS_OP_STENCIL7>, G, kCgBlock, c->stream, m->A32,
                                                 (const float*)m->p, m->q, m->partials, m->S),
                                "cg mixed: kernel launch");
                else
                    HS_TRY_CUDA(launch_dependent(k_mx_spmv_dot<HS_OP_CSR>, G, kCgBlock, c->stream, m->A32,
                                                 (const float*)m->p, m->q, m->partials, m->S),
                                "cg mixed: kernel launch");
                HS_CHECK_LAUNCH("cg mixed: spmv+dot kernel");
                HS_TRY_CUDA(launch_dependent(k_mx_update, G, kCgBlock, c->stream, n, m->d, m->r,
                                             (const float*)m->p, (const float*)m->q, m->partials, m->S),
                            "cg mixed: kernel launch");
                HS_CHECK_LAUNCH("cg mixed: update kernel");
                HS_TRY_CUDA(launch_dependent(k_mx_pupdate, G, kCgBlock, c->stream, n, (const float*)m->r, m->p,
                                             m->S),
                            "cg mixed: kernel launch");
                HS_CHECK_LAUNCH("cg mixed: p update kernel");
            }
            inner += todo;
            HS_TRY_CUDA(cudaMemcpyAsync(m->S_host, m->S, sizeof(MxScalars), cudaMemcpyDeviceToHost,
                                        c->stream),
                        "cg_run: scalar readback");
            HS_TRY_CUDA(cudaStreamSynchronize(c->stream), "cg_run: synchronize");
            if (m->S_host->inner_done) break;
            if (chunk < 32) chunk *= 2;
        }
        if (m->S_host->inner_done == 2) {
            breakdown = true;
            break;
        }
        if (m->S_host->inner_done == 3)
            return fail(HS_ETIMEOUT, "cg_run: a bounded wait in the TMA-staged FP32 SpMV ran out");
        if (m->S_host->inner_done == 4)
            return fail(HS_ECUDA, "cg_run: a bounded wait in the TMA-staged FP32 SpMV ran out and its loads "
                                  "in flight did not complete in time; treat the CUDA context as suspect");
        k_mx_correct<<<G, kCgBlock, 0, c->stream>>>(n, x, m->d);   // x += d (FP64)
        HS_CHECK_LAUNCH("cg mixed: correction kernel");
        ++outer;
    }
    if (m->S_host->zero_rhs) HS_TRY_CUDA(cudaMemsetAsync(x, 0, vbytes, c->stream), "cg_run: zero solution");
    if (host_buffers) {
        const int rc_ = copy_host(x_inout, x, vbytes, false, c->stream, "cg_run: copy of x");
        if (rc_ != HS_OK) return rc_;
    }
    HS_TRY_CUDA(cudaStreamSynchronize(c->stream), "cg_run: synchronize");
    if (breakdown) return fail(HS_ECUDA, "cg_run: breakdown in the FP32 inner solve");
    const MxScalars f = *m->S_host;   // from the last residual evaluation
    const double relres = f.zero_rhs ? 0.0 : sqrt(f.rr64) / f.bnorm;
    if (info) {
        info->iters = f.iters;
        info->relres_recur = relres;
        info->relres_true = relres;   // the outer residual is recomputed in FP64
        info->status = converged ? HS_OK : HS_ENOCONV;
        info->refinements = outer;
        info->reserved = 0;
    }
    if (!converged) {
        set_error("cg_run: mixed precision stopped at %d inner iterations (relres %g > rtol %g)",
                  f.iters, relres, rtol);
        return HS_ENOCONV;
    }
    return HS_OK;
}

}  // namespace hcg

using namespace hcg;

extern "C" {

int cg_create_mixed(hs_cg_t* out, const hs_op* A, const hs_cg_mixed_opts* opts, void* stream)
{
    if (!out) return fail(HS_EINVAL, "cg_create_mixed: out is NULL");
    *out = nullptr;
    double inner_rtol = 1e-4;
    int32_t max_inner = 1 << 20;
    if (opts) {
        if (opts->inner_rtol != 0.0) inner_rtol = opts->inner_rtol;
        if (opts->max_inner != 0) max_inner = opts->max_inner;
    }
    if (!(inner_rtol > 0.0 && inner_rtol < 1.0))
        return fail(HS_EINVAL, "cg_create_mixed: inner_rtol %g not in (0, 1)", inner_rtol);
    if (max_inner < 1) return fail(HS_EINVAL, "cg_create_mixed: max_inner < 1");
    hs_cg_t c = nullptr;
    int rc = cg_create(&c, A, stream);
    if (rc != HS_OK) return rc;
    CgMixed* m = new (std::nothrow) CgMixed();
    if (!m) {
        cg_destroy(c);
        return fail(HS_ENOMEM, "cg_create_mixed: host allocation failed");
    }
    c->mx = m;
    m->inner_rtol = inner_rtol;
    m->max_inner = max_inner;
    const int64_t n = c->A.n;
    const int G = c->grid;
    cudaError_t e = cudaSuccess;
    const cudaStream_t s = c->stream;
    for (float** v : {&m->d, &m->r, &m->p, &m->q})
        if (e == cudaSuccess) e = dev_alloc((void**)v, sizeof(float) * (size_t)n, s);
    // the FP64 residual and A x live in the context's FP64 r and q; its p is not needed
    m->r64 = c->r;
    m->q64 = c->q;
    dev_free(c->p, s);
    c->p = nullptr;
    if (e == cudaSuccess) e = dev_alloc((void**)&m->partials, sizeof(double) * 3 * (size_t)G, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&m->S, sizeof(MxScalars), s);
    if (e == cudaSuccess) {
        m->S_host = new (std::nothrow) MxScalars();
        if (!m->S_host) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess && c->A.kind == HS_OP_CSR) {
        const int64_t nnz = c->A.rowptr ? A->nnz : 0;
        e = dev_alloc((void**)&m->val32, sizeof(float) * (size_t)(nnz > 0 ? nnz : 1), s);
        if (e == cudaSuccess && nnz > 0) {
            k_mx_to_f32<<<grid_for(nnz), kCgBlock, 0, c->stream>>>(nnz, c->A.val, m->val32);
            e = cudaPeekAtLastError();
            count_launch();
        }
    }
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "cg_create_mixed: allocation");
        cg_destroy(c);
        return rc;
    }
    m->A32.kind = c->A.kind;
    m->A32.nx = c->A.nx;
    m->A32.ny = c->A.ny;
    m->A32.nz = c->A.nz;
    m->A32.n = n;
    m->A32.rowptr = c->A.rowptr;
    m->A32.col = c->A.col;
    m->A32.val = m->val32;
    // the FP32 matrix-free SpMV stages r and p by TMA, with the p update folded in,
    // when rows are a 16-byte multiple (the vectors start 256-byte aligned)
    m->tma = false;
    m->pcur = 0;
    if (m->A32.kind == HS_OP_STENCIL7 && m->A32.nx % 4 == 0) {
        e = dev_alloc((void**)&m->p2, sizeof(float) * (size_t)n, s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cg_create_mixed: allocation");
            cg_destroy(c);
            return rc;
        }
        const float* v[3] = {m->r, m->p, m->p2};
        CUtensorMap* maps[3] = {&m->rmap, &m->pmaps[0], &m->pmaps[1]};
        bool ok = true;
        for (int i = 0; i < 3 && ok; ++i)
            ok = (reinterpret_cast<uintptr_t>(v[i]) & 15) == 0 &&
                 encode_field_map(maps[i], const_cast<float*>(v[i]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                  sizeof(float), (uint64_t)m->A32.nx, (uint64_t)m->A32.ny, (uint64_t)m->A32.nz,
                                  kMxBW, kMxTY + 2) == 0;
        ok = ok && (reinterpret_cast<uintptr_t>(m->q) & 15) == 0;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mx_spmv_tma, kCgBlock, 0);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || per_sm < 1 || sms < 1) {
            rc = cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidConfiguration,
                           "cg_create_mixed: occupancy of the FP32 SpMV");
            cg_destroy(c);
            return rc;
        }
        m->spmv_grid = per_sm * sms < G ? per_sm * sms : G;
        m->tma = ok;
        if (!ok) {
            dev_free(m->p2, s);
            m->p2 = nullptr;
        }
    }
    *out = c;
    return HS_OK;
}

}  // extern "C"
