// Batched heat stepping: many independent grids (their own sizes, r, step
// counts, FP32 or FP64), every step of every grid, in ONE persistent kernel
// launch, optionally replayed from a captured CUDA graph.
//
// Work items are (step m, grid g, column tile, chunk of planes); a persistent
// grid of co-resident blocks takes them from an atomic counter in a fixed
// order that spreads every grid's steps over the whole run.
// An item of step m of grid g may start once all items of step m-1 of grid g
// have finished (a per-grid completion counter, published with a fence), so
// each step of a grid reads a complete previous time level -- the Interior
// and Boundary work of one step of Section 4's update, over the whole grid.
// Items of step m-1 always come earlier in the order, so they have been taken
// by running blocks and the wait ends; it is still bounded (about a second of
// SM clock unless heat_batch_set_wait_limit set another limit before the batch
// was created), after which the kernel records HS_ETIMEOUT and stops: blocks
// finish the item they hold and take no further one.
//
// Loads use ld.global.cg (L2 only): a block must never see another SM's
// freshly written plane through its own stale L1 lines.
//
// Plain FP64 grids run the exact-sum arithmetic of heat_step (heat_common.cuh):
// every item of step m reads the field maximum of step m from the grid's slot
// (m3 + m) % 3, which the items of step m-1 completed before the wait above
// let step m start; each item adds its outputs' maximum to slot (m3 + m + 1) % 3,
// and item 0 clears slot (m3 + m + 2) % 3, which no unfinished item reads.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <vector>

#include "heat_common.cuh"
#include "tma.cuh"

namespace hcg {

constexpr long long kBatchWaitCycles = 2000000000ll;   // about one second at GB300 clocks
// Wait limit that batches created from now on get (heat_batch_set_wait_limit).
static std::atomic<long long> g_batch_wait_cycles{kBatchWaitCycles};

// K_F64_XS_NATIVE: an exact-sum grid whose field is outside the convertible
// exponent range this step, stepped on the FP64 pipe (never a grid's kind).
enum BatchKind { K_F64_PIPE = 0, K_F32 = 1, K_F64_XS = 2, K_F64_XS_NATIVE = 3 };

struct BatchGrid {
    HeatGeom g;
    void* buf[2];
    double r;
    FxState* fx;        // K_F64_XS: the grid's per-step maxima
    int32_t kind;       // BatchKind
    int32_t cur;        // buffer holding the field when the batch starts
    int32_t m3;         // K_F64_XS: slot of the field when the batch starts
    int32_t tiles_x;    // column tiles per row of tiles
    int32_t tiles_xy;   // column tiles
    int32_t kz;         // planes per work item (the last chunk may be shorter)
    int32_t tiles;      // work items per step: column tiles x z-chunks
    int32_t tw;         // tile width: 64 (64 x 8 tiles) or 32 (32 x 16)
    int32_t pad;
    int64_t steps;
};

struct BatchDev {
    const BatchGrid* grids;
    // one descriptor per work item, in schedule order: step << 40 | grid << 24 |
    // item within the grid's step, so a block finds its item with one load
    const unsigned long long* sched;
    const CUtensorMap* maps;      // per grid: TMA maps of its two buffers (box BW x 10)
    unsigned long long* next;     // work counter
    unsigned long long* done;     // per grid: items completed, all steps
    int* err;
    int64_t items;
    long long wait_cycles;        // limit of the step wait, in SM clock cycles
};

// One work item of step m -- a column tile and a chunk [kb, ke) of its planes.
// A block of 32 x 4 threads owns a TW x TY tile of the grid's columns and
// marches up the chunk; every thread computes one 16-byte vector of
// consecutive x points (two doubles or four floats) in each of two adjacent
// rows.  Each plane of the tile with its one-point halo
// ((8 + 2) rows of BW elements) arrives by TMA into a ring of kBatchNst stages
// up to kBatchNst - 2 planes ahead of use, through a tensor map of the grid's
// source buffer kept in the batch's device memory; the ring and its mbarrier
// phases run on across the items a block takes (`seq` counts the planes
// staged so far).  Exact-sum FP64 planes are converted in place to fixed point
// once they land (every thread its own vectors, warps 0 and 1 the halo rows,
// warp 2 the halo columns), exactly as in heat_step's Interior kernel; FP32
// and FP64-pipe planes are used as they are.  The per-point arithmetic is that
// of heat_step, so every grid matches stepping it alone bit for bit.  Returns
// false when a bounded wait ran out (the block then stops).
// Tiles are TW x TY columns, TW = 64 or, for narrow grids, 32: FP64 64 x 8 (a
// warp per two rows of 64 points) or 32 x 16, FP32 64 x 16 or 32 x 32.
constexpr int kBatchRT = 2, kBatchTY = 4;   // rows per thread, warps per block
constexpr int kBatchNst = 4;
constexpr int kBatchSlot = 688;   // stage stride in 8-byte words: the largest box, 5440 B, to 128 B

template <typename T, int TW>
struct BatchShape {
    static constexpr int V = Vec<T>::V;                          // points per thread row: 16 bytes
    static constexpr int LPR = TW / V;                           // lanes per tile row
    static constexpr int TY = kBatchTY * (32 / LPR) * kBatchRT;  // tile rows
    static constexpr int A = 16 / (int)sizeof(T);                // elements per 16 bytes
    static constexpr int D = A;                                  // offset of the tile's first point
    static constexpr int BW = (D + TW + 1 + A - 1) / A * A;      // stage row, a 16-byte multiple
    static constexpr uint32_t BOX_BYTES = (TY + 2) * BW * (uint32_t)sizeof(T);
    static_assert(BOX_BYTES <= kBatchSlot * 8, "a box fits a stage");
};

// Tile rows and stage row width of a grid's tiles (host side).
inline int batch_tile_rows(int tw, bool f32)
{
    return f32 ? (tw == 64 ? BatchShape<float, 64>::TY : BatchShape<float, 32>::TY)
               : (tw == 64 ? BatchShape<double, 64>::TY : BatchShape<double, 32>::TY);
}
inline int batch_stage_row(int tw, bool f32)
{
    return f32 ? (tw == 64 ? BatchShape<float, 64>::BW : BatchShape<float, 32>::BW)
               : (tw == 64 ? BatchShape<double, 64>::BW : BatchShape<double, 32>::BW);
}

template <typename T, int KIND, int TW>
__device__ __forceinline__ bool batch_item(const BatchGrid& G, const CUtensorMap* map, int m, int item,
                                           long long* ring, uint64_t* bars, uint32_t& seq, unsigned& mx,
                                           int* err)
{
    using S = BatchShape<T, TW>;
    constexpr int V = S::V, RT = kBatchRT, BW = S::BW, NST = kBatchNst, TY = S::TY, LPR = S::LPR;
    constexpr bool CONV = KIND == K_F64_XS;
    static_assert(!CONV || (V == 2 && 2 * TY <= 32), "the halo conversion roles below are FP64's");
    // stage words: fixed-point integers (exact-sum FP64), raw bits otherwise
    using Q = typename std::conditional<CONV, long long, T>::type;
    const HeatGeom& g = G.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int t = item % G.tiles_xy;
    const int kb = (item / G.tiles_xy) * G.kz, ke = min(kb + G.kz, g.nz);
    const int x0 = (t % G.tiles_x) * TW, y0 = (t / G.tiles_x) * TY;
    const int lx = tx % LPR, row0 = (ty * (32 / LPR) + tx / LPR) * RT;   // this thread's first row in the tile
    const int X = x0 + V * lx, Y0 = y0 + row0;
    const int xs = g.lead + x0 - S::D;                 // padded x of the box, 16-byte aligned
    const int own = (row0 + 1) * BW + S::D + V * lx;
    const int nx_ok = min(V, g.nx - X);
    const int emax = CONV ? xs_emax(G.fx, (G.m3 + m) % 3) : 0;
    const double r = G.r;
    const double r2 = CONV ? xs_r2(r, emax) : 0.0;
    T* __restrict__ dst = (T*)G.buf[((G.cur + m) & 1) ^ 1];
    // besides its own vectors: a halo-row vector (64-wide tiles: warps 0 and 1;
    // 32-wide: warp 0, half a warp per row) or a halo-column value (the next warp)
    int extra = -1;
    bool xvec = false;
    constexpr int HCW = TW == 64 ? 2 : 1;   // the warp that converts the halo columns
    if (ty < HCW) {
        const int hrow = TW == 64 ? (ty == 0 ? 0 : TY + 1) : (tx < LPR ? 0 : TY + 1);
        extra = hrow * BW + S::D + V * lx;
        xvec = true;
    } else if (ty == HCW && tx < 2 * TY) {
        extra = tx < TY ? (tx + 1) * BW + S::D - 1 : (tx - TY + 1) * BW + S::D + TW;
    }
    const int np = ke - kb + 2;   // planes kb-1 .. ke
    auto slot = [&](int sl) { return reinterpret_cast<Q*>(ring + sl * kBatchSlot); };
    bool bad = false;
    auto wait = [&](int sl, uint32_t ph) {
        if (!mbar_wait_bounded(&bars[sl], ph)) bad = true;
    };
    auto convert = [&](Q* pl, Q (&q)[RT][V], T (&raw)[RT][V]) {
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            ld_vec(reinterpret_cast<const T*>(pl) + own + j * BW, raw[j]);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if constexpr (CONV) q[j][i] = xs_fix(__double_as_longlong(raw[j][i]), emax);
                else q[j][i] = raw[j][i];
            }
            if constexpr (CONV) {
#pragma unroll
                for (int i = 0; i < V; ++i) pl[own + j * BW + i] = q[j][i];
            }
        }
        if constexpr (CONV) {
            if (xvec) {
                pl[extra] = xs_fix(pl[extra], emax);
                pl[extra + 1] = xs_fix(pl[extra + 1], emax);
            } else if (extra >= 0) {
                pl[extra] = xs_fix(pl[extra], emax);
            }
        }
    };

    const int s0 = (int)(seq % NST);
    const uint32_t ph0 = (seq / NST) & 1u;
    int issued = 0;
    if (tid == 0) {
        // the source planes were written by other blocks' generic stores, which
        // the step wait has made visible to this thread: order them before the
        // async-proxy loads
        asm volatile("fence.proxy.async.global;" ::: "memory");
        fence_proxy_async_smem();
        for (int sl = s0; issued < NST && issued < np; ++issued, sl = sl + 1 == NST ? 0 : sl + 1) {
            mbar_arrive_expect_tx(&bars[sl], S::BOX_BYTES);
            tma_load_3d(ring + sl * kBatchSlot, map, xs, y0, kb + issued, &bars[sl]);
        }
    }
    Q below[RT][V], cur[RT][V], above[RT][V];
    T craw[RT][V], araw[RT][V];
    int s_cur = s0;
    uint32_t ph_cur = ph0;
    wait(s_cur, ph_cur);
#pragma unroll
    for (int j = 0; j < RT; ++j) {
        T b[V];
        ld_vec(reinterpret_cast<const T*>(slot(s_cur)) + own + j * BW, b);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            if constexpr (CONV) below[j][i] = xs_fix(__double_as_longlong(b[i]), emax);
            else below[j][i] = b[i];
        }
    }
    if (++s_cur == NST) {
        s_cur = 0;
        ph_cur ^= 1u;
    }
    wait(s_cur, ph_cur);
    convert(slot(s_cur), cur, craw);
    if constexpr (CONV) fence_proxy_async_smem();
    bool aborted = __syncthreads_or(bad) != 0;

    T* out = dst + g.at(X < g.nx ? X : 0, 0, kb) + (int64_t)Y0 * g.pitch;   // used for rows inside the grid
    for (int k = kb; !aborted && k < ke; ++k) {
        const int s_nxt = s_cur + 1 == NST ? 0 : s_cur + 1;
        const uint32_t ph_nxt = s_nxt == 0 ? ph_cur ^ 1u : ph_cur;
        wait(s_nxt, ph_nxt);
        convert(slot(s_nxt), above, araw);
        const Q* pl = slot(s_cur) + own;
        Q ym[V], yp[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            ym[i] = pl[i - BW];
            yp[i] = pl[RT * BW + i];
        }
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            const Q left = pl[j * BW - 1], right = pl[j * BW + V];
            T v[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const Q xm = i == 0 ? left : cur[j][i - 1];
                const Q xp = i == V - 1 ? right : cur[j][i + 1];
                const Q yl = j == 0 ? ym[i] : cur[j - 1][i];
                const Q yh = j == RT - 1 ? yp[i] : cur[j + 1][i];
                if constexpr (CONV) {
                    const long long L = xs_numerator(cur[j][i], xm, xp, yl, yh, below[j][i], above[j][i]);
                    v[i] = (j == 0 && i == 0) ? xs_apply<true>(craw[j][i], L, r, r2, emax)
                                              : xs_apply<false>(craw[j][i], L, r, r2, emax);
                } else {
                    v[i] = Point<T, false>::update(cur[j][i], xm, xp, yl, yh, below[j][i], above[j][i], (T)r, 0);
                }
            }
            const int nvalid = Y0 + j < g.ny ? nx_ok : 0;
            T* o = out + j * g.pitch;
            if (nvalid == V) {
                st_vec(o, v);
            } else {
#pragma unroll
                for (int i = 0; i < V - 1; ++i)
                    if (i < nvalid) o[i] = v[i];
            }
            if constexpr (KIND == K_F64_XS || KIND == K_F64_XS_NATIVE) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const unsigned a = i < nvalid ? xs_abs_hi((double)v[i]) : 0u;
                    mx = a > mx ? a : mx;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < RT; ++j)
#pragma unroll
            for (int i = 0; i < V; ++i) {
                below[j][i] = cur[j][i];
                cur[j][i] = above[j][i];
                craw[j][i] = araw[j][i];
            }
        out += g.plane;
        if constexpr (CONV) fence_proxy_async_smem();
        aborted = __syncthreads_or(bad) != 0;
        // the slot of plane k-1 is free: every thread is past its last use
        if (!aborted && tid == 0 && issued < np) {
            const int sl = s_cur == 0 ? NST - 1 : s_cur - 1;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[sl], S::BOX_BYTES);
            tma_load_3d(ring + sl * kBatchSlot, map, xs, y0, kb + issued, &bars[sl]);
            ++issued;
        }
        s_cur = s_nxt;
        ph_cur = ph_nxt;
    }
    if (aborted && tid == 0) {
        // the last load issued into each slot, consumed or not, completes
        // before the block may end or reuse the ring
        atomicMax(err, 1);
        const long long t0 = clock64();   // one time budget for the whole drain
        for (int j = issued > NST ? issued - NST : 0; j < issued; ++j)
            if (!mbar_wait_until(&bars[(seq + j) % NST], ((seq + j) / NST) & 1u, t0, kWaitCycles)) {
                atomicMax(err, 2);   // loads may still be landing: the context is suspect
                break;
            }
    }
    seq += (uint32_t)np;
    return !aborted;
}

template <int TW>
__device__ __forceinline__ bool batch_dispatch(const BatchGrid& G, const CUtensorMap* map, int m, int t,
                                               long long* ring, uint64_t* bars, uint32_t& seq, unsigned& mx,
                                               int* err)
{
    if (G.kind == K_F64_XS)   // fields outside the convertible exponent range take the FP64 pipe
        return xs_native(xs_emax(G.fx, (G.m3 + m) % 3), G.r)
                   ? batch_item<double, K_F64_XS_NATIVE, TW>(G, map, m, t, ring, bars, seq, mx, err)
                   : batch_item<double, K_F64_XS, TW>(G, map, m, t, ring, bars, seq, mx, err);
    if (G.kind == K_F64_PIPE) return batch_item<double, K_F64_PIPE, TW>(G, map, m, t, ring, bars, seq, mx, err);
    return batch_item<float, K_F32, TW>(G, map, m, t, ring, bars, seq, mx, err);
}

__global__ void __launch_bounds__(32 * kBatchTY, 8) k_heat_batch(BatchDev B)
{
    __shared__ __align__(128) long long ring[kBatchNst * kBatchSlot];
    __shared__ __align__(8) uint64_t bars[kBatchNst];
    __shared__ long long s_item;
    __shared__ int s_abort;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (tid == 0) {
        for (int sl = 0; sl < kBatchNst; ++sl) mbar_init(&bars[sl], 1);
        fence_mbar_init();
    }
    uint32_t seq = 0;   // planes this block has staged through the ring
    for (;;) {
        if (tid == 0) {
            s_abort = *(volatile int*)B.err;
            s_item = s_abort ? B.items : (long long)atomicAdd(B.next, 1ull);
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= B.items) break;
        const unsigned long long desc = __ldg(B.sched + item);
        const int m = (int)(desc >> 40);
        const int gi = (int)((desc >> 24) & 0xffffu);
        const int t = (int)(desc & 0xffffffu);
        const BatchGrid& G = B.grids[gi];
        if (tid == 0 && m > 0) {
            // wait until step m-1 of this grid is complete
            const unsigned long long need = (unsigned long long)m * (unsigned long long)G.tiles;
            const long long t0 = clock64();
            while (*(volatile unsigned long long*)&B.done[gi] < need) {
                if (clock64() - t0 > B.wait_cycles) {
                    atomicExch(B.err, 1);
                    s_abort = 1;
                    break;
                }
            }
            __threadfence();
        }
        __syncthreads();
        if (s_abort) break;
        // the map of this step's source buffer
        const CUtensorMap* map = B.maps + 2 * gi + ((G.cur + m) & 1);
        unsigned mx = 0;
        const bool ok = G.tw == 64 ? batch_dispatch<64>(G, map, m, t, ring, bars, seq, mx, B.err)
                                   : batch_dispatch<32>(G, map, m, t, ring, bars, seq, mx, B.err);
        if (ok && G.kind == K_F64_XS)
            fx_finish<32 * kBatchTY>((unsigned long long)mx << 32, G.fx, (G.m3 + m) % 3, 0, t == 0);
        if (!ok) break;   // the same in every thread
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(&B.done[gi], 1ull);
    }
}

}  // namespace hcg

using namespace hcg;

namespace {

// Planes per work item when the caller leaves it to the library: chunks of 32
// planes.  A grid's step may start only when its previous step is complete,
// so the time one item takes bounds how fast a grid's chain of steps can go;
// 32-plane chunks measured fastest on the 256-grid workload (ahead of whole
// columns by 1.5x and of 16-plane chunks).
int batch_default_kz(const HeatGeom& g, int)
{
    return g.nz < 32 ? g.nz : 32;
}

// Tile width when the caller leaves it to the library: the one that stages
// fewer values per plane (tiles with their halo rows and columns), so narrow
// grids do not leave half of every warp idle.
int batch_default_tw(const HeatGeom& g, bool f32)
{
    auto staged = [&](int tw) {
        const int ty = batch_tile_rows(tw, f32);
        return (int64_t)((g.nx + tw - 1) / tw) * ((g.ny + ty - 1) / ty) * batch_stage_row(tw, f32) * (ty + 2);
    };
    return staged(32) < staged(64) ? 32 : 64;
}

}  // namespace

struct hs_batch {
    cudaStream_t stream;
    std::vector<hs_heat_t> handles;
    std::vector<int64_t> steps;
    BatchDev dev;
    void* arena;          // device: grids, schedule, counters
    size_t counter_bytes;
    void* counters;       // next + done[] + err (cleared before each run)
    int blocks;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaStream_t capture;   // private stream the graph is captured on
    int64_t lups;
};

extern "C" {

int heat_batch_destroy(hs_batch_t b)
{
    if (!b) return HS_OK;
    int rc = HS_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "heat_batch_destroy: synchronize");
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    dev_free(b->arena, b->stream);
    delete b;
    return rc;
}

int heat_batch_create(hs_batch_t* out, const hs_heat_t* grids, const int64_t* steps, int32_t n,
                      void* stream)
{
    return heat_batch_create_tiled(out, grids, steps, nullptr, nullptr, n, stream);
}

int heat_batch_create_tiled(hs_batch_t* out, const hs_heat_t* grids, const int64_t* steps,
                            const int32_t* kz, const int32_t* tw, int32_t n, void* stream)
{
    if (!out) return fail(HS_EINVAL, "heat_batch_create: out is NULL");
    *out = nullptr;
    if (!grids || !steps || n < 1) return fail(HS_EINVAL, "heat_batch_create: no grids");
    std::vector<BatchGrid> hg((size_t)n);
    int64_t max_steps = 0;
    int64_t lups = 0;
    for (int32_t i = 0; i < n; ++i) {
        const hs_heat_t h = grids[i];
        if (!h) return fail(HS_EINVAL, "heat_batch_create: grid %d is NULL", i);
        if (steps[i] < 0) return fail(HS_EINVAL, "heat_batch_create: steps[%d] < 0", i);
        HeatBatchView v;
        int rc = heat_batch_view(h, &v);
        if (rc != HS_OK) return rc;
        if ((v.arith != A_F64 && v.arith != A_F64_XS && v.arith != A_F32) || v.vk)
            return fail(HS_EINVAL, "heat_batch_create: grid %d must be plain FP64 or FP32", i);
        for (int32_t k = 0; k < i; ++k)
            if (grids[k] == h) return fail(HS_EINVAL, "heat_batch_create: grid %d appears twice", i);
        BatchGrid& G = hg[(size_t)i];
        G.g = v.g;
        G.buf[0] = v.buf[0];
        G.buf[1] = v.buf[1];
        G.r = v.r;
        G.kind = v.arith == A_F64 ? K_F64_PIPE : v.arith == A_F64_XS ? K_F64_XS : K_F32;
        G.fx = v.fx;
        G.cur = 0;   // cur and m3 are set at each run
        G.m3 = 0;
        if (tw && tw[i] != 0 && tw[i] != 32 && tw[i] != 64)
            return fail(HS_EINVAL, "heat_batch_create: tile width %d of grid %d is not 0, 32 or 64", tw[i], i);
        const bool f32 = G.kind == K_F32;
        G.tw = (tw && tw[i]) ? tw[i] : batch_default_tw(v.g, f32);
        G.pad = 0;
        G.tiles_x = (v.g.nx + G.tw - 1) / G.tw;
        const int tyr = batch_tile_rows(G.tw, f32);
        G.tiles_xy = G.tiles_x * ((v.g.ny + tyr - 1) / tyr);
        if (kz && kz[i] < 0) return fail(HS_EINVAL, "heat_batch_create: kz[%d] < 0", i);
        G.kz = (kz && kz[i]) ? std::min(kz[i], v.g.nz) : batch_default_kz(v.g, G.tiles_xy);
        G.tiles = G.tiles_xy * ((v.g.nz + G.kz - 1) / G.kz);
        G.steps = steps[i];
        if (steps[i] > max_steps) max_steps = steps[i];
        lups += (int64_t)v.g.nx * v.g.ny * v.g.nz * steps[i];
    }
    if (max_steps > (1 << 30)) return fail(HS_EINVAL, "heat_batch_create: too many steps");
    // step-major schedule: one descriptor per item
    if (max_steps >= (1 << 24) || n > 0xffff)
        return fail(HS_EINVAL, "heat_batch_create: at most 2^24 - 1 steps and 65535 grids");
    int64_t items = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (hg[(size_t)i].tiles >= (1 << 24)) return fail(HS_EINVAL, "heat_batch_create: grid %d too large", i);
        items += (int64_t)hg[(size_t)i].tiles * hg[(size_t)i].steps;
    }
    if (items > ((int64_t)1 << 28))
        return fail(HS_EINVAL, "heat_batch_create: %lld work items exceed the schedule limit 2^28",
                    (long long)items);
    std::vector<unsigned long long> sched;
    try {
        sched.reserve((size_t)items);
    } catch (...) {
        return fail(HS_ENOMEM, "heat_batch_create: host allocation failed");
    }
    // Stretched order: step m of a grid of S steps goes in round
    // floor(m * max_steps / S), so every grid advances throughout the run and
    // all finish together -- the longest chains of steps never run alone at
    // the end.  Consecutive steps of a grid land in increasing rounds (S <=
    // max_steps), so every item comes after the items it waits for.
    {
        std::vector<std::pair<int64_t, int64_t>> order;   // (round, grid << 32 | step)
        order.reserve((size_t)(max_steps > 0 ? max_steps : 1) * (size_t)n / 2 + 16);
        for (int32_t i = 0; i < n; ++i) {
            const int64_t S = hg[(size_t)i].steps;
            for (int64_t mm = 0; mm < S; ++mm)
                order.emplace_back(mm * max_steps / S, ((int64_t)i << 32) | mm);
        }
        std::stable_sort(order.begin(), order.end(),
                         [](const std::pair<int64_t, int64_t>& a, const std::pair<int64_t, int64_t>& b) {
                             return a.first < b.first;
                         });
        for (const auto& o : order) {
            const int32_t i = (int32_t)(o.second >> 32);
            const int64_t mm = o.second & 0xffffffffll;
            const unsigned long long base = ((unsigned long long)mm << 40) | ((unsigned long long)i << 24);
            for (int32_t t = 0; t < hg[(size_t)i].tiles; ++t) sched.push_back(base | (unsigned long long)t);
        }
    }
    hs_batch* b = new (std::nothrow) hs_batch();
    if (!b) return fail(HS_ENOMEM, "heat_batch_create: host allocation failed");
    b->stream = (cudaStream_t)stream;
    b->handles.assign(grids, grids + n);
    b->steps.assign(steps, steps + n);
    b->lups = lups;
    // TMA maps of every grid's two buffers, boxes of one tile plane with its halo
    std::vector<CUtensorMap> maps(2 * (size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        const BatchGrid& G = hg[(size_t)i];
        const bool f32 = G.kind == K_F32;
        const uint32_t bx = (uint32_t)batch_stage_row(G.tw, f32);
        const uint32_t by = (uint32_t)batch_tile_rows(G.tw, f32) + 2;
        for (int bi = 0; bi < 2; ++bi) {
            const int e = encode_field_map(&maps[2 * (size_t)i + bi], G.buf[bi],
                                           f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                           f32 ? sizeof(float) : sizeof(double), (uint64_t)G.g.pitch,
                                           (uint64_t)(G.g.ny + 2), (uint64_t)(G.g.nz + 2), bx, by);
            if (e != 0) return cuda_fail((cudaError_t)e, "heat_batch_create: TMA tensor map");
        }
    }
    // one arena: maps | grids | schedule | counters (maps first: 128-byte aligned)
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t s_maps = align(sizeof(CUtensorMap) * maps.size());
    const size_t s_grids = align(sizeof(BatchGrid) * hg.size());
    const size_t s_sched = align(sizeof(unsigned long long) * (sched.size() ? sched.size() : 1));
    b->counter_bytes = align(sizeof(unsigned long long) * (1 + (size_t)n) + sizeof(int));
    const size_t total = s_maps + s_grids + s_sched + b->counter_bytes;
    cudaError_t e = dev_alloc(&b->arena, total, b->stream);
    if (e != cudaSuccess) {
        b->arena = nullptr;
        const int rc = cuda_fail(e, "heat_batch_create: device allocation");
        heat_batch_destroy(b);
        return rc;
    }
    CUtensorMap* d_maps = (CUtensorMap*)b->arena;
    char* base = (char*)b->arena + s_maps;
    BatchGrid* d_grids = (BatchGrid*)base;
    unsigned long long* d_sched = (unsigned long long*)(base + s_grids);
    b->counters = base + s_grids + s_sched;
    // grids are re-uploaded at each run (cur changes); the schedule once.  The
    // arena is ordered on the batch stream, so the copies are too (and finish
    // before the host arrays go away).
    const cudaStream_t bs = b->stream;
    e = cudaSuccess;
    if (!sched.empty())
        e = cudaMemcpyAsync(d_sched, sched.data(), sizeof(unsigned long long) * sched.size(),
                            cudaMemcpyHostToDevice, bs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_grids, hg.data(), sizeof(BatchGrid) * hg.size(), cudaMemcpyHostToDevice, bs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice, bs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "heat_batch_create: schedule upload");
        heat_batch_destroy(b);
        return rc;
    }
    unsigned long long* ctr = (unsigned long long*)b->counters;
    b->dev.grids = d_grids;
    b->dev.sched = d_sched;
    b->dev.maps = d_maps;
    b->dev.next = ctr;
    b->dev.done = ctr + 1;
    b->dev.err = (int*)(ctr + 1 + n);
    b->dev.items = items;
    b->dev.wait_cycles = g_batch_wait_cycles.load();
    // persistent grid: every block resident at once
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heat_batch, 32 * kBatchTY, 0);
    int sms = kNumSMs;
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || per_sm < 1) {
        const int rc = cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidConfiguration,
                                 "heat_batch_create: occupancy");
        heat_batch_destroy(b);
        return rc;
    }
    b->blocks = per_sm * sms;
    *out = b;
    return HS_OK;
}

// Enqueue: refresh each grid's current buffer, clear the counters, launch.
static int batch_enqueue(hs_batch* b)
{
    const int n = (int)b->handles.size();
    std::vector<BatchGrid> hg((size_t)n);
    HS_TRY_CUDA(cudaMemcpyAsync(hg.data(), b->dev.grids, sizeof(BatchGrid) * n, cudaMemcpyDeviceToHost, b->stream),
                "heat_batch_run: grid table");
    HS_TRY_CUDA(cudaStreamSynchronize(b->stream), "heat_batch_run: grid table");
    bool changed = false;
    for (int i = 0; i < n; ++i) {
        HeatBatchView v;
        int rc = heat_batch_view(b->handles[(size_t)i], &v);
        if (rc != HS_OK) return rc;
        // the grid's own stream may still be uploading into it
        if (v.stream != b->stream)
            HS_TRY_CUDA(cudaStreamSynchronize(v.stream), "heat_batch_run: grid stream");
        if (hg[(size_t)i].cur != v.cur || hg[(size_t)i].m3 != v.m3) {
            hg[(size_t)i].cur = v.cur;
            hg[(size_t)i].m3 = v.m3;
            changed = true;
        }
    }
    if (changed)
        HS_TRY_CUDA(cudaMemcpyAsync((void*)b->dev.grids, hg.data(), sizeof(BatchGrid) * n,
                                    cudaMemcpyHostToDevice, b->stream),
                    "heat_batch_run: grid table");
    HS_TRY_CUDA(cudaStreamSynchronize(b->stream), "heat_batch_run: synchronize");
    return changed ? 1 : 0;
}

int heat_batch_run(hs_batch_t b, int use_graph)
{
    if (!b) return fail(HS_EINVAL, "heat_batch_run: NULL batch");
    int rc = batch_enqueue(b);
    if (rc < 0) return rc;
    if (use_graph) {
        if (!b->exec) {
            // capture on a private stream (the caller's may be the legacy
            // default stream, which cannot be captured); launch on the caller's
            if (!b->capture)
                HS_TRY_CUDA(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking),
                            "heat_batch_run: capture stream");
            HS_TRY_CUDA(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal),
                        "heat_batch_run: begin capture");
            cudaError_t e1 = cudaMemsetAsync(b->counters, 0, b->counter_bytes, b->capture);
            k_heat_batch<<<b->blocks, dim3(32, kBatchTY), 0, b->capture>>>(b->dev);
            cudaError_t e2 = cudaPeekAtLastError();
            cudaGraph_t graph = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(b->capture, &graph);
            if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
                (void)cudaGetLastError();
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3,
                                 "heat_batch_run: capture");
            }
            b->graph = graph;
            HS_TRY_CUDA(cudaGraphInstantiate(&b->exec, graph, 0), "heat_batch_run: instantiate");
        }
        HS_TRY_CUDA(cudaGraphLaunch(b->exec, b->stream), "heat_batch_run: graph launch");
        count_launch();
    } else {
        HS_TRY_CUDA(cudaMemsetAsync(b->counters, 0, b->counter_bytes, b->stream), "heat_batch_run: memset");
        k_heat_batch<<<b->blocks, dim3(32, kBatchTY), 0, b->stream>>>(b->dev);
        HS_CHECK_LAUNCH("heat batch kernel");
    }
    // every grid advanced by its steps: update the handles' bookkeeping
    for (size_t i = 0; i < b->handles.size(); ++i) {
        rc = heat_batch_advance(b->handles[i], b->steps[i]);
        if (rc != HS_OK) return rc;
    }
    return HS_OK;
}

int heat_batch_wait(hs_batch_t b)
{
    if (!b) return fail(HS_EINVAL, "heat_batch_wait: NULL batch");
    int err = 0;
    HS_TRY_CUDA(cudaMemcpyAsync(&err, b->dev.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
                "heat_batch_wait: status");
    HS_TRY_CUDA(cudaStreamSynchronize(b->stream), "heat_batch_wait: synchronize");
    if (err) return fail(HS_ETIMEOUT, "heat_batch_wait: a bounded wait in the batch kernel ran out");
    return HS_OK;
}

int heat_batch_set_wait_limit(int64_t cycles)
{
    if (cycles < 0) return fail(HS_EINVAL, "heat_batch_set_wait_limit: cycles < 0");
    g_batch_wait_cycles.store(cycles ? (long long)cycles : kBatchWaitCycles);
    return HS_OK;
}

int heat_batch_info(hs_batch_t b, int64_t* lups, int32_t* blocks)
{
    if (!b) return fail(HS_EINVAL, "heat_batch_info: NULL batch");
    if (lups) *lups = b->lups;
    if (blocks) *blocks = b->blocks;
    return HS_OK;
}

}  // extern "C"
