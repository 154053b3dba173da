// Batched heat stepping: many independent grids (their own sizes, r, step
// counts, FP32 or FP64), every step of every grid, in ONE persistent kernel
// launch, optionally replayed from a captured CUDA graph.
//
// Work items are (step m, grid g, column tile, chunk of planes) in step-major
// order; a persistent grid of co-resident blocks takes them from an atomic
// counter.
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

namespace hcg {

constexpr int kBatchBX = 32, kBatchBY = 8;
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
    int64_t steps;
};

struct BatchDev {
    const BatchGrid* grids;
    const int64_t* step_item0;    // first item of step m (size max_steps + 1)
    const int32_t* step_list0;    // first entry of step m in the active lists (size max_steps + 1)
    const int32_t* list_grid;     // active grid of each entry
    const int64_t* list_item0;    // first item (within its step) of each entry
    unsigned long long* next;     // work counter
    unsigned long long* done;     // per grid: items completed, all steps
    int* err;
    int64_t items;
    long long wait_cycles;        // limit of the step wait, in SM clock cycles
    int32_t max_steps;
};

// One work item of step m -- a column tile and a chunk [kb, ke) of its planes:
// a block of 32 x 8 threads owns a 64 x 8 tile of the grid's columns and
// marches up the chunk's planes, every thread two
// consecutive x points of one row.  Each plane of the tile with its one-point
// halo is loaded once with coalesced L2 loads two planes ahead of use (kept in
// registers), converted once (exact-sum FP64: to fixed point on the field's
// scale; otherwise kept as is) into one of two shared plane buffers; a thread
// keeps its own values at k-1, k and k+1 in registers, reads the in-plane
// neighbours from the buffer of plane k, and one block barrier per plane
// orders the buffers.  Positions past the grid's boundary layer (x > nx,
// y > ny, possible in the last tiles) are never loaded: they hold zeros and
// feed no output.  The per-point arithmetic is that of heat_step, so the
// result matches the grid stepped alone bit for bit.  Returns the largest
// |u| high word of the outputs (exact-sum FP64 only).
constexpr int kBatchTW = 64, kBatchBW = 68, kBatchD = 2;   // tile width, buffer row, x offset
constexpr int kBatchPlane = (kBatchBY + 2) * kBatchBW;     // buffer elements per plane
static_assert(kBatchBX * 2 == kBatchTW, "two points per thread");

template <typename T>
__device__ __forceinline__ void st_pair(T* p, const T (&v)[2])
{
    if constexpr (sizeof(T) == 8)
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    else
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}

template <typename T, int KIND>
__device__ __forceinline__ unsigned batch_tile(const BatchGrid& G, int m, int item, long long* sbuf)
{
    constexpr int V = 2, BW = kBatchBW;
    constexpr bool CONV = KIND == K_F64_XS;
    // shared values: fixed-point integers (exact-sum FP64), raw bits otherwise
    using Q = typename std::conditional<CONV, long long, T>::type;
    Q* buf = reinterpret_cast<Q*>(sbuf);
    const HeatGeom& g = G.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kBatchBX + tx;
    const int t = item % G.tiles_xy;
    const int kb = (item / G.tiles_xy) * G.kz, ke = min(kb + G.kz, g.nz);
    const int x0 = (t % G.tiles_x) * kBatchTW, y0 = (t / G.tiles_x) * kBatchBY;
    const int X = x0 + V * tx, Y = y0 + ty;
    const int own = (ty + 1) * BW + kBatchD + V * tx;
    const int emax = CONV ? xs_emax(G.fx, (G.m3 + m) % 3) : 0;
    const double r = G.r;
    const double r2 = CONV ? xs_r2(r, emax) : 0.0;
    const int src_b = (G.cur + m) & 1;
    const T* __restrict__ src = (const T*)G.buf[src_b];
    T* __restrict__ dst = (T*)G.buf[src_b ^ 1];
    // own points: loaded where they lie in the padded buffer (y <= ny, x <= nx
    // reach the boundary layer), computed and stored where interior
    const bool ld0 = Y <= g.ny && X <= g.nx, ld1 = Y <= g.ny && X + 1 <= g.nx;
    const bool ok0 = Y < g.ny && X < g.nx, ok1 = Y < g.ny && X + 1 < g.nx;
    const int64_t rowoff = g.at(X, Y, -1);   // plane k adds (k + 1) plane
    // one halo value per thread for the first 2*64 + 2*8 threads
    int hidx = -1;
    int64_t hoff = 0;
    bool hld = false;
    if (tid < 2 * kBatchTW) {
        const int rr = tid < kBatchTW ? 0 : kBatchBY + 1;
        const int c = tid % kBatchTW;
        const int hx = x0 + c, hy = rr == 0 ? y0 - 1 : y0 + kBatchBY;
        hidx = rr * BW + kBatchD + c;
        hld = hx <= g.nx && hy <= g.ny;
        hoff = g.at(hx, hy, -1);
    } else if (tid < 2 * kBatchTW + 2 * kBatchBY) {
        const int u = tid - 2 * kBatchTW;
        const int rr = 1 + u % kBatchBY;
        const bool right = u >= kBatchBY;
        const int hx = right ? x0 + kBatchTW : x0 - 1, hy = y0 + rr - 1;
        hidx = rr * BW + (right ? kBatchD + kBatchTW : kBatchD - 1);
        hld = hx <= g.nx && hy <= g.ny;
        hoff = g.at(hx, hy, -1);
    }
    auto ld_own = [&](int k, T (&o)[V]) {   // k in [-1, nz]: boundary planes included
        const T* p = src + rowoff + (int64_t)(k + 1) * g.plane;
        o[0] = ld0 ? __ldcg(p) : T(0);
        o[1] = ld1 ? __ldcg(p + 1) : T(0);
    };
    auto ld_halo = [&](int k) -> T { return hld ? __ldcg(src + hoff + (int64_t)(k + 1) * g.plane) : T(0); };
    auto fix = [&](T v) -> Q {
        if constexpr (CONV) return xs_fix(__double_as_longlong(v), emax);
        else return v;
    };

    Q below[V], cur[V], above[V];
    T craw[V], araw[V], nown[V], tt[V];
    ld_own(kb - 1, tt);
    below[0] = fix(tt[0]);
    below[1] = fix(tt[1]);
    ld_own(kb, tt);
    craw[0] = tt[0];
    craw[1] = tt[1];
    cur[0] = fix(tt[0]);
    cur[1] = fix(tt[1]);
    {
        Q* b0 = buf + (kb & 1) * kBatchPlane;
        b0[own] = cur[0];
        b0[own + 1] = cur[1];
        if (hidx >= 0) b0[hidx] = fix(ld_halo(kb));
    }
    ld_own(kb + 1, araw);
    T h1 = ld_halo(kb + 1), nh = T(0);
    nown[0] = T(0);
    nown[1] = T(0);
    if (kb + 2 <= ke) {
        ld_own(kb + 2, nown);
        nh = ld_halo(kb + 2);
    }
    above[0] = fix(araw[0]);
    above[1] = fix(araw[1]);
    __syncthreads();

    unsigned mx = 0;
    T* out = dst + rowoff + (int64_t)(kb + 1) * g.plane;   // plane kb
    for (int k = kb; k < ke; ++k) {
        Q* bn = buf + ((k + 1) & 1) * kBatchPlane;   // plane k+1, read in the next iteration
        bn[own] = above[0];
        bn[own + 1] = above[1];
        if (hidx >= 0) bn[hidx] = fix(h1);
        const Q* pc = buf + (k & 1) * kBatchPlane + own;
        const Q ym0 = pc[-BW], ym1 = pc[1 - BW], yp0 = pc[BW], yp1 = pc[1 + BW];
        const Q left = pc[-1], right = pc[V];
        T v[V];
        if constexpr (CONV) {
            const long long L0 = xs_numerator(cur[0], left, cur[1], ym0, yp0, below[0], above[0]);
            const long long L1 = xs_numerator(cur[1], cur[0], right, ym1, yp1, below[1], above[1]);
            v[0] = xs_apply<true>(craw[0], L0, r, r2, emax);
            v[1] = xs_apply<false>(craw[1], L1, r, r2, emax);
            const unsigned a0 = ok0 ? xs_abs_hi(v[0]) : 0u, a1 = ok1 ? xs_abs_hi(v[1]) : 0u;
            mx = max(mx, max(a0, a1));
        } else {
            const T rr = (T)r;
            v[0] = Point<T, false>::update(cur[0], left, cur[1], ym0, yp0, below[0], above[0], rr, 0);
            v[1] = Point<T, false>::update(cur[1], cur[0], right, ym1, yp1, below[1], above[1], rr, 0);
            if constexpr (KIND == K_F64_XS_NATIVE) {
                const unsigned a0 = ok0 ? xs_abs_hi(v[0]) : 0u, a1 = ok1 ? xs_abs_hi(v[1]) : 0u;
                mx = max(mx, max(a0, a1));
            }
        }
        if (ok1) {
            st_pair(out, v);
        } else if (ok0) {
            out[0] = v[0];
        }
        out += g.plane;
        below[0] = cur[0];
        below[1] = cur[1];
        cur[0] = above[0];
        cur[1] = above[1];
        craw[0] = araw[0];
        craw[1] = araw[1];
        araw[0] = nown[0];
        araw[1] = nown[1];
        above[0] = fix(nown[0]);
        above[1] = fix(nown[1]);
        h1 = nh;
        if (k + 3 <= ke) {
            ld_own(k + 3, nown);
            nh = ld_halo(k + 3);
        }
        __syncthreads();
    }
    return mx;
}

__global__ void __launch_bounds__(kBatchBX* kBatchBY, 4) k_heat_batch(BatchDev B)
{
    __shared__ __align__(16) long long sbuf[2 * kBatchPlane];
    __shared__ long long s_item;
    __shared__ int s_abort;
    const int tid = threadIdx.y * kBatchBX + threadIdx.x;
    for (;;) {
        if (tid == 0) {
            s_abort = *(volatile int*)B.err;
            s_item = s_abort ? B.items : (long long)atomicAdd(B.next, 1ull);
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= B.items) break;
        // step m: the last m with step_item0[m] <= item
        int lo = 0, hi = B.max_steps - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.step_item0[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int m = lo;
        const long long in_step = item - B.step_item0[m];
        int a = B.step_list0[m], z = B.step_list0[m + 1] - 1;
        while (a < z) {
            const int mid = (a + z + 1) >> 1;
            if (B.list_item0[mid] <= in_step) a = mid; else z = mid - 1;
        }
        const int gi = B.list_grid[a];
        const BatchGrid& G = B.grids[gi];
        const int t = (int)(in_step - B.list_item0[a]);
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
        if (G.kind == K_F64_XS) {
            // fields outside the convertible exponent range take the FP64 pipe
            const unsigned mx = xs_native(xs_emax(G.fx, (G.m3 + m) % 3), G.r)
                                    ? batch_tile<double, K_F64_XS_NATIVE>(G, m, t, sbuf)
                                    : batch_tile<double, K_F64_XS>(G, m, t, sbuf);
            fx_finish<kBatchBX * kBatchBY>((unsigned long long)mx << 32, G.fx, (G.m3 + m) % 3, 0, t == 0);
        } else if (G.kind == K_F64_PIPE) {
            batch_tile<double, K_F64_PIPE>(G, m, t, sbuf);
        } else {
            batch_tile<float, K_F32>(G, m, t, sbuf);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(&B.done[gi], 1ull);
    }
}

}  // namespace hcg

using namespace hcg;

namespace {

// Planes per work item when the caller leaves it to the library: a grid with
// few column tiles splits each step into z-chunks of at least 16 planes, so
// that about 16 items share a step and the chain of its steps (each waits for
// the one before) does not hang on one block marching the whole column.
int batch_default_kz(const HeatGeom& g, int tiles_xy)
{
    const int want = 16;
    if (tiles_xy >= want) return g.nz;
    const int chunks = (want + tiles_xy - 1) / tiles_xy;
    int kz = (g.nz + chunks - 1) / chunks;
    if (kz < 16) kz = 16;
    return kz < g.nz ? kz : g.nz;
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
    return heat_batch_create_tiled(out, grids, steps, nullptr, n, stream);
}

int heat_batch_create_tiled(hs_batch_t* out, const hs_heat_t* grids, const int64_t* steps,
                            const int32_t* kz, int32_t n, void* stream)
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
        G.tiles_x = (v.g.nx + kBatchTW - 1) / kBatchTW;
        G.tiles_xy = G.tiles_x * ((v.g.ny + kBatchBY - 1) / kBatchBY);
        if (kz && kz[i] < 0) return fail(HS_EINVAL, "heat_batch_create: kz[%d] < 0", i);
        G.kz = (kz && kz[i]) ? std::min(kz[i], v.g.nz) : batch_default_kz(v.g, G.tiles_xy);
        G.tiles = G.tiles_xy * ((v.g.nz + G.kz - 1) / G.kz);
        G.steps = steps[i];
        if (steps[i] > max_steps) max_steps = steps[i];
        lups += (int64_t)v.g.nx * v.g.ny * v.g.nz * steps[i];
    }
    if (max_steps > (1 << 30)) return fail(HS_EINVAL, "heat_batch_create: too many steps");
    // step-major schedule
    std::vector<int64_t> step_item0((size_t)max_steps + 1, 0);
    std::vector<int32_t> step_list0((size_t)max_steps + 1, 0);
    std::vector<int32_t> list_grid;
    std::vector<int64_t> list_item0;
    int64_t items = 0;
    for (int64_t m = 0; m < max_steps; ++m) {
        step_item0[(size_t)m] = items;
        step_list0[(size_t)m] = (int32_t)list_grid.size();
        int64_t in_step = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (hg[(size_t)i].steps <= m) continue;
            list_grid.push_back(i);
            list_item0.push_back(in_step);
            in_step += hg[(size_t)i].tiles;
        }
        items += in_step;
    }
    step_item0[(size_t)max_steps] = items;
    step_list0[(size_t)max_steps] = (int32_t)list_grid.size();
    if (list_grid.size() > (size_t)INT32_MAX) return fail(HS_EINVAL, "heat_batch_create: schedule too large");

    hs_batch* b = new (std::nothrow) hs_batch();
    if (!b) return fail(HS_ENOMEM, "heat_batch_create: host allocation failed");
    b->stream = (cudaStream_t)stream;
    b->handles.assign(grids, grids + n);
    b->steps.assign(steps, steps + n);
    b->lups = lups;
    // one arena: grids | step_item0 | list_item0 | step_list0 | list_grid | counters
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t s_grids = align(sizeof(BatchGrid) * hg.size());
    const size_t s_si = align(sizeof(int64_t) * step_item0.size());
    const size_t s_li = align(sizeof(int64_t) * (list_item0.size() ? list_item0.size() : 1));
    const size_t s_sl = align(sizeof(int32_t) * step_list0.size());
    const size_t s_lg = align(sizeof(int32_t) * (list_grid.size() ? list_grid.size() : 1));
    b->counter_bytes = align(sizeof(unsigned long long) * (1 + (size_t)n) + sizeof(int));
    const size_t total = s_grids + s_si + s_li + s_sl + s_lg + b->counter_bytes;
    cudaError_t e = dev_alloc(&b->arena, total, b->stream);
    if (e != cudaSuccess) {
        b->arena = nullptr;
        const int rc = cuda_fail(e, "heat_batch_create: device allocation");
        heat_batch_destroy(b);
        return rc;
    }
    char* base = (char*)b->arena;
    BatchGrid* d_grids = (BatchGrid*)base;
    int64_t* d_si = (int64_t*)(base + s_grids);
    int64_t* d_li = (int64_t*)(base + s_grids + s_si);
    int32_t* d_sl = (int32_t*)(base + s_grids + s_si + s_li);
    int32_t* d_lg = (int32_t*)(base + s_grids + s_si + s_li + s_sl);
    b->counters = base + s_grids + s_si + s_li + s_sl + s_lg;
    // grids are re-uploaded at each run (cur changes); the schedule once.  The
    // arena is ordered on the batch stream, so the copies are too (and finish
    // before the host arrays go away).
    const cudaStream_t bs = b->stream;
    e = cudaMemcpyAsync(d_si, step_item0.data(), sizeof(int64_t) * step_item0.size(), cudaMemcpyHostToDevice, bs);
    if (e == cudaSuccess && !list_item0.empty())
        e = cudaMemcpyAsync(d_li, list_item0.data(), sizeof(int64_t) * list_item0.size(), cudaMemcpyHostToDevice,
                            bs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_sl, step_list0.data(), sizeof(int32_t) * step_list0.size(), cudaMemcpyHostToDevice,
                            bs);
    if (e == cudaSuccess && !list_grid.empty())
        e = cudaMemcpyAsync(d_lg, list_grid.data(), sizeof(int32_t) * list_grid.size(), cudaMemcpyHostToDevice, bs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_grids, hg.data(), sizeof(BatchGrid) * hg.size(), cudaMemcpyHostToDevice, bs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "heat_batch_create: schedule upload");
        heat_batch_destroy(b);
        return rc;
    }
    unsigned long long* ctr = (unsigned long long*)b->counters;
    b->dev.grids = d_grids;
    b->dev.step_item0 = d_si;
    b->dev.step_list0 = d_sl;
    b->dev.list_grid = d_lg;
    b->dev.list_item0 = d_li;
    b->dev.next = ctr;
    b->dev.done = ctr + 1;
    b->dev.err = (int*)(ctr + 1 + n);
    b->dev.items = items;
    b->dev.wait_cycles = g_batch_wait_cycles.load();
    b->dev.max_steps = (int32_t)(max_steps > 0 ? max_steps : 1);
    // persistent grid: every block resident at once
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heat_batch, kBatchBX * kBatchBY, 0);
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
            k_heat_batch<<<b->blocks, dim3(kBatchBX, kBatchBY), 0, b->capture>>>(b->dev);
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
        k_heat_batch<<<b->blocks, dim3(kBatchBX, kBatchBY), 0, b->stream>>>(b->dev);
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
