// Streaming Interior kernel: one step of the update of Section 4, Eq. 4 over
// a range of k-planes, with the planes staged in shared memory by TMA.
//
// A block of 32 x RY threads owns a (32 V) x RY column tile -- every thread
// computes V consecutive x points (4 floats, or 2 doubles / int64s, one
// 16-byte vector) -- and a chunk of k-planes.  Each plane of the tile plus a
// one-point halo ((RY + 2) rows of BW elements) arrives by TMA into a ring of
// NST stages, up to NST - 2 planes ahead of use, so each SM keeps tens of
// kilobytes of loads in flight.  A thread keeps its own values at k-1 and k in
// registers, reads the values at k+1 and the rows at y-1 and y+1 as 16-byte
// vectors from shared memory, and the two x neighbours beyond its vector as
// scalars; the result goes out as one 16-byte store.  The per-point arithmetic is that of the other heat kernels,
// so results match them bit for bit.
//
// Every mbarrier wait is bounded: one that runs out sets the handle's device
// error word (HS_ETIMEOUT at the next heat_read), waits (bounded) for the
// block's loads in flight and ends the block.
#include <cuda.h>

#include "heat_common.cuh"
#include "tma.cuh"

namespace hcg {


// Tile geometry.  Interior rows start 32 bytes into a padded row (lead *
// sizeof(T) = 32) and a tile is 32 V points = 512 bytes wide, so a box that
// starts D = 16 bytes before the tile's first point starts 16-byte aligned
// (as TMA requires), and the tile's first point -- hence every thread's
// vector -- sits 16-byte aligned in the stage row.  The row is wide enough
// for the halo point on each side and rounded up to 16 bytes.
template <typename T>
struct StreamShape {
    static constexpr int V = Vec<T>::V;
    static constexpr int A = 16 / (int)sizeof(T);                // elements per 16 bytes
    static constexpr int D = A;                                  // offset of the tile's first point
    static constexpr int BW = (D + 32 * V + 1 + A - 1) / A * A;  // stage row width, 16-byte multiple
};

template <typename T, bool EXACT, int RY, int NST, int UNR = kIsFixed<T> ? 3 : 1>
__global__ void __launch_bounds__(32 * RY)
    k_heat_stream(const __grid_constant__ CUtensorMap map, T* __restrict__ dst, HeatGeom g, T r,
                  int kbeg, int kend, int kc, FxState* fx, int m3, int* err)
{
    using S = StreamShape<T>;
    constexpr int V = S::V;
    constexpr int BW = S::BW;
    constexpr int ROWS = RY + 2;
    constexpr uint32_t BOX_BYTES = ROWS * BW * (uint32_t)sizeof(T);
    constexpr int STAGE = (int)((BOX_BYTES + 127) / 128 * 128 / sizeof(T));   // 128-byte aligned slots
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stage = reinterpret_cast<T*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage + NST * STAGE);
    __shared__ int s_abort;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const int x0 = blockIdx.x * 32 * V, y0 = blockIdx.y * RY;
    const int X = x0 + V * tx, Y = y0 + ty;
    const int kb = kbeg + blockIdx.z * kc;
    const int ke = min(kb + kc, kend);
    const int xs = g.lead + x0 - S::D;                 // padded x of the box (16-byte aligned)
    const int own = (ty + 1) * BW + S::D + V * tx;     // this thread's first point in a stage
    const bool row_ok = (Y < g.ny);
    const int nvalid = row_ok ? min(V, g.nx - X) : 0;  // points of this thread inside the box
    const int p_first = kb - 1, p_last = ke;           // planes staged: kb-1 .. ke

    int issued = p_first - 1;
    int drain_from = p_first;
    if (tid == 0) {
        // a block that starts after another one gave up does no work at all
        s_abort = *(volatile int*)err;
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_abort) return;
    if (tid == 0) {
        for (int s = 0; s < NST && p_first + s <= p_last; ++s) {
            mbar_arrive_expect_tx(&bars[s], BOX_BYTES);
            tma_load_3d(stage + s * STAGE, &map, xs, y0, p_first + s + 1, &bars[s]);
            issued = p_first + s;
        }
    }
    int ks = 0;
    if constexpr (kIsFixed<T>) ks = fx_shift(fx, m3);
    unsigned long long mx = 0;

    T below[V], cur[V], above[V], ym[V], yp[V], v[V];
    int s_cur = 0, n_cur = 0;
    bool ok = mbar_wait_bounded(&bars[0], 0);
    ld_vec(stage + own, below);
    int s_nxt = 1 % NST, n_nxt = 1 / NST;
    ok = ok && mbar_wait_bounded(&bars[s_nxt], (uint32_t)n_nxt & 1u);
    ld_vec(stage + s_nxt * STAGE + own, cur);
    s_cur = s_nxt;
    n_cur = n_nxt;
    if (!ok) {
        atomicExch(err, 1);
        s_abort = 1;
    }
    __syncthreads();

    T* out = dst + g.at(X < g.nx ? X : 0, row_ok ? Y : 0, kb);   // only used when nvalid > 0
    int k = kb;
    if (!s_abort) {
        // FIXED64: unrolled by three, the period of the rotation below <- cur <-
        // above, so the 64-bit registers are renamed instead of copied every
        // plane (0.364 ms against 0.398 per 512^3 launch; FP32 and the FP64
        // pipe gain nothing, and the exact-sum kernel loses a little)
#pragma unroll UNR
        for (; k < ke; ++k) {
            s_nxt = s_cur + 1 == NST ? 0 : s_cur + 1;
            n_nxt = s_nxt == 0 ? n_cur + 1 : n_cur;
            if (!mbar_wait_bounded(&bars[s_nxt], (uint32_t)n_nxt & 1u)) {
                atomicExch(err, 1);
                s_abort = 1;
            }
            const T* pl = stage + s_cur * STAGE + own;
            ld_vec(stage + s_nxt * STAGE + own, above);
            ld_vec(pl - BW, ym);
            ld_vec(pl + BW, yp);
            const T left = pl[-1], right = pl[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const T xm = i == 0 ? left : cur[i - 1];
                const T xp = i == V - 1 ? right : cur[i + 1];
                v[i] = Point<T, EXACT>::update(cur[i], xm, xp, ym[i], yp[i], below[i], above[i], r, ks);
            }
            if (nvalid == V) {
                st_vec(out, v);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (i < nvalid) out[i] = v[i];
            }
            if constexpr (kIsFixed<T>) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const unsigned long long a = i < nvalid ? fx_abs(v[i]) : 0ull;
                    mx = a > mx ? a : mx;
                }
            }
#pragma unroll
            for (int i = 0; i < V; ++i) {
                below[i] = cur[i];
                cur[i] = above[i];
            }
            out += g.plane;
            __syncthreads();
            if (s_abort) {
                drain_from = k + 1;
                break;
            }
            if (tid == 0 && issued < p_last) {
                const int slot = s_cur == 0 ? NST - 1 : s_cur - 1;   // plane k-1's slot is free
                const int pn = issued + 1;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[slot], BOX_BYTES);
                tma_load_3d(stage + slot * STAGE, &map, xs, y0, pn + 1, &bars[slot]);
                issued = pn;
            }
            s_cur = s_nxt;
            n_cur = n_nxt;
        }
    }
    if (s_abort) {
        if (tid == 0) {
            const long long t0 = clock64();   // one time budget for the whole drain
            for (int p = drain_from; p <= issued; ++p) {
                const int i = p - p_first;
                if (!mbar_wait_until(&bars[i % NST], (uint32_t)(i / NST) & 1u, t0, kWaitCycles)) {
                    atomicExch(err, 2);   // loads may still be landing: the context is suspect
                    break;
                }
            }
        }
        return;
    }
    if constexpr (kIsFixed<T>)
        fx_finish<32 * RY>(mx, fx, m3, ks, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

// ---- FP64 with the exact neighbour sum (A_F64_XS) -------------------------------------
// The ring, waits and error handling of k_heat_stream, for FP64 fields in the
// exact-sum arithmetic (heat_common.cuh).  A block of 32 x (RY / RT) threads
// owns a 64 x RY tile; every thread two consecutive x points of RT adjacent
// rows, so the per-plane work of a thread (its waits, barrier, address and
// loop arithmetic) is shared by 2 RT points, and the y neighbours between its
// own rows come from its registers.  Once plane k+1 has landed, the block
// converts it in place to fixed point on the field's scale: every thread its
// own vectors (keeping the raw doubles, the centre values of the next
// iteration), warps 0 and 1 the halo rows, warp 2 the two halo columns, so
// each staged value is converted once.  Plane k, converted one iteration
// earlier, gives the neighbours from outside the thread's own values.  A point
// then costs the exact integer sum, one conversion back (on the FP64 pipe for
// one of a thread's four points, with integer instructions for the others)
// and one FP64 fused multiply-add.  Converted slots are written through the
// generic proxy and refilled later by TMA (the async proxy), so every thread
// fences the async proxy after its conversion stores, before the block
// barrier that precedes a refill.  CONV = false is the FP64-pipe update on the
// raw planes, for fields outside the conversion's exponent range.
template <int RY, int RT, int NST, bool CONV>
__device__ __forceinline__ void xs_stream_body(const CUtensorMap* map, double* __restrict__ dst,
                                               const HeatGeom& g, double r, int kb, int ke, int emax,
                                               long long* stage, uint64_t* bars, int& s_abort,
                                               unsigned& mx, int* err)
{
    using S = StreamShape<double>;
    constexpr int V = S::V;
    constexpr int BW = S::BW;
    constexpr int TY = RY / RT;
    constexpr int ROWS = RY + 2;
    constexpr uint32_t BOX_BYTES = ROWS * BW * (uint32_t)sizeof(double);
    constexpr int STAGE = (int)((BOX_BYTES + 127) / 128 * 128 / sizeof(double));
    static_assert(V == 2 && RY % RT == 0 && TY >= 3 && 2 * RY <= 32,
                  "warps 0, 1 convert the halo rows, warp 2 the 2 RY halo-column values");

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const int x0 = blockIdx.x * 32 * V, y0 = blockIdx.y * RY;
    const int X = x0 + V * tx, Y0 = y0 + ty * RT;      // this thread's first point
    const int xs = g.lead + x0 - S::D;
    const int own = (ty * RT + 1) * BW + S::D + V * tx;  // its first point in a stage (row j: + j BW)
    const int nx_ok = min(V, g.nx - X);                // points per row inside the box
    const int p_first = kb - 1, p_last = ke;
    const double r2 = CONV ? xs_r2(r, emax) : 0.0;
    // what this thread converts besides its own vectors: a vector of halo row 0
    // (warp 0) or RY+1 (warp 1), or one halo-column value (warp 2)
    int extra = -1;
    if (ty == 0) extra = S::D + V * tx;
    else if (ty == 1) extra = (RY + 1) * BW + S::D + V * tx;
    else if (ty == 2 && tx < 2 * RY)
        extra = tx < RY ? (tx + 1) * BW + S::D - 1 : (tx - RY + 1) * BW + S::D + 32 * V;

    // converts this thread's part of the staged plane at `pl`; returns its own raw vectors
    auto convert = [&](long long* pl, long long (&q)[RT][V], double (&raw)[RT][V]) {
#pragma unroll
        for (int j = 0; j < RT; ++j) {
            long long b[V];
            ld_vec(pl + own + j * BW, b);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                raw[j][i] = __longlong_as_double(b[i]);
                q[j][i] = CONV ? xs_fix(b[i], emax) : b[i];
            }
            if constexpr (CONV) st_vec(pl + own + j * BW, q[j]);
        }
        if constexpr (CONV) {
            if (ty < 2) {
                long long h[V];
                ld_vec(pl + extra, h);
#pragma unroll
                for (int i = 0; i < V; ++i) h[i] = xs_fix(h[i], emax);
                st_vec(pl + extra, h);
            } else if (extra >= 0) {
                pl[extra] = xs_fix(pl[extra], emax);
            }
        }
    };

    int issued = p_first - 1;
    int drain_from = p_first;
    if (tid == 0) {
        for (int s = 0; s < NST && p_first + s <= p_last; ++s) {
            mbar_arrive_expect_tx(&bars[s], BOX_BYTES);
            tma_load_3d(stage + s * STAGE, map, xs, y0, p_first + s + 1, &bars[s]);
            issued = p_first + s;
        }
    }
    long long below[RT][V], cur[RT][V], above[RT][V];
    double craw[RT][V], araw[RT][V];
    int s_cur = 0, n_cur = 0;
    bool ok = mbar_wait_bounded(&bars[0], 0);
#pragma unroll
    for (int j = 0; j < RT; ++j) {
        long long b[V];
        ld_vec(stage + own + j * BW, b);
#pragma unroll
        for (int i = 0; i < V; ++i) below[j][i] = CONV ? xs_fix(b[i], emax) : b[i];
    }
    int s_nxt = 1 % NST, n_nxt = 1 / NST;
    ok = ok && mbar_wait_bounded(&bars[s_nxt], (uint32_t)n_nxt & 1u);
    convert(stage + s_nxt * STAGE, cur, craw);
    s_cur = s_nxt;
    n_cur = n_nxt;
    if (!ok) {
        atomicExch(err, 1);
        s_abort = 1;
    }
    if constexpr (CONV) fence_proxy_async_smem();
    __syncthreads();

    // row j of this thread's points at plane kb; only used for rows inside the box
    double* out = dst + g.at(X < g.nx ? X : 0, 0, kb) + (int64_t)Y0 * g.pitch;
    if (!s_abort) {
        for (int k = kb; k < ke; ++k) {
            s_nxt = s_cur + 1 == NST ? 0 : s_cur + 1;
            n_nxt = s_nxt == 0 ? n_cur + 1 : n_cur;
            if (!mbar_wait_bounded(&bars[s_nxt], (uint32_t)n_nxt & 1u)) {
                atomicExch(err, 1);
                s_abort = 1;
            }
            convert(stage + s_nxt * STAGE, above, araw);
            const long long* pl = stage + s_cur * STAGE + own;
            long long ym[V], yp[V];
            ld_vec(pl - BW, ym);        // the row below the thread's first row
            ld_vec(pl + RT * BW, yp);   // the row above its last row
#pragma unroll
            for (int j = 0; j < RT; ++j) {
                const long long left = pl[j * BW - 1], right = pl[j * BW + V];
                double v[V];
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const long long xm = i == 0 ? left : cur[j][i - 1];
                    const long long xp = i == V - 1 ? right : cur[j][i + 1];
                    const long long yl = j == 0 ? ym[i] : cur[j - 1][i];
                    const long long yh = j == RT - 1 ? yp[i] : cur[j + 1][i];
                    if constexpr (CONV) {
                        // one of the thread's four points converts L on the FP64 pipe,
                        // the other three with integer instructions: the same result,
                        // the FP64 pipe left with 1.25 instructions per point (measured
                        // ahead of 1.5 and of 1)
                        const long long L = xs_numerator(cur[j][i], xm, xp, yl, yh, below[j][i], above[j][i]);
                        v[i] = (j == 0 && i == 0) ? xs_apply<true>(craw[j][i], L, r, r2, emax)
                                                  : xs_apply<false>(craw[j][i], L, r, r2, emax);
                    } else {
                        auto d = [](long long b) { return __longlong_as_double(b); };
                        v[i] = Point<double, false>::update(craw[j][i], d(xm), d(xp), d(yl), d(yh),
                                                            d(below[j][i]), d(above[j][i]), r, 0);
                    }
                }
                const int nvalid = Y0 + j < g.ny ? nx_ok : 0;
                double* o = out + j * g.pitch;
                if (nvalid == V) {
                    st_vec(o, v);
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i)
                        if (i < nvalid) o[i] = v[i];
                }
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const unsigned a = i < nvalid ? xs_abs_hi(v[i]) : 0u;
                    mx = a > mx ? a : mx;
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
            __syncthreads();
            if (s_abort) {
                drain_from = k + 1;
                break;
            }
            if (tid == 0 && issued < p_last) {
                const int slot = s_cur == 0 ? NST - 1 : s_cur - 1;   // plane k-1's slot is free
                const int pn = issued + 1;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[slot], BOX_BYTES);
                tma_load_3d(stage + slot * STAGE, map, xs, y0, pn + 1, &bars[slot]);
                issued = pn;
            }
            s_cur = s_nxt;
            n_cur = n_nxt;
        }
    } else {
        drain_from = p_first;
    }
    if (s_abort && tid == 0) {
        const long long t0 = clock64();   // one time budget for the whole drain
        for (int p = drain_from; p <= issued; ++p) {
            const int i = p - p_first;
            if (!mbar_wait_until(&bars[i % NST], (uint32_t)(i / NST) & 1u, t0, kWaitCycles)) {
                atomicExch(err, 2);   // loads may still be landing: the context is suspect
                break;
            }
        }
    }
}

// kXsRows rows per tile, kXsRowsPerThread per thread: 128 threads, 64
// registers (eight blocks per SM, each with a ring of kXsStages planes).
template <int RY, int RT, int NST>
__global__ void __launch_bounds__(32 * (RY / RT), 8)
    k_heat_stream_xs(const __grid_constant__ CUtensorMap map, double* __restrict__ dst, HeatGeom g,
                     double r, int kbeg, int kend, int kc, FxState* fx, int m3, int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using S = StreamShape<double>;
    constexpr uint32_t BOX_BYTES = (RY + 2) * S::BW * (uint32_t)sizeof(double);
    constexpr int STAGE = (int)((BOX_BYTES + 127) / 128 * 128 / sizeof(double));
    long long* stage = reinterpret_cast<long long*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage + NST * STAGE);
    __shared__ int s_abort;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int kb = kbeg + blockIdx.z * kc;
    const int ke = min(kb + kc, kend);
    if (tid == 0) {
        // a block that starts after another one gave up does no work at all
        s_abort = *(volatile int*)err;
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_abort) return;
    const int emax = xs_emax(fx, m3);
    unsigned mx = 0;
    if (xs_native(emax, r))
        xs_stream_body<RY, RT, NST, false>(&map, dst, g, r, kb, ke, emax, stage, bars, s_abort, mx, err);
    else
        xs_stream_body<RY, RT, NST, true>(&map, dst, g, r, kb, ke, emax, stage, bars, s_abort, mx, err);
    if (s_abort) return;   // uniform: every thread passed the barrier that saw it
    fx_finish<32 * (RY / RT)>((unsigned long long)mx << 32, fx, m3, 0,
                              blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

template <typename T>
constexpr int stream_rows()
{
    return 16;
}

int stream_launch_xs(const StreamCall& c)
{
    constexpr int RY = kXsRows, RT = kXsRowsPerThread, NST = kXsStages;
    constexpr size_t box_bytes = sizeof(double) * (size_t)(RY + 2) * StreamShape<double>::BW;
    constexpr size_t smem = NST * ((box_bytes + 127) / 128 * 128) + NST * sizeof(uint64_t);
    if (c.box[0] != (uint32_t)StreamShape<double>::BW || c.box[1] != (uint32_t)(RY + 2))
        return fail(HS_EINVAL, "heat: tensor map box %ux%u does not match the kernel's %dx%d", c.box[0],
                    c.box[1], StreamShape<double>::BW, RY + 2);
    auto kern = k_heat_stream_xs<RY, RT, NST>;
    // once per process, under the thread-safe initialisation of a local static
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    HS_TRY_CUDA(configured, "heat: streaming kernel smem attribute");
    const HeatGeom& g = *c.g;
    const int planes = c.kend - c.kbeg;
    if (planes <= 0) return HS_OK;
    constexpr int TXW = 32 * StreamShape<double>::V;
    dim3 grid((g.nx + TXW - 1) / TXW, (g.ny + RY - 1) / RY, (planes + c.kc - 1) / c.kc);
    dim3 block(32, RY / RT, 1);
    kern<<<grid, block, smem, c.stream>>>(*c.map, (double*)c.dst, g, c.r, c.kbeg, c.kend, c.kc, c.fx,
                                          c.m3, c.err);
    HS_CHECK_LAUNCH("heat streaming Interior kernel (FP64 exact sum)");
    return HS_OK;
}

template <typename T, bool EXACT>
int stream_launch_t(const StreamCall& c)
{
    constexpr int RY = stream_rows<T>();
    constexpr int NST = 6;
    constexpr size_t box_bytes = sizeof(T) * (size_t)(RY + 2) * StreamShape<T>::BW;
    constexpr size_t smem = NST * ((box_bytes + 127) / 128 * 128) + NST * sizeof(uint64_t);
    if (c.box[0] != (uint32_t)StreamShape<T>::BW || c.box[1] != (uint32_t)(RY + 2))
        return fail(HS_EINVAL, "heat: tensor map box %ux%u does not match the kernel's %dx%d", c.box[0],
                    c.box[1], StreamShape<T>::BW, RY + 2);
    auto kern = k_heat_stream<T, EXACT, RY, NST>;
    // once per process, under the thread-safe initialisation of a local static
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    HS_TRY_CUDA(configured, "heat: streaming kernel smem attribute");
    const HeatGeom& g = *c.g;
    const int planes = c.kend - c.kbeg;
    if (planes <= 0) return HS_OK;
    constexpr int TXW = 32 * Vec<T>::V;
    dim3 grid((g.nx + TXW - 1) / TXW, (g.ny + RY - 1) / RY, (planes + c.kc - 1) / c.kc);
    dim3 block(32, RY, 1);
    kern<<<grid, block, smem, c.stream>>>(*c.map, (T*)c.dst, g, stream_param<T>(c), c.kbeg, c.kend,
                                          c.kc, c.fx, c.m3, c.err);
    HS_CHECK_LAUNCH("heat streaming Interior kernel");
    return HS_OK;
}

int stream_launch(const StreamCall& c)
{
    switch (c.arith) {
    case A_F64: return stream_launch_t<double, false>(c);
    case A_F64_EXACT: return stream_launch_t<double, true>(c);
    case A_F32: return stream_launch_t<float, false>(c);
    case A_FX64: return stream_launch_t<long long, false>(c);
    case A_F64_XS: return stream_launch_xs(c);
    }
    return fail(HS_EINVAL, "heat: unknown arithmetic");
}

int stream_box(int arith, uint32_t* box_x, uint32_t* box_y)
{
    switch (arith) {
    case A_F64_XS:
        *box_x = StreamShape<double>::BW;
        *box_y = kXsRows + 2;
        return 0;
    case A_F32:
        *box_x = StreamShape<float>::BW;
        *box_y = stream_rows<float>() + 2;
        return 0;
    default:
        *box_x = StreamShape<double>::BW;
        *box_y = stream_rows<double>() + 2;
        return 0;
    }
}

}  // namespace hcg
