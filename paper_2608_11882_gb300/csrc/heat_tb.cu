// Temporally blocked heat kernel: L steps of the update of Section 4, Eq. 4
// per pass over HBM.
//
// A block owns an output tile of TX x TY columns and a chunk of k-planes, and
// streams up the chunk.  Its W x RR threads each own one 16-byte vector of x
// points (4 floats, or 2 doubles / int64s) in two consecutive rows of the tile
// plus its halo.  Level-0 planes (the field in HBM) arrive by TMA into a ring
// of NST shared-memory stages, several planes ahead of use, each completing on
// its own mbarrier.  Level t (1..L) is computed one plane behind level t-1: a
// thread keeps level t-1's values at k-1 and k in registers and receives the
// value at k+1 from the level just computed; the x/y neighbours come from a
// ping-pong shared plane per level (the neighbour between a thread's two rows
// from its own registers).  Only level L reaches HBM, so a pass moves
// (8 or 16 bytes)/L per point-step plus the halo.  Positions outside the
// interior and planes outside [0, nz) are the Dirichlet zeros at every level;
// level 0 reads them from the zero boundary layer of the padded buffer or from
// TMA's zero fill beyond it.  Blocks whose every computed point lies inside
// the interior skip the masks.
//
// Every mbarrier wait is bounded; a wait that runs out sets the handle's
// device error word (read as HS_ETIMEOUT by heat_read), waits (again bounded)
// for the block's copies in flight, and ends the block.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "heat_common.cuh"
#include "tma.cuh"

namespace hcg {

int encode_field_map(CUtensorMap* out, void* base, CUtensorMapDataType dt, size_t elem,
                     uint64_t pitch, uint64_t rows, uint64_t planes, uint32_t box_x, uint32_t box_y)
{
    // looked up once, under the thread-safe initialisation of a local static
    // (CG solves on several host threads encode maps concurrently)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                               cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess)
                   ? (PFN_cuTensorMapEncodeTiled_v12000)fn
                   : (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    if (!encode) return (int)cudaErrorNotSupported;
    const cuuint64_t dims[3] = {pitch, rows, planes};
    const cuuint64_t strides[2] = {pitch * elem, pitch * rows * elem};
    const cuuint32_t box[3] = {box_x, box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(out, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}

// Geometry of one pass.  A block of W x RR threads owns a region of RW x REG
// columns (RW = W V, REG = RR RT rows): every thread holds one 16-byte vector
// of V consecutive x points in each of RT consecutive rows.  The region is
// the output tile of TX x TY columns plus its halo: L rows on each side in y,
// and in x the halo L rounded up to whole vectors (H), so the tile and every
// thread's vector stay 16-byte aligned.  Stage and level planes share one
// layout: REG + 2 rows of BW elements, the region in rows 1..REG and columns
// A..A+RW-1, so the neighbour reads of the edge threads land in slack, never
// outside.  W is 32 (a warp per thread row, FP32 tiles 120 columns wide) or,
// for FP32 grids it covers with fewer warps, 34 (tiles 128 wide: a grid 2^k
// wide is covered exactly).  With W = 34 a warp spans two thread rows; the
// row is then padded so that the step from a row's last thread to the next
// row's first (RT rows down, RW columns back) lands on the next group of
// shared-memory banks, and 16-byte accesses stay free of bank conflicts.
template <typename T, int L, int W>
struct TbShape {
    static constexpr int V = Vec<T>::V;
    static constexpr int A = 16 / (int)sizeof(T);
    static constexpr int H = (L + V - 1) / V * V;
    static constexpr int RW = W * V;
    static constexpr int TX = RW - 2 * H;
    static constexpr int RT = kTbRowsPerThread;
    static constexpr int RR = kTbThreadRows;
    static constexpr int REG = RR * RT;
    static constexpr int TY = REG - 2 * L;
    static constexpr int NT = W * RR;
    static constexpr int WARPS = (NT + 31) / 32;
    static constexpr int pad()
    {
        if (W == 32) return 0;
        constexpr int words = (int)sizeof(T) / 4;   // 4-byte banks per element
        for (int px = 0; px < 32 * A; px += A)
            if (((RT * (RW + 2 * A + px) - RW) * words) % 32 == 0) return px;
        return 0;
    }
    static constexpr int BW = RW + 2 * A + pad();
    static constexpr int ROWS = REG + 2;
    static constexpr uint32_t BOX_BYTES = ROWS * BW * (uint32_t)sizeof(T);
    static constexpr int PLANE = (int)((BOX_BYTES + 127) / 128 * 128 / sizeof(T));
};

// Threads per row of the FP32 blocked kernel for a grid nx wide: 34 where its
// 128-column tiles need fewer warps in x than the 120-column tiles of 32.
inline int tb_row_threads(int arith, int nx)
{
    if (arith != A_F32) return 32;
    using N = TbShape<float, 2, 32>;
    using Wd = TbShape<float, 2, 34>;
    static_assert(TbShape<float, 4, 32>::TX == N::TX && TbShape<float, 4, 34>::TX == Wd::TX,
                  "the FP32 tile width must not depend on the depth (one tensor-map box)");
    const int64_t narrow = (int64_t)((nx + N::TX - 1) / N::TX) * N::WARPS;
    const int64_t wide = (int64_t)((nx + Wd::TX - 1) / Wd::TX) * Wd::WARPS;
    return wide < narrow ? 34 : 32;
}

// The pass over one chunk of planes [kb, ke).  MASK = false is taken by blocks
// whose region lies inside the interior in x and y and whose chunk with its
// z halo (every plane any level computes) lies inside [0, nz): their points
// need no Dirichlet mask.  Returns the FIXED64 maximum |U| of the block's
// outputs (0 for the floating types); on a wait that ran out, *s_abort is set
// and drain_from names the first plane whose load may still be in flight.
template <typename T, bool EXACT, int L, int W, int NST, bool MASK>
__device__ __forceinline__ unsigned long long tb_chunk(const CUtensorMap* map, T* __restrict__ dst,
                                                       const HeatGeom& g, T r, int ks, int kb, int ke,
                                                       T* stage, T* lev, uint64_t* bars, int* s_abort,
                                                       int* err, int& issued, int& drain_from)
{
    using S = TbShape<T, L, W>;
    constexpr int V = S::V, A = S::A, H = S::H, BW = S::BW, PLANE = S::PLANE, RT = S::RT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * W + tx;
    const int x0 = blockIdx.x * S::TX, y0 = blockIdx.y * S::TY;
    const int X = x0 - H + V * tx, Y0 = y0 - L + RT * ty;
    const int q0 = kb - L, qlast = ke + L - 1;
    const int xs = g.lead + x0 - H - A;   // padded x of the box: 16-byte aligned
    const int ybox = y0 - L;              // padded row of the slack row above the region
    const int own = (RT * ty + 1) * BW + A + V * tx;
    bool in_x[V], in_y[RT], out_row[RT];
#pragma unroll
    for (int i = 0; i < V; ++i) in_x[i] = X + i >= 0 && X + i < g.nx;
#pragma unroll
    for (int j = 0; j < RT; ++j) {
        in_y[j] = Y0 + j >= 0 && Y0 + j < g.ny;
        out_row[j] = RT * ty + j >= L && RT * ty + j < L + S::TY && Y0 + j < g.ny;
    }
    const int nvx = (V * tx >= H && V * tx < H + S::TX) ? min(V, g.nx - X) : 0;

    if (tid == 0) {
        for (int s = 0; s < NST && q0 + s <= qlast; ++s) {
            mbar_arrive_expect_tx(&bars[s], S::BOX_BYTES);
            tma_load_3d(stage + s * PLANE, map, xs, ybox, q0 + s + 1, &bars[s]);
            issued = q0 + s;
        }
    }
    T zb[L][RT][V], zc[L][RT][V];   // level t-1: values at the planes below and at the centre
#pragma unroll
    for (int t = 0; t < L; ++t)
#pragma unroll
        for (int j = 0; j < RT; ++j)
#pragma unroll
            for (int i = 0; i < V; ++i) zb[t][j][i] = zc[t][j][i] = T(0);
    unsigned long long mx = 0;
    T* out = dst + g.at(nvx > 0 ? X : 0, 0, 0);   // row 0 of plane 0; used when nvx > 0

    int s_cur = 0, n_cur = 0;   // slot and use count of plane q
    // unrolled by three, the period of the rotation zb <- zc <- up: the
    // compiler renames the registers instead of copying them every plane
#pragma unroll 3
    for (int q = q0; q <= qlast; ++q) {
        if (!mbar_wait_bounded(&bars[s_cur], (uint32_t)n_cur & 1u)) {
            atomicExch(err, 1);
            *s_abort = 1;
        }
        const int s_prev = s_cur == 0 ? NST - 1 : s_cur - 1;   // plane q-1 (junk at q = q0)
        T up[RT][V];
#pragma unroll
        for (int j = 0; j < RT; ++j) ld_vec(stage + s_cur * PLANE + own + j * BW, up[j]);
#pragma unroll
        for (int t = 1; t <= L; ++t) {
            const int p = q - t;
            const T* src = (t == 1) ? stage + s_prev * PLANE + own
                                    : lev + ((t - 2) * 2 + ((q - 1) & 1)) * PLANE + own;
            T ym[V], yp[V], v[RT][V];
            ld_vec(src - BW, ym);
            ld_vec(src + RT * BW, yp);
            const bool zin = p >= 0 && p < g.nz;
#pragma unroll
            for (int j = 0; j < RT; ++j) {
                const T left = src[j * BW - 1], right = src[j * BW + V];
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const T xm = i == 0 ? left : zc[t - 1][j][i - 1];
                    const T xp = i == V - 1 ? right : zc[t - 1][j][i + 1];
                    const T yl = j == 0 ? ym[i] : zc[t - 1][j - 1][i];
                    const T yh = j == RT - 1 ? yp[i] : zc[t - 1][j + 1][i];
                    const T w = Point<T, EXACT>::update(zc[t - 1][j][i], xm, xp, yl, yh, zb[t - 1][j][i],
                                                        up[j][i], r, t == 1 ? ks : 0);
                    // Dirichlet zeros outside the interior
                    if constexpr (MASK)
                        v[j][i] = (zin && in_x[i] && in_y[j]) ? w : T(0);
                    else
                        v[j][i] = w;
                }
            }
#pragma unroll
            for (int j = 0; j < RT; ++j)
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    zb[t - 1][j][i] = zc[t - 1][j][i];
                    zc[t - 1][j][i] = up[j][i];
                }
            if (t < L) {
                T* lp = lev + ((t - 1) * 2 + (q & 1)) * PLANE + own;
#pragma unroll
                for (int j = 0; j < RT; ++j) {
                    st_vec(lp + j * BW, v[j]);
#pragma unroll
                    for (int i = 0; i < V; ++i) up[j][i] = v[j][i];
                }
            } else if (nvx > 0 && p >= kb && p < ke) {
#pragma unroll
                for (int j = 0; j < RT; ++j) {
                    if (!out_row[j]) continue;
                    T* o = out + (int64_t)p * g.plane + (int64_t)(Y0 + j) * g.pitch;
                    if (nvx == V)
                        st_vec(o, v[j]);
                    else
#pragma unroll
                        for (int i = 0; i < V; ++i)
                            if (i < nvx) o[i] = v[j][i];
                    if constexpr (kIsFixed<T>) {
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            const unsigned long long a = i < nvx ? fx_abs(v[j][i]) : 0ull;
                            mx = a > mx ? a : mx;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (*s_abort) {
            drain_from = q;
            break;
        }
        if (tid == 0 && q > q0 && issued < qlast) {
            // plane q-1's slot is free: refill it with the next plane
            const int pn = issued + 1;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[s_prev], S::BOX_BYTES);
            tma_load_3d(stage + s_prev * PLANE, map, xs, ybox, pn + 1, &bars[s_prev]);
            issued = pn;
        }
        if (++s_cur == NST) {
            s_cur = 0;
            ++n_cur;
        }
    }
    return mx;
}

template <typename T, bool EXACT, int L, int W, int NST, int MINB>
__global__ void __launch_bounds__(TbShape<T, L, W>::NT, MINB)
    k_heat_tb(const __grid_constant__ CUtensorMap map, T* __restrict__ dst, HeatGeom g, T r, int kc,
              FxState* fx, int m3, int* err)
{
    using S = TbShape<T, L, W>;
    static_assert(S::TY > 0 && S::TX > 0, "tile too small for the temporal depth");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stage = reinterpret_cast<T*>(smem_raw);
    T* lev = stage + NST * S::PLANE;   // level t (1..L-1), buffer b: lev + ((t-1)*2 + b) * PLANE
    uint64_t* bars = reinterpret_cast<uint64_t*>(lev + (L - 1) * 2 * S::PLANE);
    __shared__ int s_abort;

    const int tid = threadIdx.y * W + threadIdx.x;
    if (tid == 0) {
        // a block that starts after another one gave up does no work at all
        s_abort = *(volatile int*)err;
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_abort) return;
    const int kb = blockIdx.z * kc;
    const int ke = min(kb + kc, g.nz);
    const int x0 = blockIdx.x * S::TX, y0 = blockIdx.y * S::TY;
    // the region inside the interior in x and y, every plane of the chunk's
    // levels inside [0, nz): no masks
    const bool inner = x0 - S::H >= 0 && x0 - S::H + S::RW <= g.nx && y0 - L >= 0 &&
                       y0 - L + S::REG <= g.ny && kb - 2 * L >= 0 && ke + L <= g.nz;
    int ks = 0;
    if constexpr (kIsFixed<T>) ks = fx_shift(fx, m3);
    int issued = kb - L - 1, drain_from = kb - L;
    const unsigned long long mx =
        inner ? tb_chunk<T, EXACT, L, W, NST, false>(&map, dst, g, r, ks, kb, ke, stage, lev, bars, &s_abort,
                                                 err, issued, drain_from)
              : tb_chunk<T, EXACT, L, W, NST, true>(&map, dst, g, r, ks, kb, ke, stage, lev, bars, &s_abort,
                                                err, issued, drain_from);
    if (s_abort) {
        // drain: every load still in flight must land before shared memory goes away
        if (tid == 0) {
            const int q0 = kb - L;
            const long long t0 = clock64();   // one time budget for the whole drain
            for (int p = drain_from; p <= issued; ++p) {
                const int i = p - q0;
                if (!mbar_wait_until(&bars[i % NST], (uint32_t)(i / NST) & 1u, t0, kWaitCycles)) {
                    atomicExch(err, 2);   // loads may still be landing: the context is suspect
                    break;
                }
            }
        }
        return;
    }
    if constexpr (kIsFixed<T>)
        fx_finish<S::WARPS * 32>(mx, fx, m3, ks, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

template <typename T, bool EXACT, int L, int W>
int tb_launch_w(const TbCall& c)
{
    // three staged planes ahead; two blocks per SM at depth 2 (their planes
    // take 71-77 KB of shared memory each), one at depths 3 and 4, whose
    // registers for the extra levels would not fit two
    constexpr int NST = 3;
    constexpr int MINB = L == 2 ? 2 : 1;
    using S = TbShape<T, L, W>;
    constexpr size_t smem =
        sizeof(T) * (size_t)(NST + 2 * (L - 1)) * S::PLANE + NST * sizeof(uint64_t);
    if (c.box[0] != (uint32_t)S::BW || c.box[1] != (uint32_t)S::ROWS)
        return fail(HS_EINVAL, "heat: tensor map box %ux%u does not match the kernel's %dx%d", c.box[0],
                    c.box[1], S::BW, S::ROWS);
    auto kern = k_heat_tb<T, EXACT, L, W, NST, MINB>;
    // once per process, under the thread-safe initialisation of a local static
    static const cudaError_t configured =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    HS_TRY_CUDA(configured, "heat: temporal-blocking kernel smem attribute");
    const HeatGeom& g = *c.g;
    dim3 grid((g.nx + S::TX - 1) / S::TX, (g.ny + S::TY - 1) / S::TY, (g.nz + c.kc - 1) / c.kc);
    dim3 block(W, S::RR, 1);
    kern<<<grid, block, smem, c.stream>>>(*c.map, (T*)c.dst, g, tb_param<T>(c), c.kc, c.fx, c.m3,
                                          c.err);
    HS_CHECK_LAUNCH("heat temporal-blocking kernel");
    return HS_OK;
}

template <typename T, bool EXACT, int L>
int tb_launch_t(const TbCall& c)
{
    if constexpr (std::is_same<T, float>::value)
        if (tb_row_threads(A_F32, c.g->nx) == 34) return tb_launch_w<T, EXACT, L, 34>(c);
    return tb_launch_w<T, EXACT, L, 32>(c);
}

template <typename T, bool EXACT>
int tb_dispatch_L(const TbCall& c)
{
    switch (c.L) {
    case 2: return tb_launch_t<T, EXACT, 2>(c);
    case 3: return tb_launch_t<T, EXACT, 3>(c);
    case 4: return tb_launch_t<T, EXACT, 4>(c);
    }
    return fail(HS_EINVAL, "heat: temporal depth %d not built (2, 3 or 4)", c.L);
}

int tb_box(int arith, int nx, uint32_t* box_x, uint32_t* box_y)
{
    // the box does not depend on the depth L
    if (arith == A_F32) {
        const bool wide = tb_row_threads(arith, nx) == 34;
        *box_x = wide ? TbShape<float, 2, 34>::BW : TbShape<float, 2, 32>::BW;
        *box_y = TbShape<float, 2, 32>::ROWS;
    } else {
        *box_x = TbShape<double, 2, 32>::BW;
        *box_y = TbShape<double, 2, 32>::ROWS;
    }
    return 0;
}

template <typename T, int W>
void tb_tile_t(int L, int* tx, int* ty)
{
    switch (L) {
    case 2: *tx = TbShape<T, 2, W>::TX; *ty = TbShape<T, 2, W>::TY; return;
    case 3: *tx = TbShape<T, 3, W>::TX; *ty = TbShape<T, 3, W>::TY; return;
    default: *tx = TbShape<T, 4, W>::TX; *ty = TbShape<T, 4, W>::TY; return;
    }
}

void tb_tile(int arith, int L, int nx, int* tx, int* ty)
{
    if (arith != A_F32)
        tb_tile_t<double, 32>(L, tx, ty);
    else if (tb_row_threads(arith, nx) == 34)
        tb_tile_t<float, 34>(L, tx, ty);
    else
        tb_tile_t<float, 32>(L, tx, ty);
}

int tb_launch(const TbCall& c)
{
    switch (c.arith) {
    case A_F64: return tb_dispatch_L<double, false>(c);
    case A_F64_EXACT: return tb_dispatch_L<double, true>(c);
    case A_F32: return tb_dispatch_L<float, false>(c);
    case A_FX64: return tb_dispatch_L<long long, false>(c);
    }
    return fail(HS_EINVAL, "heat: unknown arithmetic");
}

}  // namespace hcg
