// Temporally blocked heat kernel: L steps of the update of Section 4, Eq. 4
// per pass over HBM.
//
// A block owns an output tile of TX x TY columns and a chunk of k-planes, and
// streams up the chunk.  Its 32 x RY threads each own one 16-byte vector of x
// points (4 floats, or 2 doubles / int64s) in one row of the tile plus its
// halo.  Level-0 planes (the
// field in HBM) arrive by TMA into a ring of NST shared-memory stages, several
// planes ahead of use, each completing on its own mbarrier.  Level t (1..L)
// is computed one plane behind level t-1: a thread keeps level t-1's values
// at k-1 and k in registers and receives the value at k+1 from the level just
// computed; the x/y neighbours come from a ping-pong shared plane per level.
// Only level L reaches HBM, so a pass moves (8 or 16 bytes)/L per point-step
// plus the halo.  Positions outside the interior and planes outside [0, nz)
// are the Dirichlet zeros at every level; level 0 reads them from the zero
// boundary layer of the padded buffer or from TMA's zero fill beyond it.
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

// Geometry of one pass: every thread holds V consecutive x points (one
// 16-byte vector) of one row.  The x halo H is L rounded up to whole vectors,
// so the tile and every thread's vector stay 16-byte aligned; rows carry the
// exact halo L.  Stage and level planes share one layout: RY + 2 rows of
// RW + 2A elements, the data in rows 1..RY and columns A..A+RW-1, so the
// neighbour reads of the edge threads land in slack, never outside.
template <typename T, int L, int RY>
struct TbShape {
    static constexpr int V = Vec<T>::V;
    static constexpr int A = 16 / (int)sizeof(T);
    static constexpr int H = (L + V - 1) / V * V;
    static constexpr int RW = 32 * V;
    static constexpr int TX = RW - 2 * H;
    static constexpr int TY = RY - 2 * L;
    static constexpr int BW = RW + 2 * A;
    static constexpr int ROWS = RY + 2;
    static constexpr uint32_t BOX_BYTES = ROWS * BW * (uint32_t)sizeof(T);
    static constexpr int PLANE = (int)((BOX_BYTES + 127) / 128 * 128 / sizeof(T));
};

template <typename T, bool EXACT, int L, int RY, int NST>
__global__ void __launch_bounds__(32 * RY, 1)
    k_heat_tb(const __grid_constant__ CUtensorMap map, T* __restrict__ dst, HeatGeom g, T r, int kc,
              FxState* fx, int m3, int* err)
{
    using S = TbShape<T, L, RY>;
    constexpr int V = S::V, A = S::A, H = S::H, TX = S::TX, TY = S::TY, BW = S::BW;
    constexpr int PLANE = S::PLANE;
    static_assert(TY > 0 && TX > 0, "tile too small for the temporal depth");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stage = reinterpret_cast<T*>(smem_raw);
    T* lev = stage + NST * PLANE;   // level t (1..L-1), buffer b: lev + ((t-1)*2 + b) * PLANE
    uint64_t* bars = reinterpret_cast<uint64_t*>(lev + (L - 1) * 2 * PLANE);
    __shared__ int s_abort;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int X = x0 - H + V * tx, Y = y0 - L + ty;
    const int kb = blockIdx.z * kc;
    const int ke = min(kb + kc, g.nz);
    const int q0 = kb - L, qlast = ke + L - 1;
    const int xs = g.lead + x0 - H - A;   // padded x of the box: 16-byte aligned
    const int ybox = y0 - L;              // padded row of the slack row above the region
    const int own = (ty + 1) * BW + A + V * tx;
    const bool row_in = (Y >= 0 && Y < g.ny);
    bool in_x[V];
#pragma unroll
    for (int i = 0; i < V; ++i) in_x[i] = (X + i >= 0 && X + i < g.nx);
    const bool out_rows = (ty >= L && ty < L + TY && row_in);
    const bool out_cols = (V * tx >= H && V * tx < H + TX);
    const int nvalid = (out_rows && out_cols) ? min(V, g.nx - X) : 0;

    int issued = q0 - 1;
    int drain_from = q0;
    if (tid == 0) {
        // a block that starts after another one gave up does no work at all
        s_abort = *(volatile int*)err;
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_abort) return;
    if (tid == 0) {
        for (int s = 0; s < NST && q0 + s <= qlast; ++s) {
            mbar_arrive_expect_tx(&bars[s], S::BOX_BYTES);
            tma_load_3d(stage + s * PLANE, &map, xs, ybox, q0 + s + 1, &bars[s]);
            issued = q0 + s;
        }
    }
    int ks = 0;
    if constexpr (kIsFixed<T>) ks = fx_shift(fx, m3);
    T zb[L][V], zc[L][V];   // level t-1: values at the planes below and at the centre
#pragma unroll
    for (int t = 0; t < L; ++t)
#pragma unroll
        for (int i = 0; i < V; ++i) zb[t][i] = zc[t][i] = T(0);
    unsigned long long mx = 0;
    T* out = dst + g.at(nvalid > 0 ? X : 0, nvalid > 0 ? Y : 0, 0);   // plane 0; used when nvalid > 0

    int s_cur = 0, n_cur = 0;   // slot and use count of plane q
    int q = q0;
    for (; q <= qlast; ++q) {
        if (!mbar_wait_bounded(&bars[s_cur], (uint32_t)n_cur & 1u)) {
            atomicExch(err, 1);
            s_abort = 1;
        }
        const int s_prev = s_cur == 0 ? NST - 1 : s_cur - 1;   // plane q-1 (junk at q = q0)
        T up[V];
        ld_vec(stage + s_cur * PLANE + own, up);
#pragma unroll
        for (int t = 1; t <= L; ++t) {
            const int p = q - t;
            const T* src = (t == 1) ? stage + s_prev * PLANE + own
                                    : lev + ((t - 2) * 2 + ((q - 1) & 1)) * PLANE + own;
            T ym[V], yp[V], v[V];
            ld_vec(src - BW, ym);
            ld_vec(src + BW, yp);
            const T left = src[-1], right = src[V];
            const bool zin = row_in && p >= 0 && p < g.nz;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const T xm = i == 0 ? left : zc[t - 1][i - 1];
                const T xp = i == V - 1 ? right : zc[t - 1][i + 1];
                const T w = Point<T, EXACT>::update(zc[t - 1][i], xm, xp, ym[i], yp[i], zb[t - 1][i],
                                                    up[i], r, t == 1 ? ks : 0);
                v[i] = (zin && in_x[i]) ? w : T(0);   // Dirichlet zeros outside the interior
            }
#pragma unroll
            for (int i = 0; i < V; ++i) {
                zb[t - 1][i] = zc[t - 1][i];
                zc[t - 1][i] = up[i];
            }
            if (t < L) {
                st_vec(lev + ((t - 1) * 2 + (q & 1)) * PLANE + own, v);
#pragma unroll
                for (int i = 0; i < V; ++i) up[i] = v[i];
            } else if (nvalid > 0 && p >= kb && p < ke) {
                T* o = out + (int64_t)p * g.plane;
                if (nvalid == V)
                    st_vec(o, v);
                else
#pragma unroll
                    for (int i = 0; i < V; ++i)
                        if (i < nvalid) o[i] = v[i];
                if constexpr (kIsFixed<T>) {
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        const unsigned long long a = i < nvalid ? fx_abs(v[i]) : 0ull;
                        mx = a > mx ? a : mx;
                    }
                }
            }
        }
        __syncthreads();
        if (s_abort) {
            drain_from = q;
            break;
        }
        if (tid == 0 && q > q0 && issued < qlast) {
            // plane q-1's slot is free: refill it with the next plane
            const int pn = issued + 1;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[s_prev], S::BOX_BYTES);
            tma_load_3d(stage + s_prev * PLANE, &map, xs, ybox, pn + 1, &bars[s_prev]);
            issued = pn;
        }
        if (++s_cur == NST) {
            s_cur = 0;
            ++n_cur;
        }
    }
    if (s_abort) {
        // drain: every load still in flight must land before shared memory goes away
        if (tid == 0) {
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
        fx_finish<32 * RY>(mx, fx, m3, ks, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

template <typename T, bool EXACT, int L>
int tb_launch_t(const TbCall& c)
{
    constexpr int RY = kTbRows;
    constexpr int NST = 4;
    using S = TbShape<T, L, RY>;
    constexpr size_t smem =
        sizeof(T) * (size_t)(NST + 2 * (L - 1)) * S::PLANE + NST * sizeof(uint64_t);
    if (c.box[0] != (uint32_t)S::BW || c.box[1] != (uint32_t)S::ROWS)
        return fail(HS_EINVAL, "heat: tensor map box %ux%u does not match the kernel's %dx%d", c.box[0],
                    c.box[1], S::BW, S::ROWS);
    auto kern = k_heat_tb<T, EXACT, L, RY, NST>;
    static bool configured = false;
    if (!configured) {
        HS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "heat: temporal-blocking kernel smem attribute");
        configured = true;
    }
    const HeatGeom& g = *c.g;
    dim3 grid((g.nx + S::TX - 1) / S::TX, (g.ny + S::TY - 1) / S::TY, (g.nz + c.kc - 1) / c.kc);
    dim3 block(32, RY, 1);
    kern<<<grid, block, smem, c.stream>>>(*c.map, (T*)c.dst, g, tb_param<T>(c), c.kc, c.fx, c.m3,
                                          c.err);
    HS_CHECK_LAUNCH("heat temporal-blocking kernel");
    return HS_OK;
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

int tb_box(int arith, uint32_t* box_x, uint32_t* box_y)
{
    // the box does not depend on the depth L
    if (arith == A_F32) {
        *box_x = TbShape<float, 2, kTbRows>::BW;
        *box_y = TbShape<float, 2, kTbRows>::ROWS;
    } else {
        *box_x = TbShape<double, 2, kTbRows>::BW;
        *box_y = TbShape<double, 2, kTbRows>::ROWS;
    }
    return 0;
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
