// Temporally blocked heat kernel: L steps of the update of Section 4, Eq. 4
// per pass over HBM.
//
// A block owns an output tile of TX x TY = (32 - 2L) x (RY - 2L) columns and
// a chunk of k-planes, and streams up the chunk.  Its 32 x RY threads each own
// one (x, y) position of the tile plus an L-wide halo.  Level-0 planes (the
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
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return (int)e;
        if (q != cudaDriverEntryPointSuccess || !fn) return (int)cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[3] = {pitch, rows, planes};
    const cuuint64_t strides[2] = {pitch * elem, pitch * rows * elem};
    const cuuint32_t box[3] = {box_x, box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(out, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}

constexpr uint32_t kMaxPolls = 1u << 22;   // bounded mbarrier wait (well over a second)

template <typename T, bool EXACT, int L, int RY, int NST>
__global__ void __launch_bounds__(32 * RY, 1)
    k_heat_tb(const __grid_constant__ CUtensorMap map, T* __restrict__ dst, HeatGeom g, T r, int kc,
              FxState* fx, int m3, int* err)
{
    constexpr int A = 16 / (int)sizeof(T);   // TMA x start must be 16-byte aligned
    constexpr int BW = 32 + A;               // stage row width (box width)
    constexpr int TX = 32 - 2 * L, TY = RY - 2 * L;
    constexpr int STAGE = RY * BW;           // elements per stage
    constexpr int LEV = 32 * RY;             // elements per level plane
    static_assert(TY > 0, "tile too small for the temporal depth");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stage = reinterpret_cast<T*>(smem_raw);
    T* lev = stage + NST * STAGE;   // level t (1..L-1) buffer b at lev + ((t-1)*2 + b) * LEV
    uint64_t* bars = reinterpret_cast<uint64_t*>(lev + (L > 1 ? (L - 1) * 2 * LEV : 0));
    __shared__ int s_abort;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int X = x0 - L + tx, Y = y0 - L + ty;
    const int kb = blockIdx.z * kc;
    const int ke = min(kb + kc, g.nz);
    const int q0 = kb - L, qlast = ke + L - 1;
    const int xpad = g.lead + x0 - L;
    const int xs = xpad & ~(A - 1);
    const int d = xpad - xs;
    const int ybox = y0 - L + 1;   // padded row of the region's first row
    const bool inside = (X >= 0 && X < g.nx && Y >= 0 && Y < g.ny);
    const bool out_tile = (tx >= L && tx < L + TX && ty >= L && ty < L + TY && inside);

    int issued = q0 - 1;   // last plane whose load thread 0 has issued
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < NST && q0 + s <= qlast; ++s) {
            mbar_arrive_expect_tx(&bars[s], STAGE * (uint32_t)sizeof(T));
            tma_load_3d(stage + s * STAGE, &map, xs, ybox, q0 + s + 1, &bars[s]);
            issued = q0 + s;
        }
    }
    int ks = 0;
    if constexpr (kIsFixed<T>) ks = fx_shift(fx, m3);
    T zb[L], zc[L];   // level t-1 (index t-1): values at planes below and at the centre
#pragma unroll
    for (int t = 0; t < L; ++t) zb[t] = zc[t] = T(0);
    unsigned long long mx = 0;

    int q = q0;
    for (; q <= qlast; ++q) {
        const int s = (q - q0) % NST;
        const uint32_t par = (uint32_t)((q - q0) / NST) & 1u;
        if (!mbar_wait_bounded(&bars[s], par, kMaxPolls)) {
            atomicExch(err, 1);
            s_abort = 1;
        }
        const int sp = (q - q0 + NST - 1) % NST;   // stage of plane q-1 (junk at q = q0)
        const T* st_prev = stage + sp * STAGE + ty * BW + tx + d;
        T up = stage[s * STAGE + ty * BW + tx + d];   // level 0 at plane q
#pragma unroll
        for (int t = 1; t <= L; ++t) {
            const int p = q - t;
            T v = T(0);
            const bool inreg = (tx >= t && tx < 32 - t && ty >= t && ty < RY - t);
            if (inreg && inside && p >= 0 && p < g.nz) {
                T xm, xp, ym, yp;
                if (t == 1) {
                    xm = st_prev[-1];
                    xp = st_prev[1];
                    ym = st_prev[-BW];
                    yp = st_prev[BW];
                } else {
                    const T* b = lev + ((t - 2) * 2 + ((q - 1) & 1)) * LEV + ty * 32 + tx;
                    xm = b[-1];
                    xp = b[1];
                    ym = b[-32];
                    yp = b[32];
                }
                v = Point<T, EXACT>::update(zc[t - 1], xm, xp, ym, yp, zb[t - 1], up, r,
                                            t == 1 ? ks : 0);
            }
            zb[t - 1] = zc[t - 1];
            zc[t - 1] = up;
            if (t < L) {
                lev[((t - 1) * 2 + (q & 1)) * LEV + ty * 32 + tx] = v;
                up = v;
            } else if (out_tile && p >= kb && p < ke) {
                dst[g.at(X, Y, p)] = v;
                if constexpr (kIsFixed<T>) {
                    const unsigned long long a = fx_abs(v);
                    mx = a > mx ? a : mx;
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
        if (tid == 0 && q > q0 && issued < qlast) {
            // the stage of plane q-1 is free: refill it with the next plane
            const int pn = issued + 1;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[sp], STAGE * (uint32_t)sizeof(T));
            tma_load_3d(stage + sp * STAGE, &map, xs, ybox, pn + 1, &bars[sp]);
            issued = pn;
        }
    }
    if (s_abort) {
        // drain: every load still in flight (planes q..issued) must land
        // before the block's shared memory goes away
        if (tid == 0) {
            for (int p = q; p <= issued; ++p) {
                const int s = (p - q0) % NST;
                (void)mbar_wait_bounded(&bars[s], (uint32_t)((p - q0) / NST) & 1u, kMaxPolls);
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
    constexpr int NST = 6;
    constexpr int A = 16 / (int)sizeof(T);
    constexpr int BW = 32 + A;
    constexpr int TX = 32 - 2 * L, TY = RY - 2 * L;
    const size_t smem = sizeof(T) * ((size_t)NST * RY * BW + (L > 1 ? (size_t)(L - 1) * 2 * 32 * RY : 0)) +
                        NST * sizeof(uint64_t);
    auto kern = k_heat_tb<T, EXACT, L, RY, NST>;
    static bool configured = false;
    if (!configured) {
        HS_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "heat: temporal-blocking kernel smem attribute");
        configured = true;
    }
    const HeatGeom& g = *c.g;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + c.kc - 1) / c.kc);
    dim3 block(32, RY, 1);
    kern<<<grid, block, smem, c.stream>>>(*c.map, (T*)c.dst, g, tb_param<T>(c), c.kc, c.fx,
                                          c.m3, c.err);
    HS_CHECK_LAUNCH("heat temporal-blocking kernel");
    return HS_OK;
}

template <typename T, bool EXACT>
int tb_dispatch_L(const TbCall& c)
{
    switch (c.L) {
    case 1: return tb_launch_t<T, EXACT, 1>(c);
    case 2: return tb_launch_t<T, EXACT, 2>(c);
    case 3: return tb_launch_t<T, EXACT, 3>(c);
    case 4: return tb_launch_t<T, EXACT, 4>(c);
    case 6: return tb_launch_t<T, EXACT, 6>(c);
    case 8: return tb_launch_t<T, EXACT, 8>(c);
    }
    return fail(HS_EINVAL, "heat: temporal depth %d not built (1, 2, 3, 4, 6 or 8)", c.L);
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
