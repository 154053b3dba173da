// Definitions shared by the heat kernels: the padded field geometry, the
// FIXED64 scale bookkeeping, and the point update in each arithmetic.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "xsum.cuh"

namespace hcg {

struct HeatGeom {
    int32_t nx, ny, nz;
    int32_t lead;    // element offset of interior x = 0 within a row
    int64_t pitch;   // elements per row
    int64_t plane;   // elements per plane = pitch * (ny + 2)
    int64_t total;   // elements per buffer = plane * (nz + 2)
    int32_t elem;    // bytes per element
    int32_t pad;
    __host__ __device__ __forceinline__ int64_t at(int i, int j, int k) const
    {
        return (int64_t)(k + 1) * plane + (int64_t)(j + 1) * pitch + lead + i;
    }
};

inline HeatGeom make_geom(int nx, int ny, int nz, size_t elem)
{
    HeatGeom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.lead = (int32_t)(32 / elem);
    const int64_t row_quant = (int64_t)(128 / elem);
    g.pitch = ((int64_t)g.lead + nx + 1 + row_quant - 1) / row_quant * row_quant;
    g.plane = g.pitch * (ny + 2);
    g.total = g.plane * (nz + 2);
    g.elem = (int32_t)elem;
    g.pad = 0;
    return g;
}

// Fixed-point bookkeeping of a FIXED64 field (device memory).  The field at
// step m has scale E_m (U = round(u 2^E_m)) and integer max M_m = max|U|, kept
// in slot m % 3.  The kernels of step m read slot m % 3, write slot (m+1) % 3
// (atomic max of their outputs, and E_{m+1}) and clear slot (m+2) % 3, which no
// kernel of step m reads -- so no kernel ever races on a slot.
struct FxSlot {
    unsigned long long maxU;   // max |U| of the field
    int32_t E;                 // scale exponent of the field
    int32_t pad;
};

struct FxState {
    unsigned long long maxabs_bits;   // bit pattern of max|u0| (non-negative doubles order like integers)
    int32_t nonfinite;                // 1 if the uploaded field held NaN or Inf
    int32_t pad;
    FxSlot slot[3];
};

// Left shift that keeps a shrinking field near full precision: the largest k
// with M 2^k < 2^57, so |S - 6U| 2^k <= 12 M 2^k < 2^61 never overflows.
__device__ __forceinline__ int fx_shift(const FxState* fx, int m3)
{
    const unsigned long long M = fx->slot[m3].maxU;
    if (M == 0) return 0;
    const int k = 57 - (64 - __clzll((long long)M));
    return k > 0 ? k : 0;
}

__device__ __forceinline__ unsigned long long fx_abs(long long v)
{
    return v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
}

// Block-wide max of the outputs into slot (m3+1) % 3; the grid leader also
// records E_{m+1} = E_m + k and clears slot (m3+2) % 3 for the next step.
template <int NT>
__device__ __forceinline__ void fx_finish(unsigned long long m, FxState* fx, int m3, int k,
                                          bool leader)
{
    __shared__ unsigned long long wmax[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) wmax[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < NT / 32; ++w) b = wmax[w] > b ? wmax[w] : b;
        // the slot only grows during a step: a block whose maximum is already
        // there skips the atomic, so thousands of blocks finishing together
        // do not queue on one address
        unsigned long long* mu = &fx->slot[(m3 + 1) % 3].maxU;
        if (b > *(volatile unsigned long long*)mu) atomicMax(mu, b);
        if (leader) {
            fx->slot[(m3 + 1) % 3].E = fx->slot[m3].E + k;
            fx->slot[(m3 + 2) % 3].maxU = 0;
        }
    }
}

// ---- the point update -------------------------------------------------------
// k is the FIXED64 rescaling shift of this step (unused by the floating types).
template <typename T, bool EXACT>
struct Point;

template <bool EXACT>
struct Point<double, EXACT> {
    // Default: the six-neighbour sum in the written order, then two fused
    // multiply-adds t = s - 6u, u' = u + r t (7 FP64 instructions per point).
    // Exact: one rounding per operation in the written order, no fusion.
    static __device__ __forceinline__ double update(double c, double xm, double xp, double ym,
                                                    double yp, double zm, double zp, double r, int)
    {
        const double s = __dadd_rn(__dadd_rn(__dadd_rn(xm, xp), __dadd_rn(ym, yp)),
                                   __dadd_rn(zm, zp));
        if (EXACT) return __dadd_rn(c, __dmul_rn(r, __dsub_rn(s, __dmul_rn(6.0, c))));
        return __fma_rn(r, __fma_rn(-6.0, c, s), c);
    }
};

template <bool EXACT>
struct Point<float, EXACT> {
    static __device__ __forceinline__ float update(float c, float xm, float xp, float ym, float yp,
                                                   float zm, float zp, float r, int)
    {
        const float s = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)),
                                  __fadd_rn(zm, zp));
        if (EXACT) return __fadd_rn(c, __fmul_rn(r, __fsub_rn(s, __fmul_rn(6.0f, c))));
        return __fmaf_rn(r, __fmaf_rn(-6.0f, c, s), c);
    }
};

template <bool EXACT>
struct Point<long long, EXACT> {
    // FIXED64: R = r 2^64 (a non-negative int64: r <= 1/6 < 1/2).  S - 6U is
    // exact; it and U are moved to the new scale by the exact shift k; then
    // t R / 2^64 is rounded to nearest (ties up): floor((t R + 2^63) / 2^64)
    // = high word of t R plus the top bit of its low word.
    static __device__ __forceinline__ long long update(long long c, long long xm, long long xp,
                                                       long long ym, long long yp, long long zm,
                                                       long long zp, long long R, int k)
    {
        const long long s = ((xm + xp) + (ym + yp)) + (zm + zp);
        const long long t = (long long)((unsigned long long)(s - 6 * c) << k);
        const long long cs = (long long)((unsigned long long)c << k);
        const long long hi = __mul64hi(t, R);
        const unsigned long long lo = (unsigned long long)t * (unsigned long long)R;
        return cs + hi + (long long)(lo >> 63);
    }
};

template <typename T>
constexpr bool kIsFixed = std::is_same<T, long long>::value;

// ---- FP64 with an exact neighbour sum (the arithmetic is in xsum.cuh) -----------------
// The heat update in this arithmetic: u' = fma(r, L 2^(e - 1080), u) with the
// exact numerator L = S - 6U, one or two FP64 instructions per point; its
// error against the exact update of the same field is below r 24 2^-57 max|u|
// plus two FP64 roundings.  e is tracked per step like the FIXED64 scale: slot
// m % 3 of an FxState holds the largest |u| bit pattern of the field at step
// m.  Fields outside the convertible range take Point<double, false>.
// The field's largest exponent field at step m: slot m % 3 of its FxState.
__device__ __forceinline__ int xs_emax(const FxState* fx, int m3)
{
    return (int)(__ldcg(&fx->slot[m3].maxU) >> 52);
}

// The whole update from seven doubles (kernels that convert per point).
__device__ __forceinline__ double xs_point(double c, double xm, double xp, double ym, double yp,
                                           double zm, double zp, double r, int emax)
{
    if (xs_native(emax, r)) return Point<double, false>::update(c, xm, xp, ym, yp, zm, zp, r, 0);
    auto f = [emax](double v) { return xs_fix(__double_as_longlong(v), emax); };
    const long long L = xs_numerator(f(c), f(xm), f(xp), f(ym), f(yp), f(zm), f(zp));
    return xs_apply<false>(c, L, r, 0.0, emax);
}


// V consecutive x points per thread, moved as one 16-byte vector.
template <typename T>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int V = 4;
    using type = float4;
};
template <>
struct Vec<double> {
    static constexpr int V = 2;
    using type = double2;
};
template <>
struct Vec<long long> {
    static constexpr int V = 2;
    using type = longlong2;
};

template <typename T>
__device__ __forceinline__ void ld_vec(const T* p, T (&o)[Vec<T>::V])
{
    const typename Vec<T>::type v = *reinterpret_cast<const typename Vec<T>::type*>(p);
    if constexpr (Vec<T>::V == 4) {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    } else {
        o[0] = v.x;
        o[1] = v.y;
    }
}

template <typename T>
__device__ __forceinline__ void st_vec(T* p, const T (&o)[Vec<T>::V])
{
    typename Vec<T>::type v;
    if constexpr (Vec<T>::V == 4) {
        v.x = o[0];
        v.y = o[1];
        v.z = o[2];
        v.w = o[3];
    } else {
        v.x = o[0];
        v.y = o[1];
    }
    *reinterpret_cast<typename Vec<T>::type*>(p) = v;
}

// Arithmetic of a heat handle.
// A_F64: every operation on the FP64 pipe; A_F64_XS: FP64 fields with the exact
// integer neighbour sum and one FP64 FMA per point (above).
enum Arith { A_F64 = 0, A_F64_EXACT = 1, A_F32 = 2, A_FX64 = 3, A_F64_XS = 4 };

// One launch of the temporally blocked kernel (heat_tb.cu).
struct TbCall {
    int arith;
    int L;                   // steps in this pass
    int kc;                  // k-planes per block
    const CUtensorMap* map;  // tensor map of the source buffer
    void* dst;
    const HeatGeom* g;
    double r;
    long long R;             // FIXED64: r 2^64
    FxState* fx;
    int m3;
    int* err;                // device error word (1 = a bounded wait ran out)
    cudaStream_t stream;
    uint32_t box[2];         // box the map was encoded with (checked against the kernel's)
};

template <typename T>
inline T tb_param(const TbCall& c)
{
    if constexpr (std::is_same<T, long long>::value)
        return c.R;
    else
        return (T)c.r;
}

int tb_launch(const TbCall& c);
// TMA box (elements x rows) the temporally blocked kernel loads for an
// arithmetic and a grid nx points wide.
int tb_box(int arith, int nx, uint32_t* box_x, uint32_t* box_y);

// One launch of the streaming Interior kernel (heat_stream.cu): one step over
// the k-planes [kbeg, kend).
struct StreamCall {
    int arith;
    int kbeg, kend;          // planes to update
    int kc;                  // k-planes per block
    const CUtensorMap* map;  // stream tensor map of the source buffer
    void* dst;
    const HeatGeom* g;
    double r;
    long long R;
    FxState* fx;
    int m3;
    int* err;
    cudaStream_t stream;
    uint32_t box[2];         // box the map was encoded with (checked against the kernel's)
};

template <typename T>
inline T stream_param(const StreamCall& c)
{
    if constexpr (std::is_same<T, long long>::value)
        return c.R;
    else
        return (T)c.r;
}

int stream_launch(const StreamCall& c);
// TMA box (elements x rows) the streaming kernel loads for an arithmetic.
int stream_box(int arith, uint32_t* box_x, uint32_t* box_y);
// Rows of the streaming kernels' tiles: 16 for k_heat_stream (a thread per
// row), kXsRows for the exact-sum FP64 kernel (kXsRowsPerThread rows per
// thread, a ring of kXsStages staged planes).
constexpr int kStreamRowsHost = 16;
constexpr int kXsRows = 8;
constexpr int kXsRowsPerThread = 2;
constexpr int kXsStages = 4;
inline int stream_rows_for(int arith) { return arith == A_F64_XS ? kXsRows : kStreamRowsHost; }

// One launch of a variable-coefficient kernel (heat_vk.cu).
struct VkCall {
    int part;                // 0: Interior (planes 1..nz-2), 1: Boundary (planes 0, nz-1)
    int f64;                 // 1: FP64, 0: FP32
    const void* src;
    void* dst;
    void* kap;               // FP32: kappa on every padded node; FP64: the three face
                             // sums of kappa (x, y, z arrays of g.total elements each)
    void* fdt;               // dt f on the interior
    const HeatGeom* g;
    double bx, by, bz;       // dt / (2 h_d^2)
    int kchunk;
    cudaStream_t stream;
    FxState* fx;             // FP64: the per-step maxima of the exact-sum form
                             // (nullptr: the FP64 form, no maxima)
    int m3;                  // slot of the current field in fx
    int* face_off;           // vk_init, FP64: device word set to 1 if a face sum lies outside [1, 2)
};
int vk_init(const VkCall& c, double dt);
int vk_launch(const VkCall& c);

// What the batched kernel needs to know about a heat handle (heat.cu).
struct HeatBatchView {
    HeatGeom g;
    void* buf[2];
    double r;
    int arith;
    int cur;
    int vk;                  // 1 for the variable-coefficient problem
    FxState* fx;             // A_F64_XS: the per-step maxima
    int m3;                  // A_F64_XS: slot of the current field
    cudaStream_t stream;
};
int heat_batch_view(hs_heat_t h, HeatBatchView* v);
// Records that a batch advanced the handle by `steps` steps.
int heat_batch_advance(hs_heat_t h, int64_t steps);

// Thread rows of the temporally blocked kernel's block and rows per thread:
// its region is kTbThreadRows kTbRowsPerThread rows high (the tile that plus
// the halo of L rows on each side).
constexpr int kTbThreadRows = 12;
constexpr int kTbRowsPerThread = 2;
// Output tile (x columns, y rows) of the temporally blocked kernel.
void tb_tile(int arith, int L, int nx, int* tx, int* ty);

}  // namespace hcg
