// Explicit 7-point heat stepping on one GPU: the Interior and Boundary kernels
// of Algorithms INTERIOR and BOUNDARY, the full-step kernel of Algorithm
// COMPUTE_SINGLE_GPU, and the heat_* entry points of the C ABI.
//
// Update (Section 4, Eq. 4 with kappa = 1 and f = 0, r = alpha dt / h^2):
//     u' = u + r * (((u[i-1] + u[i+1]) + (u[j-1] + u[j+1])) + (u[k-1] + u[k+1]) - 6 u)
// on interior points; the boundary layer stays zero (Dirichlet).
//
// Arithmetic, chosen per handle:
//   FP64      (default) FP64 fields, the six-neighbour sum and S - 6u exact in
//             64-bit fixed point on the field's current scale, rounded back to
//             a double and applied with one FP64 fused multiply-add
//             (heat_common.cuh);
//   FP64 pipe (HS_FP64_PIPE, and temporal blocking) the update in double
//             precision with two fused multiply-adds;
//   FP64 exact one rounding per operation in the written order (no FMA), the
//             oracle's rounding sequence bit for bit;
//   FP32      the update in single precision (storage and arithmetic);
//   FIXED64   FP64 interface, field held as 64-bit fixed-point integers
//             U = round(u 2^E).  The six-neighbour sum and S - 6U are exact;
//             r is held as R = r 2^64 (exactly for r >= 2^-11); the one rounding
//             per point is of R (S - 6U) / 2^64 to the nearest integer.  E is set
//             at upload from max|u0| so that 12 max|U| < 2^61, and grows during
//             the run: every step's kernels track max|U| of their output, and
//             when the field has shrunk the next step shifts all values left by
//             k bits (exact), keeping max|U| in [2^56, 2^57) -- about 57
//             significant bits relative to the current maximum.  For r <= 1/6
//             the update is a convex combination, so |U| never grows and
//             nothing overflows.  GB300's integer pipes run about 60x the rate
//             of its FP64 pipe, which makes this the FP64-accuracy form that is
//             bound by HBM rather than by FP64 issue.
//
// Layout in HBM: each field buffer holds (nz+2) planes of (ny+2) rows.  A row
// has `pitch` elements (a multiple of 128 bytes); interior x = 0 sits at
// element `lead` (32 bytes in), so interior rows start 32-byte aligned, and
// the x-boundary cells sit at lead-1 and lead+nx.  Planes 0 and nz+1, rows 0
// and ny+1 and the x-boundary cells hold the Dirichlet zeros in both buffers
// and are never written after creation, so a pointer swap keeps them intact.
#include <cmath>
#include <vector>
#include <cstdlib>
#include <new>
#include <type_traits>

#include "heat_common.cuh"
#include "tma.cuh"

namespace hcg {

// ---- Interior kernel ----------------------------------------------------------
// One thread per (i, j) column marches up a chunk of k-planes, keeping the
// values at k-1, k and k+1 in registers (rotated each plane); the four
// in-plane neighbours come through the read-only cache, where the block's
// neighbouring columns have just loaded them.
constexpr int kBX = 32, kBY = 8;

template <typename T, bool EXACT>
__global__ void __launch_bounds__(kBX* kBY)
    k_heat_interior(const T* __restrict__ src, T* __restrict__ dst, HeatGeom g, T r, int kbeg,
                    int kend, int kchunk, FxState* fx, int m3)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = kbeg + (int)blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, kend);
    int ks = 0;
    if constexpr (kIsFixed<T>) ks = fx_shift(fx, m3);
    unsigned long long mx = 0;
    if (i < g.nx && j < g.ny && k0 < k1) {
        const int64_t P = g.plane, Y = g.pitch;
        int64_t c = g.at(i, j, k0);
        T below = __ldg(src + c - P);
        T cur = __ldg(src + c);
        for (int k = k0; k < k1; ++k) {
            const T above = __ldg(src + c + P);
            const T xm = __ldg(src + c - 1), xp = __ldg(src + c + 1);
            const T ym = __ldg(src + c - Y), yp = __ldg(src + c + Y);
            const T v = Point<T, EXACT>::update(cur, xm, xp, ym, yp, below, above, r, ks);
            dst[c] = v;
            if constexpr (kIsFixed<T>) {
                const unsigned long long a = fx_abs(v);
                mx = a > mx ? a : mx;
            }
            below = cur;
            cur = above;
            c += P;
        }
    }
    if constexpr (kIsFixed<T>)
        fx_finish<kBX * kBY>(mx, fx, m3, ks,
                             blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

// ---- Boundary kernel ------------------------------------------------------------
// The outermost interior k-planes (k = 0 and k = nz-1): the planes a k-split
// across devices would exchange.  blockIdx.z selects the plane.
template <typename T, bool EXACT>
__global__ void __launch_bounds__(kBX* kBY)
    k_heat_boundary(const T* __restrict__ src, T* __restrict__ dst, HeatGeom g, T r, FxState* fx,
                    int m3)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    int ks = 0;
    if constexpr (kIsFixed<T>) ks = fx_shift(fx, m3);
    unsigned long long mx = 0;
    if (i < g.nx && j < g.ny) {
        const int k = (blockIdx.z == 0) ? 0 : g.nz - 1;
        const int64_t P = g.plane, Y = g.pitch;
        const int64_t c = g.at(i, j, k);
        const T v = Point<T, EXACT>::update(__ldg(src + c), __ldg(src + c - 1), __ldg(src + c + 1),
                                            __ldg(src + c - Y), __ldg(src + c + Y),
                                            __ldg(src + c - P), __ldg(src + c + P), r, ks);
        dst[c] = v;
        if constexpr (kIsFixed<T>) mx = fx_abs(v);
    }
    if constexpr (kIsFixed<T>)
        fx_finish<kBX * kBY>(mx, fx, m3, ks,
                             blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

// ---- full-step kernel -------------------------------------------------------------
// Algorithm COMPUTE_SINGLE_GPU: one thread per interior point over the whole
// box, all seven values loaded directly.  A separate code path from the
// Interior/Boundary pair, used to cross-check it bit for bit.
template <typename T, bool EXACT>
__global__ void __launch_bounds__(256)
    k_heat_full(const T* __restrict__ src, T* __restrict__ dst, HeatGeom g, T r, FxState* fx,
                int m3)
{
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const int64_t P = g.plane, Y = g.pitch;
    int ks = 0;
    if constexpr (kIsFixed<T>) ks = fx_shift(fx, m3);
    unsigned long long mx = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const int64_t jk = t / g.nx;
        const int j = (int)(jk % g.ny);
        const int k = (int)(jk / g.ny);
        const int64_t c = g.at(i, j, k);
        const T v = Point<T, EXACT>::update(src[c], src[c - 1], src[c + 1], src[c - Y], src[c + Y],
                                            src[c - P], src[c + P], r, ks);
        dst[c] = v;
        if constexpr (kIsFixed<T>) {
            const unsigned long long a = fx_abs(v);
            mx = a > mx ? a : mx;
        }
    }
    if constexpr (kIsFixed<T>) fx_finish<256>(mx, fx, m3, ks, blockIdx.x == 0);
}

// ---- Boundary and full-step kernels in the FP64 exact-sum arithmetic ------------------
// Per point the seven doubles are converted, then updated as in the streaming
// Interior kernel (xs_point); every output joins the step's maximum.
__global__ void __launch_bounds__(kBX* kBY)
    k_heat_boundary_xs(const double* __restrict__ src, double* __restrict__ dst, HeatGeom g, double r,
                       FxState* fx, int m3)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int emax = xs_emax(fx, m3);
    unsigned mx = 0;
    if (i < g.nx && j < g.ny) {
        const int k = (blockIdx.z == 0) ? 0 : g.nz - 1;
        const int64_t P = g.plane, Y = g.pitch;
        const int64_t c = g.at(i, j, k);
        const double v = xs_point(__ldg(src + c), __ldg(src + c - 1), __ldg(src + c + 1),
                                  __ldg(src + c - Y), __ldg(src + c + Y), __ldg(src + c - P),
                                  __ldg(src + c + P), r, emax);
        dst[c] = v;
        mx = xs_abs_hi(v);
    }
    fx_finish<kBX * kBY>((unsigned long long)mx << 32, fx, m3, 0,
                         blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
}

__global__ void __launch_bounds__(256)
    k_heat_full_xs(const double* __restrict__ src, double* __restrict__ dst, HeatGeom g, double r,
                   FxState* fx, int m3)
{
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const int64_t P = g.plane, Y = g.pitch;
    const int emax = xs_emax(fx, m3);
    unsigned mx = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const int64_t jk = t / g.nx;
        const int j = (int)(jk % g.ny);
        const int k = (int)(jk / g.ny);
        const int64_t c = g.at(i, j, k);
        const double v = xs_point(src[c], src[c - 1], src[c + 1], src[c - Y], src[c + Y], src[c - P],
                                  src[c + P], r, emax);
        dst[c] = v;
        const unsigned a = xs_abs_hi(v);
        mx = a > mx ? a : mx;
    }
    fx_finish<256>((unsigned long long)mx << 32, fx, m3, 0, blockIdx.x == 0);
}

// ---- FIXED64 conversions (at upload and read only) --------------------------------
// Grid-stride over the interior points of a padded buffer.
__global__ void __launch_bounds__(256) k_fx_maxabs(const double* __restrict__ buf, HeatGeom g,
                                                   FxState* st)
{
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    unsigned long long m = 0;
    int bad = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const int64_t jk = t / g.nx;
        const double v = buf[g.at(i, (int)(jk % g.ny), (int)(jk / g.ny))];
        if (!isfinite(v)) bad = 1;
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->maxabs_bits, m);
        atomicMax(&st->slot[0].maxU, m);   // the exact-sum FP64 arithmetic's step-0 maximum
        if (bad) atomicOr(&st->nonfinite, 1);
    }
}

// E such that 12 max|u| 2^E < 2^61: with 12 M = f 2^e, f in [0.5, 1), E = 61 - e.
__device__ __forceinline__ int fx_scale_exp(const FxState* st)
{
    const double m = __longlong_as_double((long long)st->maxabs_bits);
    if (st->nonfinite || !(m > 0.0)) return 0;
    int e = 0;
    (void)frexp(12.0 * m, &e);
    return 61 - e;
}

// In place: the interior doubles of buf become round(u 2^E); slot 0 describes
// the encoded field, slot 1 is cleared for the first step.
__global__ void __launch_bounds__(256) k_fx_encode(double* __restrict__ buf, HeatGeom g,
                                                   FxState* st)
{
    const int E = fx_scale_exp(st);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double m = __longlong_as_double((long long)st->maxabs_bits);
        st->slot[0].E = E;
        st->slot[0].maxU = (st->nonfinite || !(m > 0.0))
                               ? 0ull
                               : (unsigned long long)__double2ll_rn(scalbn(m, E));
        st->slot[1].maxU = 0;
    }
    long long* out = reinterpret_cast<long long*>(buf);
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const int64_t jk = t / g.nx;
        const int64_t c = g.at(i, (int)(jk % g.ny), (int)(jk / g.ny));
        const double v = buf[c];
        out[c] = isfinite(v) ? __double2ll_rn(scalbn(v, E)) : 0;
    }
}

// The interior of src (fixed point, the field of slot m3) as doubles u = U 2^-E in dst.
__global__ void __launch_bounds__(256) k_fx_decode(const long long* __restrict__ src,
                                                   double* __restrict__ dst, HeatGeom g,
                                                   const FxState* st, int m3)
{
    const int E = st->slot[m3].E;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const int64_t jk = t / g.nx;
        const int64_t c = g.at(i, (int)(jk % g.ny), (int)(jk / g.ny));
        dst[c] = scalbn(__ll2double_rn(src[c]), -E);
    }
}

}  // namespace hcg

using namespace hcg;

struct hs_heat {
    HeatGeom g;
    int32_t dtype;
    Arith arith;
    size_t elem;
    double r;
    long long R;       // FIXED64: r 2^64
    uint32_t flags;
    cudaStream_t stream;
    void* buf[2];
    bool owns_buf;     // false: buf[] are the caller's dev_buf0/dev_buf1
    FxState* fx;       // FIXED64 only
    int* err;          // device error word: 1 when a bounded device wait ran out
    int cur;           // buffer holding the current time level
    int64_t steps;     // steps since the last upload
    int64_t fxseq;     // fields produced since the last upload (FIXED64 slot = fxseq % 3)
    int kchunk;        // planes per Interior-kernel block
    int tdepth;        // steps per pass of the temporally blocked kernel (1: Interior + Boundary)
    int kc_tb;         // k-planes per block of the temporally blocked kernel
    CUtensorMap maps[2];   // TMA maps of the two buffers (temporal blocking)
    CUtensorMap smaps[2];  // TMA maps of the two buffers (streaming Interior kernel)
    uint32_t tbox[2];      // box of maps[]
    uint32_t sbox[2];      // box of smaps[]
    int kc_stream;         // k-planes per block of the streaming Interior kernel
    void* kap;             // HS_VARKAPPA: FP32 kappa on every padded node, FP64 its three face sums
    void* fdt;             // HS_VARKAPPA: dt f on the interior
    double vbx, vby, vbz;  // HS_VARKAPPA: dt / (2 h_d^2)
    // Large grids run each step's Boundary kernel on a side stream, beside the
    // Interior kernel: forked from `stream` after the previous step (ev_fork)
    // and joined back before the next one (ev_join).  Null: one stream.
    cudaStream_t bstream;
    cudaEvent_t ev_fork, ev_join;
    // heat_time_interior: event pairs around the Interior launches of heat_step
    bool timing;
    std::vector<cudaEvent_t> tev;   // 2 per recorded launch, reused
    size_t tev_used;                // pairs recorded since the last heat_interior_time
};

namespace {

constexpr int64_t kForkMinPoints = (int64_t)1 << 22;
constexpr size_t kMaxTimedLaunches = 8192;   // event pairs a handle keeps for heat_interior_time

constexpr uint32_t kKnownFlags =
    HS_ALLOW_UNSTABLE | HS_EXACT_ROUNDING | HS_SCHED_FULL | HS_FIXED64 | HS_VARKAPPA | HS_FP64_PIPE;
constexpr double kKappaMax = 0.95;   // max of 0.5 + 0.45 sin sin sin (Section 4, Eq. 2)

int check_desc(const hs_heat_desc* d)
{
    if (!d) return fail(HS_EINVAL, "heat: desc is NULL");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1)
        return fail(HS_EINVAL, "heat: grid %d x %d x %d must have at least one interior point per axis",
                    d->nx, d->ny, d->nz);
    if (d->nx > (1 << 30) || d->ny > 65535 * kBY || d->nz > (1 << 30))
        return fail(HS_EINVAL, "heat: grid axis too large (ny <= %d)", 65535 * kBY);
    if (!std::isfinite(d->r) || d->r < 0.0)
        return fail(HS_EINVAL, "heat: r = %g must be finite and >= 0", d->r);
    if (d->flags & ~kKnownFlags) return fail(HS_EINVAL, "heat: unknown flag bits 0x%x", d->flags);
    if (d->dtype != HS_F64 && d->dtype != HS_F32)
        return fail(HS_EINVAL, "heat: dtype %d is not HS_F64 or HS_F32", d->dtype);
    if ((d->flags & HS_EXACT_ROUNDING) && d->dtype != HS_F64)
        return fail(HS_EINVAL, "heat: HS_EXACT_ROUNDING applies to HS_F64 only");
    if ((d->flags & HS_FP64_PIPE) && (d->dtype != HS_F64 || (d->flags & HS_FIXED64)))
        return fail(HS_EINVAL, "heat: HS_FP64_PIPE applies to plain HS_F64 only");
    if (d->flags & HS_FIXED64) {
        if (d->dtype != HS_F64) return fail(HS_EINVAL, "heat: HS_FIXED64 applies to HS_F64 only");
        if (d->flags & HS_EXACT_ROUNDING)
            return fail(HS_EINVAL, "heat: HS_FIXED64 and HS_EXACT_ROUNDING exclude each other");
        if (d->flags & HS_ALLOW_UNSTABLE)
            return fail(HS_EINVAL, "heat: HS_FIXED64 needs r <= 1/6 (a growing field would overflow)");
    }
    if (d->tdepth < 0 || d->tdepth > 4)
        return fail(HS_EINVAL, "heat: tdepth %d not in {0, 1, 2, 3, 4}", d->tdepth);
    if ((d->flags & HS_SCHED_FULL) && d->tdepth > 1)
        return fail(HS_EINVAL, "heat: HS_SCHED_FULL runs one step per pass (tdepth 0 or 1)");
    if (d->flags & HS_VARKAPPA) {
        if (d->flags & (HS_FIXED64 | HS_EXACT_ROUNDING | HS_SCHED_FULL))
            return fail(HS_EINVAL, "heat: HS_VARKAPPA runs plain FP64 or FP32, Interior + Boundary");
        if (d->tdepth > 1) return fail(HS_EINVAL, "heat: HS_VARKAPPA runs one step per pass");
        // the update stays a convex combination (without the source) while
        // dt (kappa_max) sum_d 2/h_d^2 <= 1, which r = dt/h_min^2 <= 1/(6 kappa_max) ensures
        if (d->r > 1.0 / (6.0 * kKappaMax) && !(d->flags & HS_ALLOW_UNSTABLE))
            return fail(HS_EUNSTABLE, "heat: r = %.17g exceeds 1/(6 kappa_max) = %.6g", d->r,
                        1.0 / (6.0 * kKappaMax));
        return HS_OK;
    }
    // Three-dimensional stability of the explicit update: r <= 1/6.
    if (d->r > 1.0 / 6.0 && !(d->flags & HS_ALLOW_UNSTABLE))
        return fail(HS_EUNSTABLE, "heat: r = %.17g exceeds the stability bound 1/6", d->r);
    return HS_OK;
}

size_t elem_size(int dtype) { return dtype == HS_F64 ? sizeof(double) : sizeof(float); }

// Caller-owned time-level buffers: both or neither, distinct, not
// overlapping, 256-byte aligned (TMA and the 16-byte vector accesses need
// less; every CUDA allocator gives this).
int check_user_buffers(const hs_heat_desc* d, size_t bytes)
{
    if (!d->dev_buf0 && !d->dev_buf1) return HS_OK;
    if (!d->dev_buf0 || !d->dev_buf1)
        return fail(HS_EINVAL, "heat: give both dev_buf0 and dev_buf1, or neither");
    const uintptr_t a = reinterpret_cast<uintptr_t>(d->dev_buf0), b = reinterpret_cast<uintptr_t>(d->dev_buf1);
    if ((a | b) & 255) return fail(HS_EINVAL, "heat: dev_buf0 and dev_buf1 must be 256-byte aligned");
    if ((a < b ? b - a : a - b) < bytes)
        return fail(HS_EINVAL, "heat: dev_buf0 and dev_buf1 overlap (each needs %zu bytes)", bytes);
    return HS_OK;
}

// Plain FP64 runs the exact-sum arithmetic, except where a kernel has only the
// FP64-pipe form: temporal blocking and the variable-coefficient problem.
Arith pick_arith(const hs_heat_desc* d)
{
    const int depth = d->tdepth ? d->tdepth : 1;
    if (d->flags & HS_FIXED64) return A_FX64;
    if (d->flags & HS_EXACT_ROUNDING) return A_F64_EXACT;
    if (d->dtype == HS_F32) return A_F32;
    if ((d->flags & (HS_FP64_PIPE | HS_VARKAPPA)) || depth > 1) return A_F64;
    return A_F64_XS;
}

int pick_kchunk(const HeatGeom& g, uint32_t flags = 0, int dtype = HS_F64)
{
    // the FP32 variable-kappa kernel waits on its loads: short chunks (more
    // blocks in flight) measured 340 GLUP/s at 8 planes against 265 at the
    // 102 planes of the rule below (510^3)
    if ((flags & HS_VARKAPPA) && dtype == HS_F32) return g.nz > 2 ? std::min(8, g.nz - 2) : 1;
    // the FP64 variable-kappa kernels: 32-plane chunks (77.0 GLUP/s at 510^3
    // against 75.8 with the 102 of the rule below)
    if (flags & HS_VARKAPPA) return g.nz > 2 ? std::min(32, g.nz - 2) : 1;
    const int64_t blocks_xy = (int64_t)((g.nx + kBX - 1) / kBX) * ((g.ny + kBY - 1) / kBY);
    const int64_t target = (int64_t)kNumSMs * 8 * 4;   // about four waves of 8 blocks per SM
    const int64_t nzi = g.nz > 2 ? g.nz - 2 : 1;
    int64_t chunks = (target + blocks_xy - 1) / blocks_xy;
    if (chunks < 1) chunks = 1;
    int64_t kc = (nzi + chunks - 1) / chunks;
    if (kc < 8) kc = 8;
    if (kc > nzi) kc = nzi;
    return (int)kc;
}

template <typename T, bool EXACT>
int launch_interior_t(hs_heat* h, T param)
{
    const HeatGeom& g = h->g;
    if (g.nz < 3) return HS_OK;   // no plane lies strictly between the boundary planes
    const int kbeg = 1, kend = g.nz - 1;
    const int nchunks = (kend - kbeg + h->kchunk - 1) / h->kchunk;
    dim3 block(kBX, kBY, 1);
    dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, nchunks);
    k_heat_interior<T, EXACT><<<grid, block, 0, h->stream>>>(
        (const T*)h->buf[h->cur], (T*)h->buf[1 - h->cur], g, param, kbeg, kend, h->kchunk, h->fx,
        (int)(h->fxseq % 3));
    HS_CHECK_LAUNCH("heat interior kernel");
    return HS_OK;
}

template <typename T, bool EXACT>
int launch_boundary_t(hs_heat* h, T param, cudaStream_t s)
{
    const HeatGeom& g = h->g;
    dim3 block(kBX, kBY, 1);
    dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, g.nz >= 2 ? 2 : 1);
    k_heat_boundary<T, EXACT><<<grid, block, 0, s>>>(
        (const T*)h->buf[h->cur], (T*)h->buf[1 - h->cur], g, param, h->fx, (int)(h->fxseq % 3));
    HS_CHECK_LAUNCH("heat boundary kernel");
    return HS_OK;
}

template <typename T, bool EXACT>
int launch_full_t(hs_heat* h, T param)
{
    const HeatGeom& g = h->g;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)kNumSMs * 64) blocks = (int64_t)kNumSMs * 64;
    k_heat_full<T, EXACT><<<(unsigned)blocks, 256, 0, h->stream>>>(
        (const T*)h->buf[h->cur], (T*)h->buf[1 - h->cur], g, param, h->fx, (int)(h->fxseq % 3));
    HS_CHECK_LAUNCH("heat full-step kernel");
    return HS_OK;
}

enum Part { P_INTERIOR, P_BOUNDARY, P_FULL };

// The Interior kernel: planes 1 .. nz-2, staged through shared memory by TMA.
int launch_stream_interior(hs_heat* h)
{
    if (h->g.nz < 3) return HS_OK;   // no plane lies strictly between the boundary planes
    StreamCall c;
    c.arith = h->arith;
    c.kbeg = 1;
    c.kend = h->g.nz - 1;
    c.kc = h->kc_stream;
    c.map = &h->smaps[h->cur];
    c.dst = h->buf[1 - h->cur];
    c.g = &h->g;
    c.r = h->r;
    c.R = h->R;
    c.fx = h->fx;
    c.m3 = (int)(h->fxseq % 3);
    c.err = h->err;
    c.stream = h->stream;
    c.box[0] = h->sbox[0];
    c.box[1] = h->sbox[1];
    return stream_launch(c);
}

int launch_part_xs(hs_heat* h, Part p, cudaStream_t s)
{
    const HeatGeom& g = h->g;
    const double* src = (const double*)h->buf[h->cur];
    double* dst = (double*)h->buf[1 - h->cur];
    const int m3 = (int)(h->fxseq % 3);
    if (p == P_INTERIOR) return launch_stream_interior(h);
    if (p == P_BOUNDARY) {
        dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, g.nz >= 2 ? 2 : 1);
        k_heat_boundary_xs<<<grid, dim3(kBX, kBY, 1), 0, s>>>(src, dst, g, h->r, h->fx, m3);
        HS_CHECK_LAUNCH("heat boundary kernel (FP64 exact sum)");
        return HS_OK;
    }
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)kNumSMs * 64) blocks = (int64_t)kNumSMs * 64;
    k_heat_full_xs<<<(unsigned)blocks, 256, 0, h->stream>>>(src, dst, g, h->r, h->fx, m3);
    HS_CHECK_LAUNCH("heat full-step kernel (FP64 exact sum)");
    return HS_OK;
}

template <typename T, bool EXACT>
int launch_part(hs_heat* h, Part p, T param, cudaStream_t s)
{
    // FP64 is bound by the FP64 pipe, where the register z-march issues the
    // fewest extra instructions; the HBM-bound arithmetics stream through TMA.
    if (p == P_INTERIOR)
        return std::is_same<T, double>::value ? launch_interior_t<T, EXACT>(h, param)
                                              : launch_stream_interior(h);
    if (p == P_BOUNDARY) return launch_boundary_t<T, EXACT>(h, param, s);
    return launch_full_t<T, EXACT>(h, param);
}

int vk_part(hs_heat* h, Part p, cudaStream_t s)
{
    VkCall c;
    c.part = (p == P_INTERIOR) ? 0 : 1;
    c.f64 = h->dtype == HS_F64;
    c.src = h->buf[h->cur];
    c.dst = h->buf[1 - h->cur];
    c.kap = h->kap;
    c.fdt = h->fdt;
    c.g = &h->g;
    c.bx = h->vbx;
    c.by = h->vby;
    c.bz = h->vbz;
    c.kchunk = h->kchunk;
    c.stream = s;
    c.fx = h->fx;   // FP64 only
    c.m3 = (int)(h->fxseq % 3);
    return vk_launch(c);
}

// Launches one part of a step.  The Boundary kernel goes to stream s (the
// handle's own stream unless given); the other parts always to h->stream.
int do_part(hs_heat* h, Part p, cudaStream_t s = nullptr)
{
    if (!s || p != P_BOUNDARY) s = h->stream;
    if (h->flags & HS_VARKAPPA) return vk_part(h, p, s);
    switch (h->arith) {
    case A_F64: return launch_part<double, false>(h, p, h->r, s);
    case A_F64_EXACT: return launch_part<double, true>(h, p, h->r, s);
    case A_F32: return launch_part<float, false>(h, p, (float)h->r, s);
    case A_FX64: return launch_part<long long, false>(h, p, h->R, s);
    case A_F64_XS: return launch_part_xs(h, p, s);
    }
    return fail(HS_EINVAL, "heat: unknown arithmetic");
}

// The Interior part of a heat_step step, between a pair of timing events on
// the handle's stream while heat_time_interior is on.
int timed_interior(hs_heat* h)
{
    // past kMaxTimedLaunches unread records the launches go untimed
    if (!h->timing || h->tev_used >= kMaxTimedLaunches) return do_part(h, P_INTERIOR);
    const size_t i = 2 * h->tev_used;
    while (h->tev.size() < i + 2) {
        cudaEvent_t e;
        HS_TRY_CUDA(cudaEventCreate(&e), "heat_step: timing event");
        h->tev.push_back(e);
    }
    HS_TRY_CUDA(cudaEventRecord(h->tev[i], h->stream), "heat_step: timing event");
    const int rc = do_part(h, P_INTERIOR);
    if (rc != HS_OK) return rc;
    HS_TRY_CUDA(cudaEventRecord(h->tev[i + 1], h->stream), "heat_step: timing event");
    h->tev_used += 1;
    return HS_OK;
}

// Temporal depth when the descriptor leaves it to the library.  FP32 is bound
// by HBM, and two steps per pass move half the bytes of one: at 512^3 the
// L = 2 pass runs 880 GLUP/s against 761 for one step per pass, while depths 3
// and 4 (one block per SM) fall below one step per pass.  FP64 and FIXED64 are
// bound by the FP64 pipe and the integer pipes: blocking saves only bytes and
// adds the halo's work.  The variable-coefficient problem runs one step per
// pass.
int default_tdepth(Arith a, uint32_t flags)
{
    return (a == A_F32 && !(flags & HS_VARKAPPA)) ? 2 : 1;
}

int pick_kc_tb(const HeatGeom& g, int arith, int L)
{
    int TX = 0, TY = 0;
    tb_tile(arith, L, g.nx, &TX, &TY);
    const int64_t tiles = (int64_t)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    // about six waves of two blocks per SM: 35-plane chunks at 512^3 in FP32,
    // measured ahead of 27 (eight waves) and 52 or 64 (three or four)
    const int64_t target = (int64_t)kNumSMs * 12;
    int64_t chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int64_t kc = (g.nz + chunks - 1) / chunks;
    const int64_t floor_kc = 8 * L;                    // keep the z halo (2L planes) small
    if (kc < floor_kc) kc = floor_kc;
    if (kc > g.nz) kc = g.nz;
    return (int)kc;
}

int pick_kc_stream(const HeatGeom& g, int arith)
{
    const int tw = 512 / (int)g.elem;                  // tile width: 32 threads x one 16-byte vector
    const int ry = stream_rows_for(arith);
    const int64_t tiles = (int64_t)((g.nx + tw - 1) / tw) * ((g.ny + ry - 1) / ry);
    // about four waves of 3 blocks of 16 rows per SM; the exact-sum kernel (8 rows,
    // 8 resident blocks of 128 threads per SM) gets 64 blocks per SM, about 8
    // waves of 27-plane chunks at 512^3 -- measured ahead of 4 waves of longer
    // chunks and 12 waves of shorter ones
    const int64_t target = (int64_t)kNumSMs * (arith == A_F64_XS ? 16 : 3) * 4;
    const int64_t planes = g.nz > 2 ? g.nz - 2 : 1;
    int64_t chunks = (target + tiles - 1) / tiles;
    if (chunks < 1) chunks = 1;
    int64_t kc = (planes + chunks - 1) / chunks;
    if (kc < 8) kc = 8;
    if (kc > planes) kc = planes;
    return (int)kc;
}

// One pass of L steps with the temporally blocked kernel.
int tb_pass(hs_heat* h, int L)
{
    TbCall c;
    c.arith = h->arith;
    c.L = L;
    c.kc = pick_kc_tb(h->g, h->arith, L);
    c.map = &h->maps[h->cur];
    c.dst = h->buf[1 - h->cur];
    c.g = &h->g;
    c.r = h->r;
    c.R = h->R;
    c.fx = h->fx;
    c.m3 = (int)(h->fxseq % 3);
    c.err = h->err;
    c.stream = h->stream;
    c.box[0] = h->tbox[0];
    c.box[1] = h->tbox[1];
    int rc = tb_launch(c);
    if (rc != HS_OK) return rc;
    h->cur = 1 - h->cur;
    h->steps += L;
    h->fxseq += 1;
    return HS_OK;
}

// Copies between a dense nx*ny*nz array and the interior of a padded buffer.
int copy_interior(hs_heat* h, void* buf, const void* dense, void* dense_out, cudaMemcpyKind kind)
{
    const HeatGeom& g = h->g;
    const size_t e = h->elem;
    cudaMemcpy3DParms p = {};
    p.extent = make_cudaExtent((size_t)g.nx * e, (size_t)g.ny, (size_t)g.nz);
    cudaPitchedPtr padded = make_cudaPitchedPtr(buf, (size_t)g.pitch * e, (size_t)g.pitch,
                                                (size_t)(g.ny + 2));
    cudaPos inner = make_cudaPos((size_t)g.lead * e, 1, 1);
    if (dense) {   // dense -> padded
        p.srcPtr = make_cudaPitchedPtr(const_cast<void*>(dense), (size_t)g.nx * e, (size_t)g.nx,
                                       (size_t)g.ny);
        p.dstPtr = padded;
        p.dstPos = inner;
    } else {       // padded -> dense
        p.srcPtr = padded;
        p.srcPos = inner;
        p.dstPtr = make_cudaPitchedPtr(dense_out, (size_t)g.nx * e, (size_t)g.nx, (size_t)g.ny);
    }
    p.kind = kind;
    HS_TRY_CUDA(cudaMemcpy3DAsync(&p, h->stream), "heat: interior copy");
    return HS_OK;
}

// The interior between the dense layout (x fastest, nx * ny * nz) and the
// padded one, a row of x per block step, as raw W-sized words (16-byte words
// when a row and the dense base allow; every padded interior row starts
// 16-byte aligned).  All sizes and offsets are in words.
template <typename W>
__global__ void __launch_bounds__(256)
    k_interior_copy(const W* __restrict__ src, W* __restrict__ dst, int64_t nxw, int64_t pitch_w,
                    int64_t plane_w, int64_t lead_w, int ny, int nz, int to_padded)
{
    const int64_t rows = (int64_t)ny * nz;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t j = r % ny, k = r / ny;
        const int64_t pd = (k + 1) * plane_w + (j + 1) * pitch_w + lead_w, dn = r * nxw;
        const W* s = src + (to_padded ? dn : pd);
        W* d = dst + (to_padded ? pd : dn);
        for (int64_t i = threadIdx.x; i < nxw; i += blockDim.x) d[i] = s[i];
    }
}

// Device-side re-layout of the interior: dense -> padded (to_padded) or back.
int interior_copy(hs_heat* h, const void* src, void* dst, bool to_padded)
{
    const HeatGeom& g = h->g;
    const int64_t e = (int64_t)h->elem;
    const void* dense = to_padded ? src : dst;
    const int64_t rows = (int64_t)g.ny * g.nz;
    const unsigned blocks = (unsigned)(rows < (int64_t)kNumSMs * 16 ? rows : (int64_t)kNumSMs * 16);
    if ((g.nx * e) % 16 == 0 && (reinterpret_cast<uintptr_t>(dense) & 15) == 0) {
        k_interior_copy<uint4><<<blocks, 256, 0, h->stream>>>(
            (const uint4*)src, (uint4*)dst, g.nx * e / 16, g.pitch * e / 16, g.plane * e / 16, g.lead * e / 16,
            g.ny, g.nz, to_padded);
    } else if (e == 8) {
        k_interior_copy<unsigned long long><<<blocks, 256, 0, h->stream>>>(
            (const unsigned long long*)src, (unsigned long long*)dst, g.nx, g.pitch, g.plane, g.lead, g.ny, g.nz,
            to_padded);
    } else {
        k_interior_copy<unsigned><<<blocks, 256, 0, h->stream>>>((const unsigned*)src, (unsigned*)dst, g.nx, g.pitch,
                                                                 g.plane, g.lead, g.ny, g.nz, to_padded);
    }
    HS_CHECK_LAUNCH("heat: interior copy kernel");
    return HS_OK;
}

unsigned conv_blocks(const HeatGeom& g)
{
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)kNumSMs * 16;
    return (unsigned)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

namespace hcg {

int heat_batch_view(hs_heat_t h, HeatBatchView* v)
{
    if (!h || !v) return fail(HS_EINVAL, "heat batch: NULL handle");
    v->g = h->g;
    v->buf[0] = h->buf[0];
    v->buf[1] = h->buf[1];
    v->r = h->r;
    v->arith = h->arith;
    v->cur = h->cur;
    v->vk = (h->flags & HS_VARKAPPA) ? 1 : 0;
    v->fx = h->fx;
    v->m3 = (int)(h->fxseq % 3);
    v->stream = h->stream;
    return HS_OK;
}

int heat_batch_advance(hs_heat_t h, int64_t steps)
{
    if (!h) return fail(HS_EINVAL, "heat batch: NULL handle");
    h->cur = (int)((h->cur + steps) & 1);
    h->steps += steps;
    h->fxseq += steps;
    return HS_OK;
}

}  // namespace hcg

extern "C" {

int heat_buffer_bytes(const hs_heat_desc* desc, size_t* bytes)
{
    int rc = check_desc(desc);
    if (rc != HS_OK) return rc;
    if (!bytes) return fail(HS_EINVAL, "heat_buffer_bytes: bytes is NULL");
    const HeatGeom g = make_geom(desc->nx, desc->ny, desc->nz, elem_size(desc->dtype));
    *bytes = (size_t)g.total * elem_size(desc->dtype);
    return HS_OK;
}

int heat_device_bytes(const hs_heat_desc* desc, size_t* bytes)
{
    int rc = check_desc(desc);
    if (rc != HS_OK) return rc;
    if (!bytes) return fail(HS_EINVAL, "heat_device_bytes: bytes is NULL");
    const HeatGeom g = make_geom(desc->nx, desc->ny, desc->nz, elem_size(desc->dtype));
    const bool user_bufs = desc->dev_buf0 || desc->dev_buf1;
    *bytes = user_bufs ? 0 : 2 * (size_t)g.total * elem_size(desc->dtype);
    const Arith a = pick_arith(desc);
    if (a == A_FX64 || a == A_F64_XS) *bytes += sizeof(FxState);
    if (desc->flags & HS_VARKAPPA)   // coefficients (FP64: three face arrays) and dt f
        *bytes += (desc->dtype == HS_F64 ? 4 : 2) * (size_t)g.total * elem_size(desc->dtype) +
                  (desc->dtype == HS_F64 ? sizeof(FxState) : 0);
    return HS_OK;
}

int heat_create(hs_heat_t* out, const hs_heat_desc* desc)
{
    if (!out) return fail(HS_EINVAL, "heat_create: out is NULL");
    *out = nullptr;
    int rc = check_desc(desc);
    if (rc != HS_OK) return rc;
    hs_heat* h = new (std::nothrow) hs_heat();
    if (!h) return fail(HS_ENOMEM, "heat_create: host allocation failed");
    h->dtype = desc->dtype;
    h->elem = elem_size(desc->dtype);
    h->g = make_geom(desc->nx, desc->ny, desc->nz, h->elem);
    h->r = desc->r;
    h->flags = desc->flags;
    h->arith = pick_arith(desc);
    // r <= 1/6 < 1/2, so r 2^64 < 2^63.  For r >= 2^-11 it is an integer (r's
    // last bit is worth at least 2^-64), so R holds r exactly; a smaller r is
    // rounded to the nearest multiple of 2^-64.
    h->R = (h->arith == A_FX64) ? std::llrint(std::ldexp(desc->r, 64)) : 0;
    h->stream = (cudaStream_t)desc->stream;
    h->cur = 0;
    h->steps = 0;
    h->kchunk = pick_kchunk(h->g, desc->flags, desc->dtype);
    h->tdepth = desc->tdepth ? desc->tdepth : default_tdepth(h->arith, desc->flags);
    if (h->flags & HS_SCHED_FULL) h->tdepth = 1;
    const size_t bytes = (size_t)h->g.total * h->elem;
    rc = check_user_buffers(desc, bytes);
    if (rc != HS_OK) {
        delete h;
        return rc;
    }
    h->owns_buf = !desc->dev_buf0;
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = cudaSuccess;
        if (h->owns_buf) {
            e = dev_alloc(&h->buf[b], bytes, h->stream);
        } else {
            h->buf[b] = b == 0 ? desc->dev_buf0 : desc->dev_buf1;
        }
        if (e != cudaSuccess) {
            h->buf[b] = nullptr;
            rc = cuda_fail(e, "heat_create: device allocation");
            heat_destroy(h);
            return rc;
        }
        e = cudaMemsetAsync(h->buf[b], 0, bytes, h->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "heat_create: cudaMemsetAsync");
            heat_destroy(h);
            return rc;
        }
    }
    {
        cudaError_t e = dev_alloc((void**)&h->err, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "heat_create: error word");
            heat_destroy(h);
            return rc;
        }
    }
    {
        const CUtensorMapDataType dt = h->arith == A_FX64   ? CU_TENSOR_MAP_DATA_TYPE_INT64
                                       : h->dtype == HS_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        uint32_t bx = 0, by = 0;
        stream_box(h->arith, &bx, &by);
        h->sbox[0] = bx;
        h->sbox[1] = by;
        for (int b = 0; b < 2; ++b) {
            const int e = encode_field_map(&h->smaps[b], h->buf[b], dt, h->elem, (uint64_t)h->g.pitch,
                                           (uint64_t)(h->g.ny + 2), (uint64_t)(h->g.nz + 2), bx, by);
            if (e != 0) {
                rc = cuda_fail((cudaError_t)e, "heat_create: TMA tensor map (streaming)");
                heat_destroy(h);
                return rc;
            }
        }
        h->kc_stream = pick_kc_stream(h->g, h->arith);
    }
    if (h->tdepth > 1) {
        const CUtensorMapDataType dt = h->arith == A_FX64   ? CU_TENSOR_MAP_DATA_TYPE_INT64
                                       : h->dtype == HS_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        uint32_t box_x = 0, box_y = 0;
        tb_box(h->arith, h->g.nx, &box_x, &box_y);
        h->tbox[0] = box_x;
        h->tbox[1] = box_y;
        for (int b = 0; b < 2; ++b) {
            const int e = encode_field_map(&h->maps[b], h->buf[b], dt, h->elem, (uint64_t)h->g.pitch,
                                           (uint64_t)(h->g.ny + 2), (uint64_t)(h->g.nz + 2), box_x,
                                           box_y);
            if (e != 0) {
                rc = cuda_fail((cudaError_t)e, "heat_create: TMA tensor map");
                heat_destroy(h);
                return rc;
            }
        }
    }
    if (h->arith == A_FX64 || h->arith == A_F64_XS) {
        cudaError_t e = dev_alloc((void**)&h->fx, sizeof(FxState), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->fx, 0, sizeof(FxState), h->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "heat_create: fixed-point state");
            heat_destroy(h);
            return rc;
        }
    }
    if (h->flags & HS_VARKAPPA) {
        const size_t bytes = (size_t)h->g.total * h->elem;
        // FP64 keeps the three face sums of kappa, FP32 kappa itself
        const size_t cbytes = h->dtype == HS_F64 ? 3 * bytes : bytes;
        cudaError_t e = dev_alloc(&h->kap, cbytes, h->stream);
        if (e == cudaSuccess) e = dev_alloc(&h->fdt, bytes, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->kap, 0, cbytes, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->fdt, 0, bytes, h->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "heat_create: kappa/source arrays");
            heat_destroy(h);
            return rc;
        }
        const double hx = 1.0 / (h->g.nx + 1), hy = 1.0 / (h->g.ny + 1), hz = 1.0 / (h->g.nz + 1);
        const double hmin = std::fmin(hx, std::fmin(hy, hz));
        const double dt = desc->r * hmin * hmin;
        h->vbx = dt / (2.0 * hx * hx);
        h->vby = dt / (2.0 * hy * hy);
        h->vbz = dt / (2.0 * hz * hz);
        VkCall c = {};
        c.f64 = h->dtype == HS_F64;
        c.kap = h->kap;
        c.fdt = h->fdt;
        c.g = &h->g;
        c.stream = h->stream;
        int face_off = 1;
        if (c.f64) {
            e = dev_alloc((void**)&c.face_off, sizeof(int), h->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c.face_off, 0, sizeof(int), h->stream);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "heat_create: face-sum check word");
                heat_destroy(h);
                return rc;
            }
        }
        rc = vk_init(c, dt);
        if (rc == HS_OK && c.f64) {
            cudaError_t e2 = cudaMemcpyAsync(&face_off, c.face_off, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(h->stream);
            if (e2 != cudaSuccess) rc = cuda_fail(e2, "heat_create: face-sum check");
        }
        if (c.face_off) dev_free(c.face_off, h->stream);
        if (rc != HS_OK) {
            heat_destroy(h);
            return rc;
        }
        // FP64 with every face sum of kappa in [1, 2): the exact-sum form,
        // which tracks the field's largest exponent step by step
        if (h->dtype == HS_F64 && face_off == 0) {
            e = dev_alloc((void**)&h->fx, sizeof(FxState), h->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->fx, 0, sizeof(FxState), h->stream);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "heat_create: exact-sum state");
                heat_destroy(h);
                return rc;
            }
        }
    }
    // A Boundary kernel beside the Interior one pays for its extra API calls
    // once the Interior kernel takes tens of microseconds (2^22 points and up).
    const int64_t npts = (int64_t)h->g.nx * h->g.ny * h->g.nz;
    if (!(h->flags & HS_SCHED_FULL) && h->tdepth == 1 && npts >= kForkMinPoints && h->g.nz >= 3) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->bstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "heat_create: side stream");
            heat_destroy(h);
            return rc;
        }
    }
    *out = h;
    return HS_OK;
}

int heat_upload(hs_heat_t h, const void* u, int src_is_device)
{
    if (!h || !u) return fail(HS_EINVAL, "heat_upload: NULL handle or field");
    // The field goes to buffer 0 only.  The spare buffer needs no copy: every
    // interior value of it is written by the next step before it is read, and
    // its boundary layer has been zero since creation -- the same state the
    // paper reaches by uploading u_old and u_new alike.
    // device sources and pinned, mapped host sources are re-laid out by a
    // kernel (the latter reading host memory directly); pageable host sources
    // go through one strided 3-D copy (measured faster over the host link than
    // a contiguous copy into a staging buffer plus the re-layout)
    const void* mapped = src_is_device ? nullptr : mapped_host_ptr(u);
    int rc = src_is_device ? interior_copy(h, u, h->buf[0], true)
             : mapped      ? interior_copy(h, mapped, h->buf[0], true)
                           : copy_interior(h, h->buf[0], u, nullptr, cudaMemcpyHostToDevice);
    if (rc != HS_OK) return rc;
    if (h->arith == A_FX64) {
        HS_TRY_CUDA(cudaMemsetAsync(h->fx, 0, sizeof(FxState), h->stream), "heat_upload: memset");
        const unsigned blocks = conv_blocks(h->g);
        k_fx_maxabs<<<blocks, 256, 0, h->stream>>>((const double*)h->buf[0], h->g, h->fx);
        HS_CHECK_LAUNCH("heat_upload: max|u| kernel");
        k_fx_encode<<<blocks, 256, 0, h->stream>>>((double*)h->buf[0], h->g, h->fx);
        HS_CHECK_LAUNCH("heat_upload: fixed-point encode kernel");
    } else if (h->arith == A_F64_XS || (h->fx && (h->flags & HS_VARKAPPA))) {
        // slot 0: the largest |u| bit pattern of the uploaded field
        HS_TRY_CUDA(cudaMemsetAsync(h->fx, 0, sizeof(FxState), h->stream), "heat_upload: memset");
        k_fx_maxabs<<<conv_blocks(h->g), 256, 0, h->stream>>>((const double*)h->buf[0], h->g, h->fx);
        HS_CHECK_LAUNCH("heat_upload: max|u| kernel");
    }
    h->cur = 0;
    h->steps = 0;
    h->fxseq = 0;
    return HS_OK;
}

int heat_interior(hs_heat_t h)
{
    if (!h) return fail(HS_EINVAL, "heat_interior: NULL handle");
    return do_part(h, P_INTERIOR);
}

int heat_boundary(hs_heat_t h)
{
    if (!h) return fail(HS_EINVAL, "heat_boundary: NULL handle");
    return do_part(h, P_BOUNDARY);
}

int heat_swap(hs_heat_t h)
{
    if (!h) return fail(HS_EINVAL, "heat_swap: NULL handle");
    h->cur = 1 - h->cur;
    h->steps += 1;
    h->fxseq += 1;
    return HS_OK;
}

int heat_step(hs_heat_t h, int64_t n_steps)
{
    if (!h) return fail(HS_EINVAL, "heat_step: NULL handle");
    if (n_steps < 0) return fail(HS_EINVAL, "heat_step: n_steps = %lld < 0", (long long)n_steps);
    if (h->tdepth > 1) {
        // passes of tdepth steps, then the remainder in the largest built depths
        int64_t left = n_steps;
        static const int depths[] = {4, 3, 2};
        for (int L : depths) {
            if (L > h->tdepth) continue;
            for (; left >= L; left -= L) {
                const int rc = tb_pass(h, L);
                if (rc != HS_OK) return rc;
            }
        }
        for (; left > 0; --left) {   // a last single step: Boundary + Interior
            int rc = do_part(h, P_BOUNDARY);
            if (rc == HS_OK) rc = do_part(h, P_INTERIOR);
            if (rc != HS_OK) return rc;
            h->cur = 1 - h->cur;
            h->steps += 1;
            h->fxseq += 1;
        }
        return HS_OK;
    }
    for (int64_t m = 0; m < n_steps; ++m) {
        int rc;
        if (h->flags & HS_SCHED_FULL) {
            rc = do_part(h, P_FULL);
        } else if (h->bstream) {
            // Interior on the handle's stream, Boundary beside it on the side
            // stream (the two write disjoint planes of the new level and fold
            // into the step maximum with atomics); the next step starts after both
            HS_TRY_CUDA(cudaEventRecord(h->ev_fork, h->stream), "heat_step: fork event");
            rc = timed_interior(h);
            if (rc != HS_OK) return rc;
            HS_TRY_CUDA(cudaStreamWaitEvent(h->bstream, h->ev_fork, 0), "heat_step: fork wait");
            rc = do_part(h, P_BOUNDARY, h->bstream);
            if (rc != HS_OK) return rc;
            HS_TRY_CUDA(cudaEventRecord(h->ev_join, h->bstream), "heat_step: join event");
            HS_TRY_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0), "heat_step: join wait");
        } else {
            rc = do_part(h, P_BOUNDARY);
            if (rc == HS_OK) rc = timed_interior(h);
        }
        if (rc != HS_OK) return rc;
        h->cur = 1 - h->cur;
        h->steps += 1;
        h->fxseq += 1;
    }
    return HS_OK;
}

int heat_time_interior(hs_heat_t h, int enable)
{
    if (!h) return fail(HS_EINVAL, "heat_time_interior: NULL handle");
    h->timing = enable != 0;
    return HS_OK;
}

int heat_interior_time(hs_heat_t h, double* mean_ms, int64_t* launches)
{
    if (!h) return fail(HS_EINVAL, "heat_interior_time: NULL handle");
    double total = 0.0;
    const size_t n = h->tev_used;
    if (n > 0) HS_TRY_CUDA(cudaEventSynchronize(h->tev[2 * n - 1]), "heat_interior_time: synchronize");
    for (size_t i = 0; i < n; ++i) {
        float ms = 0.0f;
        HS_TRY_CUDA(cudaEventElapsedTime(&ms, h->tev[2 * i], h->tev[2 * i + 1]),
                    "heat_interior_time: elapsed time");
        total += ms;
    }
    h->tev_used = 0;
    if (mean_ms) *mean_ms = n ? total / (double)n : 0.0;
    if (launches) *launches = (int64_t)n;
    return HS_OK;
}

int heat_read(hs_heat_t h, void* dst, int dst_is_device)
{
    if (!h || !dst) return fail(HS_EINVAL, "heat_read: NULL handle or destination");
    void* src = h->buf[h->cur];
    void* spare = h->buf[1 - h->cur];
    if (h->arith == A_FX64) {
        // Decode into the spare buffer's interior; the next step overwrites
        // all of it, and its boundary layer stays zero.
        k_fx_decode<<<conv_blocks(h->g), 256, 0, h->stream>>>(
            (const long long*)h->buf[h->cur], (double*)spare, h->g, h->fx, (int)(h->fxseq % 3));
        HS_CHECK_LAUNCH("heat_read: fixed-point decode kernel");
        src = spare;
    }
    // device and pinned, mapped host destinations by a kernel, pageable host
    // ones by one strided 3-D copy
    void* mapped = dst_is_device ? nullptr : mapped_host_ptr(dst);
    int rc = dst_is_device ? interior_copy(h, src, dst, false)
             : mapped      ? interior_copy(h, src, mapped, false)
                           : copy_interior(h, src, nullptr, dst, cudaMemcpyDeviceToHost);
    if (rc != HS_OK) return rc;
    // status reads on the handle's own stream (a legacy-stream copy would also
    // wait for every other blocking stream, e.g. a batch running elsewhere)
    int err = 0;
    HS_TRY_CUDA(cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
                "heat_read: error word");
    HS_TRY_CUDA(cudaStreamSynchronize(h->stream), "heat_read: stream synchronize");
    if (err == 2)
        return fail(HS_ECUDA, "heat_read: a bounded wait inside a TMA-staged heat kernel ran out and "
                              "the block's loads in flight did not complete in time; the field is not "
                              "valid and the CUDA context should be treated as suspect");
    if (err)
        return fail(HS_ETIMEOUT, "heat_read: a bounded wait inside a TMA-staged heat kernel ran out; "
                                 "the field is not valid");
    if (h->arith == A_FX64) {
        FxState st;
        HS_TRY_CUDA(cudaMemcpyAsync(&st, h->fx, sizeof(st), cudaMemcpyDeviceToHost, h->stream),
                    "heat_read: state");
        HS_TRY_CUDA(cudaStreamSynchronize(h->stream), "heat_read: stream synchronize");
        if (st.nonfinite)
            return fail(HS_ERANGE, "heat_read: the uploaded field held NaN or Inf, which the "
                                   "fixed-point form cannot carry");
    }
    return HS_OK;
}

int heat_steps_done(hs_heat_t h, int64_t* steps)
{
    if (!h || !steps) return fail(HS_EINVAL, "heat_steps_done: NULL argument");
    *steps = h->steps;
    return HS_OK;
}

int heat_set_kchunk(hs_heat_t h, int32_t planes)
{
    if (!h) return fail(HS_EINVAL, "heat_set_kchunk: NULL handle");
    if (planes < 0) return fail(HS_EINVAL, "heat_set_kchunk: planes = %d < 0", planes);
    const int interior = h->g.nz > 2 ? h->g.nz - 2 : 1;
    if (planes == 0) {
        h->kchunk = pick_kchunk(h->g, h->flags, h->dtype);
        h->kc_stream = pick_kc_stream(h->g, h->arith);
    } else {
        h->kchunk = h->kc_stream = planes < interior ? planes : interior;
    }
    return HS_OK;
}

int heat_get_kchunk(hs_heat_t h, int32_t* planes)
{
    if (!h || !planes) return fail(HS_EINVAL, "heat_get_kchunk: NULL argument");
    const bool streaming = !(h->flags & HS_VARKAPPA) && h->arith != A_F64 && h->arith != A_F64_EXACT;
    *planes = streaming ? h->kc_stream : h->kchunk;
    return HS_OK;
}

int heat_get_tdepth(hs_heat_t h, int32_t* tdepth)
{
    if (!h || !tdepth) return fail(HS_EINVAL, "heat_get_tdepth: NULL argument");
    *tdepth = h->tdepth;
    return HS_OK;
}

int heat_destroy(hs_heat_t h)
{
    if (!h) return HS_OK;
    int rc = HS_OK;
    if (h->buf[0] || h->buf[1]) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "heat_destroy: stream synchronize");
    }
    if (h->bstream) {
        cudaError_t e = cudaStreamSynchronize(h->bstream);
        if (e != cudaSuccess && rc == HS_OK) rc = cuda_fail(e, "heat_destroy: side stream synchronize");
        (void)cudaStreamDestroy(h->bstream);
    }
    for (cudaEvent_t e : h->tev) (void)cudaEventDestroy(e);
    if (h->ev_fork) (void)cudaEventDestroy(h->ev_fork);
    if (h->ev_join) (void)cudaEventDestroy(h->ev_join);
    if (h->owns_buf)
        for (int b = 0; b < 2; ++b) dev_free(h->buf[b], h->stream);
    dev_free(h->fx, h->stream);
    dev_free(h->err, h->stream);
    dev_free(h->kap, h->stream);
    dev_free(h->fdt, h->stream);
    delete h;
    return rc;
}

}  // extern "C"
