// Explicit 7-point heat stepping on one GPU: the Interior and Boundary kernels
// of Algorithms INTERIOR and BOUNDARY, the full-step kernel of Algorithm
// COMPUTE_SINGLE_GPU, and the heat_* entry points of the C ABI.
//
// Update (Section 4, Eq. 4 with kappa = 1 and f = 0, r = alpha dt / h^2):
//     u' = u + r * (((u[i-1] + u[i+1]) + (u[j-1] + u[j+1])) + (u[k-1] + u[k+1]) - 6 u)
// on interior points; the boundary layer stays zero (Dirichlet).
//
// Layout in HBM: each field buffer holds (nz+2) planes of (ny+2) rows.  A row
// has `pitch` elements (a multiple of 128 bytes); interior x = 0 sits at
// element `lead` (32 bytes in), so interior rows start 32-byte aligned, and
// the x-boundary cells sit at lead-1 and lead+nx.  Planes 0 and nz+1, rows 0
// and ny+1 and the x-boundary cells hold the Dirichlet zeros in both buffers
// and are never written after creation, so a pointer swap keeps them intact.
#include <cmath>
#include <cstdlib>
#include <new>

#include "common.cuh"

namespace hcg {

struct HeatGeom {
    int32_t nx, ny, nz;
    int32_t lead;    // element offset of interior x = 0 within a row
    int64_t pitch;   // elements per row
    int64_t plane;   // elements per plane = pitch * (ny + 2)
    int64_t total;   // elements per buffer = plane * (nz + 2)
    __host__ __device__ __forceinline__ int64_t at(int i, int j, int k) const
    {
        return (int64_t)(k + 1) * plane + (int64_t)(j + 1) * pitch + lead + i;
    }
};

static HeatGeom make_geom(int nx, int ny, int nz, size_t elem)
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
    return g;
}

// ---- the point update -------------------------------------------------------
// Default: the six-neighbour sum in the written order, then two fused
// multiply-adds: t = s - 6u, u' = u + r t (7 FP64 instructions per point).
// Exact: one rounding per operation in the written order, no fusion.
template <typename T, bool EXACT>
struct Point;

template <bool EXACT>
struct Point<double, EXACT> {
    static __device__ __forceinline__ double update(double c, double xm, double xp, double ym,
                                                    double yp, double zm, double zp, double r)
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
                                                   float zm, float zp, float r)
    {
        const float s = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)),
                                  __fadd_rn(zm, zp));
        if (EXACT) return __fadd_rn(c, __fmul_rn(r, __fsub_rn(s, __fmul_rn(6.0f, c))));
        return __fmaf_rn(r, __fmaf_rn(-6.0f, c, s), c);
    }
};

// ---- Interior kernel ----------------------------------------------------------
// One thread per (i, j) column marches up a chunk of k-planes, keeping the
// values at k-1, k and k+1 in registers (rotated each plane); the four
// in-plane neighbours come through the read-only cache, where the block's
// neighbouring columns have just loaded them.
constexpr int kBX = 32, kBY = 8;

template <typename T, bool EXACT>
__global__ void __launch_bounds__(kBX* kBY)
    k_heat_interior(const T* __restrict__ src, T* __restrict__ dst, HeatGeom g, T r, int kbeg,
                    int kend, int kchunk)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k0 = kbeg + (int)blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, kend);
    if (k0 >= k1) return;
    const int64_t P = g.plane, Y = g.pitch;
    int64_t c = g.at(i, j, k0);
    T below = __ldg(src + c - P);
    T cur = __ldg(src + c);
    for (int k = k0; k < k1; ++k) {
        const T above = __ldg(src + c + P);
        const T xm = __ldg(src + c - 1), xp = __ldg(src + c + 1);
        const T ym = __ldg(src + c - Y), yp = __ldg(src + c + Y);
        dst[c] = Point<T, EXACT>::update(cur, xm, xp, ym, yp, below, above, r);
        below = cur;
        cur = above;
        c += P;
    }
}

// ---- Boundary kernel ------------------------------------------------------------
// The outermost interior k-planes (k = 0 and k = nz-1): the planes a k-split
// across devices would exchange.  blockIdx.z selects the plane.
template <typename T, bool EXACT>
__global__ void __launch_bounds__(kBX* kBY)
    k_heat_boundary(const T* __restrict__ src, T* __restrict__ dst, HeatGeom g, T r)
{
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int k = (blockIdx.z == 0) ? 0 : g.nz - 1;
    const int64_t P = g.plane, Y = g.pitch;
    const int64_t c = g.at(i, j, k);
    dst[c] = Point<T, EXACT>::update(__ldg(src + c), __ldg(src + c - 1), __ldg(src + c + 1),
                                     __ldg(src + c - Y), __ldg(src + c + Y), __ldg(src + c - P),
                                     __ldg(src + c + P), r);
}

// ---- full-step kernel -------------------------------------------------------------
// Algorithm COMPUTE_SINGLE_GPU: one thread per interior point over the whole
// box, all seven values loaded directly.  A separate code path from the
// Interior/Boundary pair, used to cross-check it bit for bit.
template <typename T, bool EXACT>
__global__ void __launch_bounds__(256)
    k_heat_full(const T* __restrict__ src, T* __restrict__ dst, HeatGeom g, T r)
{
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const int64_t P = g.plane, Y = g.pitch;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx);
        const int64_t jk = t / g.nx;
        const int j = (int)(jk % g.ny);
        const int k = (int)(jk / g.ny);
        const int64_t c = g.at(i, j, k);
        dst[c] = Point<T, EXACT>::update(src[c], src[c - 1], src[c + 1], src[c - Y], src[c + Y],
                                         src[c - P], src[c + P], r);
    }
}

}  // namespace hcg

using namespace hcg;

struct hs_heat {
    HeatGeom g;
    int32_t dtype;
    size_t elem;
    double r;
    uint32_t flags;
    cudaStream_t stream;
    void* buf[2];
    int cur;           // buffer holding the current time level
    int64_t steps;     // steps since the last upload
    int kchunk;        // planes per Interior-kernel block
};

namespace {

constexpr uint32_t kKnownFlags = HS_ALLOW_UNSTABLE | HS_EXACT_ROUNDING | HS_SCHED_FULL;

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
    if (d->reserved0 != 0) return fail(HS_EINVAL, "heat: reserved0 must be 0");
    // Three-dimensional stability of the explicit update: r <= 1/6.
    if (d->r > 1.0 / 6.0 && !(d->flags & HS_ALLOW_UNSTABLE))
        return fail(HS_EUNSTABLE, "heat: r = %.17g exceeds the stability bound 1/6", d->r);
    return HS_OK;
}

size_t elem_size(int dtype) { return dtype == HS_F64 ? sizeof(double) : sizeof(float); }

int pick_kchunk(const HeatGeom& g)
{
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

template <typename T>
int launch_interior(hs_heat* h)
{
    const HeatGeom& g = h->g;
    if (g.nz < 3) return HS_OK;   // no plane lies strictly between the boundary planes
    const int kbeg = 1, kend = g.nz - 1;
    const int nchunks = (kend - kbeg + h->kchunk - 1) / h->kchunk;
    dim3 block(kBX, kBY, 1);
    dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, nchunks);
    const T* src = (const T*)h->buf[h->cur];
    T* dst = (T*)h->buf[1 - h->cur];
    if (h->flags & HS_EXACT_ROUNDING)
        k_heat_interior<T, true><<<grid, block, 0, h->stream>>>(src, dst, g, (T)h->r, kbeg, kend,
                                                                 h->kchunk);
    else
        k_heat_interior<T, false><<<grid, block, 0, h->stream>>>(src, dst, g, (T)h->r, kbeg, kend,
                                                                  h->kchunk);
    HS_CHECK_LAUNCH("heat interior kernel");
    return HS_OK;
}

template <typename T>
int launch_boundary(hs_heat* h)
{
    const HeatGeom& g = h->g;
    dim3 block(kBX, kBY, 1);
    dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, g.nz >= 2 ? 2 : 1);
    const T* src = (const T*)h->buf[h->cur];
    T* dst = (T*)h->buf[1 - h->cur];
    if (h->flags & HS_EXACT_ROUNDING)
        k_heat_boundary<T, true><<<grid, block, 0, h->stream>>>(src, dst, g, (T)h->r);
    else
        k_heat_boundary<T, false><<<grid, block, 0, h->stream>>>(src, dst, g, (T)h->r);
    HS_CHECK_LAUNCH("heat boundary kernel");
    return HS_OK;
}

template <typename T>
int launch_full(hs_heat* h)
{
    const HeatGeom& g = h->g;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)kNumSMs * 64) blocks = (int64_t)kNumSMs * 64;
    const T* src = (const T*)h->buf[h->cur];
    T* dst = (T*)h->buf[1 - h->cur];
    if (h->flags & HS_EXACT_ROUNDING)
        k_heat_full<T, true><<<(unsigned)blocks, 256, 0, h->stream>>>(src, dst, g, (T)h->r);
    else
        k_heat_full<T, false><<<(unsigned)blocks, 256, 0, h->stream>>>(src, dst, g, (T)h->r);
    HS_CHECK_LAUNCH("heat full-step kernel");
    return HS_OK;
}

int do_interior(hs_heat* h)
{
    return h->dtype == HS_F64 ? launch_interior<double>(h) : launch_interior<float>(h);
}
int do_boundary(hs_heat* h)
{
    return h->dtype == HS_F64 ? launch_boundary<double>(h) : launch_boundary<float>(h);
}
int do_full(hs_heat* h) { return h->dtype == HS_F64 ? launch_full<double>(h) : launch_full<float>(h); }

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

}  // namespace

extern "C" {

int heat_device_bytes(const hs_heat_desc* desc, size_t* bytes)
{
    int rc = check_desc(desc);
    if (rc != HS_OK) return rc;
    if (!bytes) return fail(HS_EINVAL, "heat_device_bytes: bytes is NULL");
    const HeatGeom g = make_geom(desc->nx, desc->ny, desc->nz, elem_size(desc->dtype));
    *bytes = 2 * (size_t)g.total * elem_size(desc->dtype);
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
    h->stream = (cudaStream_t)desc->stream;
    h->cur = 0;
    h->steps = 0;
    h->kchunk = pick_kchunk(h->g);
    const size_t bytes = (size_t)h->g.total * h->elem;
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = cudaMalloc(&h->buf[b], bytes);
        if (e != cudaSuccess) {
            h->buf[b] = nullptr;
            rc = cuda_fail(e, "heat_create: cudaMalloc");
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
    *out = h;
    return HS_OK;
}

int heat_upload(hs_heat_t h, const void* u, int src_is_device)
{
    if (!h || !u) return fail(HS_EINVAL, "heat_upload: NULL handle or field");
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // The field goes to buffer 0 only.  The spare buffer needs no copy: every
    // interior value of it is written by the next step before it is read, and
    // its boundary layer has been zero since creation -- the same state the
    // paper reaches by uploading u_old and u_new alike.
    int rc = copy_interior(h, h->buf[0], u, nullptr, kind);
    if (rc != HS_OK) return rc;
    h->cur = 0;
    h->steps = 0;
    return HS_OK;
}

int heat_interior(hs_heat_t h)
{
    if (!h) return fail(HS_EINVAL, "heat_interior: NULL handle");
    return do_interior(h);
}

int heat_boundary(hs_heat_t h)
{
    if (!h) return fail(HS_EINVAL, "heat_boundary: NULL handle");
    return do_boundary(h);
}

int heat_swap(hs_heat_t h)
{
    if (!h) return fail(HS_EINVAL, "heat_swap: NULL handle");
    h->cur = 1 - h->cur;
    h->steps += 1;
    return HS_OK;
}

int heat_step(hs_heat_t h, int64_t n_steps)
{
    if (!h) return fail(HS_EINVAL, "heat_step: NULL handle");
    if (n_steps < 0) return fail(HS_EINVAL, "heat_step: n_steps = %lld < 0", (long long)n_steps);
    for (int64_t m = 0; m < n_steps; ++m) {
        int rc;
        if (h->flags & HS_SCHED_FULL) {
            rc = do_full(h);
        } else {
            rc = do_boundary(h);
            if (rc == HS_OK) rc = do_interior(h);
        }
        if (rc != HS_OK) return rc;
        h->cur = 1 - h->cur;
        h->steps += 1;
    }
    return HS_OK;
}

int heat_read(hs_heat_t h, void* dst, int dst_is_device)
{
    if (!h || !dst) return fail(HS_EINVAL, "heat_read: NULL handle or destination");
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int rc = copy_interior(h, h->buf[h->cur], nullptr, dst, kind);
    if (rc != HS_OK) return rc;
    HS_TRY_CUDA(cudaStreamSynchronize(h->stream), "heat_read: stream synchronize");
    return HS_OK;
}

int heat_steps_done(hs_heat_t h, int64_t* steps)
{
    if (!h || !steps) return fail(HS_EINVAL, "heat_steps_done: NULL argument");
    *steps = h->steps;
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
    for (int b = 0; b < 2; ++b)
        if (h->buf[b]) cudaFree(h->buf[b]);
    delete h;
    return rc;
}

}  // extern "C"
