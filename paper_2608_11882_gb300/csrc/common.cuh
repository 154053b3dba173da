// Shared host/device helpers of the heat + CG library (status handling,
// launch accounting, deterministic block reductions).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "heatcg.h"

namespace hcg {

// Records a printf-style message as the calling thread's last error.
void set_error(const char* fmt, ...);
// Records a failed CUDA call and maps it to HS_ENOMEM or HS_ECUDA.
int cuda_fail(cudaError_t e, const char* what);
// Returns code after recording msg (for argument errors).
int fail(int code, const char* fmt, ...);

extern std::atomic<int64_t> g_launches;
inline void count_launch(int64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace hcg

#define HS_TRY_CUDA(call, what)                                          \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::hcg::cuda_fail(e_, what);        \
    } while (0)

// Checks the launch just issued and counts it.
#define HS_CHECK_LAUNCH(what)                                            \
    do {                                                                 \
        cudaError_t e_ = cudaPeekAtLastError();                          \
        if (e_ != cudaSuccess) {                                         \
            (void)cudaGetLastError();                                    \
            return ::hcg::cuda_fail(e_, what);                           \
        }                                                                \
        ::hcg::count_launch();                                           \
    } while (0)

namespace hcg {

constexpr int kNumSMs = 152;   // GB300: 2 dies x 76 SMs (queried at run time where it matters)

// The device address of pinned, mapped host memory, or nullptr for any other
// pointer (pageable host memory in particular) -- api.cu.
void* mapped_host_ptr(const void* p);
// bytes between host memory and device memory, enqueued on s: a copy kernel
// through the mapped address when the host side is pinned and mapped, else
// cudaMemcpyAsync -- api.cu.
int copy_host(void* dst, const void* src, size_t bytes, bool to_device, cudaStream_t s, const char* what);

// Device memory of handles and contexts comes from the stream-ordered
// allocator on the object's own stream: unlike cudaMalloc/cudaFree these calls
// never synchronise the whole device, so creating or releasing one object does
// not stall the work other streams have in flight (a server that opens and
// closes requests while others run).  Memory freed this way returns to the pool
// once the stream's earlier work is done.
inline cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) { return cudaMallocAsync(p, bytes, s); }
inline void dev_free(void* p, cudaStream_t s)
{
    if (p) (void)cudaFreeAsync(p, s);
}

// Programmatic dependent launch.  A kernel started by launch_dependent() may
// begin while the kernel before it on the stream is still finishing: it runs
// its own set-up, then grid_dependency_wait() holds it until that kernel has
// completed and its writes are visible.  allow_dependents() marks the point
// from which this block no longer needs its SM to itself; once every block
// of the grid has passed it (or exited), the next kernel may start to launch.
// In a launch without the attribute both are no-ops.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kern)(KArgs...), int grid, int block, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (e != cudaSuccess) (void)cudaGetLastError();   // reported through the return value only
    return e;
}

// Sum of v over a block of BLOCK threads, in a fixed order (warp shuffles,
// then warp 0 over the per-warp sums).  The result is valid in thread 0.
// sh must hold BLOCK/32 doubles.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = 0.0;
    if (warp == 0) {
        v = (lane < BLOCK / 32) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

}  // namespace hcg
