// Error reporting, version and launch accounting of the C ABI.
#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace hcg {

static thread_local char t_last_error[512] = "";
std::atomic<int64_t> g_launches{0};

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
    va_end(ap);
}

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA;
}

// The device address of pinned, mapped host memory (page-locked by
// cudaHostAlloc / cudaMallocHost or registered with cudaHostRegister), or
// nullptr for any other pointer -- pageable host memory in particular, which
// a kernel must not touch.  Host buffers of this kind are moved by kernels
// that read or write host memory directly: as fast as a DMA copy on a quiet
// box (5.6 ms per GiB each way), and unaffected where the copy engines slow
// down next to long kernels (measured after a long run of other GPU work on
// the same box: 56-83 ms per GiB by DMA, 5.6 ms by a kernel).
void* mapped_host_ptr(const void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <typename W>
__global__ void __launch_bounds__(256) k_copy_words(const W* __restrict__ src, W* __restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

int copy_host(void* dst, const void* src, size_t bytes, bool to_device, cudaStream_t s, const char* what)
{
    if (bytes == 0) return HS_OK;
    void* mapped = mapped_host_ptr(to_device ? src : dst);
    if (!mapped) {
        HS_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, s),
                    what);
        return HS_OK;
    }
    const void* from = to_device ? mapped : src;
    void* to = to_device ? dst : mapped;
    const uintptr_t al = reinterpret_cast<uintptr_t>(from) | reinterpret_cast<uintptr_t>(to) | bytes;
    const int64_t w = (al & 15) == 0 ? 16 : (al & 7) == 0 ? 8 : (al & 3) == 0 ? 4 : 1;
    const int64_t n = (int64_t)bytes / w;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)kNumSMs * 16);
    if (w == 16)
        k_copy_words<uint4><<<blocks, 256, 0, s>>>((const uint4*)from, (uint4*)to, n);
    else if (w == 8)
        k_copy_words<unsigned long long><<<blocks, 256, 0, s>>>((const unsigned long long*)from, (unsigned long long*)to, n);
    else if (w == 4)
        k_copy_words<unsigned><<<blocks, 256, 0, s>>>((const unsigned*)from, (unsigned*)to, n);
    else
        k_copy_words<unsigned char><<<blocks, 256, 0, s>>>((const unsigned char*)from, (unsigned char*)to, n);
    HS_CHECK_LAUNCH(what);
    return HS_OK;
}

}  // namespace hcg

extern "C" {

const char* hs_last_error(void) { return hcg::t_last_error; }

int hs_version(void) { return 100; }

int64_t hs_launch_count(void) { return hcg::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
