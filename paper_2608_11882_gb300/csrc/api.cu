// Error reporting, version and launch accounting of the C ABI.
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

}  // namespace hcg

extern "C" {

const char* hs_last_error(void) { return hcg::t_last_error; }

int hs_version(void) { return 100; }

int64_t hs_launch_count(void) { return hcg::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
