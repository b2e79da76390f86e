// Error reporting and version of libtdq.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include "tdq_internal.cuh"

namespace {
thread_local char g_err[512] = "";
// allocations left before the injected failure (< 0: none injected)
std::atomic<long long> g_alloc_countdown{-1};
}

namespace tdq {

tdq_status set_error(tdq_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

tdq_status cuda_error(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a non-sticky error
    if (e == cudaErrorMemoryAllocation) return set_error(TDQ_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(TDQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t alloc_gate()
{
    long long c = g_alloc_countdown.load();
    while (c >= 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0 ? cudaErrorMemoryAllocation : cudaSuccess;
    }
    return cudaSuccess;
}

}  // namespace tdq

extern "C" void tdq_debug_fail_allocations(int64_t after) { g_alloc_countdown.store(after < 0 ? -1 : after); }

extern "C" const char *tdq_last_error(void) { return g_err; }

#ifdef TDQ_DEBUG
extern "C" const char *tdq_version(void) { return "tdq 0.2 (sm_103a, bounds-checked debug build)"; }
#else
extern "C" const char *tdq_version(void) { return "tdq 0.2 (sm_103a)"; }
#endif
