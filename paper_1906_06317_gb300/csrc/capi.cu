// Library state shared by all entry points: error messages, allocation, device info.
#include <cstdarg>
#include <cstring>

#include "fgb_internal.cuh"

namespace fgb {

static thread_local char g_err[1024] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

int dalloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? FGB_ERR_OOM : FGB_ERR_CUDA, "device allocation of %zu bytes failed: %s",
                    bytes, cudaGetErrorString(e));
    }
    return FGB_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace fgb

extern "C" const char *fgb_last_error(void) { return fgb::g_err; }

extern "C" int32_t fgb_version(void) { return 10000; }
