// Library state shared by all entry points: error messages, allocation, device info.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

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

// ------------------------------------------------------------------ launch accounting

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_timing{0};

struct PendingTiming {
    std::string name;
    cudaEvent_t start, stop;
};
static std::mutex g_tmu;
static std::vector<PendingTiming> g_pending;
static std::map<std::string, std::pair<double, long long>> g_totals;
static thread_local std::vector<std::pair<std::string, cudaEvent_t>> g_open;

void note_launch(const char *name, cudaStream_t s, bool begin) {
    if (begin) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_timing.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (begin) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, s);
        g_open.emplace_back(name, e);
    } else {
        for (size_t k = g_open.size(); k-- > 0;) {
            if (g_open[k].first == name) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                cudaEventRecord(e, s);
                std::lock_guard<std::mutex> lk(g_tmu);
                g_pending.push_back({name, g_open[k].second, e});
                g_open.erase(g_open.begin() + k);
                return;
            }
        }
    }
}

static void resolve_timings() {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            auto &t = g_totals[p.name];
            t.first += ms;
            t.second += 1;
        }
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    g_pending.clear();
}

}  // namespace fgb

extern "C" int64_t fgb_kernel_launches(void) { return fgb::g_launches.load(); }

extern "C" int fgb_timing_enable(int32_t on) {
    fgb::g_timing.store(on ? 1 : 0);
    return FGB_OK;
}

extern "C" int fgb_timing_read(const char *name, double *total_ms, int64_t *count) {
    if (!name) return fgb::fail(FGB_ERR_INVALID_ARG, "name is NULL");
    fgb::resolve_timings();
    std::lock_guard<std::mutex> lk(fgb::g_tmu);
    auto it = fgb::g_totals.find(name);
    if (total_ms) *total_ms = it == fgb::g_totals.end() ? 0.0 : it->second.first;
    if (count) *count = it == fgb::g_totals.end() ? 0 : it->second.second;
    return FGB_OK;
}

extern "C" int fgb_timing_reset(void) {
    fgb::resolve_timings();
    std::lock_guard<std::mutex> lk(fgb::g_tmu);
    fgb::g_totals.clear();
    return FGB_OK;
}

extern "C" const char *fgb_last_error(void) { return fgb::g_err; }

extern "C" int32_t fgb_version(void) { return 10000; }
