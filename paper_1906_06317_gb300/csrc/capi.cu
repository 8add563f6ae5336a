// Library state shared by all entry points: error messages, allocation, device info.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>

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

// The device's default memory pool returns freed memory to the system at every
// synchronisation unless told otherwise; then each neighbor list (gigabytes) is mapped
// again on the next query.  Keep freed blocks cached in this process instead.
static void keep_pool_cached() {
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

// Large blocks (neighbor lists, sort buffers) are kept for reuse instead of being freed:
// even from a cached memory pool, mapping a fresh gigabyte-sized block takes about a
// millisecond per call.  A kept block carries an event recorded on the stream that freed
// it; the stream that reuses it waits on that event first, so reuse is ordered on any
// stream.  fgb_trim_memory() releases everything kept.
namespace {
constexpr size_t kKeepMin = size_t(1) << 20;
constexpr size_t kKeepMax = size_t(48) << 30;
struct Kept {
    void *p;
    size_t bytes;
    int dev;
    cudaEvent_t done;
};
std::mutex g_amu;
std::vector<Kept> g_kept;
size_t g_kept_bytes = 0;
std::unordered_map<void *, size_t> g_sizes;

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}
}  // namespace

int dalloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    keep_pool_cached();
    if (bytes == 0) bytes = 16;
    if (bytes >= kKeepMin && !capturing(s)) {
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(g_amu);
        size_t best = SIZE_MAX;
        int bi = -1;
        for (size_t k = 0; k < g_kept.size(); ++k) {
            const Kept &b = g_kept[k];
            if (b.dev == dev && b.bytes >= bytes && b.bytes <= 2 * bytes && b.bytes < best) {
                best = b.bytes;
                bi = (int)k;
            }
        }
        if (bi >= 0) {
            Kept b = g_kept[bi];
            g_kept.erase(g_kept.begin() + bi);
            g_kept_bytes -= b.bytes;
            cudaStreamWaitEvent(s, b.done, 0);
            cudaEventDestroy(b.done);
            *p = b.p;
            g_sizes[b.p] = b.bytes;
            return FGB_OK;
        }
    }
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? FGB_ERR_OOM : FGB_ERR_CUDA, "device allocation of %zu bytes failed: %s",
                    bytes, cudaGetErrorString(e));
    }
    if (bytes >= kKeepMin) {
        std::lock_guard<std::mutex> lk(g_amu);
        g_sizes[*p] = bytes;
    }
    return FGB_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_amu);
        auto it = g_sizes.find(p);
        if (it != g_sizes.end()) {
            const size_t bytes = it->second;
            g_sizes.erase(it);
            cudaEvent_t ev;
            if (g_kept_bytes + bytes <= kKeepMax && !capturing(s) &&
                cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
                if (cudaEventRecord(ev, s) == cudaSuccess) {
                    int dev = 0;
                    cudaGetDevice(&dev);
                    g_kept.push_back({p, bytes, dev, ev});
                    g_kept_bytes += bytes;
                    return;
                }
                cudaEventDestroy(ev);
            }
        }
    }
    cudaFreeAsync(p, s);
}

int trim_memory() {
    std::lock_guard<std::mutex> lk(g_amu);
    for (Kept &b : g_kept) {
        cudaEventSynchronize(b.done);
        cudaEventDestroy(b.done);
        cudaFree(b.p);
    }
    g_kept.clear();
    g_kept_bytes = 0;
    return FGB_OK;
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

extern "C" int fgb_trim_memory(void) { return fgb::trim_memory(); }

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
