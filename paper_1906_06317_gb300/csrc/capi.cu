// Library state shared by all entry points: error messages, allocation, device info.
#include <atomic>
#include <cstdarg>
#include <cstdlib>
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

// Device memory comes from a memory pool of the library's own on each device (the
// device's default pool, which torch and other libraries share, keeps its settings).
// The pool keeps up to the cache limit of freed memory mapped, so a neighbor list
// (gigabytes) is not mapped again on every query.
namespace {
std::mutex g_amu;
cudaMemPool_t g_pool[64];
bool g_pool_failed[64];

size_t cache_limit_default() {
    const char *e = getenv("FGB_MEMORY_CACHE_MB");
    if (e && *e) {
        const long long mb = atoll(e);
        if (mb >= 0) return (size_t)mb << 20;
    }
    return size_t(4) << 30;  // 4 GB
}
size_t g_cache_limit = cache_limit_default();

// The library's pool on device dev (created on first use), or nullptr when the device
// cannot create one (allocations then use the default pool, left as it is).  g_amu held.
cudaMemPool_t lib_pool_locked(int dev) {
    if (dev < 0 || dev >= 64 || g_pool_failed[dev]) return nullptr;
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&g_pool[dev], &props) != cudaSuccess) {
            cudaGetLastError();
            g_pool[dev] = nullptr;
            g_pool_failed[dev] = true;
            return nullptr;
        }
        uint64_t keep = g_cache_limit;
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return g_pool[dev];
}

// Large blocks (neighbor lists, sort buffers) are also kept for reuse instead of being
// freed: even from a pool that keeps its memory, mapping a fresh gigabyte-sized block
// takes about a millisecond per call.  A kept block carries an event recorded on the
// stream that freed it; the stream that reuses it waits on that event first, so reuse
// is ordered on any stream.  The kept blocks total at most the cache limit;
// fgb_trim_memory() releases everything kept.
constexpr size_t kKeepMin = size_t(1) << 20;
struct Kept {
    void *p;
    size_t bytes;
    int dev;
    cudaEvent_t done;
};
std::vector<Kept> g_kept;
size_t g_kept_bytes = 0;
std::unordered_map<void *, size_t> g_sizes;

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

// Releases kept blocks (oldest first) until they total at most `limit`.  g_amu held.
void release_kept_locked(size_t limit) {
    while (g_kept_bytes > limit && !g_kept.empty()) {
        Kept b = g_kept.front();
        g_kept.erase(g_kept.begin());
        g_kept_bytes -= b.bytes;
        cudaEventSynchronize(b.done);
        cudaEventDestroy(b.done);
        cudaFree(b.p);
    }
}
}  // namespace

int dalloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_amu);
        pool = lib_pool_locked(dev);
        if (bytes >= kKeepMin && !capturing(s)) {
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
    }
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
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
            if (g_kept_bytes + bytes <= g_cache_limit && !capturing(s) &&
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

// Pinned host slots (64 bytes each) that asynchronous calls copy their status words
// into.  A released slot is handed out again once the event recorded after its last copy
// has completed (the event is the slot's to destroy).
namespace {
std::mutex g_pmu;
constexpr size_t kPinnedSlot = 64, kPinnedChunk = 64;
struct PinnedFree {
    void *p;
    cudaEvent_t after;
};
std::vector<PinnedFree> g_pinned_free;
}  // namespace

int pinned_slot(void **p) {
    std::lock_guard<std::mutex> lk(g_pmu);
    for (size_t k = 0; k < g_pinned_free.size(); ++k) {
        const PinnedFree f = g_pinned_free[k];
        if (f.after && cudaEventQuery(f.after) != cudaSuccess) continue;
        if (f.after) cudaEventDestroy(f.after);
        g_pinned_free.erase(g_pinned_free.begin() + k);
        *p = f.p;
        return FGB_OK;
    }
    void *chunk = nullptr;
    if (cudaHostAlloc(&chunk, kPinnedSlot * kPinnedChunk, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(FGB_ERR_OOM, "pinned host allocation failed");
    }
    for (size_t k = 1; k < kPinnedChunk; ++k)
        g_pinned_free.push_back(PinnedFree{static_cast<char *>(chunk) + k * kPinnedSlot, nullptr});
    *p = chunk;
    return FGB_OK;
}

void pinned_release(void *p, cudaEvent_t after) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    g_pinned_free.push_back(PinnedFree{p, after});
}

int set_memory_cache(size_t bytes) {
    std::lock_guard<std::mutex> lk(g_amu);
    g_cache_limit = bytes;
    release_kept_locked(bytes);
    uint64_t keep = bytes;
    for (int d = 0; d < 64; ++d)
        if (g_pool[d]) cudaMemPoolSetAttribute(g_pool[d], cudaMemPoolAttrReleaseThreshold, &keep);
    return FGB_OK;
}

int trim_memory() {
    std::lock_guard<std::mutex> lk(g_amu);
    release_kept_locked(0);
    for (int d = 0; d < 64; ++d)
        if (g_pool[d]) cudaMemPoolTrimTo(g_pool[d], 0);
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

extern "C" int fgb_set_memory_cache(uint64_t bytes) { return fgb::set_memory_cache((size_t)bytes); }

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
