// Exclusive prefix sums: per-tile reduce, scan of tile sums, per-tile downsweep.
// No device-side waits: three ordinary launches.
#include "fgb_internal.cuh"

namespace fgb {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr int kTopThreads = 1024;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += u;
    }
    return v;
}

// Exclusive block scan of one value per thread; returns the block total in `total`.
template <class T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T &total) {
    __shared__ T warp_sums[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < NT / 32 ? warp_sums[lane] : T(0);
        s = warp_incl_scan(s);
        if (lane < NT / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    T base = w ? warp_sums[w - 1] : T(0);
    total = warp_sums[NT / 32 - 1];
    __syncthreads();
    return base + inc - v;
}

template <class TI, class TO>
__global__ void __launch_bounds__(kThreads) k_reduce(const TI *__restrict__ in, int64_t n, TO *__restrict__ partial,
                                                     uint32_t *__restrict__ pmax) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    TO sum = 0;
    uint32_t mx = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + k * kThreads + threadIdx.x;
        if (i < n) {
            TI v = in[i];
            sum += (TO)v;
            mx = max(mx, (uint32_t)v);
        }
    }
    __shared__ TO s_sum[kThreads / 32];
    __shared__ uint32_t s_max[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s_sum[threadIdx.x >> 5] = sum;
        s_max[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        TO t = 0;
        uint32_t m = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            t += s_sum[w];
            m = max(m, s_max[w]);
        }
        partial[blockIdx.x] = t;
        if (pmax) pmax[blockIdx.x] = m;
    }
}

template <class TO>
__global__ void __launch_bounds__(kTopThreads) k_top(TO *partial, int64_t nb, TO *total_out, const uint32_t *pmax,
                                                     uint32_t *max_out) {
    TO carry = 0;
    uint32_t mx = 0;
    for (int64_t c = 0; c < nb; c += kTopThreads) {
        int64_t i = c + threadIdx.x;
        TO v = i < nb ? partial[i] : TO(0);
        if (pmax && i < nb) mx = max(mx, pmax[i]);
        TO tot;
        TO ex = block_excl_scan<TO, kTopThreads>(v, tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
    if (max_out) {
        __shared__ uint32_t s_m[kTopThreads / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t m = 0;
            for (int w = 0; w < kTopThreads / 32; ++w) m = max(m, s_m[w]);
            *max_out = m;
        }
    }
}

template <class TI, class TO>
__global__ void __launch_bounds__(kThreads) k_down(const TI *__restrict__ in, int64_t n, const TO *__restrict__ partial,
                                                   TO *__restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    TO v[kItems];
    TO run = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + k;
        TO x = i < n ? (TO)in[i] : TO(0);
        v[k] = run;
        run += x;
    }
    TO tot;
    TO pre = block_excl_scan<TO, kThreads>(run, tot) + partial[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = pre + v[k];
    }
}

// ws: at least nb * (sizeof(TO) + 4) bytes, nb = ceil(n / kTile); NULL allocates.
template <class TI, class TO>
int scan_impl(const TI *in, TO *out, int64_t n, uint32_t *max_out, void *ws, cudaStream_t s) {
    if (n < 0) return fail(FGB_ERR_INVALID_ARG, "scan: negative length");
    if (n == 0) {
        FGB_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), s));
        if (max_out) FGB_CUDA(cudaMemsetAsync(max_out, 0, sizeof(uint32_t), s));
        return FGB_OK;
    }
    const int64_t nb = (n + kTile - 1) / kTile;
    TO *partial = nullptr;
    uint32_t *pmax = nullptr;
    const bool own = ws == nullptr;
    if (own) {
        FGB_TRY(dalloc(&ws, nb * (sizeof(TO) + sizeof(uint32_t)) + 256, s));
    }
    partial = static_cast<TO *>(ws);
    if (max_out) pmax = reinterpret_cast<uint32_t *>(partial + nb);
    {
        FGB_KSCOPE("k_reduce", s);
        k_reduce<TI, TO><<<(unsigned)nb, kThreads, 0, s>>>(in, n, partial, pmax);
    }
    {
        FGB_KSCOPE("k_top", s);
        k_top<TO><<<1, kTopThreads, 0, s>>>(partial, nb, out + n, pmax, max_out);
    }
    {
        FGB_KSCOPE("k_down", s);
        k_down<TI, TO><<<(unsigned)nb, kThreads, 0, s>>>(in, n, partial, out);
    }
    cudaError_t e = cudaGetLastError();
    if (own) dfree(ws, s);
    if (e != cudaSuccess) return fail(FGB_ERR_CUDA, "scan launch failed: %s", cudaGetErrorString(e));
    return FGB_OK;
}

}  // namespace

size_t scan_ws_bytes(int64_t n) { return (size_t)((n + kTile - 1) / kTile) * 12 + 256; }

int scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n, uint32_t *max_out, cudaStream_t s) {
    return scan_impl<uint32_t, int64_t>(in, out, n, max_out, nullptr, s);
}

int scan_u32_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<uint32_t, uint32_t>(in, out, n, nullptr, nullptr, s);
}

int scan_u32_u32_ws(const uint32_t *in, uint32_t *out, int64_t n, void *ws, cudaStream_t s) {
    return scan_impl<uint32_t, uint32_t>(in, out, n, nullptr, ws, s);
}

}  // namespace fgb
