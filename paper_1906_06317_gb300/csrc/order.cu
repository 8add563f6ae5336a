// Variants of the Steinhardt order parameters and the per-bond descriptors built on the
// same spherical harmonics (order and environment modules, Section "Analysis Modules"):
//
//  * W_l, the third-order rotational invariant of Steinhardt, Nelson and Ronchetti (1983):
//      w_l(i) = sum_{m1+m2+m3=0} (l l l; m1 m2 m3) Q_lm1(i) Q_lm2(i) Q_lm3(i),
//    and its normalised form w_l / (sum_m |Q_lm(i)|^2)^{3/2};
//  * the neighbor-averaged q_l of Lechner and Dellago (2008):
//      Qbar_lm(i) = (Q_lm(i) + sum_{k in nb(i)} Q_lm(k)) / (n_i + 1);
//  * LocalDescriptors: Y_lm of every bond of a NeighborList, l <= l_max.
//
// Q_lm for m < 0 follow from Q_{l,-m} = (-1)^m conj(Q_lm).  The Wigner 3j symbols come
// from Racah's closed formula, summed in long double on the host, once per l.
#include <cmath>
#include <cstring>
#include <vector>

#include "fgb_device.cuh"
#include "fgb_ylm.cuh"

namespace fgb {

// ------------------------------------------------------------------ Wigner 3j (host)

static long double lfact(int n) {
    long double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// (j1 j2 j3; m1 m2 m3) by Racah's formula: a sign, the square root of the triangle
// coefficient and of the six (j +- m)! factors, and an alternating sum over the integers
// k for which every factorial argument is non-negative.
static double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
    const long double tri = lfact(j1 + j2 - j3) * lfact(j1 - j2 + j3) * lfact(-j1 + j2 + j3) / lfact(j1 + j2 + j3 + 1);
    const long double pre = std::sqrt(tri * lfact(j1 + m1) * lfact(j1 - m1) * lfact(j2 + m2) * lfact(j2 - m2) *
                                      lfact(j3 + m3) * lfact(j3 - m3));
    const int kmin = std::max(0, std::max(j2 - j3 - m1, j1 - j3 + m2));
    const int kmax = std::min(j1 + j2 - j3, std::min(j1 - m1, j2 + m2));
    long double sum = 0;
    for (int k = kmin; k <= kmax; ++k) {
        const long double den = lfact(k) * lfact(j3 - j2 + k + m1) * lfact(j3 - j1 + k - m2) * lfact(j1 + j2 - j3 - k) *
                                lfact(j1 - k - m1) * lfact(j2 - k + m2);
        sum += ((k & 1) ? -1.0L : 1.0L) / den;
    }
    const int e = j1 - j2 - m3;
    const long double sign = (((e % 2) + 2) % 2) ? -1.0L : 1.0L;
    return (double)(sign * pre * sum);
}

// Table t[(m1 + l)(2l + 1) + m2 + l] = (l l l; m1 m2 -m1-m2) on the device.
static int ensure_w3j(fgb_steinhardt *st, cudaStream_t s) {
    if (st->w3j) return FGB_OK;
    const int l = st->l, w = 2 * l + 1;
    std::vector<float> t((size_t)w * w, 0.f);
    for (int m1 = -l; m1 <= l; ++m1)
        for (int m2 = -l; m2 <= l; ++m2)
            if (std::abs(m1 + m2) <= l) t[(size_t)(m1 + l) * w + (m2 + l)] = (float)wigner3j(l, l, l, m1, m2, -m1 - m2);
    FGB_TRY(dalloc_n(&st->w3j, (size_t)w * w, s));
    FGB_CUDA(cudaMemcpyAsync(st->w3j, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice, s));
    FGB_CUDA(cudaStreamSynchronize(s));  // t is a host temporary
    return FGB_OK;
}

// ------------------------------------------------------------------ W_l

// Q_lm for m = -L..L from the stored m >= 0 half.
template <int L>
__device__ __forceinline__ void full_q(const float2 *Qi, float (&qr)[2 * L + 1], float (&qi)[2 * L + 1]) {
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        const float2 v = Qi[m];
        qr[L + m] = v.x;
        qi[L + m] = v.y;
        const float sg = (m & 1) ? -1.f : 1.f;
        qr[L - m] = sg * v.x;
        qi[L - m] = -sg * v.y;
    }
}

template <int L>
__global__ void __launch_bounds__(128) k_st_wl(const float2 *__restrict__ Q, int64_t n, const float *__restrict__ t,
                                               int normalize, float *__restrict__ w_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int W = 2 * L + 1;
    float qr[W], qi[W];
    full_q<L>(Q + i * (L + 1), qr, qi);
    float w = 0.f;
#pragma unroll
    for (int a = 0; a < W; ++a) {
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const int c = 3 * L - a - b;  // m3 = -m1 - m2 in index space
            if (c < 0 || c >= W) continue;
            // Re(Q_a Q_b Q_c)
            const float pr = qr[a] * qr[b] - qi[a] * qi[b];
            const float pi = qr[a] * qi[b] + qi[a] * qr[b];
            w = fmaf(__ldg(t + a * W + b), pr * qr[c] - pi * qi[c], w);
        }
    }
    if (normalize) {
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < W; ++a) s = fmaf(qr[a], qr[a], fmaf(qi[a], qi[a], s));
        w = s > 0.f ? w / (s * sqrtf(s)) : 0.f;
    }
    w_out[i] = w;
}

// ------------------------------------------------------------------ averaged q_l

template <int L>
__global__ void __launch_bounds__(128) k_st_average(const float2 *__restrict__ Q, const int64_t *__restrict__ seg,
                                                    const int32_t *__restrict__ pj, int64_t n, float2 *__restrict__ Qbar,
                                                    float *__restrict__ q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float sr[L + 1], si[L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        const float2 v = Q[i * (L + 1) + m];
        sr[m] = v.x;
        si[m] = v.y;
    }
    const int64_t beg = seg[i], end = seg[i + 1];
    for (int64_t e = beg; e < end; ++e) {
        const float2 *Qk = Q + (int64_t)pj[e] * (L + 1);
#pragma unroll
        for (int m = 0; m <= L; ++m) {
            const float2 v = __ldg(Qk + m);
            sr[m] += v.x;
            si[m] += v.y;
        }
    }
    const float inv = 1.f / (float)(end - beg + 1);
    float s = 0.f;
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        sr[m] *= inv;
        si[m] *= inv;
        s += (m == 0 ? 1.f : 2.f) * (sr[m] * sr[m] + si[m] * si[m]);
        Qbar[i * (L + 1) + m] = make_float2(sr[m], si[m]);
    }
    q[i] = sqrtf(4.f * (float)M_PI / (2 * L + 1) * s);
}

// ------------------------------------------------------------------ LocalDescriptors

// Y_lm of one bond for l = 0..LM, m = 0..l, as Abar_lm(z) (x + i y)^m.  Row l of Abar is
// built by the same recurrence in l at fixed m as the Steinhardt kernels.
template <int LM>
__device__ __forceinline__ void ylm_all(float3 u, float (&yr)[(LM + 1) * (LM + 2) / 2], float (&yi)[(LM + 1) * (LM + 2) / 2]) {
    float wr[LM + 1], wi[LM + 1];
    powers<LM>(u.x, u.y, wr, wi);
#pragma unroll
    for (int m = 0; m <= LM; ++m) {
        float p0 = c_leg.amm[m], p1 = 0.f;
#pragma unroll
        for (int l = m; l <= LM; ++l) {
            float a;
            if (l == m) {
                a = p0;
            } else if (l == m + 1) {
                p1 = c_leg.first[m] * u.z * p0;
                a = p1;
            } else {
                const float p2 = c_leg.alpha[l][m] * u.z * p1 - c_leg.beta[l][m] * p0;
                p0 = p1;
                p1 = p2;
                a = p2;
            }
            const int idx = l * (l + 1) / 2 + m;
            yr[idx] = a * wr[m];
            yi[idx] = a * wi[m];
        }
    }
}

constexpr int kDescWarps = 2;

// One thread per bond writes its n_sph values into a per-warp shared block, then the warp
// stores the 32 bonds' contiguous output with coalesced 8-byte stores.
template <int LM>
__global__ void __launch_bounds__(kDescWarps * 32) k_descriptors(BoxF b, const float *__restrict__ p,
                                                                 const float *__restrict__ qp,
                                                                 const int32_t *__restrict__ qi,
                                                                 const int32_t *__restrict__ pj, int64_t m,
                                                                 int negative_m, int nsph, float2 *__restrict__ out) {
    extern __shared__ float2 sdesc[];  // kDescWarps * 32 * nsph
    constexpr int NT = (LM + 1) * (LM + 2) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e0 = ((int64_t)blockIdx.x * kDescWarps + warp) * 32;
    if (e0 >= m) return;
    float2 *blk = sdesc + (size_t)warp * 32 * nsph;
    const int64_t e = e0 + lane;
    if (e < m) {
        const int i = qi[e], j = pj[e];
        const float3 d = bond_f32v(b, __ldg(qp + 3 * i), __ldg(qp + 3 * i + 1), __ldg(qp + 3 * i + 2), __ldg(p + 3 * j),
                                   __ldg(p + 3 * j + 1), __ldg(p + 3 * j + 2));
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        float yr[NT], yi[NT];
        if (r2 > 0.f) {
            const float inv = rsqrtf(r2);
            ylm_all<LM>(make_float3(d.x * inv, d.y * inv, d.z * inv), yr, yi);
        } else {
#pragma unroll
            for (int k = 0; k < NT; ++k) yr[k] = yi[k] = 0.f;  // coincident points: no bond direction
        }
        float2 *row = blk + (size_t)lane * nsph;
        int o = 0;
#pragma unroll
        for (int l = 0; l <= LM; ++l) {
            if (negative_m) {
#pragma unroll
                for (int mm = l; mm >= 1; --mm) {  // m = -l .. -1: (-1)^m conj(Y_l|m|)
                    const int idx = l * (l + 1) / 2 + mm;
                    const float sg = (mm & 1) ? -1.f : 1.f;
                    row[o++] = make_float2(sg * yr[idx], -sg * yi[idx]);
                }
            }
#pragma unroll
            for (int mm = 0; mm <= l; ++mm) {
                const int idx = l * (l + 1) / 2 + mm;
                row[o++] = make_float2(yr[idx], yi[idx]);
            }
        }
    }
    __syncwarp();
    const int64_t nb = min((int64_t)32, m - e0);
    const int64_t total = nb * nsph;
    float2 *dst = out + e0 * nsph;
    for (int64_t k = lane; k < total; k += 32) __stcs(dst + k, blk[k]);
}

// ------------------------------------------------------------------ launchers

template <template <int> class F, class... Args>
static bool dispatch_order(int l, Args &&...args) {
    switch (l) {
#define FGB_L(V)                                \
    case V:                                     \
        F<V>::run(std::forward<Args>(args)...); \
        return true;
        FGB_L(0) FGB_L(1) FGB_L(2) FGB_L(3) FGB_L(4) FGB_L(5) FGB_L(6) FGB_L(7) FGB_L(8) FGB_L(9) FGB_L(10) FGB_L(11)
        FGB_L(12)
#undef FGB_L
    }
    return false;
}

template <int L>
struct RunWl {
    static void run(const float2 *Q, int64_t n, const float *t, int normalize, float *w, cudaStream_t s) {
        FGB_KSCOPE("k_st_wl", s);
        k_st_wl<L><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(Q, n, t, normalize, w);
    }
};

template <int L>
struct RunAverage {
    static void run(const float2 *Q, const fgb_nlist *nl, int64_t n, float2 *Qbar, float *q, cudaStream_t s) {
        FGB_KSCOPE("k_st_average", s);
        k_st_average<L><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(Q, nl->segments, nl->pj, n, Qbar, q);
    }
};

template <int L>
struct RunDesc {
    static int run(const BoxF &b, const float *p, const float *qp, const fgb_nlist *nl, int negative_m, int nsph,
                   float2 *out, cudaStream_t s) {
        const size_t smem = (size_t)kDescWarps * 32 * nsph * sizeof(float2);
        FGB_CUDA(cudaFuncSetAttribute(k_descriptors<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int64_t blocks = (nl->n_pairs + kDescWarps * 32 - 1) / (kDescWarps * 32);
        FGB_KSCOPE("k_descriptors", s);
        k_descriptors<L><<<(unsigned)blocks, kDescWarps * 32, smem, s>>>(b, p, qp, nl->qi, nl->pj, nl->n_pairs,
                                                                          negative_m, nsph, out);
        return FGB_OK;
    }
};

}  // namespace fgb

using namespace fgb;

extern "C" int fgb_steinhardt_wl(fgb_steinhardt *st, int32_t normalize, float *w_out, void *stream) {
    clear_error();
    if (!st) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    if (!st->Q) return fail(FGB_ERR_INVALID_ARG, "call fgb_steinhardt_compute first");
    if (st->n > 0 && !w_out) return fail(FGB_ERR_INVALID_ARG, "w_out is NULL");
    cudaStream_t s = as_stream(stream);
    FGB_TRY(ensure_w3j(st, s));
    if (st->n == 0) return FGB_OK;
    dispatch_order<RunWl>(st->l, st->Q, st->n, st->w3j, normalize ? 1 : 0, w_out, s);
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}

extern "C" int fgb_steinhardt_average(fgb_steinhardt *st, const fgb_nlist *nlist, float *q_out, void *stream) {
    clear_error();
    if (!st || !nlist) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    if (!st->Q) return fail(FGB_ERR_INVALID_ARG, "call fgb_steinhardt_compute first");
    if (nlist->n_query != st->n || nlist->n_points != st->n)
        return fail(FGB_ERR_INVALID_ARG, "the averaging needs a self neighbor list over the same points");
    if (st->n > 0 && !q_out) return fail(FGB_ERR_INVALID_ARG, "q_out is NULL");
    cudaStream_t s = as_stream(stream);
    if (!st->Qtmp) FGB_TRY(dalloc_n(&st->Qtmp, (size_t)st->n * (st->l + 1), s));
    if (st->n > 0) {
        dispatch_order<RunAverage>(st->l, st->Q, nlist, st->n, st->Qtmp, q_out, s);
        FGB_LAUNCH_CHECK();
    }
    std::swap(st->Q, st->Qtmp);
    st->averaged = 1;
    return FGB_OK;
}

extern "C" int fgb_local_descriptors(const fgb_box *box, const float *points, const float *query_points,
                                     const fgb_nlist *nlist, int32_t l_max, int32_t negative_m, float *out,
                                     void *stream) {
    clear_error();
    if (!box || !points || !nlist) return fail(FGB_ERR_INVALID_ARG, "NULL argument");
    FGB_TRY(nlist_ready(nlist));
    if (l_max < 0 || l_max > kLMax) return fail(FGB_ERR_INVALID_ARG, "l_max must be in [0, %d]", kLMax);
    if (nlist->n_pairs > 0 && !out) return fail(FGB_ERR_INVALID_ARG, "out is NULL");
    BoxHost b;
    FGB_TRY(make_box(box, &b));
    FGB_TRY(ensure_consts());
    if (nlist->n_pairs == 0) return FGB_OK;
    const int nsph = negative_m ? (l_max + 1) * (l_max + 1) : (l_max + 1) * (l_max + 2) / 2;
    cudaStream_t s = as_stream(stream);
    int st = FGB_OK;
    switch (l_max) {
#define FGB_D(V)                                                                                                   \
    case V:                                                                                                        \
        st = RunDesc<V>::run(b.f, points, query_points ? query_points : points, nlist, negative_m ? 1 : 0, nsph, \
                             reinterpret_cast<float2 *>(out), s);                                                  \
        break;
        FGB_D(0) FGB_D(1) FGB_D(2) FGB_D(3) FGB_D(4) FGB_D(5) FGB_D(6) FGB_D(7) FGB_D(8) FGB_D(9) FGB_D(10) FGB_D(11)
        FGB_D(12)
#undef FGB_D
    }
    FGB_TRY(st);
    FGB_LAUNCH_CHECK();
    return FGB_OK;
}
