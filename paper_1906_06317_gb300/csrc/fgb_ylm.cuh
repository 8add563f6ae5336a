// Steinhardt bond-orientational order q_l (order module, Section "Analysis Modules";
// definition of Steinhardt, Nelson and Ronchetti 1983) and the gradient of the global
// Q = (1/N) sum_i q_l(i) with respect to the positions, neighbor list held fixed.
//
// Spherical harmonics in FP32 without trigonometry: for a unit bond u = (x, y, z),
//   Y_lm(u) = Abar_lm(z) (x + i y)^m,   Abar_lm = c_lm d^m P_l / dz^m,
//   c_lm = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
// with Abar_lm built by the three-term recurrence in l at fixed m (normalisation folded
// into the coefficients) and (x + i y)^m by repeated complex products.  m < 0 follows
// from Y_{l,-m} = (-1)^m conj(Y_lm), so sum_m |Q_lm|^2 = |Q_l0|^2 + 2 sum_{m>0} |Q_lm|^2.
// The gradient uses the same basis: Y~_lm(u) = Abar_lm(z) (x + i y)^m is a homogeneous
// polynomial of degree l, so
//   d/dx Y~ = m Abar_lm w^(m-1),  d/dy Y~ = i m Abar_lm w^(m-1),
//   d/dz Y~ = (c_lm / c_l,m+1) Abar_l,m+1 w^m,
// projected on the sphere with (I - u u^T)/|d|, and the gradient at -u is (-1)^(l-1)
// times the gradient at u.
#pragma once

#include <cmath>
#include <cstring>

#include "fgb_internal.cuh"

namespace fgb {

constexpr int kLMax = 12;

struct LegendreConsts {
    float amm[kLMax + 1];                  // Abar_mm
    float first[kLMax + 1];                // Abar_{m+1,m} = first[m] z Abar_mm
    float alpha[kLMax + 1][kLMax + 1];     // Abar_lm = alpha z Abar_{l-1,m} - beta Abar_{l-2,m}
    float beta[kLMax + 1][kLMax + 1];
    float gamma[kLMax + 1][kLMax + 2];     // d Abar_lm / dz = gamma Abar_{l,m+1}
};

// Each translation unit that includes this header holds its own copy, filled by
// ensure_consts() before its first launch.
static __constant__ LegendreConsts c_leg;

static int ensure_consts() {
    static bool done = false;
    if (done) return FGB_OK;
    auto fact = [](int n) {
        double f = 1;
        for (int i = 2; i <= n; ++i) f *= i;
        return f;
    };
    auto c = [&](int l, int m) {
        return ((m & 1) ? -1.0 : 1.0) * std::sqrt((2 * l + 1) / (4.0 * M_PI) * fact(l - m) / fact(l + m));
    };
    LegendreConsts h;
    memset(&h, 0, sizeof(h));
    for (int m = 0; m <= kLMax; ++m) {
        double dfact = 1;  // (2m-1)!!
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
        h.amm[m] = (float)(c(m, m) * dfact);
        if (m + 1 <= kLMax) h.first[m] = (float)((2 * m + 1) * c(m + 1, m) / c(m, m));
        for (int l = m + 2; l <= kLMax; ++l) {
            h.alpha[l][m] = (float)((2.0 * l - 1) / (l - m) * c(l, m) / c(l - 1, m));
            h.beta[l][m] = (float)((double)(l + m - 1) / (l - m) * c(l, m) / c(l - 2, m));
        }
    }
    for (int l = 0; l <= kLMax; ++l)
        for (int m = 0; m < l; ++m) h.gamma[l][m] = (float)(c(l, m) / c(l, m + 1));
    FGB_CUDA(cudaMemcpyToSymbol(c_leg, &h, sizeof(h)));
    done = true;
    return FGB_OK;
}

// Abar_Lm(z) for m = 0..L (A[L+1] = 0 for the derivative).
template <int L>
__device__ __forceinline__ void legendre_row(float z, float (&A)[L + 2]) {
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        float p0 = c_leg.amm[m];
        if (m == L) {
            A[m] = p0;
            continue;
        }
        float p1 = c_leg.first[m] * z * p0;
#pragma unroll
        for (int l = m + 2; l <= L; ++l) {
            const float p2 = c_leg.alpha[l][m] * z * p1 - c_leg.beta[l][m] * p0;
            p0 = p1;
            p1 = p2;
        }
        A[m] = p1;
    }
    A[L + 1] = 0.f;
}

template <int L>
__device__ __forceinline__ void powers(float x, float y, float (&wr)[L + 1], float (&wi)[L + 1]) {
    wr[0] = 1.f;
    wi[0] = 0.f;
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        wr[m] = wr[m - 1] * x - wi[m - 1] * y;
        wi[m] = wr[m - 1] * y + wi[m - 1] * x;
    }
}

template <int L>
__device__ __forceinline__ void accumulate_bond(float3 d, float (&sr)[L + 1], float (&si)[L + 1]) {
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    if (!(r2 > 0.f)) return;  // coincident points have no bond direction
    const float inv = rsqrtf(r2);
    float A[L + 2], wr[L + 1], wi[L + 1];
    legendre_row<L>(d.z * inv, A);
    powers<L>(d.x * inv, d.y * inv, wr, wi);
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        sr[m] += A[m] * wr[m];
        si[m] += A[m] * wi[m];
    }
}

// Y~_Lm(u) for m = 0..L of one bond (real and imaginary parts); all zero for a zero
// displacement, which has no bond direction.
template <int L>
__device__ __forceinline__ void bond_harmonics(float3 d, float (&yr)[L + 1], float (&yi)[L + 1]) {
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    if (!(r2 > 0.f)) {
#pragma unroll
        for (int m = 0; m <= L; ++m) yr[m] = yi[m] = 0.f;
        return;
    }
    const float inv = rsqrtf(r2);
    float A[L + 2], wr[L + 1], wi[L + 1];
    legendre_row<L>(d.z * inv, A);
    powers<L>(d.x * inv, d.y * inv, wr, wi);
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        yr[m] = A[m] * wr[m];
        yi[m] = A[m] * wi[m];
    }
}

// Bonds met during a neighbor walk, accumulated after it (or whenever the buffer fills):
// inside the walk only the hit branch would evaluate the harmonics, with the warp's lanes
// that found no neighbor idle, while a separate loop keeps them in step.  Bonds are
// accumulated in the order met, so the sums equal accumulating them in the walk.
constexpr int kBondBuf = 32;

template <int L>
struct BondBuffer {
    float3 d[kBondBuf];
    int nb = 0;
    __device__ __forceinline__ void add(float3 v, float (&sr)[L + 1], float (&si)[L + 1]) {
        d[nb++] = v;
        if (nb == kBondBuf) flush(sr, si);
    }
    __device__ __forceinline__ void flush(float (&sr)[L + 1], float (&si)[L + 1]) {
        for (int k = 0; k < nb; ++k) accumulate_bond<L>(d[k], sr, si);
        nb = 0;
    }
};

// Raw gradient of Re sum_m f_m conj(Q_m) Y~_m at u (before projection), f_0 = 1, f_m = 2.
template <int L>
__device__ __forceinline__ float3 contract_grad(const float (&A)[L + 2], const float (&wr)[L + 1],
                                                const float (&wi)[L + 1], const float2 *Q) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        const float2 q = Q[m];
        const float f = m == 0 ? 1.f : 2.f;
        if (m > 0) {
            const float am = A[m] * (float)m;
            const float pr = wr[m - 1], pi = wi[m - 1];
            gx += f * am * (q.x * pr + q.y * pi);
            gy += f * am * (q.y * pr - q.x * pi);
        }
        if (m < L) {
            const float g = c_leg.gamma[L][m] * A[m + 1];
            gz += f * g * (q.x * wr[m] + q.y * wi[m]);
        }
    }
    return make_float3(gx, gy, gz);
}

// (I - u u^T) g / r
__device__ __forceinline__ float3 project(float3 g, float3 u, float inv_r) {
    const float ug = u.x * g.x + u.y * g.y + u.z * g.z;
    return make_float3((g.x - ug * u.x) * inv_r, (g.y - ug * u.y) * inv_r, (g.z - ug * u.z) * inv_r);
}

template <int L>
__device__ __forceinline__ void finish(int64_t i, int n, const float (&sr)[L + 1], const float (&si)[L + 1], float *q,
                                       float2 *Q, int32_t *nn) {
    float s = sr[0] * sr[0] + si[0] * si[0];
#pragma unroll
    for (int m = 1; m <= L; ++m) s += 2.f * (sr[m] * sr[m] + si[m] * si[m]);
    const float invn = n > 0 ? 1.f / (float)n : 0.f;
    q[i] = n > 0 ? sqrtf(4.f * (float)M_PI / (2 * L + 1) * s) * invn : 0.f;
#pragma unroll
    for (int m = 0; m <= L; ++m) Q[i * (L + 1) + m] = make_float2(sr[m] * invn, si[m] * invn);
    nn[i] = n;
}

}  // namespace fgb
