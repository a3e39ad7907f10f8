// Pair kernels of the regularized Stokeslet and rotlet in FP32 or FP64,
// shared by the evaluator and the per-cluster error measurement.
#pragma once

#include "common.cuh"

namespace {

// ---------------------------------------------------------------------------
// Kernel math.  d = x - y, rho^2 = r^2 + eps^2, ri = 1/rho.  With
// r^2 = rho^2 - eps^2 the MRS functions of Eq. MRS_kernels become (times 8 pi):
//   H1 = ri + eps^2 ri^3,  H2 = ri^3,  Q = 2 ri^3 + 3 eps^2 ri^5,
//   D1 = -2 ri^3 - 3 eps^2 ri^5 + 15 eps^4 ri^7,  D2 = 6 ri^5 + 15 eps^2 ri^7.
// The common factor 1/(8 pi) is applied once per target at the end.
// A pair with rho = 0 (eps = 0, x = y) contributes nothing (Sec. 1).
// ---------------------------------------------------------------------------
template <int K> struct KT;
template <> struct KT<KITC_STOKESLET> { static constexpr int WIN = 3, WOUT = 3; };
template <> struct KT<KITC_ROTLET> { static constexpr int WIN = 3, WOUT = 6; };
template <> struct KT<KITC_STOKESLET_ROTLET> { static constexpr int WIN = 6, WOUT = 6; };
template <> struct KT<KITC_TEST_POLY> { static constexpr int WIN = 3, WOUT = 3; };

// 1/sqrt(v) on the MUFU in one instruction (approximate, <= 2 ulp; inputs are
// never subnormal: v >= eps^2 or a squared distance).  With EPS0 (eps = 0) a
// coincident pair (v = 0) gives 0, otherwise v > 0 and no guard is needed.
__device__ __forceinline__ float rsqrt_mufu(float v)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
template <bool EPS0> __device__ __forceinline__ float rsq(float v)
{
    if constexpr (EPS0) return v > 0.f ? rsqrt_mufu(v) : 0.f;
    else return rsqrt_mufu(v);
}
template <bool EPS0> __device__ __forceinline__ double rsq(double v)
{
    if constexpr (EPS0) return v > 0.0 ? rsqrt(v) : 0.0;
    else return rsqrt(v);
}

// u += k(x, y) f for one pair, given d = x - y and r2 = |d|^2 + eps^2
// (Eqs. Velocity_1, MRS_2).
template <int K, bool EPS0, typename R>
__device__ __forceinline__ void pair(R dx, R dy, R dz, const R *f, R e2, R e4, R *u, R r2)
{
    R ri = rsq<EPS0>(r2);
    R ri2 = ri * ri;
    R ri3 = ri2 * ri;
    if (K == KITC_STOKESLET || K == KITC_STOKESLET_ROTLET) {
        R H1 = fma(e2, ri3, ri);
        R fd = fma(f[0], dx, fma(f[1], dy, f[2] * dz));
        R s = fd * ri3;
        u[0] = fma(f[0], H1, fma(dx, s, u[0]));
        u[1] = fma(f[1], H1, fma(dy, s, u[1]));
        u[2] = fma(f[2], H1, fma(dz, s, u[2]));
    }
    if (K == KITC_ROTLET || K == KITC_STOKESLET_ROTLET) {
        const R *n = (K == KITC_ROTLET) ? f : f + 3;
        R ri5 = ri3 * ri2;
        R ri7 = ri5 * ri2;
        R hQ = fma(R(1.5) * e2, ri5, ri3);                              // Q / 2
        R qD1 = fma(R(3.75) * e4, ri7, fma(R(-0.75) * e2, ri5, R(-0.5) * ri3));  // D1 / 4
        R qD2 = fma(R(3.75) * e2, ri7, R(1.5) * ri5);                   // D2 / 4
        R nd = fma(n[0], dx, fma(n[1], dy, n[2] * dz));
        R t = nd * qD2;
        u[0] = fma(hQ, n[1] * dz - n[2] * dy, u[0]);
        u[1] = fma(hQ, n[2] * dx - n[0] * dz, u[1]);
        u[2] = fma(hQ, n[0] * dy - n[1] * dx, u[2]);
        u[3] = fma(n[0], qD1, fma(dx, t, u[3]));
        u[4] = fma(n[1], qD1, fma(dy, t, u[4]));
        u[5] = fma(n[2], qD1, fma(dz, t, u[5]));
        if (K == KITC_STOKESLET_ROTLET) {
            u[3] = fma(hQ, f[1] * dz - f[2] * dy, u[3]);
            u[4] = fma(hQ, f[2] * dx - f[0] * dz, u[4]);
            u[5] = fma(hQ, f[0] * dy - f[1] * dx, u[5]);
        }
    }
}

}  // namespace
