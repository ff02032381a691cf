// Device building blocks of the SANS trace: Philox4x32-10, the neutron
// history geometry, the fourteen form-factor models with their
// polydispersity and orientation quadratures (or per-event draws), the
// shape-independent laws, the Percus-Yevick structure factor and the
// self-attenuation table. Templated on the
// arithmetic type: float (FP32 trace: sin, cos and sine from the
// special-function unit where the tolerances allow, own polynomial forms of
// 2 J1(x)/x and of the small-argument series) or double (FP64 trace, CUDA's
// double precision math functions).
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>
#include "sas_math.cuh"
#include "sas_types.h"

namespace sas {

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplications with the round constants 0xD2511F53 and
// 0xCD9E8D57, key schedule incremented by the Weyl constants 0x9E3779B9 and
// 0xBB67AE85.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// uniform on (0,1): 23 random bits plus one half (exact in float and double)
template <typename T>
__device__ __forceinline__ T u01(uint32_t x)
{
    return (T)((x >> 9) | 0u) * (T)(1.0 / 8388608.0) + (T)(0.5 / 8388608.0);
}

// FP32: the same value without an integer-to-float conversion: the 23 bits
// as the mantissa of a float in [1, 2), minus (1 - 2^-24); exact.
template <>
__device__ __forceinline__ float u01<float>(uint32_t x)
{
    return __uint_as_float((x >> 9) | 0x3F800000u) - 0.99999994f;
}

// (float)k for 0 <= k < 2^23 without a conversion instruction (exact)
__device__ __forceinline__ float small_uint_to_float(uint32_t k)
{
    return __uint_as_float(k | 0x4B000000u) - 8388608.0f;
}

// --------------------------------------------------------------- math glue
template <typename T> struct M;

template <> struct M<float> {
    static __device__ __forceinline__ float erfcinv_(float y) { return erfcinvf(y); }
    static __device__ __forceinline__ void sincospi_(float u, float& s, float& c) { sincospif(u, &s, &c); }
    // approximate reciprocal (2 ulp; the trace's tolerances are 1e-5)
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    // approximate square root (1 ulp; 0 -> 0)
    static __device__ __forceinline__ float sqrt_(float x)
    {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    // x > 0 only: x / sqrt(x) by the approximate reciprocal square root
    static __device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrtf(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float exp_(float x) { return __expf(x); }
    // sin, cos of 2 pi u for u in (0, 1) from the special-function unit
    // (absolute error about 1e-6: pinhole points to a few nanometres)
    static __device__ __forceinline__ void sincos2pi(float u, float& s, float& c)
    {
        __sincosf(6.283185307f * u, &s, &c);
    }
    static __device__ __forceinline__ void sincos_(float x, float& s, float& c)
    {
        sas_sincosf(x, s, c);
    }
    // (sin x - x cos x) / x^3 = f(x) / 3 for x >= 0, inv = 1 / x: sin and
    // cos from the special-function unit for x >= 1.5 (relative error of
    // the closed form below 2e-6 there), the five-term series below
    static __device__ __forceinline__ float sphere_g(float x, float inv)
    {
        float s, c;
        __sincosf(x, &s, &c);
        const float big = fmaf(-x, c, s) * (inv * inv * inv);
        const float t = x * x;
        float h = fmaf(2.505210839e-07f, t, -2.204585538e-05f);
        h = fmaf(h, t, 1.190476190e-03f);
        h = fmaf(h, t, -3.333333333e-02f);
        h = fmaf(h, t, 3.333333333e-01f);
        return x < 1.5f ? h : big;
    }
    // sin(y) / y for y >= 0, inv = 1 / y: the SFU's sine (absolute error
    // about 1e-6, so 1e-6 / y in the sinc) for y >= 0.5, the series to y^6
    // below (truncation 1e-8)
    static __device__ __forceinline__ float sinc(float y, float inv)
    {
        const float t = y * y;
        float h = fmaf(-1.984126984e-04f, t, 8.333333333e-03f);
        h = fmaf(h, t, -1.666666667e-01f);
        h = fmaf(h, t, 1.0f);
        return y < 0.5f ? h : __sinf(y) * inv;
    }
    static __device__ __forceinline__ float cyl_a(float x, float inv, float rsx)
    {
        return sas_cyl_a(x, inv, rsx);
    }
};

template <> struct M<double> {
    static __device__ __forceinline__ double erfcinv_(double y) { return erfcinv(y); }
    static __device__ __forceinline__ void sincospi_(double u, double& s, double& c) { sincospi(u, &s, &c); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double sqrt_(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double sqrt_pos(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    static __device__ __forceinline__ double exp_(double x) { return ::exp(x); }
    static __device__ __forceinline__ void sincos2pi(double u, double& s, double& c)
    {
        sincospi(2.0 * u, &s, &c);
    }
    static __device__ __forceinline__ void sincos_(double x, double& s, double& c)
    {
        sincos(x, &s, &c);
    }
    // (sin x - x cos x) / x^3 = f(x) / 3
    static __device__ __forceinline__ double sphere_g(double x, double inv)
    {
        if (x < 0.1) {   // Taylor series of j1(x)/x
            const double t = x * x;
            return (1.0 - t * (1.0 / 10.0) + t * t * (1.0 / 280.0) - t * t * t * (1.0 / 15120.0)
                    + t * t * t * t * (1.0 / 1330560.0)) * (1.0 / 3.0);
        }
        double s, c;
        sincos(x, &s, &c);
        return (s - x * c) * inv * inv * inv;
    }
    static __device__ __forceinline__ double sinc(double y, double inv)
    {
        return (y < 1e-8) ? 1.0 : sin(y) * inv;
    }
    static __device__ __forceinline__ double cyl_a(double x, double inv, double)
    {
        return (x < 1e-6) ? 1.0 - 0.125 * x * x : 2.0 * j1(x) * inv;
    }
};

// ----------------------------------------------------------- Percus-Yevick
// S(q) = 1 / (1 + 24 phi G(A)/A), A = 2 q R (hard-sphere closed form);
// below A = switch the series of G(A)/A in A^2 prepared on the host.
template <typename T>
__device__ __forceinline__ T structure_factor(T q, const ModelConst<T>& mc)
{
    if (mc.sq_kind == SAS_SQ_HAYTER_MSA) {
        // cubic Hermite on the host-solved table; beyond it S - 1 decays as Q^-2
        const T s = q * mc.sq_inv_dq;
        const int last = mc.sq_n - 1;
        if (!(s < (T)last)) {
            const T r = (T)last / s;
            return (T)1 + (mc.sq_tab[2 * last] - (T)1) * r * r;
        }
        const int i = (int)s;
        const T f = s - (T)i, f1 = (T)1 - f;
        const T* p = mc.sq_tab + 2 * i;
        // h00 = (1 + 2f)(1 - f)^2, h10 = f (1 - f)^2, h01 = f^2 (3 - 2f), h11 = f^2 (f - 1)
        return f1 * f1 * fma((T)2 * f + (T)1, p[0], f * p[1]) + f * f * fma((T)3 - (T)2 * f, p[2], -f1 * p[3]);
    }
    if (mc.sq_kind != SAS_SQ_HARD_SPHERE_PY) return (T)1;
    const T A = q * mc.sq_2r;
    T ga;
    if (A < mc.sq_switch) {
        const T a2 = A * A;
        T r = mc.sq_series[SAS_SQ_NSER - 1];
#pragma unroll
        for (int k = SAS_SQ_NSER - 2; k >= 0; --k) r = fma(r, a2, mc.sq_series[k]);
        ga = r;
    } else {
        T s, c;
        M<T>::sincos_(A, s, c);
        const T iA = M<T>::rcp(A);
        const T A2 = A * A;
        const T b1 = s - A * c;
        const T b2 = (T)2 * A * s + ((T)2 - A2) * c - (T)2;
        const T b3 = -A2 * A2 * c + (T)4 * (((T)3 * A2 - (T)6) * c + (A2 * A - (T)6 * A) * s + (T)6);
        const T i3 = iA * iA * iA;
        ga = i3 * (mc.sq_alpha * b1 + iA * (mc.sq_beta * b2 + iA * iA * mc.sq_gamma * b3));
    }
    return M<T>::rcp((T)1 + mc.sq_24phi * ga);
}

// ---------------------------------------------------------------- models
// Quadrature tables (see sas_types.h for the per-kind layout):
//   poly   [n_poly][8]  nodes of the polydisperse radius with folded weights
//   orient [n_orient][4] axis unit vector and normalised weight
// Returns <|F|^2> (without the phi/<V> factor and S(Q)).

template <typename T>
__device__ __forceinline__ T avg_sphere(T q, T iq, const T* __restrict__ poly, int np)
{
    T acc = 0;
#pragma unroll 4
    for (int i = 0; i < np; ++i) {
        const T* p = poly + 8 * i;
        const T g = M<T>::sphere_g(q * p[0], iq * p[4]);
        acc = fma(p[2], g * g, acc);
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ T avg_core_shell(T q, T iq, const T* __restrict__ poly, int np, T shell)
{
    T acc = 0;
    if constexpr (sizeof(T) == sizeof(float)) {
        // sin and cos of x1 = q r_c and x2 = q r_o from the special-function
        // unit (absolute error about 1e-6 over these arguments). The
        // amplitude term c g(x) is (iq^3 c / r^3) (sin x - x cos x) for
        // x >= 1.5 and c h(x^2) below, h the series of g to x^8 (truncation
        // 4e-7 relative at 1.5), where the closed form's cancellation would
        // exceed 2e-6 relative.
        (void)shell;
        const float iq3 = iq * iq * iq;
        const float gs[5] = {3.333333333e-01f, -3.333333333e-02f, 1.190476190e-03f, -2.204585538e-05f,
                             2.505210839e-07f};
#pragma unroll 8
        for (int i = 0; i < np; ++i) {
            const float4 pa = *reinterpret_cast<const float4*>(poly + 8 * i);       // r_c^2, r_o^2, c_1, c_2
            const float4 pb = *reinterpret_cast<const float4*>(poly + 8 * i + 4);   // c_1/r_c^3, c_2/r_o^3, r_c, r_o
            const float x1 = q * pb.z, x2 = q * pb.w;
            float s1, c1, s2, c2;
            __sincosf(x1, &s1, &c1);
            __sincosf(x2, &s2, &c2);
            const float A1 = fmaf(-x1, c1, s1), A2 = fmaf(-x2, c2, s2);
            const float h1 = sas_horner(gs, x1 * x1), h2 = sas_horner(gs, x2 * x2);
            // select (coefficient, value) pairs, then one FMA combines them
            const bool s1b = x1 < 1.5f, s2b = x2 < 1.5f;
            const float k1 = s1b ? pa.z : iq3 * pb.x, v1 = s1b ? h1 : A1;
            const float k2 = s2b ? pa.w : iq3 * pb.y, v2 = s2b ? h2 : A2;
            const float F = fmaf(k1, v1, k2 * v2);
            acc = fmaf(F, F, acc);
        }
    } else {
#pragma unroll 4
        for (int i = 0; i < np; ++i) {
            const T* p = poly + 8 * i;
            const T x1 = q * p[6], x2 = q * p[7];
            const T g1 = M<T>::sphere_g(x1, M<T>::rcp(x1));
            const T g2 = M<T>::sphere_g(x2, M<T>::rcp(x2));
            const T F = fma(p[2], g1, p[3] * g2);
            acc = fma(F, F, acc);
        }
    }
    return acc;
}

// ---------------------------------------------- |Q|-ordered warps (FP32)
// When the histories of a warp carry nearby |Q| (the trace kernel orders a
// CTA's histories by |Q|^2 first), most nodes of the radius table fall on one
// side of the series/closed-form switch x = 1.5 for every lane. With the
// nodes in ascending radius, the warp's smallest and largest |Q| cut the
// table into three runs:
//   [0, iA)   series for every lane (largest Q times the outer radius < 1.5),
//   [iA, iC)  the per-lane selection of the plain loops,
//   [iC, np)  closed form for every lane (smallest Q times the radius >= 1.5),
// and each run does only its own branch's work. Every lane takes the same
// branch per node as the plain loops; only the closed-form run accumulates
// its terms before the common factor iq^3 (resp. iq^6) is applied once,
// which is safe there because q >= 1.5 / r_max.
struct NodeSplit {
    int iA, iC;
};

// qlo, qhi: the warp's extreme |Q|; radius columns ri (inner) and ro (outer)
// of a table with SAS_POLY_STRIDE floats per node
__device__ __forceinline__ NodeSplit node_split(const float* __restrict__ poly, int np, int ri, int ro,
                                                float qlo, float qhi)
{
    const int lane = threadIdx.x & 31;
    int nA = 0, nC = 0;
    for (int c0 = 0; c0 < np; c0 += 32) {
        const int i = c0 + lane;
        bool a = false, c = false;
        if (i < np) {
            a = qhi * poly[SAS_POLY_STRIDE * i + ro] < 1.5f;
            c = qlo * poly[SAS_POLY_STRIDE * i + ri] >= 1.5f;
        }
        nA += __popc(__ballot_sync(0xffffffffu, a));
        nC += __popc(__ballot_sync(0xffffffffu, c));
    }
    return NodeSplit{nA, np - nC};
}

// The runs for NV histories per lane at once (NV independent chains per
// node, one shared-memory load of the node for all of them); q, q2 = q^2,
// iq = 1/q per history, out[v] = <|F|^2> of history v.
template <int NV>
__device__ __forceinline__ void avg_core_shell_split(const float (&q)[NV], const float (&q2)[NV], const float (&iq)[NV],
                                                     const float* __restrict__ poly, int np, float shell, NodeSplit sp,
                                                     float (&out)[NV])
{
    const float gs[5] = {3.333333333e-01f, -3.333333333e-02f, 1.190476190e-03f, -2.204585538e-05f,
                         2.505210839e-07f};
    float acc[NV], accC[NV], iq3[NV], St[NV], Ct[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        acc[v] = 0.f;
        accC[v] = 0.f;
        iq3[v] = iq[v] * iq[v] * iq[v];
    }
#pragma unroll 2
    for (int i = 0; i < sp.iA; ++i) {   // series for both radii, in x^2 = q^2 r^2
        const float4 pa = *reinterpret_cast<const float4*>(poly + 8 * i);   // r_c^2, r_o^2, c_1, c_2
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float F = fmaf(pa.z, sas_horner(gs, q2[v] * pa.x), pa.w * sas_horner(gs, q2[v] * pa.y));
            acc[v] = fmaf(F, F, acc[v]);
        }
    }
    for (int i = sp.iA; i < sp.iC; ++i) {   // per-lane selection
        const float4 pa = *reinterpret_cast<const float4*>(poly + 8 * i);       // r_c^2, r_o^2, c_1, c_2
        const float4 pb = *reinterpret_cast<const float4*>(poly + 8 * i + 4);   // c_1/r_c^3, c_2/r_o^3, r_c, r_o
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float x1 = q[v] * pb.z, x2 = q[v] * pb.w;
            float s1, c1, s2, c2;
            __sincosf(x1, &s1, &c1);
            __sincosf(x2, &s2, &c2);
            const bool s1b = x1 < 1.5f, s2b = x2 < 1.5f;
            const float k1 = s1b ? pa.z : iq3[v] * pb.x, v1 = s1b ? sas_horner(gs, x1 * x1) : fmaf(-x1, c1, s1);
            const float k2 = s2b ? pa.w : iq3[v] * pb.y, v2 = s2b ? sas_horner(gs, x2 * x2) : fmaf(-x2, c2, s2);
            const float F = fmaf(k1, v1, k2 * v2);
            acc[v] = fmaf(F, F, acc[v]);
        }
    }
    // Closed form for both radii. The outer radius is r_c + t at every node,
    // so sin and cos of x2 follow from those of x1 and of q t (accurate,
    // once per history) by the angle-addition identities: two special-function
    // operations per node instead of four and one shared load, which keeps
    // this run below the MIO queue's limit. With S = sin qt, C = cos qt,
    //   sin x2 - x2 cos x2 = s1 (C + x2 S) + c1 (S - x2 C),
    // so the node's amplitude k1 (s1 - x1 c1) + k2 (sin x2 - x2 cos x2) is
    //   s1 (k1 + k2 (C + x2 S)) + c1 (k2 (S - x2 C) - k1 x1).
#pragma unroll
    for (int v = 0; v < NV; ++v) sincospif(q[v] * shell * 0.318309886f, &St[v], &Ct[v]);
#pragma unroll 2
    for (int i = sp.iC; i < np; ++i) {
        const float4 pb = *reinterpret_cast<const float4*>(poly + 8 * i + 4);   // k_1, k_2, r_c, r_o
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float x1 = q[v] * pb.z, x2 = q[v] * pb.w;
            float s1, c1;
            __sincosf(x1, &s1, &c1);
            const float gam = fmaf(pb.y, fmaf(x2, St[v], Ct[v]), pb.x);
            const float del = fmaf(pb.y, fmaf(-x2, Ct[v], St[v]), -pb.x * x1);
            const float F = fmaf(s1, gam, c1 * del);
            accC[v] = fmaf(F, F, accC[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)   // iq3^2 may overflow below q = 4e-7: only with a closed-form run
        out[v] = sp.iC < np ? fmaf(iq3[v] * iq3[v], accC[v], acc[v]) : acc[v];
}

template <int NV>
__device__ __forceinline__ void avg_sphere_split(const float (&q)[NV], const float (&q2)[NV], const float (&iq)[NV],
                                                 const float* __restrict__ poly, int np, NodeSplit sp,
                                                 float (&out)[NV])
{
    const float gs[5] = {3.333333333e-01f, -3.333333333e-02f, 1.190476190e-03f, -2.204585538e-05f,
                         2.505210839e-07f};
    float acc[NV], accC[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = accC[v] = 0.f;
#pragma unroll 2
    for (int i = 0; i < sp.iA; ++i) {
        const float2 p = *reinterpret_cast<const float2*>(poly + 8 * i + 2);   // c, r^2
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float g = sas_horner(gs, q2[v] * p.y);
            acc[v] = fmaf(p.x, g * g, acc[v]);
        }
    }
    for (int i = sp.iA; i < sp.iC; ++i) {
        const float* p = poly + 8 * i;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float g = M<float>::sphere_g(q[v] * p[0], iq[v] * p[4]);
            acc[v] = fmaf(p[2], g * g, acc[v]);
        }
    }
#pragma unroll 2
    for (int i = sp.iC; i < np; ++i) {
        const float2 p = *reinterpret_cast<const float2*>(poly + 8 * i);   // r, c / r^6
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float x = q[v] * p.x;
            float s, c;
            __sincosf(x, &s, &c);
            const float A = fmaf(-x, c, s);
            accC[v] = fmaf(p.y, A * A, accC[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float iq3 = iq[v] * iq[v] * iq[v];
        out[v] = sp.iC < np ? fmaf(iq3 * iq3, accC[v], acc[v]) : acc[v];
    }
}

// dSigma/dOmega at |Q|^2 = q2[v] for the NV histories of a lane of a
// |Q|-ordered warp (sphere and core-shell sphere, quadrature averages);
// inactive histories (q2 < 0) give 0. Every lane of the warp calls it.
template <int KIND, int NV>
__device__ __forceinline__ void dsigma_sorted(const float (&q2)[NV], const ModelConst<float>& mc,
                                              const float* __restrict__ poly, float (&out)[NV])
{
    unsigned lo = 0x7F800000u, hi = 0u;
    float q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        q[v] = q2[v] >= 0.f ? M<float>::sqrt_(q2[v]) : 0.f;
        if (q2[v] >= 0.f) {
            lo = min(lo, __float_as_uint(q[v]));
            hi = max(hi, __float_as_uint(q[v]));
        }
    }
    const float qlo = __uint_as_float(__reduce_min_sync(0xffffffffu, lo));
    const float qhi = __uint_as_float(__reduce_max_sync(0xffffffffu, hi));
    if (qlo == __uint_as_float(0x7F800000u)) {   // no live history in the warp
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = 0.f;
        return;
    }
    float qe[NV], qe2[NV], iq[NV], avg[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const bool on = q2[v] >= 0.f;
        qe[v] = on ? q[v] : qhi;
        qe2[v] = on ? q2[v] : qhi * qhi;
        iq[v] = M<float>::rcp(qe[v]);
    }
    if constexpr (KIND == SAS_CORE_SHELL) {
        avg_core_shell_split<NV>(qe, qe2, iq, poly, mc.n_poly, mc.shell, node_split(poly, mc.n_poly, 6, 7, qlo, qhi),
                                 avg);
    } else {
        avg_sphere_split<NV>(qe, qe2, iq, poly, mc.n_poly, node_split(poly, mc.n_poly, 0, 0, qlo, qhi), avg);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
        out[v] = q2[v] >= 0.f ? mc.scale * avg[v] * structure_factor<float>(qe[v], mc) : 0.f;
    if constexpr (KIND == SAS_SPHERE) {   // fuzzy sphere: the Gaussian interface
        if (mc.fuzz2 > 0.f) {
#pragma unroll
            for (int v = 0; v < NV; ++v) out[v] *= exp2f(-qe2[v] * mc.fuzz2);
        }
    }
}

// Kahan-compensated accumulation of the orientation sum.
template <typename T>
struct Kahan {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T v)
    {
        const T y = v - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Number of the ascending radius nodes whose r^2 qm stays <= smax (binary
// search on value `col` of each poly row, the first by default).
__device__ __forceinline__ int cyl_tier_end(const float* __restrict__ poly, int lo, int np, float qm, float smax,
                                            int col = 0)
{
    int hi = np;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (poly[8 * mid + col] * qm <= smax) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Orientation and polydispersity average of the cylinder. FP32: 2 J1(x)/x
// from s = x^2 = |Q x c|^2 r^2 without a square root per term, by the
// cheapest polynomial form valid for the node's tier; the modulus-phase form
// beyond x = 12 (tails of broad size distributions). FP64: CUDA's j1.
template <typename T>
__device__ __forceinline__ T avg_cylinder(const T qv[3], const T* __restrict__ poly, int np,
                                          const T* __restrict__ orient, int no, T half_len)
{
    Kahan<T> k;
    if constexpr (sizeof(T) == sizeof(float)) {
        // FP32: 2 J1(x)/x in the cheapest form valid for x = |Q x c| r. Since
        // |Q x c|^2 <= |Q|^2 for every axis c, the nodes (sorted by radius)
        // are split once per history, uniformly over the warp's lanes, by
        // the largest |Q|^2 of the warp: x <= 4, 6, 8, 12 and beyond.
        const float q2 = fma(qv[0], qv[0], fma(qv[1], qv[1], qv[2] * qv[2]));
        const float qm = __uint_as_float(__reduce_max_sync(__activemask(), __float_as_uint(q2)));
        const int t4 = cyl_tier_end(poly, 0, np, qm, SAS_J1R_SMAX);
        const int t6 = cyl_tier_end(poly, t4, np, qm, SAS_J1V_SMAX);
        const int t8 = cyl_tier_end(poly, t6, np, qm, SAS_J1P_SMAX);
        const int t12 = cyl_tier_end(poly, t8, np, qm, SAS_J1Q_SMAX);
        for (int o = 0; o < no; ++o) {
            const T* c = orient + 4 * o;
            const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
            const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
            const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
            const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
            const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
            const T y = fabs(qc) * half_len;
            const T sn = M<T>::sinc(y, M<T>::rcp(y));
            float inner = 0.f;
#pragma unroll 8
            for (int i = 0; i < t4; ++i) {
                const float2 rc = *reinterpret_cast<const float2*>(poly + 8 * i);   // (r^2, c)
                const float a = sas_cyl_a_r(qab2 * rc.x);
                inner = fma(rc.y, a * a, inner);
            }
#pragma unroll 8
            for (int i = t4; i < t6; ++i) {
                const float2 rc = *reinterpret_cast<const float2*>(poly + 8 * i);
                const float a = sas_cyl_a_v(qab2 * rc.x);
                inner = fma(rc.y, a * a, inner);
            }
#pragma unroll 4
            for (int i = t6; i < t8; ++i) {
                const float2 rc = *reinterpret_cast<const float2*>(poly + 8 * i);
                const float a = sas_cyl_a_s(qab2 * rc.x);
                inner = fma(rc.y, a * a, inner);
            }
#pragma unroll 4
            for (int i = t8; i < t12; ++i) {
                const float2 rc = *reinterpret_cast<const float2*>(poly + 8 * i);
                const float a = sas_cyl_a_s3(qab2 * rc.x);
                inner = fma(rc.y, a * a, inner);
            }
            if (t12 < np) {
                const float qab = M<T>::sqrt_(qab2);
                for (int i = t12; i < np; ++i) {
                    const T* p = poly + 8 * i;
                    const float sx = qab2 * p[0];
                    float a;
                    if (sx <= SAS_J1Q_SMAX) {
                        a = sas_cyl_a_s3(sx);
                    } else {
                        const float x = qab * p[2];
                        a = sas_cyl_a_large(x, __frcp_rn(x), rsqrtf(x));
                    }
                    inner = fma(p[1], a * a, inner);
                }
            }
            k.add(c[3] * sn * sn * inner);
        }
    } else {
        for (int o = 0; o < no; ++o) {
            const T* c = orient + 4 * o;
            const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
            const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
            const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
            const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
            const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
            const T y = fabs(qc) * half_len;
            const T sn = M<T>::sinc(y, M<T>::rcp(y));
            const T qab = M<T>::sqrt_(qab2);
            const T iq = M<T>::rcp(qab);
            T inner = 0;
#pragma unroll 4
            for (int i = 0; i < np; ++i) {
                const T* p = poly + 8 * i;
                const T a = M<T>::cyl_a(qab * p[2], iq * p[3], 0);
                inner = fma(p[1], a * a, inner);
            }
            k.add(c[3] * sn * sn * inner);
        }
    }
    return k.s;
}

// Cylinder with a radial table: the polydisperse radial sum of an
// orientation node is tab_c0 G(q_AB rbar), G by cubic Hermite interpolation
// of (G, h G') at the grid points; beyond the table, the direct sum over the
// radius nodes.
template <typename T>
__device__ __forceinline__ T avg_cylinder_tab(const T qv[3], const T* __restrict__ poly, const ModelConst<T>& mc,
                                              const T* __restrict__ orient, int no)
{
    const T* __restrict__ tab = poly + SAS_POLY_STRIDE * mc.n_rad;
    Kahan<T> k;
    constexpr int kUnroll = sizeof(T) == sizeof(float) ? 4 : 1;   // FP32: four orientation nodes in flight
#pragma unroll kUnroll
    for (int o = 0; o < no; ++o) {
        const T* c = orient + 4 * o;
        const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
        const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
        const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
        const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
        const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
        const T y = fabs(qc) * mc.half_length;
        const T sn = M<T>::sinc(y, M<T>::rcp(y));
        const T qab = M<T>::sqrt_(qab2);
        const T x = qab * mc.tab_rbar;
        T inner = 0;
        if (x < mc.tab_xmax) {
            const T s = x * mc.tab_inv_h;
            int i;
            T fi;
            if constexpr (sizeof(T) == sizeof(float)) {   // floor without conversion instructions (s < 2^23)
                const float tz = __fadd_rz(s, 8388608.0f);
                i = min(__float_as_int(tz) - 0x4B000000, mc.n_tab - 2);
                fi = small_uint_to_float((uint32_t)i);
            } else {
                i = min((int)s, mc.n_tab - 2);
                fi = (T)i;
            }
            const T f = s - fi, f1 = (T)1 - f;
            const T g0 = tab[2 * i], d0 = tab[2 * i + 1], g1 = tab[2 * i + 2], d1 = tab[2 * i + 3];
            // h00 = (1 + 2f)(1 - f)^2, h10 = f (1 - f)^2, h01 = f^2 (3 - 2f), h11 = f^2 (f - 1)
            inner = mc.tab_c0 * (f1 * f1 * fma((T)2 * f + (T)1, g0, f * d0) + f * f * fma((T)3 - (T)2 * f, g1, -f1 * d1));
        } else {
            for (int j = 0; j < mc.n_rad; ++j) {
                const T* p = poly + SAS_POLY_STRIDE * j;
                const T xr = qab * p[2];
                T a;
                if constexpr (sizeof(T) == 4) {
                    const float sx = xr * xr;
                    if (sx <= SAS_J1P_SMAX) a = sas_cyl_a_s(sx);
                    else if (sx <= SAS_J1Q_SMAX) a = sas_cyl_a_s3(sx);
                    else a = sas_cyl_a_large(xr, __frcp_rn(xr), rsqrtf(xr));
                } else {
                    a = M<T>::cyl_a(xr, M<T>::rcp(xr), (T)0);
                }
                inner = fma(p[1], a * a, inner);
            }
        }
        k.add(c[3] * sn * sn * inner);
    }
    return k.s;
}

// 2 J1(x)/x from s = x^2 in the form of tier TIER: x <= 4, 6, 8, 12, and
// any x (the modulus-phase form beyond 12, chosen per term).
template <int TIER>
__device__ __forceinline__ float cyl_a_tier(float sx)
{
    if constexpr (TIER == 0) return sas_cyl_a_r(sx);
    else if constexpr (TIER == 1) return sas_cyl_a_v(sx);
    else if constexpr (TIER == 2) return sas_cyl_a_s(sx);
    else if constexpr (TIER == 3) return sas_cyl_a_s3(sx);
    else {
        if (sx <= SAS_J1Q_SMAX) return sas_cyl_a_s3(sx);
        const float x = sqrtf(sx);
        return sas_cyl_a_large(x, __frcp_rn(x), rsqrtf(x));
    }
}

// FP32 amplitude of one capped-cylinder or barbell node over its slices:
//   body a(u r^2) + sum_j c_j cos(w z_j) a(u rho_j^2),
// u = (s |Q x c|)^2, w = s Q_C; cos from the special-function unit.
template <int TIER>
__device__ __forceinline__ float capped_amp(float body, float u, float w, const float* __restrict__ cap, int nc,
                                            float r2)
{
    float f = body * cyl_a_tier<TIER>(u * r2);
#pragma unroll 4
    for (int j = 0; j < nc; ++j) {
        const float4 c = *reinterpret_cast<const float4*>(cap + 4 * j);   // z, rho^2, c, 0
        f = fmaf(c.z * __cosf(w * c.x), cyl_a_tier<TIER>(u * c.y), f);
    }
    return f;
}

// Capped cylinder and barbell (Eq. 1 over disk slices normal to the axis):
// per orientation node and polydisperse scale s (poly node {s, coefficient,
// s^2}), F / (drho s^3) = pi r^2 L sinc(s Q_C L / 2) a(s Q_AB r)
//   + sum_j c_j cos(s Q_C z_j) a(s Q_AB rho_j), a(x) = 2 J1(x)/x, the cap
// slices {z_j, rho_j^2, c_j} behind the nodes. FP32: the 2 J1(x)/x form is
// chosen per node, uniformly over the warp, from the warp's largest |Q|^2
// times s^2 times the largest slice radius squared.
template <typename T>
__device__ __forceinline__ T avg_capped(const T qv[3], const T* __restrict__ poly, int np,
                                        const T* __restrict__ orient, int no, const ModelConst<T>& mc)
{
    const T* __restrict__ cap = poly + SAS_POLY_STRIDE * np;
    const int nc = mc.n_cap;
    Kahan<T> k;
    float qm = 0.f;
    if constexpr (sizeof(T) == sizeof(float)) {
        const float q2 = fma(qv[0], qv[0], fma(qv[1], qv[1], qv[2] * qv[2]));
        qm = __uint_as_float(__reduce_max_sync(__activemask(), __float_as_uint(q2))) * mc.cap_rho2max;
    }
    for (int o = 0; o < no; ++o) {
        const T* c = orient + 4 * o;
        const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
        const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
        const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
        const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
        const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
        T inner = 0;
        for (int i = 0; i < np; ++i) {
            const T* p = poly + SAS_POLY_STRIDE * i;
            const T w = p[0] * qc;
            const T y = fabs(w) * mc.half_length;
            const T body = mc.cap_body * M<T>::sinc(y, M<T>::rcp(y));
            T F;
            if constexpr (sizeof(T) == sizeof(float)) {
                const float u = qab2 * p[2];
                const float bound = qm * p[2];   // warp-uniform
                if (bound <= SAS_J1R_SMAX) F = capped_amp<0>(body, u, w, cap, nc, mc.cap_r2);
                else if (bound <= SAS_J1V_SMAX) F = capped_amp<1>(body, u, w, cap, nc, mc.cap_r2);
                else if (bound <= SAS_J1P_SMAX) F = capped_amp<2>(body, u, w, cap, nc, mc.cap_r2);
                else if (bound <= SAS_J1Q_SMAX) F = capped_amp<3>(body, u, w, cap, nc, mc.cap_r2);
                else F = capped_amp<4>(body, u, w, cap, nc, mc.cap_r2);
            } else {
                const T qs = M<T>::sqrt_(qab2) * p[0];
                T x = qs * M<T>::sqrt_(mc.cap_r2);
                F = body * M<T>::cyl_a(x, M<T>::rcp(x), (T)0);
                for (int j = 0; j < nc; ++j) {
                    const T* cj = cap + 4 * j;
                    x = qs * M<T>::sqrt_(cj[1]);
                    F = fma(cj[2] * cos(w * cj[0]), M<T>::cyl_a(x, M<T>::rcp(x), (T)0), F);
                }
            }
            inner = fma(p[1], F * F, inner);
        }
        k.add(c[3] * inner);
    }
    return k.s;
}

// FP32 amplitude of one node of the shelled cylinders: the two nested
// cylinders' terms k1 a(Q_AB r) + k2 a(Q_AB r_o), 2 J1(x)/x in the form of
// tier TIER for both.
template <int TIER>
__device__ __forceinline__ float cs_cyl_amp(float k1, float k2, float qab2, float r2, float ro2)
{
    return fmaf(k1, cyl_a_tier<TIER>(qab2 * r2), k2 * cyl_a_tier<TIER>(qab2 * ro2));
}

// F of one shelled-cylinder radius node {r^2, r_o^2, c_1, c_2 | c_3, c_4, r, r_o}
// in the 2 J1(x)/x form of tier TIER, s1 and s2 the node's two sincs.
template <int TIER>
__device__ __forceinline__ float cs_cyl_node(const float* __restrict__ poly, int i, float s1, float s2, float qab2)
{
    const float4 p = *reinterpret_cast<const float4*>(poly + SAS_POLY_STRIDE * i);      // r^2, r_o^2, c_1, c_2
    const float2 pc = *reinterpret_cast<const float2*>(poly + SAS_POLY_STRIDE * i + 4); // c_3, c_4
    const float k1 = fmaf(s1, p.z, s2 * p.w), k2 = fmaf(s1, pc.x, s2 * pc.y);
    return cs_cyl_amp<TIER>(k1, k2, qab2, p.x, p.y);
}

// Core-shell and hollow cylinders, core-shell bicelle (Eq. 1 region by
// region, four nested cylinders): per orientation node and radius node
// {r^2, r_o^2, c_1, c_2, c_3, c_4, r, r_o},
//   F = (c_1 s_L + c_2 s_Lo) a(Q_AB r) + (c_3 s_L + c_4 s_Lo) a(Q_AB r_o),
// s_H = sinc(Q_C H/2), L_o = L + 2 t_f. FP32: the 2 J1(x)/x form of a node
// is chosen uniformly over the warp from the warp's largest |Q|^2 times
// r_o^2. RUNS: the radius nodes ascend, so the forms split them into
// consecutive runs found once per history, each run a loop of its own form;
// otherwise (the batch kernel, whose registers are shared by every kind)
// the form is chosen node by node.
template <typename T, bool RUNS = true>
__device__ __forceinline__ T avg_cs_cylinder(const T qv[3], const T* __restrict__ poly, int np,
                                             const T* __restrict__ orient, int no, const ModelConst<T>& mc)
{
    Kahan<T> k;
    if constexpr (sizeof(T) == sizeof(float) && !RUNS) {
        const float q2 = fma(qv[0], qv[0], fma(qv[1], qv[1], qv[2] * qv[2]));
        const float qm = __uint_as_float(__reduce_max_sync(__activemask(), __float_as_uint(q2)));
        for (int o = 0; o < no; ++o) {
            const T* c = orient + 4 * o;
            const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
            const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
            const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
            const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
            const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
            const T y1 = fabs(qc) * mc.half_length, y2 = fabs(qc) * mc.half_length_o;
            const T s1 = M<T>::sinc(y1, M<T>::rcp(y1)), s2 = M<T>::sinc(y2, M<T>::rcp(y2));
            float inner = 0.f;
            for (int i = 0; i < np; ++i) {
                const float bound = qm * poly[SAS_POLY_STRIDE * i + 1];   // warp-uniform
                float F;
                if (bound <= SAS_J1R_SMAX) F = cs_cyl_node<0>(poly, i, s1, s2, qab2);
                else if (bound <= SAS_J1V_SMAX) F = cs_cyl_node<1>(poly, i, s1, s2, qab2);
                else if (bound <= SAS_J1P_SMAX) F = cs_cyl_node<2>(poly, i, s1, s2, qab2);
                else if (bound <= SAS_J1Q_SMAX) F = cs_cyl_node<3>(poly, i, s1, s2, qab2);
                else F = cs_cyl_node<4>(poly, i, s1, s2, qab2);
                inner = fmaf(F, F, inner);
            }
            k.add(c[3] * inner);
        }
        return k.s;
    } else if constexpr (sizeof(T) == sizeof(float)) {
        const float q2 = fma(qv[0], qv[0], fma(qv[1], qv[1], qv[2] * qv[2]));
        const float qm = __uint_as_float(__reduce_max_sync(__activemask(), __float_as_uint(q2)));
        const int t4 = cyl_tier_end(poly, 0, np, qm, SAS_J1R_SMAX, 1);
        const int t6 = cyl_tier_end(poly, t4, np, qm, SAS_J1V_SMAX, 1);
        const int t8 = cyl_tier_end(poly, t6, np, qm, SAS_J1P_SMAX, 1);
        const int t12 = cyl_tier_end(poly, t8, np, qm, SAS_J1Q_SMAX, 1);
        for (int o = 0; o < no; ++o) {
            const T* c = orient + 4 * o;
            const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
            const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
            const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
            const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
            const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
            const T y1 = fabs(qc) * mc.half_length, y2 = fabs(qc) * mc.half_length_o;
            const T s1 = M<T>::sinc(y1, M<T>::rcp(y1)), s2 = M<T>::sinc(y2, M<T>::rcp(y2));
            float inner = 0.f;
#pragma unroll 4
            for (int i = 0; i < t4; ++i) {
                const float F = cs_cyl_node<0>(poly, i, s1, s2, qab2);
                inner = fmaf(F, F, inner);
            }
#pragma unroll 4
            for (int i = t4; i < t6; ++i) {
                const float F = cs_cyl_node<1>(poly, i, s1, s2, qab2);
                inner = fmaf(F, F, inner);
            }
#pragma unroll 2
            for (int i = t6; i < t8; ++i) {
                const float F = cs_cyl_node<2>(poly, i, s1, s2, qab2);
                inner = fmaf(F, F, inner);
            }
#pragma unroll 2
            for (int i = t8; i < t12; ++i) {
                const float F = cs_cyl_node<3>(poly, i, s1, s2, qab2);
                inner = fmaf(F, F, inner);
            }
            for (int i = t12; i < np; ++i) {
                const float F = cs_cyl_node<4>(poly, i, s1, s2, qab2);
                inner = fmaf(F, F, inner);
            }
            k.add(c[3] * inner);
        }
        return k.s;
    } else {
        for (int o = 0; o < no; ++o) {
            const T* c = orient + 4 * o;
            const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
            const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
            const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
            const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
            const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
            const T y1 = fabs(qc) * mc.half_length, y2 = fabs(qc) * mc.half_length_o;
            const T s1 = M<T>::sinc(y1, M<T>::rcp(y1)), s2 = M<T>::sinc(y2, M<T>::rcp(y2));
            T inner = 0;
            const T qab = M<T>::sqrt_(qab2), iq = M<T>::rcp(qab);
            for (int i = 0; i < np; ++i) {
                const T* p = poly + SAS_POLY_STRIDE * i;
                const T xa = qab * p[6], xb = qab * p[7];
                const T F = fma(s1, p[2], s2 * p[3]) * M<T>::cyl_a(xa, iq / p[6], 0) +
                            fma(s1, p[4], s2 * p[5]) * M<T>::cyl_a(xb, iq / p[7], 0);
                inner = fma(F, F, inner);
            }
            k.add(c[3] * inner);
        }
        return k.s;
    }
}

// Core-shell ellipsoid of revolution: per orientation node and radius node
// {r_e^2, r_o^2, 3 c_1, 3 c_2}, F = 3 c_1 g(x_c) + 3 c_2 g(x_o) with
// x^2 = r^2 Q_AB^2 + r_p^2 Q_C^2 for the core and the outer surface.
template <typename T>
__device__ __forceinline__ T avg_cs_ellipsoid(const T qv[3], const T* __restrict__ poly, int np,
                                              const T* __restrict__ orient, int no, const ModelConst<T>& mc)
{
    Kahan<T> k;
    for (int o = 0; o < no; ++o) {
        const T* c = orient + 4 * o;
        const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
        const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
        const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
        const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
        const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
        const T qc2 = qc * qc;
        const T pc = mc.rp2 * qc2, po = mc.rp2o * qc2;
        T inner = 0;
        for (int i = 0; i < np; ++i) {
            const T* p = poly + SAS_POLY_STRIDE * i;
            // floored so that Q = 0 gives x = 0 (the series branch), not 0 * inf
            const T xc2 = fmax(fma(p[0], qab2, pc), (T)1e-30), xo2 = fmax(fma(p[1], qab2, po), (T)1e-30);
            const T ic = M<T>::rsqrt(xc2), io = M<T>::rsqrt(xo2);
            const T F = p[2] * M<T>::sphere_g(xc2 * ic, ic) + p[3] * M<T>::sphere_g(xo2 * io, io);
            inner = fma(F, F, inner);
        }
        k.add(c[3] * inner);
    }
    return k.s;
}

// Particles without a symmetry axis (Eq. 1 for the body): per frame
// (rows A, B, C of the orientation table, weight in row A) and polydisperse
// scale s_i (poly node: s_i, coefficient):
//   triaxial ellipsoid  F = drho V(s) 3 g(s |(a Q_A, b Q_B, c Q_C)|)
//   parallelepiped      F = drho V(s) sinc(s a Q_A) sinc(s b Q_B) sinc(s c Q_C)
template <typename T, int KIND>
__device__ __forceinline__ T avg_axes3(const T qv[3], const T* __restrict__ poly, int np,
                                       const T* __restrict__ orient, int nrows, const ModelConst<T>& mc)
{
    Kahan<T> k;
    for (int o = 0; o + 2 < nrows; o += 3) {
        const T* A = orient + 4 * o;
        const T* B = A + 4;
        const T* C = A + 8;
        const T pa = fma(qv[0], A[0], fma(qv[1], A[1], qv[2] * A[2]));
        const T pb = fma(qv[0], B[0], fma(qv[1], B[1], qv[2] * B[2]));
        const T pc = fma(qv[0], C[0], fma(qv[1], C[1], qv[2] * C[2]));
        const T qa = mc.ax_a * pa, qb = mc.ax_b * pb, qc = mc.ax_c * pc;
        T inner = 0;
        if constexpr (KIND == SAS_ELLIPTICAL_CYLINDER) {
            const T xab2 = fma(qa, qa, qb * qb), yc0 = fabs(qc);
            for (int i = 0; i < np; ++i) {
                const T sc = poly[SAS_POLY_STRIDE * i];
                const T y = sc * yc0;
                T a;
                if constexpr (sizeof(T) == sizeof(float)) {
                    a = cyl_a_tier<4>(sc * sc * xab2);
                } else {
                    const T x = sc * M<T>::sqrt_(xab2);
                    a = M<T>::cyl_a(x, M<T>::rcp(x), (T)0);
                }
                const T amp = M<T>::sinc(y, M<T>::rcp(y)) * a;
                inner = fma(poly[SAS_POLY_STRIDE * i + 1], amp * amp, inner);
            }
        } else if constexpr (KIND == SAS_HOLLOW_RECTANGULAR_PRISM) {
            const T ya0 = fabs(qa), yb0 = fabs(qb), yc0 = fabs(qc);
            const T za0 = fabs(mc.ax_ai * pa), zb0 = fabs(mc.ax_bi * pb), zc0 = fabs(mc.ax_ci * pc);
            for (int i = 0; i < np; ++i) {
                const T sc = poly[SAS_POLY_STRIDE * i];
                const T ya = sc * ya0, yb = sc * yb0, yc = sc * yc0;
                const T za = sc * za0, zb = sc * zb0, zc = sc * zc0;
                const T outer = M<T>::sinc(ya, M<T>::rcp(ya)) * M<T>::sinc(yb, M<T>::rcp(yb)) *
                                M<T>::sinc(yc, M<T>::rcp(yc));
                const T hole = M<T>::sinc(za, M<T>::rcp(za)) * M<T>::sinc(zb, M<T>::rcp(zb)) *
                               M<T>::sinc(zc, M<T>::rcp(zc));
                const T amp = fma(mc.ax_v, outer, -mc.ax_vi * hole);
                inner = fma(poly[SAS_POLY_STRIDE * i + 1], amp * amp, inner);
            }
        } else if (KIND == SAS_TRIAXIAL_ELLIPSOID) {
            const T x0 = M<T>::sqrt_(fma(qa, qa, fma(qb, qb, qc * qc)));
            for (int i = 0; i < np; ++i) {
                const T x = poly[SAS_POLY_STRIDE * i] * x0;
                const T g = M<T>::sphere_g(x, M<T>::rcp(x));
                inner = fma(poly[SAS_POLY_STRIDE * i + 1], g * g, inner);
            }
        } else {
            const T ya0 = fabs(qa), yb0 = fabs(qb), yc0 = fabs(qc);
            for (int i = 0; i < np; ++i) {
                const T sc = poly[SAS_POLY_STRIDE * i];
                const T ya = sc * ya0, yb = sc * yb0, yc = sc * yc0;
                const T amp = M<T>::sinc(ya, M<T>::rcp(ya)) * M<T>::sinc(yb, M<T>::rcp(yb)) *
                              M<T>::sinc(yc, M<T>::rcp(yc));
                inner = fma(poly[SAS_POLY_STRIDE * i + 1], amp * amp, inner);
            }
        }
        k.add(A[3] * inner);
    }
    return k.s;
}

template <typename T>
__device__ __forceinline__ T avg_ellipsoid(const T qv[3], const T* __restrict__ poly, int np,
                                           const T* __restrict__ orient, int no, T rp2)
{
    Kahan<T> k;
    for (int o = 0; o < no; ++o) {
        const T* c = orient + 4 * o;
        const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
        const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
        const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
        const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
        const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
        const T pol = rp2 * qc * qc;
        T inner = 0;
#pragma unroll 4
        for (int i = 0; i < np; ++i) {
            const T* p = poly + 8 * i;
            const T x2e = fma(p[0], qab2, pol);
            const T inv = M<T>::rsqrt(x2e);
            const T g = M<T>::sphere_g(x2e * inv, inv);
            inner = fma(p[1], g * g, inner);
        }
        k.add(c[3] * inner);
    }
    return k.s;
}

// Shape-independent laws f(|Q|) (parameters prepared on the host in f_a,
// f_b, f_c): CUDA's accurate exp, expm1 and pow, one call per history. The
// Gaussian coil takes its series sum_k 2 (-u)^k / (k + 2)! below u = 1
// (FP32; 0.1 in FP64), where 2 (exp(-u) - 1 + u) / u^2 cancels.
// Debye's function of a Gaussian coil, D(u) = 2 (exp(-u) - 1 + u) / u^2:
// its series below u = 1 (FP32; 0.1 in FP64), where the closed form cancels.
template <typename T>
__device__ __forceinline__ T debye_fn(T u)
{
    constexpr bool fp32 = sizeof(T) == sizeof(float);
    if (u < (fp32 ? (T)1 : (T)0.1)) {
        constexpr int nt = fp32 ? 10 : 12;
        T sum = 0, c = (T)2;   // c = 2 / (k + 2)!, from k = 0
        T term[nt];
#pragma unroll
        for (int k = 0; k < nt; ++k) {
            c = k == 0 ? (T)1 : c / (T)(k + 2);
            term[k] = c;
        }
#pragma unroll
        for (int k = nt - 1; k >= 0; --k) sum = fma(sum, -u, term[k]);
        return sum;
    }
    return (T)2 * (expm1(-u) + u) / (u * u);
}

// y - log(1 + y) for y >= 0 without cancellation: its series below 0.3
// (FP32; 1e-3 in FP64), the direct difference above.
template <typename T>
__device__ __forceinline__ T y_minus_log1p(T y)
{
    constexpr bool fp32 = sizeof(T) == sizeof(float);
    if (y < (fp32 ? (T)0.3 : (T)1e-3)) {
        constexpr int nt = fp32 ? 12 : 4;   // y^2 (1/2 - y/3 + y^2/4 - ...)
        T sum = 0;
#pragma unroll
        for (int k = nt - 1; k >= 0; --k) sum = fma(sum, -y, (T)1 / (T)(k + 2));
        return y * y * sum;
    }
    return y - log1p(y);
}

// Sphere factor (3 (sin x - x cos x) / x^3)^2, x = q r (1 at r = 0): the
// series to x^8 below x = 0.5 (truncation 2e-12 relative), CUDA's accurate
// sincos above (one evaluation per history, so no special-function-unit form).
template <typename T>
__device__ __forceinline__ T si_sphere_p(T q, T r)
{
    const T x = q * r;
    T g;
    if (x < (T)0.5) {
        const T t = x * x;
        g = fma(t, fma(t, fma(t, fma(t, (T)(1.0 / 3991680.0), (T)(-1.0 / 45360.0)), (T)(1.0 / 840.0)),
                       (T)(-1.0 / 30.0)), (T)(1.0 / 3.0));
    } else {
        T s, c;
        sincos(x, &s, &c);
        g = (s - x * c) / (x * x * x);
    }
    const T a = (T)3 * g;
    return a * a;
}

// Fractal factor M(y; D) = sin(e atan y) / (e y (1 + y^2)^(e/2)), e = D - 1 > 0,
// as (sin z / z)(atan y / y)(1 + y^2)^(-e/2) with z = e atan y (M(0) = 1).
template <typename T>
__device__ __forceinline__ T fractal_m(T y, T e)
{
    if (y < (T)1e-30) return (T)1;
    const T th = atan(y);
    const T z = e * th;
    return (sin(z) / z) * (th / y) * pow(fma(y, y, (T)1), (T)-0.5 * e);
}

// x^-a gamma(a, x), the scaled lower incomplete gamma function (a > 0,
// x > 0; gamma_a = Gamma(a)): the power series e^-x sum_n x^n / (a (a+1)
// ... (a+n)) below x = a + 1, above it Gamma(a) x^-a - e^-x CF with the
// continued fraction of Gamma(a, x) by Lentz's method (Abramowitz-Stegun
// 6.5.29 and 6.5.31). Both converge within 200 steps for a <= 6.
template <typename T>
__device__ __forceinline__ T scaled_lower_gamma(T a, T x, T gamma_a)
{
    constexpr bool fp32 = sizeof(T) == sizeof(float);
    const T eps = fp32 ? (T)3e-8 : (T)1e-17;
    if (x < a + (T)1) {
        T term = (T)1 / a, sum = term;
        for (int n = 1; n < 200 && term > eps * sum; ++n) {
            term *= x / (a + (T)n);
            sum += term;
        }
        return exp(-x) * sum;
    }
    const T tiny = fp32 ? (T)1e-30 : (T)1e-300;
    T b = x + (T)1 - a, f = (T)1 / b, C = (T)1 / tiny, D = (T)1 / b;
    for (int i = 1; i < 200; ++i) {
        const T an = -(T)i * ((T)i - a);
        b += (T)2;
        D = fma(an, D, b);
        if (fabs(D) < tiny) D = tiny;
        C = b + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = (T)1 / D;
        const T delta = C * D;
        f *= delta;
        if (fabs(delta - (T)1) < eps) break;
    }
    return gamma_a * pow(x, -a) - exp(-x) * f;
}

template <typename T>
__device__ __forceinline__ T shape_independent(T q2, T q, const ModelConst<T>& mc)
{
    switch (mc.function) {
    case SAS_FN_GUINIER: return exp(-q2 * mc.f_a);
    case SAS_FN_GAUSS_COIL: return debye_fn<T>(q2 * mc.f_a);
    case SAS_FN_LORENTZ: return (T)1 / fma(q2, mc.f_a, (T)1);
    case SAS_FN_DAB: {
        const T d = fma(q2, mc.f_a, (T)1);
        return (T)1 / (d * d);
    }
    case SAS_FN_POWER_LAW: return pow(q, -mc.f_a);
    case SAS_FN_GAUSS_PEAK: {
        const T d = q - mc.f_a;
        return exp(-d * d * mc.f_b);
    }
    case SAS_FN_TEUBNER_STREY: return (T)1 / fma(q2, fma(q2, mc.f_c, mc.f_b), mc.f_a);
    case SAS_FN_PEAK_LORENTZ: {   // f_a = Q0, f_b = 1 / B
        const T d = (q - mc.f_a) * mc.f_b;
        return (T)1 / fma(d, d, (T)1);
    }
    case SAS_FN_TWO_POWER_LAW:    // f_a = Qc, f_b = m1, f_c = m2, f_d = Qc^(m2 - m1)
        return q <= mc.f_a ? pow(q, -mc.f_b) : mc.f_d * pow(q, -mc.f_c);
    case SAS_FN_GUINIER_POROD:    // f_a = Rg^2 / (3 - s), f_b = s, f_c = m, f_d = Q1, f_e = D
        return q <= mc.f_d ? pow(q, -mc.f_b) * exp(-q2 * mc.f_a) : mc.f_e * pow(q, -mc.f_c);
    case SAS_FN_GAUSS_LORENTZ_GEL:   // f_a = Xi^2 / 2, f_b = xi^2, f_c = r
        return exp(-q2 * mc.f_a) + mc.f_c / fma(q2, mc.f_b, (T)1);
    case SAS_FN_POLY_GAUSS_COIL: {   // f_a = Rg^2 / (1 + 2U), f_b = U
        // with t = log(1 + U x) / U: (1 + U x)^(-1/U) - 1 + x
        //   = (exp(-t) - 1 + t) + (x - t) = t^2 D(t) / 2 + (U x - log(1 + U x)) / U,
        // two non-negative terms, so the numerator does not cancel
        const T x = q2 * mc.f_a, U = mc.f_b;
        if (x < (T)1e-30) return (T)1;
        const T y = U * x;
        const T t = U > (T)0 ? log1p(y) / U : x;
        const T h = U > (T)0 ? y_minus_log1p<T>(y) / U : (T)0;
        return (t * t * debye_fn<T>(t) + (T)2 * h) / (((T)1 + U) * x * x);
    }
    case SAS_FN_MASS_FRACTAL:     // f_a = R, f_b = D - 1, f_c = xi
        return si_sphere_p<T>(q, mc.f_a) * fractal_m<T>(q * mc.f_c, mc.f_b);
    case SAS_FN_FRACTAL:          // f_a = R0, f_b = D - 1, f_c = xi, f_d = Gamma(D + 1) (xi / R0)^D
        return si_sphere_p<T>(q, mc.f_a) * fma(mc.f_d, fractal_m<T>(q * mc.f_c, mc.f_b), (T)1);
    case SAS_FN_SPINODAL: {       // f_a = 1 / Qmax, f_b = g, f_c = g / 2, f_d = 1 + g / 2
        const T x = q * mc.f_a;
        return mc.f_d * x * x / (mc.f_c + pow(x, (T)2 + mc.f_b));
    }
    case SAS_FN_LINEAR_PEARLS: {  // f_a = R, f_b = d, f_c = N, f_d = 1 / N^2
        if (q < (T)1e-30) return (T)1;
        const int n = (int)mc.f_c;
        const T y1 = q * mc.f_b;
        T pairs = mc.f_c;
        for (int k = 1; k < n; ++k) {
            const T y = y1 * (T)k;
            pairs = fma((T)2 * (T)(n - k), sin(y) / y, pairs);
        }
        return si_sphere_p<T>(q, mc.f_a) * pairs * mc.f_d;
    }
    case SAS_FN_POLYMER_EXCL_VOLUME: {   // f_a: U = Q^2 f_a; f_b = m = 1/nu, f_c = Gamma(m/2), f_d = Gamma(m)
        const T U = q2 * mc.f_a;
        if (U < (T)1e-30) return (T)1;
        return mc.f_b * (scaled_lower_gamma<T>((T)0.5 * mc.f_b, U, mc.f_c) - scaled_lower_gamma<T>(mc.f_b, U, mc.f_d));
    }
    default: {                    // star polymer: f_a = Rg^2 f / (3f - 2), f_b = f
        const T v = q2 * mc.f_a;
        const T g = v > (T)1e-30 ? -expm1(-v) / v : (T)1;
        return (debye_fn<T>(v) + (mc.f_b - (T)1) * g * g) / mc.f_b;
    }
    }
}

// dSigma/dOmega(Q) in 1/angstrom. LEAN: the forms that need fewer
// registers, for the batch kernel (same values).
template <typename T, int KIND, bool LEAN = false>
__device__ __forceinline__ T dsigma(const T qv[3], const ModelConst<T>& mc,
                                    const T* __restrict__ poly, const T* __restrict__ orient)
{
    const T q2 = fma(qv[0], qv[0], fma(qv[1], qv[1], qv[2] * qv[2]));
    if constexpr (KIND == SAS_SHAPE_INDEPENDENT) {
        (void)poly;
        (void)orient;
        return mc.scale * shape_independent<T>(q2, ::sqrt(q2), mc);
    }
    const T q = M<T>::sqrt_(q2);
    T avg;
    if (KIND == SAS_SPHERE) {
        avg = avg_sphere<T>(q, M<T>::rcp(q), poly, mc.n_poly);
        if (mc.fuzz2 > (T)0) avg *= exp2(-q2 * mc.fuzz2);   // fuzzy sphere: the Gaussian interface
    } else if (KIND == SAS_CORE_SHELL) {
        avg = avg_core_shell<T>(q, M<T>::rcp(q), poly, mc.n_poly, mc.shell);
    } else if (KIND == SAS_CYLINDER) {
        avg = mc.n_tab > 0 ? avg_cylinder_tab<T>(qv, poly, mc, orient, mc.n_orient)
                           : avg_cylinder<T>(qv, poly, mc.n_rad, orient, mc.n_orient, mc.half_length);
    } else if (KIND == SAS_ELLIPSOID) {
        avg = avg_ellipsoid<T>(qv, poly, mc.n_poly, orient, mc.n_orient, mc.rp2);
    } else if (KIND == SAS_CAPPED_CYLINDER || KIND == SAS_BARBELL) {
        avg = avg_capped<T>(qv, poly, mc.n_rad, orient, mc.n_orient, mc);
    } else if (KIND == SAS_CORE_SHELL_CYLINDER || KIND == SAS_HOLLOW_CYLINDER || KIND == SAS_CORE_SHELL_BICELLE) {
        avg = avg_cs_cylinder<T, !LEAN>(qv, poly, mc.n_rad, orient, mc.n_orient, mc);
    } else if (KIND == SAS_CORE_SHELL_ELLIPSOID) {
        avg = avg_cs_ellipsoid<T>(qv, poly, mc.n_rad, orient, mc.n_orient, mc);
    } else {
        avg = avg_axes3<T, KIND>(qv, poly, mc.n_rad, orient, mc.n_orient, mc);
    }
    return mc.scale * avg * structure_factor<T>(q, mc);
}

// ------------------------------------------------ per-event sampling
// Philox block 2 of a history: radius, axis polar, axis azimuth, spare.
__device__ __forceinline__ uint4 event_draws(uint64_t seed, uint32_t exp_id, uint64_t index)
{
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    return philox(make_uint4(2u, exp_id, (uint32_t)index, (uint32_t)(index >> 32)), key);
}

// 1 - u01(x), exact
template <typename T>
__device__ __forceinline__ T u01c(uint32_t x)
{
    return ((T)(8388607u - (x >> 9)) + (T)0.5) * (T)(1.0 / 8388608.0);
}

// One event of the model (Sec. II.B): the radius from N(R, (pR)^2)
// restricted to R > 0, sampled by inversion z = Phi^-1(lo + u (1 - lo)),
// Phi^-1(v) = -sqrt(2) erfcinv(2 v) (upper half through 1 - v = (1 - u)(1 - lo));
// the axis uniform on the sphere or in the angles. Returns
// (phi / <V>) |F(Q; r, axis)|^2 S(Q); its expectation over the draws is the
// quadrature average over the same laws.
template <typename T, int KIND>
__device__ __forceinline__ T dsigma_event(const T qv[3], const ModelConst<T>& mc, const T* __restrict__ poly,
                                          uint4 rb)
{
    const T q2 = fma(qv[0], qv[0], fma(qv[1], qv[1], qv[2] * qv[2]));
    const T q = M<T>::sqrt_(q2);
    T r = mc.ev_r;
    if (mc.ev_p > (T)0) {
        const T u = u01<T>(rb.x);
        const T v = fma(u, mc.ev_1mlo, mc.ev_lo);
        const T z = (v < (T)0.5) ? -(T)1.41421356237309515 * M<T>::erfcinv_((T)2 * v)
                                 : (T)1.41421356237309515 * M<T>::erfcinv_((T)2 * u01c<T>(rb.x) * mc.ev_1mlo);
        r = mc.ev_r * fma(mc.ev_p, z, (T)1);
    }
    const T pi = (T)3.14159265358979323846;
    T F2;
    if constexpr (KIND == SAS_TRIAXIAL_ELLIPSOID || KIND == SAS_PARALLELEPIPED || KIND == SAS_ELLIPTICAL_CYLINDER ||
                  KIND == SAS_HOLLOW_RECTANGULAR_PRISM) {
        // frame of this event: C from (theta, phi), A and B rotated by psi
        T A[3], B[3], C[3];
        if (mc.orient_mode == 0) {
            for (int k = 0; k < 3; ++k) {
                A[k] = mc.ev_frame[k];
                B[k] = mc.ev_frame[3 + k];
                C[k] = mc.ev_axis[k];
            }
        } else {
            T ct, st, sp, cp, sq, cq;
            if (mc.orient_mode == 1) {
                ct = (T)1 - (T)2 * u01<T>(rb.y);
                st = M<T>::sqrt_(fmax((T)0, (T)1 - ct * ct));
            } else {
                M<T>::sincospi_(u01<T>(rb.y), st, ct);
            }
            M<T>::sincospi_((T)2 * u01<T>(rb.z), sp, cp);
            M<T>::sincospi_((T)2 * u01<T>(rb.w), sq, cq);
            const T et[3] = {ct * cp, ct * sp, -st}, ep[3] = {-sp, cp, (T)0};
            for (int k = 0; k < 3; ++k) {
                A[k] = cq * et[k] + sq * ep[k];
                B[k] = -sq * et[k] + cq * ep[k];
            }
            C[0] = st * cp;
            C[1] = st * sp;
            C[2] = ct;
        }
        const T sc = r / mc.ev_r;
        const T pa = sc * fma(qv[0], A[0], fma(qv[1], A[1], qv[2] * A[2]));
        const T pb = sc * fma(qv[0], B[0], fma(qv[1], B[1], qv[2] * B[2]));
        const T pc = sc * fma(qv[0], C[0], fma(qv[1], C[1], qv[2] * C[2]));
        const T qa = mc.ax_a * pa, qb = mc.ax_b * pb, qc = mc.ax_c * pc;
        const T v3 = mc.ax_a * mc.ax_b * mc.ax_c * sc * sc * sc;
        T F;
        if constexpr (KIND == SAS_ELLIPTICAL_CYLINDER) {
            // V = pi a b L = 2 pi a b c
            const T x = M<T>::sqrt_(fma(qa, qa, qb * qb)), y = fabs(qc);
            T a;
            if constexpr (sizeof(T) == sizeof(float)) a = cyl_a_tier<4>(x * x);
            else a = M<T>::cyl_a(x, M<T>::rcp(x), (T)0);
            F = mc.ev_c1 * (T)2 * pi * v3 * M<T>::sinc(y, M<T>::rcp(y)) * a;
        } else if constexpr (KIND == SAS_HOLLOW_RECTANGULAR_PRISM) {
            const T ya = fabs(qa), yb = fabs(qb), yc = fabs(qc);
            const T za = fabs(mc.ax_ai * pa), zb = fabs(mc.ax_bi * pb), zc = fabs(mc.ax_ci * pc);
            const T outer = M<T>::sinc(ya, M<T>::rcp(ya)) * M<T>::sinc(yb, M<T>::rcp(yb)) *
                            M<T>::sinc(yc, M<T>::rcp(yc));
            const T hole = M<T>::sinc(za, M<T>::rcp(za)) * M<T>::sinc(zb, M<T>::rcp(zb)) *
                           M<T>::sinc(zc, M<T>::rcp(zc));
            F = mc.ev_c1 * (T)8 * sc * sc * sc * fma(mc.ax_v, outer, -mc.ax_vi * hole);
        } else if (KIND == SAS_TRIAXIAL_ELLIPSOID) {
            const T x = M<T>::sqrt_(fma(qa, qa, fma(qb, qb, qc * qc)));
            F = (T)3 * mc.ev_c1 * (T)(4.0 / 3.0) * pi * v3 * M<T>::sphere_g(x, M<T>::rcp(x));
        } else {
            const T ya = fabs(qa), yb = fabs(qb), yc = fabs(qc);
            F = mc.ev_c1 * (T)8 * v3 * M<T>::sinc(ya, M<T>::rcp(ya)) * M<T>::sinc(yb, M<T>::rcp(yb)) *
                M<T>::sinc(yc, M<T>::rcp(yc));
        }
        F2 = F * F;
    } else if (KIND == SAS_SPHERE) {
        const T x = q * r;
        const T g = M<T>::sphere_g(x, M<T>::rcp(x));
        const T V = (T)(4.0 / 3.0) * pi * r * r * r;
        const T F = (T)3 * mc.ev_c1 * V * g;
        F2 = F * F;
        if (mc.fuzz2 > (T)0) F2 *= exp2(-q2 * mc.fuzz2);
    } else if (KIND == SAS_CORE_SHELL) {
        const T ro = r + mc.shell;
        const T xc = q * r, xo = q * ro;
        const T Vc = (T)(4.0 / 3.0) * pi * r * r * r, Vo = (T)(4.0 / 3.0) * pi * ro * ro * ro;
        const T F = (T)3 * (mc.ev_c1 * Vc * M<T>::sphere_g(xc, M<T>::rcp(xc)) +
                            mc.ev_c2 * Vo * M<T>::sphere_g(xo, M<T>::rcp(xo)));
        F2 = F * F;
    } else {
        T c[3];
        if (mc.orient_mode == 0) {
            c[0] = mc.ev_axis[0];
            c[1] = mc.ev_axis[1];
            c[2] = mc.ev_axis[2];
        } else {
            T ct, st, sp, cp;
            if (mc.orient_mode == 1) {
                ct = (T)1 - (T)2 * u01<T>(rb.y);
                st = M<T>::sqrt_(fmax((T)0, (T)1 - ct * ct));
            } else {
                M<T>::sincospi_(u01<T>(rb.y), st, ct);
            }
            M<T>::sincospi_((T)2 * u01<T>(rb.z), sp, cp);
            c[0] = st * cp;
            c[1] = st * sp;
            c[2] = ct;
        }
        const T qc = fma(qv[0], c[0], fma(qv[1], c[1], qv[2] * c[2]));
        const T x0 = fma(qv[1], c[2], -qv[2] * c[1]);
        const T x1 = fma(qv[2], c[0], -qv[0] * c[2]);
        const T x2 = fma(qv[0], c[1], -qv[1] * c[0]);
        const T qab2 = fma(x0, x0, fma(x1, x1, x2 * x2));
        if constexpr (KIND == SAS_CAPPED_CYLINDER || KIND == SAS_BARBELL) {
            // the drawn scale s = r / r_mean on every size; the cap slices sit
            // behind the single node row
            const T sc = r / mc.ev_r;
            const T w = sc * qc;
            const T y = fabs(w) * mc.half_length;
            const T body = mc.cap_body * M<T>::sinc(y, M<T>::rcp(y));
            const T* __restrict__ cap = poly + SAS_POLY_STRIDE;
            const int nc = mc.n_cap;
            T A;
            if constexpr (sizeof(T) == sizeof(float)) {
                const float s2 = sc * sc, u = qab2 * s2;
                const float bound = __uint_as_float(__reduce_max_sync(__activemask(), __float_as_uint(q2 * s2))) *
                                    mc.cap_rho2max;   // warp-uniform
                if (bound <= SAS_J1R_SMAX) A = capped_amp<0>(body, u, w, cap, nc, mc.cap_r2);
                else if (bound <= SAS_J1V_SMAX) A = capped_amp<1>(body, u, w, cap, nc, mc.cap_r2);
                else if (bound <= SAS_J1P_SMAX) A = capped_amp<2>(body, u, w, cap, nc, mc.cap_r2);
                else if (bound <= SAS_J1Q_SMAX) A = capped_amp<3>(body, u, w, cap, nc, mc.cap_r2);
                else A = capped_amp<4>(body, u, w, cap, nc, mc.cap_r2);
            } else {
                const T qs = M<T>::sqrt_(qab2) * sc;
                T x = qs * M<T>::sqrt_(mc.cap_r2);
                A = body * M<T>::cyl_a(x, M<T>::rcp(x), (T)0);
                for (int j = 0; j < nc; ++j) {
                    const T* cj = cap + 4 * j;
                    x = qs * M<T>::sqrt_(cj[1]);
                    A = fma(cj[2] * cos(w * cj[0]), M<T>::cyl_a(x, M<T>::rcp(x), (T)0), A);
                }
            }
            const T F = mc.ev_c1 * sc * sc * sc * A;
            F2 = F * F;
        } else if constexpr (KIND == SAS_CORE_SHELL_CYLINDER || KIND == SAS_HOLLOW_CYLINDER ||
                             KIND == SAS_CORE_SHELL_BICELLE) {
            // the four nested cylinders of the drawn core radius r and r + t
            const T ro = r + mc.shell;
            const T y1 = fabs(qc) * mc.half_length, y2 = fabs(qc) * mc.half_length_o;
            const T qab = M<T>::sqrt_(qab2);
            const T xa = qab * r, xb = qab * ro;
            T a1, a2;
            if constexpr (sizeof(T) == 4) {
                a1 = cyl_a_tier<4>(xa * xa);
                a2 = cyl_a_tier<4>(xb * xb);
            } else {
                a1 = M<T>::cyl_a(xa, M<T>::rcp(xa), (T)0);
                a2 = M<T>::cyl_a(xb, M<T>::rcp(xb), (T)0);
            }
            const T sL = (T)2 * mc.half_length * M<T>::sinc(y1, M<T>::rcp(y1));
            const T sLo = (T)2 * mc.half_length_o * M<T>::sinc(y2, M<T>::rcp(y2));
            const T F = pi * (r * r * fma(mc.ev_k[0], sL, mc.ev_k[1] * sLo) * a1 +
                              ro * ro * fma(mc.ev_k[2], sL, mc.ev_k[3] * sLo) * a2);
            F2 = F * F;
        } else if constexpr (KIND == SAS_CORE_SHELL_ELLIPSOID) {
            const T ro = r + mc.shell;
            const T xc = M<T>::sqrt_(fma(r * r, qab2, mc.ev_rp * mc.ev_rp * qc * qc));
            const T xo = M<T>::sqrt_(fma(ro * ro, qab2, mc.rp2o * qc * qc));
            const T F = (T)4 * pi * (mc.ev_c1 * mc.ev_rp * r * r * M<T>::sphere_g(xc, M<T>::rcp(xc)) +
                                     mc.ev_c2 * mc.rp_o * ro * ro * M<T>::sphere_g(xo, M<T>::rcp(xo)));
            F2 = F * F;
        } else if (KIND == SAS_CYLINDER) {
            const T y = fabs(qc) * (T)0.5 * mc.ev_len;
            const T sn = M<T>::sinc(y, M<T>::rcp(y));
            const T x = M<T>::sqrt_(qab2) * r;
            T a;
            if constexpr (sizeof(T) == 4) {
                const float s = x * x;
                if (s <= SAS_J1P_SMAX) a = sas_cyl_a_s(s);
                else if (s <= SAS_J1Q_SMAX) a = sas_cyl_a_s3(s);
                else a = sas_cyl_a_large(x, __frcp_rn(x), rsqrtf(x));
            } else {
                a = M<T>::cyl_a(x, M<T>::rcp(x), (T)0);
            }
            const T F = mc.ev_c1 * pi * r * r * mc.ev_len * sn * a;
            F2 = F * F;
        } else {
            const T x = M<T>::sqrt_(fma(r * r, qab2, mc.ev_rp * mc.ev_rp * qc * qc));
            const T V = (T)(4.0 / 3.0) * pi * mc.ev_rp * r * r;
            const T F = (T)3 * mc.ev_c1 * V * M<T>::sphere_g(x, M<T>::rcp(x));
            F2 = F * F;
        }
    }
    return mc.scale * F2 * structure_factor<T>(q, mc);
}

// dSigma/dOmega of history `index` of experiment `exp_id`: the quadrature
// average, or the per-event estimate from the history's own draws.
template <typename T, int KIND, bool LEAN = false>
__device__ __forceinline__ T dsigma_history(const T qv[3], const ModelConst<T>& mc, const T* __restrict__ poly,
                                            const T* __restrict__ orient, uint64_t seed, uint32_t exp_id,
                                            uint64_t index)
{
    if constexpr (KIND != SAS_SHAPE_INDEPENDENT) {   // no draws: a law of |Q| only
        if (mc.event) return dsigma_event<T, KIND>(qv, mc, poly, event_draws(seed, exp_id, index));
    }
    return dsigma<T, KIND, LEAN>(qv, mc, poly, orient);
}

// ------------------------------------------------------------- geometry
template <typename T>
struct History {
    T q[3];      // scattering vector, 1/angstrom
    T pref;      // l * dOmega * attenuation * 1e10 (1/angstrom -> 1/m)
    T wt;        // transmitted (unscattered) weight
    int pixel;   // -1: the neutron missed the sample
};

// entry/exit ray parameters of the box |x|<=hx, |y|<=hy, 0<=z<=t
template <typename T>
__device__ __forceinline__ bool slab(const InstConst<T>& in, const T o[3], const T d[3], T& a, T& b)
{
    const T lo[3] = {-in.hx, -in.hy, (T)0};
    const T hi[3] = {in.hx, in.hy, in.thick};
    a = (T)-1e30;
    b = (T)1e30;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] == (T)0) {
            ok = ok && (o[k] >= lo[k]) && (o[k] <= hi[k]);
        } else {
            const T id = M<T>::rcp(d[k]);
            T t1 = (lo[k] - o[k]) * id, t2 = (hi[k] - o[k]) * id;
            const T mn = fmin(t1, t2), mx = fmax(t1, t2);
            a = fmax(a, mn);
            b = fmin(b, mx);
        }
    }
    a = fmax(a, (T)0);
    return ok && (b > a);
}

// mu_s(lambda) in 1/m from its Chebyshev interpolant (Clenshaw's recurrence).
template <typename T>
__device__ __forceinline__ T att_mu(const AttTable<T>& a, T lambda)
{
    const T t = fma(lambda, a.t_mul, a.t_add);
    const T t2 = t + t;
    T b1 = (T)0, b2 = (T)0;
#pragma unroll
    for (int j = SAS_ATT_MAX - 1; j >= 1; --j) {
        if (j < a.n) {
            const T b0 = fma(t2, b1, a.c[j] - b2);
            b2 = b1;
            b1 = b0;
        }
    }
    return fma(t, b1, a.c[0] - b2);
}

// One history up to the scattering vector and the weight prefactor. The
// beam inside the sample is attenuated with the instrument's mu plus, when
// ATT and att.n > 0, the particles' own total scattering mu_s(lambda)
// (ATT = false compiles the plain path without the table).
template <typename T, bool ATT = true>
__device__ __forceinline__ History<T> history(const InstConst<T>& in, const AttTable<T>& att, uint64_t seed,
                                              uint32_t exp_id, uint64_t index)
{
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 r0 = philox(make_uint4(0u, exp_id, (uint32_t)index, (uint32_t)(index >> 32)), key);
    const uint4 r1 = philox(make_uint4(1u, exp_id, (uint32_t)index, (uint32_t)(index >> 32)), key);
    History<T> h;
    // source wavelength: triangular spread by inverse CDF
    const T u = u01<T>(r0.x);
    const bool lower = u < (T)0.5;
    const T sq = M<T>::sqrt_pos((T)2 * (lower ? u : (T)1 - u));
    const T tri = lower ? sq - (T)1 : (T)1 - sq;
    const T lambda = in.lambda0 * ((T)1 + in.dlambda * tri);
    // pinholes: area-uniform points on both discs
    T s1, c1, s2, c2;
    M<T>::sincos2pi(u01<T>(r0.z), s1, c1);
    M<T>::sincos2pi(u01<T>(r1.x), s2, c2);
    const T rr1 = in.ap1_r * M<T>::sqrt_pos(u01<T>(r0.y));
    const T rr2 = in.ap2_r * M<T>::sqrt_pos(u01<T>(r0.w));
    const T p2[3] = {rr2 * c2, rr2 * s2, in.ap2_z};
    T d[3] = {p2[0] - rr1 * c1, p2[1] - rr1 * s1, in.ap2_z - in.ap1_z};
    const T idn = M<T>::rsqrt(fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2])));
    const T ki[3] = {d[0] * idn, d[1] * idn, d[2] * idn};
    T t_in, t_out;
    if (!slab<T>(in, p2, ki, t_in, t_out)) {
        h.pixel = -1;
        h.wt = (T)1;
        h.pref = (T)0;
        h.q[0] = h.q[1] = h.q[2] = (T)0;
        return h;
    }
    const T l = t_out - t_in;
    T mu = in.mu;
    if constexpr (ATT) {
        if (att.n > 0) mu += att_mu<T>(att, lambda);
    }
    h.wt = (mu > (T)0) ? M<T>::exp_(-mu * l) : (T)1;
    const T s = u01<T>(r1.y) * l;
    const T ps[3] = {fma(t_in + s, ki[0], p2[0]), fma(t_in + s, ki[1], p2[1]),
                     fma(t_in + s, ki[2], p2[2])};
    // detector point: integer pixel choice, sub-pixel position from the remainder
    const uint64_t mx = (uint64_t)(r1.z >> 9) * (uint64_t)in.nx;
    const uint64_t my = (uint64_t)(r1.w >> 9) * (uint64_t)in.ny;
    const int ix = (int)(mx >> 23), iy = (int)(my >> 23);
    T fx, fy, fix, fiy;
    if constexpr (sizeof(T) == sizeof(float)) {   // the same values, no conversion instructions
        fx = __uint_as_float((uint32_t)(mx & 0x7FFFFFu) | 0x3F800000u) - 0.99999994f;
        fy = __uint_as_float((uint32_t)(my & 0x7FFFFFu) | 0x3F800000u) - 0.99999994f;
        fix = small_uint_to_float((uint32_t)ix);
        fiy = small_uint_to_float((uint32_t)iy);
    } else {
        fx = (T)(uint32_t)(mx & 0x7FFFFFu) * (T)(1.0 / 8388608.0) + (T)(0.5 / 8388608.0);
        fy = (T)(uint32_t)(my & 0x7FFFFFu) * (T)(1.0 / 8388608.0) + (T)(0.5 / 8388608.0);
        fix = (T)ix;
        fiy = (T)iy;
    }
    const T pd0 = fma(fix + fx, in.px, -in.half_wx);
    const T pd1 = fma(fiy + fy, in.py, -in.half_wy);
    const T v[3] = {pd0 - ps[0], pd1 - ps[1], in.det_z - ps[2]};
    const T ir = M<T>::rsqrt(fma(v[0], v[0], fma(v[1], v[1], v[2] * v[2])));
    const T ko[3] = {v[0] * ir, v[1] * ir, v[2] * ir};
    const T domega = in.area * ko[2] * ir * ir;
    // Q = k (k_out - k_in); the z difference without cancellation
    const T k = in.two_pi * M<T>::rcp(lambda);
    const T tin = fma(ki[0], ki[0], ki[1] * ki[1]);
    const T tout = fma(ko[0], ko[0], ko[1] * ko[1]);
    h.q[0] = k * (ko[0] - ki[0]);
    h.q[1] = k * (ko[1] - ki[1]);
    h.q[2] = k * (tin - tout) * M<T>::rcp(ko[2] + ki[2]);
    T out_att = (T)1;
    if (mu > (T)0) {
        T e_in, e_out, l_out = (T)0;
        if (slab<T>(in, ps, ko, e_in, e_out)) l_out = e_out - e_in;
        out_att = M<T>::exp_(-mu * (s + l_out));
    }
    h.pref = l * domega * out_att * (T)1e10;
    h.pixel = iy * in.nx + ix;
    return h;
}

}  // namespace sas
