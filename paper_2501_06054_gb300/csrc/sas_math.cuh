// FP32 special functions of the form factors (sinc, spherical and cylindrical
// Bessel amplitudes) on the FMA pipe.
//
// Written for the device; the same source compiles as plain C++ (SAS_HD
// empty) so that its arithmetic can be checked against FP64 references on a
// host without a GPU. Only IEEE-exact primitives are used (fmaf, rintf,
// multiplication, addition), so host and device give identical bits.
//
//  * sin / cos: Cody-Waite reduction by pi/2 in three parts, Taylor
//    polynomials on [-pi/4, pi/4] (Abramowitz and Stegun 4.3.65/4.3.66 style).
//  * sphere amplitude f(x) = 3 (sin x - x cos x) / x^3: in the first
//    quadrant it is evaluated as 3 (S - C) from the same polynomials, which
//    removes the cancellation of the closed form at small x.
//  * cylinder radial factor a(x) = 2 J1(x) / x: a fitted polynomial in
//    (x / X1)^2 below X1 = 4, the modulus-phase form of J1 above it.
#pragma once

#include <math.h>
#include "sas_coeffs.h"

#if defined(__CUDACC__)
#define SAS_HD __host__ __device__ __forceinline__
#else
#define SAS_HD inline
#endif

template <int N>
SAS_HD float sas_horner(const float (&c)[N], float x)
{
    float r = c[N - 1];
#pragma unroll
    for (int i = N - 2; i >= 0; --i) r = fmaf(r, x, c[i]);
    return r;
}

struct SasTrig {
    float r;   // reduced argument
    float t;   // r^2
    float S;   // sin r = r + r^3 S(t)
    float C;   // cos r = 1 + t C(t)
    int q;     // quadrant k mod 4
};

// x = k pi/2 + r, |r| <= pi/4 (up to rounding), valid for |x| < 2^12 pi/2.
SAS_HD SasTrig sas_reduce_pio2(float x)
{
    const float cs[4] = {-1.666666667e-01f, 8.333333333e-03f, -1.984126984e-04f,
                         2.755731922e-06f};
    const float cc[5] = SAS_COS_C;
    SasTrig o;
    float k = rintf(x * 0.636619772f);
    float r = fmaf(-k, SAS_PIO2_1, x);
    r = fmaf(-k, SAS_PIO2_2, r);
    r = fmaf(-k, SAS_PIO2_3, r);
    o.r = r;
    o.t = r * r;
    o.S = sas_horner(cs, o.t);
    o.C = sas_horner(cc, o.t);
    o.q = ((int)k) & 3;
    return o;
}

SAS_HD void sas_trig_sincos(const SasTrig& g, float& s, float& c)
{
    float sr = fmaf(g.r * g.t, g.S, g.r);
    float cr = fmaf(g.t, g.C, 1.0f);
    float a = (g.q & 1) ? cr : sr;      // sin of the quadrant-shifted angle
    float b = (g.q & 1) ? sr : cr;
    s = (g.q & 2) ? -a : a;
    c = ((g.q + 1) & 2) ? -b : b;
}

SAS_HD void sas_sincosf(float x, float& s, float& c)
{
    sas_trig_sincos(sas_reduce_pio2(x), s, c);
}

// sin(y) / y for y >= 0; inv = 1 / y (may be inf at y = 0)
SAS_HD float sas_sinc(float y, float inv)
{
    SasTrig g = sas_reduce_pio2(y);
    float s, c;
    sas_trig_sincos(g, s, c);
    float big = s * inv;
    float small = fmaf(g.t, g.S, 1.0f);   // k = 0: r = y exactly
    return (g.q == 0 && fabsf(y) < 1.0f) ? small : big;
}

// f(x) = 3 (sin x - x cos x) / x^3, x >= 0; inv = 1 / x (may be inf at x = 0)
SAS_HD float sas_sphere_f(float x, float inv)
{
    SasTrig g = sas_reduce_pio2(x);
    float s, c;
    sas_trig_sincos(g, s, c);
    float num = fmaf(-x, c, s);
    float inv3 = inv * inv * inv;
    float big = 3.0f * num * inv3;
    float small = 3.0f * (g.S - g.C);     // first quadrant: r = x
    return (x < 0.78539816f) ? small : big;
}

// a(x) = 2 J1(x) / x for 0 <= x <= X1
SAS_HD float sas_cyl_a_small(float x)
{
    const float cj[8] = SAS_J1S_C;
    float s = x * x * (1.0f / (SAS_J1_X1 * SAS_J1_X1));
    return sas_horner(cj, s);
}

// a(x) = 2 J1(x) / x for x > X1; inv = 1 / x, rsx = 1 / sqrt(x)
SAS_HD float sas_cyl_a_large(float x, float inv, float rsx)
{
    const float cm[6] = SAS_J1M_C;
    const float ch[6] = SAS_J1H_C;
    float u = (SAS_J1_X1 * SAS_J1_X1) * inv * inv;
    float m = sas_horner(cm, u);
    float eps = sas_horner(ch, u) * inv;
    // y' = x + eps - pi/4 = k pi/2 + r  ->  cos(theta) = sin(y')
    float k = rintf(fmaf(x + eps, 0.636619772f, -0.5f));
    float K = fmaf(2.0f, k, 1.0f);
    float r = fmaf(-K, SAS_PIO4_1, x);
    r = fmaf(-K, SAS_PIO4_2, r);
    r = fmaf(-K, SAS_PIO4_3, r);
    r = r + eps;
    const float cs[4] = {-1.666666667e-01f, 8.333333333e-03f, -1.984126984e-04f,
                         2.755731922e-06f};
    const float cc[5] = SAS_COS_C;
    float t = r * r;
    SasTrig g;
    g.r = r; g.t = t; g.S = sas_horner(cs, t); g.C = sas_horner(cc, t); g.q = ((int)k) & 3;
    float s, c;
    sas_trig_sincos(g, s, c);
    // 2 sqrt(2/pi) = 1.5957691216
    return 1.5957691216f * m * inv * rsx * s;
}

SAS_HD float sas_cyl_a(float x, float inv, float rsx)
{
    return (x <= SAS_J1_X1) ? sas_cyl_a_small(x) : sas_cyl_a_large(x, inv, rsx);
}
