// FP32 special functions of the form factors (sinc, spherical and cylindrical
// Bessel amplitudes) on the FMA pipe.
//
// Written for the device; the same source compiles as plain C++ (SAS_HD
// empty) so that its arithmetic can be checked against FP64 references on a
// host without a GPU. Only IEEE-exact primitives are used (fmaf,
// multiplication, addition, bit moves), so host and device give identical bits.
//
//  * sin / cos: two-part FMA Cody-Waite reduction by pi/2, polynomials on
//    [-pi/4, pi/4] fitted toward minimax (gen_coeffs.py).
//  * sphere amplitude f(x) = 3 (sin x - x cos x) / x^3: quadrant handled by
//    two FMAs, one select and a sign flip; in the first quadrant it is
//    3 (S - C) from the same polynomials, free of the closed form's
//    cancellation at small x. (The trace kernels take sin and cos from the
//    special-function unit instead; these forms serve the surrogate's exact
//    targets and the host checks.)
//  * cylinder radial factor a(x) = 2 J1(x) / x: fitted polynomials in x^2
//    (plain to x = 4, centred to x = 6, with the first two or three zeros of
//    J1 as exact factors to x = 8 and 12), the modulus-phase form of J1
//    beyond.
#pragma once

#include <math.h>
#include <string.h>
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
    int kb;    // low bits of the quadrant index k (k mod 4 = kb & 3)
};

// Round to the nearest integer with the 1.5 * 2^23 constant (valid for
// |v| < 2^22): v + C lands on an integer grid; k = (v + C) - C and the low
// bits of (v + C) hold k mod 2^22. Two FP32 adds, no conversion instruction.
#define SAS_RND_C 12582912.0f

SAS_HD float sas_round_magic(float v, int& kbits)
{
    const float t = v + SAS_RND_C;
    float bits_src = t;
    unsigned u;
    memcpy(&u, &bits_src, sizeof(u));
    kbits = (int)u;
    return t - SAS_RND_C;
}

SAS_HD float sas_flip_sign(float v, int bit31)
{
    unsigned u;
    memcpy(&u, &v, sizeof(u));
    u ^= (unsigned)bit31 & 0x80000000u;
    float o;
    memcpy(&o, &u, sizeof(o));
    return o;
}

// x = k pi/2 + r, |r| <= pi/4 (up to rounding), for |x| < 2^20. Two-part
// Cody-Waite in FMA form: the products k * part are exact inside the FMA.
SAS_HD SasTrig sas_reduce_pio2(float x)
{
    const float cs[3] = SAS_SIN_C;
    const float cc[4] = SAS_COS_C;
    SasTrig o;
    float k = sas_round_magic(x * 0.636619772f, o.kb);
    float r = fmaf(-k, SAS_PIO2_1, x);
    r = fmaf(-k, SAS_PIO2_2, r);
    o.r = r;
    o.t = r * r;
    o.S = sas_horner(cs, o.t);
    o.C = sas_horner(cc, o.t);
    return o;
}

SAS_HD void sas_trig_sincos(const SasTrig& g, float& s, float& c)
{
    const float sr = fmaf(g.r * g.t, g.S, g.r);
    const float cr = fmaf(g.t, g.C, 1.0f);
    const int q = g.kb & 3;
    const float a = (q & 1) ? cr : sr;      // sin of the quadrant-shifted angle
    const float b = (q & 1) ? sr : cr;
    s = (q & 2) ? -a : a;
    c = ((q + 1) & 2) ? -b : b;
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
    const float big = s * inv;
    const float small = fmaf(g.t, g.S, 1.0f);   // k = 0: r = y exactly
    return (y < 0.78539816f) ? small : big;
}

// g(x) = f(x) / 3 = (sin x - x cos x) / x^3 for x >= 0 (f is the sphere
// amplitude 3 j1(x) / x); inv = 1 / x (may be inf at x = 0).
// With x = k pi/2 + r: sin x - x cos x = +-(sin r - x cos r) for even k and
// +-(cos r + x sin r) for odd k, the sign being (-1)^(k >> 1). In the first
// quadrant (r = x) it is r^3 (S - C), free of cancellation.
SAS_HD float sas_sphere_g(float x, float inv)
{
    const SasTrig g = sas_reduce_pio2(x);
    const float sr = fmaf(g.r * g.t, g.S, g.r);
    const float cr = fmaf(g.t, g.C, 1.0f);
    const float A = fmaf(-x, cr, sr);
    const float B = fmaf(x, sr, cr);
    float num = (g.kb & 1) ? B : A;
    num = sas_flip_sign(num, g.kb << 30);
    const float big = num * inv * inv * inv;
    const float small = g.S - g.C;
    return (x < 0.78539816f) ? small : big;
}

// f(x) = 3 (sin x - x cos x) / x^3
SAS_HD float sas_sphere_f(float x, float inv) { return 3.0f * sas_sphere_g(x, inv); }

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
    int kb;
    const float k = sas_round_magic(fmaf(x + eps, 0.636619772f, -0.5f), kb);
    const float K = fmaf(2.0f, k, 1.0f);
    float r = fmaf(-K, SAS_PIO4_1, x);
    r = fmaf(-K, SAS_PIO4_2, r);
    r = r + eps;
    const float cs[3] = SAS_SIN_C;
    const float cc[4] = SAS_COS_C;
    const float t = r * r;
    SasTrig g;
    g.r = r; g.t = t; g.S = sas_horner(cs, t); g.C = sas_horner(cc, t); g.kb = kb;
    float s, c;
    sas_trig_sincos(g, s, c);
    // 2 sqrt(2/pi) = 1.5957691216
    return 1.5957691216f * m * inv * rsx * s;
}

// a(x) = 2 J1(x) / x from s = x^2 <= SAS_J1P_SMAX (x <= 8): product of the
// first two zero factors and a fitted polynomial; no square root needed.
SAS_HD float sas_cyl_a_s(float s)
{
    const float c[9] = SAS_J1P_C;
    const float h = sas_horner(c, s);
    const float p1 = fmaf(-s, SAS_J1P_Z1, 1.0f);
    const float p2 = fmaf(-s, SAS_J1P_Z2, 1.0f);
    return p1 * p2 * h;
}

// a(x) for s = x^2 <= SAS_J1R_SMAX (x <= 4): a degree-6 polynomial in s.
SAS_HD float sas_cyl_a_r(float s)
{
    const float c[SAS_J1R_C_N] = SAS_J1R_C;
    return sas_horner(c, s);
}

// a(x) for s = x^2 <= SAS_J1V_SMAX (x <= 6): a degree-7 polynomial in the
// centred variable 2 s / 36 - 1.
SAS_HD float sas_cyl_a_v(float s)
{
    const float c[SAS_J1V_C_N] = SAS_J1V_C;
    return sas_horner(c, fmaf(s, 2.0f / SAS_J1V_SMAX, -1.0f));
}

// a(x) for s = x^2 <= SAS_J1Q_SMAX (x <= 12): three zero factors and a fit.
SAS_HD float sas_cyl_a_s3(float s)
{
    const float c[11] = SAS_J1Q_C;
    const float g = sas_horner(c, fmaf(s, 2.0f / SAS_J1Q_SMAX, -1.0f));
    const float p1 = fmaf(-s, SAS_J1Q_Z1, 1.0f);
    const float p2 = fmaf(-s, SAS_J1Q_Z2, 1.0f);
    const float p3 = fmaf(-s, SAS_J1Q_Z3, 1.0f);
    return (p1 * p2) * (p3 * g);
}

SAS_HD float sas_cyl_a(float x, float inv, float rsx)
{
    return (x <= SAS_J1_X1) ? sas_cyl_a_small(x) : sas_cyl_a_large(x, inv, rsx);
}
