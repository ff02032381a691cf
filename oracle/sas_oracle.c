/*
 * FP64 CPU oracle of the SANS Monte Carlo trace.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use this file. It shares no code, header,
 * table or constant with the CUDA library and must never be linked into it.
 *
 * It follows the method step by step in double precision, in the order the
 * paper describes one neutron history (Sec. II.A, instrument chain: source,
 * collimation, sample, 2D position-sensitive detector; single scattering,
 * Sec. I), and evaluates the averaged model by its plain definition:
 *
 *   amplitude A(Q) = integral of drho exp(-i Q.r) dV          (Eq. 1)
 *   intensity  I = (Phi / V) A A*                             (Eq. 2)
 *   dilute isotropic I = n drho^2 V^2 P(Q) S(Q)               (Eq. 3)
 *   model M = A* A / V                                        (Eq. 4)
 *   uniaxial particles A(Q_AB, Q_C)                           (Eq. 7)
 *   cylinder amplitude, volume pi r^2 L                       (Eq. 8)
 *
 * Optionally the beam inside the sample is also depleted by the particles'
 * own scattering: mu(lambda) = mu + Sigma_s(lambda), Sigma_s the model's
 * dSigma/dOmega integrated over all directions (single scattering: a
 * neutron scattered twice is lost, not redistributed).
 *
 * The quadrature nodes (Schulz polydispersity, orientation distribution) are
 * computed by the Python side of the oracle and passed in as arrays.
 * Special functions come from the C library (sin, cos, j1, exp, sqrt).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11),
 * key = (seed low 32 bits, seed high 32 bits), counter = (draw block,
 * experiment id, neutron index low 32 bits, neutron index high 32 bits).
 * With draw block 0 and experiment 0, neutron i reads the same four words as
 * block i of cuRAND's host Philox4x32-10 generator seeded with the same seed.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

static void gl_nodes(int n, double *x, double *w);

/* ---------------------------------------------------------------- Philox */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform on (0,1): 23 random bits plus one half, exact in float and double */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }
/* 1 - u01(x), also exact */
static double u01c(uint32_t x) { return ((double)(8388607u - (x >> 9)) + 0.5) * (1.0 / 8388608.0); }

/* ------------------------------------------------------------ structures */

typedef struct {
    double lambda0, dlambda_rel;
    double ap1_radius, ap1_z, ap2_radius, ap2_z;
    double sample_half_x, sample_half_y, sample_thickness;
    double mu;
    double det_distance, pixel_x, pixel_y;
    int64_t nx, ny;
} oracle_instrument;

typedef struct {
    int64_t kind;          /* 0 sphere, 1 core-shell, 2 cylinder, 3 ellipsoid, 4 triaxial
                              ellipsoid, 5 parallelepiped, 6 capped cylinder, 7 barbell,
                              8 core-shell cylinder, 9 hollow cylinder, 10 core-shell ellipsoid,
                              11 core-shell bicelle, 12 elliptical cylinder,
                              13 hollow rectangular prism, 14 shape-independent */
    int64_t sq_kind;       /* 0 none, 1 Percus-Yevick hard spheres, 2 Hayter-Penfold (table) */
    int64_t n_poly;        /* polydispersity nodes */
    int64_t n_orient;      /* orientation nodes */
    double radius, thickness, length, radius_polar;
    double sld, sld_shell, sld_solvent;
    double volume_fraction;
    double sq_radius, sq_fraction;
    const double *poly_r;  /* [n_poly] radii of the polydisperse radius */
    const double *poly_w;  /* [n_poly] normalised weights */
    const double *orient_c;/* [n_orient][3] particle axis unit vectors */
    const double *orient_w;/* [n_orient] normalised weights */
    /* per-event sampling (Sec. II.B): each history draws one radius and one
     * axis instead of averaging over the nodes above, which then serve only
     * for <V> of the radius distribution */
    int64_t event;         /* 0: quadrature average, 1: per-event draws */
    int64_t orient_mode;   /* axis draw: 0 fixed mean axis, 1 uniform on the sphere,
                              2 theta ~ U[0, pi], phi ~ U[0, 2 pi] */
    double poly;           /* sigma / mean of the Gaussian radius (0: monodisperse) */
    double axis_theta, axis_phi;   /* fixed axis (orient_mode 0) */
    /* particles without a symmetry axis (kinds 4, 5; Sec. II.B): sizes
     * (radius, radius_b, radius_polar) along the particle axes (A, B, C),
     * the orientation nodes are frames (A, B, C) of 9 doubles, and the
     * polydisperse nodes poly_r / radius scale all three sizes alike */
    double radius_b;
    double axis_psi;       /* rotation about C of the fixed frame (event mode 0) */
    /* 1: the beam inside the sample is attenuated by the particles' own
     * scattering as well, mu(lambda) = mu + Sigma_s(lambda) */
    int64_t self_att;
    /* capped cylinder and barbell (kinds 6, 7): Gauss-Legendre nodes of the
     * integral over each spherical end cap (1 to 64) */
    int64_t n_cap;
    /* core-shell cylinder (kind 8): thickness of the shell on the end faces;
     * core-shell ellipsoid (kind 10): thickness of the shell along the axis
     * (`thickness` is the shell's radial / equatorial thickness) */
    double thickness_face;
    /* core-shell bicelle (kind 11): density of the face layers */
    double sld_face;
    /* shape-independent models (kind 14): dSigma/dOmega = f_scale f(|Q|), f
     * selected by `function` with parameters f_p0..f_p2 */
    int64_t function;
    double f_scale, f_p0, f_p1, f_p2;
    /* Hayter-Penfold S(Q) (sq_kind 2), solved in oracle/msa.py: S_j and
     * dS/dQ_j interleaved at Q_j = j sq_dq, j < sq_n */
    const double *sq_tab;
    int64_t sq_n;
    double sq_dq;
    /* fuzzy sphere: width of the Gaussian the sphere's density is convolved with (0: sharp) */
    double fuzz;
} oracle_model;

/* --------------------------------------------------------- model pieces */

/* normalised sphere amplitude 3 (sin x - x cos x) / x^3, f(0) = 1 */
double oracle_sphere_f(double x)
{
    x = fabs(x);
    if (x < 0.1) {
        /* Taylor series: sum_m (-1)^m 6 (m+1) x^(2m) / (2m+3)! */
        double t = x * x;
        return 1.0 - t / 10.0 * (1.0 - t / 28.0 * (1.0 - t / 54.0 * (1.0 - t / 88.0
                                                        * (1.0 - t / 130.0))));
    }
    return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
}

/* 2 J1(x) / x, value 1 at x = 0 */
double oracle_cyl_a(double x)
{
    x = fabs(x);
    if (x < 1e-6) return 1.0 - x * x / 8.0;
    return 2.0 * j1(x) / x;
}

/* sin(y) / y */
double oracle_sinc(double y)
{
    y = fabs(y);
    if (y < 1e-8) return 1.0;
    return sin(y) / y;
}

/* Taylor coefficient (of A^(2m)) of each bracket of the Percus-Yevick G(A).
 * b1 = sin A - A cos A
 * b2 = 2 A sin A + (2 - A^2) cos A - 2
 * b3 = -A^4 cos A + 4 [ (3 A^2 - 6) cos A + (A^3 - 6 A) sin A + 6 ]
 * sin A = sum (-1)^n A^(2n+1)/(2n+1)!,  cos A = sum (-1)^n A^(2n)/(2n)!    */
static double fact(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }
static double sgn(int n) { return (n % 2 == 0) ? 1.0 : -1.0; }
/* coefficient of A^k in sin A and cos A */
static double sin_c(int k) { return (k % 2 == 1) ? sgn((k - 1) / 2) / fact(k) : 0.0; }
static double cos_c(int k) { return (k % 2 == 0) ? sgn(k / 2) / fact(k) : 0.0; }
static double b1_c(int k) { return sin_c(k) - (k >= 1 ? cos_c(k - 1) : 0.0); }
static double b2_c(int k)
{
    double c = (k >= 1 ? 2.0 * sin_c(k - 1) : 0.0) + 2.0 * cos_c(k)
             - (k >= 2 ? cos_c(k - 2) : 0.0) - (k == 0 ? 2.0 : 0.0);
    return c;
}
static double b3_c(int k)
{
    double c = -(k >= 4 ? cos_c(k - 4) : 0.0);
    double in = (k >= 2 ? 3.0 * cos_c(k - 2) : 0.0) - 6.0 * cos_c(k)
              + (k >= 3 ? sin_c(k - 3) : 0.0) - (k >= 1 ? 6.0 * sin_c(k - 1) : 0.0)
              + (k == 0 ? 6.0 : 0.0);
    return c + 4.0 * in;
}

/* Percus-Yevick hard-sphere structure factor (Wertheim / Thiele closed form).
 * S(q) = 1 / (1 + 24 phi G(A) / A), A = 2 q R, with
 * G(A) = alpha b1/A^2 + beta b2/A^3 + gamma b3/A^5,
 * alpha = (1+2phi)^2/(1-phi)^4, beta = -6 phi (1+phi/2)^2/(1-phi)^4,
 * gamma = phi alpha / 2.                                                    */
double oracle_sq_py(double q, double radius, double phi);

/* S(Q) from the table of a solved Hayter-Penfold model: cubic Hermite
 * interpolation of S and dS/dQ; beyond the table S - 1 decays as Q^-2. */
static double oracle_sq_table(const oracle_model *m, double q)
{
    double s = q / m->sq_dq;
    int64_t last = m->sq_n - 1;
    if (s >= (double)last) {
        double r = (double)last / s;
        return 1.0 + (m->sq_tab[2 * last] - 1.0) * r * r;
    }
    int64_t i = (int64_t)s;
    double f = s - (double)i, h = m->sq_dq;
    double s0 = m->sq_tab[2 * i], d0 = m->sq_tab[2 * i + 1] * h;
    double s1 = m->sq_tab[2 * i + 2], d1 = m->sq_tab[2 * i + 3] * h;
    double h00 = (1.0 + 2.0 * f) * (1.0 - f) * (1.0 - f), h10 = f * (1.0 - f) * (1.0 - f);
    double h01 = f * f * (3.0 - 2.0 * f), h11 = f * f * (f - 1.0);
    return h00 * s0 + h10 * d0 + h01 * s1 + h11 * d1;
}

double oracle_sq_py(double q, double radius, double phi)
{
    double A = 2.0 * fabs(q) * radius;
    double d = pow(1.0 - phi, 4);
    double alpha = (1.0 + 2.0 * phi) * (1.0 + 2.0 * phi) / d;
    double beta = -6.0 * phi * (1.0 + 0.5 * phi) * (1.0 + 0.5 * phi) / d;
    double gamma = 0.5 * phi * alpha;
    double GA; /* G(A)/A */
    if (A < 0.5) {
        /* series of each bracket: b1 ~ A^3, b2 ~ A^4, b3 ~ A^6 */
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, Ak;
        Ak = 1.0; for (int k = 3; k <= 3 + 30; ++k) { s1 += b1_c(k) * Ak; Ak *= A; }
        Ak = 1.0; for (int k = 4; k <= 4 + 30; ++k) { s2 += b2_c(k) * Ak; Ak *= A; }
        Ak = 1.0; for (int k = 6; k <= 6 + 30; ++k) { s3 += b3_c(k) * Ak; Ak *= A; }
        /* b1/A^3 = s1, b2/A^4 = s2, b3/A^6 = s3 */
        GA = alpha * s1 + beta * s2 + gamma * s3;
    } else {
        double sA = sin(A), cA = cos(A);
        double b1 = sA - A * cA;
        double b2 = 2.0 * A * sA + (2.0 - A * A) * cA - 2.0;
        double b3 = -A * A * A * A * cA
                  + 4.0 * ((3.0 * A * A - 6.0) * cA + (A * A * A - 6.0 * A) * sA + 6.0);
        GA = alpha * b1 / (A * A * A) + beta * b2 / (A * A * A * A)
           + gamma * b3 / (A * A * A * A * A * A);
    }
    return 1.0 / (1.0 + 24.0 * phi * GA);
}

static double sphere_volume(double r) { return 4.0 / 3.0 * PI * r * r * r; }

/* x^-a gamma(a, x) = x^-a int_0^x t^(a-1) e^-t dt, the scaled lower
 * incomplete gamma function (a > 0, x > 0): the power series
 * e^-x sum_n x^n / (a (a+1) ... (a+n)) (Abramowitz-Stegun 6.5.29) for
 * x < a + 1; above, Gamma(a) x^-a - e^-x CF(a, x) with the continued
 * fraction of Gamma(a, x) (A-S 6.5.31, even part) evaluated by Lentz's
 * method. */
static double oracle_scaled_lower_gamma(double a, double x)
{
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term;
        for (int n = 1; n < 1000 && term > 1e-18 * sum; ++n) {
            term *= x / (a + n);
            sum += term;
        }
        return exp(-x) * sum;
    }
    /* Gamma(a, x) = e^-x x^a / (x + 1 - a - 1 (1 - a) / (x + 3 - a - 2 (2 - a) / (x + 5 - a - ...))) */
    const double tiny = 1e-300;
    double b = x + 1.0 - a, f = 1.0 / b, C = 1.0 / tiny, D = 1.0 / b;
    for (int i = 1; i < 1000; ++i) {
        double an = -i * (i - a);
        b += 2.0;
        D = an * D + b;
        if (fabs(D) < tiny) D = tiny;
        C = b + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-16) break;
    }
    return tgamma(a) * pow(x, -a) - exp(-x) * f;
}

/* Scattering cross section per unit volume dSigma/dOmega(Q) in 1/angstrom:
 * (phi / <V>) <|F|^2> S(Q), F = drho V f, averages over the polydispersity
 * nodes (and, for the uniaxial models, over the orientation nodes).      */
/* Shape-independent models (the isotropic group G): dSigma/dOmega as a
 * function of |Q| alone, f_scale times
 *   0 Guinier            exp(-Q^2 Rg^2 / 3)                    (p0 = Rg)
 *   1 Gaussian coil      Debye's 2 (exp(-u) - 1 + u) / u^2,
 *                        u = (Q Rg)^2                          (p0 = Rg)
 *   2 Lorentzian         1 / (1 + (Q xi)^2)                    (p0 = xi)
 *   3 Debye-Anderson-Brumberger 1 / (1 + (Q xi)^2)^2           (p0 = xi)
 *   4 power law          Q^-m                                  (p0 = m)
 *   5 Gaussian peak      exp(-(Q - Q0)^2 / (2 sigma^2))        (p0 = Q0, p1 = sigma)
 *   6 Teubner-Strey      1 / (a2 + c1 Q^2 + c2 Q^4)            (p0 = a2, p1 = c1, p2 = c2)
 * The coil below u = 1e-3 by its series 1 - u/3 + u^2/12 (the closed form
 * cancels there), above it with expm1. */
static double oracle_shape_independent(const oracle_model *m, double q)
{
    double q2 = q * q, f;
    switch (m->function) {
    case 0: f = exp(-q2 * m->f_p0 * m->f_p0 / 3.0); break;
    case 1: {
        double u = q2 * m->f_p0 * m->f_p0;
        f = u < 1e-3 ? 1.0 - u / 3.0 + u * u / 12.0 : 2.0 * (expm1(-u) + u) / (u * u);
        break;
    }
    case 2: f = 1.0 / (1.0 + q2 * m->f_p0 * m->f_p0); break;
    case 3: { double d = 1.0 + q2 * m->f_p0 * m->f_p0; f = 1.0 / (d * d); break; }
    case 4: f = pow(q, -m->f_p0); break;
    case 5: { double d = (q - m->f_p0) / m->f_p1; f = exp(-0.5 * d * d); break; }
    case 6: f = 1.0 / (m->f_p0 + q2 * (m->f_p1 + q2 * m->f_p2)); break;
    case 7: { double d = (q - m->f_p0) / m->f_p1; f = 1.0 / (1.0 + d * d); break; }   /* peak Lorentz */
    case 8:   /* two power laws meeting at q_c = f_p0: q^-m1 below, q_c^(m2 - m1) q^-m2 above */
        f = q <= m->f_p0 ? pow(q, -m->f_p1) : pow(m->f_p0, m->f_p2 - m->f_p1) * pow(q, -m->f_p2);
        break;
    case 9: {   /* Guinier-Porod (Hammouda): Rg = f_p0, dimension variable s = f_p1, Porod exponent m = f_p2 */
        double rg = m->f_p0, sd = m->f_p1, mp = m->f_p2;
        double q1 = sqrt((mp - sd) * (3.0 - sd) / 2.0) / rg;
        if (q <= q1) f = pow(q, -sd) * exp(-q2 * rg * rg / (3.0 - sd));
        else f = pow(q1, mp - sd) * exp(-(mp - sd) / 2.0) * pow(q, -mp);
        break;
    }
    case 10: {  /* Gauss-Lorentz gel: exp(-q^2 Xi^2 / 2) + r / (1 + q^2 xi^2) */
        f = exp(-0.5 * q2 * m->f_p0 * m->f_p0) + m->f_p2 / (1.0 + q2 * m->f_p1 * m->f_p1);
        break;
    }
    case 11: {  /* polydisperse Gaussian coil (Schulz-Zimm): Rg = f_p0, U = Mw/Mn - 1 = f_p1 */
        double U = m->f_p1, x = q2 * m->f_p0 * m->f_p0 / (1.0 + 2.0 * U);
        if (x * (1.0 + U) < 1e-2) {
            /* 2 / (1 + U) sum_{k>=2} (-x)^(k-2) prod_{j=1}^{k-1} (1 + jU) / k!, to k = 9: successive
               terms shrink by x (1 + (k - 1) U) / k < 0.09 / k here, so the first omitted one is
               below 1e-14 of the sum */
            double c = (1.0 + U) / 2.0, sum = c;
            for (int k = 3; k <= 9; ++k) {
                c *= -x * (1.0 + (k - 1) * U) / k;
                sum += c;
            }
            f = 2.0 * sum / (1.0 + U);
        } else {
            double t = U > 0.0 ? log1p(U * x) / U : x;
            /* exp(-t) + x - 1 written as expm1(-t) + x: rounding then scales as eps / x, not eps / x^2 */
            f = 2.0 * (expm1(-t) + x) / ((1.0 + U) * x * x);
        }
        break;
    }
    case 13:    /* mass fractal (Mildner-Hall): spheres of radius f_p0, dimension f_p1, cutoff f_p2 */
    case 14: {  /* fractal aggregate (Teixeira): spheres of radius f_p0, dimension f_p1, cutoff f_p2 */
        double D = m->f_p1, y = q * m->f_p2, e = D - 1.0, P = oracle_sphere_f(q * m->f_p0);
        /* transform of r^(D - 3) exp(-r / xi), normalised to 1 at Q = 0 */
        double M = y < 1e-8 ? 1.0 : sin(e * atan(y)) / (e * y * pow(1.0 + y * y, 0.5 * e));
        f = P * P * (m->function == 13 ? M : 1.0 + tgamma(D + 1.0) * pow(m->f_p2 / m->f_p0, D) * M);
        break;
    }
    case 15: {  /* spinodal (Furukawa): Qmax = f_p0, exponent g = f_p1 */
        double x = q / m->f_p0, g = m->f_p1;
        f = (1.0 + g / 2.0) * x * x / (g / 2.0 + pow(x, 2.0 + g));
        break;
    }
    case 16: {  /* polymer with excluded volume (Hammouda): Rg = f_p0, Porod exponent m = 1/nu = f_p1;
                   P = 2 int_0^1 (1 - x) exp(-U x^(2 nu)) dx, U = Q^2 Rg^2 (2 nu + 1)(2 nu + 2) / 6,
                   = m (U^(-m/2) gamma(m/2, U) - U^(-m) gamma(m, U)) */
        double mp = m->f_p1, nu = 1.0 / mp;
        double U = q2 * m->f_p0 * m->f_p0 * (2.0 * nu + 1.0) * (2.0 * nu + 2.0) / 6.0;
        f = U < 1e-300 ? 1.0
                       : mp * (oracle_scaled_lower_gamma(0.5 * mp, U) - oracle_scaled_lower_gamma(mp, U));
        break;
    }
    case 17: {  /* linear pearls: N = f_p2 spheres of radius R = f_p0 on a line, centres d = 2R + f_p1 apart;
                   Debye's sum over the pairs, normalised to 1 at Q = 0 */
        double R = m->f_p0, d = 2.0 * R + m->f_p1, P = oracle_sphere_f(q * R);
        int64_t N = (int64_t)m->f_p2;
        double pairs = (double)N;
        for (int64_t k = 1; k < N; ++k) {
            double y = q * k * d;
            pairs += 2.0 * (double)(N - k) * (y < 1e-8 ? 1.0 : sin(y) / y);
        }
        f = P * P * pairs / ((double)N * (double)N);
        break;
    }
    default: {  /* star polymer (Benoit): Rg = f_p0 of the star, f_p1 arms */
        double fa = m->f_p1, v = q2 * m->f_p0 * m->f_p0 * fa / (3.0 * fa - 2.0);
        double deb, g;
        if (v < 1e-3) {
            deb = 1.0 - v / 3.0 + v * v / 12.0;
            g = 1.0 - v / 2.0 + v * v / 6.0;
        } else {
            deb = 2.0 * (expm1(-v) + v) / (v * v);
            g = -expm1(-v) / v;
        }
        f = (deb + (fa - 1.0) * g * g) / fa;
        break;
    }
    }
    return m->f_scale * f;
}

double oracle_dsigma(const oracle_model *m, const double q[3])
{
    double qq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    if (m->kind == 14) return oracle_shape_independent(m, qq);
    double sum = 0.0, vmean = 0.0;
    int64_t np = m->n_poly;
    if (m->kind == 0) {              /* sphere; fuzzy: the amplitude of its density convolved with a
                                        Gaussian of width fuzz, the product with exp(-(Q fuzz)^2 / 2) */
        double drho = m->sld - m->sld_solvent, blur = exp(-0.5 * qq * qq * m->fuzz * m->fuzz);
        for (int64_t i = 0; i < np; ++i) {
            double r = m->poly_r[i], V = sphere_volume(r);
            double F = drho * V * oracle_sphere_f(qq * r) * blur;
            sum += m->poly_w[i] * F * F;
            vmean += m->poly_w[i] * V;
        }
    } else if (m->kind == 1) {       /* core-shell sphere: core radius polydisperse */
        for (int64_t i = 0; i < np; ++i) {
            double rc = m->poly_r[i], ro = rc + m->thickness;
            double Vc = sphere_volume(rc), Vo = sphere_volume(ro);
            double F = (m->sld - m->sld_shell) * Vc * oracle_sphere_f(qq * rc)
                     + (m->sld_shell - m->sld_solvent) * Vo * oracle_sphere_f(qq * ro);
            sum += m->poly_w[i] * F * F;
            vmean += m->poly_w[i] * Vo;
        }
    } else if (m->kind == 2) {       /* cylinder: radius polydisperse, length fixed */
        double drho = m->sld - m->sld_solvent;
        for (int64_t i = 0; i < np; ++i)
            vmean += m->poly_w[i] * PI * m->poly_r[i] * m->poly_r[i] * m->length;
        for (int64_t o = 0; o < m->n_orient; ++o) {
            const double *c = m->orient_c + 3 * o;
            double qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2];
            double x0 = q[1] * c[2] - q[2] * c[1];
            double x1 = q[2] * c[0] - q[0] * c[2];
            double x2 = q[0] * c[1] - q[1] * c[0];
            double qab = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
            double s = oracle_sinc(0.5 * qc * m->length);
            double inner = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double r = m->poly_r[i];
                double V = PI * r * r * m->length;
                double F = drho * V * s * oracle_cyl_a(qab * r);
                inner += m->poly_w[i] * F * F;
            }
            sum += m->orient_w[o] * inner;
        }
    } else if (m->kind == 4 || m->kind == 5 || m->kind == 12 || m->kind == 13) {
        /* triaxial ellipsoid (semi-axes a, b, c): F = drho V f(x),
         * x = |(a Q_A, b Q_B, c Q_C)|, V = 4/3 pi a b c (Eq. 1 on the affine
         * image of a sphere); rectangular parallelepiped (half-edges a, b, c):
         * F = drho V sinc(a Q_A) sinc(b Q_B) sinc(c Q_C), V = 8 a b c.
         * Elliptical cylinder (12): cross-section semi-axes a, b along A, B,
         * length L along C (c = L/2): F = drho V sinc(c Q_C) a(|(a Q_A, b Q_B)|),
         * a(x) = 2 J1(x)/x (the affine image of the circular cylinder),
         * V = pi a b L. Hollow rectangular prism (13): the parallelepiped of
         * half-edges (a, b, c) less the inner one (a - t, b - t, c - t), walls
         * t thick: F = drho [V sinc sinc sinc - V_i sinc_i sinc_i sinc_i],
         * normalised by the wall volume V - V_i. */
        double drho = m->sld - m->sld_solvent;
        double a0 = m->radius, b0 = m->radius_b, c0 = m->kind == 12 ? 0.5 * m->length : m->radius_polar;
        double t = m->kind == 13 ? m->thickness : 0.0;
        double ai = a0 - t, bi = b0 - t, ci = c0 - t;
        double vo = m->kind == 4 ? 4.0 / 3.0 * PI * a0 * b0 * c0
                  : m->kind == 12 ? PI * a0 * b0 * 2.0 * c0 : 8.0 * a0 * b0 * c0;
        double vi = m->kind == 13 ? 8.0 * ai * bi * ci : 0.0;
        double v0 = vo - vi;
        for (int64_t i = 0; i < np; ++i) {
            double s = m->poly_r[i] / m->radius;
            vmean += m->poly_w[i] * v0 * s * s * s;
        }
        for (int64_t o = 0; o < m->n_orient; ++o) {
            const double *f = m->orient_c + 9 * o;
            double qa = q[0] * f[0] + q[1] * f[1] + q[2] * f[2];
            double qb = q[0] * f[3] + q[1] * f[4] + q[2] * f[5];
            double qc = q[0] * f[6] + q[1] * f[7] + q[2] * f[8];
            double inner = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double s = m->poly_r[i] / m->radius;
                double V = v0 * s * s * s, F;
                if (m->kind == 4) {
                    double xa = s * a0 * qa, xb = s * b0 * qb, xc = s * c0 * qc;
                    F = drho * V * oracle_sphere_f(sqrt(xa * xa + xb * xb + xc * xc));
                } else if (m->kind == 12) {
                    double xa = s * a0 * qa, xb = s * b0 * qb;
                    F = drho * V * oracle_sinc(s * c0 * qc) * oracle_cyl_a(sqrt(xa * xa + xb * xb));
                } else if (m->kind == 13) {
                    double s3 = s * s * s;
                    F = drho * s3 * (vo * oracle_sinc(s * a0 * qa) * oracle_sinc(s * b0 * qb) * oracle_sinc(s * c0 * qc)
                                     - vi * oracle_sinc(s * ai * qa) * oracle_sinc(s * bi * qb) * oracle_sinc(s * ci * qc));
                } else {
                    F = drho * V * oracle_sinc(s * a0 * qa) * oracle_sinc(s * b0 * qb)
                      * oracle_sinc(s * c0 * qc);
                }
                inner += m->poly_w[i] * F * F;
            }
            sum += m->orient_w[o] * inner;
        }
    } else if (m->kind == 6 || m->kind == 7) {
        /* capped cylinder (6) and barbell (7): a cylinder of radius r and
         * length L along the axis with two spherical end caps of radius R >= r.
         * The caps are the parts of the spheres beyond the end faces z = +-L/2;
         * the sphere centres sit at +-(L/2 -+ h), h = sqrt(R^2 - r^2), inside
         * the cylinder for the capped cylinder and outside for the barbell,
         * so each cap is H = R -+ h high. Eq. 1 summed over slices normal to
         * the axis, each a disk of radius rho(z) with amplitude
         * pi rho^2 a(Q_AB rho) e^(i Q_C z), a(x) = 2 J1(x)/x; on a cap the
         * slice at depth R u below its tip has rho^2 = R^2 u (2 - u):
         *   F = drho [pi r^2 L sinc(Q_C L / 2) a(Q_AB r)
         *      + 2 pi R^3 int_0^(H/R) cos(Q_C (L/2 + H - R u)) u (2 - u) a(Q_AB R sqrt(u (2 - u))) du],
         * the cap integral by an n_cap point Gauss-Legendre rule. (u = 1 - t
         * with t the slice's height above the sphere centre in units of R;
         * written in u the rule has no cancellation for R >> r.) The
         * capped cylinder's H = R - h is formed as r^2 / (R + h). One
         * polydisperse factor s = r_i / radius scales r, R and L alike. */
        double drho = m->sld - m->sld_solvent;
        double r0 = m->radius, R0 = m->radius_polar, L0 = m->length;
        double h0 = sqrt(fmax(R0 * R0 - r0 * r0, 0.0));
        double H0 = m->kind == 6 ? r0 * r0 / (R0 + h0) : R0 + h0;
        int nc = (int)m->n_cap;
        double gx[64], gw[64], uj[64], wj[64];
        gl_nodes(nc, gx, gw);
        for (int j = 0; j < nc; ++j) {
            uj[j] = 0.5 * (H0 / R0) * (1.0 + gx[j]);
            wj[j] = 0.5 * (H0 / R0) * gw[j];
        }
        /* int_0^(H/R) u (2 - u) du = (H/R)^2 (1 - H / 3R) */
        double v0 = PI * r0 * r0 * L0 + 2.0 * PI * R0 * H0 * H0 * (1.0 - H0 / (3.0 * R0));
        for (int64_t i = 0; i < np; ++i) {
            double sc = m->poly_r[i] / r0;
            vmean += m->poly_w[i] * v0 * sc * sc * sc;
        }
        for (int64_t o = 0; o < m->n_orient; ++o) {
            const double *c = m->orient_c + 3 * o;
            double qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2];
            double x0 = q[1] * c[2] - q[2] * c[1];
            double x1 = q[2] * c[0] - q[0] * c[2];
            double x2 = q[0] * c[1] - q[1] * c[0];
            double qab = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
            double inner = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double sc = m->poly_r[i] / r0;
                double r = sc * r0, R = sc * R0, L = sc * L0, H = sc * H0;
                double F = PI * r * r * L * oracle_sinc(0.5 * qc * L) * oracle_cyl_a(qab * r);
                double cap = 0.0;
                for (int j = 0; j < nc; ++j) {
                    double v = uj[j] * (2.0 - uj[j]);
                    cap += wj[j] * cos(qc * (0.5 * L + H - R * uj[j])) * v
                         * oracle_cyl_a(qab * R * sqrt(v));
                }
                F = drho * (F + 2.0 * PI * R * R * R * cap);
                inner += m->poly_w[i] * F * F;
            }
            sum += m->orient_w[o] * inner;
        }
    } else if (m->kind == 8 || m->kind == 9) {
        /* core-shell cylinder (8): a core cylinder (r, L, rho_core) inside a
         * shell that adds t around it and t_f on each end face (rho_shell);
         * by Eq. 1 each region's amplitude is the difference of two nested
         * cylinders, so
         *   F = (rho_c - rho_s) pi r^2 L sinc(Q_C L/2) a(Q_AB r)
         *     + (rho_s - rho_solv) V_o sinc(Q_C (L/2 + t_f)) a(Q_AB (r + t)),
         * V_o = pi (r + t)^2 (L + 2 t_f), normalised by <V_o>.
         * Hollow cylinder (9): a tube of wall material (sld) between r and
         * r + t over the length L, solvent inside:
         *   F = (rho - rho_solv) sinc(Q_C L/2) [pi (r + t)^2 L a(Q_AB (r + t)) - pi r^2 L a(Q_AB r)],
         * normalised by the wall volume <pi ((r + t)^2 - r^2) L>.
         * The core (hollow) radius r is polydisperse, t, t_f and L fixed. */
        double t = m->thickness, L = m->length;
        double tf = m->kind == 8 ? m->thickness_face : 0.0;
        double d1 = m->kind == 8 ? m->sld - m->sld_shell : -(m->sld - m->sld_solvent);
        double d2 = m->kind == 8 ? m->sld_shell - m->sld_solvent : m->sld - m->sld_solvent;
        for (int64_t i = 0; i < np; ++i) {
            double r = m->poly_r[i], ro = r + t;
            vmean += m->poly_w[i] * (m->kind == 8 ? PI * ro * ro * (L + 2.0 * tf) : PI * (ro * ro - r * r) * L);
        }
        for (int64_t o = 0; o < m->n_orient; ++o) {
            const double *c = m->orient_c + 3 * o;
            double qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2];
            double x0 = q[1] * c[2] - q[2] * c[1];
            double x1 = q[2] * c[0] - q[0] * c[2];
            double x2 = q[0] * c[1] - q[1] * c[0];
            double qab = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
            double s1 = oracle_sinc(0.5 * qc * L);
            double s2 = oracle_sinc(qc * (0.5 * L + tf));
            double inner = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double r = m->poly_r[i], ro = r + t;
                double F = d1 * PI * r * r * L * s1 * oracle_cyl_a(qab * r)
                         + d2 * PI * ro * ro * (L + 2.0 * tf) * s2 * oracle_cyl_a(qab * ro);
                inner += m->poly_w[i] * F * F;
            }
            sum += m->orient_w[o] * inner;
        }
    } else if (m->kind == 11) {
        /* core-shell bicelle: a core cylinder (r, L, rho_core) closed on each
         * end face by a layer t_f thick of the core's radius (rho_face), the
         * whole wrapped in a rim t thick over the full length L + 2 t_f
         * (rho_rim = sld_shell). Nested cylinders C1 = (r, L),
         * C2 = (r, L + 2 t_f), C3 = (r + t, L + 2 t_f), so by Eq. 1
         *   F = (rho_c - rho_f) C1 + (rho_f - rho_r) C2 + (rho_r - rho_solv) C3,
         * C = pi R^2 H sinc(Q_C H/2) a(Q_AB R); normalised by <V(C3)>. The
         * core radius is polydisperse, t, t_f and L fixed. */
        double t = m->thickness, L = m->length, tf = m->thickness_face, Lo = L + 2.0 * tf;
        double dc = m->sld - m->sld_face, df = m->sld_face - m->sld_shell, dr = m->sld_shell - m->sld_solvent;
        for (int64_t i = 0; i < np; ++i) {
            double ro = m->poly_r[i] + t;
            vmean += m->poly_w[i] * PI * ro * ro * Lo;
        }
        for (int64_t o = 0; o < m->n_orient; ++o) {
            const double *c = m->orient_c + 3 * o;
            double qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2];
            double x0 = q[1] * c[2] - q[2] * c[1];
            double x1 = q[2] * c[0] - q[0] * c[2];
            double x2 = q[0] * c[1] - q[1] * c[0];
            double qab = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
            double s1 = oracle_sinc(0.5 * qc * L), s2 = oracle_sinc(0.5 * qc * Lo);
            double inner = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double r = m->poly_r[i], ro = r + t;
                double ar = oracle_cyl_a(qab * r), ao = oracle_cyl_a(qab * ro);
                double F = dc * PI * r * r * L * s1 * ar
                         + df * PI * r * r * Lo * s2 * ar
                         + dr * PI * ro * ro * Lo * s2 * ao;
                inner += m->poly_w[i] * F * F;
            }
            sum += m->orient_w[o] * inner;
        }
    } else if (m->kind == 10) {
        /* core-shell ellipsoid of revolution: core radii (r, r_p), the shell
         * adds t at the equator and t_p at the poles; by Eq. 1 with the
         * ellipsoid's amplitude f(x) = 3 (sin x - x cos x) / x^3,
         *   F = (rho_c - rho_s) V_c f(x_c) + (rho_s - rho_solv) V_o f(x_o),
         * x^2 = (Q_AB r_e)^2 + (Q_C r_p)^2 for the core and the outer
         * surface, V = 4/3 pi r_e^2 r_p; normalised by <V_o>. The core's
         * equatorial radius is polydisperse, r_p, t and t_p fixed. */
        double rp = m->radius_polar, t = m->thickness;
        double rpo = rp + m->thickness_face;
        for (int64_t i = 0; i < np; ++i) {
            double ro = m->poly_r[i] + t;
            vmean += m->poly_w[i] * 4.0 / 3.0 * PI * ro * ro * (rp + m->thickness_face);
        }
        for (int64_t o = 0; o < m->n_orient; ++o) {
            const double *c = m->orient_c + 3 * o;
            double qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2];
            double x0 = q[1] * c[2] - q[2] * c[1];
            double x1 = q[2] * c[0] - q[0] * c[2];
            double x2 = q[0] * c[1] - q[1] * c[0];
            double qab2 = x0 * x0 + x1 * x1 + x2 * x2;
            double inner = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double re = m->poly_r[i], ro = re + t;
                double Vc = 4.0 / 3.0 * PI * re * re * rp, Vo = 4.0 / 3.0 * PI * ro * ro * rpo;
                double xc = sqrt(re * re * qab2 + rp * rp * qc * qc);
                double xo = sqrt(ro * ro * qab2 + rpo * rpo * qc * qc);
                double F = (m->sld - m->sld_shell) * Vc * oracle_sphere_f(xc)
                         + (m->sld_shell - m->sld_solvent) * Vo * oracle_sphere_f(xo);
                inner += m->poly_w[i] * F * F;
            }
            sum += m->orient_w[o] * inner;
        }
    } else {                         /* ellipsoid of revolution: equatorial radius polydisperse */
        double drho = m->sld - m->sld_solvent;
        double rp = m->radius_polar;
        for (int64_t i = 0; i < np; ++i)
            vmean += m->poly_w[i] * 4.0 / 3.0 * PI * rp * m->poly_r[i] * m->poly_r[i];
        for (int64_t o = 0; o < m->n_orient; ++o) {
            const double *c = m->orient_c + 3 * o;
            double qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2];
            double x0 = q[1] * c[2] - q[2] * c[1];
            double x1 = q[2] * c[0] - q[0] * c[2];
            double x2 = q[0] * c[1] - q[1] * c[0];
            double qab2 = x0 * x0 + x1 * x1 + x2 * x2;
            double inner = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double re = m->poly_r[i];
                double V = 4.0 / 3.0 * PI * rp * re * re;
                double x = sqrt(re * re * qab2 + rp * rp * qc * qc);
                double F = drho * V * oracle_sphere_f(x);
                inner += m->poly_w[i] * F * F;
            }
            sum += m->orient_w[o] * inner;
        }
    }
    double S = 1.0;
    if (m->sq_kind == 1) S = oracle_sq_py(qq, m->sq_radius, m->sq_fraction);
    else if (m->sq_kind == 2) S = oracle_sq_table(m, qq);
    return m->volume_fraction / vmean * sum * S;
}

void oracle_dsigma_many(const oracle_model *m, const double *q, int64_t n, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_dsigma(m, q + 3 * i);
}

/* ------------------------------------------------- per-event sampling */

/* Inverse complementary error function on (0, 2): the x with erfc(x) = y,
 * by bisection on the monotone erfc to 1e-6 and Newton steps on
 * erfc(x) - y (derivative -2/sqrt(pi) exp(-x^2)) to full precision. */
double oracle_erfcinv(double y)
{
    if (!(y > 0.0 && y < 2.0)) return y <= 0.0 ? INFINITY : -INFINITY;
    double lo = -27.0, hi = 27.0;           /* erfc(lo) = 2, erfc(hi) = 0 to double range */
    while (hi - lo > 1e-6) {
        double mid = 0.5 * (lo + hi);
        if (erfc(mid) > y) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 8; ++it) {
        double f = erfc(x) - y;
        double d = -2.0 / sqrt(PI) * exp(-x * x);
        if (d == 0.0) break;
        double step = f / d;
        x -= step;
        if (fabs(step) <= 1e-16 * fabs(x)) break;
    }
    return x;
}

/* Polydisperse radius of one event: Gaussian N(R, (p R)^2) restricted to
 * R > 0 (Sec. II.B: non-positive draws are redrawn). The restricted law is
 * sampled by inversion, z = Phi^-1(lo + u (1 - lo)) with lo = Phi(-1/p) and
 * Phi^-1(v) = -sqrt(2) erfcinv(2 v); u and 1 - u are both exact, and the
 * upper half uses 1 - v = (1 - u)(1 - lo) so neither tail loses digits.  */
double oracle_event_radius(double R, double p, uint32_t x)
{
    if (p <= 0.0) return R;
    double lo = 0.5 * erfc(1.0 / (p * sqrt(2.0)));
    double u = u01(x), uc = u01c(x);
    double v = lo + u * (1.0 - lo), z;
    if (v < 0.5) z = -sqrt(2.0) * oracle_erfcinv(2.0 * v);
    else z = sqrt(2.0) * oracle_erfcinv(2.0 * uc * (1.0 - lo));
    return R * (1.0 + p * z);
}

/* Particle axis of one event from two uniforms (Sec. II.B): mode 1 uniform
 * on the sphere (cos theta = 1 - 2 u), mode 2 theta = pi u, phi = 2 pi u'. */
void oracle_event_axis(int64_t mode, double theta0, double phi0, uint32_t xa, uint32_t xb, double c[3])
{
    double ct, st;
    if (mode == 1) {
        ct = 1.0 - 2.0 * u01(xa);
        st = sqrt(fmax(0.0, 1.0 - ct * ct));
    } else if (mode == 2) {
        double th = PI * u01(xa);
        ct = cos(th); st = sin(th);
    } else {
        ct = cos(theta0); st = sin(theta0);
        c[0] = st * cos(phi0); c[1] = st * sin(phi0); c[2] = ct;
        return;
    }
    double ph = 2.0 * PI * u01(xb);
    c[0] = st * cos(ph); c[1] = st * sin(ph); c[2] = ct;
}

/* Particle frame (A, B, C) from the three angles (Sec. II.B): C along
 * (theta, phi), A and B the spherical unit vectors e_theta, e_phi of C
 * rotated by psi about C. */
void oracle_frame(double theta, double phi, double psi, double f[9])
{
    double st = sin(theta), ct = cos(theta), sp = sin(phi), cp = cos(phi);
    double sq = sin(psi), cq = cos(psi);
    double et[3] = {ct * cp, ct * sp, -st}, ep[3] = {-sp, cp, 0.0};
    for (int k = 0; k < 3; ++k) {
        f[k] = cq * et[k] + sq * ep[k];
        f[3 + k] = -sq * et[k] + cq * ep[k];
    }
    f[6] = st * cp; f[7] = st * sp; f[8] = ct;
}

/* Frame of one event for the particles without a symmetry axis: mode 1 a
 * uniform rotation (cos theta = 1 - 2u, phi, psi uniform), mode 2 the
 * angles uniform, theta ~ U[0, pi], phi, psi ~ U[0, 2 pi]; mode 0 the
 * fixed frame. */
void oracle_event_frame(int64_t mode, double theta0, double phi0, double psi0, uint32_t xa, uint32_t xb,
                        uint32_t xc, double f[9])
{
    if (mode == 0) { oracle_frame(theta0, phi0, psi0, f); return; }
    double th = mode == 1 ? acos(1.0 - 2.0 * u01(xa)) : PI * u01(xa);
    oracle_frame(th, 2.0 * PI * u01(xb), 2.0 * PI * u01(xc), f);
}

/* Volume of one particle of the polydisperse parameter r (the quantity the
 * cross section is normalised by through <V>). */
static double model_volume(const oracle_model *m, double r)
{
    if (m->kind == 0) return sphere_volume(r);
    if (m->kind == 1) return sphere_volume(r + m->thickness);
    if (m->kind == 2) return PI * r * r * m->length;
    if (m->kind == 4 || m->kind == 5) {
        double s = r / m->radius;
        return (m->kind == 4 ? 4.0 / 3.0 * PI : 8.0) * m->radius * m->radius_b * m->radius_polar * s * s * s;
    }
    if (m->kind == 12) {
        double s = r / m->radius;
        return PI * m->radius * m->radius_b * m->length * s * s * s;
    }
    if (m->kind == 13) {
        double s = r / m->radius, t = m->thickness;
        return 8.0 * (m->radius * m->radius_b * m->radius_polar -
                      (m->radius - t) * (m->radius_b - t) * (m->radius_polar - t)) * s * s * s;
    }
    if (m->kind == 8) {
        double ro = r + m->thickness;
        return PI * ro * ro * (m->length + 2.0 * m->thickness_face);
    }
    if (m->kind == 9) return PI * ((r + m->thickness) * (r + m->thickness) - r * r) * m->length;
    if (m->kind == 11)
        return PI * (r + m->thickness) * (r + m->thickness) * (m->length + 2.0 * m->thickness_face);
    if (m->kind == 10)
        return 4.0 / 3.0 * PI * (r + m->thickness) * (r + m->thickness) * (m->radius_polar + m->thickness_face);
    if (m->kind == 6 || m->kind == 7) {
        double s = r / m->radius, R = m->radius_polar, r0 = m->radius;
        double h = sqrt(fmax(R * R - r0 * r0, 0.0));
        double H = m->kind == 6 ? r0 * r0 / (R + h) : R + h;
        return (PI * r0 * r0 * m->length + 2.0 * PI * R * H * H * (1.0 - H / (3.0 * R))) * s * s * s;
    }
    return 4.0 / 3.0 * PI * m->radius_polar * r * r;
}

/* Per-event estimate of dSigma/dOmega(Q): (phi / <V>) |F(Q; r, c)|^2 S(Q)
 * for the radius r and axis c drawn from Philox block 2 of the history
 * (words: radius, axis polar, axis azimuth, rotation about the axis). <V> is the mean over
 * the radius distribution (the model's nodes). Its expectation over the
 * draws is the quadrature average of oracle_dsigma with matching nodes. */
double oracle_dsigma_event(const oracle_model *m, const double q[3], uint64_t seed,
                           uint32_t exp_id, uint64_t index)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c2[4] = {2u, exp_id, (uint32_t)index, (uint32_t)(index >> 32)};
    uint32_t x[4];
    oracle_philox4x32_10(c2, key, x);
    double r = oracle_event_radius(m->radius, m->poly, x[0]);
    double c[9];
    if (m->kind == 4 || m->kind == 5 || m->kind == 12 || m->kind == 13)
        oracle_event_frame(m->orient_mode, m->axis_theta, m->axis_phi, m->axis_psi, x[1], x[2], x[3], c);
    else
        oracle_event_axis(m->kind >= 2 ? m->orient_mode : 0, m->axis_theta, m->axis_phi, x[1], x[2], c);
    double one = 1.0;
    oracle_model single = *m;
    single.n_poly = 1; single.poly_r = &r; single.poly_w = &one;
    single.n_orient = 1; single.orient_c = c; single.orient_w = &one;
    double vmean = 0.0;
    for (int64_t i = 0; i < m->n_poly; ++i) vmean += m->poly_w[i] * model_volume(m, m->poly_r[i]);
    /* oracle_dsigma of the single node carries phi / V(r); rescale to phi / <V> */
    return oracle_dsigma(&single, q) * model_volume(m, r) / vmean;
}

void oracle_dsigma_event_many(const oracle_model *m, const double *q, uint64_t seed, uint32_t exp_id,
                              uint64_t first, int64_t n, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        out[i] = oracle_dsigma_event(m, q + 3 * i, seed, exp_id, first + (uint64_t)i);
}

/* ------------------------------------------- scattering attenuation */
/*
 * The particles remove neutrons from the beam at the rate of their total
 * scattering cross section per unit volume,
 *
 *   Sigma_s(lambda) = integral over all directions k_f of dSigma/dOmega(Q) dOmega,
 *   Q = k (k_f - k_i),  k = 2 pi / lambda,  k_i along the beam axis (+z).
 *
 * Parametrising k_f by |Q| and the azimuth phi about z:
 *   Q = (Q s cos phi, Q s sin phi, -Q^2 / (2 k)),  s = sqrt(1 - Q^2 / (4 k^2)),
 *   dOmega = Q dQ dphi / k^2,  0 <= Q <= 2k.
 *
 * The integral is taken by a fixed product rule, built once at the shortest
 * wavelength of the source (k_max) and scaled with k, so that Sigma_s is a
 * smooth function of lambda:
 *   - |Q| panels [a, b] from 0 to 2 k_max with b - a = max(pi / D, a / 8),
 *     D the largest extent of the particle over its polydisperse nodes (a
 *     panel is at most half a period of the amplitude's oscillation near
 *     the origin, and grows geometrically further out); the last panel ends
 *     at 2 k_max; 8 Gauss-Legendre nodes per panel;
 *   - phi: the midpoint rule with n_phi = 8 clamp(ceil(Q_mid D / 2), 2, 64)
 *     points on the panel (Q_mid its midpoint at k_max); one point for the
 *     sphere and the core-shell sphere, whose dSigma/dOmega depends on |Q|
 *     only.
 * In the trace, Sigma_s(lambda) over the source's wavelength band enters as
 * its interpolant at 8 Chebyshev points (one point without a spread).
 */

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n. */
static void gl_nodes(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Largest extent of the particle (angstrom) over its polydisperse nodes. */
double oracle_model_extent(const oracle_model *m)
{
    double r = 0.0;
    for (int64_t i = 0; i < m->n_poly; ++i) r = fmax(r, m->poly_r[i]);
    switch (m->kind) {
    case 0: return 2.0 * r;
    case 1: return 2.0 * (r + m->thickness);
    case 2: return sqrt(m->length * m->length + 4.0 * r * r);
    case 3: return 2.0 * fmax(r, m->radius_polar);
    case 4: {
        double f = r / m->radius;
        return 2.0 * f * fmax(m->radius, fmax(m->radius_b, m->radius_polar));
    }
    case 6:
    case 7: {   /* tip to tip along the axis, L + 2H, or the caps' diameter */
        double f = r / m->radius, R = m->radius_polar, r0 = m->radius;
        double h = sqrt(fmax(R * R - r0 * r0, 0.0));
        double H = m->kind == 6 ? r0 * r0 / (R + h) : R + h;
        return f * fmax(m->length + 2.0 * H, 2.0 * R);
    }
    case 8:
    case 11: {
        double lo = m->length + 2.0 * m->thickness_face, ro = r + m->thickness;
        return sqrt(lo * lo + 4.0 * ro * ro);
    }
    case 9: return sqrt(m->length * m->length + 4.0 * (r + m->thickness) * (r + m->thickness));
    case 10: return 2.0 * fmax(r + m->thickness, m->radius_polar + m->thickness_face);
    case 12: {
        double f = r / m->radius, a = fmax(m->radius, m->radius_b);
        return 2.0 * f * sqrt(a * a + 0.25 * m->length * m->length);
    }
    default: {
        double f = r / m->radius;
        return 2.0 * f * sqrt(m->radius * m->radius + m->radius_b * m->radius_b +
                              m->radius_polar * m->radius_polar);
    }
    }
}

/* Sigma_s(lambda) in 1/angstrom by the rule above (built at lambda_min):
 * the sum over the |Q| panels, or only panel `only` (>= 0); *n_pan gets the
 * number of panels. */
static double sigma_s_panels(const oracle_model *m, double lambda, double lambda_min, int only, int *n_pan)
{
    const double D = oracle_model_extent(m);
    const double kmax = 2.0 * PI / lambda_min, k = 2.0 * PI / lambda, sc = k / kmax;
    const int iso = m->kind == 0 || m->kind == 1;
    double gx[8], gw[8];
    gl_nodes(8, gx, gw);
    double total = 0.0, a = 0.0;
    int idx = 0;
    while (a < 2.0 * kmax) {
        double b = a + fmax(PI / D, a / 8.0);
        if (b > 2.0 * kmax) b = 2.0 * kmax;
        int nphi = 1;
        if (!iso) {
            double c = ceil(0.5 * (a + b) * D / 2.0);
            nphi = 8 * (int)fmin(fmax(c, 2.0), 64.0);
        }
        if (only < 0 || idx == only) {
            double panel = 0.0;
            for (int g = 0; g < 8; ++g) {
                double Q = sc * (0.5 * (a + b) + 0.5 * (b - a) * gx[g]);
                double wq = sc * 0.5 * (b - a) * gw[g];
                double st = sqrt(fmax(1.0 - Q * Q / (4.0 * k * k), 0.0));
                double qz = -Q * Q / (2.0 * k);
                double ring = 0.0;
#pragma omp parallel for reduction(+ : ring) schedule(static) if (nphi >= 64)
                for (int j = 0; j < nphi; ++j) {
                    double ph = 2.0 * PI * (j + 0.5) / nphi;
                    double q[3] = {Q * st * cos(ph), Q * st * sin(ph), qz};
                    ring += oracle_dsigma(m, q);
                }
                panel += wq * Q * ring * (2.0 * PI / nphi);
            }
            total += panel;
        }
        a = b;
        ++idx;
    }
    *n_pan = idx;
    return total / (k * k);
}

double oracle_sigma_s(const oracle_model *m, double lambda, double lambda_min)
{
    int n;
    return sigma_s_panels(m, lambda, lambda_min, -1, &n);
}

/* The share of panel i in Sigma_s(lambda) (NAN if there is no panel i). */
double oracle_sigma_s_panel(const oracle_model *m, double lambda, double lambda_min, int i)
{
    int n;
    double v = sigma_s_panels(m, lambda, lambda_min, i, &n);
    return (i >= 0 && i < n) ? v : NAN;
}

/* Number of |Q| panels of the rule built at lambda_min. */
int oracle_sigma_s_npanels(const oracle_model *m, double lambda_min)
{
    int n;
    sigma_s_panels(m, lambda_min, lambda_min, 1 << 30, &n);
    return n;
}

/* The trace's attenuation table: mu_s(lambda) = 1e10 Sigma_s(lambda) in 1/m
 * at n Chebyshev points of [lmin, lmax] and the coefficients of its
 * interpolant sum_j c_j T_j(t), t = (2 lambda - lmin - lmax) / (lmax - lmin). */
typedef struct {
    int n;
    double lmin, lmax;
    double lam[8], mu[8], c[8];
} oracle_att;

static void att_setup(const oracle_instrument *in, const oracle_model *m, oracle_att *a)
{
    a->n = 0;
    if (!m || !m->self_att) return;
    a->lmin = in->lambda0 * (1.0 - in->dlambda_rel);
    a->lmax = in->lambda0 * (1.0 + in->dlambda_rel);
    const int n = in->dlambda_rel > 0.0 ? 8 : 1;
    a->n = n;
    for (int j = 0; j < n; ++j) {
        double t = cos(PI * (j + 0.5) / n);
        a->lam[j] = n > 1 ? 0.5 * (a->lmin + a->lmax) + 0.5 * (a->lmax - a->lmin) * t : in->lambda0;
        a->mu[j] = 1e10 * oracle_sigma_s(m, a->lam[j], a->lmin);
    }
    for (int i = 0; i < n; ++i) {
        double c = 0.0;
        for (int j = 0; j < n; ++j) c += a->mu[j] * cos(PI * i * (j + 0.5) / n);
        a->c[i] = (i == 0 ? 1.0 : 2.0) * c / n;
    }
}

/* mu_s(lambda) in 1/m from the table: T_j(t) = cos(j arccos t). */
static double att_mu(const oracle_att *a, double lambda)
{
    if (!a || a->n == 0) return 0.0;
    if (a->n == 1) return a->c[0];
    double t = (2.0 * lambda - a->lmin - a->lmax) / (a->lmax - a->lmin);
    t = fmin(fmax(t, -1.0), 1.0);
    double th = acos(t), v = 0.0;
    for (int j = 0; j < a->n; ++j) v += a->c[j] * cos(j * th);
    return v;
}

/* Exposes the table: lam, mu (1/m) and c, each [8]; returns n (0: off). */
int oracle_att_table(const oracle_instrument *in, const oracle_model *m, double *lam, double *mu,
                     double *c)
{
    oracle_att a;
    att_setup(in, m, &a);
    for (int j = 0; j < a.n; ++j) { lam[j] = a.lam[j]; mu[j] = a.mu[j]; c[j] = a.c[j]; }
    return a.n;
}

/* mu_s at the wavelengths lam[n] from the table (1/m). */
void oracle_att_eval(const oracle_instrument *in, const oracle_model *m, const double *lam, int64_t n,
                     double *out)
{
    oracle_att a;
    att_setup(in, m, &a);
    for (int64_t i = 0; i < n; ++i) out[i] = att_mu(&a, lam[i]);
}

/* ------------------------------------------------------------- geometry */

/* source wavelength from one uniform: triangular on [l0 (1-d), l0 (1+d)],
 * mode l0, by inverse cumulative distribution */
double oracle_sample_lambda(double lambda0, double drel, double u)
{
    double T = (u < 0.5) ? sqrt(2.0 * u) - 1.0 : 1.0 - sqrt(2.0 * (1.0 - u));
    return lambda0 * (1.0 + drel * T);
}

/* entry and exit ray parameters of the sample box |x|<=hx, |y|<=hy, 0<=z<=t.
 * Returns 0 on a miss. */
static int slab(const oracle_instrument *in, const double o[3], const double d[3],
                double *t_in, double *t_out)
{
    double lo[3] = {-in->sample_half_x, -in->sample_half_y, 0.0};
    double hi[3] = {in->sample_half_x, in->sample_half_y, in->sample_thickness};
    double a = -INFINITY, b = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < lo[k] || o[k] > hi[k]) return 0;
            continue;
        }
        double t1 = (lo[k] - o[k]) / d[k], t2 = (hi[k] - o[k]) / d[k];
        if (t1 > t2) { double s = t1; t1 = t2; t2 = s; }
        if (t1 > a) a = t1;
        if (t2 < b) b = t2;
    }
    if (a < 0.0) a = 0.0;
    if (b <= a) return 0;
    *t_in = a; *t_out = b;
    return 1;
}

/* Geometry of one neutron history (everything but the cross section).
 * Returns 1 if it scattered onto the detector, with its pixel, the path
 * length l in the sample, the solid-angle factor, the attenuation and Q;
 * *w_trans gets the unscattered (transmitted) weight. */
static int history_geometry(const oracle_instrument *in, const oracle_att *att, uint64_t seed,
                            uint32_t exp_id, uint64_t index, int64_t *pixel, double *l_path,
                            double *d_omega, double *atten, double q_out[3], double *w_trans)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c0[4] = {0u, exp_id, (uint32_t)index, (uint32_t)(index >> 32)};
    uint32_t c1[4] = {1u, exp_id, (uint32_t)index, (uint32_t)(index >> 32)};
    uint32_t x[8];
    oracle_philox4x32_10(c0, key, x);
    oracle_philox4x32_10(c1, key, x + 4);

    /* source: triangular wavelength spread by inverse CDF */
    double lambda = oracle_sample_lambda(in->lambda0, in->dlambda_rel, u01(x[0]));
    /* attenuation: the instrument's mu plus, optionally, the particles' own scattering */
    const double mu = in->mu + att_mu(att, lambda);
    /* collimation: uniform points on the two pinhole discs */
    double r1 = in->ap1_radius * sqrt(u01(x[1])), f1 = 2.0 * PI * u01(x[2]);
    double r2 = in->ap2_radius * sqrt(u01(x[3])), f2 = 2.0 * PI * u01(x[4]);
    double p1[3] = {r1 * cos(f1), r1 * sin(f1), in->ap1_z};
    double p2[3] = {r2 * cos(f2), r2 * sin(f2), in->ap2_z};
    double d[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double k_in[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    /* sample */
    double t_in, t_out;
    if (!slab(in, p2, k_in, &t_in, &t_out)) { *w_trans = 1.0; return 0; }
    double l = t_out - t_in;
    *w_trans = exp(-mu * l);
    double s = u01(x[5]) * l;
    double ps[3] = {p2[0] + (t_in + s) * k_in[0], p2[1] + (t_in + s) * k_in[1],
                    p2[2] + (t_in + s) * k_in[2]};
    /* detector point: pixel from the integer draw, position inside it from the remainder */
    uint64_t mx = (uint64_t)(x[6] >> 9) * (uint64_t)in->nx;
    uint64_t my = (uint64_t)(x[7] >> 9) * (uint64_t)in->ny;
    int64_t ix = (int64_t)(mx >> 23), iy = (int64_t)(my >> 23);
    double fx = ((double)(mx & 0x7FFFFF) + 0.5) / 8388608.0;
    double fy = ((double)(my & 0x7FFFFF) + 0.5) / 8388608.0;
    double pd[3] = {((double)ix + fx) * in->pixel_x - 0.5 * (double)in->nx * in->pixel_x,
                    ((double)iy + fy) * in->pixel_y - 0.5 * (double)in->ny * in->pixel_y,
                    in->det_distance};
    double v[3] = {pd[0] - ps[0], pd[1] - ps[1], pd[2] - ps[2]};
    double rr = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double k_out[3] = {v[0] / rr, v[1] / rr, v[2] / rr};
    /* solid-angle factor of the area-uniform detector point */
    double area = (double)in->nx * in->pixel_x * (double)in->ny * in->pixel_y;
    double domega = area * k_out[2] / (rr * rr);
    /* scattering vector Q = k_f - k_i in 1/angstrom */
    double k = 2.0 * PI / lambda;
    q_out[0] = k * (k_out[0] - k_in[0]);
    q_out[1] = k * (k_out[1] - k_in[1]);
    q_out[2] = k * (k_out[2] - k_in[2]);
    /* path to the exit of the sample along the scattered direction */
    double e_in, e_out, l_out = 0.0;
    if (slab(in, ps, k_out, &e_in, &e_out)) l_out = e_out - e_in;
    *atten = exp(-mu * (s + l_out));
    *l_path = l;
    *d_omega = domega;
    *pixel = iy * in->nx + ix;
    return 1;
}

/* One neutron history. Returns 1 if it scattered onto the detector, with
 * its pixel and weight l dSigma/dOmega(Q) dOmega att; *w_trans gets the
 * unscattered (transmitted) weight. */
static int history_att(const oracle_instrument *in, const oracle_model *m, const oracle_att *at,
                       uint64_t seed, uint32_t exp_id, uint64_t index, int64_t *pixel, double *w,
                       double *w_trans)
{
    double l, domega, att, q[3];
    if (!history_geometry(in, at, seed, exp_id, index, pixel, &l, &domega, &att, q, w_trans)) return 0;
    double ds = (m->event ? oracle_dsigma_event(m, q, seed, exp_id, index) : oracle_dsigma(m, q))
              * 1e10; /* 1/angstrom -> 1/m */
    *w = l * ds * domega * att;
    return 1;
}

int oracle_history(const oracle_instrument *in, const oracle_model *m, uint64_t seed,
                   uint32_t exp_id, uint64_t index, int64_t *pixel, double *w,
                   double *w_trans)
{
    oracle_att a;
    att_setup(in, m, &a);
    return history_att(in, m, &a, seed, exp_id, index, pixel, w, w_trans);
}

/* Per-neutron geometry records: pixel (-1 on a miss), Q [n][3], the
 * prefactor l dOmega att (1/m per 1/angstrom of cross section, so that the
 * weight is prefactor * dSigma/dOmega(Q) with dSigma/dOmega in 1/angstrom)
 * and the transmitted weight. Lets a test weight the histories with a cross
 * section of its own. */
void oracle_geometry_records(const oracle_instrument *in, uint64_t seed, uint32_t exp_id,
                             uint64_t first, uint64_t n, int64_t *pixel, double *q,
                             double *pref, double *w_trans)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)n; ++j) {
        int64_t pix; double l, domega, att;
        if (history_geometry(in, NULL, seed, exp_id, first + (uint64_t)j, &pix, &l, &domega, &att,
                             q + 3 * j, w_trans + j)) {
            pixel[j] = pix;
            pref[j] = l * 1e10 * domega * att;
        } else {
            pixel[j] = -1;
            pref[j] = 0.0;
            q[3 * j] = q[3 * j + 1] = q[3 * j + 2] = 0.0;
        }
    }
}

/* Trace neutrons [first, first+n) and accumulate the detector in place.
 * sum_w, sum_w2: [ny*nx] doubles; count: [ny*nx] uint64; trans: scalar. */
void oracle_trace(const oracle_instrument *in, const oracle_model *m, uint64_t seed,
                  uint32_t exp_id, uint64_t first, uint64_t n, double *sum_w,
                  double *sum_w2, uint64_t *count, double *trans, int threads)
{
    int64_t npix = in->nx * in->ny;
    int nt = 1;
#ifdef _OPENMP
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
    double *pw = calloc((size_t)nt * npix, sizeof(double));
    double *pw2 = calloc((size_t)nt * npix, sizeof(double));
    uint64_t *pc = calloc((size_t)nt * npix, sizeof(uint64_t));
    double *pt = calloc((size_t)nt, sizeof(double));
    oracle_att at;
    att_setup(in, m, &at);
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *w1 = pw + (size_t)tid * npix, *w2 = pw2 + (size_t)tid * npix;
        uint64_t *c = pc + (size_t)tid * npix;
        double tr = 0.0;
#pragma omp for schedule(static)
        for (int64_t j = 0; j < (int64_t)n; ++j) {
            int64_t pix; double w, wt;
            if (history_att(in, m, &at, seed, exp_id, first + (uint64_t)j, &pix, &w, &wt)) {
                w1[pix] += w; w2[pix] += w * w; c[pix] += 1;
            }
            tr += wt;
        }
        pt[tid] = tr;
    }
    for (int t = 0; t < nt; ++t) {
        for (int64_t p = 0; p < npix; ++p) {
            sum_w[p] += pw[(size_t)t * npix + p];
            sum_w2[p] += pw2[(size_t)t * npix + p];
            count[p] += pc[(size_t)t * npix + p];
        }
        *trans += pt[t];
    }
    free(pw); free(pw2); free(pc); free(pt);
}

/* Per-neutron records for brute-force comparisons: pixel (-1 on a miss), weight. */
void oracle_records(const oracle_instrument *in, const oracle_model *m, uint64_t seed,
                    uint32_t exp_id, uint64_t first, uint64_t n, int64_t *pixel, double *w)
{
    oracle_att at;
    att_setup(in, m, &at);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)n; ++j) {
        int64_t pix; double ww, wt;
        if (history_att(in, m, &at, seed, exp_id, first + (uint64_t)j, &pix, &ww, &wt)) {
            pixel[j] = pix; w[j] = ww;
        } else {
            pixel[j] = -1; w[j] = 0.0;
        }
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
