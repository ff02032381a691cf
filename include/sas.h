/*
 * sas.h -- C ABI of the GB300 SANS Monte Carlo trace library (libsas.so).
 *
 * One neutron history (Sec. II.A, instrument chain; single scattering,
 * Sec. I): a neutron is drawn from the source (wavelength with a triangular
 * spread), passes two pinholes (collimation), enters the sample slab, is
 * split into a transmitted weight and a scattered branch, gets a scattering
 * vector Q toward an area-uniform point of the 2D position-sensitive detector
 * and the weight  l * dSigma/dOmega(Q) * dOmega,  where
 *
 *   dSigma/dOmega(Q) = (phi / <V>) <|F(Q)|^2> S(Q),   F = drho V f(Q)
 *
 * follows Eqs. (1)-(4) (amplitude, intensity, dilute-limit intensity
 * n drho^2 V^2 P S, model A*A/V), Eq. (7) (uniaxial particles: F depends on
 * Q_AB and Q_C) and Eq. (8) (cylinder). <.> averages over the polydispersity
 * distribution and, for uniaxial particles, the orientation distribution
 * (Sec. II.B). The weight is tallied on the detector pixel.
 *
 * Conventions for every entry point:
 *  - Return SAS_OK or an error code; nothing aborts or prints. The text of
 *    the last error of the calling thread is in sas_last_error().
 *  - Units: instrument lengths in m, wavelength and particle sizes in
 *    angstrom, SLD in 1/angstrom^2, angles in rad, Q in 1/angstrom,
 *    dSigma/dOmega in 1/angstrom (model evaluation) or 1/m (trace weights).
 *    The beam runs along +z; the sample front face is the plane z = 0.
 *  - Device memory of an experiment or a batch is owned by the library.
 *    Host buffers passed in are owned by the caller, who states their length.
 *  - "stream" arguments are cudaStream_t values passed as void* (NULL: the
 *    legacy default stream). Work is enqueued asynchronously on the stream;
 *    the sas_read_* calls synchronise it.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *    key = (seed low 32 bits, seed high 32 bits) and counter =
 *    (draw block, experiment id, neutron index low, neutron index high).
 *    A neutron's history depends only on (seed, experiment id, index), so
 *    any split of an index range into sub-ranges gives the same histories.
 */
#ifndef SAS_H
#define SAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sas_status {
    SAS_OK = 0,
    SAS_ERR_ARG = 1,         /* invalid argument, size mismatch, NULL pointer */
    SAS_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    SAS_ERR_OOM = 3,         /* device allocation failed */
    SAS_ERR_STATE = 4,       /* call out of order (e.g. trace before set_model) */
    SAS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    SAS_ERR_OUT_OF_BOX = 6,  /* surrogate input outside its training box */
    SAS_ERR_NUMERIC = 7      /* non-finite value detected */
} sas_status;

enum { SAS_SPHERE = 0, SAS_CORE_SHELL = 1, SAS_CYLINDER = 2, SAS_ELLIPSOID = 3,
       /* no symmetry axis (Sec. II.B): sizes along the particle axes A, B, C */
       SAS_TRIAXIAL_ELLIPSOID = 4, SAS_PARALLELEPIPED = 5,
       /* cylinders with spherical end caps (Sec. III: the expensive models) */
       SAS_CAPPED_CYLINDER = 6, SAS_BARBELL = 7,
       /* shelled uniaxial models (the cylinder and ellipsoid groups of Sec. II.B) */
       SAS_CORE_SHELL_CYLINDER = 8, SAS_HOLLOW_CYLINDER = 9, SAS_CORE_SHELL_ELLIPSOID = 10,
       SAS_CORE_SHELL_BICELLE = 11,
       /* no symmetry axis (Sec. II.B, the ellipsoid and parallelepiped groups) */
       SAS_ELLIPTICAL_CYLINDER = 12, SAS_HOLLOW_RECTANGULAR_PRISM = 13,
       /* shape-independent laws of |Q| (the isotropic group G) */
       SAS_SHAPE_INDEPENDENT = 14 };
/* sas_model_desc.function of SAS_SHAPE_INDEPENDENT */
enum { SAS_FN_GUINIER = 0, SAS_FN_GAUSS_COIL = 1, SAS_FN_LORENTZ = 2, SAS_FN_DAB = 3, SAS_FN_POWER_LAW = 4,
       SAS_FN_GAUSS_PEAK = 5, SAS_FN_TEUBNER_STREY = 6, SAS_FN_PEAK_LORENTZ = 7, SAS_FN_TWO_POWER_LAW = 8,
       SAS_FN_GUINIER_POROD = 9, SAS_FN_GAUSS_LORENTZ_GEL = 10, SAS_FN_POLY_GAUSS_COIL = 11,
       SAS_FN_STAR_POLYMER = 12, SAS_FN_MASS_FRACTAL = 13, SAS_FN_FRACTAL = 14, SAS_FN_SPINODAL = 15,
       SAS_FN_POLYMER_EXCL_VOLUME = 16, SAS_FN_LINEAR_PEARLS = 17 };
/* largest Gauss-Legendre rule over an end cap */
#define SAS_MAX_CAP_NODES 64
enum { SAS_SQ_NONE = 0, SAS_SQ_HARD_SPHERE_PY = 1, SAS_SQ_HAYTER_MSA = 2 };
enum { SAS_FP32 = 0, SAS_FP64 = 1 };
/* sampling: average every history over the quadrature nodes, or draw one
 * polydisperse radius and one particle axis per history (the paper's
 * per-event estimator, Sec. II.B) */
enum { SAS_QUADRATURE = 0, SAS_PER_EVENT = 1 };
/* law of the polydisperse radius: Schulz, or the Gaussian of Sec. II.B
 * restricted to positive radii */
enum { SAS_POLY_SCHULZ = 0, SAS_POLY_GAUSSIAN = 1 };
/* largest cylinder radial table (points; 64 KB of FP32 values) */
#define SAS_MAX_RADIAL_TABLE 8192

/* Instrument (Sec. II.A: source, collimation, sample, 2D PSD). */
typedef struct sas_instrument {
    double lambda0;          /* mean wavelength, angstrom */
    double dlambda_rel;      /* half width of the triangular spread / lambda0 */
    double ap1_radius;       /* first pinhole radius, m */
    double ap1_z;            /* first pinhole plane, m (< ap2_z) */
    double ap2_radius;       /* second pinhole radius, m */
    double ap2_z;            /* second pinhole plane, m (<= 0) */
    double sample_half_x;    /* sample slab |x| <= half_x, m */
    double sample_half_y;    /* sample slab |y| <= half_y, m */
    double sample_thickness; /* slab 0 <= z <= thickness, m */
    double mu;               /* attenuation coefficient inside the sample, 1/m */
    double det_distance;     /* detector plane z, m */
    double pixel_x;          /* pixel pitch in x, m */
    double pixel_y;          /* pixel pitch in y, m */
    int64_t nx;              /* pixels in x (1..4096) */
    int64_t ny;              /* pixels in y (1..4096); pixel index = iy * nx + ix */
} sas_instrument;

/* Sample model (Eqs. 1-4, 7, 8; polydispersity and orientation Sec. II.B). */
typedef struct sas_model_desc {
    int64_t kind;            /* SAS_SPHERE, SAS_CORE_SHELL, SAS_CYLINDER, SAS_ELLIPSOID,
                                SAS_TRIAXIAL_ELLIPSOID, SAS_PARALLELEPIPED, SAS_CAPPED_CYLINDER,
                                SAS_BARBELL, SAS_CORE_SHELL_CYLINDER, SAS_HOLLOW_CYLINDER,
                                SAS_CORE_SHELL_ELLIPSOID, SAS_CORE_SHELL_BICELLE,
                                SAS_ELLIPTICAL_CYLINDER, SAS_HOLLOW_RECTANGULAR_PRISM,
                                SAS_SHAPE_INDEPENDENT */
    int64_t sq_kind;         /* SAS_SQ_NONE, SAS_SQ_HARD_SPHERE_PY or SAS_SQ_HAYTER_MSA */
    int64_t precision;       /* SAS_FP32 (tallies FP32 Kahan + FP64 reduction) or SAS_FP64 */
    int64_t n_poly;          /* Schulz nodes of the polydisperse radius (1..64) */
    int64_t n_gamma;         /* orientation nodes in the polar angle about the axis (1..128) */
    int64_t n_psi;           /* orientation nodes in the azimuth about the axis (1..128) */
    int64_t isotropic;       /* axis law of the uniaxial models: 0 Gaussian cap about the mean
                                axis (width sigma_orient), 1 uniform on the sphere, 2 uniform in
                                the angles, theta ~ U[0, pi], phi ~ U[0, 2 pi] (Sec. II.B) */
    double radius;           /* sphere R; core radius; cylinder R; ellipsoid equatorial R */
    double thickness;        /* core-shell shell thickness */
    double length;           /* cylinder length L */
    double radius_polar;     /* ellipsoid polar radius (along the axis) */
    double sld;              /* particle (core) scattering length density */
    double sld_shell;        /* core-shell shell SLD */
    double sld_solvent;      /* solvent SLD */
    double volume_fraction;  /* phi */
    double poly;             /* sigma / mean of the polydisperse radius (0: none) */
    double sigma_orient;     /* Gaussian width of the axis about its mean, rad */
    double axis_theta;       /* mean axis polar angle from +z, rad */
    double axis_phi;         /* mean axis azimuth, rad */
    double sq_radius;        /* hard-sphere (effective) radius of S(Q), angstrom */
    double sq_fraction;      /* volume fraction of S(Q) */
    int64_t sampling;        /* SAS_QUADRATURE or SAS_PER_EVENT. Per-event histories draw the
                                radius from the Gaussian law (poly_dist must be SAS_POLY_GAUSSIAN
                                unless poly = 0) by inversion of its distribution function, and
                                the axis uniformly (isotropic 1 or 2; or fixed: sigma_orient 0),
                                from Philox block 2 of the history; dSigma/dOmega is then
                                (phi / <V>) |F(Q; r, axis)|^2 S(Q), whose mean over the draws is
                                the quadrature average over the same laws. */
    int64_t poly_dist;       /* SAS_POLY_SCHULZ or SAS_POLY_GAUSSIAN */
    int64_t radial_table;    /* cylinder quadrature only: 1 replaces the polydisperse radial sum of
                                every orientation node by the interpolated table
                                G(x) = sum_i w_i t_i^4 [2 J1(x t_i)/(x t_i)]^2, x = Q_AB rbar,
                                t_i = r_i / rbar (built in FP64 per model up to the instrument's
                                largest |Q|, grid doubled until the cubic Hermite error is at
                                most 1e-7 G(0), 1e-13 for FP64 models; at most
                                SAS_MAX_RADIAL_TABLE points, else the direct sum is kept);
                                0 sums over the radius nodes */
    /* The 3-axis kinds: triaxial ellipsoid with semi-axes (radius, radius_b,
     * radius_polar) along (A, B, C), F = drho V f(|(a Q_A, b Q_B, c Q_C)|),
     * V = 4/3 pi a b c; rectangular parallelepiped with half-edges (radius,
     * radius_b, radius_polar), F = drho V sinc(a Q_A) sinc(b Q_B) sinc(c Q_C),
     * V = 8 a b c (Eq. 1 for both bodies). The frame: C along (axis_theta,
     * axis_phi), A and B rotated by axis_psi about C. Orientation laws as
     * for the uniaxial kinds (isotropic 0: the C axis in the Gaussian cap,
     * the mean frame carried along; 1: uniform rotations; 2: theta, phi and
     * psi uniform), with n_rot nodes in psi. The polydisperse factor
     * radius_i / radius scales all three sizes. Two more bodies use the
     * same frames: the elliptical cylinder, cross-section semi-axes
     * (radius, radius_b) along (A, B) and `length` L along C,
     * F = drho V sinc(Q_C L/2) 2 J1(x)/x, x = |(a Q_A, b Q_B)|, V = pi a b L;
     * the hollow rectangular prism, half-edges (radius, radius_b,
     * radius_polar) with walls `thickness` t thick (0 < t < every
     * half-edge), F = drho [8 a b c sinc(a Q_A) sinc(b Q_B) sinc(c Q_C) - the
     * same for the inner half-edges (a - t, b - t, c - t)], normalised by
     * the wall volume. */
    double radius_b;         /* 3-axis kinds: size along B */
    double axis_psi;         /* 3-axis kinds: rotation of the frame about C, rad */
    int64_t n_rot;           /* 3-axis kinds: quadrature nodes in psi (1..128) */
    /* Attenuation by the particles' own scattering (single scattering: a
     * neutron that would scatter twice is lost, not redistributed). 1: the
     * beam inside the sample is attenuated with mu + mu_s(lambda), where
     * mu_s = Sigma_s = the model's dSigma/dOmega integrated over all
     * directions for a neutron along +z (in 1/m), on the way to the
     * scattering point and out of the sample; the transmitted weight too.
     * Sigma_s is taken on the GPU when the model is set, by a fixed
     * (|Q|, phi) product rule (8-node Gauss-Legendre |Q| panels of width
     * max(pi / D, Q / 8), D the particle's largest extent; midpoint rule in
     * phi), at the 8 Chebyshev wavelengths of the source band, and
     * interpolated per history. Quadrature sampling only; 0: off. */
    int64_t self_attenuation;
    /* Capped cylinder and barbell: a cylinder of radius `radius` and length
     * `length` (>= 0) along the axis, closed by two spherical caps of radius
     * R = `radius_polar` >= radius: the parts of two spheres beyond the end
     * faces, their centres h = sqrt(R^2 - r^2) inside the cylinder (capped
     * cylinder; caps H = R - h high) or outside it (barbell; H = R + h).
     * Eq. 1 summed over disk slices normal to the axis:
     *   F = drho [pi r^2 L sinc(Q_C L / 2) 2 J1(Q_AB r) / (Q_AB r)
     *      + sum_j c_j cos(Q_C z_j) 2 J1(Q_AB rho_j) / (Q_AB rho_j)],
     * over the n_cap Gauss-Legendre slices of a cap at depth R u_j below its
     * tip, u_j in [0, H / R]: z_j = L / 2 + H - R u_j,
     * rho_j^2 = R^2 u_j (2 - u_j), c_j = 2 pi R^3 w_j u_j (2 - u_j);
     * V = pi r^2 L + 2 pi R H^2 (1 - H / 3R). The polydisperse factor
     * radius_i / radius scales r, R and L alike. Axis laws as for the
     * cylinder; quadrature sampling only; radial_table does not apply. */
    int64_t n_cap;           /* slices per cap (1..SAS_MAX_CAP_NODES); other kinds ignore it */
    /* Shelled uniaxial kinds (Eq. 1 region by region; the core radius
     * `radius` is polydisperse, the other sizes fixed; a(x) = 2 J1(x)/x,
     * f(x) = 3 (sin x - x cos x) / x^3):
     * - core-shell cylinder: core (radius r, length L, sld) in a shell
     *   (sld_shell) `thickness` t thick around it and `thickness_face` t_f
     *   on each end face; F = (sld - sld_shell) pi r^2 L sinc(Q_C L/2) a(Q_AB r)
     *   + (sld_shell - sld_solvent) V_o sinc(Q_C (L/2 + t_f)) a(Q_AB (r + t)),
     *   V_o = pi (r + t)^2 (L + 2 t_f), normalised by <V_o>;
     * - hollow cylinder: a tube of wall material (sld) between r and r + t
     *   over the length L with solvent inside; F = (sld - sld_solvent)
     *   sinc(Q_C L/2) [pi (r + t)^2 L a(Q_AB (r + t)) - pi r^2 L a(Q_AB r)],
     *   normalised by the wall volume <pi ((r + t)^2 - r^2) L>;
     * - core-shell ellipsoid of revolution: core radii (r, radius_polar r_p),
     *   shell t at the equator and t_f at the poles; F = (sld - sld_shell)
     *   V_c f(x_c) + (sld_shell - sld_solvent) V_o f(x_o), x^2 = (Q_AB r_e)^2
     *   + (Q_C r_p)^2 for the core and the outer surface, V = 4/3 pi r_e^2 r_p,
     *   normalised by <V_o>;
     * - core-shell bicelle: core (r, L, sld) closed on each end face by a
     *   layer `thickness_face` t_f thick of the core's radius (sld_face), the
     *   whole wrapped in a rim `thickness` t thick over L + 2 t_f
     *   (sld_shell); with the nested cylinders C(R, H) = pi R^2 H
     *   sinc(Q_C H/2) a(Q_AB R): F = (sld - sld_face) C(r, L) + (sld_face -
     *   sld_shell) C(r, L + 2 t_f) + (sld_shell - sld_solvent) C(r + t, L + 2 t_f),
     *   normalised by <pi (r + t)^2 (L + 2 t_f)>. */
    double thickness_face;   /* core-shell cylinder, bicelle: face layer; core-shell ellipsoid: polar shell (>= 0) */
    double sld_face;         /* core-shell bicelle: SLD of the face layers */
    /* Shape-independent laws: dSigma/dOmega(Q) = f_scale f(|Q|) in
     * 1/angstrom (no particle, no S(Q), no orientation or size average;
     * quadrature sampling, no self-attenuation), f by `function`:
     *   SAS_FN_GUINIER        exp(-Q^2 Rg^2 / 3)                   f_p0 = Rg > 0
     *   SAS_FN_GAUSS_COIL     2 (exp(-u) - 1 + u) / u^2, u = (Q Rg)^2  f_p0 = Rg > 0
     *   SAS_FN_LORENTZ        1 / (1 + (Q xi)^2)                   f_p0 = xi > 0
     *   SAS_FN_DAB            1 / (1 + (Q xi)^2)^2                 f_p0 = xi > 0
     *   SAS_FN_POWER_LAW      Q^-m                                 f_p0 = m
     *   SAS_FN_GAUSS_PEAK     exp(-(Q - Q0)^2 / (2 sigma^2))       f_p0 = Q0, f_p1 = sigma > 0
     *   SAS_FN_TEUBNER_STREY  1 / (a2 + c1 Q^2 + c2 Q^4)           f_p0 = a2 > 0, f_p1 = c1,
     *                         f_p2 = c2 >= 0, positive for every Q (c1 >= 0 or c1^2 < 4 a2 c2)
     *   SAS_FN_PEAK_LORENTZ   1 / (1 + ((Q - Q0) / B)^2)           f_p0 = Q0, f_p1 = B > 0
     *   SAS_FN_TWO_POWER_LAW  Q^-m1 for Q <= Qc, Qc^(m2 - m1) Q^-m2 above
     *                                                              f_p0 = Qc > 0, f_p1 = m1, f_p2 = m2
     *   SAS_FN_GUINIER_POROD  Q^-s exp(-Q^2 Rg^2 / (3 - s)) for Q <= Q1, D Q^-m above, with
     *                         Q1 = sqrt((m - s)(3 - s) / 2) / Rg and D joining value and slope
     *                                                              f_p0 = Rg > 0, f_p1 = s in [0, 3),
     *                                                              f_p2 = m > s
     *   SAS_FN_GAUSS_LORENTZ_GEL  exp(-Q^2 Xi^2 / 2) + r / (1 + (Q xi)^2)
     *                                                              f_p0 = Xi > 0, f_p1 = xi > 0, f_p2 = r >= 0
     *   SAS_FN_POLY_GAUSS_COIL  Schulz-Zimm polydisperse coil: 2 ((1 + U x)^(-1/U) + x - 1) /
     *                         ((1 + U) x^2), x = (Q Rg)^2 / (1 + 2U), Rg the z-average
     *                                                              f_p0 = Rg > 0, f_p1 = U = Mw/Mn - 1 >= 0
     *   SAS_FN_STAR_POLYMER   star of f Gaussian arms: (D(v) + (f - 1) g(v)^2) / f, D Debye's
     *                         function, g(v) = (1 - exp(-v)) / v, v = (Q Rg)^2 f / (3f - 2)
     *                                                              f_p0 = Rg (of the star) > 0, f_p1 = f >= 1
     *   SAS_FN_MASS_FRACTAL   spheres of radius R in a mass fractal of dimension D and cutoff xi:
     *                         P(Q R) M(Q xi; D), P(x) = (3 (sin x - x cos x) / x^3)^2 (1 at R = 0),
     *                         M(y; D) = sin((D - 1) atan y) / ((D - 1) y (1 + y^2)^((D - 1) / 2)),
     *                         the transform of r^(D - 3) exp(-r / xi) normalised to M(0) = 1
     *                                                              f_p0 = R >= 0, f_p1 = D in (1, 6),
     *                                                              f_p2 = xi > 0
     *   SAS_FN_FRACTAL        Teixeira's fractal aggregate of spheres of radius R0:
     *                         P(Q R0) (1 + Gamma(D + 1) (xi / R0)^D M(Q xi; D))
     *                                                              f_p0 = R0 > 0, f_p1 = D in (1, 6),
     *                                                              f_p2 = xi > 0
     *   SAS_FN_SPINODAL       Furukawa's spinodal peak: (1 + g/2) x^2 / (g/2 + x^(2 + g)),
     *                         x = Q / Qmax (1 at Q = Qmax)         f_p0 = Qmax > 0, f_p1 = g > 0
     *   SAS_FN_POLYMER_EXCL_VOLUME  Hammouda's chain with excluded volume, Flory exponent
     *                         nu = 1/m: 2 int_0^1 (1 - x) exp(-U x^(2 nu)) dx,
     *                         U = (Q Rg)^2 (2 nu + 1)(2 nu + 2) / 6   f_p0 = Rg > 0, f_p1 = m in (1, 6)
     *   SAS_FN_LINEAR_PEARLS  N spheres of radius R on a line, centres d = 2R + s apart:
     *                         P(Q R) (N + 2 sum_k (N - k) sin(Q k d) / (Q k d)) / N^2
     *                                                              f_p0 = R > 0, f_p1 = s >= 0,
     *                                                              f_p2 = N (an integer, 1 .. 1000) */
    int64_t function;
    double f_scale;          /* >= 0 */
    double f_p0, f_p1, f_p2;
    /* Hayter-Penfold S(Q) of charged spheres (Table II, "Hayter MSA";
     * sq_kind SAS_SQ_HAYTER_MSA): hard spheres of diameter sigma =
     * 2 sq_radius at volume fraction eta = sq_fraction (0 < eta < 0.45),
     * carrying sq_charge elementary charges, in a 1:1 electrolyte of
     * sq_salt mol/L at sq_temperature K with relative permittivity
     * sq_dielectric. Pair potential outside the core (screened Coulomb):
     *   beta u(r) = gamma_c sigma exp(-kappa (r - sigma)) / r,
     *   gamma_c = Z^2 l_B / ((1 + kappa sigma / 2)^2 sigma),
     *   l_B = e^2 / (4 pi eps0 eps_r k_B T),
     *   kappa^2 = 4 pi l_B (2 n_salt + |Z| n_particles)   (counter-ions monovalent).
     * The mean spherical approximation closes the Ornstein-Zernike equation
     * (g = 0 in the core, c = -beta u outside); where it gives g(sigma+) < 0
     * the core is widened to s sigma (volume fraction eta s^3, same
     * potential) until g(s sigma+) = 0 (Hansen-Hayter rescaling).
     * sas_set_model solves this on the host (Newton's method on a grid,
     * Richardson-extrapolated over two grid spacings, about 1e-8 from the
     * continuum) and tabulates S and dS/dQ from Q = 0 past the instrument's
     * largest |Q| and 1/angstrom; the trace interpolates (cubic Hermite,
     * about 1e-7). Beyond the table S - 1 decays as Q^-2 from its last
     * value. SAS_ERR_ARG for parameters out of range, a screening length
     * beyond 500 sigma, or no convergence. Single experiments only (a
     * batch refuses it). */
    double sq_charge;        /* Z >= 0, elementary charges per particle */
    double sq_temperature;   /* K > 0 */
    double sq_salt;          /* mol/L >= 0 */
    double sq_dielectric;    /* relative permittivity of the solvent > 0 */
    /* Fuzzy sphere (Table I, group F; SAS_SPHERE only, 0 elsewhere): the
     * sphere's density convolved with an isotropic Gaussian of width sigma
     * = fuzziness (angstrom, >= 0), so that every amplitude carries
     * exp(-(Q sigma)^2 / 2) (convolution theorem) and dSigma/dOmega the
     * factor exp(-(Q sigma)^2); 0 is the sharp sphere. */
    double fuzziness;
} sas_model_desc;

typedef struct sas_experiment sas_experiment;   /* opaque, library-owned */

/* Create an experiment on the current CUDA device (Sec. II.A: the virtual
 * instrument of a test run -- source, collimation by two pinholes, sample,
 * 2D position-sensitive detector at a set distance): validates the
 * instrument and allocates its FP64 detector (sum w, sum w^2, counts) and
 * the transmitted-weight scalar in device memory. *out is owned by the
 * caller until sas_destroy_experiment. SAS_ERR_ARG on invalid geometry. */
sas_status sas_create_experiment(const sas_instrument *inst, void *stream,
                                 sas_experiment **out);

/* Replace the sample model (Sec. II.A, Eqs. 1-4: amplitude, intensity and
 * the dilute-limit cross section phi drho^2 V P S; Eq. 7 for uniaxial
 * bodies; Eq. 8, the cylinder; Sec. II.B: distributions of the radii and of
 * the particle axis): validates it, builds the FP64 quadrature tables
 * (Schulz generalised Gauss-Laguerre nodes, Gaussian-cap orientation nodes
 * on a Gauss-Legendre grid in (gamma, psi)) and the Percus-Yevick series,
 * rounds them to the trace precision and uploads them (stream-ordered).
 * SAS_ERR_ARG on an invalid model (the message names the field). */
sas_status sas_set_model(sas_experiment *exp, const sas_model_desc *model);

/* Select the Philox experiment id (counter word 1) used by later traces
 * (default 0). */
sas_status sas_set_experiment_id(sas_experiment *exp, uint32_t id);

/* Change the stream later calls enqueue on. */
sas_status sas_set_stream(sas_experiment *exp, void *stream);

/* Zero the detector, then trace neutrons [0, n_neutrons) (Sec. I: each
 * neutron history is independent of the others, single scattering; Sec.
 * II.A: the instrument chain; Eqs. 1-4 weight every history by the model's
 * cross section). Asynchronous on the experiment's stream; SAS_ERR_STATE
 * before sas_set_model. */
sas_status sas_trace(sas_experiment *exp, uint64_t n_neutrons, uint64_t seed);

/* Trace neutrons [first, first + n) and ADD them to the detector: resume a
 * run, or trace one share of a scatter/gather split of the index range
 * across processes or GPUs (Sec. II.C; the histories of any split are the
 * histories of the whole range). Asynchronous; SAS_ERR_STATE before
 * sas_set_model; SAS_ERR_ARG if first + n overflows 64 bits. */
sas_status sas_trace_range(sas_experiment *exp, uint64_t first, uint64_t n, uint64_t seed);

/* Zero the detector and transmitted weight. Asynchronous. */
sas_status sas_reset_detector(sas_experiment *exp);

/* Copy the detector (the 2D PSD of Sec. II.A: per pixel sum of weights,
 * sum of squared weights, histories) into caller-owned HOST buffers of
 * n_pixels entries (n_pixels must equal nx*ny, else SAS_ERR_ARG; any
 * pointer may be NULL to skip it) and the transmitted weight (may be NULL).
 * Intensity per incident neutron = sum_w / histories traced. Synchronises
 * the stream. */
sas_status sas_read_detector(const sas_experiment *exp, double *sum_w, double *sum_w2,
                             uint64_t *count, size_t n_pixels, double *transmitted);

/* Library-owned DEVICE pointers of the detector arrays (valid until destroy). */
sas_status sas_detector_device(const sas_experiment *exp, const double **sum_w,
                               const double **sum_w2, const uint64_t **count,
                               const double **transmitted);

/* Parity hook: dSigma/dOmega (1/angstrom; Eqs. 1-4, 7, 8 averaged per
 * Sec. II.B) of the experiment's model at n scattering vectors. q_xyz: DEVICE float[n][3]; out: DEVICE float[n]
 * (model precision FP32) -- or double pointers if the model is FP64.
 * Asynchronous on the experiment's stream. SAS_ERR_STATE for a per-event
 * model (its cross section is a random draw per history; the records below
 * give its per-history values). */
sas_status sas_eval_model(sas_experiment *exp, const void *q_xyz, size_t n, void *out);

/* The experiment's self-attenuation table (sas_model_desc.self_attenuation):
 * HOST arrays of SAS_ATT_MAX doubles receive the wavelengths (angstrom), the
 * GPU-evaluated mu_s (1/m) there, and the Chebyshev coefficients c of the
 * interpolant sum_j c_j T_j(t), t = (2 lambda - lmin - lmax) / (lmax - lmin),
 * with lmin_lmax[2] the source band; *n = points (1 without a wavelength
 * spread, 0 if the model has no self-attenuation). Any array may be NULL.
 * SAS_ERR_STATE before sas_set_model. */
#define SAS_ATT_MAX 8
sas_status sas_attenuation_table(const sas_experiment *exp, int *n, double *lambda, double *mu_s,
                                 double *coef, double *lmin_lmax);

/* Total scattering cross section per unit volume Sigma_s(lambda) in
 * 1/angstrom: the experiment's dSigma/dOmega integrated over all directions
 * for a neutron along +z, by the rule of sas_model_desc.self_attenuation
 * (built at the shortest wavelength of the instrument's band), evaluated on
 * the GPU at any lambda > 0 whether or not the model attenuates itself.
 * HOST outputs: *sigma; panels[min(n, max_panels)] the share of each |Q|
 * panel (may be NULL with max_panels 0); *n_panels = n. Synchronous.
 * SAS_ERR_STATE before sas_set_model or for a per-event model. */
sas_status sas_total_cross_section(sas_experiment *exp, double lambda, double *sigma, double *panels,
                                   int max_panels, int *n_panels);

/* Parity hook: per-neutron records of neutrons [first, first+n): DEVICE
 * int32 pixel[n] (-1: missed the sample) and DEVICE double weight[n] (1/m
 * units of the tally). Does not touch the detector. Asynchronous. */
sas_status sas_trace_records(sas_experiment *exp, uint64_t first, uint64_t n, uint64_t seed,
                             int32_t *pixel, double *weight);

/* Block until all work on the experiment's stream is done. */
sas_status sas_sync(sas_experiment *exp);

/* Free the experiment and its device memory (NULL is accepted). */
sas_status sas_destroy_experiment(sas_experiment *exp);

/* Thread-local text of the last error (empty string if none). */
const char *sas_last_error(void);

/* Device properties used by the launch heuristics. */
sas_status sas_device_info(int *sm_count, int *smem_per_block_optin, int *cc_major,
                           int *cc_minor);

/* ---- launch configuration and autotuning (single experiment) ---------- */

typedef struct sas_launch_config {
    int32_t block;           /* threads per CTA: multiple of 32 in [32, 1024] */
    int32_t tally;           /* 0: FP64 global atomics per history;
                                1: per-CTA FP32 Kahan shared-memory histogram (FP32 only) */
    int32_t agg;             /* 1: combine lanes of a warp hitting the same pixel first */
    int32_t ctas_per_sm;     /* resident CTAs per SM of the persistent grid (0: all that fit) */
    int32_t stage_orient;    /* 1: copy the orientation table into shared memory */
    int32_t order_q;         /* 1: each CTA orders its histories by |Q| before the model's
                                average, so that a warp's lanes take the same branch of the
                                sphere amplitude (series or closed form) at most radius nodes.
                                Applies to FP32 sphere and core-shell sphere quadrature traces
                                with >= 4 radius nodes and room for the ordering buffers
                                (24 bytes per thread + 1032 bytes) in shared memory; ignored
                                otherwise. The histories, their weights and tallies are the
                                same either way. */
} sas_launch_config;

/* Read / replace the launch configuration of the experiment's trace kernel.
 * SAS_ERR_ARG if it does not fit (shared memory) or is malformed;
 * SAS_ERR_STATE before sas_set_model. */
sas_status sas_get_launch_config(const sas_experiment *exp, sas_launch_config *cfg);
sas_status sas_set_launch_config(sas_experiment *exp, const sas_launch_config *cfg);

/* Autotuner: times every valid configuration (block 256/512/1024, tally,
 * warp aggregation, orientation staging) on n_sample histories with CUDA
 * events, keeps the fastest and caches it per (model kind, precision, node
 * counts, detector size, S(Q)): later sas_set_model calls with the same key
 * start from it. Zeroes the detector. Synchronous. */
sas_status sas_autotune(sas_experiment *exp, uint64_t n_sample, uint64_t seed,
                        sas_launch_config *best, double *best_ms);

/* ---- batched form (many experiments, one persistent graph launch) ----- */

typedef struct sas_batch sas_batch;                 /* opaque, library-owned */

typedef struct sas_batch_config {
    int32_t block;             /* threads per CTA: multiple of 32 in [32, 1024] */
    int32_t ctas_per_sm;       /* 0: as many as fit */
    int32_t use_hist;          /* 1: models without an orientation average tally
                                  through the shared-memory histogram */
    int32_t reserved;
    double target_item_flop;   /* work-item size (FLOP) the index ranges are cut to; an item
                                  holds at least 4 x block histories, in whole multiples of
                                  block (default block 1024, target 2e9) */
} sas_batch_config;

/* Create a batch of n_exp experiments sharing one instrument (Sec. II.A),
 * each with its own model (FP32 only) and neutron count; experiment e uses
 * Philox experiment id e and its own FP64 detector. Builds all quadrature
 * tables, cuts the index ranges into work items ordered longest-first and
 * allocates n_exp * nx * ny * 24 bytes of detectors. SAS_ERR_ARG for an FP64
 * model or a shape-independent law (those trace one by one). */
sas_status sas_create_batch(const sas_instrument *inst, const sas_model_desc *models,
                            const uint64_t *counts, size_t n_exp, void *stream, sas_batch **out);

/* Zero all detectors and trace every experiment: one CUDA-graph launch
 * (memsets + one persistent kernel pulling work items from an atomic
 * counter). The graph is captured on first use and after config changes.
 * Sec. I motivates the batch: large data sets of virtual experiments over a
 * model's parameter space; each experiment's histories are those of
 * sas_trace with experiment id e. Asynchronous on the batch's stream. */
sas_status sas_trace_batch(sas_batch *batch, uint64_t seed);

/* Copy experiment exp's detector (as sas_read_detector) into caller-owned
 * host buffers (n_pixels = nx*ny, else SAS_ERR_ARG; exp >= n_exp is
 * SAS_ERR_ARG; NULL pointers skip). Synchronises the stream. */
sas_status sas_read_batch_detector(const sas_batch *batch, size_t exp, double *sum_w, double *sum_w2,
                                   uint64_t *count, size_t n_pixels, double *transmitted);

/* Library-owned device arrays [n_exp][nx*ny] (transmitted: [n_exp]). */
sas_status sas_batch_detector_device(const sas_batch *batch, const double **sum_w,
                                     const double **sum_w2, const uint64_t **count,
                                     const double **transmitted);

sas_status sas_batch_set_config(sas_batch *batch, const sas_batch_config *cfg);
sas_status sas_batch_get_config(const sas_batch *batch, sas_batch_config *cfg);

/* Work items, persistent grid size, dynamic shared memory, total histories. */
sas_status sas_batch_info(const sas_batch *batch, uint32_t *n_items, int *grid, size_t *smem,
                          uint64_t *total_histories);

/* Autotuner of the batch: times block size x item size x histogram on/off
 * (one traced batch each, CUDA events) and keeps the fastest. Synchronous. */
sas_status sas_batch_autotune(sas_batch *batch, uint64_t seed, sas_batch_config *best,
                              double *best_ms);

sas_status sas_destroy_batch(sas_batch *batch);

/* Batched trace that allocates nothing. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, for example
 * code whose device memory belongs to another allocator or a fixed budget,
 * plugins whose host application forbids device allocations, or loops that
 * cannot accept the implicit synchronisation of an allocation.
 *
 * Same histories and results as sas_create_batch + sas_trace_batch with the
 * default configuration (Philox experiment id = index e). The caller passes
 * host inputs (instrument, n_exp models (FP32), neutron counts) and DEVICE
 * outputs: sum_w, sum_w2, count [n_exp][nx*ny] and transmitted [n_exp]; the
 * call zeroes them, uploads the tables and launches the batch kernel on
 * `stream`, asynchronously.
 * Scratch: model constants, quadrature tables, work items, the work counter
 * and the seed go to one static device array of 8 MiB that every GPU loading
 * the library holds until process exit. A batch whose tables and items do
 * not fit returns SAS_ERR_ARG with the bytes it would need.
 * Every call looks up the array's device address in the caller's current
 * CUDA context (cudaGetSymbolAddress, with the caller's device current):
 * each context that loads the library, e.g. a plugin host's own driver-API
 * context, or the primary context re-created after cudaDeviceReset, has its
 * own copy of the array. The first call in a context also loads the
 * library's device code there; make that first call before any stream
 * capture. The uploads are copies from pageable host memory, so the call may
 * block until they are staged.
 * All calls share the array and it keeps the last call's contents: calls
 * that overlap on the GPU (e.g. on two streams) race, so issue them in
 * order on one stream or synchronise between them. */
sas_status sas_trace_batch_static(const sas_instrument *inst, const sas_model_desc *models,
                                  const uint64_t *counts, size_t n_exp, uint64_t seed,
                                  double *sum_w, double *sum_w2, uint64_t *count,
                                  double *transmitted, void *stream);

/* ---- learned surrogate of the averaged form factor of uniaxial bodies --
 * The paper has no learned part. The network stands in for the cross
 * section of Eq. 8 of a cylinder or an ellipsoid of revolution averaged over
 * the radius and axis distributions of Sec. II.B, the costly step of the
 * anisotropic models (Sec. III.B names the cylinder family among those that
 * gain most on a GPU). One surrogate serves one body. */

typedef struct sas_surrogate sas_surrogate;          /* opaque, library-owned */

/* Training box. The surrogate reproduces, for oriented polydisperse bodies
 * of its kind inside it, the normalised averaged form factor
 * P = <|F|^2> / (drho^2 <V^2>) that sas_set_model's quadrature gives with
 * the same node counts (n_poly Schulz nodes on the radius; n_gamma x n_psi
 * orientation nodes). L is the body's length along its axis: the cylinder's
 * length, or twice the polar semi-axis R_p of the ellipsoid (whose
 * equatorial semi-axis is R). Its inputs are the rotation-invariant features
 * (q_par L / 2, q_perp R, L / (2R), sigma_orient, sigma_poly) plus
 * n_fourier (sin, cos) pairs of k q_par L / 4 (k = 1..n), where q_par and
 * q_perp are the components of Q along and across the mean axis; its output
 * is log P (trained on log max(P, 1e-6)).
 * sigma_poly is learned on n_buckets values spread evenly over the range. */
typedef struct sas_surrogate_box {
    double q_max;                                 /* 1/angstrom */
    double r_min, r_max;                          /* radius R, angstrom */
    double l_min, l_max;                          /* length L along the axis, angstrom */
    double sigma_orient_min, sigma_orient_max;    /* rad */
    double poly_min, poly_max;                    /* Schulz relative width */
    int32_t n_poly, n_gamma, n_psi;               /* quadrature it reproduces */
    int32_t n_buckets;                            /* sigma_poly values in the training set */
    int32_t n_fourier;                            /* Fourier feature pairs (0..13) */
    int32_t model;                                /* SAS_CYLINDER (0 reads as it) or SAS_ELLIPSOID */
} sas_surrogate_box;

/* MLP 64 -> 256 -> 256 -> 256 -> 256 -> 1, SiLU, BF16 hidden weights (FP32
 * master copy, biases and output layer), initialised from Philox(seed). */
sas_status sas_create_surrogate(const sas_surrogate_box *box, uint64_t seed, void *stream,
                                sas_surrogate **out);

/* Draw n training samples uniformly in the box (Philox experiment id
 * 0x80000001) and compute their exact targets log P on the GPU with the
 * trace's quadrature. The data set stays in device memory. */
sas_status sas_surrogate_generate(sas_surrogate *s, uint64_t n, uint64_t seed);

/* Device pointers of the data set: raw parameters [n][8] floats
 * (q_par, q_perp, R, L, sigma_orient, sigma_poly, bucket, 0) and log P [n]. */
sas_status sas_surrogate_dataset(const sas_surrogate *s, const void **raw, const float **log_p,
                                 uint64_t *n);

/* Exact log P (the target quadrature) at raw parameters (DEVICE [n][8]
 * floats, bucket index in column 6) into DEVICE log_p[n]. */
sas_status sas_surrogate_exact(sas_surrogate *s, const void *raw, size_t n, float *log_p);

/* Surrogate log P (tensor-core inference) at raw parameters (DEVICE). */
sas_status sas_surrogate_eval(sas_surrogate *s, const void *raw, size_t n, float *log_p);

/* One forward + backward pass (no update) of the mean squared error of log P
 * over n rows (multiple of 128) of DEVICE raw / log_p; the FP32 gradient of
 * all parameters goes to the HOST buffer grad[n_params]. */
sas_status sas_surrogate_grad(sas_surrogate *s, const void *raw, const float *log_p, uint32_t n,
                              float *grad, size_t n_params);

/* n_steps Adam steps (CUDA-graph replay of forward, backward, weight
 * gradients and update) over consecutive minibatches of `batch` rows
 * (multiple of 128) of the generated data set; learning rate lr with
 * cosine decay over total_steps. */
sas_status sas_surrogate_train(sas_surrogate *s, uint32_t n_steps, uint32_t batch, double lr,
                               uint32_t total_steps);

/* FP32 master parameters (flat layout: W1 [256][64] (column 63 is the
 * layer-1 bias), W2, W3, W4 [256][256] (out, in), b1 (unused, 0), b2, b3, b4,
 * w5 [256], b5), host buffers of n_params floats. */
sas_status sas_surrogate_get_params(const sas_surrogate *s, float *params, size_t n_params);
sas_status sas_surrogate_set_params(sas_surrogate *s, const float *params, size_t n_params);
sas_status sas_surrogate_info(const sas_surrogate *s, size_t *n_params, uint32_t *steps_done);

/* Test hook of the bounded device waits (failure detection without a GPU
 * fault): the next sas_surrogate_eval makes its first CTA wait, before any
 * copy or tensor-core operation is issued, on a barrier that nothing
 * completes; after wait_ns (1 .. 1e9 ns, else SAS_ERR_ARG) it gives up, every
 * CTA frees its tensor memory and returns, and the call reports
 * SAS_ERR_TIMEOUT with no output written. The hook then clears itself, so
 * the following calls run normally. 0 disarms it. */
sas_status sas_surrogate_test_stall(sas_surrogate *s, uint64_t wait_ns);
sas_status sas_destroy_surrogate(sas_surrogate *s);

/* Use the surrogate for the experiment's model when it is of the
 * surrogate's kind and lies in the training box (same node counts);
 * histories whose |Q| leaves the box fall back to the exact quadrature.
 * NULL detaches. The surrogate must outlive the attachment. */
sas_status sas_attach_surrogate(sas_experiment *exp, const sas_surrogate *s);

/* Same for every in-box experiment of the surrogate's kind in a batch: they
 * are traced by a persistent tensor-core kernel in the batch's graph. A
 * batch holds one surrogate per kind (a cylinder and an ellipsoid one);
 * attaching replaces the one of the same kind, NULL detaches both. */
sas_status sas_batch_attach_surrogate(sas_batch *batch, const sas_surrogate *s);

/* Experiments of the batch that the attached surrogates cover (their model
 * lies in a box) and their histories; the other experiments run the exact
 * quadrature. Of the covered histories, those whose |Q| leaves the box are
 * counted by sas_surrogate_fallbacks. NULL outputs are skipped. */
sas_status sas_batch_surrogate_share(const sas_batch *batch, uint64_t *experiments, uint64_t *histories);

/* Histories of surrogate-covered experiments that were evaluated by the
 * exact fallback (|Q| outside the box) since the last attach. */
sas_status sas_surrogate_fallbacks(const sas_experiment *exp, const sas_batch *batch,
                                   uint64_t *count);

/* ---- host-side utilities (no GPU needed): the library's own FP64 tables.
 * They are the quadrature rules sas_set_model builds for the trace. */

/* n-point Gauss-Legendre rule on [-1, 1] (Newton on P_n), n in 1..1024. */
sas_status sas_gauss_legendre(int n, double *x, double *w);

/* Schulz distribution (mean, relative width p) as n generalised
 * Gauss-Laguerre nodes r[n] with normalised weights w[n] (Sec. II.B reading:
 * Schulz instead of per-event Gaussian draws). p == 0: one node at the mean. */
sas_status sas_schulz_nodes(double mean, double p, int n, double *r, double *w);

/* The cylinder radial table of sas_model_desc.radial_table on HOST arrays:
 * radius nodes r[n_nodes] with normalised weights w, mean radius rbar,
 * points x_k = k xmax / (n_points - 1): G[k] and D[k] = h G'(x_k).
 * *max_err: largest error of the cubic Hermite interpolant at the interval
 * midpoints. SAS_ERR_ARG on sizes < 2 or non-positive rbar, xmax. */
sas_status sas_cylinder_radial_table(const double *r, const double *w, int n_nodes, double rbar,
                                     double xmax, int n_points, double *G, double *D, double *max_err);

/* Orientation nodes of the axis distribution about (theta, phi): Gaussian
 * cap of width sigma (or isotropic), n_gamma x n_psi Gauss-Legendre grid.
 * c_xyz[3 * n_gamma * n_psi], w[n_gamma * n_psi]; *n_out = nodes written. */
sas_status sas_orientation_nodes(double theta, double phi, double sigma, int n_gamma, int n_psi,
                                 int isotropic, double *c_xyz, double *w, int *n_out);

/* The Hayter-Penfold S(Q) that sas_set_model tabulates (sq_kind
 * SAS_SQ_HAYTER_MSA; parameters as in sas_model_desc), on HOST arrays:
 * S(Q_j) and dS/dQ(Q_j) interleaved in s_dsdq[2 j], s_dsdq[2 j + 1] at
 * Q_j = j * (*dq) (1/angstrom), j < *n_out, from 0 past q_max; *s_rescale
 * the Hansen-Hayter factor (1 when the plain MSA has g(sigma+) >= 0),
 * *contact the extrapolated g at the (rescaled) contact, *gamma_c the
 * contact potential beta u(sigma+) and *kappa (1/angstrom) the inverse
 * screening length of the unrescaled system. Any output may be NULL except
 * s_dsdq when n_max > 0. SAS_ERR_ARG on parameters out of range or a solve
 * that does not converge; SAS_ERR_ARG when the table needs more than n_max
 * points (*n_out then holds the number needed). */
sas_status sas_hayter_msa_table(double radius_eff, double fraction, double charge, double temperature,
                                double salt, double dielectric, double q_max, int n_max, double *dq,
                                double *s_dsdq, int *n_out, double *s_rescale, double *contact,
                                double *gamma_c, double *kappa);

/* Percus-Yevick constants (alpha, beta, gamma) and the first nser
 * coefficients of G(A)/A in powers of A^2. */
sas_status sas_py_series(double phi, double *alpha_beta_gamma, double *series, int nser);

#ifdef __cplusplus
}
#endif

#endif /* SAS_H */
