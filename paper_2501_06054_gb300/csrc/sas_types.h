// Plain-data structures passed from the host runtime to the kernels.
#pragma once

#include <stdint.h>
#include "../../include/sas.h"

#define SAS_SQ_NSER 14        // terms of the Percus-Yevick G(A)/A series in A^2
#define SAS_MAX_POLY 64
#define SAS_MAX_ORIENT_SIDE 128
#define SAS_POLY_STRIDE 8     // values per polydispersity node
#define SAS_ORIENT_STRIDE 4   // values per orientation node
#define SAS_ATT_GL 8          // Gauss-Legendre nodes per |Q| panel of the total cross section

namespace sas {

// Instrument in the trace precision (derived quantities precomputed).
template <typename T>
struct InstConst {
    T lambda0, dlambda;
    T ap1_r, ap1_z, ap2_r, ap2_z;
    T hx, hy, thick, mu;
    T det_z, px, py, half_wx, half_wy, area;
    T two_pi;
    int nx, ny;
};

// Attenuation of the beam by the particles' own scattering, mu_s(lambda) in
// 1/m, as sum_j c[j] T_j(t), t = lambda * t_mul + t_add (n = 0: off).
template <typename T>
struct AttTable {
    int n;
    T t_mul, t_add;
    T c[SAS_ATT_MAX];
};

// One |Q| panel of the total-cross-section rule at k_max: Gauss-Legendre
// nodes q and weights w (1/angstrom) and the azimuthal points on its rings.
struct AttPanel {
    double q[SAS_ATT_GL];
    double w[SAS_ATT_GL];
    int n_phi;
    int pad;
};

// Model constants in the trace precision.
//   poly table per node (SAS_POLY_STRIDE values); the sphere amplitude is
//   evaluated as g = f / 3, so its factor 3 is folded in here:
//     sphere     {r, c / r^6, c = 9 w (drho V)^2, r^2, 1/r, 0...}  (ascending r)
//     core-shell {r_c^2, r_o^2, c_1 = 3 sqrt(w) (rho_c - rho_s) V_c,
//                 c_2 = 3 sqrt(w) (rho_s - rho_solv) V_o, c_1 / r_c^3, c_2 / r_o^3, r_c, r_o}
//                (ascending r_c)
//     cylinder   {r^2, w (drho V)^2, r, 1/r, 1/sqrt(r), 0...}  (ascending r)
//     ellipsoid  {r_e^2, 9 w (drho V)^2, 0...}
//     elliptical cylinder {s, w (drho V(s))^2, 0...}; hollow rectangular prism
//                {s, w (8 drho s^3)^2, 0...} (frames as for the 3-axis kinds)
//     capped cylinder, barbell {s, w (drho s^3)^2, s^2, 0...} (s = r_i / r),
//                followed by the cap slices, two per row: {z_j, rho_j^2, c_j, 0}
//     core-shell / hollow cylinder, bicelle {r^2, r_o^2, c_1, c_2, c_3, c_4, r, r_o}
//                (ascending r): F = (c_1 s_L + c_2 s_Lo) a(Q_AB r) + (c_3 s_L + c_4 s_Lo) a(Q_AB r_o),
//                s_H = sinc(Q_C H / 2), L_o = L + 2 t_f, c_k = sqrt(w) times the contrast
//                times the volume of its nested cylinder (ModelConst ev_k: the contrasts)
//     core-shell ellipsoid {r_e^2, r_o^2, 3 sqrt(w) (rho_c - rho_s) V_c,
//                3 sqrt(w) (rho_s - rho_solv) V_o, 0...}
//   orient table per node: {c_x, c_y, c_z, weight}
template <typename T>
struct ModelConst {
    int kind, sq_kind, n_poly, n_orient;
    T scale;         // phi / <V>
    T half_length;   // cylinder L / 2
    T shell;         // core-shell shell thickness
    T rp2;           // ellipsoid polar radius squared
    T sq_2r;         // 2 R_hs
    T sq_24phi;      // 24 phi_hs
    T sq_alpha, sq_beta, sq_gamma;
    T sq_switch;     // A below which the series is used
    T sq_series[SAS_SQ_NSER];
    const T* sq_tab;  // Hayter-Penfold S(Q): {S_j, dq dS/dQ_j} at Q_j = j dq (device, global memory)
    int sq_n;
    T sq_inv_dq;
    // per-event sampling (Sec. II.B): one radius and one axis per history
    int event;       // 0: quadrature average over the tables, 1: per-event draws
    int orient_mode; // axis draw: 0 fixed (ev_axis), 1 uniform on the sphere, 2 uniform angles
    T ev_r;          // mean of the polydisperse radius
    T ev_p;          // sigma / mean of its Gaussian (0: monodisperse)
    T ev_lo;         // Phi(-1/p): probability mass of r <= 0, removed by the restriction
    T ev_1mlo;       // 1 - ev_lo
    T ev_c1, ev_c2;  // contrasts: (drho, 0), core-shell (rho_core - rho_shell, rho_shell - rho_solvent)
    T ev_len;        // cylinder L
    T ev_rp;         // ellipsoid polar radius
    T ev_axis[3];    // fixed axis (orient_mode 0)
    // cylinder radial table: inner(q_AB) = tab_c0 G(q_AB rbar), G interpolated
    int n_rad;       // radius nodes (the direct sum beyond the table)
    int n_tab;       // table points (0: direct sum)
    T tab_inv_h, tab_xmax, tab_c0, tab_rbar;
    // 3-axis kinds: sizes along (A, B, C) (poly nodes hold scale factors);
    // orientation rows come in threes: (A, w), (B, 0), (C, 0)
    T ax_a, ax_b, ax_c;
    T ev_frame[6];   // rows A and B of the fixed frame (C is ev_axis)
    AttTable<T> att; // self-attenuation mu_s(lambda) (n = 0: the instrument's mu only)
    // capped cylinder and barbell: the cylinder's amplitude pi r^2 L, r^2,
    // the largest squared slice radius (cylinder or cap) and the cap slices
    // stored behind the n_rad radius nodes
    int n_cap;
    T cap_body, cap_r2, cap_rho2max;
    // shelled uniaxial kinds: the shell's half length L/2 + t_f (cylinders),
    // the outer polar radius r_p + t_p and its square (ellipsoid)
    T half_length_o, rp_o, rp2o;
    T ev_k[4];       // shelled cylinders: the contrasts of c_1..c_4 (per-event amplitudes)
    // hollow rectangular prism: inner half-edges and the two a b c products
    T ax_ai, ax_bi, ax_ci, ax_v, ax_vi;
    // shape-independent laws: the function and its parameters (Rg^2 / 3,
    // Rg^2, xi^2, m, Q0 and 1 / (2 sigma^2), or a2, c1, c2 in f_a, f_b, f_c;
    // the later laws as set in model_const)
    int function;
    T f_a, f_b, f_c, f_d, f_e;
    T fuzz2;         // fuzzy sphere: sigma^2 log2(e) (dSigma/dOmega times 2^(-Q^2 fuzz2)); 0 otherwise
};

}  // namespace sas
