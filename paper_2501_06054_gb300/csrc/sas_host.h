// Host-side tables of a model (FP64) and the functions that build them.
#pragma once

#include <vector>
#include <cuda_runtime.h>
#include "sas_types.h"

namespace sas {

struct ModelTables {
    std::vector<double> poly;     // n_poly * SAS_POLY_STRIDE
    std::vector<double> orient;   // n_orient * SAS_ORIENT_STRIDE
    int n_poly = 0, n_orient = 0;
    double scale = 0, vmean = 0, half_length = 0, rp2 = 0;
    int sq_kind = 0;
    double sq_2r = 0, sq_24phi = 0, sq_alpha = 0, sq_beta = 0, sq_gamma = 0, sq_switch = 0;
    std::vector<double> sq_series;
    // Hayter-Penfold S(Q): {S_j, dq dS/dQ_j} at Q_j = j sq_dq
    std::vector<double> sq_tab;
    double sq_dq = 0, sq_rescale = 1, sq_contact = 0;
    // cylinder radial table (radial_table = 1): G(x) and h G'(x) on a grid,
    // stored behind the radius nodes in `poly`
    int n_rad = 0;                // radius nodes (n_poly counts the table rows too)
    int n_tab = 0;                // table points (0: no table)
    double tab_inv_h = 0, tab_xmax = 0, tab_c0 = 0, tab_rbar = 0, tab_err = 0;
    double r_max = 0;             // largest polydisperse radius node
    // capped cylinder and barbell: cap slices behind the radius nodes
    int n_cap = 0;
    double cap_body = 0, cap_r2 = 0, cap_rho2max = 0;
    // self-attenuation: mu_s (1/m) at the Chebyshev wavelengths and its
    // interpolant (att_n = 0: off)
    int att_n = 0;
    double att_lmin = 0, att_lmax = 0;
    double att_lam[SAS_ATT_MAX] = {}, att_mu[SAS_ATT_MAX] = {}, att_c[SAS_ATT_MAX] = {};
};

// The total-cross-section rule of a model for an instrument's band.
struct AttRule {
    int n_lambda = 0;
    double lmin = 0, lmax = 0, kmax = 0;
    double lam[SAS_ATT_MAX] = {};
    std::vector<AttPanel> panels;
};

void gauss_legendre(int n, double* x, double* w);
void gauss_laguerre_gen(int n, double alpha, double* x, double* w);
void schulz_nodes(double mean, double p, int n, double* r, double* w);
int orientation_nodes(double theta, double phi, double sigma, int ng, int npsi, int isotropic,
                      double* c, double* w);
void py_constants(double phi, double* alpha, double* beta, double* gamma, double* series, int nser);
// q_max: upper bound of |Q| over the instrument (for the radial table; 0: none)
sas_status build_model_tables(const sas_model_desc& m, ModelTables& t, double q_max);
double instrument_q_max(const sas_instrument& in);
// G(x) = sum_i w_i t_i^4 a(x t_i)^2, a(y) = 2 J1(y) / y, t_i = r_i / rbar, and
// D = h G'(x) at x_k = k h, h = xmax / (n - 1); returns the largest error of
// the cubic Hermite interpolant at the interval midpoints.
double cylinder_radial_table(const double* r, const double* w, int np, double rbar, double xmax, int n,
                             double* G, double* D);
sas_status validate_instrument(const sas_instrument* in);
sas_status validate_model(const sas_model_desc* m);
template <typename T> ModelConst<T> model_const(const sas_model_desc& m, const ModelTables& t);
// extent of the particle, the rule, and the table from mu_s at the nodes
double model_extent(const sas_model_desc& m, const ModelTables& t);
double cap_height(const sas_model_desc& m);
double capped_volume(const sas_model_desc& m);
bool shelled_cylinder(int64_t kind);
bool axes3_kind(int64_t kind);
double face_layer(const sas_model_desc& m);
void shelled_contrasts(const sas_model_desc& m, double d[4]);
void att_rule(const sas_instrument& in, const sas_model_desc& m, const ModelTables& t, AttRule& r);
void att_fit(const AttRule& r, const double* mu, ModelTables& t);
// evaluates mu_s (1/m) at the rule's wavelengths on the GPU (kernels of the
// model's kind and precision, tables already on the device)
cudaError_t att_nodes(const sas_model_desc& m, const ModelTables& t, const void* d_poly, const void* d_orient,
                      const AttRule& r, cudaStream_t s, double* mu_out);
// the same at nl wavelengths lam (<= SAS_ATT_MAX): mu_s (1/m) and, if
// partial_out is given, each panel's share of Sigma_s (1/angstrom), [nl][panels]
cudaError_t att_run(const sas_model_desc& m, const ModelTables& t, const void* d_poly, const void* d_orient,
                    const AttRule& r, const double* lam, int nl, cudaStream_t s, double* mu_out, double* partial_out);
template <typename T> InstConst<T> inst_const(const sas_instrument& in);

}  // namespace sas
