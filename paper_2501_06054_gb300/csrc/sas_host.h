// Host-side tables of a model (FP64) and the functions that build them.
#pragma once

#include <vector>
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
};

void gauss_legendre(int n, double* x, double* w);
void gauss_laguerre_gen(int n, double alpha, double* x, double* w);
void schulz_nodes(double mean, double p, int n, double* r, double* w);
int orientation_nodes(double theta, double phi, double sigma, int ng, int npsi, int isotropic,
                      double* c, double* w);
void py_constants(double phi, double* alpha, double* beta, double* gamma, double* series, int nser);
sas_status build_model_tables(const sas_model_desc& m, ModelTables& t);
sas_status validate_instrument(const sas_instrument* in);
sas_status validate_model(const sas_model_desc* m);
template <typename T> ModelConst<T> model_const(const sas_model_desc& m, const ModelTables& t);
template <typename T> InstConst<T> inst_const(const sas_instrument& in);

}  // namespace sas
