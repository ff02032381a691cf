// Hayter-Penfold structure factor of charged spheres (Table II, "Hayter
// MSA"): host solver of the mean spherical approximation and the table the
// trace interpolates. Host code only.
#pragma once

#include <string>
#include <vector>

namespace sas {
namespace msa {

// The hard-core screened Coulomb fluid in reduced units (lengths in the
// hard-core diameter sigma): volume fraction eta, contact potential gamma_c
// = beta u(sigma+), inverse screening length k = kappa sigma.
struct Reduced {
    double sigma;     // angstrom
    double eta;
    double gamma_c;
    double k;
    double l_b;       // Bjerrum length, angstrom
    double kappa;     // 1/angstrom
};

// From the physical parameters (radius in angstrom, charge in e, K, mol/L).
Reduced reduce(double radius_eff, double fraction, double charge, double temperature, double salt,
               double dielectric);

// S(Q) and dS/dQ on Q_j = j dq (1/angstrom), j < S.size(), interleaved
// {S_0, D_0, S_1, D_1, ...}; s_rescale is the Hansen-Hayter factor (1: the
// plain MSA), contact the extrapolated g(s sigma+).
struct Table {
    double dq = 0.0;
    std::vector<double> sd;
    double s_rescale = 1.0;
    double contact = 0.0;
};

// Solve and tabulate up to at least q_max (1/angstrom). Returns false with
// a message on parameters it cannot handle or a solve that does not
// converge.
bool build_table(const Reduced& r, double q_max, Table& out, std::string& err);

}  // namespace msa
}  // namespace sas
