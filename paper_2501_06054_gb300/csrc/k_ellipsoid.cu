// Instantiates the trace, records and evaluation kernels for the ellipsoid model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_ELLIPSOID>;
template struct Launcher<double, SAS_ELLIPSOID>;
}  // namespace sas
