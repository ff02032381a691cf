// Instantiates the trace, records and evaluation kernels for the triaxial ellipsoid.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_TRIAXIAL_ELLIPSOID>;
template struct Launcher<double, SAS_TRIAXIAL_ELLIPSOID>;
}  // namespace sas
