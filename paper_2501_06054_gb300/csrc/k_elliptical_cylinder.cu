// Instantiates the trace, records and evaluation kernels for the elliptical cylinder model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_ELLIPTICAL_CYLINDER>;
template struct Launcher<double, SAS_ELLIPTICAL_CYLINDER>;
}  // namespace sas
