// Instantiates the trace, records and evaluation kernels for the cylinder model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_CYLINDER>;
template struct Launcher<double, SAS_CYLINDER>;
}  // namespace sas
