// Instantiates the trace, records and evaluation kernels for the hollow cylinder model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_HOLLOW_CYLINDER>;
template struct Launcher<double, SAS_HOLLOW_CYLINDER>;
}  // namespace sas
