// Instantiates the trace, records and evaluation kernels for the capped cylinder model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_CAPPED_CYLINDER>;
template struct Launcher<double, SAS_CAPPED_CYLINDER>;
}  // namespace sas
