// Instantiates the trace, records and evaluation kernels for the core-shell cylinder model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_CORE_SHELL_CYLINDER>;
template struct Launcher<double, SAS_CORE_SHELL_CYLINDER>;
}  // namespace sas
