// Instantiates the trace, records and evaluation kernels for the core-shell bicelle model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_CORE_SHELL_BICELLE>;
template struct Launcher<double, SAS_CORE_SHELL_BICELLE>;
}  // namespace sas
