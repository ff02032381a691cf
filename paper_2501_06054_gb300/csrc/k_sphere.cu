// Instantiates the trace, records and evaluation kernels for the sphere model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_SPHERE>;
template struct Launcher<double, SAS_SPHERE>;
}  // namespace sas
