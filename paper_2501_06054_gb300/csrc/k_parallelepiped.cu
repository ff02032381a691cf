// Instantiates the trace, records and evaluation kernels for the rectangular parallelepiped.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_PARALLELEPIPED>;
template struct Launcher<double, SAS_PARALLELEPIPED>;
}  // namespace sas
