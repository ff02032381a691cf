// Instantiates the trace, records and evaluation kernels for the hollow rectangular prism model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_HOLLOW_RECTANGULAR_PRISM>;
template struct Launcher<double, SAS_HOLLOW_RECTANGULAR_PRISM>;
}  // namespace sas
