// Instantiates the trace, records and evaluation kernels for the shape-independent laws.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_SHAPE_INDEPENDENT>;
template struct Launcher<double, SAS_SHAPE_INDEPENDENT>;
}  // namespace sas
