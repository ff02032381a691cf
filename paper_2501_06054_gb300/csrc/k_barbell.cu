// Instantiates the trace, records and evaluation kernels for the barbell model.
#include "sas_kernels.cuh"

namespace sas {
template struct Launcher<float, SAS_BARBELL>;
template struct Launcher<double, SAS_BARBELL>;
}  // namespace sas
