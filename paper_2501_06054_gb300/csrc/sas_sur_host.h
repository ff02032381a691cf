// Host-side hooks of the surrogate used by the experiment and batch runtimes.
#pragma once

#include <cuda_runtime.h>
#include "sas_surrogate.cuh"

namespace sas {
bool surrogate_covers(const sas_surrogate* s, const sas_model_desc& m);
sur::SurExp surrogate_exp(const sas_model_desc& m, bool in_box);
cudaError_t launch_sur_trace(const sas_surrogate* s, const sur::STParams& P, int sm_count, cudaStream_t st);
const float* surrogate_params(const sas_surrogate* s);
sur::Box surrogate_dbox(const sas_surrogate* s);
int* surrogate_err(const sas_surrogate* s);
}  // namespace sas
