// Host-side hooks of the surrogate used by the experiment and batch runtimes.
#pragma once

#include <cuda_runtime.h>

#include <vector>
#include "sas_surrogate.cuh"

namespace sas {
bool surrogate_covers(const sas_surrogate* s, const sas_model_desc& m);
int surrogate_kind(const sas_surrogate* s);   // SAS_CYLINDER or SAS_ELLIPSOID
sur::SurExp surrogate_exp(const sas_model_desc& m, bool in_box);
// Launches min(sm_count, P.n_pairs) CTAs (one per SM); nothing when there are no pairs.
cudaError_t launch_sur_trace(const sas_surrogate* s, const sur::STParams& P, int sm_count, cudaStream_t st);
// prefix[i] = 256-history pairs in items [0, i); returns the total.
uint64_t surrogate_pair_prefix(const std::vector<WorkItem>& items, std::vector<uint32_t>& prefix);
// Trace epilogue constants [1281]: b_l / 2 (4 x 256), w5, b5 (kept current by training and set_params).
const float* surrogate_epi(const sas_surrogate* s);
sur::Box surrogate_dbox(const sas_surrogate* s);
int* surrogate_err(const sas_surrogate* s);
// SAS_ERR_TIMEOUT (and clears the flag) if a surrogate kernel on stream st gave up a wait.
sas_status surrogate_take_error(const sas_surrogate* s, cudaStream_t st);
}  // namespace sas
