// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/apsp.h"

namespace apsp {

// Number of SMs of the current device (cached).
int sm_count();

// n rounded up to the working tile order (a multiple of 128).
int padded_order(int n);

// Single-graph run on device buffers (the body of apsp_fw_ex).
apsp_status fw_run(const float* W, float* D, int32_t* P, int n, const apsp_options* opt, void* workspace,
                   size_t workspace_bytes, apsp_run_info* info, cudaStream_t s);

}  // namespace apsp
