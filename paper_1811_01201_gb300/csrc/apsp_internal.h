// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/apsp.h"

namespace apsp {

// Number of SMs of the current device (cached).
int sm_count();

// n rounded up to the working tile order (a multiple of 128).
int padded_order(int n);

// Workspace bytes of fw_exec for a given arithmetic.
size_t fw_exec_workspace(int n, int bs, int dtype);

// Block rounds with the arithmetic already chosen (no input scan; async).
// graph_int: every finite weight is an integer (enables exact keys in phase 3).
// workspace may be NULL (stream-ordered allocation inside).
apsp_status fw_exec(const float* W, float* D, int32_t* P, int n, int bs, int dtype, int graph_int, int flags,
                    void* workspace, size_t workspace_bytes, apsp_run_info* info, cudaStream_t s);

// Single-graph run on device buffers (the body of apsp_fw_ex).
apsp_status fw_run(const float* W, float* D, int32_t* P, int n, const apsp_options* opt, void* workspace,
                   size_t workspace_bytes, apsp_run_info* info, cudaStream_t s);

// Descriptor of one graph of an asynchronous batch (same layout as the
// batched kernel's table entry).
struct BatchGraphDesc {
  const float* W;
  float* D;
  int32_t* P;
  int n;
  int ph3_rows;  // phase-3 tile height of keyed graphs (0 = the kernel's default)
};

// Largest graph order of the batched kernel.
constexpr int kBatchMaxN = 512;

// One-shot asynchronous batch launch for pre-validated graphs. host_graphs
// points to `count` descriptors followed by `count` ints (the processing
// order, largest first), all page-locked and alive until the stream passes.
apsp_status batch_launch_async(const BatchGraphDesc* host_graphs, int count, cudaStream_t s);

// Phase-3 tile height the batched kernel uses for a keyed graph of order n
// unless an autotuning run chose another.
int default_ph3_rows(int n);

}  // namespace apsp
