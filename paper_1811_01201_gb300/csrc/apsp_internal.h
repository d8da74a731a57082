// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/apsp.h"

namespace apsp {

// Devices the library keeps per-device state for (function attributes, SM
// count, the allocation-free workspace address).
constexpr int kMaxDevices = 64;

// The current CUDA device, or -1 (error cleared) if it cannot be read or is
// kMaxDevices or above.
int current_device();

// Number of SMs of the current device (cached per device).
int sm_count();

// n rounded up to the working tile order (a multiple of 128).
int padded_order(int n);

// Workspace bytes of fw_exec for a given arithmetic, block size and D / P
// (NULL counts as 16-byte aligned).
size_t fw_exec_workspace(int n, int bs, int dtype, const void* D, const void* P);

// Workspace bytes apsp_fw_ex needs for (n, opt) and these D and P: the larger
// of the two arithmetics the options allow; 0 for invalid arguments.
size_t fw_workspace_need(int n, const apsp_options* opt, const void* D, const void* P);

// Block rounds with the arithmetic already chosen (no input scan; async).
// graph_int: every finite weight is an integer (enables exact keys in phase 3).
// workspace may be NULL (stream-ordered allocation inside).
apsp_status fw_exec(const float* W, float* D, int32_t* P, int n, int bs, int dtype, int graph_int, int flags,
                    void* workspace, size_t workspace_bytes, apsp_run_info* info, cudaStream_t s);

// Byte offset of a solve's own fault word inside its workspace (set when a
// bounded device wait of that solve expired; zeroed by the solve's first kernel).
size_t fw_fault_word_offset();

// Eligibility of the exact 16-bit path: integer weights and either every
// simple path length below 65535 (max_w * (n - 1) < 65535), or a complete
// graph (no absent edge) with max_w < 65535.
bool u16_eligible(bool all_integer, bool complete, float max_w, int n);

// Library default block size for order n once the arithmetic is chosen.
int default_bs_for(int n, int dtype);

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
