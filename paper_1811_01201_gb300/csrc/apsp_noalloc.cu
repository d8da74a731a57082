// Allocation-free single-graph solve: apsp_fw_noalloc (declared in include/apsp.h).
//
// Some callers cannot allocate device memory at the point where they need a
// shortest-path solve: code embedded in a host framework that owns the whole
// device memory (its own pool, no spare room for another allocator), code
// that must never block on, or fail inside, an allocator while it runs, and
// drivers or environments where the stream-ordered allocator that apsp_fw
// uses for its workspace is unavailable. For them this entry point takes its
// workspace from one fixed array in device memory that is part of the library
// itself, so the call performs no cudaMalloc, cudaMallocAsync, cudaFree or
// other allocation; the caller still provides W, D and P.
//
// The array is sized once (APSP_NOALLOC_SCRATCH_BYTES); every GPU that loads
// the library holds it until the process exits. All calls on a device share
// it, so calls that overlap on the GPU (different streams or threads without
// ordering between them) race on it and corrupt each other's results. Each
// call rewrites everything it reads from the array before reading it (the
// input-scan counters are zeroed on the stream, the round maxima are reset by
// every round's first kernel, the padded working matrices are fully
// initialised), so no state carries over from the previous call.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/apsp.h"
#include "apsp_internal.h"

// The shared workspace (device global memory owned by the library).
static __device__ __align__(256) unsigned char g_apsp_noalloc_scratch[APSP_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device. In host code the array's
// name only stands in for it; the address has to be asked for, once per device,
// with that device current.
apsp_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return APSP_ECUDA;
  }
  std::lock_guard<std::mutex> g(g_setup_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_apsp_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return APSP_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return APSP_OK;
}

}  // namespace

extern "C" size_t apsp_noalloc_scratch_bytes(void) { return (size_t)APSP_NOALLOC_SCRATCH_BYTES; }

extern "C" apsp_status apsp_fw_noalloc(const float* W, float* D, int32_t* P, int n, const apsp_options* opt,
                                       apsp_run_info* info, void* stream) {
  if (n < 1 || !W || !D || !P) return APSP_EINVAL;
  apsp_options o;
  if (opt) {
    o = *opt;
  } else {
    o.bs = 0;
    o.dtype = APSP_DTYPE_AUTO;
    o.validate = 1;
    o.flags = 0;
  }
  // per-phase timing creates CUDA events; this entry point creates nothing
  if (o.flags & APSP_FLAG_TIME_PHASES) return APSP_EINVAL;
  // sized for the D and P given (a misaligned D or P needs a working copy in the array)
  const size_t need = apsp::fw_workspace_need(n, &o, D, P);
  if (need == 0) return APSP_EINVAL;
  if (need > (size_t)APSP_NOALLOC_SCRATCH_BYTES) return APSP_ENOMEM;  // too large for the fixed array
  void* scratch = nullptr;
  apsp_status st = scratch_for_current_device(&scratch);
  if (st != APSP_OK) return st;
  return apsp_fw_ex(W, D, P, n, &o, scratch, (size_t)APSP_NOALLOC_SCRATCH_BYTES, info, stream);
}
