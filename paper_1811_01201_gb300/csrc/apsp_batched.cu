// Batched APSP: host side of the persistent many-graph launch (C ABI in
// include/apsp.h). The descriptor table and the largest-first order live in
// device memory owned by an apsp_batch; a launch is a queue reset plus one
// kernel, so it can be captured into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/apsp.h"
#include "apsp_internal.h"
#include "fw_batched.cuh"

namespace apsp {

// Phase-3 tile of a keyed graph before any autotuning, by its height (32: 32 x 64 tiles, 64:
// 64 x 64, 128: 128 x 64): the shape whose tile grid over the compressed (n - 32) x (n - 32)
// index space costs least, counting the padded area times the instructions a relaxation takes
// on that shape (hot loop plus per-tile load and epilogue: 1.78, 1.59 and 1.53).
int default_ph3_rows(int n) {
  const long m = std::max(1, n - kBBS);
  const struct { int rows, cols; double cost; } shapes[3] = {{32, 64, 1.78}, {64, 64, 1.59}, {128, 64, 1.53}};
  int best = 128;
  double best_v = 0.0;
  for (const auto& sh : shapes) {
    const double v = (double)((m + sh.rows - 1) / sh.rows * sh.rows) * (double)((m + sh.cols - 1) / sh.cols * sh.cols) *
                     sh.cost;
    if (best_v == 0.0 || v < best_v) {
      best_v = v;
      best = sh.rows;
    }
  }
  return best;
}

// The batched kernel's shared-memory limit, set once per device (function
// attributes belong to the device that was current when they were set).
static cudaError_t batched_kernel_attributes() {
  static std::once_flag once[kMaxDevices];
  static cudaError_t errs[kMaxDevices];
  const int dev = current_device();
  if (dev < 0) return cudaErrorInvalidDevice;
  std::call_once(once[dev], [dev] {
    errs[dev] = cudaFuncSetAttribute(fw_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)batched_smem_bytes(kBMaxN));
  });
  return errs[dev];
}

// One CTA per graph: count negative / NaN off-diagonal weights.
__global__ void scan_batch_kernel(const BatchGraph* __restrict__ graphs, int count, unsigned* bad) {
  __shared__ unsigned s_bad;
  for (int g = blockIdx.x; g < count; g += gridDim.x) {
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const BatchGraph G = graphs[g];
    unsigned b = 0;
    for (size_t t = threadIdx.x; t < (size_t)G.n * G.n; t += blockDim.x) {
      const size_t i = t / G.n, j = t - i * G.n;
      const float v = G.W[t];
      if (i != j && (v != v || v < 0.f)) b = 1;
    }
    if (b) s_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicAdd(bad, 1u);
    __syncthreads();
  }
}

}  // namespace apsp

using namespace apsp;

struct apsp_batch {
  BatchGraph* d_graphs = nullptr;
  int* d_order = nullptr;
  BatchQueue* d_queue = nullptr;
  int count = 0;
  int n_max = 0;
  int sp = 0;
  size_t smem = 0;
  int grid = 0;
  std::vector<BatchGraph> hg;  // host copy of the descriptor table
  std::vector<int> order;      // largest first
};

extern "C" int apsp_batched_bs(int /*n*/) { return kBBS; }

static apsp_status batch_free(apsp_batch* b) {
  if (!b) return APSP_OK;
  cudaFree(b->d_graphs);
  cudaFree(b->d_order);
  cudaFree(b->d_queue);
  delete b;
  return APSP_OK;
}

extern "C" apsp_status apsp_batch_create(const float* const* W, float* const* D, int32_t* const* P, const int* n,
                                         int count, const apsp_options* opt, apsp_batch** out, void* stream) {
  if (!out) return APSP_EINVAL;
  *out = nullptr;
  if (count < 1 || !W || !D || !P || !n) return APSP_EINVAL;
  int validate = 1;
  if (opt) {
    if (opt->bs != 0 && opt->bs != kBBS) return APSP_EINVAL;
    if (opt->dtype != APSP_DTYPE_AUTO && opt->dtype != APSP_DTYPE_F32) return APSP_EINVAL;
    validate = opt->validate;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<BatchGraph> hg(count);
  int n_max = 1;
  for (int g = 0; g < count; ++g) {
    if (n[g] < 1 || n[g] > kBMaxN || !W[g] || !D[g] || !P[g]) return APSP_EINVAL;
    hg[g] = BatchGraph{W[g], D[g], P[g], n[g], default_ph3_rows(n[g])};
    n_max = std::max(n_max, n[g]);
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });

  apsp_batch* b = new apsp_batch();
  b->hg = hg;
  b->order = order;
  b->count = count;
  b->n_max = n_max;
  b->sp = batched_sp(n_max);
  b->smem = batched_smem_bytes(n_max);
  if (cudaMalloc(&b->d_graphs, sizeof(BatchGraph) * count) != cudaSuccess ||
      cudaMalloc(&b->d_order, sizeof(int) * count) != cudaSuccess ||
      cudaMalloc(&b->d_queue, sizeof(BatchQueue) + sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    return APSP_ENOMEM;
  }
  apsp_status st = APSP_OK;
  if (cudaMemcpyAsync(b->d_graphs, hg.data(), sizeof(BatchGraph) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = APSP_ECUDA;
  if (st == APSP_OK && validate) {
    unsigned* d_bad = reinterpret_cast<unsigned*>(b->d_queue + 1);
    cudaMemsetAsync(d_bad, 0, sizeof(unsigned), s);
    scan_batch_kernel<<<std::min(count, sm_count() * 8), 256, 0, s>>>(b->d_graphs, count, d_bad);
    unsigned h_bad = 0;
    if (cudaMemcpyAsync(&h_bad, d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) st = APSP_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) st = APSP_ECUDA;
    if (st == APSP_OK && h_bad) st = APSP_EINVAL;
  } else if (st == APSP_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    st = APSP_ECUDA;
  }
  if (st == APSP_OK) {
    if (batched_kernel_attributes() != cudaSuccess) st = APSP_ECUDA;
    int per_sm = 0;
    if (st == APSP_OK &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_batched_kernel, kBThreads, b->smem) != cudaSuccess)
      st = APSP_ECUDA;
    b->grid = std::max(1, std::min(count, std::max(1, per_sm) * sm_count()));
  }
  if (st != APSP_OK) {
    cudaGetLastError();
    batch_free(b);
    return st;
  }
  *out = b;
  return APSP_OK;
}

extern "C" apsp_status apsp_batch_launch(apsp_batch* b, void* stream) {
  if (!b) return APSP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(b->d_queue, 0, sizeof(BatchQueue), s) != cudaSuccess) return APSP_ECUDA;
  fw_batched_kernel<<<b->grid, kBThreads, b->smem, s>>>(b->d_graphs, b->d_order, b->count, b->d_queue, b->sp, 0);
  return cudaGetLastError() == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

namespace {
// Size classes of the phase-3 tile autotuner: n <= 64, <= 128, <= 256, <= 512.
constexpr int kTuneClasses = 4;
constexpr int kTuneClassMax[kTuneClasses] = {64, 128, 256, 512};
// Candidates: 0 = each graph's size rule (default_ph3_rows), then one tile for the whole class.
constexpr int kTuneRows[4] = {0, 32, 64, 128};

int tune_class(int n) {
  for (int c = 0; c < kTuneClasses; ++c)
    if (n <= kTuneClassMax[c]) return c;
  return kTuneClasses - 1;
}
}  // namespace

extern "C" apsp_status apsp_batch_autotune(apsp_batch* b, int* rows_out, void* stream) {
  if (!b) return APSP_EINVAL;
  for (const BatchGraph& g : b->hg)
    if (static_cast<const void*>(g.W) == static_cast<const void*>(g.D)) return APSP_EINVAL;  // reruns need W
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int> cls_order[kTuneClasses];
  for (int idx : b->order) cls_order[tune_class(b->hg[idx].n)].push_back(idx);  // largest first per class
  int* d_sub = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  apsp_status st = APSP_OK;
  if (cudaMalloc(&d_sub, sizeof(int) * b->count) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    st = APSP_ECUDA;
  // the size-rule candidate runs on the table's own tiles: put the rule back first
  for (BatchGraph& g : b->hg) g.ph3_rows = default_ph3_rows(g.n);
  if (st == APSP_OK &&
      cudaMemcpyAsync(b->d_graphs, b->hg.data(), sizeof(BatchGraph) * b->count, cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    st = APSP_ECUDA;
  int chosen[kTuneClasses] = {-1, -1, -1, -1};
  for (int c = 0; c < kTuneClasses && st == APSP_OK; ++c) {
    const std::vector<int>& sub = cls_order[c];
    if (sub.empty()) continue;
    const int cnt = (int)sub.size();
    if (cudaMemcpyAsync(d_sub, sub.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = APSP_ECUDA;
      break;
    }
    const int grid = std::min(b->grid, cnt);
    float best = 0.f;
    for (int rows : kTuneRows) {
      float t = 0.f;
      for (int rep = 0; rep < 3 && st == APSP_OK; ++rep) {  // the first run warms up
        cudaMemsetAsync(b->d_queue, 0, sizeof(BatchQueue), s);
        cudaEventRecord(e0, s);
        fw_batched_kernel<<<grid, kBThreads, b->smem, s>>>(b->d_graphs, d_sub, cnt, b->d_queue, b->sp, rows);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          st = APSP_ECUDA;
        if (rep > 0) t += ms;
      }
      if (st != APSP_OK) break;
      if (chosen[c] < 0 || t < best) {
        best = t;
        chosen[c] = rows;
      }
    }
  }
  if (st == APSP_OK) {
    for (BatchGraph& g : b->hg) {
      const int ch = chosen[tune_class(g.n)];
      g.ph3_rows = ch > 0 ? ch : default_ph3_rows(g.n);
    }
    if (cudaMemcpyAsync(b->d_graphs, b->hg.data(), sizeof(BatchGraph) * b->count, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = APSP_ECUDA;
  }
  if (rows_out)
    for (int c = 0; c < kTuneClasses; ++c) rows_out[c] = chosen[c];
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_sub) cudaFree(d_sub);
  if (st != APSP_OK) cudaGetLastError();
  return st;
}

extern "C" apsp_status apsp_batch_destroy(apsp_batch* b) { return batch_free(b); }

namespace apsp {

// Asynchronous one-shot batch for callers that already validated the graphs
// (the server): descriptor table, order and queue go into one stream-ordered
// allocation that is released on the same stream after the kernel.
// host_graphs must be page-locked and stay valid until the stream passes it.
apsp_status batch_launch_async(const BatchGraphDesc* host_graphs, int count, cudaStream_t s) {
  if (count < 1) return APSP_OK;
  int n_max = 1;
  for (int g = 0; g < count; ++g) {
    if (host_graphs[g].n < 1 || host_graphs[g].n > kBMaxN) return APSP_EINVAL;
    n_max = std::max(n_max, host_graphs[g].n);
  }
  static_assert(sizeof(BatchGraphDesc) == sizeof(BatchGraph), "descriptor layouts differ");
  const size_t tbl = sizeof(BatchGraph) * count, ord = sizeof(int) * count;
  const size_t bytes = ((tbl + 255) & ~(size_t)255) + ((ord + 255) & ~(size_t)255) + 256;
  char* buf = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&buf), bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return APSP_ENOMEM;
  }
  BatchGraph* d_graphs = reinterpret_cast<BatchGraph*>(buf);
  int* d_order = reinterpret_cast<int*>(buf + ((tbl + 255) & ~(size_t)255));
  BatchQueue* d_q = reinterpret_cast<BatchQueue*>(buf + ((tbl + 255) & ~(size_t)255) + ((ord + 255) & ~(size_t)255));
  // host_graphs is already in the caller's order; the order array is the identity
  // (the caller sorts largest first). It is written from a page-locked table
  // that follows the descriptors in the caller's staging block.
  const int* host_order = reinterpret_cast<const int*>(host_graphs + count);
  cudaError_t e = cudaMemcpyAsync(d_graphs, host_graphs, tbl, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, host_order, ord, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_q, 0, sizeof(BatchQueue), s);
  const size_t smem = batched_smem_bytes(n_max);
  if (e == cudaSuccess) e = batched_kernel_attributes();
  if (e == cudaSuccess) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_batched_kernel, kBThreads, smem);
    const int grid = std::max(1, std::min(count, std::max(1, per_sm) * sm_count()));
    fw_batched_kernel<<<grid, kBThreads, smem, s>>>(d_graphs, d_order, count, d_q, batched_sp(n_max), 0);
    e = cudaGetLastError();
  }
  cudaFreeAsync(buf, s);
  return e == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

}  // namespace apsp

extern "C" apsp_status apsp_fw_batched(const float* const* W, float* const* D, int32_t* const* P, const int* n,
                                       int count, const apsp_options* opt, int* bs_used, void* stream) {
  apsp_batch* b = nullptr;
  apsp_status st = apsp_batch_create(W, D, P, n, count, opt, &b, stream);
  if (st != APSP_OK) return st;
  st = apsp_batch_launch(b, stream);
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && st == APSP_OK) st = APSP_ECUDA;
  batch_free(b);
  if (st == APSP_OK && bs_used)
    for (int g = 0; g < count; ++g) bs_used[g] = kBBS;
  return st;
}
