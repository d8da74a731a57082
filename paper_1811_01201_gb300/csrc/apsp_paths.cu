// Batched path reconstruction on the device (C ABI in include/apsp.h).
//
// Section 3 of arXiv 1811.01201: P[i][j] is the intermediate vertex added
// last to the path i -> j, kept so that the path can be rebuilt. The path
// splits as path(i, P[i][j]) ++ path(P[i][j], j); P == -1 is the direct edge.
//
// One thread walks one pair. The walk keeps a stack of pending sub-walk
// targets only: the source of the sub-walk on top is always the vertex written
// last, so (source, target) pairs are not needed. The stack grows down from
// the end of the pair's own output row while the path grows up from its
// start; every stacked target is still to be written, so the two meet only
// when the path would exceed the row's capacity, which is the failure case.
// Each step is one read of P, and a path of L vertices takes 2L - 3 steps.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/apsp.h"

namespace apsp {

constexpr int kPathThreads = 128;

__global__ void __launch_bounds__(kPathThreads) paths_kernel(const int32_t* __restrict__ P, int n,
                                                             const int32_t* __restrict__ pairs, int count,
                                                             int32_t* __restrict__ out, int cap,
                                                             int32_t* __restrict__ len) {
  const int t = blockIdx.x * kPathThreads + threadIdx.x;
  if (t >= count) return;
  const int i = pairs[2 * (size_t)t], j = pairs[2 * (size_t)t + 1];
  if (i < 0 || j < 0 || i >= n || j >= n) {
    len[t] = -1;
    return;
  }
  int32_t* o = out + (size_t)t * cap;
  const int limit = cap < n ? cap : n;
  o[0] = i;
  if (i == j) {
    len[t] = 1;
    return;
  }
  if (limit < 2) {
    len[t] = -1;
    return;
  }
  int cnt = 1, depth = 1, cur = i;
  o[cap - 1] = j;
  while (depth > 0) {
    const int b = o[cap - depth];
    const int k = __ldg(P + (size_t)cur * n + b);
    if (k == -1) {
      o[cnt++] = b;  // cnt + depth <= limit still holds: one moves from the stack to the path
      cur = b;
      --depth;
    } else {
      if (k < 0 || k >= n || k == cur || k == b || cnt + depth + 1 > limit) {
        len[t] = -1;
        return;
      }
      ++depth;
      o[cap - depth] = k;
    }
  }
  len[t] = cnt;
}

}  // namespace apsp

extern "C" apsp_status apsp_paths(const int32_t* P, int n, const int32_t* pairs, int count, int32_t* out, int cap,
                                  int32_t* len, void* stream) {
  if (n < 1 || count < 0 || cap < 1) return APSP_EINVAL;
  if (count == 0) return APSP_OK;
  if (!P || !pairs || !out || !len) return APSP_EINVAL;
  const int blocks = (int)(((int64_t)count + apsp::kPathThreads - 1) / apsp::kPathThreads);
  apsp::paths_kernel<<<blocks, apsp::kPathThreads, 0, (cudaStream_t)stream>>>(P, n, pairs, count, out, cap, len);
  return cudaGetLastError() == cudaSuccess ? APSP_OK : APSP_ECUDA;
}
