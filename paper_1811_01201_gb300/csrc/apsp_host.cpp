// Host-side helpers of the C ABI (no device code).
#include <cstdint>
#include <vector>

#include "../../include/apsp.h"

// Path walk on a host copy of P: P[i][j] is the most recently added
// intermediate vertex (Section 3 of arXiv 1811.01201), so the path splits as
// path(i, P[i][j]) ++ path(P[i][j], j); P == -1 is the direct edge. Iterative
// with an explicit stack; rejects malformed matrices instead of looping.
extern "C" int apsp_path(const int32_t* P, int n, int i, int j, int32_t* out, int cap) {
  if (!P || !out || n < 1 || cap < 1 || i < 0 || j < 0 || i >= n || j >= n) return -1;
  const int64_t limit = cap < n ? cap : n;
  int cnt = 0;
  out[cnt++] = i;
  if (i == j) return cnt;
  std::vector<int32_t> st;
  st.reserve(64);
  st.push_back(i);
  st.push_back(j);
  int64_t steps = 0;
  while (!st.empty()) {
    if (++steps > 4 * (int64_t)n + 8) return -1;
    const int32_t b = st.back(); st.pop_back();
    const int32_t a = st.back(); st.pop_back();
    const int32_t k = P[(int64_t)a * n + b];
    if (k == -1) {
      if (cnt >= limit) return -1;
      out[cnt++] = b;
    } else {
      if (k < 0 || k >= n || k == a || k == b) return -1;
      st.push_back(k); st.push_back(b);  // expanded second
      st.push_back(a); st.push_back(k);  // expanded first
    }
  }
  return cnt;
}
