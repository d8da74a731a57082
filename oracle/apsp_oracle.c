/*
 * Serial CPU oracle for blocked Floyd-Warshall all-pairs shortest paths
 * (Rucci, De Giusti, Naiouf, "Blocked All-Pairs Shortest Paths Algorithm on
 * Intel Xeon Phi KNL Processor: A Case Study", arXiv 1811.01201).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * restatement of the method that the CUDA library is checked against. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the library itself never calls it and shares no code with it.
 *
 * Arithmetic: IEEE-754 binary32, round-to-nearest, built with
 * -ffp-contract=off and without -ffast-math, so every candidate D[i][k]+D[k][j]
 * is one correctly rounded fp32 addition, exactly as on the GPU.
 *
 * Readings of the paper taken here (the figures holding its pseudo-code are
 * missing from the text, so the algorithm is rebuilt from the prose):
 *  - Relaxation uses a strict '<' (Section 4.2: the loop body is one addition,
 *    one comparison and at most two assignments): on a tie the existing
 *    distance and its path entry are kept.
 *  - P[i][j] holds the most recently added intermediate vertex (Section 3),
 *    as a global vertex index; -1 means "direct edge, i==j, or unreachable".
 *  - D starts as the input weights with the diagonal forced to 0; absent edges
 *    are +INF, and INF + x == INF, INF < INF is false.
 *  - A last block that is cut short by n is clipped to n (equivalent to
 *    padding with isolated vertices).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "apsp_oracle.h"

static void init_dp(const float* W, int64_t n, float* D, int32_t* P) {
  /* Section 3: D is initialised with the original distances; P records
   * intermediates, so it starts empty (-1). The diagonal is forced to 0. */
  if (D != W) memcpy(D, W, (size_t)(n * n) * sizeof(float));
  for (int64_t i = 0; i < n * n; ++i) P[i] = -1;
  for (int64_t i = 0; i < n; ++i) D[i * n + i] = 0.0f;
}

/* Naive Floyd-Warshall (Section 3, Fig. 1): N iterations of k, each relaxing
 * every pair (i, j) through intermediate vertex k. */
void oracle_fw_naive(const float* W, int n_, float* D, int32_t* P) {
  const int64_t n = n_;
  init_dp(W, n, D, P);
  for (int64_t k = 0; k < n; ++k)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        float c = D[i * n + k] + D[k * n + j];
        if (c < D[i * n + j]) {
          D[i * n + j] = c;
          P[i * n + j] = (int32_t)k;
        }
      }
}

/* FW_BLOCK(C, A, B) of Section 4.1 / Fig. 3 with C = block (bi, bj),
 * A = block (bi, r), B = block (r, bj), all views into D: for every k of block
 * r in ascending order, for every i of row-block bi, for every j of
 * column-block bj, relax C[i][j] through A[i][k] + B[k][j]. */
static void fw_block(float* D, int32_t* P, int64_t n, int64_t bs, int64_t bi, int64_t bj, int64_t r) {
  const int64_t k0 = r * bs, k1 = (k0 + bs < n) ? k0 + bs : n;
  const int64_t i0 = bi * bs, i1 = (i0 + bs < n) ? i0 + bs : n;
  const int64_t j0 = bj * bs, j1 = (j0 + bs < n) ? j0 + bs : n;
  for (int64_t k = k0; k < k1; ++k)
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t j = j0; j < j1; ++j) {
        float c = D[i * n + k] + D[k * n + j];
        if (c < D[i * n + j]) {
          D[i * n + j] = c;
          P[i * n + j] = (int32_t)k;
        }
      }
}

/* Blocked Floyd-Warshall (Section 4.1, Fig. 2-3): R = ceil(N/BS) rounds, each
 * in four phases: (1) the self-dependent diagonal block (r,r); (2) the other
 * blocks of row r, which depend on themselves and block (r,r); (3) the other
 * blocks of column r, likewise; (4) every remaining block (i,j), which depends
 * on block (i,r) of its row and block (r,j) of its column. */
void oracle_fw_blocked(const float* W, int n_, int bs_, float* D, int32_t* P) {
  const int64_t n = n_, bs = bs_;
  const int64_t R = (n + bs - 1) / bs;
  init_dp(W, n, D, P);
  for (int64_t r = 0; r < R; ++r) {
    fw_block(D, P, n, bs, r, r, r);                                  /* phase 1 */
    for (int64_t j = 0; j < R; ++j)
      if (j != r) fw_block(D, P, n, bs, r, j, r);                    /* phase 2 */
    for (int64_t i = 0; i < R; ++i)
      if (i != r) fw_block(D, P, n, bs, i, r, r);                    /* phase 3 */
    for (int64_t i = 0; i < R; ++i)
      if (i != r)
        for (int64_t j = 0; j < R; ++j)
          if (j != r) fw_block(D, P, n, bs, i, j, r);                /* phase 4 */
  }
}

/* Textbook dense Dijkstra from one source, in double precision: the exact
 * shortest distance for non-negative weights (a check of the oracle above,
 * not part of the paper's method). */
void oracle_dijkstra(const float* W, int n_, int src, double* dist) {
  const int64_t n = n_;
  char* done = (char*)calloc((size_t)n, 1);
  for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
  dist[src] = 0.0;
  for (int64_t it = 0; it < n; ++it) {
    int64_t u = -1;
    double best = INFINITY;
    for (int64_t v = 0; v < n; ++v)
      if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
    if (u < 0) break;
    done[u] = 1;
    const float* row = W + u * n;
    for (int64_t v = 0; v < n; ++v) {
      if (v == u) continue;
      double c = dist[u] + (double)row[v];
      if (c < dist[v]) dist[v] = c;
    }
  }
  free(done);
}

/* Textbook Bellman-Ford from one source, double precision. */
void oracle_bellman_ford(const float* W, int n_, int src, double* dist) {
  const int64_t n = n_;
  for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
  dist[src] = 0.0;
  for (int64_t pass = 0; pass + 1 < n; ++pass) {
    int changed = 0;
    for (int64_t u = 0; u < n; ++u) {
      if (dist[u] == INFINITY) continue;
      for (int64_t v = 0; v < n; ++v) {
        if (v == u) continue;
        double c = dist[u] + (double)W[u * n + v];
        if (c < dist[v]) { dist[v] = c; changed = 1; }
      }
    }
    if (!changed) break;
  }
}

/* Reconstruct the path i -> j from P (Section 3: P[i][j] is the most recently
 * added intermediate vertex; the paper does not print the walk, so the
 * standard split path(i,j) = path(i,P[i][j]) ++ path(P[i][j],j) is used, with
 * P == -1 meaning the direct edge). Writes the vertices i..j into out and
 * returns their count, or -1 if the walk is malformed or longer than
 * min(cap, n) vertices. */
int oracle_path(const int32_t* P, int n_, int i, int j, int32_t* out, int cap) {
  const int64_t n = n_;
  if (i < 0 || j < 0 || i >= n || j >= n || cap < 1) return -1;
  int64_t limit = cap < n ? cap : n;
  int cnt = 0;
  out[cnt++] = i;
  if (i == j) return cnt;
  /* explicit stack of (a, b) sub-walks still to expand, deepest last */
  int64_t sc = 2 * n + 4;
  int32_t* st = (int32_t*)malloc((size_t)sc * 2 * sizeof(int32_t));
  int64_t sp = 0;
  st[0] = i; st[1] = j; sp = 1;
  int64_t steps = 0;
  while (sp > 0) {
    if (++steps > 4 * n + 8) { cnt = -1; break; }
    --sp;
    int32_t a = st[2 * sp], b = st[2 * sp + 1];
    int32_t k = P[(int64_t)a * n + b];
    if (k == -1) {
      if (cnt >= limit) { cnt = -1; break; }
      out[cnt++] = b;
    } else {
      if (k < 0 || k >= n || k == a || k == b || sp + 2 > sc) { cnt = -1; break; }
      st[2 * sp] = k; st[2 * sp + 1] = b; ++sp;   /* expanded second */
      st[2 * sp] = a; st[2 * sp + 1] = k; ++sp;   /* expanded first */
    }
  }
  free(st);
  return cnt;
}

/* Walk P for each (i, j) pair and check it against W and D: the walk starts at
 * i, ends at j, visits distinct vertices, uses only present edges, and its
 * weight (summed in double) equals D[i][j] within rtol (0 = exactly). An
 * unreachable pair must have D == +INF and P == -1. Returns the number of
 * failing pairs. */
int64_t oracle_check_paths(const float* W, const float* D, const int32_t* P, int n_, const int32_t* pairs,
                           int64_t npairs, double rtol) {
  const int64_t n = n_;
  int32_t* path = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  char* seen = (char*)calloc((size_t)n, 1);
  int64_t bad = 0;
  for (int64_t q = 0; q < npairs; ++q) {
    int32_t i = pairs[2 * q], j = pairs[2 * q + 1];
    float d = D[(int64_t)i * n + j];
    if (i == j) {
      if (d != 0.0f || P[(int64_t)i * n + j] != -1) ++bad;
      continue;
    }
    if (isinf(d)) {
      if (P[(int64_t)i * n + j] != -1 || !isinf(W[(int64_t)i * n + j])) ++bad;
      continue;
    }
    int cnt = oracle_path(P, n_, i, j, path, n_);
    if (cnt < 2 || path[0] != i || path[cnt - 1] != j) { ++bad; continue; }
    double sum = 0.0;
    int ok = 1;
    for (int t = 0; t < cnt; ++t) {
      if (seen[path[t]]) ok = 0;
      seen[path[t]] = 1;
    }
    for (int t = 0; t < cnt; ++t) seen[path[t]] = 0;
    for (int t = 0; ok && t + 1 < cnt; ++t) {
      float w = W[(int64_t)path[t] * n + path[t + 1]];
      if (isinf(w)) ok = 0;
      sum += (double)w;
    }
    if (ok) {
      double dd = (double)d;
      double tol = rtol * fabs(dd);
      if (!(fabs(sum - dd) <= tol)) ok = 0;
    }
    if (!ok) ++bad;
  }
  free(seen);
  free(path);
  return bad;
}

/* Invariants of a finished APSP distance matrix: D[i][i] == 0, D <= W
 * elementwise, and the triangle inequality D[i][j] <= D[i][k] + D[k][j] for
 * all k (checked as D[i][j] <= (D[i][k] + D[k][j]) * (1 + rtol) in double).
 * Returns the number of violations. O(n^3): small n only. */
int64_t oracle_check_invariants(const float* W, const float* D, int n_, double rtol) {
  const int64_t n = n_;
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (D[i * n + i] != 0.0f) ++bad;
    for (int64_t j = 0; j < n; ++j)
      if (i != j && D[i * n + j] > W[i * n + j]) ++bad;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = 0; k < n; ++k) {
      double dik = D[i * n + k];
      if (isinf(dik)) continue;
      for (int64_t j = 0; j < n; ++j) {
        double s = dik + (double)D[k * n + j];
        if ((double)D[i * n + j] > s * (1.0 + rtol)) ++bad;
      }
    }
  return bad;
}

/* Bellman optimality certificate for one source row s: D[s][j] <= D[s][k] +
 * W[k][j] for every k, j (within rtol). Together with a path of weight D[s][j]
 * this certifies that row s holds exact shortest distances. Returns the number
 * of violations. O(n^2). */
int64_t oracle_check_bellman_row(const float* W, const float* Drow, int n_, double rtol) {
  const int64_t n = n_;
  int64_t bad = 0;
  for (int64_t k = 0; k < n; ++k) {
    double dk = Drow[k];
    if (isinf(dk)) continue;
    const float* wrow = W + k * n;
    for (int64_t j = 0; j < n; ++j) {
      if (j == k) continue;
      double s = dk + (double)wrow[j];
      if ((double)Drow[j] > s * (1.0 + rtol)) ++bad;
    }
  }
  return bad;
}
