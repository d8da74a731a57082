/* Serial CPU oracle for blocked Floyd-Warshall (arXiv 1811.01201).
 * Test infrastructure only: never linked into the CUDA library. */
#ifndef APSP_ORACLE_H
#define APSP_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif
void oracle_fw_naive(const float* W, int n, float* D, int32_t* P);
void oracle_fw_blocked(const float* W, int n, int bs, float* D, int32_t* P);
void oracle_dijkstra(const float* W, int n, int src, double* dist);
void oracle_bellman_ford(const float* W, int n, int src, double* dist);
int oracle_path(const int32_t* P, int n, int i, int j, int32_t* out, int cap);
int64_t oracle_check_paths(const float* W, const float* D, const int32_t* P, int n, const int32_t* pairs,
                           int64_t npairs, double rtol);
int64_t oracle_check_invariants(const float* W, const float* D, int n, double rtol);
int64_t oracle_check_bellman_row(const float* W, const float* Drow, int n, double rtol);
#ifdef __cplusplus
}
#endif
#endif
