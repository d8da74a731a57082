/*
 * CPU BASELINE: the paper's own blocked design run on the host cores.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the oracle next to it: the
 * benchmark times it beside the GPU library as a parallel CPU baseline, and a
 * test pins it bit for bit to oracle_fw_blocked. The library never calls it.
 *
 * Rucci, De Giusti, Naiouf (arXiv 1811.01201), Section 4: the distance matrix
 * is split into BS x BS blocks and every round r runs the diagonal block
 * alone (phase 1), then the blocks of row r and of column r in parallel
 * (phases 2 and 3, which depend only on the diagonal block), then all other
 * blocks in parallel (phase 4); threads take blocks (OpenMP), the innermost
 * loop over j is vectorised, and the update is branch-free (compare, then
 * select the new distance and path entry). Phase-4 blocks 64 columns wide keep
 * each output row in registers across the block's k.
 *
 * Every element sees the same candidates in the same order (k ascending within
 * each block round) as oracle_fw_blocked, with one correctly rounded fp32
 * addition each (-ffp-contract=off, no -ffast-math) and a strict '<', so D
 * and P equal the oracle's exactly. In-place updates of the diagonal and panel
 * blocks are safe in vector form because row k and column k do not change
 * during step k (D[k][k] == 0).
 */
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Update block C (rows i0.., columns j0..) through the intermediates
 * kb .. kb+kn-1, A = block (rows of C, columns of k), B = block (rows of k,
 * columns of C). All three are views into D (leading dimension n). */
static void block_update(float* D, int32_t* P, int64_t n, int64_t i0, int64_t in, int64_t j0, int64_t jn,
                         int64_t kb, int64_t kn) {
  for (int64_t k = kb; k < kb + kn; ++k) {
    const float* Bk = D + k * n + j0;
    for (int64_t i = i0; i < i0 + in; ++i) {
      const float a = D[i * n + k];
      float* Ci = D + i * n + j0;
      int32_t* Pi = P + i * n + j0;
      const int32_t kk = (int32_t)k;
#pragma omp simd
      for (int64_t j = 0; j < jn; ++j) {
        const float c = a + Bk[j], old = Ci[j];
        const int32_t m = -(int32_t)(c < old);  /* all ones where strictly better */
        Ci[j] = c < old ? c : old;
        Pi[j] = (Pi[j] & ~m) | (kk & m);
      }
    }
  }
}

/* Phase-4 block of full width 64: A and B are fixed during the round, so each
 * output row can run through all k of the block while it stays in registers
 * (i, then k, then j). Every element still sees its candidates with k
 * ascending, so the result equals block_update's. */
#define ROW 64
static void block_update_fixed64(float* D, int32_t* P, int64_t n, int64_t i0, int64_t in, int64_t j0,
                                 int64_t kb, int64_t kn) {
  for (int64_t i = i0; i < i0 + in; ++i) {
    float c[ROW];
    int32_t p[ROW];
    float* Ci = D + i * n + j0;
    int32_t* Pi = P + i * n + j0;
    const float* Ai = D + i * n + kb;
    for (int j = 0; j < ROW; ++j) {
      c[j] = Ci[j];
      p[j] = Pi[j];
    }
    for (int64_t k = 0; k < kn; ++k) {
      const float a = Ai[k];
      const float* Bk = D + (kb + k) * n + j0;
      const int32_t kk = (int32_t)(kb + k);
#pragma omp simd
      for (int j = 0; j < ROW; ++j) {
        const float t = a + Bk[j], old = c[j];
        const int32_t m = -(int32_t)(t < old);
        c[j] = t < old ? t : old;
        p[j] = (p[j] & ~m) | (kk & m);
      }
    }
    for (int j = 0; j < ROW; ++j) {
      Ci[j] = c[j];
      Pi[j] = p[j];
    }
  }
}

int host_fw_blocked_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* D <- W with a zero diagonal, P <- -1, then R = ceil(n / bs) rounds. */
void host_fw_blocked(const float* W, int n_, int bs_, float* D, int32_t* P) {
  const int64_t n = n_, bs = bs_;
  if (n < 1 || bs < 1) return;
  if (D != W) memcpy(D, W, (size_t)(n * n) * sizeof(float));
  for (int64_t t = 0; t < n * n; ++t) P[t] = -1;
  for (int64_t i = 0; i < n; ++i) D[i * n + i] = 0.0f;
  const int64_t R = (n + bs - 1) / bs;
#pragma omp parallel
  for (int64_t r = 0; r < R; ++r) {
    const int64_t kb = r * bs, kn = (n - kb < bs) ? n - kb : bs;
    /* phase 1: the diagonal block, one thread */
#pragma omp single
    block_update(D, P, n, kb, kn, kb, kn, kb, kn);
    /* phases 2 and 3: row r and column r blocks, in parallel */
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < 2 * R; ++t) {
      const int64_t b = t % R;
      if (b == r) continue;
      const int64_t b0 = b * bs, bn = (n - b0 < bs) ? n - b0 : bs;
      if (t < R)
        block_update(D, P, n, kb, kn, b0, bn, kb, kn);   /* block (r, b) */
      else
        block_update(D, P, n, b0, bn, kb, kn, kb, kn);   /* block (b, r) */
    }
    /* phase 4: every other block, in parallel */
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < R * R; ++t) {
      const int64_t bi = t / R, bj = t % R;
      if (bi == r || bj == r) continue;
      const int64_t i0 = bi * bs, in = (n - i0 < bs) ? n - i0 : bs;
      const int64_t j0 = bj * bs, jn = (n - j0 < bs) ? n - j0 : bs;
      if (jn == ROW)
        block_update_fixed64(D, P, n, i0, in, j0, kb, kn);
      else
        block_update(D, P, n, i0, in, j0, jn, kb, kn);
    }
  }
}
