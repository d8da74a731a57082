// Many small graphs in one persistent launch: one CTA runs the whole blocked
// Floyd-Warshall of one graph (Section 4.1 of arXiv 1811.01201: R rounds of
// diagonal block, row/column blocks, remaining blocks), then takes the next
// graph from a device work queue (largest first).
//
// Block size BS = 32; the last block is clipped to n (equivalent to padding
// with isolated vertices), so results equal the single-graph path with
// BS = 32 bit for bit.
//
// Per round, inside the CTA:
//  * phase 1: the 32x32 diagonal tile in shared memory, one barrier per k; a
//    thread updates its two elements only on strict improvement, so row k and
//    column k (which cannot improve at step k because D[k][k] = 0) are never
//    written during step k.
//  * phase 2: one warp per line -- a column of the row panel or a row of the
//    column panel. Lane t holds element t of the line and the matching row
//    (or column) of the diagonal tile in registers; step k broadcasts the
//    line's element k with a shuffle, and each lane applies the strict-'<'
//    update with its path entry. The finished lines are written to global
//    memory and into the shared panels phase 3 reads.
//  * phase 3: every element outside row/column band r relaxes through the 32
//    panel entries (no barriers: the panels are fixed). Keyed graphs use
//    TR x 128 tiles (TR = 128, 64 or 32, chosen per graph by the host's
//    autotuner), others 4x4 elements per thread per 64x128 tile.
//
// Exact P at one FADD + FMNMX per phase-3 update: for graphs whose weights are
// all integers and whose longest possible path keeps every key below 2^24,
// phase 3 runs on keys M*d + slot (M = 64): the column panel carries slot
// k+1, the old value slot 0. min over keys then reproduces the strict-'<'
// sweep exactly (the old value wins ties; among equal new values the smallest
// k). Other graphs use a warp-cooperative first-k search for the improved
// elements of phase 3.
#pragma once

#include "fw_common.cuh"

namespace apsp {

constexpr int kBBS = 32;         // batched block size
constexpr int kBThreads = 512;   // threads per CTA
constexpr int kBMaxN = 512;      // largest graph order of the batched kernel
constexpr float kBKeyM = 64.f;   // key scale (power of two > BS)

struct BatchGraph {
  const float* W;
  float* D;
  int32_t* P;
  int n;
  int ph3_rows;  // phase-3 tile height on keyed graphs: 128, 64 or 32 (0 = 128); set by the autotuner
};

struct BatchQueue {
  unsigned int next;     // next index into the order array
  unsigned int done;     // graphs finished
};

// Shared-memory layout (floats): diag[32][33], gR[32][36], gC[32][36], As[32][ldp], Bs[32][ldp]
constexpr int kBG = 36;  // row stride of the key-form diagonal copies (16-byte aligned rows)
__host__ __device__ constexpr int batched_ldp(int n_max) { return ((n_max + 31) / 32) * 32 + 8; }
__host__ __device__ constexpr size_t batched_smem_bytes(int n_max) {
  return sizeof(float) * ((size_t)32 * 33 + 2 * (size_t)32 * kBG + 2 * (size_t)32 * batched_ldp(n_max)) + 64;
}

__device__ __forceinline__ float floor_small(float v) {
  // floor for 0 <= v < 2^23 on the FMA pipe: round-down add of 2^23, then subtract
  return __fsub_rn(__fadd_rd(v, 8388608.f), 8388608.f);
}

__device__ __forceinline__ float key_floor(float key) {
  // M * floor(key / M): the value part of a key (exact for integer keys < 2^24; INF stays INF)
  return floor_small(key * (1.f / kBKeyM)) * kBKeyM;
}

// Phase-3 tile of keyed graphs: TR rows x 128 columns, 16 x 32 threads with
// TR/16 x 4 elements each (TR = 128, 64 or 32).
template <bool KEYED, int TR>
__device__ __forceinline__ void batched_graph(const BatchGraph& g, float* sm, int ldp) {
  float* diag = sm;                 // [32][33]
  float* gR = sm + 32 * 33;         // gR[k * kBG + i] = M * diag[i][k] + k + 1   (key form, row-panel lines)
  float* gC = gR + 32 * kBG;        // gC[k * kBG + j] = M * diag[k][j] + k + 1   (key form, column-panel lines)
  float* As = gC + 32 * kBG;        // As[k * ldp + i] = D[i][kb + k]   (column panel, transposed)
  float* Bs = As + 32 * ldp;        // Bs[k * ldp + j] = D[kb + k][j]   (row panel)
  const int n = g.n;
  float* __restrict__ D = g.D;
  int32_t* __restrict__ P = g.P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kBThreads / 32;
  const float INF = f32_inf();
  const int R = (n + kBBS - 1) / kBBS;

  for (int r = 0; r < R; ++r) {
    const int kb = r * kBBS;
    const int kw = min(kBBS, n - kb);

    // ---------------- phase 1: diagonal tile (padded with isolated vertices)
    for (int t = tid; t < 32 * 32; t += kBThreads) {
      const int i = t >> 5, j = t & 31;
      float v;
      if (i < kw && j < kw) v = D[(size_t)(kb + i) * n + kb + j];
      else v = (i == j) ? 0.f : INF;
      diag[i * 33 + j] = v;
    }
    __syncthreads();
    {
      const int i = tid >> 4, j0 = (tid & 15) * 2;  // 512 threads x 2 elements
      int32_t p0 = -1, p1 = -1;
      for (int k = 0; k < kBBS; ++k) {
        const float a = diag[i * 33 + k];
        const float c0 = __fadd_rn(a, diag[k * 33 + j0]);
        const float c1 = __fadd_rn(a, diag[k * 33 + j0 + 1]);
        if (c0 < diag[i * 33 + j0]) { diag[i * 33 + j0] = c0; p0 = kb + k; }
        if (c1 < diag[i * 33 + j0 + 1]) { diag[i * 33 + j0 + 1] = c1; p1 = kb + k; }
        __syncthreads();
      }
      if (i < kw) {
        if (p0 >= 0 && j0 < kw) { D[(size_t)(kb + i) * n + kb + j0] = diag[i * 33 + j0]; P[(size_t)(kb + i) * n + kb + j0] = p0; }
        if (p1 >= 0 && j0 + 1 < kw) { D[(size_t)(kb + i) * n + kb + j0 + 1] = diag[i * 33 + j0 + 1]; P[(size_t)(kb + i) * n + kb + j0 + 1] = p1; }
      }
    }
    // diagonal block entries of the panels (rows/cols in band r); in key form
    // the column panel carries slot k+1 and both are scaled by M
    for (int t = tid; t < 32 * 32; t += kBThreads) {
      const int k = t >> 5, x = t & 31;
      if (x < kw) {
        const float av = diag[x * 33 + k];  // D[kb+x][kb+k]
        const float bv = diag[k * 33 + x];  // D[kb+k][kb+x]
        As[k * ldp + kb + x] = KEYED ? fmaf(av, kBKeyM, (float)(k + 1)) : av;
        Bs[k * ldp + kb + x] = KEYED ? bv * kBKeyM : bv;
      }
    }

    // ---------------- phase 2: lines of the row and column panels
    if (KEYED) {
      // key-form copies of the diagonal tile, then one thread per line with the
      // line's 32 keys in registers: step k adds the line's own value part at k
      for (int t = tid; t < 32 * 32; t += kBThreads) {
        const int k = t >> 5, x = t & 31;
        gR[k * kBG + x] = fmaf(diag[x * 33 + k], kBKeyM, (float)(k + 1));
        gC[k * kBG + x] = fmaf(diag[k * 33 + x], kBKeyM, (float)(k + 1));
      }
      __syncthreads();
      const int nl = n - kw;
      for (int l = tid; l < 2 * nl; l += kBThreads) {
        const bool rowp = l < nl;  // row-panel column o, else column-panel row o
        int o = rowp ? l : l - nl;
        o = o < kb ? o : o + kw;
        const size_t base = rowp ? (size_t)kb * n + o : (size_t)o * n + kb;
        const size_t stride = rowp ? (size_t)n : 1;
        const float* g = rowp ? gR : gC;
        float x[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) x[t] = t < kw ? D[base + t * stride] * kBKeyM : INF;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const float xk = key_floor(x[k]);
#pragma unroll
          for (int t = 0; t < 32; t += 4) {
            const float4 g4 = *reinterpret_cast<const float4*>(g + k * kBG + t);
            x[t] = fminf(x[t], __fadd_rn(g4.x, xk));
            x[t + 1] = fminf(x[t + 1], __fadd_rn(g4.y, xk));
            x[t + 2] = fminf(x[t + 2], __fadd_rn(g4.z, xk));
            x[t + 3] = fminf(x[t + 3], __fadd_rn(g4.w, xk));
          }
        }
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          float v = INF;
          if (t < kw) {
            const float key = x[t];
            if (key < INF) {
              v = floor_small(key * (1.f / kBKeyM));
              const int sl = (int)__fmaf_rn(-v, kBKeyM, key);
              if (sl != 0) {
                D[base + t * stride] = v;
                P[base + t * stride] = kb + sl - 1;
              }
            }
          }
          if (rowp) Bs[t * ldp + o] = v * kBKeyM;
          else As[t * ldp + o] = fmaf(v, kBKeyM, (float)(t + 1));
        }
      }
    } else {
      // lane t: row t of the diagonal tile (row-panel lines) and column t (column-panel lines)
      float drow[32], dcol[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        drow[k] = diag[lane * 33 + k];
        dcol[k] = diag[k * 33 + lane];
      }
      const int nl = n - kw;  // lines per panel
      const bool valid = lane < kw;
      // row-panel column o: element t = D[kb+t][o]; c_t = Diag[t][k] + x_k
      for (int l = warp; l < nl; l += NW) {
        const int o = l < kb ? l : l + kw;
        const size_t off = (size_t)(kb + lane) * n + o;
        float x = valid ? D[off] : INF;
        int32_t p = -1;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const float c = __fadd_rn(drow[k], __shfl_sync(0xffffffffu, x, k));
          if (c < x) { x = c; p = kb + k; }
        }
        if (valid && p >= 0) { D[off] = x; P[off] = p; }
        Bs[lane * ldp + o] = valid ? x : INF;
      }
      // column-panel row o: element t = D[o][kb+t]; c_t = x_k + Diag[k][t]
      for (int l = warp; l < nl; l += NW) {
        const int o = l < kb ? l : l + kw;
        const size_t off = (size_t)o * n + kb + lane;
        float x = valid ? D[off] : INF;
        int32_t p = -1;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const float c = __fadd_rn(__shfl_sync(0xffffffffu, x, k), dcol[k]);
          if (c < x) { x = c; p = kb + k; }
        }
        if (valid && p >= 0) { D[off] = x; P[off] = p; }
        As[lane * ldp + o] = valid ? x : INF;
      }
    }
    __syncthreads();

    // ---------------- phase 3: every element outside band r
    if (R > 1 && KEYED) {
      // 16 x 32 threads, RA x 4 elements each: TR x 128 tiles; the next tile's
      // elements are loaded while the current one computes
      constexpr int RA = TR / 16;
      const int ty = tid >> 5, tx = lane;
      const int tiles_r = (n + TR - 1) / TR, tiles_c = (n + 127) / 128;
      const int ntile = tiles_r * tiles_c;
      float nxt[RA][4];
      auto load_tile = [&](int tile) {
        const int tr = tile / tiles_c, tc = tile - tr * tiles_c;
        const int i0 = tr * TR + ty * RA, j0 = tc * 128 + tx * 4;
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = i0 + a, j = j0 + c;
            nxt[a][c] = (i < n && j < n) ? D[(size_t)i * n + j] : INF;
          }
      };
      load_tile(0);
      for (int tile = 0; tile < ntile; ++tile) {
        const int tr = tile / tiles_c, tc = tile - tr * tiles_c;
        const int i0 = tr * TR + ty * RA, j0 = tc * 128 + tx * 4;
        float d[RA][4];
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) d[a][c] = nxt[a][c] * kBKeyM;
        if (tile + 1 < ntile) load_tile(tile + 1);
        if (i0 < n && j0 < n) {
          const float* Ap = As + i0;
          const float* Bp = Bs + j0;
#pragma unroll 8
          for (int k = 0; k < kBBS; ++k) {
            float av[RA];
            if constexpr (RA == 8) {
              const float4 a0 = *reinterpret_cast<const float4*>(Ap + k * ldp);
              const float4 a1 = *reinterpret_cast<const float4*>(Ap + k * ldp + 4);
              av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
              av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
            } else if constexpr (RA == 4) {
              const float4 a0 = *reinterpret_cast<const float4*>(Ap + k * ldp);
              av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
            } else {
              const float2 a0 = *reinterpret_cast<const float2*>(Ap + k * ldp);
              av[0] = a0.x; av[1] = a0.y;
            }
            const float4 b4 = *reinterpret_cast<const float4*>(Bp + k * ldp);
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) d[a][c] = fminf(d[a][c], __fadd_rn(av[a], bv[c]));
          }
          // slot 0 = unchanged; slot s = improved at k = s-1
#pragma unroll
          for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int i = i0 + a, j = j0 + c;
              const float key = d[a][c];
              if (i >= n || j >= n || !(key < INF)) continue;
              if ((i >= kb && i < kb + kw) || (j >= kb && j < kb + kw)) continue;
              const float v = floor_small(key * (1.f / kBKeyM));
              const int sl = (int)__fmaf_rn(-v, kBKeyM, key);
              if (sl != 0) {
                D[(size_t)i * n + j] = v;
                P[(size_t)i * n + j] = kb + sl - 1;
              }
            }
        }
      }
    } else if (R > 1) {
      const int ty = tid >> 5, tx = lane;  // 16 x 32 threads, 4 x 4 elements each: 64 x 128 tile
      const int tiles_r = (n + 63) / 64, tiles_c = (n + 127) / 128;
      for (int tile = 0; tile < tiles_r * tiles_c; ++tile) {
        const int tr = tile / tiles_c, tc = tile - tr * tiles_c;
        const int i0 = tr * 64 + ty * 4, j0 = tc * 128 + tx * 4;
        const bool any_row = i0 < n, any_col = j0 < n;
        float d[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = i0 + a, j = j0 + c;
            d[a][c] = (i < n && j < n) ? D[(size_t)i * n + j] : INF;
          }
        const float old[4][4] = {{d[0][0], d[0][1], d[0][2], d[0][3]}, {d[1][0], d[1][1], d[1][2], d[1][3]},
                                 {d[2][0], d[2][1], d[2][2], d[2][3]}, {d[3][0], d[3][1], d[3][2], d[3][3]}};
        if (any_row && any_col) {
          const float* Ap = As + i0;
          const float* Bp = Bs + j0;
#pragma unroll 8
          for (int k = 0; k < kBBS; ++k) {
            const float4 a4 = *reinterpret_cast<const float4*>(Ap + k * ldp);
            const float4 b4 = *reinterpret_cast<const float4*>(Bp + k * ldp);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) d[a][c] = fminf(d[a][c], __fadd_rn(av[a], bv[c]));
          }
        }
        uint32_t imp = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = i0 + a, j = j0 + c;
            const bool inside = i < n && j < n && !(i >= kb && i < kb + kw) && !(j >= kb && j < kb + kw);
            if (inside && d[a][c] < old[a][c]) {
              D[(size_t)i * n + j] = d[a][c];
              imp |= 1u << (a * 4 + c);
            }
          }
        if (__any_sync(0xffffffffu, imp != 0)) {
#pragma unroll
          for (int slot = 0; slot < 16; ++slot) {
            unsigned bal = __ballot_sync(0xffffffffu, (imp >> slot) & 1);
            const float dmine = d[slot >> 2][slot & 3];
            while (bal) {
              const int src = __ffs(bal) - 1;
              bal &= bal - 1;
              const int li = i0 + (slot >> 2);                 // same ty for the whole warp
              const int lj = tc * 128 + src * 4 + (slot & 3);
              const float dn = __shfl_sync(0xffffffffu, dmine, src);
              const float cand = __fadd_rn(As[lane * ldp + li], Bs[lane * ldp + lj]);
              const unsigned eq = __ballot_sync(0xffffffffu, cand == dn);
              if (lane == src) P[(size_t)li * n + lj] = kb + __ffs(eq) - 1;
            }
          }
        }
      }
    }
    __syncthreads();  // D and the shared panels are reused by the next round
  }
}

// Persistent kernel: each CTA repeatedly takes the next graph (largest first).
// force_rows != 0 overrides every graph's phase-3 tile height (autotuning runs).
__global__ void __launch_bounds__(kBThreads, 1) fw_batched_kernel(const BatchGraph* __restrict__ graphs,
                                                                  const int* __restrict__ order, int count,
                                                                  BatchQueue* q, int ldp, int force_rows) {
  extern __shared__ __align__(16) float smb[];
  __shared__ int s_g, s_keyed;
  __shared__ unsigned s_frac, s_max;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned idx = atomicAdd(&q->next, 1u);
      s_g = idx < (unsigned)count ? order[idx] : -1;
      s_frac = 0;
      s_max = 0;
    }
    __syncthreads();
    const int gi = s_g;
    if (gi < 0) return;
    const BatchGraph g = graphs[gi];
    const int n = g.n;
    // initialise D = W (zero diagonal), P = -1; find integrality and the largest finite weight
    unsigned frac = 0, mx = 0;
    const size_t nn = (size_t)n * n;
    constexpr int kInitUnroll = 8;  // loads of a thread in flight together
    for (size_t t0 = threadIdx.x; t0 < nn; t0 += (size_t)kInitUnroll * kBThreads) {
      float w[kInitUnroll];
#pragma unroll
      for (int u = 0; u < kInitUnroll; ++u) {
        const size_t t = t0 + (size_t)u * kBThreads;
        w[u] = t < nn ? g.W[t] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kInitUnroll; ++u) {
        const size_t t = t0 + (size_t)u * kBThreads;
        if (t < nn) {
          const size_t i = t / n, j = t - i * n;
          float v = w[u];
          if (i == j) v = 0.f;
          if (v < f32_inf()) {
            frac |= (v != floorf(v));
            mx = max(mx, (unsigned)__float_as_int(v));
          }
          g.D[t] = v;
          g.P[t] = -1;
        }
      }
    }
    if (frac) s_frac = 1;
    atomicMax(&s_max, mx);
    __syncthreads();
    if (threadIdx.x == 0) {
      // keys stay exact while every path length (< n * max_w) plus a panel sum keeps M*(sum) + 32 < 2^24
      const float mw = __int_as_float((int)s_max);
      s_keyed = (s_frac == 0) && (2.0f * mw * (float)n <= 262000.0f);
    }
    __syncthreads();
    const int rows = force_rows ? force_rows : g.ph3_rows;
    if (!s_keyed) batched_graph<false, 128>(g, smb, ldp);
    else if (rows == 32) batched_graph<true, 32>(g, smb, ldp);
    else if (rows == 64) batched_graph<true, 64>(g, smb, ldp);
    else batched_graph<true, 128>(g, smb, ldp);
    if (threadIdx.x == 0) atomicAdd(&q->done, 1u);
    __syncthreads();
  }
}

}  // namespace apsp
