// Phases 1 and 2 of a block round: tiles whose update depends on itself.
//
// Section 4.1 of arXiv 1811.01201: in round r the diagonal block (r,r) is
// self-dependent (phase 1); the other blocks of row r and of column r depend
// on themselves and on the finished block (r,r) (paper phases 2 and 3, run
// here as one launch). Each such tile is updated in place by FW_BLOCK: for k
// ascending over block r, every element relaxes through D[i][k] + D[k][j]
// with a strict '<', and P records the global k (Section 4.2, Section 3).
//
// GPU mapping: phase 1 is one CTA holding the diagonal tile in registers, one
// barrier per step; phase 2 is one CTA per panel tile, its lines owned by the
// lanes of a warp, no barrier per step (details at each kernel). Step k needs
// row k and/or column k as they stand after step k-1; neither changes during
// step k, because D[k][k] = 0.
#pragma once

#include <type_traits>

#include "fw_common.cuh"

namespace apsp {

// Phase 1: the diagonal block (kb..kb+BS-1)^2 of round r, updated in place
// through its own intermediates, c = C[i][k] + C[k][j] with k ascending.
// Every thread keeps a TE x TE sub-block in registers; the owners of row k
// and column k publish them into a double-buffered shared row/column, so one
// barrier per step orders the sweep exactly like the serial loop.
//
// (Exact keys, which serve phases 2 and 3, did not pay here: at BS = 32 and
// 64 this sweep is bound by the barrier and shared-memory round trip of each
// step, not by its ALU work.)
template <class T, int BS>
__device__ __forceinline__ void diag_tile(typename T::store_t* __restrict__ D, int32_t* __restrict__ P, size_t ld,
                                          int kb, typename T::reg_t* rowbuf, typename T::reg_t* colbuf, RoundMax* rm,
                                          typename T::reg_t* __restrict__ pk, typename T::reg_t* stage) {
  using S = SeqShape<BS>;
  using reg_t = typename T::reg_t;
  constexpr int TE = S::TE, TPR = S::TPR;
  const int tid = threadIdx.x, tx = tid % TPR, ty = tid / TPR;
  const int li0 = ty * TE, lj0 = tx * TE;

  reg_t d[TE][TE];
  int32_t p[TE][TE];
#pragma unroll
  for (int a = 0; a < TE; ++a)
#pragma unroll
    for (int c = 0; c < TE; ++c) {
      d[a][c] = T::load(D[(size_t)(kb + li0 + a) * ld + kb + lj0 + c]);
      p[a][c] = -1;
    }

  for (int k0 = 0; k0 < BS; k0 += TE) {
#pragma unroll
    for (int kk = 0; kk < TE; ++kk) {
      const int k = k0 + kk;
      reg_t* rb = rowbuf + (k & 1) * BS;
      reg_t* cb = colbuf + (k & 1) * BS;
      if (ty == k0 / TE) {
#pragma unroll
        for (int c = 0; c < TE; ++c) rb[lj0 + c] = d[kk][c];
      }
      if (tx == k0 / TE) {
#pragma unroll
        for (int a = 0; a < TE; ++a) cb[li0 + a] = d[a][kk];
      }
      __syncthreads();
      reg_t av[TE], bv[TE];
#pragma unroll
      for (int a = 0; a < TE; ++a) av[a] = cb[li0 + a];
#pragma unroll
      for (int c = 0; c < TE; ++c) bv[c] = rb[lj0 + c];
#pragma unroll
      for (int a = 0; a < TE; ++a)
#pragma unroll
        for (int c = 0; c < TE; ++c) {
          const reg_t cand = T::add(av[a], bv[c]);
          if (cand < d[a][c]) {
            d[a][c] = cand;
            p[a][c] = kb + k;
          }
        }
    }
  }

#pragma unroll
  for (int a = 0; a < TE; ++a)
#pragma unroll
    for (int c = 0; c < TE; ++c) {
      const size_t off = (size_t)(kb + li0 + a) * ld + kb + lj0 + c;
      if (p[a][c] >= 0) {
        D[off] = T::store(d[a][c]);
        P[off] = p[a][c];
      }
    }
  {
    // The finished tile for phase 2 in both of its layouts (see fw_phase2_kernel):
    // staged in shared memory, then written by two bulk copies.
    constexpr int PS = BS + 4;
    constexpr unsigned kBytes = (unsigned)(sizeof(reg_t) * BS * PS);
#pragma unroll
    for (int a = 0; a < TE; ++a)
#pragma unroll
      for (int c = 0; c < TE; ++c) {
        stage[(lj0 + c) * PS + li0 + a] = d[a][c];            // row panels: [k][i] = diag[i][k]
        stage[BS * PS + (li0 + a) * PS + lj0 + c] = d[a][c];  // column panels: [k][j] = diag[k][j]
      }
    bulk_store_fence();
    __syncthreads();
    if (tid == 0) {
      bulk_copy_s2g_and_wait(pk, stage, kBytes);
      bulk_copy_s2g_and_wait(pk + BS * PS, stage + BS * PS, kBytes);
    }
  }
  // Largest value of the finished tile for phase 3's per-round choice: fp32
  // takes the largest finite value (bit pattern) for the exact-key bound;
  // 16-bit takes the largest value including INF for the overflow test.
  unsigned mx = 0;
#pragma unroll
  for (int a = 0; a < TE; ++a)
#pragma unroll
    for (int c = 0; c < TE; ++c) {
      if constexpr (std::is_same<T, F32T>::value) {
        if (d[a][c] < f32_inf()) mx = max(mx, (unsigned)__float_as_int(d[a][c]));
      } else {
        mx = max(mx, (unsigned)d[a][c]);
      }
    }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&rm->a_bits, mx);
    atomicMax(&rm->b_bits, mx);
  }
}

// pk: receives the finished tile in the two layouts phase 2 copies in
// (2 * BS * (BS + 4) values), staged in dynamic shared memory of that size.
template <class T, int BS>
__global__ void __launch_bounds__(SeqShape<BS>::NT) fw_phase1_kernel(typename T::store_t* D, int32_t* P, size_t ld,
                                                                     int r, RoundMax* rm, typename T::reg_t* pk) {
  __shared__ typename T::reg_t rowbuf[2 * BS], colbuf[2 * BS];
  extern __shared__ __align__(16) unsigned char stage_raw[];
  pdl_prologue();
  const int kb = r * BS;
  if (threadIdx.x == 0) {
    rm->a_bits = 0;  // visible to this CTA's atomics after the tile's barriers
    rm->b_bits = 0;
  }
  diag_tile<T, BS>(D, P, ld, kb, rowbuf, colbuf, rm, pk, reinterpret_cast<typename T::reg_t*>(stage_raw));
}

template <class T, int BS>
constexpr size_t phase1_smem_bytes() {
  return sizeof(typename T::reg_t) * 2 * (size_t)BS * (BS + 4);
}

// Phase 2: the other blocks of row r (CTAs 0 .. R-2) and of column r
// (CTAs R-1 .. 2R-3), all against the finished diagonal block.
//
// Line owners instead of a barrier per step: in a row-panel block (r, J) the
// update c = A[i][k] + C[k][j] keeps column j of C to itself (A is the
// finished diagonal block), and in a column-panel block (I, r) the update
// c = C[i][k] + B[k][j] keeps row i to itself. Each line (column or row of
// the block) is held by TPL lanes of one warp, RPT elements each; the lane
// holding element k of the line passes it to the others with a shuffle, so
// the BS steps need no block barrier. The diagonal block sits in shared
// memory, transposed for row panels, so every lane reads its RPT operands of
// step k as 128-bit loads; phase 1 wrote it in both layouts (pk), and one
// thread pulls the needed one with a bulk copy while the lanes load their
// line elements (bounded wait, as in phase 3: wait_ns, no_copy).
//
// Exact keys (fp32, integer-valued graphs): an element is held as
// M*value + slot (M = 2*BS, slot = local k+1 of its last improvement, 0 for
// none) and step k forms the candidate key M*diag + M*v_k + k + 1 with one
// FFMA, so one FMNMX replaces the compare and the two selects: a smaller
// value wins, and on equal values the older, smaller slot is kept, as the
// strict '<' requires. The finished diagonal block obeys the triangle
// inequality, so an element improves only through a line element that has
// not improved itself; every candidate is therefore at most 2*max(diagonal)
// + max(initial line), and the keys stay exact below 2^24 when that bound
// allows. Each warp checks it for its own lines (the diagonal maximum comes
// from phase 1's round maxima) and runs the key loop or the plain loop. On
// the 16-bit path the keys are 32-bit integers and always exact.
template <int BS>
struct LineShape {
  static constexpr int NT = BS == 128 ? 1024 : 256;  // threads per CTA
  static constexpr int TPL = NT / BS;          // lanes per line
  static constexpr int RPT = BS / TPL;         // elements per lane
  static constexpr int LPW = 32 / TPL;         // lines per warp
  static constexpr int DS = BS + 4;            // shared row stride (16-byte multiple)
  static_assert(TPL * RPT == BS && LPW * TPL == 32 && RPT % 4 == 0, "bad line shape");
};

template <class T, int BS>
__global__ void __launch_bounds__(LineShape<BS>::NT, LineShape<BS>::NT == 1024 ? 1 : 2)
    fw_phase2_kernel(typename T::store_t* D, int32_t* P, size_t ld, int r, int R, RoundMax* rm,
                     const typename T::reg_t* __restrict__ pk, unsigned long long wait_ns, int no_copy,
                     int graph_int) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  using reg_t = typename T::reg_t;
  using L = LineShape<BS>;
  constexpr int RPT = L::RPT, DS = L::DS;
  constexpr unsigned kBytes = (unsigned)(sizeof(reg_t) * BS * DS);
  reg_t* S = reinterpret_cast<reg_t*>(smem_raw);
  pdl_prologue();
  const int kb = r * BS;
  const int b = blockIdx.x;
  const bool rowp = b < R - 1;
  const int bb = rowp ? b : b - (R - 1);
  const int other = (bb < r ? bb : bb + 1) * BS;  // first column (row panel) or row (column panel)
  // S[k * DS + x]: A[x][k] = diag[x][k] for row panels, B[k][x] = diag[k][x] for column panels
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, kBytes);
    if (!no_copy) bulk_copy_g2s(S, pk + (rowp ? 0 : (size_t)BS * DS), kBytes, &bar);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = lane / L::LPW, jj = lane % L::LPW;
  const int line = warp * L::LPW + jj;
  // element e of this lane: row-panel (kb + q*RPT + e, other + line), column-panel (other + line, kb + q*RPT + e)
  const size_t base = rowp ? (size_t)(kb + q * RPT) * ld + other + line : (size_t)(other + line) * ld + kb + q * RPT;
  const size_t step = rowp ? ld : 1;
  reg_t d[RPT];
  int32_t p[RPT];
#pragma unroll
  for (int e = 0; e < RPT; ++e) {
    d[e] = T::load(D[base + e * step]);
    p[e] = -1;
  }
  if (!__syncthreads_and(mbar_wait_phase0(&bar, wait_ns))) {
    if (threadIdx.x == 0) report_fault(rm, kFaultPanelCopyTimeout);
    mbar_wait_phase0(&bar, wait_ns);  // a copy still in flight lands before the CTA exits
    return;
  }
  bool keyed = false;
  if constexpr (std::is_same<T, F32T>::value) {
    if (graph_int) {
      constexpr float M = 2.0f * BS;
      unsigned vc = 0;  // largest finite initial value of this warp's lines (bit order = value order)
#pragma unroll
      for (int e = 0; e < RPT; ++e)
        if (d[e] < f32_inf()) vc = max(vc, (unsigned)__float_as_int(d[e]));
      vc = __reduce_max_sync(0xffffffffu, vc);
      const float va = __int_as_float((int)max(rm->a_bits, rm->b_bits));  // >= the diagonal block's largest
      keyed = (2.0f * va + __int_as_float((int)vc)) * M + BS <= 16777215.0f;
      if (keyed) {
#pragma unroll
        for (int e = 0; e < RPT; ++e) d[e] *= M;  // slot 0
        for (int qo = 0; qo < L::TPL; ++qo) {
          const int src = qo * L::LPW + jj;
#pragma unroll
          for (int kk = 0; kk < RPT; ++kk) {
            const int k = qo * RPT + kk;
            const float ck = __shfl_sync(0xffffffffu, d[kk], src);  // key of element k of this line
            // M * (its value) + k + 1; an INF key stays INF
            const float vkp = __fmaf_rn(__fsub_rn(__fadd_rd(ck * (1.f / M), 8388608.f), 8388608.f), M,
                                        (float)(k + 1));
            const float* Sk = reinterpret_cast<const float*>(S) + k * DS + q * RPT;
#pragma unroll
            for (int e4 = 0; e4 < RPT; e4 += 4) {
              const float4 v = *reinterpret_cast<const float4*>(Sk + e4);
              d[e4] = fminf(d[e4], __fmaf_rn(v.x, M, vkp));
              d[e4 + 1] = fminf(d[e4 + 1], __fmaf_rn(v.y, M, vkp));
              d[e4 + 2] = fminf(d[e4 + 2], __fmaf_rn(v.z, M, vkp));
              d[e4 + 3] = fminf(d[e4 + 3], __fmaf_rn(v.w, M, vkp));
            }
          }
        }
#pragma unroll
        for (int e = 0; e < RPT; ++e) {
          const float key = d[e];
          if (key < f32_inf()) {
            const float v = __fsub_rn(__fadd_rd(key * (1.f / M), 8388608.f), 8388608.f);
            const int sl = (int)__fmaf_rn(-v, M, key);
            d[e] = v;
            if (sl != 0) p[e] = kb + sl - 1;
          }
        }
      }
    }
  }
  if constexpr (std::is_same<T, U16T>::value) {
    // 16-bit path: keys M*v + slot in 32-bit integers are always exact (v <= 0xFFFF). A
    // candidate through an INF (0xFFFF) operand is at least M*0xFFFF + k + 1, above the key of
    // any value up to INF with an older slot, so it never wins, as the saturating sum never did.
    constexpr uint32_t M = 2 * BS;
#pragma unroll
    for (int e = 0; e < RPT; ++e) d[e] *= M;  // slot 0
    for (int qo = 0; qo < L::TPL; ++qo) {
      const int src = qo * L::LPW + jj;
#pragma unroll
      for (int kk = 0; kk < RPT; ++kk) {
        const int k = qo * RPT + kk;
        const uint32_t ck = __shfl_sync(0xffffffffu, d[kk], src);  // key of element k of this line
        const uint32_t vkp = (ck & ~(M - 1)) + (uint32_t)(k + 1);    // M * (its value) + k + 1
        const uint32_t* Sk = reinterpret_cast<const uint32_t*>(S) + k * DS + q * RPT;
#pragma unroll
        for (int e4 = 0; e4 < RPT; e4 += 4) {
          const uint4 v = *reinterpret_cast<const uint4*>(Sk + e4);
          d[e4] = min(d[e4], v.x * M + vkp);
          d[e4 + 1] = min(d[e4 + 1], v.y * M + vkp);
          d[e4 + 2] = min(d[e4 + 2], v.z * M + vkp);
          d[e4 + 3] = min(d[e4 + 3], v.w * M + vkp);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < RPT; ++e) {
      const uint32_t sl = d[e] & (M - 1);
      d[e] /= M;
      if (sl != 0) p[e] = kb + (int)sl - 1;
    }
    keyed = true;
  }
  if (!keyed) for (int qo = 0; qo < L::TPL; ++qo) {
    const int src = qo * L::LPW + jj;
#pragma unroll
    for (int kk = 0; kk < RPT; ++kk) {
      const int k = qo * RPT + kk;
      const reg_t ck = __shfl_sync(0xffffffffu, d[kk], src);  // element k of this line
      const reg_t* Sk = S + k * DS + q * RPT;
#pragma unroll
      for (int e4 = 0; e4 < RPT; e4 += 4) {
        reg_t sv[4];
        if constexpr (std::is_same<reg_t, float>::value) {
          const float4 v = *reinterpret_cast<const float4*>(Sk + e4);
          sv[0] = v.x; sv[1] = v.y; sv[2] = v.z; sv[3] = v.w;
        } else {
          const uint4 v = *reinterpret_cast<const uint4*>(Sk + e4);
          sv[0] = v.x; sv[1] = v.y; sv[2] = v.z; sv[3] = v.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const reg_t cand = T::add(sv[u], ck);
          if (cand < d[e4 + u]) {
            d[e4 + u] = cand;
            p[e4 + u] = kb + k;
          }
        }
      }
    }
  }
  unsigned mx = 0;
#pragma unroll
  for (int e = 0; e < RPT; ++e) {
    if (p[e] >= 0) {
      D[base + e * step] = T::store(d[e]);
      P[base + e * step] = p[e];
    }
    if constexpr (std::is_same<T, F32T>::value) {
      if (d[e] < f32_inf()) mx = max(mx, (unsigned)__float_as_int(d[e]));
    } else {
      mx = max(mx, (unsigned)d[e]);
    }
  }
  // this block's largest value for phase 3's per-round choice (see diag_tile)
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) atomicMax(rowp ? &rm->b_bits : &rm->a_bits, mx);
}

template <class T, int BS>
constexpr size_t phase2_smem_bytes() {
  return sizeof(typename T::reg_t) * (size_t)BS * LineShape<BS>::DS;
}

// Values in phase 1's packed output (both layouts).
template <int BS>
__host__ __device__ constexpr size_t packed_diag_values() {
  return 2 * (size_t)BS * LineShape<BS>::DS;
}

}  // namespace apsp
