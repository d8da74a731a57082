// Phases 1 and 2 of a block round: tiles whose update depends on itself.
//
// Section 4.1 of arXiv 1811.01201: in round r the diagonal block (r,r) is
// self-dependent (phase 1); the other blocks of row r and of column r depend
// on themselves and on the finished block (r,r) (paper phases 2 and 3, run
// here as one launch). Each such tile is updated in place by FW_BLOCK: for k
// ascending over block r, every element relaxes through D[i][k] + D[k][j]
// with a strict '<', and P records the global k (Section 4.2, Section 3).
//
// GPU mapping: one CTA per tile; every thread keeps a TE x TE sub-block of the
// tile in registers. Step k needs row k and/or column k of the tile as they
// stand after step k-1 (neither changes during step k, because D[k][k] = 0);
// their owners publish them into a double-buffered shared-memory row/column,
// so one barrier per step orders the whole update exactly like the serial
// loop. The fixed operand of a panel tile (the finished diagonal block) sits
// in shared memory.
#pragma once

#include <type_traits>

#include "fw_common.cuh"

namespace apsp {

enum SeqMode { kSeqDiag = 0, kSeqRow = 1, kSeqCol = 2 };

// Update one BS x BS tile of D (origin ti0, tj0; leading dimension ld) through
// the intermediates kb .. kb+BS-1.
//   kSeqDiag: C = A = B = block (r,r)            c = C[i][k] + C[k][j]
//   kSeqRow:  C = B = block (r,J), A = diag       c = Diag[i][k] + C[k][j]
//   kSeqCol:  C = A = block (I,r), B = diag       c = C[i][k] + Diag[k][j]
// diag_s: BS x (BS+1) shared copy of the finished diagonal block (row and
// column modes). rowbuf / colbuf: 2*BS shared scratch each.
template <class T, int BS, int MODE>
__device__ __forceinline__ void seq_tile(typename T::store_t* __restrict__ D, int32_t* __restrict__ P, size_t ld,
                                         int kb, int ti0, int tj0, const typename T::reg_t* __restrict__ diag_s,
                                         typename T::reg_t* rowbuf, typename T::reg_t* colbuf, RoundMax* rm) {
  using S = SeqShape<BS>;
  using reg_t = typename T::reg_t;
  constexpr int TE = S::TE, TPR = S::TPR, DS = BS + 1;
  const int tid = threadIdx.x, tx = tid % TPR, ty = tid / TPR;
  const int li0 = ty * TE, lj0 = tx * TE;

  reg_t d[TE][TE];
  int32_t p[TE][TE];
#pragma unroll
  for (int a = 0; a < TE; ++a)
#pragma unroll
    for (int c = 0; c < TE; ++c) {
      d[a][c] = T::load(D[(size_t)(ti0 + li0 + a) * ld + tj0 + lj0 + c]);
      p[a][c] = -1;
    }

  for (int k0 = 0; k0 < BS; k0 += TE) {
#pragma unroll
    for (int kk = 0; kk < TE; ++kk) {
      const int k = k0 + kk;
      reg_t* rb = rowbuf + (k & 1) * BS;
      reg_t* cb = colbuf + (k & 1) * BS;
      if (MODE != kSeqCol && ty == k0 / TE) {
#pragma unroll
        for (int c = 0; c < TE; ++c) rb[lj0 + c] = d[kk][c];
      }
      if (MODE != kSeqRow && tx == k0 / TE) {
#pragma unroll
        for (int a = 0; a < TE; ++a) cb[li0 + a] = d[a][kk];
      }
      __syncthreads();
      reg_t av[TE], bv[TE];
#pragma unroll
      for (int a = 0; a < TE; ++a) av[a] = (MODE == kSeqRow) ? diag_s[(li0 + a) * DS + k] : cb[li0 + a];
#pragma unroll
      for (int c = 0; c < TE; ++c) bv[c] = (MODE == kSeqCol) ? diag_s[k * DS + lj0 + c] : rb[lj0 + c];
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
      const size_t off = (size_t)(ti0 + li0 + a) * ld + tj0 + lj0 + c;
      if (p[a][c] >= 0) {
        D[off] = T::store(d[a][c]);
        P[off] = p[a][c];
      }
    }
  if (rm != nullptr) {
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
      if (MODE != kSeqRow) atomicMax(&rm->a_bits, mx);
      if (MODE != kSeqCol) atomicMax(&rm->b_bits, mx);
    }
  }
}

// Phase 1: the diagonal block of round r (one CTA).
template <class T, int BS>
__global__ void __launch_bounds__(SeqShape<BS>::NT) fw_phase1_kernel(typename T::store_t* D, int32_t* P, size_t ld,
                                                                     int r, RoundMax* rm) {
  __shared__ typename T::reg_t rowbuf[2 * BS], colbuf[2 * BS];
  const int kb = r * BS;
  if (rm != nullptr && threadIdx.x == 0) {
    rm->a_bits = 0;  // visible to this CTA's atomics after seq_tile's barriers
    rm->b_bits = 0;
  }
  seq_tile<T, BS, kSeqDiag>(D, P, ld, kb, kb, kb, nullptr, rowbuf, colbuf, rm);
}

// Phase 2: the other blocks of row r (CTAs 0 .. R-2) and of column r
// (CTAs R-1 .. 2R-3), all against the finished diagonal block.
template <class T, int BS>
__global__ void __launch_bounds__(SeqShape<BS>::NT) fw_phase2_kernel(typename T::store_t* D, int32_t* P, size_t ld,
                                                                     int r, int R, RoundMax* rm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using reg_t = typename T::reg_t;
  constexpr int DS = BS + 1;
  reg_t* diag_s = reinterpret_cast<reg_t*>(smem_raw);
  reg_t* rowbuf = diag_s + BS * DS;
  reg_t* colbuf = rowbuf + 2 * BS;
  const int kb = r * BS;
  for (int t = threadIdx.x; t < BS * BS; t += blockDim.x) {
    const int i = t / BS, j = t % BS;
    diag_s[i * DS + j] = T::load(D[(size_t)(kb + i) * ld + kb + j]);
  }
  __syncthreads();
  const int b = blockIdx.x;
  if (b < R - 1) {
    const int J = b < r ? b : b + 1;
    seq_tile<T, BS, kSeqRow>(D, P, ld, kb, kb, J * BS, diag_s, rowbuf, colbuf, rm);
  } else {
    const int bb = b - (R - 1);
    const int I = bb < r ? bb : bb + 1;
    seq_tile<T, BS, kSeqCol>(D, P, ld, kb, I * BS, kb, diag_s, rowbuf, colbuf, rm);
  }
}

template <class T, int BS>
constexpr size_t phase2_smem_bytes() {
  return sizeof(typename T::reg_t) * ((size_t)BS * (BS + 1) + 4 * BS);
}

}  // namespace apsp
