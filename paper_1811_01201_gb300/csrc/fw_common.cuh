// Shared device-side definitions of the blocked Floyd-Warshall kernels.
//
// Method: Rucci, De Giusti, Naiouf, arXiv 1811.01201. Section 3 defines the
// problem (distance matrix D, path matrix P = most recently added
// intermediate); Section 4.1 the blocking (R rounds of diagonal block, row and
// column blocks, remaining blocks); Section 4.2 the update (one addition, one
// comparison, here a strict '<').
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace apsp {

// Working layout: n rounded up to a multiple of kTile, row-major, leading
// dimension n_pad. Padding rows/columns are isolated vertices (INF off the
// diagonal, 0 on it), which never improve a real entry.
constexpr int kTile = 128;

constexpr float kInfF = __builtin_huge_valf();
constexpr uint32_t kInf16 = 0xFFFFu;

__device__ __forceinline__ float f32_inf() { return __int_as_float(0x7f800000); }

// fp32 element type: D in fp32, candidate = one correctly rounded addition.
struct F32T {
  using store_t = float;
  using reg_t = float;
  static __device__ __forceinline__ reg_t load(store_t v) { return v; }
  static __device__ __forceinline__ store_t store(reg_t v) { return v; }
  static __device__ __forceinline__ reg_t add(reg_t a, reg_t b) { return __fadd_rn(a, b); }
};

// 16-bit element type: D in uint16 with 0xFFFF = INF; candidates saturate at
// 0xFFFF, which equals the unbounded fp32 result whenever every path length
// is below 0xFFFF (the eligibility rule of the 16-bit path).
struct U16T {
  using store_t = uint16_t;
  using reg_t = uint32_t;
  static __device__ __forceinline__ reg_t load(store_t v) { return v; }
  static __device__ __forceinline__ store_t store(reg_t v) { return (store_t)v; }
  static __device__ __forceinline__ reg_t add(reg_t a, reg_t b) { return min(a + b, kInf16); }
};

// Largest panel values of the current round. Phase 1 resets it and adds the
// diagonal block; phase 2 adds its column-panel blocks to `a` (the A operand
// of phase 3) and its row-panel blocks to `b` (the B operand). fp32: largest
// finite value as a bit pattern (for non-negative floats the integer order is
// the value order). 16-bit: largest value with INF (0xFFFF) included.
struct RoundMax {
  unsigned int a_bits;
  unsigned int b_bits;
};

// Threads and per-thread sub-block of the sequential (phase 1 / phase 2) tile
// routine: BS x BS tile, each thread owns TE x TE elements.
template <int BS>
struct SeqShape {
  static constexpr int TPR = (BS == 128) ? 32 : 16;  // threads along a row (and a column)
  static constexpr int NT = TPR * TPR;               // threads per CTA
  static constexpr int TE = BS / TPR;                // elements per thread per dimension
  static_assert(TE * TPR == BS, "bad tile shape");
};

}  // namespace apsp
