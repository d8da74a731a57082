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
// `fault` is the solve's own fault word (zeroed by the init kernel, never by
// the rounds): a bounded wait of this solve that expired sets a bit in it, so
// a caller that runs several solves at once can tell which one failed.
struct RoundMax {
  unsigned int a_bits;
  unsigned int b_bits;
  unsigned int fault;
};

// Device-side fault word of this translation unit's kernels, shared by every
// solve on the device: a bounded wait that expired sets a bit here (and in the
// solve's own word) instead of hanging; the host reads and clears it.
constexpr unsigned kFaultPanelCopyTimeout = 1u;
static __device__ unsigned int g_apsp_fault = 0;

__device__ __forceinline__ void report_fault(RoundMax* rm, unsigned bit) {
  atomicOr(&rm->fault, bit);
  atomicOr(&g_apsp_fault, bit);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Single-use mbarrier on shared memory, completed by bulk-copy byte counts.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Polls phase 0 of the barrier until it completes or `limit_ns` passes; true if it completed.
__device__ __forceinline__ bool mbar_wait_phase0(uint64_t* bar, unsigned long long limit_ns) {
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done)
                 : "r"(smem_addr(bar))
                 : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// shared to global memory; the calling thread then waits until it is done.
// The shared source must be made visible to the copy engine first
// (bulk_store_fence after the threads' writes and a barrier).
__device__ __forceinline__ void bulk_store_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_copy_s2g_and_wait(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Programmatic dependent launch: the round's kernels are launched so that the
// next one may be scheduled while this one runs. Each kernel first lets its
// dependent be scheduled (once every CTA of this grid has started or exited),
// then waits until its own predecessor has completed and its writes are
// visible, before touching any data. Without the launch attribute both are
// no-ops.
__device__ __forceinline__ void pdl_prologue() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

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
