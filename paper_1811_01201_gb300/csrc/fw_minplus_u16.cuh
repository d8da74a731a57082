// Phase 3 of a block round on exact 16-bit distances, two per 32-bit lane.
//
// Same update as the fp32 kernel (Section 4.1 paper phase 4, Section 4.2
// FW_BLOCK with strict '<', P = global k per Section 3), on integer distances
// stored as uint16 with 0xFFFF = INF. A graph qualifies for this path only
// when every path length is below 0xFFFF (max_w * (n-1) < 65535), so the
// saturating sum min(a + b, 0xFFFF) equals the exact sum whenever it can
// matter, and D and P come out bit-identical to the fp32 path.
//
// The hot loop is PTX add.u16x2 + min.u16x2: two updates per instruction
// pair. A wrapping add is exact when no a + b can exceed 0xFFFF, which holds
// when the round's panel maxima (recorded by phases 1-2, INF included) sum to
// at most 0xFFFF; otherwise (typically while panels still hold INF) the round
// uses the saturating form sat(a + b) = min(a, ~b) + b (one more min per pair).
//
// P comes, as on the fp32 path, from keys where the round allows them: when
// every panel value of the round is finite and small enough (a + b below
// 65536 / M - 1 with M = 2*BS; phases 1-2 record the maxima), every operand is
// scaled by M inside its 16-bit lane and the A panel carries k+1 in the low
// bits (A' = M*a + k + 1, B' = M*b, D' = M*min(d, T) with T = 65536/M - 1).
// The same add.u16x2 + min.u16x2 loop then yields, per element, the minimum
// value and the smallest k attaining it, while the old value (slot 0) wins
// ties; an old value clamped to T (INF included) reads as unchanged, and every
// finite candidate, at most M*(T-2) + BS, still beats it. Slot 0 means
// unchanged. Other rounds (an INF or a large value in the panels) find the
// improved elements by comparing with the old tile (kept in registers); a
// warp then re-evaluates its BS candidates, one k per lane, and takes the
// first k whose saturated sum equals the new value.
//
// Tiling: 128 x 128 output tile per CTA of 256 threads; each thread owns 8
// rows (ty*4+{0..3}, 64+ty*4+{0..3}) x 8 consecutive columns (tx*8 ..), i.e.
// 8 x 4 packed words. The A panel slice is stored transposed with every value
// duplicated into both halves of a word; the B panel slice as is. A small
// kernel packs every slice of the round once; each CTA pulls its two slices
// with bulk copies while it loads its tile.
#pragma once

#include "fw_common.cuh"
#include "fw_minplus_f32.cuh"

namespace apsp {

constexpr int kSstA16 = kTile + 4;      // words per transposed-A row
constexpr int kSstB16 = kTile / 2 + 4;  // words per B row (two uint16 per word)

// 16-bit keys of phase 3 (see the top of this file): scale M = 2*BS, clamp T,
// and the largest panel sum a + b of a keyed round.
template <int BS>
struct Key16 {
  static constexpr uint32_t M = 2u * BS;
  static constexpr int log2M = BS == 32 ? 6 : (BS == 64 ? 7 : 8);
  static constexpr uint32_t T = 65536u / M - 1u;
  static constexpr uint32_t bound = T - 2u;
  static constexpr uint32_t T2 = T | (T << 16);                                // clamp, both lanes
  static constexpr uint32_t slot2 = (M - 1u) | ((M - 1u) << 16);               // slot bits, both lanes
  static constexpr uint32_t val2 = ((0xFFFFu >> log2M)) | ((0xFFFFu >> log2M) << 16);  // value bits after >> log2M
};

// Keyed 16-bit round: the round's panel maxima (INF = 0xFFFF included) sum to at most the bound.
template <int BS>
__device__ __forceinline__ bool round_keyed16(const RoundMax* rm) {
  return rm->a_bits + rm->b_bits <= Key16<BS>::bound;
}

template <int BS>
constexpr size_t minplus_u16_smem_bytes() {
  return sizeof(uint32_t) * (size_t)BS * (kSstA16 + kSstB16);
}

// Words of one packed A slice (tile row) and one packed B slice (tile column)
// in the shared-memory layout of the kernel below.
template <int BS>
__host__ __device__ constexpr size_t u16_slice_a_words() {
  return (size_t)BS * kSstA16;
}
template <int BS>
__host__ __device__ constexpr size_t u16_slice_b_words() {
  return (size_t)BS * kSstB16;
}

__device__ __forceinline__ uint32_t vadd16(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("add.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t vmin16(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t umax4(uint4 v) {
  // largest of the eight uint16 lanes of v
  uint32_t m = max(max(max(v.x & 0xFFFF, v.x >> 16), max(v.y & 0xFFFF, v.y >> 16)),
                   max(max(v.z & 0xFFFF, v.z >> 16), max(v.w & 0xFFFF, v.w >> 16)));
  return m;
}

// SAT: saturating sums (rounds whose panels may overflow 16 bits); otherwise
// no sum can exceed 0xFFFF and a wrapping add.u16x2 is exact. Both lanes' add
// and min run on the ALU pipe, which bounds this loop (a fused
// __viaddmin_u16x2 measured the same, and a 32-bit integer add, exact here too,
// measured 8% slower).
template <int BS, bool SAT>
__device__ __forceinline__ void minplus_u16_loop(uint32_t (&w)[8][4], const uint32_t* __restrict__ Ap,
                                                 const uint32_t* __restrict__ Bp) {
#pragma unroll 4
  for (int k = 0; k < BS; ++k) {
    const uint4 a0 = *reinterpret_cast<const uint4*>(Ap + k * kSstA16);
    const uint4 a1 = *reinterpret_cast<const uint4*>(Ap + k * kSstA16 + 64);
    const uint4 b4 = *reinterpret_cast<const uint4*>(Bp + k * kSstB16);
    const uint32_t av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const uint32_t bv[4] = {b4.x, b4.y, b4.z, b4.w};
    uint32_t nb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) nb[q] = ~bv[q];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (SAT) w[a][q] = vmin16(w[a][q], vadd16(vmin16(av[a], nb[q]), bv[q]));
        else w[a][q] = vmin16(w[a][q], vadd16(av[a], bv[q]));
      }
  }
}

// The round's panel slices in the kernel's shared-memory layout, packed once
// per round: CTAs 0 .. nT-1 write A slice tr (As[k * kSstA16 + i] =
// dup(D[tr*128 + i][kb + k]), transposed and duplicated into both halves),
// CTAs nT .. 2nT-1 write B slice tc (Bs[k * kSstB16 + q] = D[kb + k][tc*128 +
// 2q .. 2q+1]).
template <int BS>
__global__ void __launch_bounds__(256) fw_pack_panels_u16_kernel(const uint16_t* __restrict__ D, size_t ld, int nT,
                                                                 int r, const RoundMax* __restrict__ rm,
                                                                 uint32_t* __restrict__ Apk,
                                                                 uint32_t* __restrict__ Bpk) {
  pdl_prologue();
  const int kb = r * BS, tid = threadIdx.x;
  const bool keyed = round_keyed16<BS>(rm);  // every panel value is then at most the bound: no lane overflows
  constexpr int sh = Key16<BS>::log2M;
  if ((int)blockIdx.x < nT) {
    // 128 rows x BS uint16 (BS/8 uint4 per row), transposed + duplicated.
    const int r0 = blockIdx.x * kTile;
    uint32_t* As = Apk + u16_slice_a_words<BS>() * blockIdx.x;
#pragma unroll
    for (int m = 0; m < BS / 16; ++m) {
      const int idx = tid + 256 * m;
      const int ri = idx & 7, cq = (idx >> 3) & 3, grp = idx >> 5;
      const int i = (grp & 15) * 8 + ri;
      const int q8 = (grp >> 4) * 4 + cq;
      const uint4 v = *reinterpret_cast<const uint4*>(D + (size_t)(r0 + i) * ld + kb + q8 * 8);
      const uint32_t h[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k0 = q8 * 8 + 2 * e;
        uint32_t lo = h[e] & 0xFFFF, hi = h[e] >> 16;
        if (keyed) {
          lo = (lo << sh) + (uint32_t)(k0 + 1);
          hi = (hi << sh) + (uint32_t)(k0 + 2);
        }
        As[k0 * kSstA16 + i] = lo | (lo << 16);
        As[(k0 + 1) * kSstA16 + i] = hi | (hi << 16);
      }
    }
  } else {
    // BS rows x 128 uint16 = 16 uint4 per row.
    const int tc = blockIdx.x - nT, c0 = tc * kTile;
    uint32_t* Bs = Bpk + u16_slice_b_words<BS>() * tc;
#pragma unroll
    for (int m = 0; m < BS / 16; ++m) {
      const int idx = tid + 256 * m, k = idx >> 4, q = idx & 15;
      uint4 v = *reinterpret_cast<const uint4*>(D + (size_t)(kb + k) * ld + c0 + q * 8);
      if (keyed) {  // both lanes below 65536 / M: the shift scales each lane without spilling
        v.x <<= sh; v.y <<= sh; v.z <<= sh; v.w <<= sh;
      }
      *reinterpret_cast<uint4*>(Bs + k * kSstB16 + q * 4) = v;
    }
  }
}

// One launch per round; one CTA per 128x128 tile. Apk / Bpk: the round's
// packed slices, pulled into shared memory by two bulk copies while the CTA
// loads its tile; wait_ns / no_copy as in the fp32 kernel (a wait that
// expires sets kFaultPanelCopyTimeout and the CTA leaves its tile).
template <int BS>
__global__ void __launch_bounds__(256, 2) fw_phase3_u16_kernel(uint16_t* __restrict__ D, int32_t* __restrict__ P,
                                                               size_t ld, int nT, int r, RoundMax* rm,
                                                               const uint32_t* __restrict__ Apk,
                                                               const uint32_t* __restrict__ Bpk, int stagger, int sms,
                                                               unsigned long long wait_ns, int no_copy) {
  extern __shared__ __align__(16) uint32_t smu[];
  __shared__ uint64_t bar;
  pdl_prologue();
  uint32_t* As = smu;                 // As[k * kSstA16 + i] = dup(D[r0 + i][kb + k])
  uint32_t* Bs = smu + BS * kSstA16;  // Bs[k * kSstB16 + q] = D[kb + k][c0 + 2q .. 2q+1]

  const int kb = r * BS;
  const int tr = blockIdx.x / nT, tc = blockIdx.x - tr * nT;
  const int r0 = tr * kTile, c0 = tc * kTile;
  if (r0 >= kb && r0 + kTile <= kb + BS) return;
  if (c0 >= kb && c0 + kTile <= kb + BS) return;
  // the round's panel maxima (INF included) decide whether a wrapping add is safe, and whether
  // the round runs on keys
  const bool sat = rm->a_bits + rm->b_bits > 0xFFFFu;
  const bool keyed = round_keyed16<BS>(rm);
  if (stagger > 0 && (int)blockIdx.x >= sms && (int)blockIdx.x < 2 * sms) {
    const long long t0 = clock64();
    while (clock64() - t0 < stagger) {
    }
  }

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr unsigned a_bytes = (unsigned)(u16_slice_a_words<BS>() * sizeof(uint32_t));
  constexpr unsigned b_bytes = (unsigned)(u16_slice_b_words<BS>() * sizeof(uint32_t));
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar, a_bytes + b_bytes);
    if (!no_copy) {
      bulk_copy_g2s(As, Apk + u16_slice_a_words<BS>() * tr, a_bytes, &bar);
      bulk_copy_g2s(Bs, Bpk + u16_slice_b_words<BS>() * tc, b_bytes, &bar);
    }
  }

  uint32_t w[8][4], old[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const uint4 v = *reinterpret_cast<const uint4*>(D + (size_t)(r0 + mp_row(ty, a)) * ld + c0 + tx * 8);
    old[a][0] = v.x; old[a][1] = v.y; old[a][2] = v.z; old[a][3] = v.w;
#pragma unroll
    for (int q = 0; q < 4; ++q) w[a][q] = old[a][q];
  }
  if (!__syncthreads_and(mbar_wait_phase0(&bar, wait_ns))) {
    if (tid == 0) report_fault(rm, kFaultPanelCopyTimeout);
    mbar_wait_phase0(&bar, wait_ns);  // copies still in flight land before the CTA exits
    return;
  }

  if (keyed) {
    constexpr int sh = Key16<BS>::log2M;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) w[a][q] = vmin16(old[a][q], Key16<BS>::T2) << sh;  // slot 0
    minplus_u16_loop<BS, false>(w, As + ty * 4, Bs + tx * 4);
    // slot bits name the first k of each improved element; others keep their old value
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int gi = r0 + mp_row(ty, a);
      const int gj = c0 + tx * 8;
      if ((gi >= kb && gi < kb + BS) || (gj >= kb && gj < kb + BS)) continue;
      const uint32_t any = (w[a][0] | w[a][1] | w[a][2] | w[a][3]) & Key16<BS>::slot2;
      if (any == 0u) continue;
      uint32_t nw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t sl = w[a][q] & Key16<BS>::slot2;
        const uint32_t m = (sl & 0xFFFFu ? 0x0000FFFFu : 0u) | (sl >> 16 ? 0xFFFF0000u : 0u);
        nw[q] = (((w[a][q] >> sh) & Key16<BS>::val2) & m) | (old[a][q] & ~m);
        if (sl & 0xFFFFu) P[(size_t)gi * ld + gj + 2 * q] = kb + (int)(sl & 0xFFFFu) - 1;
        if (sl >> 16) P[(size_t)gi * ld + gj + 2 * q + 1] = kb + (int)(sl >> 16) - 1;
      }
      *reinterpret_cast<uint4*>(D + (size_t)gi * ld + gj) = make_uint4(nw[0], nw[1], nw[2], nw[3]);
    }
    return;
  }
  if (sat)
    minplus_u16_loop<BS, true>(w, As + ty * 4, Bs + tx * 4);
  else
    minplus_u16_loop<BS, false>(w, As + ty * 4, Bs + tx * 4);

  // Epilogue: write back changed 8-element groups outside block r's rows and
  // columns; flag improved elements (slot = a*8 + column).
  uint64_t imp = 0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int gi = r0 + mp_row(ty, a);
    const int gj = c0 + tx * 8;
    if ((gi >= kb && gi < kb + BS) || (gj >= kb && gj < kb + BS)) continue;
    uint16_t* dp = D + (size_t)gi * ld + gj;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if ((w[a][q] & 0xFFFF) < (old[a][q] & 0xFFFF)) imp |= 1ull << (a * 8 + 2 * q);
      if ((w[a][q] >> 16) < (old[a][q] >> 16)) imp |= 1ull << (a * 8 + 2 * q + 1);
    }
    if ((imp >> (a * 8)) & 0xFF) *reinterpret_cast<uint4*>(dp) = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
  }

  if (!__any_sync(0xffffffffu, imp != 0)) return;
#pragma unroll
  for (int slot = 0; slot < 64; ++slot) {
    unsigned bal = __ballot_sync(0xffffffffu, (imp >> slot) & 1);
    if (!bal) continue;
    const int a = slot >> 3, c = slot & 7;
    const uint32_t dmine = (c & 1) ? (w[a][c >> 1] >> 16) : (w[a][c >> 1] & 0xFFFF);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      const int stid = warp * 32 + src;
      const int li = mp_row(stid >> 4, a), lj = (stid & 15) * 8 + c;
      const uint32_t dn = __shfl_sync(0xffffffffu, dmine, src);
      int kstar = BS;
#pragma unroll
      for (int m = 0; m < BS / 32; ++m) {
        const int k = m * 32 + lane;
        const uint32_t av = As[k * kSstA16 + li] & 0xFFFF;
        const uint32_t bw = Bs[k * kSstB16 + (lj >> 1)];
        const uint32_t bvv = (lj & 1) ? (bw >> 16) : (bw & 0xFFFF);
        const uint32_t cand = min(av + bvv, kInf16);
        const unsigned eq = __ballot_sync(0xffffffffu, cand == dn);
        if (eq && kstar == BS) kstar = m * 32 + __ffs(eq) - 1;
      }
      if (lane == src) P[(size_t)(r0 + li) * ld + c0 + lj] = kb + kstar;
    }
  }
}

}  // namespace apsp
