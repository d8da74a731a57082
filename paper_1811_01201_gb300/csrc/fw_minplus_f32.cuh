// Phase 3 of a block round, fp32: every tile outside row r and column r.
//
// Section 4.1 of arXiv 1811.01201 (paper phase 4): each remaining block
// (I,J) depends only on block (I,r) of its row and block (r,J) of its column,
// which phase 3 never changes. FW_BLOCK (Section 4.2) relaxes every element
// through k = kb .. kb+BS-1 in ascending order with a strict '<' and records
// the global k in P (Section 3).
//
// With both panels fixed, the serial strict-'<' sweep over k has a closed
// form per element: D' = min(D, min_k (A[i][k] + B[k][j])) (fp32 min is exact
// and order-free), and P changes only if D' < D, to kb + the FIRST k whose
// candidate equals D'. The kernel therefore runs the hot loop as one FADD and
// one FMNMX per update and recovers P afterwards:
//
//  * integer-valued graphs whose round panels' largest finite values sum to
//    at most a bound (phases 1-2 record the maxima): every operand is scaled
//    by M = 2*BS and the A panel carries k+1 in the low bits, all above an
//    offset of 2^23 (A' = 2^23 + M*a + k + 1, B' = M*b, D' = 2^23 + M*d;
//    k+1 <= BS < M). The candidate keys 2^23 + M*(a+b) + k + 1 are exact while
//    below 2^24, so min over keys yields the minimum value and, among equal
//    values, the smallest k -- while the old D (slot 0) wins ties, as the
//    strict '<' requires. Slot 0 in the result means unchanged, so neither
//    the old tile nor a search is needed: P comes for free. Every finite key
//    lies in [2^23, 2^24), where the float's mantissa is the integer itself,
//    so the slot and the value are read from the key's bits with integer ops.
//  * rounds of integer graphs beyond that bound (rare): improved elements are
//    found by comparing with the old D; where many improved every lane
//    re-scans its own elements with k descending, else the warp re-evaluates
//    one improved element at a time, one k per lane. Real-valued graphs run
//    fw_phase3_f32_real_kernel (end of this file), which tags each element
//    with the group of k pairs of its last improvement. All searches use
//    bit-identical additions, so equality is exact.
//
// Tiling: 128 x 128 output tile per CTA of 256 threads, 8 x 8 elements per
// thread in registers (rows ty*4+{0..3}, 64+ty*4+{0..3}; columns likewise
// with tx). Both panel slices are stored as k pairs (A transposed), so each
// 128-bit shared load gives two elements' (a_k, a_k+1) pairs and one PTX
// add.rn.f32x2 forms two candidates; the min stays one FMNMX per candidate.
// A small kernel packs every slice of the round once (scaled into keys on
// keyed rounds); each phase-3 CTA pulls its two slices into shared memory
// with bulk copies (cp.async.bulk, completion counted on an mbarrier) that run
// while the CTA loads its tile.
// Rows/columns of the tile that fall in block r (the panels) are computed but
// never written.
#pragma once

#include "fw_common.cuh"

namespace apsp {

constexpr int kDenseRescan = 384;  // improved elements per warp above which lanes re-scan their own

// Key scale M = 2*BS (a power of two, so scaling is exact), the key offset
// 2^23, and the largest finite panel sum a + b for which every key
// 2^23 + M*(a+b) + BS stays below 2^24.
template <int BS>
struct KeyParams {
  static constexpr float M = 2.0f * BS;
  static constexpr int log2M = BS == 32 ? 6 : (BS == 64 ? 7 : 8);
  static constexpr float off = 8388608.0f;  // 2^23
  // Old values are keyed as min(2^23 + M*d, cap) with cap = 2^24 - M (slot 0): a D value too
  // large for an exact key (or INF) reads as unchanged, and every finite candidate, below
  // 2^23 + M*bound + BS < cap, still beats it.
  static constexpr float cap = 16777216.0f - 2.0f * BS;
  static constexpr float bound = (float)(((1 << 23) - 2 * BS) / (2 * BS) - 16);
  static_assert(BS == 32 || BS == 64 || BS == 128, "unsupported block size");
};

// B slices are stored with their 16-byte chunks swizzled (chunk c at
// c ^ ((c >> 3) & 1)), so that the 16 lanes of a half warp, which read the
// chunks 2*tx and 2*tx + 1 of their columns, fall on distinct bank groups in
// pairs: two shared-memory wavefronts per 128-bit load instead of four.
__host__ __device__ constexpr int bswz(int chunk) { return chunk ^ ((chunk >> 3) & 1); }
// float offset of column j's k pair (element e = k & 1) in a B k-pair row
__host__ __device__ constexpr int bcol(int j, int e) { return 4 * bswz(j >> 1) + 2 * (j & 1) + e; }

// Panels are stored as k pairs: As[kp*kS2 + 2i + e] = A[i][2kp+e] and
// Bs[kp*kS2 + 2j + e] = B[2kp+e][j], so one 128-bit load gives two rows' (or
// columns') consecutive-k pairs and one add.rn.f32x2 forms two candidates.
constexpr int kS2 = 2 * kTile + 8;  // floats per k-pair row (padded)

// Per-warp list of improved elements for the P search of real-valued graphs.
constexpr int kQueuePerWarp = 384;

template <int BS>
constexpr size_t minplus_f32_smem_bytes() {
  return sizeof(float) * (size_t)BS * kS2;
}

__device__ __forceinline__ float2 fadd2_rn(float2 a, float2 b) {
  // two independent IEEE round-to-nearest fp32 additions in one instruction
  unsigned long long pa, pb, pc;
  asm("mov.b64 %0, {%1,%2};" : "=l"(pa) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1,%2};" : "=l"(pb) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(pc) : "l"(pa), "l"(pb));
  float2 c;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(c.x), "=f"(c.y) : "l"(pc));
  return c;
}

__device__ __forceinline__ float pan(const float* S, int k, int x) { return S[(k >> 1) * kS2 + 2 * x + (k & 1)]; }
__device__ __forceinline__ float pan_b(const float* S, int k, int x) { return S[(k >> 1) * kS2 + bcol(x, k & 1)]; }

__device__ __forceinline__ int mp_row(int ty, int a) { return (a < 4) ? ty * 4 + a : 64 + ty * 4 + (a - 4); }
__device__ __forceinline__ int mp_col(int tx, int c) { return (c < 4) ? tx * 4 + c : 64 + tx * 4 + (c - 4); }

__device__ __forceinline__ float floor_pos(float v) {
  // floor for 0 <= v < 2^23 on the FMA pipe: round-down add of 2^23, then subtract
  return __fsub_rn(__fadd_rd(v, 8388608.f), 8388608.f);
}

// Integer-valued graphs (graphs with other weights use
// fw_phase3_f32_real_kernel below).
template <int BS>
__device__ __forceinline__ void tile_body(float* __restrict__ D, int32_t* __restrict__ P, size_t ld, int kb,
                                          int r0, int c0, bool keyed, float* As, float* Bs, uint64_t* bar,
                                          unsigned long long wait_ns, RoundMax* rm) {
  constexpr float M = KeyParams<BS>::M;
  const float INF = f32_inf();
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
  float d[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const float* row = D + (size_t)(r0 + mp_row(ty, a)) * ld + c0;
    const float4 v0 = *reinterpret_cast<const float4*>(row + tx * 4);
    const float4 v1 = *reinterpret_cast<const float4*>(row + 64 + tx * 4);
    d[a][0] = v0.x; d[a][1] = v0.y; d[a][2] = v0.z; d[a][3] = v0.w;
    d[a][4] = v1.x; d[a][5] = v1.y; d[a][6] = v1.z; d[a][7] = v1.w;
  }
  if (keyed) {
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) d[a][c] = fminf(__fmaf_rn(d[a][c], M, KeyParams<BS>::off), KeyParams<BS>::cap);
  }
  // The packed panel slices were requested by the kernel before the tile load;
  // the whole CTA goes on only if every thread saw them arrive in time.
  if (!__syncthreads_and(mbar_wait_phase0(bar, wait_ns))) {
    if (tid == 0) report_fault(rm, kFaultPanelCopyTimeout);
    mbar_wait_phase0(bar, wait_ns);  // copies still in flight land before the CTA exits
    return;
  }
  // Hot loop: per k pair, one f32x2 add and two FMNMX per element.
  const float* Ap = As + ty * 8;
  const float* Bp0 = Bs + 4 * bswz(2 * tx);      // columns tx*4, tx*4+1 (and +64 at +128)
  const float* Bp1 = Bs + 4 * bswz(2 * tx + 1);  // columns tx*4+2, tx*4+3
#pragma unroll 1
  for (int kp = 0; kp < BS / 2; ++kp) {
    const float4 a0 = *reinterpret_cast<const float4*>(Ap + kp * kS2);
    const float4 a1 = *reinterpret_cast<const float4*>(Ap + kp * kS2 + 4);
    const float4 a2 = *reinterpret_cast<const float4*>(Ap + kp * kS2 + 128);
    const float4 a3 = *reinterpret_cast<const float4*>(Ap + kp * kS2 + 132);
    const float4 b0 = *reinterpret_cast<const float4*>(Bp0 + kp * kS2);
    const float4 b1 = *reinterpret_cast<const float4*>(Bp1 + kp * kS2);
    const float4 b2 = *reinterpret_cast<const float4*>(Bp0 + kp * kS2 + 128);
    const float4 b3 = *reinterpret_cast<const float4*>(Bp1 + kp * kS2 + 128);
    const float2 av[8] = {{a0.x, a0.y}, {a0.z, a0.w}, {a1.x, a1.y}, {a1.z, a1.w},
                          {a2.x, a2.y}, {a2.z, a2.w}, {a3.x, a3.y}, {a3.z, a3.w}};
    const float2 bv[8] = {{b0.x, b0.y}, {b0.z, b0.w}, {b1.x, b1.y}, {b1.z, b1.w},
                          {b2.x, b2.y}, {b2.z, b2.w}, {b3.x, b3.y}, {b3.z, b3.w}};
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float2 s = fadd2_rn(av[a], bv[c]);
        d[a][c] = fminf(fminf(d[a][c], s.x), s.y);
      }
  }
  if (keyed) {
    // Every key lies in [2^23, 2^24), so its bits are 0x4B000000 | (M*v + slot). A group of four
    // without a slot is unchanged and costs two logic ops and a test; an improved element
    // (always an exact candidate key) gets its value v and P = kb + slot - 1.
    constexpr uint32_t kSlot = (uint32_t)(2 * BS) - 1u;
    constexpr int kSh = KeyParams<BS>::log2M;
    const uint32_t kCapBits = __float_as_uint(KeyParams<BS>::cap);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int gi = r0 + mp_row(ty, a);
      const bool band_r = (gi >= kb) && (gi < kb + BS);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gj = c0 + mp_col(tx, 4 * h);
        const bool band_c = (gj >= kb) && (gj < kb + BS);
        uint32_t kbits[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) kbits[e] = __float_as_uint(d[a][4 * h + e]);
        if (((kbits[0] | kbits[1] | kbits[2] | kbits[3]) & kSlot) != 0u && !band_r && !band_c) {
          float* dp = D + (size_t)gi * ld + gj;
          int32_t* pp = P + (size_t)gi * ld + gj;
          // v = (M*v + slot) >> log2(M), rebuilt as the float 2^23 + v minus 2^23 (exact); a clamped
          // key (a value too large for a key, or INF) does not hold its old value
          float nv[4];
          bool clamped = false;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            nv[e] = __fsub_rn(__uint_as_float(0x4B000000u | ((kbits[e] & 0x7FFFFFu) >> kSh)), KeyParams<BS>::off);
            clamped |= kbits[e] == kCapBits;
          }
          if (!clamped) {
            *reinterpret_cast<float4*>(dp) = make_float4(nv[0], nv[1], nv[2], nv[3]);  // one 16-byte store
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if ((kbits[e] & kSlot) != 0u) dp[e] = nv[e];
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint32_t sl = kbits[e] & kSlot;
            if (sl != 0u) pp[e] = kb + (int)sl - 1;
          }
        }
      }
    }
    return;
  }
  uint64_t imp = 0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int gi = r0 + mp_row(ty, a);
    const bool band_r = (gi >= kb) && (gi < kb + BS);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gj = c0 + mp_col(tx, 4 * h);
      const bool band_c = (gj >= kb) && (gj < kb + BS);
      if (band_r || band_c) continue;
      float* dp = D + (size_t)gi * ld + gj;
      const float4 o4 = *reinterpret_cast<const float4*>(dp);
      const float old[4] = {o4.x, o4.y, o4.z, o4.w};
      float nv[4];
      bool any = false;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float dn = d[a][4 * h + e];
        const bool im = dn < old[e];
        nv[e] = im ? dn : old[e];
        if (im) imp |= 1ull << (a * 8 + 4 * h + e);
        any |= im;
      }
      if (any) *reinterpret_cast<float4*>(dp) = make_float4(nv[0], nv[1], nv[2], nv[3]);
    }
  }
  if (!__any_sync(0xffffffffu, imp != 0)) return;
  // Many improvements in this warp (early rounds): every lane re-runs its own
  // candidates, 16 elements at a time, with k descending, so the last match
  // it records is the first k whose sum equals the new value.
  const int wcnt = __reduce_add_sync(0xffffffffu, __popcll(imp));
  if (wcnt > kDenseRescan) {
#pragma unroll
    for (int a0 = 0; a0 < 8; a0 += 2) {
      if (!__any_sync(0xffffffffu, ((imp >> (a0 * 8)) & 0xFFFF) != 0)) continue;
      int pk[2][8];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 8; ++c) pk[q][c] = BS;
      const int ra0 = mp_row(ty, a0), ra1 = mp_row(ty, a0 + 1);
#pragma unroll 2
      for (int k = BS - 1; k >= 0; --k) {
        const float av[2] = {pan(As, k, ra0), pan(As, k, ra1)};
        float bv[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) bv[c] = pan_b(Bs, k, mp_col(tx, c));
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (__fadd_rn(av[q], bv[c]) == d[a0 + q][c]) pk[q][c] = k;
      }
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if ((imp >> ((a0 + q) * 8 + c)) & 1)
            P[(size_t)(r0 + mp_row(ty, a0 + q)) * ld + c0 + mp_col(tx, c)] = kb + pk[q][c];
    }
    return;
  }
#pragma unroll
  for (int slot = 0; slot < 64; ++slot) {
    unsigned bal = __ballot_sync(0xffffffffu, (imp >> slot) & 1);
    if (!bal) continue;
    const int a = slot >> 3, c = slot & 7;
    const float dmine = d[a][c];
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      const int stid = warp * 32 + src;
      const int li = mp_row(stid >> 4, a), lj = mp_col(stid & 15, c);
      const float dn = __shfl_sync(0xffffffffu, dmine, src);
      int kstar = BS;
#pragma unroll
      for (int m = 0; m < BS / 32; ++m) {
        const int k = m * 32 + lane;
        const float cand = __fadd_rn(pan(As, k, li), pan_b(Bs, k, lj));
        const unsigned eq = __ballot_sync(0xffffffffu, cand == dn);
        if (eq && kstar == BS) kstar = m * 32 + __ffs(eq) - 1;
      }
      if (lane == src) P[(size_t)(r0 + li) * ld + c0 + lj] = kb + kstar;
    }
  }
}

__device__ __forceinline__ void spin_cycles(long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
  }
}

// Panel slices of round r in the layout phase 3 reads, written once per round
// by fw_pack_panels_f32_kernel: slice tr of Apk holds A[i][k] (rows tr*128 ..
// tr*128+127, the BS columns of block r) at [kp*kS2 + 2i + (k&1)], slice tc of
// Bpk holds B[k][j] (the BS rows of block r, columns tc*128 ..) at
// [kp*kS2 + bcol(j, k&1)] (swizzled chunks). On keyed rounds A holds
// 2^23 + M*a + k + 1 and B holds M*b.
template <int BS>
__host__ __device__ constexpr size_t panel_slice_floats() {
  return (size_t)(BS / 2) * kS2;
}

template <int BS>
__device__ __forceinline__ bool round_keyed(const RoundMax* rm, int graph_int) {
  return graph_int != 0 &&
         __int_as_float((int)rm->a_bits) + __int_as_float((int)rm->b_bits) <= KeyParams<BS>::bound;
}

// Floats per k-pair row of a B slice WB columns wide (128 for the integer
// kernel, 64 for the real-weight kernel), padded like kS2.
template <int WB>
__host__ __device__ constexpr int b_slice_stride() {
  return 2 * WB + 8;
}

// CTAs 0 .. nT-1 pack the A slices (tile rows), the next n_pad/WB CTAs the B
// slices (column tiles WB wide).
template <int BS, int WB = kTile>
__global__ void __launch_bounds__(256) fw_pack_panels_f32_kernel(const float* __restrict__ D, size_t ld, int nT, int r,
                                                                 const RoundMax* __restrict__ rm, int graph_int,
                                                                 float* __restrict__ Apk, float* __restrict__ Bpk) {
  constexpr float M = KeyParams<BS>::M;
  pdl_prologue();
  const bool keyed = round_keyed<BS>(rm, graph_int);
  const float mb = keyed ? M : 1.f;
  const int kb = r * BS, tid = threadIdx.x;
  if ((int)blockIdx.x < nT) {
    // 128 rows x BS columns; a 128-bit load of row i holds k = 4q4..4q4+3, i.e. two k pairs.
    // Lane -> (row ri = lane & 7 of an 8-row group, column quad cq = lane >> 3).
    const int r0 = blockIdx.x * kTile;
    float* As = Apk + panel_slice_floats<BS>() * blockIdx.x;
#pragma unroll
    for (int m = 0; m < BS / 8; ++m) {
      const int idx = tid + 256 * m;
      const int ri = idx & 7, cq = (idx >> 3) & 3, grp = idx >> 5;
      const int i = (grp % (kTile / 8)) * 8 + ri;
      const int q4 = (grp / (kTile / 8)) * 4 + cq;
      const float4 v = *reinterpret_cast<const float4*>(D + (size_t)(r0 + i) * ld + kb + q4 * 4);
      const float k0 = keyed ? KeyParams<BS>::off + (float)(q4 * 4 + 1) : 0.f;  // exact below 2^24
      const float k1 = keyed ? k0 + 1.f : 0.f, k2 = keyed ? k0 + 2.f : 0.f, k3 = keyed ? k0 + 3.f : 0.f;
      *reinterpret_cast<float2*>(As + (2 * q4) * kS2 + 2 * i) = make_float2(fmaf(v.x, mb, k0), fmaf(v.y, mb, k1));
      *reinterpret_cast<float2*>(As + (2 * q4 + 1) * kS2 + 2 * i) = make_float2(fmaf(v.z, mb, k2), fmaf(v.w, mb, k3));
    }
  } else {
    // rows 2kp and 2kp+1 of one column quad -> two interleaved 128-bit stores
    constexpr int QW = WB / 4, SB = b_slice_stride<WB>();
    const int tc = blockIdx.x - nT, c0 = tc * WB;
    float* Bs = Bpk + (size_t)(BS / 2) * SB * tc;
#pragma unroll
    for (int m = 0; m < (BS / 2) * QW / 256; ++m) {
      const int idx = tid + 256 * m, kp = idx / QW, q = idx % QW;
      const float4 x = *reinterpret_cast<const float4*>(D + (size_t)(kb + 2 * kp) * ld + c0 + q * 4);
      const float4 y = *reinterpret_cast<const float4*>(D + (size_t)(kb + 2 * kp + 1) * ld + c0 + q * 4);
      *reinterpret_cast<float4*>(Bs + kp * SB + 4 * bswz(2 * q)) = make_float4(x.x * mb, y.x * mb, x.y * mb, y.y * mb);
      *reinterpret_cast<float4*>(Bs + kp * SB + 4 * bswz(2 * q + 1)) =
          make_float4(x.z * mb, y.z * mb, x.w * mb, y.w * mb);
    }
  }
}

// One launch per round; one CTA per 128x128 tile, two CTAs per SM.
//   rm:        the round's panel maxima written by phases 1-2
//   graph_int: every weight of the graph is an integer (so every D value is)
//   Apk, Bpk:  the round's packed panel slices (fw_pack_panels_f32_kernel)
//   stagger:   CTAs sms .. 2*sms-1 (the first wave's second half) start this
//              many cycles late, so the first wave's SMs do not all load their
//              tiles from HBM at the same instant
//   wait_ns:   limit of the wait for the panel slices; when it expires the CTA
//              sets kFaultPanelCopyTimeout in g_apsp_fault and leaves its tile
//   no_copy:   testing only: announce the slices but never copy them, so the
//              wait expires (the timeout path, with no copy in flight)
// A thread issues two bulk copies (the A and B slices of this tile) before the
// CTA loads its tile, so the copies overlap the tile load.
template <int BS>
__global__ void __launch_bounds__(256, 2) fw_phase3_f32_kernel(float* __restrict__ D, int32_t* __restrict__ P,
                                                               size_t ld, int nT, int r, RoundMax* rm, int graph_int, const float* __restrict__ Apk,
                                                               const float* __restrict__ Bpk, int stagger, int sms,
                                                               unsigned long long wait_ns, int no_copy) {
  extern __shared__ __align__(16) float sm[];
  __shared__ uint64_t bar;
  pdl_prologue();
  const int kb = r * BS;
  const int tr = blockIdx.x / nT, tc = blockIdx.x - tr * nT;
  const int r0 = tr * kTile, c0 = tc * kTile;
  // Tiles entirely inside row band r or column band r belong to phases 1-2.
  if ((r0 >= kb && r0 + kTile <= kb + BS) || (c0 >= kb && c0 + kTile <= kb + BS)) return;
  const bool keyed = round_keyed<BS>(rm, graph_int);
  if (stagger > 0 && (int)blockIdx.x >= sms && (int)blockIdx.x < 2 * sms) spin_cycles(stagger);
  float* As = sm;
  float* Bs = sm + panel_slice_floats<BS>();
  constexpr unsigned slice_bytes = (unsigned)(panel_slice_floats<BS>() * sizeof(float));
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, 2 * slice_bytes);
    if (!no_copy) {
      bulk_copy_g2s(As, Apk + panel_slice_floats<BS>() * tr, slice_bytes, &bar);
      bulk_copy_g2s(Bs, Bpk + panel_slice_floats<BS>() * tc, slice_bytes, &bar);
    }
  }
  tile_body<BS>(D, P, ld, kb, r0, c0, keyed, As, Bs, &bar, wait_ns, rm);
}

// ---------------------------------------------------------------- real-valued graphs
//
// Phase 3 for graphs with non-integer weights (no keys). One CTA of 256
// threads per 128 x 64 tile, 8 x 4 elements per thread (rows as in the integer
// kernel, four consecutive columns). The BS intermediates run in groups of
// eight k pairs; at the end of each group every element compares itself with
// its value at the group's start and, if it fell, records the group (a 4-bit
// tag; the first group's start is the old D). The tags name every improved
// element and the group holding its last strict improvement, which contains
// the first k attaining its final value (an earlier group cannot reach that
// value, or the later group could not have fallen to it). So the old tile is
// never re-read, and each improved element is searched over 16 candidates only:
// the warp lists them in shared memory and each lane takes listed elements.
// The A slices are the integer kernel's; the B slices are packed 64 columns
// wide (fw_pack_panels_f32_kernel<BS, 64>).
constexpr int kRealCols = 64;
constexpr int kRealSB = 2 * kRealCols + 8;      // floats per k-pair row of a B slice
// k pairs per tagged group: 16 measured slower (n = 8192: 17.3 vs 19.4 TFLOPS;
// n = 32768: 24.3 vs 25.0), as the searches double while the bookkeeping halves.
constexpr int kRealGroup = 8;
constexpr int kRealQueueFlush = kQueuePerWarp - 128;  // a row adds at most 32 x 4 entries

template <int BS>
__host__ __device__ constexpr size_t real_b_slice_floats() {
  return (size_t)(BS / 2) * kRealSB;
}

template <int BS>
constexpr size_t minplus_f32_real_smem_bytes() {
  return sizeof(float) * (panel_slice_floats<BS>() + real_b_slice_floats<BS>()) + sizeof(int2) * 8 * kQueuePerWarp;
}

template <int BS>
__global__ void __launch_bounds__(256, 2) fw_phase3_f32_real_kernel(float* __restrict__ D, int32_t* __restrict__ P,
                                                                    size_t ld, int nT, int r, RoundMax* rm,
                                                                    const float* __restrict__ Apk,
                                                                    const float* __restrict__ Bpk, int stagger,
                                                                    int sms, unsigned long long wait_ns, int no_copy) {
  extern __shared__ __align__(16) float sm[];
  __shared__ uint64_t bar;
  pdl_prologue();
  constexpr int NG = BS / (2 * kRealGroup);  // groups of kRealGroup k pairs (tags 1..NG fit in 4 bits)
  static_assert(NG >= 1 && NG <= 15, "group tags need 4 bits");
  const int kb = r * BS;
  const int nTc = nT * (kTile / kRealCols);
  const int tr = blockIdx.x / nTc, tc = blockIdx.x - tr * nTc;
  const int r0 = tr * kTile, c0 = tc * kRealCols;
  if ((r0 >= kb && r0 + kTile <= kb + BS) || (c0 >= kb && c0 + kRealCols <= kb + BS)) return;
  if (stagger > 0 && (int)blockIdx.x >= sms && (int)blockIdx.x < 2 * sms) spin_cycles(stagger);
  float* As = sm;
  float* Bs = sm + panel_slice_floats<BS>();
  int2* queue = reinterpret_cast<int2*>(Bs + real_b_slice_floats<BS>());
  constexpr unsigned a_bytes = (unsigned)(panel_slice_floats<BS>() * sizeof(float));
  constexpr unsigned b_bytes = (unsigned)(real_b_slice_floats<BS>() * sizeof(float));
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31, warp = tid >> 5;
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar, a_bytes + b_bytes);
    if (!no_copy) {
      bulk_copy_g2s(As, Apk + panel_slice_floats<BS>() * tr, a_bytes, &bar);
      bulk_copy_g2s(Bs, Bpk + real_b_slice_floats<BS>() * tc, b_bytes, &bar);
    }
  }
  float d[8][4], ds[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const float4 v = *reinterpret_cast<const float4*>(D + (size_t)(r0 + mp_row(ty, a)) * ld + c0 + tx * 4);
    d[a][0] = v.x; d[a][1] = v.y; d[a][2] = v.z; d[a][3] = v.w;
#pragma unroll
    for (int c = 0; c < 4; ++c) ds[a][c] = d[a][c];
  }
  if (!__syncthreads_and(mbar_wait_phase0(&bar, wait_ns))) {
    if (tid == 0) report_fault(rm, kFaultPanelCopyTimeout);
    mbar_wait_phase0(&bar, wait_ns);  // copies still in flight land before the CTA exits
    return;
  }
  uint32_t tag[4] = {0u, 0u, 0u, 0u};  // element e = a*4 + c: bits 4*(e&7) of tag[e>>3]
  const float* Ap = As + ty * 8;
  const float* Bp0 = Bs + 4 * bswz(2 * tx);
  const float* Bp1 = Bs + 4 * bswz(2 * tx + 1);
#pragma unroll 1
  for (int g = 0; g < NG; ++g) {
#pragma unroll 1
    for (int u = 0; u < kRealGroup; ++u) {
      const int kp = g * kRealGroup + u;
      const float4 a0 = *reinterpret_cast<const float4*>(Ap + kp * kS2);
      const float4 a1 = *reinterpret_cast<const float4*>(Ap + kp * kS2 + 4);
      const float4 a2 = *reinterpret_cast<const float4*>(Ap + kp * kS2 + 128);
      const float4 a3 = *reinterpret_cast<const float4*>(Ap + kp * kS2 + 132);
      const float4 b0 = *reinterpret_cast<const float4*>(Bp0 + kp * kRealSB);
      const float4 b1 = *reinterpret_cast<const float4*>(Bp1 + kp * kRealSB);
      const float2 av[8] = {{a0.x, a0.y}, {a0.z, a0.w}, {a1.x, a1.y}, {a1.z, a1.w},
                            {a2.x, a2.y}, {a2.z, a2.w}, {a3.x, a3.y}, {a3.z, a3.w}};
      const float2 bv[4] = {{b0.x, b0.y}, {b0.z, b0.w}, {b1.x, b1.y}, {b1.z, b1.w}};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 sv = fadd2_rn(av[a], bv[c]);
          d[a][c] = fminf(fminf(d[a][c], sv.x), sv.y);
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int e = a * 4 + c, sh = 4 * (e & 7);
        if (d[a][c] < ds[a][c]) tag[e >> 3] = (tag[e >> 3] & ~(0xFu << sh)) | ((uint32_t)(g + 1) << sh);
        ds[a][c] = d[a][c];
      }
  }
  // Write back improved rows of four; list improved elements (group, row, column, value).
  int2* wq = queue + warp * kQueuePerWarp;
  const unsigned lt = (1u << lane) - 1u;
  const int gj = c0 + tx * 4;
  const bool band_c = (gj >= kb) && (gj < kb + BS);
  int cnt = 0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int li = mp_row(ty, a);
    const int gi = r0 + li;
    const bool band = band_c || ((gi >= kb) && (gi < kb + BS));
    const uint32_t row_tags = (tag[a >> 1] >> (16 * (a & 1))) & 0xFFFFu;  // elements a*4 .. a*4+3
    if (!band && row_tags != 0)
      *reinterpret_cast<float4*>(D + (size_t)gi * ld + gj) = make_float4(d[a][0], d[a][1], d[a][2], d[a][3]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t gt = (row_tags >> (4 * c)) & 0xFu;
      const bool bit = !band && gt != 0;
      const unsigned bal = __ballot_sync(0xffffffffu, bit);
      if (bit)
        wq[cnt + __popc(bal & lt)] = make_int2((int)(gt << 16) | (li << 8) | (tx * 4 + c), __float_as_int(d[a][c]));
      cnt += __popc(bal);
    }
    if (cnt >= kRealQueueFlush || (a == 7 && cnt > 0)) {
      __syncwarp();
#pragma unroll 1
      for (int e = lane; e < cnt; e += 32) {
        const int2 ent = wq[e];
        const int kp0 = ((ent.x >> 16) - 1) * kRealGroup;
        const int qi = (ent.x >> 8) & 255, qj = ent.x & 255;
        const float dn = __int_as_float(ent.y);
        float2 c2[kRealGroup];
#pragma unroll
        for (int u = 0; u < kRealGroup; ++u)
          c2[u] = fadd2_rn(*reinterpret_cast<const float2*>(As + (kp0 + u) * kS2 + 2 * qi),
                           *reinterpret_cast<const float2*>(Bs + (kp0 + u) * kRealSB + bcol(qj, 0)));
        int kstar = BS;
#pragma unroll
        for (int u = kRealGroup - 1; u >= 0; --u) {
          if (c2[u].y == dn) kstar = 2 * (kp0 + u) + 1;
          if (c2[u].x == dn) kstar = 2 * (kp0 + u);
        }
        P[(size_t)(r0 + qi) * ld + c0 + qj] = kb + kstar;
      }
      __syncwarp();
      cnt = 0;
    }
  }
}

}  // namespace apsp
