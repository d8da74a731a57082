// Element-wise kernels around the block rounds: input scan, initialisation of
// the working matrices, and copy-out of a padded or 16-bit working matrix.
#pragma once

#include "fw_common.cuh"

namespace apsp {

// Result of the input scan (device side; one per call).
struct WeightStats {
  unsigned int n_negative;   // weights < 0 (off the diagonal)
  unsigned int n_nan;        // NaN weights (off the diagonal)
  unsigned int n_fraction;   // finite weights that are not integers
  unsigned int max_bits;     // bit pattern of the largest finite weight (non-negative floats order as ints)
  unsigned int n_inf;        // absent edges (+INF off the diagonal)
};

// Scan W (n x n, leading dimension n) for the validity and 16-bit
// eligibility rules. Grid-stride, one atomic per counter per block.
__global__ void scan_weights_kernel(const float* __restrict__ W, int n, WeightStats* st) {
  __shared__ unsigned s_neg, s_nan, s_frac, s_max, s_inf;
  if (threadIdx.x == 0) { s_neg = 0; s_nan = 0; s_frac = 0; s_max = 0; s_inf = 0; }
  __syncthreads();
  unsigned neg = 0, nan = 0, frac = 0, mx = 0, inf = 0;
  const size_t total = (size_t)n * n;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t / n, j = t - i * n;
    if (i == j) continue;
    const float v = W[t];
    if (v != v) { ++nan; continue; }
    if (v < 0.f) { ++neg; continue; }
    if (v < f32_inf()) {
      if (v != floorf(v)) ++frac;
      mx = max(mx, (unsigned)__float_as_int(v));
    } else {
      ++inf;
    }
  }
  if (neg) atomicAdd(&s_neg, neg);
  if (nan) atomicAdd(&s_nan, nan);
  if (frac) atomicAdd(&s_frac, frac);
  if (inf) atomicAdd(&s_inf, inf);
  atomicMax(&s_max, mx);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_neg) atomicAdd(&st->n_negative, s_neg);
    if (s_nan) atomicAdd(&st->n_nan, s_nan);
    if (s_frac) atomicAdd(&st->n_fraction, s_frac);
    if (s_inf) atomicAdd(&st->n_inf, s_inf);
    atomicMax(&st->max_bits, s_max);
  }
}

// D (n_pad x n_pad) <- W (n x n) with a zero diagonal and INF padding;
// P <- -1; the solve's fault word <- 0. One thread per 4 consecutive
// destination columns.
__global__ void init_f32_kernel(const float* __restrict__ W, int n, float* __restrict__ D, int32_t* __restrict__ P,
                                int n_pad, unsigned* fault) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *fault = 0u;
  const size_t quads = (size_t)n_pad * (n_pad / 4);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < quads; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / (n_pad / 4));
    const int j0 = (int)(t - (size_t)i * (n_pad / 4)) * 4;
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = j0 + e;
      v[e] = (i < n && j < n) ? W[(size_t)i * n + j] : f32_inf();
      if (i == j) v[e] = 0.f;
    }
    *reinterpret_cast<float4*>(D + (size_t)i * n_pad + j0) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<int4*>(P + (size_t)i * n_pad + j0) = make_int4(-1, -1, -1, -1);
  }
}

// 16-bit working matrix: D16 <- W (integers below 0xFFFF, INF -> 0xFFFF).
__global__ void init_u16_kernel(const float* __restrict__ W, int n, uint16_t* __restrict__ D, int32_t* __restrict__ P,
                                int n_pad, unsigned* fault) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *fault = 0u;
  const size_t quads = (size_t)n_pad * (n_pad / 4);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < quads; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / (n_pad / 4));
    const int j0 = (int)(t - (size_t)i * (n_pad / 4)) * 4;
    uint32_t v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = j0 + e;
      const float w = (i < n && j < n) ? W[(size_t)i * n + j] : f32_inf();
      v[e] = (i == j) ? 0u : (w < f32_inf() ? (uint32_t)w : kInf16);
    }
    *reinterpret_cast<uint2*>(D + (size_t)i * n_pad + j0) = make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
    *reinterpret_cast<int4*>(P + (size_t)i * n_pad + j0) = make_int4(-1, -1, -1, -1);
  }
}

// Copy the leading n x n block of a padded working matrix out.
template <class S>
__global__ void copy_out_kernel(const S* __restrict__ src, int n_pad, S* __restrict__ dst, int n) {
  const size_t total = (size_t)n * n;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t / n, j = t - i * n;
    dst[t] = src[i * n_pad + j];
  }
}

// 16-bit working matrix -> fp32 distances (0xFFFF -> +INF).
__global__ void widen_u16_kernel(const uint16_t* __restrict__ src, int n_pad, float* __restrict__ dst, int n) {
  const size_t total = (size_t)n * n;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t / n, j = t - i * n;
    const uint32_t v = src[i * n_pad + j];
    dst[t] = (v == kInf16) ? f32_inf() : (float)v;
  }
}

}  // namespace apsp
