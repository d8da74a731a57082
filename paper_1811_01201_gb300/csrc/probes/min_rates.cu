// Issue rates of the instructions a phase-3 relaxation D = min(D, A + B) can
// be built from, measured on register operands (no memory traffic). The
// roofline of the phase-3 kernels is derived from these rates.
//
// Standalone program, not part of the library:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o min_rates min_rates.cu && ./min_rates
//
// The instruction cases run 8 (or 16) independent chains per thread; the
// register-tile cases 16 to 64, with the occupancy their registers allow. All
// launch 256 threads x 4 CTAs per SM and report units per clock per SM at
// 2070 MHz (the maximum SM clock; the clock is not sampled here). An empty volatile asm on an operand
// each step keeps the compiler from hoisting or folding; where the
// accumulator also passes through one, two successive mins cannot be fused
// into a three-input min.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ float2 add_f32x2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ uint32_t add_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("add.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

enum Case {
  kFminUnfused,     // min.f32, accumulator fenced: one FMNMX per step
  kFmin3,           // three-input min.f32 (sm_100 and later)
  kRelaxF32,        // add.rn.f32x2 + two mins per k pair (the fp32 phase-3 pattern)
  kMinS32Unfused,   // min.s32, accumulator fenced
  kMinU16x2Unfused, // min.u16x2, accumulator fenced
  kRelaxU16,        // add.u16x2 + min.u16x2 (the 16-bit phase-3 pattern)
  kAddMinS32,       // __viaddmin_s32: min(a + b, c)
  kAddMinU16x2,     // __viaddmin_u16x2
  kCases
};

template <int C, int E>
__global__ void rate_kernel(uint32_t* out, int iters, uint32_t seed) {
  float fd[E], fx[E], fy[E];
  uint32_t ud[E], ux[E], uy[E];
  float2 fa[E], fb;
  uint32_t ua[E], ub;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    fd[q] = 1e6f + q + threadIdx.x;
    fx[q] = (float)(seed + q);
    fy[q] = (float)(seed + 3 * q);
    fa[q] = make_float2((float)(seed + q), (float)(2 * seed + q));
    ud[q] = 0x7FFF7FFFu - threadIdx.x - q;
    ux[q] = seed * (q + 1);
    uy[q] = 0x7FF07FF0u - q;
    ua[q] = seed + 5u * q;
  }
  fb = make_float2((float)(5 * seed), (float)(7 * seed));
  ub = seed * 9u;
  for (int it = 0; it < iters; ++it) {
    asm volatile("" : "+f"(fb.x), "+f"(fb.y), "+r"(ub));
#pragma unroll
    for (int q = 0; q < E; ++q) {
      if (C == kFminUnfused) {
        asm volatile("" : "+f"(fx[q]));
        fd[q] = fminf(fd[q], fx[q]);
        asm volatile("" : "+f"(fd[q]));
      } else if (C == kFmin3) {
        asm volatile("" : "+f"(fx[q]), "+f"(fy[q]));
        asm("min.f32 %0, %0, %1, %2;" : "+f"(fd[q]) : "f"(fx[q]), "f"(fy[q]));
      } else if (C == kRelaxF32) {
        const float2 s = add_f32x2(fa[q], fb);
        fd[q] = fminf(fminf(fd[q], s.x), s.y);
      } else if (C == kMinS32Unfused) {
        asm volatile("" : "+r"(ux[q]));
        ud[q] = (uint32_t)min((int)ud[q], (int)ux[q]);
        asm volatile("" : "+r"(ud[q]));
      } else if (C == kMinU16x2Unfused) {
        asm volatile("" : "+r"(ux[q]));
        ud[q] = min_u16x2(ud[q], ux[q]);
        asm volatile("" : "+r"(ud[q]));
      } else if (C == kRelaxU16) {
        ud[q] = min_u16x2(ud[q], add_u16x2(ua[q], ub));
      } else if (C == kAddMinS32) {
        asm volatile("" : "+r"(ux[q]));
        ud[q] = (uint32_t)__viaddmin_s32((int)ud[q], (int)ux[q], (int)uy[q]);
      } else if (C == kAddMinU16x2) {
        asm volatile("" : "+r"(ux[q]));
        ud[q] = __viaddmin_u16x2(ud[q], ux[q], uy[q]);
      }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < E; ++q) s += ud[q] + __float_as_uint(fd[q]);
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The phase-3 register tile: RA x RC accumulators per thread, each k pair
// one add.rn.f32x2 per (a, c) and two mins, operands renewed every step (as
// the kernel renews them from shared memory) but never loaded.
template <int RA, int RC, int MINB>
__global__ void __launch_bounds__(256, MINB) outer_kernel(uint32_t* out, int iters, uint32_t seed) {
  float d[RA][RC];
  float2 av[RA], bv[RC];
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    av[a] = make_float2((float)(seed + a), (float)(2 * seed + a));
#pragma unroll
    for (int c = 0; c < RC; ++c) d[a][c] = 1e6f + a * RC + c + threadIdx.x;
  }
#pragma unroll
  for (int c = 0; c < RC; ++c) bv[c] = make_float2((float)(3 * seed + c), (float)(5 * seed + c));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int a = 0; a < RA; ++a) asm volatile("" : "+f"(av[a].x), "+f"(av[a].y));
#pragma unroll
    for (int c = 0; c < RC; ++c) asm volatile("" : "+f"(bv[c].x), "+f"(bv[c].y));
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        const float2 s = add_f32x2(av[a], bv[c]);
        d[a][c] = fminf(fminf(d[a][c], s.x), s.y);
      }
  }
  uint32_t s = 0;
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int c = 0; c < RC; ++c) s += __float_as_uint(d[a][c]);
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

struct Row {
  const char* name;
  void (*kernel)(uint32_t*, int, uint32_t);
  int chains;
  double units_per_step;  // instructions, or relaxations for the relaxation patterns
  const char* unit;
};

}  // namespace

int main() {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) return 1;
  const int threads = 256, blocks = sms * 4, iters = 1 << 15;
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, sizeof(uint32_t) * (size_t)blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const Row rows[] = {
      {"min.f32 (FMNMX), unfused", rate_kernel<kFminUnfused, 8>, 8, 1.0, "instr"},
      {"min.f32 three-input", rate_kernel<kFmin3, 8>, 8, 1.0, "instr"},
      {"add.rn.f32x2 + 2 min, 8 chains", rate_kernel<kRelaxF32, 8>, 8, 2.0, "relax"},
      {"add.rn.f32x2 + 2 min, 16 chains", rate_kernel<kRelaxF32, 16>, 16, 2.0, "relax"},
      {"min.s32, unfused", rate_kernel<kMinS32Unfused, 8>, 8, 1.0, "instr"},
      {"min.u16x2, unfused", rate_kernel<kMinU16x2Unfused, 8>, 8, 1.0, "instr"},
      {"add.u16x2 + min.u16x2, 8 chains", rate_kernel<kRelaxU16, 8>, 8, 2.0, "relax"},
      {"__viaddmin_s32", rate_kernel<kAddMinS32, 8>, 8, 1.0, "instr"},
      {"__viaddmin_u16x2", rate_kernel<kAddMinU16x2, 8>, 8, 1.0, "instr"},
      {"8x8 register tile (phase-3 kernel)", outer_kernel<8, 8, 2>, 64, 2.0, "relax"},
      {"8x4 register tile", outer_kernel<8, 4, 3>, 32, 2.0, "relax"},
      {"4x4 register tile", outer_kernel<4, 4, 4>, 16, 2.0, "relax"},
  };
  for (const Row& r : rows) {
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {  // the last of three launches is reported
      cudaEventRecord(e0);
      r.kernel<<<blocks, threads>>>(out, iters, 12345u + rep);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
      cudaEventElapsedTime(&ms, e0, e1);
    }
    const double units = (double)blocks * threads * r.chains * iters * r.units_per_step;
    std::printf("%-34s %8.3f ms  %6.1f %s/clk/SM at 2070 MHz\n", r.name, ms,
                units / (ms * 1e-3) / sms / 2.07e9, r.unit);
  }
  const cudaError_t e = cudaDeviceSynchronize();
  std::printf("%s\n", e == cudaSuccess ? "ok" : cudaGetErrorString(e));
  cudaFree(out);
  return e == cudaSuccess ? 0 : 1;
}
