// The phase-3 hot loop with its panel pairs read from shared memory, as the
// fp32 phase-3 kernel reads them, for several register tiles per thread and
// two warp footprints (timing only: no global traffic besides one checksum
// per thread). The rates it prints bound what a kernel of that tile shape can
// reach in its hot loop.
//
// Standalone program, not part of the library:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o smem_tiles smem_tiles.cu && ./smem_tiles
//
// 256 threads as 16 x 16 (ty, tx); LAYOUT 0 gives each warp 2 x 16 threads (the
// kernel's), LAYOUT 1 gives it 4 x 8. Each thread owns rows g*64 + ty*4 + {0..3}
// and columns g*64 + tx*4 + {0..3} of the CTA tile; a k pair costs two 128-bit
// shared loads per group of four rows or columns.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
constexpr int BS = 64, KP = BS / 2, TY = 16, TX = 16;
template <int TM, int TN, int MINB, int LAYOUT>
__global__ void __launch_bounds__(256, MINB) hot(uint32_t* out, int reps) {
  constexpr int ROWS = TM * TY, COLS = TN * TX;
  extern __shared__ __align__(16) float sm[];
  float* As = sm;                  // [KP][ROWS * 2]
  float* Bs = sm + KP * ROWS * 2;  // [KP][COLS * 2]
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int ty = LAYOUT ? (w >> 1) * 4 + (l >> 3) : tid / TX, tx = LAYOUT ? (w & 1) * 8 + (l & 7) : tid % TX;
  for (int i = tid; i < KP * ROWS * 2; i += 256) As[i] = (float)((i * 7 + blockIdx.x) & 1023);
  for (int i = tid; i < KP * COLS * 2; i += 256) Bs[i] = (float)((i * 13 + blockIdx.x) & 1023);
  __syncthreads();
  float d[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int c = 0; c < TN; ++c) d[a][c] = 4096.f + a + c + tid;
  for (int rep = 0; rep < reps; ++rep) {
#pragma unroll 1
    for (int kp = 0; kp < KP; ++kp) {
      float2 av[TM], bv[TN];
#pragma unroll
      for (int g = 0; g < TM / 4; ++g) {
        const float* p = As + kp * ROWS * 2 + (g * TY * 4 + ty * 4) * 2;
        const float4 x = *reinterpret_cast<const float4*>(p), y = *reinterpret_cast<const float4*>(p + 4);
        av[g * 4 + 0] = make_float2(x.x, x.y); av[g * 4 + 1] = make_float2(x.z, x.w);
        av[g * 4 + 2] = make_float2(y.x, y.y); av[g * 4 + 3] = make_float2(y.z, y.w);
      }
#pragma unroll
      for (int g = 0; g < TN / 4; ++g) {
        const float* p = Bs + kp * COLS * 2 + (g * TX * 4 + tx * 4) * 2;
        const float4 x = *reinterpret_cast<const float4*>(p), y = *reinterpret_cast<const float4*>(p + 4);
        bv[g * 4 + 0] = make_float2(x.x, x.y); bv[g * 4 + 1] = make_float2(x.z, x.w);
        bv[g * 4 + 2] = make_float2(y.x, y.y); bv[g * 4 + 3] = make_float2(y.z, y.w);
      }
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
          const float2 s = add2(av[a], bv[c]);
          d[a][c] = fminf(fminf(d[a][c], s.x), s.y);
        }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int c = 0; c < TN; ++c) s += __float_as_uint(d[a][c]);
  out[(size_t)blockIdx.x * 256 + tid] = s;
}
template <int TM, int TN, int MINB, int LAYOUT>
int run(const char* name, uint32_t* out, int sms, int ctas_per_sm) {
  const size_t smem = sizeof(float) * KP * 2 * (TM * TY + TN * TX);
  if (cudaFuncSetAttribute(hot<TM, TN, MINB, LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
  const int grid = sms * ctas_per_sm;
  const int reps = 16384 / (TM * TN);  // about the same time per launch
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms = 0.f;
  for (int it = 0; it < 3; ++it) {
    cudaEventRecord(e0); hot<TM, TN, MINB, LAYOUT><<<grid, 256, smem>>>(out, reps); cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
    cudaEventElapsedTime(&ms, e0, e1);
  }
  const double relax = (double)grid * 256 * TM * TN * BS * reps;
  printf("%-10s smem %6zu B  %8.3f ms  %6.1f relax/clk/SM (%5.1f TFLOP/s at 2070 MHz)\n", name, smem, ms,
         relax / (ms * 1e-3) / sms / 2.07e9, 2.0 * relax / (ms * 1e-3) / 1e12);
  return 0;
}
int main() {
  int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, sizeof(uint32_t) * (size_t)sms * 8 * 256) != cudaSuccess) return 1;
  int rc = 0;
  rc |= run<8, 8, 2, 0>("8x8 2x16", out, sms, 8);
  rc |= run<8, 8, 2, 1>("8x8 4x8", out, sms, 8);
  rc |= run<8, 4, 3, 0>("8x4 2x16", out, sms, 8);
  rc |= run<8, 4, 3, 1>("8x4 4x8", out, sms, 8);
  rc |= run<4, 8, 3, 0>("4x8 2x16", out, sms, 8);
  rc |= run<4, 4, 4, 0>("4x4 2x16", out, sms, 8);
  const cudaError_t e = cudaDeviceSynchronize();
  printf("%s\n", (e == cudaSuccess && !rc) ? "ok" : "failed");
  return (e == cudaSuccess && !rc) ? 0 : 1;
}
