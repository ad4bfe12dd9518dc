// Throughput probe of the special-function unit's 2^x, the bound of the
// attention softmax at small head dims.  Every thread keeps eight independent
// chains x <- 2^(a x + b) going for `iters` steps (one FMA and one ex2 each)
// and writes one float, so the rate is ex2 results per second of the launch.
//   variant 0: ex2.approx.ftz.f32 (one result per instruction)
//   variant 1: ex2.approx.ftz.bf16x2 (two results per instruction)
#include "evo.h"
#include "kernels.h"

namespace evo {
namespace {

__global__ void __launch_bounds__(256) ex2_probe_f32(int iters, float *sink) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = -0.001f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fmaf(x[k], -0.5f, -0.25f)));
      x[k] = y;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ex2_probe_bf16x2(int iters, float *sink) {
  uint32_t x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    __nv_bfloat162 v = __floats2bfloat162_rn(-0.001f * (float)(threadIdx.x + k), -0.002f * (float)k);
    x[k] = *reinterpret_cast<uint32_t *>(&v);
  }
  __nv_bfloat162 a2 = __floats2bfloat162_rn(-0.5f, -0.5f), b2 = __floats2bfloat162_rn(-0.25f, -0.25f);
  const uint32_t a = *reinterpret_cast<uint32_t *>(&a2), b = *reinterpret_cast<uint32_t *>(&b2);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t t, y;
      asm volatile("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(t) : "r"(x[k]), "r"(a), "r"(b));
      asm volatile("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(y) : "r"(t));
      x[k] = y;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&x[k]));
    s += f.x + f.y;
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace evo

extern "C" int evo_probe_ex2(int variant, int blocks, int iters, float *sink, evo_stream_t stream) {
  if (blocks <= 0 || iters <= 0 || !sink || (variant != 0 && variant != 1)) return EVO_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (variant == 0) evo::ex2_probe_f32<<<blocks, 256, 0, s>>>(iters, sink);
  else evo::ex2_probe_bf16x2<<<blocks, 256, 0, s>>>(iters, sink);
  return cudaGetLastError() == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}
