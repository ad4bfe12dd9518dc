// Shared device/host helpers of libevo (internal).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

typedef __nv_bfloat16 bf16;

#define EVO_LOG2E 1.4426950408889634f

namespace evo {

// ------------------------------------------------------------ load / store
__device__ __forceinline__ float ldf(const float *p) { return *p; }
__device__ __forceinline__ float ldf(const bf16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float *p, float v) { *p = v; }
__device__ __forceinline__ void stf(bf16 *p, float v) { *p = __float2bfloat16_rn(v); }

template <typename T> struct is_bf16 { static constexpr bool value = false; };
template <> struct is_bf16<bf16> { static constexpr bool value = true; };

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + __expf(-x)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Output index map of GEMM epilogues:
// offset(m, n) = (m / mdiv) * s_m1 + (m % mdiv) * s_m0 + (n / ndiv) * s_n1 + (n % ndiv) * s_n0
struct OutMap {
  int64_t mdiv, s_m1, s_m0, ndiv, s_n1, s_n0;
  __host__ __device__ __forceinline__ int64_t operator()(int64_t m, int64_t n) const {
    return (m / mdiv) * s_m1 + (m % mdiv) * s_m0 + (n / ndiv) * s_n1 + (n % ndiv) * s_n0;
  }
};

inline OutMap rowmajor_map(int64_t ld) { return OutMap{1ll << 40, 0, ld, 1ll << 40, 0, 1}; }

enum { ACT_NONE = 0, ACT_RELU = 1, ACT_SIGMOID = 2 };

// Epilogue of every GEMM: with acc = sum_k A(m,k) B(n,k),
//   v = alpha * acc; v += bias[n - bias_n0] (n >= bias_n0); v *= row_scale[m];
//   v *= (relu_ref[m, n] > 0); act (relu, or sigmoid for n >= act_n0);
//   aux[m, n] = v; v *= gate[m, n]; v += residual[map(m, n)];
//   C[map(m, n)] = v  (or C += v for fp32 accumulate; or split-K partial store).
struct Epi {
  void *C;
  int64_t c_bstride;
  OutMap map;
  int c_f32;        // C is fp32 (else the activation type)
  int accumulate;   // fp32 C += v
  float alpha;
  const float *bias;
  int bias_n0;
  const float *row_scale;
  int act, act_n0;
  const void *relu_ref;
  int64_t relu_ld;
  void *aux;
  int64_t aux_ld;
  const void *gate;
  int64_t gate_ld;
  const void *residual;
  float *partial;   // split-K: partial[(split * M + m) * N + n]
  int M, N;
};

template <typename T>
__device__ __forceinline__ void epi_store(const Epi &e, int b, int split, int m, int n, float acc) {
  if (e.partial) {
    e.partial[((int64_t)split * e.M + m) * e.N + n] = acc;
    return;
  }
  float v = e.alpha * acc;
  if (e.bias && n >= e.bias_n0) v += e.bias[n - e.bias_n0];
  if (e.row_scale) v *= e.row_scale[m];
  if (e.relu_ref && !(ldf((const T *)e.relu_ref + (int64_t)m * e.relu_ld + n) > 0.f)) v = 0.f;
  if (e.act == ACT_RELU) v = fmaxf(v, 0.f);
  else if (e.act == ACT_SIGMOID && n >= e.act_n0) v = 1.f / (1.f + __expf(-v));
  if (e.aux) stf((T *)e.aux + (int64_t)m * e.aux_ld + n, v);
  if (e.gate) v *= ldf((const T *)e.gate + (int64_t)m * e.gate_ld + n);
  const int64_t off = (int64_t)b * e.c_bstride + e.map(m, n);
  if (e.residual) v += ldf((const T *)e.residual + off);
  if (e.c_f32) {
    float *c = (float *)e.C + off;
    if (e.accumulate) *c += v; else *c = v;
  } else {
    stf((T *)e.C + off, v);
  }
}

}  // namespace evo
