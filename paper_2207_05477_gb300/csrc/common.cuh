// Shared device/host helpers of libevo (internal).
#pragma once
#include <utility>
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

// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_entry(): it waits until the kernels before it in the stream have
// finished and their writes are visible (griddepcontrol.wait), then lets the
// next kernel's blocks be scheduled as soon as all of this kernel's blocks
// have started (griddepcontrol.launch_dependents).  The next kernel's launch
// and prologue thus overlap this kernel's tail, while no kernel touches
// memory before its predecessors are done.  Kernels launched without the
// attribute (pdl_enabled() false) see both instructions as no-ops.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// The two halves, for kernels with a prologue that touches no global memory
// (barrier set-up, tensor-memory allocation): trigger first, wait after it.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch attribute switch (on unless EVO_PDL=0 in the environment).
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Output index map of GEMM epilogues:
// offset(m, n) = (m / mdiv) * s_m1 + (m % mdiv) * s_m0 + (n / ndiv) * s_n1 + (n % ndiv) * s_n0
// A divisor of 2^31 or more means "no split" along that index; splits use
// 32-bit division (row and column indices are below 2^31).
struct OutMap {
  int64_t mdiv, s_m1, s_m0, ndiv, s_n1, s_n0;
  __host__ __device__ __forceinline__ int64_t row(int m) const {
    if (mdiv >= (1ll << 31)) return (int64_t)m * s_m0;
    const int d = (int)mdiv, q = m / d;
    return (int64_t)q * s_m1 + (int64_t)(m - q * d) * s_m0;
  }
  __host__ __device__ __forceinline__ int64_t col(int n) const {
    if (ndiv >= (1ll << 31)) return (int64_t)n * s_n0;
    const int d = (int)ndiv, q = n / d;
    return (int64_t)q * s_n1 + (int64_t)(n - q * d) * s_n0;
  }
  __host__ __device__ __forceinline__ int64_t operator()(int m, int n) const { return row(m) + col(n); }
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
  int atomic;       // fp32 C += v with atomics (split-K; no other epilogue step)
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

// Epilogue chain up to (not including) the residual add.
template <typename T>
__device__ __forceinline__ float epi_value(const Epi &e, int m, int n, float acc) {
  float v = e.alpha * acc;
  if (e.bias && n >= e.bias_n0) v += e.bias[n - e.bias_n0];
  if (e.row_scale) v *= e.row_scale[m];
  if (e.relu_ref && !(ldf((const T *)e.relu_ref + (int64_t)m * e.relu_ld + n) > 0.f)) v = 0.f;
  if (e.act == ACT_RELU) v = fmaxf(v, 0.f);
  else if (e.act == ACT_SIGMOID && n >= e.act_n0) v = 1.f / (1.f + __expf(-v));
  if (e.aux) stf((T *)e.aux + (int64_t)m * e.aux_ld + n, v);
  if (e.gate) v *= ldf((const T *)e.gate + (int64_t)m * e.gate_ld + n);
  return v;
}

template <typename T>
__device__ __forceinline__ void epi_store(const Epi &e, int b, int split, int m, int n, float acc) {
  if (e.partial) {
    e.partial[((int64_t)split * e.M + m) * e.N + n] = acc;
    return;
  }
  float v = epi_value<T>(e, m, n, acc);
  const int64_t off = (int64_t)b * e.c_bstride + e.map(m, n);
  if (e.residual) v += ldf((const T *)e.residual + off);
  if (e.c_f32) {
    float *c = (float *)e.C + off;
    if (e.accumulate) *c += v; else *c = v;
  } else {
    stf((T *)e.C + off, v);
  }
}

// Columns n and n+1 (n even) of row m: one 2-element vector load/store where
// the two outputs are adjacent and aligned, else two scalar ones.
template <typename T>
__device__ __forceinline__ void epi_pair(const Epi &e, int b, int split, int m, int n, int64_t rowoff, float a0,
                                         float a1) {
  const bool two = n + 1 < e.N;
  if (!two) {
    epi_store<T>(e, b, split, m, n, a0);
    return;
  }
  if (e.partial) {
    float *p = e.partial + ((int64_t)split * e.M + m) * e.N + n;
    if (((uintptr_t)p & 7u) == 0) *reinterpret_cast<float2 *>(p) = make_float2(a0, a1);
    else { p[0] = a0; p[1] = a1; }
    return;
  }
  float v0 = epi_value<T>(e, m, n, a0);
  float v1 = epi_value<T>(e, m, n + 1, a1);
  const int64_t off0 = rowoff + e.map.col(n);
  const int64_t off1 = rowoff + e.map.col(n + 1);
  const bool vec = off1 == off0 + 1 && (off0 & 1) == 0;
  if (e.residual) {
    const T *r = (const T *)e.residual;
    if (vec && is_bf16<T>::value) {
      const __nv_bfloat162 rr = *reinterpret_cast<const __nv_bfloat162 *>(r + off0);
      v0 += __low2float(rr);
      v1 += __high2float(rr);
    } else {
      v0 += ldf(r + off0);
      v1 += ldf(r + off1);
    }
  }
  if (e.c_f32) {
    float *c = (float *)e.C;
    if (e.accumulate) {
      c[off0] += v0;
      c[off1] += v1;
    } else if (vec) {
      *reinterpret_cast<float2 *>(c + off0) = make_float2(v0, v1);
    } else {
      c[off0] = v0;
      c[off1] = v1;
    }
  } else {
    T *c = (T *)e.C;
    if (vec && is_bf16<T>::value) {
      *reinterpret_cast<__nv_bfloat162 *>(c + off0) = __floats2bfloat162_rn(v0, v1);
    } else if (vec) {
      *reinterpret_cast<float2 *>(c + off0) = make_float2(v0, v1);
    } else {
      stf(c + off0, v0);
      stf(c + off1, v1);
    }
  }
}

}  // namespace evo
