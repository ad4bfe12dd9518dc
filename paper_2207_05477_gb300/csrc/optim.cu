// Fused training update over the flat parameter buffer: gradient clip by
// global norm, Adam and the EMA of the parameters (HelixFold Sec. 3.2, tensor
// fusion, and its table of kernel launches per stage).
//
// The paper's fused form takes O(1) launches per stage -- two for the clip
// (norm, then scale), one for the optimizer update, one for the EMA.  Here the
// whole update is two launches over the flat buffer:
//   1. adam_norm_k: each block writes the sum of squares of its grid-stride
//      share of the gradient (fp32 lanes, double across lanes) to the
//      workspace; no atomics, so the norm is the same on every run.
//   2. adam_update_k: every block first reduces the partials in the same fixed
//      order (a few KB from L2), forms the clip factor c / max(G, c), then in
//      one pass over the buffer scales the gradient, updates both Adam moments
//      and the parameter, the EMA and the BF16 shadow copy of the parameters
//      the tensor-core path reads.
// Both kernels are bound by HBM: 4 bytes per element for the norm, 28 more
// (p, g, m, v read; p, m, v written) plus 8 for the EMA and 2 for the BF16
// copy.  16-byte accesses, several in flight per thread; the grid is a
// multiple of the 152 SMs.
#include <cmath>
#include <initializer_list>
#include <algorithm>

#include "common.cuh"
#include "evo.h"
#include "prof.h"

namespace evo {
namespace {

constexpr int kThreads = 256;
constexpr int kNormBlocks = 152 * 8;   // upper bound on the norm grid (= partials in the workspace)
constexpr int kUpdBlocks = 152 * 3;    // update grid: three resident 256-thread blocks per SM
constexpr int kNormU = 4;              // float4 loads in flight per thread (norm)
constexpr int kUpdU = 2;               // float4 groups in flight per thread (update; 4-5 streams each)

struct AdamArgs {
  float lr_bc1;   // lr / (1 - beta1^t)
  float inv_bc2;  // 1 / (1 - beta2^t)
  float b1, omb1, b2, omb2, eps;
  float decay, omd;
  double clip;    // <= 0: no clipping
  int nparts;     // partial sums written by the norm kernel
};

__device__ __forceinline__ double block_sum_d(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

__global__ void __launch_bounds__(kThreads) adam_norm_k(const float *__restrict__ g, int64_t n,
                                                        double *__restrict__ part) {
  pdl_entry();
  __shared__ double red[kThreads / 32];
  const int64_t n4 = n >> 2;
  const float4 *g4 = reinterpret_cast<const float4 *>(g);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int64_t i = t;
  for (; i + (kNormU - 1) * stride < n4; i += kNormU * stride) {
    float4 x[kNormU];
#pragma unroll
    for (int u = 0; u < kNormU; ++u) x[u] = __ldg(g4 + i + u * stride);
#pragma unroll
    for (int u = 0; u < kNormU; ++u) {
      a0 = fmaf(x[u].x, x[u].x, a0);
      a1 = fmaf(x[u].y, x[u].y, a1);
      a2 = fmaf(x[u].z, x[u].z, a2);
      a3 = fmaf(x[u].w, x[u].w, a3);
    }
  }
  for (; i < n4; i += stride) {
    const float4 x = __ldg(g4 + i);
    a0 = fmaf(x.x, x.x, a0);
    a1 = fmaf(x.y, x.y, a1);
    a2 = fmaf(x.z, x.z, a2);
    a3 = fmaf(x.w, x.w, a3);
  }
  if (t < n - 4 * n4) {  // the last n % 4 elements, one per thread of block 0
    const float x = g[4 * n4 + t];
    a0 = fmaf(x, x, a0);
  }
  const double s = block_sum_d(((double)a0 + (double)a1) + ((double)a2 + (double)a3), red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <bool EMA, bool BF>
__device__ __forceinline__ void adam_elem(float &p, float g, float &m, float &v, float &e, float sc,
                                          const AdamArgs &a) {
  const float gg = g * sc;
  m = fmaf(a.b1, m, a.omb1 * gg);
  v = fmaf(a.b2, v, a.omb2 * (gg * gg));
  const float den = sqrtf(v * a.inv_bc2) + a.eps;
  p = p - a.lr_bc1 * (m / den);
  if (EMA) e = fmaf(a.decay, e, a.omd * p);
}

template <bool EMA, bool BF>
__global__ void __launch_bounds__(kThreads) adam_update_k(float *__restrict__ p, const float *__restrict__ g,
                                                          float *__restrict__ m, float *__restrict__ v,
                                                          float *__restrict__ e, bf16 *__restrict__ pb, int64_t n,
                                                          const double *__restrict__ part, AdamArgs a,
                                                          float *__restrict__ norm_out) {
  pdl_entry();
  __shared__ double red[kThreads / 32];
  __shared__ float s_scale;
  double acc = 0.0;
  for (int k = threadIdx.x; k < a.nparts; k += blockDim.x) acc += part[k];
  acc = block_sum_d(acc, red);
  if (threadIdx.x == 0) {
    const double G = sqrt(acc);
    s_scale = (a.clip > 0.0 && G > a.clip) ? (float)(a.clip / G) : 1.f;
    if (blockIdx.x == 0 && norm_out) *norm_out = (float)G;
  }
  __syncthreads();
  const float sc = s_scale;

  const int64_t n4 = n >> 2;
  float4 *p4 = reinterpret_cast<float4 *>(p);
  const float4 *g4 = reinterpret_cast<const float4 *>(g);
  float4 *m4 = reinterpret_cast<float4 *>(m);
  float4 *v4 = reinterpret_cast<float4 *>(v);
  float4 *e4 = reinterpret_cast<float4 *>(e);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

  auto body = [&](float4 &P, const float4 &Gv, float4 &M, float4 &V, float4 &E) {
    adam_elem<EMA, BF>(P.x, Gv.x, M.x, V.x, E.x, sc, a);
    adam_elem<EMA, BF>(P.y, Gv.y, M.y, V.y, E.y, sc, a);
    adam_elem<EMA, BF>(P.z, Gv.z, M.z, V.z, E.z, sc, a);
    adam_elem<EMA, BF>(P.w, Gv.w, M.w, V.w, E.w, sc, a);
  };
  auto store = [&](int64_t j, const float4 &P, const float4 &M, const float4 &V, const float4 &E) {
    p4[j] = P;
    m4[j] = M;
    v4[j] = V;
    if (EMA) e4[j] = E;
    if (BF) {
      __nv_bfloat162 lo = __floats2bfloat162_rn(P.x, P.y), hi = __floats2bfloat162_rn(P.z, P.w);
      uint2 w;
      w.x = *reinterpret_cast<unsigned *>(&lo);
      w.y = *reinterpret_cast<unsigned *>(&hi);
      reinterpret_cast<uint2 *>(pb)[j] = w;
    }
  };

  int64_t i = t;
  for (; i + (kUpdU - 1) * stride < n4; i += kUpdU * stride) {
    float4 P[kUpdU], Gv[kUpdU], M[kUpdU], V[kUpdU], E[kUpdU];
#pragma unroll
    for (int u = 0; u < kUpdU; ++u) {
      const int64_t j = i + u * stride;
      P[u] = p4[j];
      Gv[u] = __ldg(g4 + j);
      M[u] = m4[j];
      V[u] = v4[j];
      E[u] = EMA ? e4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kUpdU; ++u) {
      body(P[u], Gv[u], M[u], V[u], E[u]);
      store(i + u * stride, P[u], M[u], V[u], E[u]);
    }
  }
  for (; i < n4; i += stride) {
    float4 P = p4[i], M = m4[i], V = v4[i], E = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 Gv = __ldg(g4 + i);
    if (EMA) E = e4[i];
    body(P, Gv, M, V, E);
    store(i, P, M, V, E);
  }
  if (t < n - 4 * n4) {  // the last n % 4 elements
    const int64_t j = 4 * n4 + t;
    float P = p[j], M = m[j], V = v[j], E = EMA ? e[j] : 0.f;
    adam_elem<EMA, BF>(P, g[j], M, V, E, sc, a);
    p[j] = P;
    m[j] = M;
    v[j] = V;
    if (EMA) e[j] = E;
    if (BF) pb[j] = __float2bfloat16_rn(P);
  }
}

bool aligned_to(const void *q, uintptr_t a) { return ((uintptr_t)q & (a - 1)) == 0; }

}  // namespace
}  // namespace evo

using namespace evo;

extern "C" size_t evo_adam_workspace_size(size_t n) { return n ? (size_t)kNormBlocks * sizeof(double) : 0; }

extern "C" int evo_adam_step(const evo_adam *h, size_t n, float *params, const float *grad, float *exp_avg,
                             float *exp_avg_sq, float *ema, void *params_bf16, float *grad_norm, void *workspace,
                             size_t ws_bytes, evo_stream_t stream) {
  if (!h) return EVO_ERR_INVALID_ARG;
  const bool hyper_ok = h->step >= 1 && h->beta1 >= 0.f && h->beta1 < 1.f && h->beta2 >= 0.f && h->beta2 < 1.f &&
                        h->eps > 0.f && std::isfinite(h->lr) && std::isfinite(h->eps) && !std::isnan(h->clip_norm) &&
                        (!ema || (h->ema_decay >= 0.f && h->ema_decay <= 1.f));
  if (!hyper_ok) return EVO_ERR_INVALID_ARG;
  if (n == 0) return EVO_OK;
  if (n > ((size_t)1 << 40)) return EVO_ERR_INVALID_ARG;
  if (!params || !grad || !exp_avg || !exp_avg_sq || !workspace) return EVO_ERR_INVALID_ARG;
  for (const void *q : {(const void *)params, (const void *)grad, (const void *)exp_avg, (const void *)exp_avg_sq,
                        (const void *)workspace})
    if (!aligned_to(q, 256)) return EVO_ERR_ALIGNMENT;
  if ((ema && !aligned_to(ema, 256)) || (params_bf16 && !aligned_to(params_bf16, 256)) ||
      (grad_norm && !aligned_to(grad_norm, 4)))
    return EVO_ERR_ALIGNMENT;
  if (ws_bytes < evo_adam_workspace_size(n)) return EVO_ERR_WORKSPACE;

  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = (int64_t)n;
  const int64_t n4 = N >> 2;
  double *part = (double *)workspace;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n4 + kThreads * kNormU - 1) / (kThreads * kNormU),
                                                             kNormBlocks));
  {
    Prof prof("adam_norm", s, 2.0 * N, 4.0 * N, 1);
    if (launch_k(adam_norm_k, nb, kThreads, 0, s, grad, N, part) != cudaSuccess) return EVO_ERR_CUDA;
  }
  AdamArgs a;
  const double bc1 = 1.0 - std::pow((double)h->beta1, (double)h->step);
  const double bc2 = 1.0 - std::pow((double)h->beta2, (double)h->step);
  a.lr_bc1 = (float)((double)h->lr / bc1);
  a.inv_bc2 = (float)(1.0 / bc2);
  a.b1 = h->beta1;
  a.omb1 = (float)(1.0 - (double)h->beta1);
  a.b2 = h->beta2;
  a.omb2 = (float)(1.0 - (double)h->beta2);
  a.eps = h->eps;
  a.decay = h->ema_decay;
  a.omd = (float)(1.0 - (double)h->ema_decay);
  a.clip = h->clip_norm;
  a.nparts = nb;
  const int ub = (int)std::max<int64_t>(1, std::min<int64_t>((n4 + kThreads * kUpdU - 1) / (kThreads * kUpdU),
                                                             kUpdBlocks));
  bf16 *pb = (bf16 *)params_bf16;
  const double bytes = (double)N * (28.0 + (ema ? 8.0 : 0.0) + (pb ? 2.0 : 0.0));
  Prof prof("adam_update", s, 12.0 * N, bytes, 1);
  cudaError_t r;
  if (ema && pb)
    r = launch_k(adam_update_k<true, true>, ub, kThreads, 0, s, params, grad, exp_avg, exp_avg_sq, ema, pb, N, part,
                 a, grad_norm);
  else if (ema)
    r = launch_k(adam_update_k<true, false>, ub, kThreads, 0, s, params, grad, exp_avg, exp_avg_sq, ema, pb, N, part,
                 a, grad_norm);
  else if (pb)
    r = launch_k(adam_update_k<false, true>, ub, kThreads, 0, s, params, grad, exp_avg, exp_avg_sq, ema, pb, N, part,
                 a, grad_norm);
  else
    r = launch_k(adam_update_k<false, false>, ub, kThreads, 0, s, params, grad, exp_avg, exp_avg_sq, ema, pb, N, part,
                 a, grad_norm);
  return r == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}
