// LayerNorm over the channel axis (AlphaFold2 LayerNorm: biased variance,
// eps 1e-5), FP32 statistics, warp-shuffle reductions: one warp per row.
// The channel-major variants serve the triangle-multiplication output, whose
// per-channel batched product is laid out [c][i][j].
#include <algorithm>

#include "kernels.h"

namespace evo {
namespace {

constexpr float LN_EPS = 1e-5f;

template <typename T, int CPL>
__global__ void __launch_bounds__(256) ln_fwd_rows(const T *x, const float *gamma, const float *beta, T *y,
                                                   int64_t M, int C) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= M) return;
  const T *xr = x + row * C;
  float v[CPL > 0 ? CPL : 1];
  float s = 0.f;
  if (CPL > 0) {
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      v[j] = ldf(xr + lane + 32 * j);
      s += v[j];
    }
    const float mu = warp_sum(s) / C;
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < CPL; ++j) q += (v[j] - mu) * (v[j] - mu);
    const float rstd = rsqrtf(warp_sum(q) / C + LN_EPS);
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int cc = lane + 32 * j;
      stf(y + row * C + cc, (v[j] - mu) * rstd * gamma[cc] + beta[cc]);
    }
  } else {
    for (int cc = lane; cc < C; cc += 32) s += ldf(xr + cc);
    const float mu = warp_sum(s) / C;
    float q = 0.f;
    for (int cc = lane; cc < C; cc += 32) {
      const float d = ldf(xr + cc) - mu;
      q += d * d;
    }
    const float rstd = rsqrtf(warp_sum(q) / C + LN_EPS);
    for (int cc = lane; cc < C; cc += 32) stf(y + row * C + cc, (ldf(xr + cc) - mu) * rstd * gamma[cc] + beta[cc]);
  }
}

// dx = rstd * (gdy - mean(gdy) - xhat * mean(gdy * xhat)), gdy = gamma * dy.
template <typename T>
__global__ void __launch_bounds__(256) ln_bwd_rows(const T *dy, const T *x, const float *gamma, float *dacc, T *dcopy,
                                                   T *dx_out, const T *dinit, int64_t M, int C, int64_t rows_per_blk,
                                                   float *dgamma, float *dbeta) {
  pdl_entry();
  extern __shared__ float sh[];  // [8][2C]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *mine = sh + warp * 2 * C;
  for (int cc = lane; cc < 2 * C; cc += 32) mine[cc] = 0.f;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
  const int64_t r1 = min(M, r0 + rows_per_blk);
  for (int64_t row = r0 + warp; row < r1; row += 8) {
    const T *xr = x + row * C;
    const T *dyr = dy + row * C;
    float s = 0.f;
    for (int cc = lane; cc < C; cc += 32) s += ldf(xr + cc);
    const float mu = warp_sum(s) / C;
    float q = 0.f;
    for (int cc = lane; cc < C; cc += 32) {
      const float d = ldf(xr + cc) - mu;
      q += d * d;
    }
    const float rstd = rsqrtf(warp_sum(q) / C + LN_EPS);
    float a1 = 0.f, a2 = 0.f;
    for (int cc = lane; cc < C; cc += 32) {
      const float xh = (ldf(xr + cc) - mu) * rstd;
      const float g = ldf(dyr + cc);
      const float gd = g * gamma[cc];
      a1 += gd;
      a2 += gd * xh;
      mine[cc] += g * xh;
      mine[C + cc] += g;
    }
    a1 = warp_sum(a1) / C;
    a2 = warp_sum(a2) / C;
    for (int cc = lane; cc < C; cc += 32) {
      const float xh = (ldf(xr + cc) - mu) * rstd;
      const float gd = ldf(dyr + cc) * gamma[cc];
      const float dx = rstd * (gd - a1 - xh * a2);
      if (dacc) {
        const float nv = (dinit ? ldf(dinit + row * C + cc) : dacc[row * C + cc]) + dx;
        dacc[row * C + cc] = nv;
        if (dcopy) stf(dcopy + row * C + cc, nv);
      } else {
        stf(dx_out + row * C + cc, dx);
      }
    }
  }
  __syncthreads();
  for (int cc = threadIdx.x; cc < 2 * C; cc += blockDim.x) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += sh[w * 2 * C + cc];
    atomicAdd(cc < C ? dgamma + cc : dbeta + cc - C, t);
  }
}


template <typename T> struct Pair;
template <> struct Pair<bf16> {
  static __device__ __forceinline__ float2 ld(const bf16 *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
  }
  static __device__ __forceinline__ void st(bf16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
  }
};
template <> struct Pair<float> {
  static __device__ __forceinline__ float2 ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }
  static __device__ __forceinline__ void st(float *p, float a, float b) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
  }
};

// LayerNorm backward with the row in registers: lane l holds channels
// 64j + 2l, 64j + 2l + 1 (j < P), so every load is a coalesced pair.  A warp
// takes NR rows at a time (all their loads issued before any reduction) so
// that the latency of one row overlaps the others.
template <typename T, int P, int NR>
__global__ void __launch_bounds__(256) ln_bwd_rows_vec(const T *dy, const T *x, const float *gamma, float *dacc,
                                                       T *dcopy, T *dx_out, const T *dinit, int64_t M,
                                                       int64_t rows_per_blk, float *dgamma, float *dbeta) {
  pdl_entry();
  constexpr int C = 64 * P;
  __shared__ float red[8][2 * C];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float g0[P], g1[P], ag[P], ag1[P], ab[P], ab1[P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const int c = 64 * j + 2 * lane;
    g0[j] = gamma[c];
    g1[j] = gamma[c + 1];
    ag[j] = ag1[j] = ab[j] = ab1[j] = 0.f;
  }
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
  const int64_t r1 = min(M, r0 + rows_per_blk);
  for (int64_t rb = r0 + (int64_t)warp * NR; rb < r1; rb += 8 * NR) {
    float2 xv[NR][P], gv[NR][P], av[NR][P];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int64_t row = rb + i;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const int c = 64 * j + 2 * lane;
        if (row < r1) {
          xv[i][j] = Pair<T>::ld(x + row * C + c);
          gv[i][j] = Pair<T>::ld(dy + row * C + c);
          av[i][j] = dinit  ? Pair<T>::ld(dinit + row * C + c)
                     : dacc ? *reinterpret_cast<const float2 *>(dacc + row * C + c)
                            : make_float2(0.f, 0.f);
        } else {
          xv[i][j] = gv[i][j] = av[i][j] = make_float2(0.f, 0.f);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int64_t row = rb + i;
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < P; ++j) s += xv[i][j].x + xv[i][j].y;
      const float mu = warp_sum(s) * (1.f / C);
      float q = 0.f;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const float d0 = xv[i][j].x - mu, d1 = xv[i][j].y - mu;
        q += d0 * d0 + d1 * d1;
      }
      const float rstd = rsqrtf(warp_sum(q) * (1.f / C) + LN_EPS);
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const float h0 = (xv[i][j].x - mu) * rstd, h1 = (xv[i][j].y - mu) * rstd;
        xv[i][j].x = h0;
        xv[i][j].y = h1;
        const float d0 = gv[i][j].x * g0[j], d1 = gv[i][j].y * g1[j];
        a1 += d0 + d1;
        a2 += d0 * h0 + d1 * h1;
        ag[j] += gv[i][j].x * h0;
        ag1[j] += gv[i][j].y * h1;
        ab[j] += gv[i][j].x;
        ab1[j] += gv[i][j].y;
      }
      a1 = warp_sum(a1) * (1.f / C);
      a2 = warp_sum(a2) * (1.f / C);
      if (row >= r1) continue;  // warp-uniform
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const int c = 64 * j + 2 * lane;
        const float dx0 = rstd * (gv[i][j].x * g0[j] - a1 - xv[i][j].x * a2);
        const float dx1 = rstd * (gv[i][j].y * g1[j] - a1 - xv[i][j].y * a2);
        if (dacc) {
          const float2 nv = make_float2(av[i][j].x + dx0, av[i][j].y + dx1);
          *reinterpret_cast<float2 *>(dacc + row * C + c) = nv;
          if (dcopy) Pair<T>::st(dcopy + row * C + c, nv.x, nv.y);
        } else {
          Pair<T>::st(dx_out + row * C + c, dx0, dx1);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const int c = 64 * j + 2 * lane;
    red[warp][c] = ag[j];
    red[warp][c + 1] = ag1[j];
    red[warp][C + c] = ab[j];
    red[warp][C + c + 1] = ab1[j];
  }
  __syncthreads();
  for (int cc = threadIdx.x; cc < 2 * C; cc += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][cc];
    atomicAdd(cc < C ? dgamma + cc : dbeta + cc - C, t);
  }
}


template <typename T, int P>
__global__ void __launch_bounds__(256) ln_fwd_rows_vec(const T *x, const float *gamma, const float *beta, T *y,
                                                       int64_t M) {
  pdl_entry();
  constexpr int C = 64 * P;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= M) return;
  float2 v[P];
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < P; ++j) {
    v[j] = Pair<T>::ld(x + row * C + 64 * j + 2 * lane);
    s += v[j].x + v[j].y;
  }
  const float mu = warp_sum(s) * (1.f / C);
  float q = 0.f;
#pragma unroll
  for (int j = 0; j < P; ++j) q += (v[j].x - mu) * (v[j].x - mu) + (v[j].y - mu) * (v[j].y - mu);
  const float rstd = rsqrtf(warp_sum(q) * (1.f / C) + LN_EPS);
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const int c = 64 * j + 2 * lane;
    Pair<T>::st(y + row * C + c, (v[j].x - mu) * rstd * gamma[c] + beta[c],
                (v[j].y - mu) * rstd * gamma[c + 1] + beta[c + 1]);
  }
}

// Eight consecutive channels per thread: one 16-byte access for bf16, two for
// fp32 (rows of C channels start 16-byte aligned).
__device__ __forceinline__ void ld8(const bf16 *p, float (&v)[8]) {
  const uint4 w = *reinterpret_cast<const uint4 *>(p);
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __bfloat1622float2(h[k]);
    v[2 * k] = f.x, v[2 * k + 1] = f.y;
  }
}
__device__ __forceinline__ void ld8(const float *p, float (&v)[8]) {
  const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}
__device__ __forceinline__ void st8(bf16 *p, const float (&v)[8]) {
  uint4 w;
  uint32_t *u = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    u[k] = *reinterpret_cast<const uint32_t *>(&h);
  }
  *reinterpret_cast<uint4 *>(p) = w;
}
__device__ __forceinline__ void st8(float *p, const float (&v)[8]) {
  reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// Row LayerNorm, C in {64, 128, 256}: a row is spread over TPR = C / 8 lanes
// (eight channels each), so a warp covers 32 / TPR rows per step; each warp
// keeps U steps of loads in flight before reducing, enough bytes per SM to
// cover the HBM latency.  Grid-stride over warp-steps.
template <typename T, int C, int U>
__global__ void __launch_bounds__(256) ln_fwd_rows_v8(const T *x, const float *gamma, const float *beta, T *y,
                                                      int64_t M) {
  pdl_entry();
  constexpr int TPR = C / 8, RPW = 32 / TPR;
  const int lane = threadIdx.x & 31;
  const int sub = lane % TPR, rw = lane / TPR;
  const int c0 = sub * 8;
  float g[8], b[8];
  ld8(gamma + c0, g);
  ld8(beta + c0, b);
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int64_t base = w0 * (RPW * U); base < M; base += nwarps * (RPW * U)) {
    float v[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t row = base + u * RPW + rw;
      if (row < M) {
        ld8(x + row * C + c0, v[u]);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[u][k] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) s += v[u][k];
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const float mu = s * (1.f / C);
      float q = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) q += (v[u][k] - mu) * (v[u][k] - mu);
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      const float rstd = rsqrtf(q * (1.f / C) + LN_EPS);
      const int64_t row = base + u * RPW + rw;
      float o8[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) o8[k] = (v[u][k] - mu) * rstd * g[k] + b[k];
      if (row < M) st8(y + row * C + c0, o8);
    }
  }
}

// Row LayerNorm backward, C in {64, 128, 256}, eight channels per lane as in
// ln_fwd_rows_v8 (U warp-steps of loads in flight).  dacc (fp32) becomes
// (dinit or dacc) + dx and dcopy its activation-type copy, or dx_out = dx;
// the gamma / beta partial sums stay in registers (fixed channel slice per
// lane) and leave through one atomic add per channel and block.
__device__ __forceinline__ void ld8f(const float *p, float (&v)[8]) { ld8(p, v); }

template <typename T, int C, int U>
__global__ void __launch_bounds__(256) ln_bwd_rows_v8(const T *dy, const T *x, const float *gamma, float *dacc,
                                                      T *dcopy, T *dx_out, const T *dinit, int64_t M, float *dgamma,
                                                      float *dbeta, float *dsum) {
  pdl_entry();
  constexpr int TPR = C / 8, RPW = 32 / TPR;
  __shared__ float red[8][3 * C];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane % TPR, rw = lane / TPR, c0 = sub * 8;
  float g[8], ag[8], ab[8], as[8];
  ld8f(gamma + c0, g);
#pragma unroll
  for (int k = 0; k < 8; ++k) ag[k] = ab[k] = as[k] = 0.f;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  const int64_t w0 = (int64_t)blockIdx.x * 8 + warp;
  for (int64_t base = w0 * (RPW * U); base < M; base += nwarps * (RPW * U)) {
    float xv[U][8], gv[U][8], av[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t row = base + u * RPW + rw;
      if (row < M) {
        ld8(x + row * C + c0, xv[u]);
        ld8(dy + row * C + c0, gv[u]);
        if (dinit) {
          ld8(dinit + row * C + c0, av[u]);
        } else if (dacc) {
          ld8f(dacc + row * C + c0, av[u]);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) av[u][k] = 0.f;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) xv[u][k] = gv[u][k] = av[u][k] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t row = base + u * RPW + rw;
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) s += xv[u][k];
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const float mu = s * (1.f / C);
      float q = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) q += (xv[u][k] - mu) * (xv[u][k] - mu);
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      const float rstd = rsqrtf(q * (1.f / C) + LN_EPS);
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float xh = (xv[u][k] - mu) * rstd;
        xv[u][k] = xh;
        const float d = gv[u][k] * g[k];
        a1 += d;
        a2 += d * xh;
        ag[k] += gv[u][k] * xh;
        ab[k] += gv[u][k];
      }
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      }
      a1 *= 1.f / C;
      a2 *= 1.f / C;
      if (row >= M) continue;
      float dx[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) dx[k] = rstd * (gv[u][k] * g[k] - a1 - xv[u][k] * a2);
      if (dacc) {
#pragma unroll
        for (int k = 0; k < 8; ++k) dx[k] += av[u][k];
        st8(dacc + row * C + c0, dx);
        if (dcopy) st8(dcopy + row * C + c0, dx);
      } else {
        st8(dx_out + row * C + c0, dx);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) as[k] += dx[k];
    }
  }
  // lanes with the same channel slice: sum over the warp's row groups, then
  // over the block's warps
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int o = TPR; o < 32; o <<= 1) {
      ag[k] += __shfl_xor_sync(0xffffffffu, ag[k], o);
      ab[k] += __shfl_xor_sync(0xffffffffu, ab[k], o);
      as[k] += __shfl_xor_sync(0xffffffffu, as[k], o);
    }
  }
  if (rw == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      red[warp][c0 + k] = ag[k], red[warp][C + c0 + k] = ab[k], red[warp][2 * C + c0 + k] = as[k];
  }
  __syncthreads();
  const int nsum = dsum ? 3 * C : 2 * C;
  for (int cc = threadIdx.x; cc < nsum; cc += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][cc];
    atomicAdd(cc < C ? dgamma + cc : cc < 2 * C ? dbeta + cc - C : dsum + cc - 2 * C, t);
  }
}

// Channel-major LayerNorm of the triangle-multiplication output x[c][i][pitch]
// (pitch a multiple of 8): one block per 32 positions j of a row i.  The
// C x 32 tile comes in with 16-byte loads (8 positions per thread) into a
// padded fp32 tile; the per-position statistics are summed by all eight warps
// over channel slices; the normalised rows are staged [j][C] so that the
// row-major output leaves in 16-byte stores.
template <typename T>
__device__ __forceinline__ void cm_load_tile(const T *x, int64_t pitch, int R, int C, int i, int j0, int nj, float *xt) {
  const int64_t plane = (int64_t)R * pitch;
  for (int idx = threadIdx.x; idx < C * 4; idx += blockDim.x) {
    const int cc = idx >> 2, q = idx & 3;
    const T *src = x + cc * plane + (int64_t)i * pitch + j0 + q * 8;
    float v[8];
    if (q * 8 + 8 <= nj) {
      ld8(src, v);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = q * 8 + k < nj ? ldf(src + k) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) xt[cc * 33 + q * 8 + k] = v[k];
  }
}

// mean and rstd of the 32 positions of an fp32 [C][33] tile into stat[0..31],
// stat[32..63] (part: [8][32] scratch); ends with the block synchronised
__device__ __forceinline__ void cm_stats(const float *xt, int C, float *part, float *stat) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float s = 0.f;
  for (int cc = warp; cc < C; cc += 8) s += xt[cc * 33 + lane];
  part[warp * 32 + lane] = s;
  __syncthreads();
  if (warp == 0) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += part[w * 32 + lane];
    stat[lane] = t / C;
  }
  __syncthreads();
  const float mu = stat[lane];
  float q = 0.f;
  for (int cc = warp; cc < C; cc += 8) {
    const float d = xt[cc * 33 + lane] - mu;
    q += d * d;
  }
  part[warp * 32 + lane] = q;
  __syncthreads();
  if (warp == 0) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += part[w * 32 + lane];
    stat[32 + lane] = rsqrtf(t / C + LN_EPS);
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) ln_fwd_cm_v(const T *x, int64_t pitch, const float *gamma, const float *beta,
                                                   T *y, int R, int C) {
  pdl_entry();
  extern __shared__ __align__(16) float smv[];
  float *xt = smv;              // [C][33]
  float *part = xt + C * 33;    // [8][32]
  float *stat = part + 8 * 32;  // mean [32], rstd [32]
  T *yt = reinterpret_cast<T *>(stat + 64);  // [32][C + 8]
  const int CP = C + 8;
  const int i = blockIdx.y, j0 = blockIdx.x * 32, nj = min(32, R - j0);
  cm_load_tile(x, pitch, R, C, i, j0, nj, xt);
  __syncthreads();
  cm_stats(xt, C, part, stat);
  for (int idx = threadIdx.x; idx < 32 * C; idx += blockDim.x) {
    const int jj = idx / C, cc = idx - jj * C;
    const float v = (xt[cc * 33 + jj] - stat[jj]) * stat[32 + jj] * gamma[cc] + beta[cc];
    if constexpr (sizeof(T) == 2) yt[jj * CP + cc] = __float2bfloat16_rn(v);
    else yt[jj * CP + cc] = v;
  }
  __syncthreads();
  const int cq = C / 8;
  for (int idx = threadIdx.x; idx < nj * cq; idx += blockDim.x) {
    const int jj = idx / cq, q = idx - jj * cq;
    const T *src = yt + jj * CP + q * 8;
    T *dst = y + ((int64_t)i * R + j0 + jj) * C + q * 8;
    if constexpr (sizeof(T) == 2) {
      *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
    } else {
      reinterpret_cast<float4 *>(dst)[0] = reinterpret_cast<const float4 *>(src)[0];
      reinterpret_cast<float4 *>(dst)[1] = reinterpret_cast<const float4 *>(src)[1];
    }
  }
}

// Backward of ln_fwd_cm_v: dy row-major [R*R][C], dx channel-major like x.
// The dy rows are staged [j][C + 2] (odd word stride: conflict-free column
// reads); dx overwrites the x tile in place and leaves in 16-byte stores.
template <typename T>
__global__ void __launch_bounds__(256) ln_bwd_cm_v(const T *dy, const T *x, int64_t pitch, const float *gamma, T *dx,
                                                   int R, int C, float *dgamma, float *dbeta) {
  pdl_entry();
  extern __shared__ __align__(16) float smv[];
  float *xt = smv;              // [C][33]
  float *part = xt + C * 33;    // [8][32]
  float *stat = part + 8 * 32;  // mean, rstd, a1, a2 [4][32]
  float *dyt = stat + 128;      // [32][C + 1] fp32
  const int DP = C + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.y, j0 = blockIdx.x * 32, nj = min(32, R - j0);
  cm_load_tile(x, pitch, R, C, i, j0, nj, xt);
  const int cq = C / 8;
  for (int idx = threadIdx.x; idx < 32 * cq; idx += blockDim.x) {
    const int jj = idx / cq, q = idx - jj * cq;
    float v[8];
    if (jj < nj) {
      ld8(dy + ((int64_t)i * R + j0 + jj) * C + q * 8, v);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) dyt[jj * DP + q * 8 + k] = v[k];
  }
  __syncthreads();
  cm_stats(xt, C, part, stat);
  // a1 = mean_c(dy gamma), a2 = mean_c(dy gamma xhat) per position (lane = j)
  {
    const float mu = stat[lane], rs = stat[32 + lane];
    float a1 = 0.f, a2 = 0.f;
    for (int cc = warp; cc < C; cc += 8) {
      const float gd = dyt[lane * DP + cc] * gamma[cc];
      a1 += gd;
      a2 += gd * (xt[cc * 33 + lane] - mu) * rs;
    }
    part[warp * 32 + lane] = a1;
    __syncthreads();
    if (warp == 0) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += part[w * 32 + lane];
      stat[64 + lane] = t / C;
    }
    __syncthreads();
    part[warp * 32 + lane] = a2;
    __syncthreads();
    if (warp == 0) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += part[w * 32 + lane];
      stat[96 + lane] = t / C;
    }
    __syncthreads();
  }
  // gamma / beta gradients: one thread per channel over the block's positions
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    float sg = 0.f, sb = 0.f;
    for (int jj = 0; jj < nj; ++jj) {
      const float g = dyt[jj * DP + cc];
      sg += g * (xt[cc * 33 + jj] - stat[jj]) * stat[32 + jj];
      sb += g;
    }
    atomicAdd(dgamma + cc, sg);
    atomicAdd(dbeta + cc, sb);
  }
  __syncthreads();  // every read of xt above is done before it is overwritten
  for (int idx = threadIdx.x; idx < 32 * C; idx += blockDim.x) {
    const int cc = idx >> 5, jj = idx & 31;
    const float xh = (xt[cc * 33 + jj] - stat[jj]) * stat[32 + jj];
    xt[cc * 33 + jj] = stat[32 + jj] * (dyt[jj * DP + cc] * gamma[cc] - stat[64 + jj] - xh * stat[96 + jj]);
  }
  __syncthreads();
  const int64_t plane = (int64_t)R * pitch;
  for (int idx = threadIdx.x; idx < C * 4; idx += blockDim.x) {
    const int cc = idx >> 2, q = idx & 3;
    T *dst = dx + cc * plane + (int64_t)i * pitch + j0 + q * 8;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = xt[cc * 33 + q * 8 + k];
    if (q * 8 + 8 <= nj) {
      st8(dst, v);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (q * 8 + k < nj) stf(dst + k, v[k]);
    }
  }
}

// Channel-major input: block = 32 consecutive j of one row i.
template <typename T>
__global__ void __launch_bounds__(256) ln_fwd_cm_k(const T *x, int64_t pitch, const float *gamma, const float *beta,
                                                   T *y, int R, int C) {
  pdl_entry();
  extern __shared__ float tile[];  // [C][33]
  const int i = blockIdx.y, j0 = blockIdx.x * 32;
  const int64_t plane = (int64_t)R * pitch;
  for (int idx = threadIdx.x; idx < C * 32; idx += blockDim.x) {
    const int cc = idx >> 5, jj = idx & 31;
    tile[cc * 33 + jj] = (j0 + jj < R) ? ldf(x + cc * plane + (int64_t)i * pitch + j0 + jj) : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jj = warp; jj < 32; jj += 8) {
    if (j0 + jj >= R) break;
    float s = 0.f;
    for (int cc = lane; cc < C; cc += 32) s += tile[cc * 33 + jj];
    const float mu = warp_sum(s) / C;
    float q = 0.f;
    for (int cc = lane; cc < C; cc += 32) {
      const float d = tile[cc * 33 + jj] - mu;
      q += d * d;
    }
    const float rstd = rsqrtf(warp_sum(q) / C + LN_EPS);
    const int64_t p = (int64_t)i * R + j0 + jj;
    for (int cc = lane; cc < C; cc += 32)
      stf(y + p * C + cc, (tile[cc * 33 + jj] - mu) * rstd * gamma[cc] + beta[cc]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) ln_bwd_cm_k(const T *dy, const T *x, int64_t pitch, const float *gamma, T *dx,
                                                   int R, int C, float *dgamma, float *dbeta) {
  pdl_entry();
  extern __shared__ float sm[];  // xt [C][33], dxt [C][33], acc [8][2C]
  float *xt = sm;
  float *dxt = sm + C * 33;
  float *acc = sm + 2 * C * 33;
  const int i = blockIdx.y, j0 = blockIdx.x * 32;
  const int64_t plane = (int64_t)R * pitch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < C * 32; idx += blockDim.x) {
    const int cc = idx >> 5, jj = idx & 31;
    xt[cc * 33 + jj] = (j0 + jj < R) ? ldf(x + cc * plane + (int64_t)i * pitch + j0 + jj) : 0.f;
  }
  float *mine = acc + warp * 2 * C;
  for (int cc = lane; cc < 2 * C; cc += 32) mine[cc] = 0.f;
  __syncthreads();
  for (int jj = warp; jj < 32; jj += 8) {
    if (j0 + jj >= R) {
      for (int cc = lane; cc < C; cc += 32) dxt[cc * 33 + jj] = 0.f;
      continue;
    }
    float s = 0.f;
    for (int cc = lane; cc < C; cc += 32) s += xt[cc * 33 + jj];
    const float mu = warp_sum(s) / C;
    float q = 0.f;
    for (int cc = lane; cc < C; cc += 32) {
      const float d = xt[cc * 33 + jj] - mu;
      q += d * d;
    }
    const float rstd = rsqrtf(warp_sum(q) / C + LN_EPS);
    const int64_t p = (int64_t)i * R + j0 + jj;
    float a1 = 0.f, a2 = 0.f;
    for (int cc = lane; cc < C; cc += 32) {
      const float xh = (xt[cc * 33 + jj] - mu) * rstd;
      const float g = ldf(dy + p * C + cc);
      const float gd = g * gamma[cc];
      a1 += gd;
      a2 += gd * xh;
      mine[cc] += g * xh;
      mine[C + cc] += g;
    }
    a1 = warp_sum(a1) / C;
    a2 = warp_sum(a2) / C;
    for (int cc = lane; cc < C; cc += 32) {
      const float xh = (xt[cc * 33 + jj] - mu) * rstd;
      const float gd = ldf(dy + p * C + cc) * gamma[cc];
      dxt[cc * 33 + jj] = rstd * (gd - a1 - xh * a2);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < C * 32; idx += blockDim.x) {
    const int cc = idx >> 5, jj = idx & 31;
    if (j0 + jj < R) stf(dx + cc * plane + (int64_t)i * pitch + j0 + jj, dxt[cc * 33 + jj]);
  }
  for (int cc = threadIdx.x; cc < 2 * C; cc += blockDim.x) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += acc[w * 2 * C + cc];
    atomicAdd(cc < C ? dgamma + cc : dbeta + cc - C, t);
  }
}

template <typename T, int C>
void launch_ln_fwd_v8(const T *x, const float *gamma, const float *beta, T *y, int64_t M, cudaStream_t s) {
  constexpr int U = 4, RPW = 32 / (C / 8);
  const int64_t steps = (M + RPW * U - 1) / (RPW * U);  // warp-steps
  const int64_t blocks = std::min<int64_t>((steps + 7) / 8, (int64_t)152 * 4);  // one resident wave
  launch_k(ln_fwd_rows_v8<T, C, U>, (unsigned)std::max<int64_t>(blocks, 1), 256, 0, s, x, gamma, beta, y, M);
}

template <typename T>
cudaError_t ln_fwd_t(const void *x, const float *gamma, const float *beta, void *y, int64_t M, int C, cudaStream_t s) {
  const dim3 grid((unsigned)((M + 7) / 8));
  const T *xx = (const T *)x;
  T *yy = (T *)y;
  auto a16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (a16(x) && a16(y) && a16(gamma) && a16(beta)) {
    switch (C) {
      case 64: launch_ln_fwd_v8<T, 64>(xx, gamma, beta, yy, M, s); return cudaGetLastError();
      case 128: launch_ln_fwd_v8<T, 128>(xx, gamma, beta, yy, M, s); return cudaGetLastError();
      case 256: launch_ln_fwd_v8<T, 256>(xx, gamma, beta, yy, M, s); return cudaGetLastError();
      default: break;
    }
  }
  switch (C) {
    case 64: launch_k(ln_fwd_rows_vec<T, 1>, grid, 256, 0, s, xx, gamma, beta, yy, M); break;
    case 128: launch_k(ln_fwd_rows_vec<T, 2>, grid, 256, 0, s, xx, gamma, beta, yy, M); break;
    case 256: launch_k(ln_fwd_rows_vec<T, 4>, grid, 256, 0, s, xx, gamma, beta, yy, M); break;
    default: launch_k(ln_fwd_rows<T, 0>, grid, 256, 0, s, xx, gamma, beta, yy, M, C); break;
  }
  return cudaGetLastError();
}

}  // namespace

int ln_bwd_blocks(int64_t M) {
  // four blocks per SM (each adds its gamma / beta partial sums with atomics)
  int64_t b = (M + 63) / 64;
  return (int)(b < 608 ? (b < 1 ? 1 : b) : 608);
}

cudaError_t ln_fwd(const void *x, const float *gamma, const float *beta, void *y, int64_t M, int C, int use_bf16,
                   cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  Prof p("ln_fwd", s, 0, (use_bf16 ? 4.0 : 8.0) * M * C);
  return use_bf16 ? ln_fwd_t<bf16>(x, gamma, beta, y, M, C, s) : ln_fwd_t<float>(x, gamma, beta, y, M, C, s);
}

cudaError_t ln_fwd_cm(const void *x, int64_t pitch, const float *gamma, const float *beta, void *y, int R, int C,
                      int use_bf16, cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  Prof p("ln_fwd_cm", s, 0, (use_bf16 ? 4.0 : 8.0) * R * (double)R * C);
  if (use_bf16 && ln_cm_tma_supported(x, pitch, y, R, C)) {
    const cudaError_t e = ln_fwd_cm_tma_launch(x, pitch, gamma, beta, y, R, C, s);
    if (e != cudaErrorNotSupported) return e;
  }
  dim3 grid((R + 31) / 32, R);
  auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
  if (pitch % 8 == 0 && C % 8 == 0 && a16(x) && a16(y)) {
    const size_t smv = (size_t)(C * 33 + 8 * 32 + 64) * 4 + (size_t)32 * (C + 8) * (use_bf16 ? 2 : 4);
    if (smv > 48 * 1024) {
      cudaError_t e = use_bf16 ? cudaFuncSetAttribute(ln_fwd_cm_v<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv)
                               : cudaFuncSetAttribute(ln_fwd_cm_v<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv);
      if (e != cudaSuccess) return e;
    }
    if (use_bf16)
      launch_k(ln_fwd_cm_v<bf16>, grid, 256, smv, s, (const bf16 *)x, pitch, gamma, beta, (bf16 *)y, R, C);
    else
      launch_k(ln_fwd_cm_v<float>, grid, 256, smv, s, (const float *)x, pitch, gamma, beta, (float *)y, R, C);
    return cudaGetLastError();
  }
  const size_t sm = (size_t)C * 33 * sizeof(float);
  if (use_bf16)
    launch_k(ln_fwd_cm_k<bf16>, grid, 256, sm, s, (const bf16 *)x, pitch, gamma, beta, (bf16 *)y, R, C);
  else
    launch_k(ln_fwd_cm_k<float>, grid, 256, sm, s, (const float *)x, pitch, gamma, beta, (float *)y, R, C);
  return cudaGetLastError();
}

// LayerNorm backward without the fused column sums (any C; the vectorised
// kernels for C = 64 P).
cudaError_t ln_bwd_rows_any(const void *dy, const void *x, const float *gamma, float *dacc, void *dcopy,
                            void *dx_out, int64_t M, int C, int use_bf16, cudaStream_t s, float *dgamma, float *dbeta,
                            const void *dinit) {
  const int nb = ln_bwd_blocks(M);
  const int64_t rpb = (M + nb - 1) / nb;
#define EVO_LN_BWD_VEC(P, NR)                                                                                    \
  if (C == 64 * P) {                                                                                             \
    if (use_bf16)                                                                                                \
      launch_k(ln_bwd_rows_vec<bf16, P, NR>, nb, 256, 0, s, (const bf16 *)dy, (const bf16 *)x, gamma, dacc,           \
                                                      (bf16 *)dcopy, (bf16 *)dx_out, (const bf16 *)dinit, M, rpb, dgamma, dbeta);     \
    else                                                                                                         \
      launch_k(ln_bwd_rows_vec<float, P, NR>, nb, 256, 0, s, (const float *)dy, (const float *)x, gamma, dacc,        \
                                                       (float *)dcopy, (float *)dx_out, (const float *)dinit, M, rpb, dgamma, dbeta);  \
    return cudaGetLastError();                                                                                   \
  }
  EVO_LN_BWD_VEC(1, 4)
  EVO_LN_BWD_VEC(2, 4)
  EVO_LN_BWD_VEC(4, 2)
#undef EVO_LN_BWD_VEC
  const size_t sm = (size_t)8 * 2 * C * sizeof(float);
  if (use_bf16)
    launch_k(ln_bwd_rows<bf16>, nb, 256, sm, s, (const bf16 *)dy, (const bf16 *)x, gamma, dacc, (bf16 *)dcopy,
                                          (bf16 *)dx_out, (const bf16 *)dinit, M, C, rpb, dgamma, dbeta);
  else
    launch_k(ln_bwd_rows<float>, nb, 256, sm, s, (const float *)dy, (const float *)x, gamma, dacc, (float *)dcopy,
                                           (float *)dx_out, (const float *)dinit, M, C, rpb, dgamma, dbeta);
  return cudaGetLastError();
}

cudaError_t ln_bwd(const void *dy, const void *x, const float *gamma, float *dacc, void *dcopy, void *dx_out,
                   int64_t M, int C, int use_bf16, cudaStream_t s, float *dgamma, float *dbeta, const void *dinit,
                   float *dsum) {
  if (M <= 0) return cudaSuccess;
  Prof p("ln_bwd", s, 0, (use_bf16 ? 2.0 : 4.0) * M * C * (dcopy ? 3 : 2) + (dacc ? 8.0 * M * C : 0.0));
  {
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    const bool al = a16(dy) && a16(x) && a16(gamma) && (!dacc || a16(dacc)) && (!dcopy || a16(dcopy)) &&
                    (!dx_out || a16(dx_out)) && (!dinit || a16(dinit));
    if (al && (C == 64 || C == 128 || C == 256)) {
      constexpr int U = 2;
      const int64_t rpw = 32 / (C / 8);
      const int64_t steps = (M + rpw * U - 1) / (rpw * U);
      const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((steps + 7) / 8, 152 * 2));
#define EVO_LN_BWD_V8(CC)                                                                                        \
  if (C == CC) {                                                                                                 \
    if (use_bf16)                                                                                                \
      launch_k(ln_bwd_rows_v8<bf16, CC, U>, blocks, 256, 0, s, (const bf16 *)dy, (const bf16 *)x, gamma, dacc,   \
               (bf16 *)dcopy, (bf16 *)dx_out, (const bf16 *)dinit, M, dgamma, dbeta, dsum);                    \
    else                                                                                                         \
      launch_k(ln_bwd_rows_v8<float, CC, U>, blocks, 256, 0, s, (const float *)dy, (const float *)x, gamma, dacc, \
               (float *)dcopy, (float *)dx_out, (const float *)dinit, M, dgamma, dbeta, dsum);                 \
    return cudaGetLastError();                                                                                   \
  }
      EVO_LN_BWD_V8(64)
      EVO_LN_BWD_V8(128)
      EVO_LN_BWD_V8(256)
#undef EVO_LN_BWD_V8
    }
  }
  cudaError_t e = ln_bwd_rows_any(dy, x, gamma, dacc, dcopy, dx_out, M, C, use_bf16, s, dgamma, dbeta, dinit);
  if (e == cudaSuccess && dsum) {
    e = dacc ? colsum(dacc, C, M, C, 0, s, dsum) : colsum(dx_out, C, M, C, use_bf16, s, dsum);
  }
  return e;
}

cudaError_t ln_bwd_cm(const void *dy, const void *x, int64_t pitch, const float *gamma, void *dx, int R,
                      int C, int use_bf16, cudaStream_t s, float *dgamma, float *dbeta) {
  if (R <= 0) return cudaSuccess;
  Prof p("ln_bwd_cm", s, 0, (use_bf16 ? 6.0 : 12.0) * R * (double)R * C);
  if (use_bf16 && ln_cm_tma_supported(x, pitch, dx, R, C) && (((uintptr_t)dy) & 15u) == 0) {
    const cudaError_t e = ln_bwd_cm_tma_launch(dy, x, pitch, gamma, dx, R, C, dgamma, dbeta, s);
    if (e != cudaErrorNotSupported) return e;
  }
  dim3 grid((R + 31) / 32, R);
  auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
  if (pitch % 8 == 0 && C % 8 == 0 && a16(x) && a16(dy) && a16(dx)) {
    const size_t smv = (size_t)(C * 33 + 8 * 32 + 128 + 32 * (C + 1)) * 4;
    if (smv > 48 * 1024) {
      cudaError_t e = use_bf16 ? cudaFuncSetAttribute(ln_bwd_cm_v<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv)
                               : cudaFuncSetAttribute(ln_bwd_cm_v<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv);
      if (e != cudaSuccess) return e;
    }
    if (use_bf16)
      launch_k(ln_bwd_cm_v<bf16>, grid, 256, smv, s, (const bf16 *)dy, (const bf16 *)x, pitch, gamma, (bf16 *)dx, R, C,
               dgamma, dbeta);
    else
      launch_k(ln_bwd_cm_v<float>, grid, 256, smv, s, (const float *)dy, (const float *)x, pitch, gamma, (float *)dx, R,
               C, dgamma, dbeta);
    return cudaGetLastError();
  }
  const size_t sm = ((size_t)2 * C * 33 + (size_t)8 * 2 * C) * sizeof(float);
  if (sm > 48 * 1024) {
    cudaError_t e = use_bf16 ? cudaFuncSetAttribute(ln_bwd_cm_k<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                         : cudaFuncSetAttribute(ln_bwd_cm_k<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (use_bf16)
    launch_k(ln_bwd_cm_k<bf16>, grid, 256, sm, s, (const bf16 *)dy, (const bf16 *)x, pitch, gamma, (bf16 *)dx, R, C,
                                            dgamma, dbeta);
  else
    launch_k(ln_bwd_cm_k<float>, grid, 256, sm, s, (const float *)dy, (const float *)x, pitch, gamma, (float *)dx, R,
                                             C, dgamma, dbeta);
  return cudaGetLastError();
}

}  // namespace evo
