// Bandwidth-bound helpers of the Evoformer block: pair-bias projection,
// triangle-multiplication gating (with the [c][i][k] relayout the per-channel
// product needs), gate backwards, outer-product-mean normaliser, column sums
// and partial reductions, dtype conversions.
#include <algorithm>

#include "kernels.h"

namespace evo {
namespace {

// q = i / d, r = i % d with 32-bit division when i fits.
__device__ __forceinline__ void divmod(int64_t i, int d, int64_t &q, int &r) {
  if (i < (1ll << 31)) {
    const int ii = (int)i, qq = ii / d;
    q = qq;
    r = ii - qq * d;
  } else {
    q = i / d;
    r = (int)(i - q * d);
  }
}

__device__ __forceinline__ void ld8(const bf16 *p, float (&v)[8]) {
  const uint4 w = *reinterpret_cast<const uint4 *>(p);
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __bfloat1622float2(h[k]);
    v[2 * k] = f.x;
    v[2 * k + 1] = f.y;
  }
}
__device__ __forceinline__ void st8(bf16 *p, const float (&v)[8]) {
  uint4 w;
  __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&w);
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
  *reinterpret_cast<uint4 *>(p) = w;
}

// ------------------------------------------------------------- reductions
// 32 columns per block; the 8 warps split the partial rows, then combine.
__global__ void __launch_bounds__(256) reduce_partials_k(const float *part, int nblk, int64_t ld, int N, float *out) {
  pdl_entry();
  __shared__ float s[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = blockIdx.x * 32 + lane;
  float t = 0.f;
  if (n < N)
    for (int b = w; b < nblk; b += 8) t += part[(int64_t)b * ld + n];
  s[w][lane] = t;
  __syncthreads();
  if (w == 0 && n < N) {
    float tot = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) tot += s[k][lane];
    out[n] += tot;
  }
}

// Column sums: block (64 columns, a range of rows); each lane owns two
// adjacent columns, the 8 warps split the rows, then combine.
template <typename T>
__global__ void __launch_bounds__(256) colsum_k(const T *x, int64_t ld, int64_t M, int N,
                                                int64_t rows_per_blk, float *out) {
  pdl_entry();
  __shared__ float s[8][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = blockIdx.x * 64 + 2 * lane;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_blk;
  const int64_t r1 = min(M, r0 + rows_per_blk);
  float t0 = 0.f, t1 = 0.f;
  for (int64_t r = r0 + w; r < r1; r += 8) {
    if (n < N) t0 += ldf(x + r * ld + n);
    if (n + 1 < N) t1 += ldf(x + r * ld + n + 1);
  }
  s[w][2 * lane] = t0;
  s[w][2 * lane + 1] = t1;
  __syncthreads();
  if (threadIdx.x < 64) {
    const int nn = blockIdx.x * 64 + threadIdx.x;
    float tot = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) tot += s[k][threadIdx.x];
    if (nn < N) atomicAdd(out + nn, tot);
  }
}

// bf16 column sums with 16-byte loads: a thread owns 8 adjacent columns of
// every (256 / (N / 8))-th row of the block's row range; the rows meet in
// shared memory and the block adds its N sums with atomics.  N % 8 == 0,
// N <= 2048, 16-byte aligned rows.
__global__ void __launch_bounds__(256) colsum_v8_k(const bf16 *x, int64_t ld, int64_t M, int N, int64_t rows_per_blk,
                                                   float *out) {
  pdl_entry();
  extern __shared__ float part[];  // [256 / tpr][N]
  const int tpr = N / 8;           // threads per row
  const int rpi = blockDim.x / tpr;  // rows per iteration
  const int t = threadIdx.x;
  const int r_in = t / tpr, c8 = (t % tpr) * 8;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk, r1 = min(M, r0 + rows_per_blk);
  if (r_in < rpi) {
    // four rows of loads in flight per thread
    int64_t r = r0 + r_in;
    for (; r + 3 * rpi < r1; r += 4 * rpi) {
      float v[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) ld8(x + (r + u * rpi) * ld + c8, v[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += v[u][k];
    }
    for (; r < r1; r += rpi) {
      float v[8];
      ld8(x + r * ld + c8, v);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += v[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) part[r_in * N + c8 + k] = acc[k];
  }
  __syncthreads();
  for (int c = t; c < N; c += blockDim.x) {
    float sum = 0.f;
    for (int i = 0; i < rpi; ++i) sum += part[i * N + c];
    atomicAdd(out + c, sum);
  }
}

__global__ void reduce_splits_k(const float *part, int splits, int64_t n, float *out) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float t = 0.f;
  for (int s = 0; s < splits; ++s) t += part[(int64_t)s * n + i];
  out[i] += t;
}

// out(m, n) = sum_s part[(s*M + m)*N + n] in bf16 at offset map(m, n); a
// thread owns two adjacent columns (N even).
__global__ void reduce_splits_map_k(const float *part, int splits, int M, int N, OutMap map, bf16 *out) {
  pdl_entry();
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (i >= (int64_t)M * N) return;
  const int m = (int)(i / N), n = (int)(i - (int64_t)m * N);
  float t0 = 0.f, t1 = 0.f;
  for (int s = 0; s < splits; ++s) {
    const float2 v = *reinterpret_cast<const float2 *>(part + (int64_t)s * M * N + i);
    t0 += v.x;
    t1 += v.y;
  }
  const int64_t o0 = map.row(m) + map.col(n), o1 = map.row(m) + map.col(n + 1);
  if (o1 == o0 + 1 && (o0 & 1) == 0) {
    *reinterpret_cast<__nv_bfloat162 *>(out + o0) = __floats2bfloat162_rn(t0, t1);
  } else {
    out[o0] = __float2bfloat16_rn(t0);
    out[o1] = __float2bfloat16_rn(t1);
  }
}

// ------------------------------------------------------------- pair bias
template <typename T, typename OT>
__global__ void head_proj_fwd_k(const T *x, const float *w, OT *out, int R, int C, int H, int transpose) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t P = (int64_t)R * R;
  if (p >= P) return;
  float acc[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) acc[h] = 0.f;
  for (int cc = lane; cc < C; cc += 32) {
    const float xv = ldf(x + p * C + cc);
#pragma unroll
    for (int h = 0; h < 8; ++h)
      if (h < H) acc[h] = fmaf(xv, w[h * C + cc], acc[h]);
  }
  int64_t i;
  int j;
  divmod(p, R, i, j);
  const int64_t pp = transpose ? (int64_t)j * R + i : p;
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    if (h >= H) break;
    const float v = warp_sum(acc[h]);
    if (lane == 0) stf(out + h * P + pp, v);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) head_proj_bwd_k(const float *dbias, const T *x, const float *w, T *dx,
                                                       int accumulate, int R, int C, int H, int transpose,
                                                       int64_t pos_per_blk, float *dw) {
  pdl_entry();
  extern __shared__ float acc[];  // [8 warps][H*C]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *mine = acc + warp * H * C;
  for (int k = lane; k < H * C; k += 32) mine[k] = 0.f;
  const int64_t P = (int64_t)R * R;
  const int64_t p0 = (int64_t)blockIdx.x * pos_per_blk;
  const int64_t p1 = min(P, p0 + pos_per_blk);
  for (int64_t p = p0 + warp; p < p1; p += 8) {
    int64_t i;
    int j;
    divmod(p, R, i, j);
    const int64_t pp = transpose ? (int64_t)j * R + i : p;
    float g[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) g[h] = h < H ? dbias[h * P + pp] : 0.f;
    for (int cc = lane; cc < C; cc += 32) {
      float d = 0.f;
      const float xv = ldf(x + p * C + cc);
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        if (h < H) {
          d = fmaf(g[h], w[h * C + cc], d);
          mine[h * C + cc] += g[h] * xv;
        }
      }
      T *dp = dx + p * C + cc;
      stf(dp, accumulate ? ldf(dp) + d : d);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < H * C; k += blockDim.x) {
    float t = 0.f;
    for (int ww = 0; ww < 8; ++ww) t += acc[ww * H * C + k];
    atomicAdd(dw + k, t);
  }
}


// CPL consecutive bf16 channels per lane as floats (CPL = 4 or 8).
template <int CPL>
__device__ __forceinline__ void ldc(const bf16 *p, float (&v)[CPL]) {
  if constexpr (CPL == 8) {
    ld8(p, v);
  } else {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.y));
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
}
template <int CPL>
__device__ __forceinline__ void stc(bf16 *p, const float (&v)[CPL]) {
  if constexpr (CPL == 8) {
    st8(p, v);
  } else {
    uint2 w;
    *reinterpret_cast<__nv_bfloat162 *>(&w.x) = __floats2bfloat162_rn(v[0], v[1]);
    *reinterpret_cast<__nv_bfloat162 *>(&w.y) = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2 *>(p) = w;
  }
}

// Sum of H per-lane values over the TPR lanes of a position group (aligned
// groups of TPR lanes), by halving exchanges: at the step with offset o the
// lane with bit o set keeps the upper half of its remaining heads and sends
// the lower half.  Lane l ends with the full sum of head head_of_lane(l).
template <int H, int TPR>
__device__ __forceinline__ float head_reduce(float (&a)[H], int lane) {
  int n = H;
#pragma unroll
  for (int o = TPR / 2; o >= 1; o >>= 1) {
    if (n > 1) {
      const int half = n / 2;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < H / 2; ++i) {
        if (i < half) {
          const float send = up ? a[i] : a[i + half];
          const float keep = up ? a[i + half] : a[i];
          a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      n = half;
    } else {
      a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
    }
  }
  return a[0];
}
// the head whose sum lane l holds after head_reduce, and whether l is the
// lowest lane holding it
template <int H, int TPR>
__device__ __forceinline__ int head_of_lane(int lane, bool &writer) {
  int h = 0, n = H, low = 0;
#pragma unroll
  for (int o = TPR / 2; o >= 1; o >>= 1) {
    if (n > 1) {
      n /= 2;
      if (lane & o) h += n;
    } else {
      low |= lane & o;
    }
  }
  writer = low == 0;
  return h;
}

// Pair-bias projection, BF16: a position's C channels are spread over
// TPR = C / CPL lanes with CPL channels each, so the lane's slice of w stays
// in registers; U warp-steps of loads are in flight before the products are
// reduced over the group (head_reduce).  Grid-stride over warp-steps in the
// order of the output index q; with transpose the input position is the
// transposed one (i, j) -> (j, i), whose C channels are one contiguous row,
// so both the reads and the bf16 writes stay coalesced.
template <int H, int C, int CPL, int U>
__global__ void __launch_bounds__(256, H == 4 ? 3 : 2) head_proj_fwd_w(const bf16 *x, const float *w, bf16 *out, int R,
                                                       int transpose, int64_t P, int64_t hstride) {
  pdl_entry();
  constexpr int TPR = C / CPL, PPW = 32 / TPR;
  const int lane = threadIdx.x & 31;
  const int sub = lane % TPR, pw = lane / TPR;
  float wl[H][CPL];
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int k = 0; k < CPL; ++k) wl[h][k] = w[h * C + sub * CPL + k];
  bool writer;
  const int hsel = head_of_lane<H, TPR>(lane, writer);
  // P positions from x (all R * R, or the rows of an i-slab), head h at out + h * hstride
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int64_t base = w0 * (PPW * U); base < P; base += nwarps * (PPW * U)) {
    float v[U][CPL];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = base + u * PPW + pw;
      if (q < P) {
        int64_t p = q;
        if (transpose) {
          int64_t i;
          int j;
          divmod(q, R, i, j);
          p = (int64_t)j * R + i;
        }
        ldc<CPL>(x + p * C + sub * CPL, v[u]);
      } else {
#pragma unroll
        for (int k = 0; k < CPL; ++k) v[u][k] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float acc[H];
#pragma unroll
      for (int h = 0; h < H; ++h) {
        acc[h] = 0.f;
#pragma unroll
        for (int k = 0; k < CPL; ++k) acc[h] = fmaf(v[u][k], wl[h][k], acc[h]);
      }
      const float r = head_reduce<H, TPR>(acc, lane);
      const int64_t q = base + u * PPW + pw;
      if (writer && q < P) out[hsel * hstride + q] = __float2bfloat16_rn(r);
    }
  }
}

// Backward: dx (+)= sum_h dbias[h][pos'] w[h] over the lane's CPL channels,
// and the lane's slice of dw accumulates in registers (one atomic add per
// element and block at the end).  Positions are taken in the order of the
// dbias index q (the input position is the transposed one with transpose),
// so the dbias loads are coalesced.
template <int H, int C, int CPL, int U>
__global__ void __launch_bounds__(256, 2) head_proj_bwd_w(const float *dbias, const bf16 *x, const float *w, bf16 *dx,
                                                       int accumulate, int R, int transpose, float *dw) {
  pdl_entry();
  constexpr int TPR = C / CPL, PPW = 32 / TPR;
  __shared__ float red[8][H * C];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane % TPR, pw = lane / TPR;
  float wl[H][CPL], aw[H][CPL];
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int k = 0; k < CPL; ++k) wl[h][k] = w[h * C + sub * CPL + k], aw[h][k] = 0.f;
  const int64_t P = (int64_t)R * R;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  const int64_t w0 = (int64_t)blockIdx.x * 8 + warp;
  for (int64_t base = w0 * (PPW * U); base < P; base += nwarps * (PPW * U)) {
    float v[U][CPL], d[U][CPL], g[U][H];
    int64_t pos[U];  // input / dx position of step u (-1 past the end)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = base + u * PPW + pw;
      pos[u] = -1;
      if (q < P) {
        int64_t p = q;
        if (transpose) {
          int64_t i;
          int j;
          divmod(q, R, i, j);
          p = (int64_t)j * R + i;
        }
        pos[u] = p;
#pragma unroll
        for (int h = 0; h < H; ++h) g[u][h] = dbias[h * P + q];
        ldc<CPL>(x + p * C + sub * CPL, v[u]);
        if (accumulate) {
          ldc<CPL>(dx + p * C + sub * CPL, d[u]);
        } else {
#pragma unroll
          for (int k = 0; k < CPL; ++k) d[u][k] = 0.f;
        }
      } else {
#pragma unroll
        for (int h = 0; h < H; ++h) g[u][h] = 0.f;
#pragma unroll
        for (int k = 0; k < CPL; ++k) v[u][k] = d[u][k] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int h = 0; h < H; ++h)
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
          d[u][k] = fmaf(g[u][h], wl[h][k], d[u][k]);
          aw[h][k] = fmaf(g[u][h], v[u][k], aw[h][k]);
        }
      if (pos[u] >= 0) stc<CPL>(dx + pos[u] * C + sub * CPL, d[u]);
    }
  }
  // dw: lanes of the same sub hold the same channels; sum over the warp's
  // position groups, then over the block's warps
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      float t = aw[h][k];
#pragma unroll
      for (int o = TPR; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (pw == 0) red[warp][h * C + sub * CPL + k] = t;
    }
  __syncthreads();
  for (int k = threadIdx.x; k < H * C; k += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) t += red[ww][k];
    atomicAdd(dw + k, t);
  }
}

// Pair-bias projection, BF16 fast path: one thread per position, the
// position's C channels read as 16-byte vectors, w staged in shared memory.
template <int H, typename OT>
__global__ void __launch_bounds__(128) head_proj_fwd_v8(const bf16 *x, const float *w, OT *out, int R, int C,
                                                        int transpose) {
  pdl_entry();
  extern __shared__ float ws[];  // [H][C]
  for (int k = threadIdx.x; k < H * C; k += blockDim.x) ws[k] = w[k];
  __syncthreads();
  const int64_t P = (int64_t)R * R;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float acc[H];
#pragma unroll
  for (int h = 0; h < H; ++h) acc[h] = 0.f;
  const bf16 *row = x + p * C;
  for (int c0 = 0; c0 < C; c0 += 8) {
    float v[8];
    ld8(row + c0, v);
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[h] = fmaf(v[k], ws[h * C + c0 + k], acc[h]);
  }
  int64_t i;
  int j;
  divmod(p, R, i, j);
  const int64_t pp = transpose ? (int64_t)j * R + i : p;
#pragma unroll
  for (int h = 0; h < H; ++h) stf(out + h * P + pp, acc[h]);
}

// Backward, BF16 fast path: warp per position, lane owns channel pairs
// 64j + 2*lane (+1); the weight gradient accumulates in registers.
template <int H, int PJ>
__global__ void __launch_bounds__(256) head_proj_bwd_v8(const float *dbias, const bf16 *x, const float *w, bf16 *dx,
                                                        int accumulate, int R, int transpose,
                                                        int64_t pos_per_blk, float *dw) {
  pdl_entry();
  constexpr int C = 64 * PJ;
  __shared__ float red[8][H * C];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[H][2 * PJ];
  float wl[H][2 * PJ];
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int j = 0; j < PJ; ++j) {
      acc[h][2 * j] = acc[h][2 * j + 1] = 0.f;
      wl[h][2 * j] = w[h * C + 64 * j + 2 * lane];
      wl[h][2 * j + 1] = w[h * C + 64 * j + 2 * lane + 1];
    }
  const int64_t P = (int64_t)R * R;
  const int64_t p0 = (int64_t)blockIdx.x * pos_per_blk;
  const int64_t p1 = min(P, p0 + pos_per_blk);
  for (int64_t p = p0 + warp; p < p1; p += 8) {
    int64_t i;
    int jj;
    divmod(p, R, i, jj);
    const int64_t pp = transpose ? (int64_t)jj * R + i : p;
    float g[H];
#pragma unroll
    for (int h = 0; h < H; ++h) g[h] = dbias[h * P + pp];
#pragma unroll
    for (int j = 0; j < PJ; ++j) {
      const int c = 64 * j + 2 * lane;
      const float2 xv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(x + p * C + c));
      float d0 = 0.f, d1 = 0.f;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        d0 = fmaf(g[h], wl[h][2 * j], d0);
        d1 = fmaf(g[h], wl[h][2 * j + 1], d1);
        acc[h][2 * j] = fmaf(g[h], xv.x, acc[h][2 * j]);
        acc[h][2 * j + 1] = fmaf(g[h], xv.y, acc[h][2 * j + 1]);
      }
      __nv_bfloat162 *dp = reinterpret_cast<__nv_bfloat162 *>(dx + p * C + c);
      if (accumulate) {
        const float2 old = __bfloat1622float2(*dp);
        d0 += old.x;
        d1 += old.y;
      }
      *dp = __floats2bfloat162_rn(d0, d1);
    }
  }
#pragma unroll
  for (int h = 0; h < H; ++h)
#pragma unroll
    for (int j = 0; j < PJ; ++j) {
      red[warp][h * C + 64 * j + 2 * lane] = acc[h][2 * j];
      red[warp][h * C + 64 * j + 2 * lane + 1] = acc[h][2 * j + 1];
    }
  __syncthreads();
  for (int k = threadIdx.x; k < H * C; k += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) t += red[ww][k];
    atomicAdd(dw + k, t);
  }
}

// ---------------------------------------------------- triangle multiplication
// Tile of 32 (orow) x 32 (ocol) positions, 4 channels. Outgoing: position
// (p0,p1) = (orow, ocol); incoming: (p0,p1) = (ocol, orow). Channel-major
// element (c, orow, ocol) sits at c*R*pitch + orow*pitch + ocol.
template <typename T>
__global__ void __launch_bounds__(256) trimul_gate_fwd_k(const T *abg, int64_t ld, const float *mask, T *A, T *B,
                                                         int64_t pitch, int R, int cm, int incoming) {
  pdl_entry();
  __shared__ float as[4][32][33], bs[4][32][33];
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c0 = blockIdx.z * 4;
  for (int idx = threadIdx.x; idx < 32 * 32 * 4; idx += blockDim.x) {
    const int cc = idx & 3, ocl = (idx >> 2) & 31, orl = idx >> 7;
    const int orow = r0 + orl, ocol = q0 + ocl, c = c0 + cc;
    float av = 0.f, bv = 0.f;
    if (orow < R && ocol < R && c < cm) {
      const int64_t p = incoming ? (int64_t)ocol * R + orow : (int64_t)orow * R + ocol;
      const T *row = abg + p * ld;
      const float mk = mask[p];
      const float ap = ldf(row + c), ag = ldf(row + cm + c), bp = ldf(row + 2 * cm + c), bg = ldf(row + 3 * cm + c);
      av = mk * sigmoidf_(ag) * ap;
      bv = mk * sigmoidf_(bg) * bp;
    }
    as[cc][orl][ocl] = av;
    bs[cc][orl][ocl] = bv;
  }
  __syncthreads();
  const int64_t plane = (int64_t)R * pitch;
  for (int idx = threadIdx.x; idx < 32 * 32 * 4; idx += blockDim.x) {
    const int ocl = idx & 31, orl = (idx >> 5) & 31, cc = idx >> 10;
    const int orow = r0 + orl, ocol = q0 + ocl, c = c0 + cc;
    if (orow < R && ocol < R && c < cm) {
      const int64_t o = (int64_t)c * plane + (int64_t)orow * pitch + ocol;
      stf(A + o, as[cc][orl][ocl]);
      stf(B + o, bs[cc][orl][ocl]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) trimul_gate_bwd_k(const T *dA, const T *dB, int64_t pitch, const T *abg,
                                                         int64_t ld, const float *mask, T *dabg, int R, int cm,
                                                         int incoming) {
  pdl_entry();
  __shared__ float as[4][32][33], bs[4][32][33];
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c0 = blockIdx.z * 4;
  const int64_t plane = (int64_t)R * pitch;
  for (int idx = threadIdx.x; idx < 32 * 32 * 4; idx += blockDim.x) {
    const int ocl = idx & 31, orl = (idx >> 5) & 31, cc = idx >> 10;
    const int orow = r0 + orl, ocol = q0 + ocl, c = c0 + cc;
    float av = 0.f, bv = 0.f;
    if (orow < R && ocol < R && c < cm) {
      const int64_t o = (int64_t)c * plane + (int64_t)orow * pitch + ocol;
      av = ldf(dA + o);
      bv = ldf(dB + o);
    }
    as[cc][orl][ocl] = av;
    bs[cc][orl][ocl] = bv;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * 32 * 4; idx += blockDim.x) {
    const int cc = idx & 3, ocl = (idx >> 2) & 31, orl = idx >> 7;
    const int orow = r0 + orl, ocol = q0 + ocl, c = c0 + cc;
    if (orow < R && ocol < R && c < cm) {
      const int64_t p = incoming ? (int64_t)ocol * R + orow : (int64_t)orow * R + ocol;
      const T *row = abg + p * ld;
      T *drow = dabg + p * ld;
      const float mk = mask[p];
      const float ap = ldf(row + c), ag = ldf(row + cm + c), bp = ldf(row + 2 * cm + c), bg = ldf(row + 3 * cm + c);
      const float sa = sigmoidf_(ag), sb = sigmoidf_(bg);
      const float da = as[cc][orl][ocl] * mk, db = bs[cc][orl][ocl] * mk;
      stf(drow + c, da * sa);
      stf(drow + cm + c, da * ap * sa * (1.f - sa));
      stf(drow + 2 * cm + c, db * sb);
      stf(drow + 3 * cm + c, db * bp * sb * (1.f - sb));
    }
  }
}


// BF16 fast path of the gating relayout: a block owns 32 x 32 positions and
// 8 channels; each position's 8 channels of a_proj, a_gate, b_proj, b_gate
// arrive as four 16-byte loads; the sigmoid of the g columns is folded in
// (block z handles g columns z*8.., z*8 + 8).
__global__ void __launch_bounds__(256) trimul_gate_fwd_v8(const bf16 *abg, int64_t ld, const float *mask, bf16 *A,
                                                          bf16 *B, int64_t pitch, int R, int cm, int incoming) {
  pdl_entry();
  __shared__ bf16 as[8][32][34], bs[8][32][34];
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c0 = blockIdx.z * 8;
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int ocl = idx & 31, orl = idx >> 5;
    const int orow = r0 + orl, ocol = q0 + ocl;
    float av[8] = {}, bv[8] = {};
    if (orow < R && ocol < R) {
      const int64_t p = incoming ? (int64_t)ocol * R + orow : (int64_t)orow * R + ocol;
      const bf16 *row = abg + p * ld;
      const float mk = mask[p];
      float ap[8], ag[8], bp[8], bg[8];
      ld8(row + c0, ap);
      ld8(row + cm + c0, ag);
      ld8(row + 2 * cm + c0, bp);
      ld8(row + 3 * cm + c0, bg);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        av[k] = mk * __fdividef(ap[k], 1.f + __expf(-ag[k]));
        bv[k] = mk * __fdividef(bp[k], 1.f + __expf(-bg[k]));
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      as[k][orl][ocl] = __float2bfloat16_rn(av[k]);
      bs[k][orl][ocl] = __float2bfloat16_rn(bv[k]);
    }
  }
  __syncthreads();
  const int64_t plane = (int64_t)R * pitch;
  for (int idx = threadIdx.x; idx < 8 * 32 * 16; idx += blockDim.x) {  // pairs of columns
    const int oc2 = (idx & 15) * 2, orl = (idx >> 4) & 31, k = idx >> 9;
    const int orow = r0 + orl, ocol = q0 + oc2, c = c0 + k;
    if (orow >= R || c >= cm) continue;
    const int64_t o = (int64_t)c * plane + (int64_t)orow * pitch + ocol;
    if (ocol + 1 < R && (o & 1) == 0) {
      __nv_bfloat162 a2, b2;
      a2.x = as[k][orl][oc2], a2.y = as[k][orl][oc2 + 1];
      b2.x = bs[k][orl][oc2], b2.y = bs[k][orl][oc2 + 1];
      *reinterpret_cast<__nv_bfloat162 *>(A + o) = a2;
      *reinterpret_cast<__nv_bfloat162 *>(B + o) = b2;
    } else {
      if (ocol < R) {
        A[o] = as[k][orl][oc2];
        B[o] = bs[k][orl][oc2];
      }
      if (ocol + 1 < R) {
        A[o + 1] = as[k][orl][oc2 + 1];
        B[o + 1] = bs[k][orl][oc2 + 1];
      }
    }
  }
}

__global__ void __launch_bounds__(256) trimul_gate_bwd_v8(const bf16 *dA, const bf16 *dB, int64_t pitch,
                                                          const bf16 *abg, int64_t ld, const float *mask, bf16 *dabg,
                                                          int R, int cm, int incoming) {
  pdl_entry();
  __shared__ bf16 as[8][32][34], bs[8][32][34];
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c0 = blockIdx.z * 8;
  const int64_t plane = (int64_t)R * pitch;
  for (int idx = threadIdx.x; idx < 8 * 32 * 32; idx += blockDim.x) {
    const int ocl = idx & 31, orl = (idx >> 5) & 31, k = idx >> 10;
    const int orow = r0 + orl, ocol = q0 + ocl, c = c0 + k;
    bf16 av = __float2bfloat16_rn(0.f), bv = av;
    if (orow < R && ocol < R && c < cm) {
      const int64_t o = (int64_t)c * plane + (int64_t)orow * pitch + ocol;
      av = dA[o];
      bv = dB[o];
    }
    as[k][orl][ocl] = av;
    bs[k][orl][ocl] = bv;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
    const int ocl = idx & 31, orl = idx >> 5;
    const int orow = r0 + orl, ocol = q0 + ocl;
    if (orow >= R || ocol >= R) continue;
    const int64_t p = incoming ? (int64_t)ocol * R + orow : (int64_t)orow * R + ocol;
    const bf16 *row = abg + p * ld;
    bf16 *drow = dabg + p * ld;
    const float mk = mask[p];
    float ap[8], ag[8], bp[8], bg[8], dap[8], dag[8], dbp[8], dbg[8];
    ld8(row + c0, ap);
    ld8(row + cm + c0, ag);
    ld8(row + 2 * cm + c0, bp);
    ld8(row + 3 * cm + c0, bg);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float sa = __fdividef(1.f, 1.f + __expf(-ag[k])), sb = __fdividef(1.f, 1.f + __expf(-bg[k]));
      const float da = __bfloat162float(as[k][orl][ocl]) * mk, db = __bfloat162float(bs[k][orl][ocl]) * mk;
      dap[k] = da * sa;
      dag[k] = da * ap[k] * sa * (1.f - sa);
      dbp[k] = db * sb;
      dbg[k] = db * bp[k] * sb * (1.f - sb);
    }
    st8(drow + c0, dap);
    st8(drow + cm + c0, dag);
    st8(drow + 2 * cm + c0, dbp);
    st8(drow + 3 * cm + c0, dbg);
  }
}

// Triangle-multiplication gates, tiled for bf16 with cm a multiple of 64:
// block = 2 rows x 64 columns of the (row, col) output grid and 64 of the cm
// channels (blockIdx.z).  A warp reads one position's 64-channel segments of
// ap | ag | bp | bg (4 x 128 B: lanes 0-7, 8-15, 16-23, 24-31), exchanges the
// gate halves by shuffles, and the channel-major A, B rows leave as 128-byte
// rows through a shared-memory transposition ([row][col][channel] with an odd
// channel pitch, so both the channel-wise and the column-wise accesses are
// free of bank conflicts).  Position of (row, col): row * R + col (outgoing)
// or col * R + row (incoming).
constexpr int TG_ROWS = 2, TG_COLS = 64, TG_CH = 64, TG_LDC = TG_CH + 1, TG_U = 4;

__device__ __forceinline__ float sigm(float x) { return __fdividef(1.f, 1.f + __expf(-x)); }

__global__ void __launch_bounds__(256) trimul_gate_fwd_t(const bf16 *abg, int64_t ld, const float *mask, bf16 *A,
                                                         bf16 *B, int64_t pitch, int R, int cm, int incoming) {
  pdl_entry();
  __shared__ bf16 as[TG_ROWS][TG_COLS][TG_LDC];
  __shared__ bf16 bs[TG_ROWS][TG_COLS][TG_LDC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q0 = blockIdx.x * TG_COLS, r0 = blockIdx.y * TG_ROWS, c0 = blockIdx.z * TG_CH;
  const int seg = lane >> 3, sub = lane & 7;  // segment (ap, ag, bp, bg) and its 8-channel piece
  // a warp takes positions warp + 8u + 32k; the loads of TG_U positions are
  // issued before any of them is used
  for (int pb = warp; pb < TG_ROWS * TG_COLS; pb += 8 * TG_U) {
    float v[TG_U][8], mk[TG_U];
#pragma unroll
    for (int u = 0; u < TG_U; ++u) {
      const int pi = pb + 8 * u;
      const int orow = r0 + pi / TG_COLS, ocol = q0 + pi % TG_COLS;
      mk[u] = 0.f;
      if (orow < R && ocol < R) {
        const int64_t p = incoming ? (int64_t)ocol * R + orow : (int64_t)orow * R + ocol;
        mk[u] = mask[p];
        ld8(abg + p * ld + seg * cm + c0 + sub * 8, v[u]);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[u][k] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < TG_U; ++u) {
      const int pi = pb + 8 * u;
      const int orl = pi / TG_COLS, ocl = pi % TG_COLS;
      // lanes 0-7 (ap) take ag from lanes 8-15; lanes 16-23 (bp) take bg from 24-31
      float gv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) gv[k] = __shfl_down_sync(0xffffffffu, v[u][k], 8);
      if ((seg & 1) == 0) {
        bf16 *dst = seg == 0 ? &as[orl][ocl][sub * 8] : &bs[orl][ocl][sub * 8];
#pragma unroll
        for (int k = 0; k < 8; ++k) dst[k] = __float2bfloat16_rn(mk[u] * v[u][k] * sigm(gv[k]));
      }
    }
  }
  __syncthreads();
  // channel-major rows: A[c][orow][q0 ..] (64 bf16 = 128 B per warp instruction)
  const int64_t plane = (int64_t)R * pitch;
  for (int t = warp; t < 2 * TG_CH * TG_ROWS; t += 8) {
    const int which = t / (TG_CH * TG_ROWS), rem = t % (TG_CH * TG_ROWS);
    const int ch = rem / TG_ROWS, orl = rem % TG_ROWS;
    const int c = c0 + ch, orow = r0 + orl, ocol = q0 + 2 * lane;
    if (c >= cm || orow >= R || ocol >= R) continue;
    const bf16 (*src)[TG_COLS][TG_LDC] = which ? bs : as;
    const bf16 v0 = src[orl][2 * lane][ch], v1 = src[orl][2 * lane + 1][ch];
    bf16 *dst = (which ? B : A) + (int64_t)c * plane + (int64_t)orow * pitch + ocol;
    if (ocol + 1 < R && ((((uintptr_t)dst) & 3u) == 0)) {
      __nv_bfloat162 w;
      w.x = v0, w.y = v1;
      *reinterpret_cast<__nv_bfloat162 *>(dst) = w;
    } else {
      dst[0] = v0;
      if (ocol + 1 < R) dst[1] = v1;
    }
  }
}

__global__ void __launch_bounds__(256) trimul_gate_bwd_t(const bf16 *dA, const bf16 *dB, int64_t pitch,
                                                         const bf16 *abg, int64_t ld, const float *mask, bf16 *dabg,
                                                         int R, int cm, int incoming) {
  pdl_entry();
  __shared__ bf16 as[TG_ROWS][TG_COLS][TG_LDC];
  __shared__ bf16 bs[TG_ROWS][TG_COLS][TG_LDC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q0 = blockIdx.x * TG_COLS, r0 = blockIdx.y * TG_ROWS, c0 = blockIdx.z * TG_CH;
  const int64_t plane = (int64_t)R * pitch;
  // channel-major gradient rows in (128 B per warp instruction), eight rows
  // of a warp in flight together
  constexpr int NROW = 2 * TG_CH * TG_ROWS, RU = 8;
  for (int tb = warp; tb < NROW; tb += 8 * RU) {
    __nv_bfloat162 w[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int t = tb + 8 * u;
      const int which = t / (TG_CH * TG_ROWS), rem = t % (TG_CH * TG_ROWS);
      const int ch = rem / TG_ROWS, orl = rem % TG_ROWS;
      const int c = c0 + ch, orow = r0 + orl, ocol = q0 + 2 * lane;
      w[u].x = w[u].y = __float2bfloat16_rn(0.f);
      if (c < cm && orow < R && ocol < R) {
        const bf16 *src = (which ? dB : dA) + (int64_t)c * plane + (int64_t)orow * pitch + ocol;
        if (ocol + 1 < R && ((((uintptr_t)src) & 3u) == 0)) {
          w[u] = *reinterpret_cast<const __nv_bfloat162 *>(src);
        } else {
          w[u].x = src[0];
          if (ocol + 1 < R) w[u].y = src[1];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int t = tb + 8 * u;
      const int which = t / (TG_CH * TG_ROWS), rem = t % (TG_CH * TG_ROWS);
      const int ch = rem / TG_ROWS, orl = rem % TG_ROWS;
      bf16 (*dst)[TG_COLS][TG_LDC] = which ? bs : as;
      dst[orl][2 * lane][ch] = w[u].x;
      dst[orl][2 * lane + 1][ch] = w[u].y;
    }
  }
  __syncthreads();
  const int seg = lane >> 3, sub = lane & 7;
  for (int pb = warp; pb < TG_ROWS * TG_COLS; pb += 8 * TG_U) {
    float v[TG_U][8], mk[TG_U];
    int64_t pp[TG_U];
#pragma unroll
    for (int u = 0; u < TG_U; ++u) {
      const int pi = pb + 8 * u;
      const int orow = r0 + pi / TG_COLS, ocol = q0 + pi % TG_COLS;
      mk[u] = 0.f;
      pp[u] = -1;
      if (orow < R && ocol < R) {
        pp[u] = incoming ? (int64_t)ocol * R + orow : (int64_t)orow * R + ocol;
        mk[u] = mask[pp[u]];
        ld8(abg + pp[u] * ld + seg * cm + c0 + sub * 8, v[u]);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[u][k] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < TG_U; ++u) {
      const int pi = pb + 8 * u;
      const int orl = pi / TG_COLS, ocl = pi % TG_COLS;
      float gv[8], pv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        gv[k] = __shfl_down_sync(0xffffffffu, v[u][k], 8);  // the gate pre-activation, for lanes of ap / bp
        pv[k] = __shfl_up_sync(0xffffffffu, v[u][k], 8);    // the projection, for lanes of ag / bg
      }
      if (pp[u] < 0) continue;  // warp-uniform
      const bf16 *src = seg < 2 ? &as[orl][ocl][sub * 8] : &bs[orl][ocl][sub * 8];
      float out[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float d = __bfloat162float(src[k]) * mk[u];
        if ((seg & 1) == 0) {
          out[k] = d * sigm(gv[k]);  // d proj = d * sigmoid(gate)
        } else {
          const float sg = sigm(v[u][k]);
          out[k] = d * pv[k] * sg * (1.f - sg);  // d gate = d * proj * sigmoid'(gate)
        }
      }
      st8(dabg + pp[u] * ld + seg * cm + c0 + sub * 8, out);
    }
  }
}

template <typename T>
__global__ void gate_out_bwd_k(const T *dz, const T *g, int64_t g_ld, const T *y, T *dy, T *dgpre, int64_t dg_ld,
                               int64_t P, int C) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * C) return;
  int64_t p;
  int c;
  divmod(i, C, p, c);
  const float d = ldf(dz + i), gv = ldf(g + p * g_ld + c), yv = ldf(y + i);
  stf(dy + i, d * gv);
  stf(dgpre + p * dg_ld + c, d * yv * gv * (1.f - gv));
}

// bf16, C = 8k: eight channels per thread with 16-byte accesses, two groups
// of loads in flight per thread
// Column sums of a grid-stride pass whose thread keeps one 8-channel chunk
// (the stride is a multiple of C / 8): lanes of a warp holding the same chunk
// are combined by shuffles, the warps of a block in shared memory, then one
// atomic add per channel and block.  red: [8][C] floats (C <= 256).
__device__ __forceinline__ void chunk_colsum_flush(float (&cs)[8], int C, float *red, float *dsum) {
  const int cq = C / 8, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = cq; o < 32; o <<= 1)
#pragma unroll
    for (int k = 0; k < 8; ++k) cs[k] += __shfl_xor_sync(0xffffffffu, cs[k], o);
  if (lane < cq) {
#pragma unroll
    for (int k = 0; k < 8; ++k) red[warp * C + lane * 8 + k] = cs[k];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w * C + c];
    atomicAdd(dsum + c, t);
  }
}

__device__ __forceinline__ void unpack8(const uint4 &w, float (&v)[8]) {
  const uint32_t q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) v[2 * k] = __uint_as_float(q[k] << 16), v[2 * k + 1] = __uint_as_float(q[k] & 0xffff0000u);
}

// Grid-stride kernels over (position, 8-channel chunk) items with C / 8
// chunks per position: the grid stride is a multiple of C / 8 (which divides
// 256), so a thread keeps its eight channels c .. c + 7 (the ones whose
// column sums it accumulates) and steps over positions.
struct ChunkWalk {
  int64_t p0, pstep;
  int c;
  __device__ __forceinline__ explicit ChunkWalk(int C) {
    const int cq = C / 8;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    c = (int)(i0 % cq) * 8;
    p0 = i0 / cq;
    pstep = (int64_t)gridDim.x * blockDim.x / cq;
  }
};

// Output-gate backward: dy = dz g, dgpre = dz y g (1 - g), four positions'
// 16-byte loads in flight per thread (kept packed).
__global__ void __launch_bounds__(256) gate_out_bwd_v8(const bf16 *dz, const bf16 *g, int64_t g_ld, const bf16 *y,
                                                       bf16 *dy, bf16 *dgpre, int64_t dg_ld, int64_t P, int C,
                                                       float *dsum) {
  pdl_entry();
  constexpr int U = 4;
  __shared__ float red[8 * 256];
  float cs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const ChunkWalk w(C);
  const int c = w.c;
  for (int64_t p0 = w.p0; p0 < P; p0 += U * w.pstep) {
    uint4 dr[U], gr[U], yr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = p0 + u * w.pstep;
      if (p < P) {
        dr[u] = *reinterpret_cast<const uint4 *>(dz + p * C + c);
        gr[u] = *reinterpret_cast<const uint4 *>(g + p * g_ld + c);
        yr[u] = *reinterpret_cast<const uint4 *>(y + p * C + c);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = p0 + u * w.pstep;
      if (p < P) {
        float d[8], gv[8], yv[8], a[8], b[8];
        unpack8(dr[u], d);
        unpack8(gr[u], gv);
        unpack8(yr[u], yv);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          a[k] = d[k] * gv[k];
          b[k] = d[k] * yv[k] * gv[k] * (1.f - gv[k]);
        }
        st8(dy + p * C + c, a);
        st8(dgpre + p * dg_ld + c, b);
#pragma unroll
        for (int k = 0; k < 8; ++k) cs[k] += a[k];
      }
    }
  }
  if (dsum) chunk_colsum_flush(cs, C, red, dsum);
}

// ------------------------------------------------------------------ dropout
// out[p, c] = (res ? res[p, c] : 0) + upd[p, c] * scale[q(p), c], q(p) = p % R
// (row-wise: one draw per column, shared by every row) or p / R (column-wise).
template <typename T>
__global__ void dropout_apply_k(const T *upd, const float *scale, const T *res, T *out, int64_t P, int C, int R,
                                int colwise) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * C) return;
  int64_t p;
  int c;
  divmod(i, C, p, c);
  const int64_t q = colwise ? p / R : p % R;
  const float v = ldf(upd + i) * scale[q * C + c];
  stf(out + i, res ? ldf(res + i) + v : v);
}

__global__ void __launch_bounds__(256) dropout_apply_v8(const bf16 *upd, const float *scale, const bf16 *res,
                                                        bf16 *out, int64_t P, int C, int R, int colwise) {
  pdl_entry();
  const int cq = C / 8;
  const int64_t n = P * cq;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t p = e / cq;
    const int c = (int)(e - p * cq) * 8;
    const int64_t q = colwise ? p / R : p % R;
    float u[8], r[8];
    ld8(upd + p * C + c, u);
    const float4 s0 = reinterpret_cast<const float4 *>(scale + q * C + c)[0];
    const float4 s1 = reinterpret_cast<const float4 *>(scale + q * C + c)[1];
    const float sc[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    if (res) {
      ld8(res + p * C + c, r);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) r[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] += u[k] * sc[k];
    st8(out + p * C + c, r);
  }
}

// ------------------------------------------------------------ attention gate
template <typename T>
__global__ void attn_gate_bwd_k(AttnArgs a, const T *dog, T *dgpre, int64_t sGb_d, int64_t sGx_d, T *do_att,
                                float *D) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= (int64_t)a.B1 * a.X) return;
  int64_t b;
  int x;
  divmod(row, a.X, b, x);
  const int64_t ob = b * a.sOb + x * a.sOx;
  const int64_t gb = b * a.sQb + x * a.sQx;
  const int64_t db = b * sGb_d + x * sGx_d;
  for (int h = 0; h < a.H; ++h) {
    float s = 0.f;
    for (int d = lane; d < a.c; d += 32) {
      const int64_t k = h * a.c + d;
      const float dg = ldf(dog + ob + k), gv = ldf((const T *)a.g + gb + k), ov = ldf((const T *)a.o_att + ob + k);
      const float doa = dg * gv;
      stf(do_att + ob + k, doa);
      stf(dgpre + db + k, dg * ov * gv * (1.f - gv));
      s += doa * ov;
    }
    s = warp_sum(s);
    if (lane == 0) D[(b * a.H + h) * a.X + x] = s;
  }
}

template <typename T>
__global__ void attn_dq_store_k(AttnArgs a, T *dq) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int hc = a.H * a.c;
  if (i >= (int64_t)a.B1 * a.X * hc) return;
  int64_t row, b;
  int k, x;
  divmod(i, hc, row, k);
  divmod(row, a.X, b, x);
  stf(dq + b * a.sQb + x * a.sQx + k, a.scale * a.dq_acc[b * a.sOb + x * a.sOx + k]);
}

// ------------------------------------------------------------ OPM, scaling
// inv[i*R + j] = 1 / (eps + sum_s mask[s,i] mask[s,j]): a 32 x 32 tile of
// (i, j) per block, the mask columns of the tile staged in shared memory 64
// rows s at a time, 2 x 2 outputs per thread.
__global__ void __launch_bounds__(256) opm_inv_norm_k(const float *mask, float *inv, int S, int R, float eps) {
  pdl_entry();
  __shared__ float mi[64][32], mj[64][32];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // outputs (i0 + 2ty + a, j0 + 2tx + b)
  float n00 = 0.f, n01 = 0.f, n10 = 0.f, n11 = 0.f;
  for (int s0 = 0; s0 < S; s0 += 64) {
    for (int idx = threadIdx.x; idx < 64 * 32; idx += blockDim.x) {
      const int ss = idx >> 5, c = idx & 31, srow = s0 + ss;
      mi[ss][c] = srow < S && i0 + c < R ? mask[(int64_t)srow * R + i0 + c] : 0.f;
      mj[ss][c] = srow < S && j0 + c < R ? mask[(int64_t)srow * R + j0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int ss = 0; ss < 64; ++ss) {
      const float a0 = mi[ss][2 * ty], a1 = mi[ss][2 * ty + 1];
      const float b0 = mj[ss][2 * tx], b1 = mj[ss][2 * tx + 1];
      n00 = fmaf(a0, b0, n00), n01 = fmaf(a0, b1, n01);
      n10 = fmaf(a1, b0, n10), n11 = fmaf(a1, b1, n11);
    }
    __syncthreads();
  }
  const int i = i0 + 2 * ty, j = j0 + 2 * tx;
  if (i < R && j < R) inv[(int64_t)i * R + j] = 1.f / (eps + n00);
  if (i < R && j + 1 < R) inv[(int64_t)i * R + j + 1] = 1.f / (eps + n01);
  if (i + 1 < R && j < R) inv[(int64_t)(i + 1) * R + j] = 1.f / (eps + n10);
  if (i + 1 < R && j + 1 < R) inv[(int64_t)(i + 1) * R + j + 1] = 1.f / (eps + n11);
}

// bf16 rows of C = 8k channels, 16 bytes per access, two in flight per thread
__global__ void __launch_bounds__(256) row_scale_v8(const bf16 *x, const float *scale, bf16 *y, int64_t M, int C,
                                                    float *dsum) {
  pdl_entry();
  constexpr int U = 4;
  __shared__ float red[8 * 256];
  float cs[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const ChunkWalk w(C);
  const int c = w.c;
  for (int64_t r0 = w.p0; r0 < M; r0 += U * w.pstep) {
    uint4 xr[U];
    float sc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = r0 + u * w.pstep;
      if (r < M) xr[u] = *reinterpret_cast<const uint4 *>(x + r * C + c), sc[u] = scale[r];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = r0 + u * w.pstep;
      if (r < M) {
        float v[8];
        unpack8(xr[u], v);
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] *= sc[u], cs[k] += v[k];
        st8(y + r * C + c, v);
      }
    }
  }
  if (dsum) chunk_colsum_flush(cs, C, red, dsum);
}

template <typename T>
__global__ void row_scale_k(const T *x, const float *scale, T *y, int64_t M, int C) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * C) return;
  int64_t r;
  int c;
  divmod(i, C, r, c);
  stf(y + i, ldf(x + i) * scale[r]);
}

template <typename T>
__global__ void to_f32_k(const T *src, float *dst, int64_t n) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = ldf(src + i);
}
template <typename T>
__global__ void from_f32_k(const float *src, T *dst, int64_t n) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) stf(dst + i, src[i]);
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t reduce_partials(const float *part, int nb, int N, float *out, cudaStream_t s) {
  Prof prof("reduce_partials", s, 0, 4.0 * nb * (double)N, 1);
  launch_k(reduce_partials_k, (N + 31) / 32, 256, 0, s, part, nb, N, N, out);
  return cudaGetLastError();
}
// Variant with a leading dimension (LayerNorm partials hold gamma and beta sums).
cudaError_t reduce_partials_ld(const float *part, int nb, int64_t ld, int N, float *out, cudaStream_t s) {
  Prof prof("reduce_partials", s, 0, 4.0 * nb * (double)N, 1);
  launch_k(reduce_partials_k, (N + 31) / 32, 256, 0, s, part, nb, ld, N, out);
  return cudaGetLastError();
}

int colsum_blocks(int64_t M) {
  int64_t b = (M + 255) / 256;
  return (int)(b < 296 ? (b < 1 ? 1 : b) : 296);
}
cudaError_t colsum(const void *x, int64_t ld, int64_t M, int N, int use_bf16, cudaStream_t s, float *out) {
  Prof prof("colsum", s, 0, (use_bf16 ? 2.0 : 4.0) * M * (double)N, 1);
  if (M <= 0) return cudaSuccess;
  if (use_bf16 && N % 8 == 0 && N <= 2048 && ld % 8 == 0 && (((uintptr_t)x) & 15u) == 0) {
    // about four blocks per SM, each over a contiguous row range
    const int64_t nbv = std::min<int64_t>(608, (M + 63) / 64);
    const int64_t rpb = (M + nbv - 1) / nbv;
    const size_t sm = (size_t)(256 / (N / 8)) * N * sizeof(float);
    return launch_k(colsum_v8_k, (unsigned)nbv, 256, sm, s, (const bf16 *)x, ld, M, N, rpb, out);
  }
  const int nb = colsum_blocks(M);
  const int64_t rpb = (M + nb - 1) / nb;
  const dim3 grid((N + 63) / 64, nb);
  if (use_bf16) launch_k(colsum_k<bf16>, grid, 256, 0, s, (const bf16 *)x, ld, M, N, rpb, out);
  else launch_k(colsum_k<float>, grid, 256, 0, s, (const float *)x, ld, M, N, rpb, out);
  return cudaGetLastError();
}

cudaError_t reduce_splits(const float *part, int splits, int64_t n, float *out, cudaStream_t s) {
  Prof prof("reduce_splits", s, 0, 4.0 * (splits + 2) * (double)n, 1);
  launch_k(reduce_splits_k, nblk(n), 256, 0, s, part, splits, n, out);
  return cudaGetLastError();
}

cudaError_t reduce_splits_map(const float *part, int splits, int M, int N, const OutMap &map, void *out,
                              cudaStream_t s) {
  if (N % 2) return cudaErrorInvalidValue;
  Prof prof("reduce_splits", s, 0, (4.0 * splits + 2.0) * (double)M * N, 1);
  const int64_t pairs = (int64_t)M * N / 2;
  launch_k(reduce_splits_map_k, nblk(pairs), 256, 0, s, part, splits, M, N, map, (bf16 *)out);
  return cudaGetLastError();
}

// Grid of a grid-stride kernel of 256-thread blocks (no dynamic shared
// memory): the blocks that fit on all SMs at once, at most `want`; a grid
// of one whole wave leaves no SM with a partial second round.
template <typename K>
unsigned one_wave(K kern, int64_t want) {
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * sms));
}

cudaError_t head_proj_fwd(const void *x, const float *w, void *out, int R, int C, int H, int transpose, int use_bf16,
                          cudaStream_t s) {
  Prof prof("head_proj_fwd", s, 2.0 * R * (double)R * C * H, (use_bf16 ? 2.0 : 4.0) * R * (double)R * C + 4.0 * H * R * (double)R, 1);
  if (H > 8) return cudaErrorInvalidValue;
  const int64_t P = (int64_t)R * R;
  if (use_bf16 && C == 128 && (((uintptr_t)x) & 15u) == 0 && (H == 4 || H == 8)) {
    constexpr int U = 4;
    const int64_t steps = (P + 2 * U - 1) / (2 * U);  // warp-steps (two positions each)
    if (H == 4)
      launch_k(head_proj_fwd_w<4, 128, 8, U>, one_wave(head_proj_fwd_w<4, 128, 8, U>, (steps + 7) / 8), 256, 0, s,
               (const bf16 *)x, w, (bf16 *)out, R, transpose, P, P);
    else
      launch_k(head_proj_fwd_w<8, 128, 8, U>, one_wave(head_proj_fwd_w<8, 128, 8, U>, (steps + 7) / 8), 256, 0, s,
               (const bf16 *)x, w, (bf16 *)out, R, transpose, P, P);
  } else if (use_bf16 && C % 8 == 0 && (((uintptr_t)x) & 15u) == 0 && (H == 4 || H == 8)) {
    const size_t sm = (size_t)H * C * sizeof(float);
    if (H == 4) launch_k(head_proj_fwd_v8<4, bf16>, nblk(P, 128), 128, sm, s, (const bf16 *)x, w, (bf16 *)out, R, C, transpose);
    else launch_k(head_proj_fwd_v8<8, bf16>, nblk(P, 128), 128, sm, s, (const bf16 *)x, w, (bf16 *)out, R, C, transpose);
  } else if (use_bf16) {
    launch_k(head_proj_fwd_k<bf16, bf16>, nblk(P, 8), 256, 0, s, (const bf16 *)x, w, (bf16 *)out, R, C, H, transpose);
  } else {
    launch_k(head_proj_fwd_k<float, float>, nblk(P, 8), 256, 0, s, (const float *)x, w, (float *)out, R, C, H,
             transpose);
  }
  return cudaGetLastError();
}

cudaError_t head_proj_fwd_rows(const void *x, const float *w, void *out, int64_t npos, int64_t hstride, int C, int H,
                               cudaStream_t s) {
  Prof prof("head_proj_fwd", s, 2.0 * npos * C * H, 2.0 * npos * C + 2.0 * H * npos, 1);
  if (C != 128 || (H != 4 && H != 8) || (((uintptr_t)x) & 15u)) return cudaErrorNotSupported;
  if (npos <= 0) return cudaSuccess;
  constexpr int U = 4;
  const int64_t steps = (npos + 2 * U - 1) / (2 * U);
  if (H == 4)
    launch_k(head_proj_fwd_w<4, 128, 8, U>, one_wave(head_proj_fwd_w<4, 128, 8, U>, (steps + 7) / 8), 256, 0, s,
             (const bf16 *)x, w, (bf16 *)out, 1, 0, npos, hstride);
  else
    launch_k(head_proj_fwd_w<8, 128, 8, U>, one_wave(head_proj_fwd_w<8, 128, 8, U>, (steps + 7) / 8), 256, 0, s,
             (const bf16 *)x, w, (bf16 *)out, 1, 0, npos, hstride);
  return cudaGetLastError();
}

int head_proj_blocks(int R) {
  int64_t b = ((int64_t)R * R + 63) / 64;
  return (int)(b < 296 ? (b < 1 ? 1 : b) : 296);
}
cudaError_t head_proj_bwd(const float *dbias, const void *x, const float *w, void *dx, int accumulate, int R, int C, int H, int transpose, int use_bf16, cudaStream_t s, float *dw) {
  Prof prof("head_proj_bwd", s, 4.0 * R * (double)R * C * H, (use_bf16 ? 2.0 : 4.0) * R * (double)R * C * (accumulate ? 3 : 2) + 4.0 * H * R * (double)R, 1);
  if (H > 8) return cudaErrorInvalidValue;
  const int nb = head_proj_blocks(R);
  const int64_t ppb = ((int64_t)R * R + nb - 1) / nb;
  const size_t sm = (size_t)8 * H * C * sizeof(float);
  if (sm > 48 * 1024) return cudaErrorInvalidValue;
  if (use_bf16 && C == 128 && (H == 4 || H == 8) && (((uintptr_t)x) & 15u) == 0 && (((uintptr_t)dx) & 15u) == 0) {
    // H = 4: eight channels per lane (16 positions' worth of w and dw in
    // registers); H = 8: four channels per lane
    constexpr int U = 2;
    const int64_t P = (int64_t)R * R;
    const int64_t ppw = H == 4 ? 2 : 1;
    const int64_t steps = (P + ppw * U - 1) / (ppw * U);
    if (H == 4)
      launch_k(head_proj_bwd_w<4, 128, 8, U>, one_wave(head_proj_bwd_w<4, 128, 8, U>, (steps + 7) / 8), 256, 0, s,
               dbias, (const bf16 *)x, w, (bf16 *)dx, accumulate, R, transpose, dw);
    else
      launch_k(head_proj_bwd_w<8, 128, 4, U>, one_wave(head_proj_bwd_w<8, 128, 4, U>, (steps + 7) / 8), 256, 0, s,
               dbias, (const bf16 *)x, w, (bf16 *)dx, accumulate, R, transpose, dw);
  } else if (use_bf16 && C == 128 && (H == 4 || H == 8) && (((uintptr_t)x) & 3u) == 0 && (((uintptr_t)dx) & 3u) == 0) {
    if (H == 4)
      launch_k(head_proj_bwd_v8<4, 2>, nb, 256, 0, s, dbias, (const bf16 *)x, w, (bf16 *)dx, accumulate, R, transpose,
                                                ppb, dw);
    else
      launch_k(head_proj_bwd_v8<8, 2>, nb, 256, 0, s, dbias, (const bf16 *)x, w, (bf16 *)dx, accumulate, R, transpose,
                                                ppb, dw);
  } else if (use_bf16)
    launch_k(head_proj_bwd_k<bf16>, nb, 256, sm, s, dbias, (const bf16 *)x, w, (bf16 *)dx, accumulate, R, C, H,
                                              transpose, ppb, dw);
  else
    launch_k(head_proj_bwd_k<float>, nb, 256, sm, s, dbias, (const float *)x, w, (float *)dx, accumulate, R, C, H,
                                               transpose, ppb, dw);
  return cudaGetLastError();
}

cudaError_t trimul_gate_fwd(const void *abg, int64_t ld, const float *mask, void *A, void *B, int64_t pitch, int R,
                            int cm, int incoming, int use_bf16, cudaStream_t s) {
  Prof prof("trimul_gate_fwd", s, 0, (use_bf16 ? 2.0 : 4.0) * R * (double)R * 6.0 * cm, 1);
  if (use_bf16 && trimul_gate_tma_supported(abg, ld, A, B, pitch, R, cm)) {
    const cudaError_t e = trimul_gate_fwd_tma_launch(abg, ld, mask, A, B, pitch, R, cm, incoming, s);
    if (e != cudaErrorNotSupported) return e;
  }
  dim3 grid((R + 31) / 32, (R + 31) / 32, (cm + 3) / 4);
  const bool v8 = cm % 8 == 0 && ld % 8 == 0 && (((uintptr_t)abg) & 15u) == 0;
  if (use_bf16 && v8 && cm % TG_CH == 0) {
    dim3 gt((R + TG_COLS - 1) / TG_COLS, (R + TG_ROWS - 1) / TG_ROWS, cm / TG_CH);
    launch_k(trimul_gate_fwd_t, gt, 256, 0, s, (const bf16 *)abg, ld, mask, (bf16 *)A, (bf16 *)B, pitch, R, cm,
             incoming);
  } else if (use_bf16 && v8) {
    dim3 g8((R + 31) / 32, (R + 31) / 32, cm / 8);
    launch_k(trimul_gate_fwd_v8, g8, 256, 0, s, (const bf16 *)abg, ld, mask, (bf16 *)A, (bf16 *)B, pitch, R, cm,
             incoming);
  } else if (use_bf16) {
    launch_k(trimul_gate_fwd_k<bf16>, grid, 256, 0, s, (const bf16 *)abg, ld, mask, (bf16 *)A, (bf16 *)B, pitch, R, cm,
             incoming);
  } else {
    launch_k(trimul_gate_fwd_k<float>, grid, 256, 0, s, (const float *)abg, ld, mask, (float *)A, (float *)B, pitch, R,
             cm, incoming);
  }
  return cudaGetLastError();
}

cudaError_t trimul_gate_bwd(const void *dA, const void *dB, int64_t pitch, const void *abg, int64_t ld,
                            const float *mask, void *dabg, int R, int cm, int incoming, int use_bf16, cudaStream_t s) {
  Prof prof("trimul_gate_bwd", s, 0, (use_bf16 ? 2.0 : 4.0) * R * (double)R * 10.0 * cm, 1);
  if (use_bf16 && trimul_gate_tma_supported(abg, ld, dA, dB, pitch, R, cm) && (((uintptr_t)dabg) & 15u) == 0) {
    const cudaError_t e = trimul_gate_bwd_tma_launch(dA, dB, pitch, abg, ld, mask, dabg, R, cm, incoming, s);
    if (e != cudaErrorNotSupported) return e;
  }
  dim3 grid((R + 31) / 32, (R + 31) / 32, (cm + 3) / 4);
  const bool v8 = cm % 8 == 0 && ld % 8 == 0 && (((uintptr_t)abg) & 15u) == 0 && (((uintptr_t)dabg) & 15u) == 0;
  if (use_bf16 && v8 && cm % TG_CH == 0) {
    dim3 gt((R + TG_COLS - 1) / TG_COLS, (R + TG_ROWS - 1) / TG_ROWS, cm / TG_CH);
    launch_k(trimul_gate_bwd_t, gt, 256, 0, s, (const bf16 *)dA, (const bf16 *)dB, pitch, (const bf16 *)abg, ld, mask,
                                         (bf16 *)dabg, R, cm, incoming);
  } else if (use_bf16 && v8) {
    dim3 g8((R + 31) / 32, (R + 31) / 32, cm / 8);
    launch_k(trimul_gate_bwd_v8, g8, 256, 0, s, (const bf16 *)dA, (const bf16 *)dB, pitch, (const bf16 *)abg, ld, mask,
                                          (bf16 *)dabg, R, cm, incoming);
  } else if (use_bf16)
    launch_k(trimul_gate_bwd_k<bf16>, grid, 256, 0, s, (const bf16 *)dA, (const bf16 *)dB, pitch, (const bf16 *)abg, ld,
                                                 mask, (bf16 *)dabg, R, cm, incoming);
  else
    launch_k(trimul_gate_bwd_k<float>, grid, 256, 0, s, (const float *)dA, (const float *)dB, pitch, (const float *)abg, ld,
                                                  mask, (float *)dabg, R, cm, incoming);
  return cudaGetLastError();
}

cudaError_t gate_out_bwd(const void *dz, const void *g, int64_t g_ld, const void *y, void *dy, void *dgpre,
                         int64_t dg_ld, int64_t P, int C, int use_bf16, cudaStream_t s, float *dsum) {
  Prof prof("gate_out_bwd", s, 0, (use_bf16 ? 2.0 : 4.0) * (double)P * C * 5, 1);
  auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
  if (use_bf16 && C % 8 == 0 && C <= 256 && 256 % (C / 8) == 0 && g_ld % 8 == 0 && dg_ld % 8 == 0 && a16(dz) &&
      a16(g) && a16(y) && a16(dy) && a16(dgpre)) {
    const int64_t n = P * (C / 8);
    launch_k(gate_out_bwd_v8, one_wave(gate_out_bwd_v8, (n + 1023) / 1024), 256, 0, s, (const bf16 *)dz,
             (const bf16 *)g, g_ld, (const bf16 *)y, (bf16 *)dy, (bf16 *)dgpre, dg_ld, P, C, dsum);
    return cudaGetLastError();
  } else if (use_bf16)
    launch_k(gate_out_bwd_k<bf16>, nblk(P * C), 256, 0, s, (const bf16 *)dz, (const bf16 *)g, g_ld, (const bf16 *)y,
                                                     (bf16 *)dy, (bf16 *)dgpre, dg_ld, P, C);
  else
    launch_k(gate_out_bwd_k<float>, nblk(P * C), 256, 0, s, (const float *)dz, (const float *)g, g_ld, (const float *)y,
                                                      (float *)dy, (float *)dgpre, dg_ld, P, C);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && dsum) e = colsum(dy, C, P, C, use_bf16, s, dsum);
  return e;
}

cudaError_t attn_gate_bwd(const AttnArgs &a, const void *dog, void *dgpre, int64_t sGb_d, int64_t sGx_d, void *do_att,
                          float *D, int use_bf16, cudaStream_t s) {
  Prof prof("attn_gate_bwd", s, 0, (use_bf16 ? 2.0 : 4.0) * (double)a.B1 * a.X * a.H * a.c * 5, 1);
  const int64_t rows = (int64_t)a.B1 * a.X;
  if (use_bf16)
    launch_k(attn_gate_bwd_k<bf16>, nblk(rows, 8), 256, 0, s, a, (const bf16 *)dog, (bf16 *)dgpre, sGb_d, sGx_d,
                                                        (bf16 *)do_att, D);
  else
    launch_k(attn_gate_bwd_k<float>, nblk(rows, 8), 256, 0, s, a, (const float *)dog, (float *)dgpre, sGb_d, sGx_d,
                                                         (float *)do_att, D);
  return cudaGetLastError();
}

cudaError_t attn_dq_store(const AttnArgs &a, void *dq, int use_bf16, cudaStream_t s) {
  Prof prof("attn_dq_store", s, 0, (use_bf16 ? 6.0 : 8.0) * (double)a.B1 * a.X * a.H * a.c, 1);
  const int64_t n = (int64_t)a.B1 * a.X * a.H * a.c;
  if (use_bf16) launch_k(attn_dq_store_k<bf16>, nblk(n), 256, 0, s, a, (bf16 *)dq);
  else launch_k(attn_dq_store_k<float>, nblk(n), 256, 0, s, a, (float *)dq);
  return cudaGetLastError();
}

cudaError_t opm_inv_norm(const float *mask, float *inv, int S, int R, float eps, cudaStream_t s) {
  Prof prof("opm_inv_norm", s, 0, 8.0 * S * (double)R + 4.0 * R * (double)R, 1);
  launch_k(opm_inv_norm_k, dim3((R + 31) / 32, (R + 31) / 32), 256, 0, s, mask, inv, S, R, eps);
  return cudaGetLastError();
}

cudaError_t row_scale(const void *x, const float *scale, void *y, int64_t M, int C, int use_bf16, cudaStream_t s,
                      float *dsum) {
  Prof prof("row_scale", s, 0, (use_bf16 ? 4.0 : 8.0) * M * (double)C, 1);
  if (use_bf16 && C % 8 == 0 && C <= 256 && 256 % (C / 8) == 0 && (((uintptr_t)x | (uintptr_t)y) & 15u) == 0) {
    const int64_t n = M * (C / 8);
    launch_k(row_scale_v8, one_wave(row_scale_v8, (n + 1023) / 1024), 256, 0, s, (const bf16 *)x, scale, (bf16 *)y, M,
             C, dsum);
    return cudaGetLastError();
  } else if (use_bf16) launch_k(row_scale_k<bf16>, nblk(M * C), 256, 0, s, (const bf16 *)x, scale, (bf16 *)y, M, C);
  else launch_k(row_scale_k<float>, nblk(M * C), 256, 0, s, (const float *)x, scale, (float *)y, M, C);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && dsum) e = colsum(y, C, M, C, use_bf16, s, dsum);
  return e;
}

cudaError_t to_f32(const void *src, float *dst, int64_t n, int use_bf16, cudaStream_t s) {
  Prof prof("convert", s, 0, (use_bf16 ? 6.0 : 8.0) * n, 1);
  if (use_bf16) launch_k(to_f32_k<bf16>, nblk(n), 256, 0, s, (const bf16 *)src, dst, n);
  else launch_k(to_f32_k<float>, nblk(n), 256, 0, s, (const float *)src, dst, n);
  return cudaGetLastError();
}
cudaError_t from_f32(const float *src, void *dst, int64_t n, int use_bf16, cudaStream_t s) {
  Prof prof("convert", s, 0, (use_bf16 ? 6.0 : 8.0) * n, 1);
  if (use_bf16) launch_k(from_f32_k<bf16>, nblk(n), 256, 0, s, src, (bf16 *)dst, n);
  else launch_k(from_f32_k<float>, nblk(n), 256, 0, s, src, (float *)dst, n);
  return cudaGetLastError();
}
namespace {
// dst[(a * dst_B + b) * W + w] = src[(a * src_B + b) * W + w] for a < A, b < B,
// w < W (32-bit words): one row (a, b) of W words per warp step.
__global__ void __launch_bounds__(256) copy_rows_k(const uint32_t *src, uint32_t *dst, int64_t A, int64_t B,
                                                    int64_t src_B, int64_t dst_B, int W) {
  pdl_entry();
  const int64_t rows = A * B;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t r = wid; r < rows; r += nw) {
    const int64_t a = r / B, b = r - a * B;
    const uint32_t *sp = src + (a * src_B + b) * W;
    uint32_t *dp = dst + (a * dst_B + b) * W;
    for (int w = lane; w < W; w += 32) dp[w] = sp[w];
  }
}
}  // namespace

namespace {
// dst[(b * dst_ld + a) * W + w] = src[(a * Bd + b) * W + w]: rows of W words
// on an A x Bd grid, transposed, one row per warp step (a row's reads and its
// write each one contiguous run of W words).
__global__ void __launch_bounds__(256) transpose_rows_k(const uint32_t *src, uint32_t *dst, int64_t A, int64_t Bd,
                                                        int W, int64_t dst_ld) {
  pdl_entry();
  const int64_t rows = A * Bd;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t r = wid; r < rows; r += nw) {
    const int64_t a = r / Bd, b = r - a * Bd;
    const uint32_t *sp = src + r * W;
    uint32_t *dp = dst + (b * dst_ld + a) * W;
    for (int w = lane; w < W; w += 32) dp[w] = sp[w];
  }
}
}  // namespace

cudaError_t transpose_rows(const void *src, void *dst, int64_t A, int64_t Bd, int W, int64_t dst_ld, cudaStream_t s) {
  if (A <= 0 || Bd <= 0 || W <= 0) return cudaSuccess;
  if (dst_ld < A) return cudaErrorInvalidValue;
  Prof prof("transpose_rows", s, 0, 8.0 * A * Bd * W);
  const unsigned grid = (unsigned)std::min<int64_t>((A * Bd + 7) / 8, 152 * 16);
  launch_k(transpose_rows_k, grid, 256, 0, s, (const uint32_t *)src, (uint32_t *)dst, A, Bd, W, dst_ld);
  return cudaGetLastError();
}

cudaError_t copy_rows_strided(const void *src, void *dst, int64_t A, int64_t B, int64_t src_B, int64_t dst_B, int W,
                              cudaStream_t s) {
  if (A <= 0 || B <= 0 || W <= 0) return cudaSuccess;
  Prof prof("copy_rows", s, 0, 8.0 * A * B * W);
  const int64_t warps = A * B;
  const unsigned grid = (unsigned)std::min<int64_t>((warps + 7) / 8, 152 * 16);
  launch_k(copy_rows_k, grid, 256, 0, s, (const uint32_t *)src, (uint32_t *)dst, A, B, src_B, dst_B, W);
  return cudaGetLastError();
}

cudaError_t f32_to_bf16(const float *src, bf16 *dst, int64_t n, cudaStream_t s) {
  Prof prof("convert", s, 0, 6.0 * n, 1);
  launch_k(from_f32_k<bf16>, nblk(n), 256, 0, s, src, dst, n);
  return cudaGetLastError();
}

}  // namespace evo

namespace evo {

cudaError_t dropout_apply(const void *upd, const float *scale, const void *res, void *out, int64_t P, int C, int R,
                          int colwise, int use_bf16, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  Prof prof("dropout", s, 0, (use_bf16 ? 2.0 : 4.0) * (double)P * C * (res ? 3 : 2), 1);
  auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
  if (use_bf16 && C % 8 == 0 && a16(upd) && a16(scale) && a16(out) && (!res || a16(res))) {
    const int64_t n = P * (C / 8);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    launch_k(dropout_apply_v8, blocks, 256, 0, s, (const bf16 *)upd, scale, (const bf16 *)res, (bf16 *)out, P, C, R,
             colwise);
  } else if (use_bf16) {
    launch_k(dropout_apply_k<bf16>, nblk(P * C), 256, 0, s, (const bf16 *)upd, scale, (const bf16 *)res, (bf16 *)out,
             P, C, R, colwise);
  } else {
    launch_k(dropout_apply_k<float>, nblk(P * C), 256, 0, s, (const float *)upd, scale, (const float *)res,
             (float *)out, P, C, R, colwise);
  }
  return cudaGetLastError();
}

}  // namespace evo
