// Triangle-multiplication gating (Alg. 11 and 12, the gated projections a and
// b) as TMA-tiled BF16 kernels.
//
// The projection output abg is row-major over positions p (columns
// [ap | ag | bp | bg | g], cm channels each for the first four); the batched
// per-channel products want a and b channel-major, A[c][i][j] with a row
// pitch.  One CTA moves a tile of 64 positions (64 consecutive ocol of one
// orow) x 64 channels: TMA brings the four 8 KB source tiles (128-byte
// swizzled rows of 64 channels) in at once, the threads gate and transpose
// through shared memory, and TMA stores the two channel-major 8 KB tiles
// (rows of 64 positions).  The backward reads dA, dB in the same tiles and
// writes the gradients of the four projections in place of their tiles.
// Position of (orow, ocol): orow R + ocol (outgoing) or ocol R + orow
// (incoming); the tensor maps order their dimensions by stride, so both
// cases give the same shared-memory tile, rows indexed by ocol.
#include "tc.cuh"

namespace evo {
using namespace tc;
namespace {

constexpr int TT_C = 64;                 // channels per tile
constexpr int TT_Q = 64;                 // positions per tile
constexpr int TT_TILE = TT_C * TT_Q * 2;  // bytes of one bf16 tile

// byte offset of 16-byte chunk q of row r in a tile of 128-byte rows written
// by TMA with the 128-byte swizzle (tile base 1024-byte aligned)
__device__ __forceinline__ uint32_t sw128(int r, int q) { return (uint32_t)(r * 128 + ((q ^ (r & 7)) << 4)); }

__device__ __forceinline__ float sigm_tc(float x) { return __fdividef(1.f, 1.f + __expf(-x)); }

__device__ __forceinline__ void lds8(uint32_t addr, float (&v)[8]) {
  uint32_t w0, w1, w2, w3;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3) : "r"(addr));
  // bf16 to fp32 is exact: the bf16 bits are the top half of the fp32 word
  v[0] = __uint_as_float(w0 << 16), v[1] = __uint_as_float(w0 & 0xffff0000u);
  v[2] = __uint_as_float(w1 << 16), v[3] = __uint_as_float(w1 & 0xffff0000u);
  v[4] = __uint_as_float(w2 << 16), v[5] = __uint_as_float(w2 & 0xffff0000u);
  v[6] = __uint_as_float(w3 << 16), v[7] = __uint_as_float(w3 & 0xffff0000u);
}
__device__ __forceinline__ void sts8(uint32_t addr, const float (&v)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    w[k] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k])) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k + 1])) << 16);
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
               : "memory");
}
__device__ __forceinline__ void sts16(uint32_t addr, float v) {
  asm volatile("st.shared.b16 [%0], %1;" ::"r"(addr), "h"(__bfloat16_as_ushort(__float2bfloat16_rn(v))) : "memory");
}
__device__ __forceinline__ float lds16(uint32_t addr) {
  unsigned short u;
  asm volatile("ld.shared.b16 %0, [%1];" : "=h"(u) : "r"(addr));
  return __uint_as_float((uint32_t)u << 16);
}

// mask of the positions this thread gates: ocol = q0 + 32 half + lane
__device__ __forceinline__ void load_mask(const float *mask, int R, int orow, int q0, int incoming, float (&mk)[2]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int ocol = q0 + 32 * half + lane;
    mk[half] = 0.f;
    if (ocol < R) mk[half] = mask[incoming ? (int64_t)ocol * R + orow : (int64_t)orow * R + ocol];
  }
}

// the four source tiles ap, ag, bp, bg (swap: bp, bg, ap, ag)
__device__ __forceinline__ void load_abg(const CUtensorMap *tm, uint32_t tiles, int cm, int c0, int q0, int orow,
                                         int incoming, uint64_t *bar, int swap = 0) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int src = swap ? (s ^ 2) : s;
    if (incoming) tma_load_3d(tiles + s * TT_TILE, tm, src * cm + c0, orow, q0, bar);
    else tma_load_3d(tiles + s * TT_TILE, tm, src * cm + c0, q0, orow, bar);
  }
}

// grid (ceil(R / 64), R, cm / 64): tile of ocol q0 .. q0 + 63 of row orow,
// channels c0 .. c0 + 63
__global__ void __launch_bounds__(256) trimul_gate_fwd_tma(const __grid_constant__ CUtensorMap tm_abg,
                                                           const __grid_constant__ CUtensorMap tm_A,
                                                           const __grid_constant__ CUtensorMap tm_B,
                                                           const float *mask, int R, int cm, int incoming, int swap) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int s_abort;
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const uint32_t in = base, outA = base + 4 * TT_TILE, outB = outA + TT_TILE;
  const int q0 = blockIdx.x * TT_Q, orow = blockIdx.y, c0 = blockIdx.z * TT_C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  pdl_entry();  // abg is the previous kernel's output
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, 4 * TT_TILE);
    load_abg(&tm_abg, in, cm, c0, q0, orow, incoming, &bar, swap);
  }
  float mk[2];
  load_mask(mask, R, orow, q0, incoming, mk);
  const bool ok = __syncthreads_and(mbar_wait(&bar, 0, &s_abort));
  if (!ok) {
    if (threadIdx.x == 0) mbar_drain(&bar, 0);
    return;
  }
  // items: (a or b, half, 8-channel chunk); a warp takes four
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int item = warp + 8 * it;
    const int ab = item >> 4, half = (item >> 3) & 1, chunk = item & 7;
    const int r = 32 * half + lane;
    float p[8], g[8];
    lds8(in + (2 * ab) * TT_TILE + sw128(r, chunk), p);
    lds8(in + (2 * ab + 1) * TT_TILE + sw128(r, chunk), g);
    const uint32_t out = ab ? outB : outA;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = chunk * 8 + k;
      sts16(out + sw128(c, r >> 3) + (r & 7) * 2, mk[half] * p[k] * sigm_tc(g[k]));
    }
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    tma_store_3d(&tm_A, outA, q0, orow, c0);
    tma_store_3d(&tm_B, outB, q0, orow, c0);
    bulk_commit();
    bulk_wait_read_all();
  }
}

// Backward: d ap = dA mask sigmoid(ag); d ag = dA mask ap sigmoid'(ag) (and b
// likewise), written over the abg tiles and stored to dabg.
__global__ void __launch_bounds__(256) trimul_gate_bwd_tma(const __grid_constant__ CUtensorMap tm_abg,
                                                           const __grid_constant__ CUtensorMap tm_dA,
                                                           const __grid_constant__ CUtensorMap tm_dB,
                                                           const __grid_constant__ CUtensorMap tm_dabg,
                                                           const float *mask, int R, int cm, int incoming) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int s_abort;
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const uint32_t in = base, dAt = base + 4 * TT_TILE, dBt = dAt + TT_TILE;
  const int q0 = blockIdx.x * TT_Q, orow = blockIdx.y, c0 = blockIdx.z * TT_C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  pdl_entry();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, 6 * TT_TILE);
    load_abg(&tm_abg, in, cm, c0, q0, orow, incoming, &bar);
    tma_load_3d(dAt, &tm_dA, q0, orow, c0, &bar);
    tma_load_3d(dBt, &tm_dB, q0, orow, c0, &bar);
  }
  float mk[2];
  load_mask(mask, R, orow, q0, incoming, mk);
  const bool ok = __syncthreads_and(mbar_wait(&bar, 0, &s_abort));
  if (!ok) {
    if (threadIdx.x == 0) mbar_drain(&bar, 0);
    return;
  }
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int item = warp + 8 * it;
    const int ab = item >> 4, half = (item >> 3) & 1, chunk = item & 7;
    const int r = 32 * half + lane;
    const uint32_t pa = in + (2 * ab) * TT_TILE + sw128(r, chunk), ga = in + (2 * ab + 1) * TT_TILE + sw128(r, chunk);
    float p[8], g[8], dp[8], dg[8];
    lds8(pa, p);
    lds8(ga, g);
    const uint32_t dt = ab ? dBt : dAt;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = chunk * 8 + k;
      const float d = lds16(dt + sw128(c, r >> 3) + (r & 7) * 2) * mk[half];
      const float sg = sigm_tc(g[k]);
      dp[k] = d * sg;
      dg[k] = d * p[k] * sg * (1.f - sg);
    }
    sts8(pa, dp);
    sts8(ga, dg);
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (incoming) tma_store_3d(&tm_dabg, in + s * TT_TILE, s * cm + c0, orow, q0);
      else tma_store_3d(&tm_dabg, in + s * TT_TILE, s * cm + c0, q0, orow);
    }
    bulk_commit();
    bulk_wait_read_all();
  }
}

// ---------------------------------------------------------------------------
// LayerNorm of the triangle-multiplication product (Alg. 11 and 12, the
// LayerNorm before the output projection), channel-major in, row-major out,
// and its backward.  The unit of work is a tile of 64 positions j of one row
// i with all C channels: C / 64 channel-major tiles of [64 c][64 j] (x, dx)
// and row-major tiles of [64 j][64 c] (y, dy), 8 KB each, 128-byte swizzled.
//
// Persistent CTAs of C threads walk the tiles (blockIdx.x, + gridDim.x, ...)
// with two shared-memory buffers: the next tile's TMA loads are in flight
// while the current one is worked, and the result is written in place of
// the input and stored by TMA.  Thread t owns positions 8 pg .. 8 pg + 7 and
// channels 8 cg .. 8 cg + 7 of a tile, pg = t % 8 and cg = (t / 8 + pg) mod
// (C / 8): the eight threads of a quarter-warp then read and write eight
// different 16-byte bank groups both in the channel-major tiles (row c,
// chunk pg) and in the row-major ones (row j, chunk cg).  Per-position sums
// over the channels go through shared memory (the C / 8 threads of a
// position group sit in different warps).
constexpr float LNC_EPS = 1e-5f;
constexpr int LNC_RED_LD = 68;  // floats per row of the per-position partials (68 = 4 mod 32: no bank conflicts)

template <int C>
struct LnCm {
  static constexpr int NCG = C / 8, NT = C / 64;
  static constexpr int BUF = NT * TT_TILE;  // one operand of one tile
};

// per-position partials v (positions 8 pg ..) of channel group cg into red
__device__ __forceinline__ void lnc_put(float *red, int cg, int pg, const float (&v)[8]) {
  float4 *d = reinterpret_cast<float4 *>(red + cg * LNC_RED_LD + 8 * pg);
  d[0] = make_float4(v[0], v[1], v[2], v[3]);
  d[1] = make_float4(v[4], v[5], v[6], v[7]);
}
// sum over the channel groups of position t (t < 64)
template <int NCG>
__device__ __forceinline__ float lnc_sum(const float *red, int t) {
  float s = 0.f;
#pragma unroll
  for (int g = 0; g < NCG; ++g) s += red[g * LNC_RED_LD + t];
  return s;
}
__device__ __forceinline__ void lnc_get8(const float *a, int pg, float (&v)[8]) {
  const float4 lo = reinterpret_cast<const float4 *>(a + 8 * pg)[0], hi = reinterpret_cast<const float4 *>(a + 8 * pg)[1];
  v[0] = lo.x, v[1] = lo.y, v[2] = lo.z, v[3] = lo.w, v[4] = hi.x, v[5] = hi.y, v[6] = hi.z, v[7] = hi.w;
}

// Issue the loads of tile `tile` (x channel-major; dy row-major when nsrc is
// 2) into buffer base `buf`, completing on bar.
template <int C>
__device__ __forceinline__ void lnc_load(const CUtensorMap *tm_x, const CUtensorMap *tm_dy, int nsrc, uint32_t buf,
                                         int tile, int ntj, uint64_t *bar) {
  using L = LnCm<C>;
  const int j0 = (tile % ntj) * 64, i = tile / ntj;
  mbar_arrive_expect_tx(bar, nsrc * L::BUF);
#pragma unroll
  for (int c = 0; c < L::NT; ++c) {
    tma_load_3d(buf + c * TT_TILE, tm_x, j0, i, 64 * c, bar);
    if (nsrc == 2) tma_load_3d(buf + L::BUF + c * TT_TILE, tm_dy, 64 * c, j0, i, bar);
  }
}

// After an abort: wait (bounded) for the loads still in flight into each
// buffer, and for the stores still reading one.
__device__ __forceinline__ void lnc_drain(uint64_t *full, const uint32_t (&issued)[2], const uint32_t (&used)[2]) {
  for (int b = 0; b < 2; ++b)
    for (uint32_t u = used[b]; u < issued[b]; ++u) mbar_drain(&full[b], u & 1u);
  bulk_wait_read_all();
}

// Forward: y = (x - mean) / sqrt(var + eps) gamma + beta over the C channels
// of each position; ntiles = ceil(R / 64) rows of tiles.
template <int C>
__global__ void __launch_bounds__(C) ln_fwd_cm_tma(const __grid_constant__ CUtensorMap tm_x,
                                                   const __grid_constant__ CUtensorMap tm_y, const float *gamma,
                                                   const float *beta, int ntj, int ntiles) {
  using L = LnCm<C>;
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ volatile int s_abort;
  __shared__ __align__(16) float red[L::NCG * LNC_RED_LD];
  __shared__ __align__(16) float mu[64], rs[64];
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const int t = threadIdx.x, pg = t & 7, cg = ((t >> 3) + pg) % L::NCG, cb = cg >> 3, r = cg & 7;
  uint32_t issued[2] = {0u, 0u}, used[2] = {0u, 0u};
  if (t == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  pdl_entry();
  if (t == 0) {
    for (int k = 0; k < 2; ++k) {
      const int tile = blockIdx.x + k * gridDim.x;
      if (tile < ntiles) lnc_load<C>(&tm_x, nullptr, 1, base + k * L::BUF, tile, ntj, &full[k]), ++issued[k];
    }
  }
  float gm[8], bt[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) gm[k] = gamma[8 * cg + k], bt[k] = beta[8 * cg + k];
  for (int tile = blockIdx.x, it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const uint32_t buf = base + b * L::BUF;
    const bool ok = __syncthreads_and(mbar_wait(&full[b], (uint32_t)(it >> 1) & 1u, &s_abort));
    if (!ok) {
      if (t == 0) lnc_drain(full, issued, used);
      return;
    }
    ++used[b];
    // xv[k][p]: channel 8 cg + k, position 8 pg + p
    float xv[8][8], s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) lds8(buf + cb * TT_TILE + sw128(8 * r + k, pg), xv[k]);
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      s[p] = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) s[p] += xv[k][p];
    }
    lnc_put(red, cg, pg, s);
    __syncthreads();
    if (t < 64) mu[t] = lnc_sum<L::NCG>(red, t) * (1.f / C);
    __syncthreads();
    float m8[8];
    lnc_get8(mu, pg, m8);
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      s[p] = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        xv[k][p] -= m8[p];
        s[p] += xv[k][p] * xv[k][p];
      }
    }
    lnc_put(red, cg, pg, s);
    __syncthreads();
    if (t < 64) rs[t] = rsqrtf(lnc_sum<L::NCG>(red, t) * (1.f / C) + LNC_EPS);
    __syncthreads();
    float r8[8];
    lnc_get8(rs, pg, r8);
    // y rows j = 8 pg + p of tile cb, chunk r (the x tile's reads are done)
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      float o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = xv[k][p] * r8[p] * gm[k] + bt[k];
      sts8(buf + cb * TT_TILE + sw128(8 * pg + p, r), o);
    }
    fence_proxy_async();
    __syncthreads();
    if (t == 0) {
      const int j0 = (tile % ntj) * 64, i = tile / ntj;
      for (int c = 0; c < L::NT; ++c) tma_store_3d(&tm_y, buf + c * TT_TILE, 64 * c, j0, i);
      bulk_commit();
      const int next = tile + 2 * gridDim.x;
      if (next < ntiles) {
        bulk_wait_read_all();  // the store has read the buffer
        lnc_load<C>(&tm_x, nullptr, 1, buf, next, ntj, &full[b]);
        ++issued[b];
      }
    }
  }
  if (t == 0) bulk_wait_read_all();
}

// Backward: dy row-major, x channel-major; dx channel-major (written in place
// of x); the gamma / beta gradients of the thread's channels accumulate over
// its tiles and meet in fp32 atomics once per CTA.
//   dx = rs (dy gamma - mean_c(dy gamma) - xhat mean_c(dy gamma xhat))
template <int C>
__global__ void __launch_bounds__(C) ln_bwd_cm_tma(const __grid_constant__ CUtensorMap tm_x,
                                                   const __grid_constant__ CUtensorMap tm_dy,
                                                   const __grid_constant__ CUtensorMap tm_dx, const float *gamma,
                                                   int ntj, int ntiles, float *dgamma, float *dbeta) {
  using L = LnCm<C>;
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ volatile int s_abort;
  __shared__ __align__(16) float red[L::NCG * LNC_RED_LD], red2[L::NCG * LNC_RED_LD];
  __shared__ __align__(16) float mu[64], rs[64], a1[64], a2[64];
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const int t = threadIdx.x, pg = t & 7, cg = ((t >> 3) + pg) % L::NCG, cb = cg >> 3, r = cg & 7;
  uint32_t issued[2] = {0u, 0u}, used[2] = {0u, 0u};
  if (t == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  pdl_entry();
  if (t == 0) {
    for (int k = 0; k < 2; ++k) {
      const int tile = blockIdx.x + k * gridDim.x;
      if (tile < ntiles) lnc_load<C>(&tm_x, &tm_dy, 2, base + k * 2 * L::BUF, tile, ntj, &full[k]), ++issued[k];
    }
  }
  float gm[8], dg[8], db[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) gm[k] = gamma[8 * cg + k], dg[k] = 0.f, db[k] = 0.f;
  bool ok = true;
  for (int tile = blockIdx.x, it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const uint32_t xb = base + b * 2 * L::BUF, dyb = xb + L::BUF;
    ok = __syncthreads_and(mbar_wait(&full[b], (uint32_t)(it >> 1) & 1u, &s_abort));
    if (!ok) break;
    ++used[b];
    // xv[k][p]: channel 8 cg + k, position 8 pg + p; dv[p][k]: the same element of dy
    float xv[8][8], dv[8][8], s[8], s2[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) lds8(xb + cb * TT_TILE + sw128(8 * r + k, pg), xv[k]);
#pragma unroll
    for (int p = 0; p < 8; ++p) lds8(dyb + cb * TT_TILE + sw128(8 * pg + p, r), dv[p]);
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      s[p] = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) s[p] += xv[k][p];
    }
    lnc_put(red, cg, pg, s);
    __syncthreads();
    if (t < 64) mu[t] = lnc_sum<L::NCG>(red, t) * (1.f / C);
    __syncthreads();
    float m8[8];
    lnc_get8(mu, pg, m8);
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      s[p] = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        xv[k][p] -= m8[p];
        s[p] += xv[k][p] * xv[k][p];
      }
    }
    lnc_put(red, cg, pg, s);
    __syncthreads();
    if (t < 64) rs[t] = rsqrtf(lnc_sum<L::NCG>(red, t) * (1.f / C) + LNC_EPS);
    __syncthreads();
    float r8[8];
    lnc_get8(rs, pg, r8);
    // xhat; the gamma / beta gradients; the per-position sums of dy gamma and
    // dy gamma xhat
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      s[p] = 0.f, s2[p] = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        xv[k][p] *= r8[p];
        dg[k] += dv[p][k] * xv[k][p];
        db[k] += dv[p][k];
        dv[p][k] *= gm[k];
        s[p] += dv[p][k];
        s2[p] += dv[p][k] * xv[k][p];
      }
    }
    lnc_put(red, cg, pg, s);
    lnc_put(red2, cg, pg, s2);
    __syncthreads();
    if (t < 64) a1[t] = lnc_sum<L::NCG>(red, t) * (1.f / C), a2[t] = lnc_sum<L::NCG>(red2, t) * (1.f / C);
    __syncthreads();
    float c1[8], c2[8];
    lnc_get8(a1, pg, c1);
    lnc_get8(a2, pg, c2);
    // dx rows c = 8 cg + k of tile cb, chunk pg (in place of x, read above)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float o[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) o[p] = r8[p] * (dv[p][k] - c1[p] - xv[k][p] * c2[p]);
      sts8(xb + cb * TT_TILE + sw128(8 * r + k, pg), o);
    }
    fence_proxy_async();
    __syncthreads();
    if (t == 0) {
      const int j0 = (tile % ntj) * 64, i = tile / ntj;
      for (int c = 0; c < L::NT; ++c) tma_store_3d(&tm_dx, xb + c * TT_TILE, j0, i, 64 * c);
      bulk_commit();
      const int next = tile + 2 * gridDim.x;
      if (next < ntiles) {
        bulk_wait_read_all();  // the store has read the buffer
        lnc_load<C>(&tm_x, &tm_dy, 2, xb, next, ntj, &full[b]);
        ++issued[b];
      }
    }
  }
  if (!ok) {
    if (t == 0) lnc_drain(full, issued, used);
    return;
  }
  // gamma / beta gradients: the eight threads of a channel group (pg = 0..7)
  // meet in shared memory (red, red2 reused: 8 x C floats each fit)
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; ++k) red[pg * C + 8 * cg + k] = dg[k], red2[pg * C + 8 * cg + k] = db[k];
  __syncthreads();
  float g = 0.f, bsum = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) g += red[q * C + t], bsum += red2[q * C + t];
  atomicAdd(dgamma + t, g);
  atomicAdd(dbeta + t, bsum);
  if (t == 0) bulk_wait_read_all();
}

// row-major [R][R][C] map, boxes of 64 channels x 64 positions j
bool map_rows(CUtensorMap *tm, const void *p, int R, int C, int rows = -1) {
  if (rows < 0) rows = R;
  const uint64_t dims[3] = {(uint64_t)C, (uint64_t)R, (uint64_t)rows};
  const uint64_t st[2] = {(uint64_t)C * 2, (uint64_t)R * C * 2};
  const uint32_t box[3] = {64, 64, 1};
  return make_tmap_nd(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, p, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

// abg-like map: channels [0, 4 cm) of rows of ld elements, positions in
// stride order (outgoing: ocol then orow; incoming: orow then ocol)
bool map_abg(CUtensorMap *tm, const void *p, int64_t ld, int R, int cm, int incoming, int rows = -1) {
  if (rows < 0) rows = R;  // an outgoing i-slab: rows orow of R columns
  const uint64_t dims[3] = {(uint64_t)4 * cm, (uint64_t)R, (uint64_t)rows};
  const uint64_t st[2] = {(uint64_t)ld * 2, (uint64_t)R * ld * 2};
  const uint32_t box[3] = {TT_C, incoming ? 1u : (uint32_t)TT_Q, incoming ? (uint32_t)TT_Q : 1u};
  return make_tmap_nd(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, p, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B);
}
// channel-major map: [c][orow][ocol] with row pitch, ocol clipped at R
bool map_cm(CUtensorMap *tm, const void *p, int64_t pitch, int R, int cm, int rows = -1, int64_t cstride = -1) {
  if (rows < 0) rows = R;
  if (cstride < 0) cstride = (int64_t)R * pitch;
  const uint64_t dims[3] = {(uint64_t)R, (uint64_t)rows, (uint64_t)cm};
  const uint64_t st[2] = {(uint64_t)pitch * 2, (uint64_t)cstride * 2};
  const uint32_t box[3] = {TT_Q, 1, TT_C};
  return make_tmap_nd(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, p, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

bool a16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

bool trimul_gate_tma_supported(const void *abg, int64_t ld, const void *A, const void *B, int64_t pitch, int R,
                               int cm) {
  return R > 0 && cm % TT_C == 0 && ld % 8 == 0 && pitch % 8 == 0 && a16(abg) && a16(A) && a16(B);
}

cudaError_t trimul_gate_fwd_tma_launch(const void *abg, int64_t ld, const float *mask, void *A, void *B, int64_t pitch,
                                       int R, int cm, int incoming, cudaStream_t s) {
  CUtensorMap ta, tA, tB;
  if (!map_abg(&ta, abg, ld, R, cm, incoming) || !map_cm(&tA, A, pitch, R, cm) || !map_cm(&tB, B, pitch, R, cm))
    return cudaErrorNotSupported;
  const int smem = 6 * TT_TILE + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(trimul_gate_fwd_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid((R + TT_Q - 1) / TT_Q, R, cm / TT_C);
  return launch_k(trimul_gate_fwd_tma, grid, 256, smem, s, ta, tA, tB, mask, R, cm, incoming, 0);
}

cudaError_t trimul_gate_fwd_rows(const void *abg, int64_t ld, const float *mask, void *A, int64_t a_cstride, void *B,
                                 int64_t b_cstride, int64_t pitch, int rows, int R, int cm, int swap, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (!trimul_gate_tma_supported(abg, ld, A, B, pitch, R, cm) || a_cstride % 8 || b_cstride % 8)
    return cudaErrorNotSupported;
  Prof prof("trimul_gate_fwd", s, 0, 2.0 * rows * (double)R * 6.0 * cm, 1);
  CUtensorMap ta, tA, tB;
  if (!map_abg(&ta, abg, ld, R, cm, 0, rows) || !map_cm(&tA, A, pitch, R, cm, rows, a_cstride) ||
      !map_cm(&tB, B, pitch, R, cm, rows, b_cstride))
    return cudaErrorNotSupported;
  const int smem = 6 * TT_TILE + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(trimul_gate_fwd_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid((R + TT_Q - 1) / TT_Q, rows, cm / TT_C);
  return launch_k(trimul_gate_fwd_tma, grid, 256, smem, s, ta, tA, tB, mask, R, cm, 0, swap);
}

cudaError_t trimul_gate_bwd_tma_launch(const void *dA, const void *dB, int64_t pitch, const void *abg, int64_t ld,
                                       const float *mask, void *dabg, int R, int cm, int incoming, cudaStream_t s) {
  CUtensorMap ta, tdA, tdB, tdabg;
  if (!map_abg(&ta, abg, ld, R, cm, incoming) || !map_cm(&tdA, dA, pitch, R, cm) ||
      !map_cm(&tdB, dB, pitch, R, cm) || !map_abg(&tdabg, dabg, ld, R, cm, incoming))
    return cudaErrorNotSupported;
  const int smem = 6 * TT_TILE + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(trimul_gate_bwd_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid((R + TT_Q - 1) / TT_Q, R, cm / TT_C);
  return launch_k(trimul_gate_bwd_tma, grid, 256, smem, s, ta, tdA, tdB, tdabg, mask, R, cm, incoming);
}

bool ln_cm_tma_supported(const void *x, int64_t pitch, const void *y, int R, int C) {
  return R > 0 && (C == 64 || C == 128 || C == 256) && pitch % 8 == 0 && a16(x) && a16(y);
}

namespace {
// Persistent grid of the channel-major LayerNorm kernels: as many CTAs as
// fit on the SMs at once (occupancy of the kernel at its shared memory),
// at most one per tile.
// (BWD, C) tell the kernels apart: their function types are alike
template <int BWD, int C, typename K>
cudaError_t lnc_launch_cfg(K kern, int smem, int threads, int ntiles, int *grid) {
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  *grid = std::max(1, std::min(ntiles, per_sm * sms));
  return cudaSuccess;
}

template <int C>
cudaError_t ln_fwd_cm_go(const CUtensorMap &tx, const CUtensorMap &ty, const float *gamma, const float *beta, int R,
                         int rows, cudaStream_t s) {
  const int ntj = (R + 63) / 64, ntiles = ntj * rows;
  const int smem = 2 * LnCm<C>::BUF + 1024;
  int grid = 0;
  const cudaError_t e = lnc_launch_cfg<0, C>(ln_fwd_cm_tma<C>, smem, C, ntiles, &grid);
  if (e != cudaSuccess) return e;
  return launch_k(ln_fwd_cm_tma<C>, grid, C, smem, s, tx, ty, gamma, beta, ntj, ntiles);
}
cudaError_t ln_fwd_cm_dispatch(const CUtensorMap &tx, const CUtensorMap &ty, const float *gamma, const float *beta,
                               int R, int rows, int C, cudaStream_t s) {
  if (C == 64) return ln_fwd_cm_go<64>(tx, ty, gamma, beta, R, rows, s);
  if (C == 128) return ln_fwd_cm_go<128>(tx, ty, gamma, beta, R, rows, s);
  if (C == 256) return ln_fwd_cm_go<256>(tx, ty, gamma, beta, R, rows, s);
  return cudaErrorNotSupported;
}
template <int C>
cudaError_t ln_bwd_cm_go(const CUtensorMap &tx, const CUtensorMap &tdy, const CUtensorMap &tdx, const float *gamma,
                         int R, float *dgamma, float *dbeta, cudaStream_t s) {
  const int ntj = (R + 63) / 64, ntiles = ntj * R;
  const int smem = 4 * LnCm<C>::BUF + 1024;
  int grid = 0;
  const cudaError_t e = lnc_launch_cfg<1, C>(ln_bwd_cm_tma<C>, smem, C, ntiles, &grid);
  if (e != cudaSuccess) return e;
  return launch_k(ln_bwd_cm_tma<C>, grid, C, smem, s, tx, tdy, tdx, gamma, ntj, ntiles, dgamma, dbeta);
}
}  // namespace

cudaError_t ln_fwd_cm_tma_launch(const void *x, int64_t pitch, const float *gamma, const float *beta, void *y, int R,
                                 int C, cudaStream_t s) {
  CUtensorMap tx, ty;
  if (!map_cm(&tx, x, pitch, R, C) || !map_rows(&ty, y, R, C)) return cudaErrorNotSupported;
  return ln_fwd_cm_dispatch(tx, ty, gamma, beta, R, R, C, s);
}

cudaError_t ln_fwd_cm_rows(const void *x, int64_t pitch, int64_t cstride, const float *gamma, const float *beta,
                           void *y, int rows, int R, int C, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (!ln_cm_tma_supported(x, pitch, y, R, C) || cstride % 8) return cudaErrorNotSupported;
  Prof p("ln_fwd_cm", s, 0, 4.0 * rows * (double)R * C);
  CUtensorMap tx, ty;
  if (!map_cm(&tx, x, pitch, R, C, rows, cstride) || !map_rows(&ty, y, R, C, rows)) return cudaErrorNotSupported;
  return ln_fwd_cm_dispatch(tx, ty, gamma, beta, R, rows, C, s);
}

cudaError_t ln_bwd_cm_tma_launch(const void *dy, const void *x, int64_t pitch, const float *gamma, void *dx, int R,
                                 int C, float *dgamma, float *dbeta, cudaStream_t s) {
  CUtensorMap tx, tdy, tdx;
  if (!map_cm(&tx, x, pitch, R, C) || !map_rows(&tdy, dy, R, C) || !map_cm(&tdx, dx, pitch, R, C))
    return cudaErrorNotSupported;
  if (C == 64) return ln_bwd_cm_go<64>(tx, tdy, tdx, gamma, R, dgamma, dbeta, s);
  if (C == 128) return ln_bwd_cm_go<128>(tx, tdy, tdx, gamma, R, dgamma, dbeta, s);
  if (C == 256) return ln_bwd_cm_go<256>(tx, tdy, tdx, gamma, R, dgamma, dbeta, s);
  return cudaErrorNotSupported;
}

namespace {
__global__ void trimul_tc_debug_wait_kernel(int64_t limit_ns) {
  pdl_entry();
  debug_wait_body(limit_ns);
}
}  // namespace

cudaError_t trimul_tc_debug_wait(int64_t limit_ns, cudaStream_t s) {
  launch_k(trimul_tc_debug_wait_kernel, 1, 32, 0, s, limit_ns);
  return cudaGetLastError();
}

cudaError_t trimul_tc_error_read_clear(int *out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, tc_error_word, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(tc_error_word, &zero, sizeof(int));
}

}  // namespace evo
