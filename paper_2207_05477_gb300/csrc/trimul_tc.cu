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
// LayerNorm before the output projection), channel-major in, row-major out:
// one CTA per 64 positions j of a row i, all C channels (C / 64 tiles of
// [64 c][64 j] in, [64 j][64 c] out, each 8 KB, 128-byte swizzled).
constexpr int LN_MAXC = 256;
constexpr float LNC_EPS = 1e-5f;

// mean and rstd of the 64 positions of the channel-major tiles (256 threads:
// position t % 64, channel quarter t / 64); red holds 4 x 64 floats
__device__ __forceinline__ void cm_tile_stats(uint32_t xin, int C, float *red, float *mu, float *rs) {
  const int t = threadIdx.x, j = t & 63, qt = t >> 6, cpq = C / 4;
  float sum = 0.f;
  for (int c = qt * cpq; c < (qt + 1) * cpq; ++c) sum += lds16(xin + (c >> 6) * TT_TILE + sw128(c & 63, j >> 3) + (j & 7) * 2);
  red[qt * 64 + j] = sum;
  __syncthreads();
  if (t < 64) mu[t] = (red[t] + red[64 + t] + red[128 + t] + red[192 + t]) / C;
  __syncthreads();
  const float m = mu[j];
  float q = 0.f;
  for (int c = qt * cpq; c < (qt + 1) * cpq; ++c) {
    const float d = lds16(xin + (c >> 6) * TT_TILE + sw128(c & 63, j >> 3) + (j & 7) * 2) - m;
    q += d * d;
  }
  red[qt * 64 + j] = q;
  __syncthreads();
  if (t < 64) rs[t] = rsqrtf((red[t] + red[64 + t] + red[128 + t] + red[192 + t]) / C + LNC_EPS);
  __syncthreads();
}

// grid (ceil(R / 64), R)
__global__ void __launch_bounds__(256) ln_fwd_cm_tma(const __grid_constant__ CUtensorMap tm_x,
                                                     const __grid_constant__ CUtensorMap tm_y, const float *gamma,
                                                     const float *beta, int C) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int s_abort;
  __shared__ float red[256], mu[64], rs[64], gs[LN_MAXC], bs[LN_MAXC];
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const int nt = C / 64;
  const uint32_t xin = base, yout = base + nt * TT_TILE;
  const int j0 = blockIdx.x * 64, i = blockIdx.y;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  pdl_entry();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, nt * TT_TILE);
    for (int c = 0; c < nt; ++c) tma_load_3d(xin + c * TT_TILE, &tm_x, j0, i, 64 * c, &bar);
  }
  for (int c = threadIdx.x; c < C; c += blockDim.x) gs[c] = gamma[c], bs[c] = beta[c];
  const bool ok = __syncthreads_and(mbar_wait(&bar, 0, &s_abort));
  if (!ok) {
    if (threadIdx.x == 0) mbar_drain(&bar, 0);
    return;
  }
  cm_tile_stats(xin, C, red, mu, rs);
  // item (position j, 8-channel chunk q): lanes take consecutive j
  for (int item = threadIdx.x; item < 64 * (C / 8); item += blockDim.x) {
    const int j = item & 63, q = item >> 6;
    float o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = q * 8 + k;
      const float x = lds16(xin + (c >> 6) * TT_TILE + sw128(c & 63, j >> 3) + (j & 7) * 2);
      o[k] = (x - mu[j]) * rs[j] * gs[c] + bs[c];
    }
    sts8(yout + (q >> 3) * TT_TILE + sw128(j, q & 7), o);
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < nt; ++c) tma_store_3d(&tm_y, yout + c * TT_TILE, 64 * c, j0, i);
    bulk_commit();
    bulk_wait_read_all();
  }
}

// Backward: dy row-major tiles [64 j][64 c], x channel-major; dx channel-major
// (written over the x tiles), gamma / beta gradients by fp32 atomics.
__global__ void __launch_bounds__(256) ln_bwd_cm_tma(const __grid_constant__ CUtensorMap tm_x,
                                                     const __grid_constant__ CUtensorMap tm_dy,
                                                     const __grid_constant__ CUtensorMap tm_dx, const float *gamma,
                                                     int C, float *dgamma, float *dbeta) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int s_abort;
  __shared__ float red[256], red2[512], mu[64], rs[64], a1[64], a2[64], gs[LN_MAXC];
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const int nt = C / 64;
  const uint32_t xin = base, dyin = base + nt * TT_TILE;
  const int j0 = blockIdx.x * 64, i = blockIdx.y;
  const int t = threadIdx.x, j = t & 63, qt = t >> 6, cpq = C / 4;
  if (t == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  pdl_entry();
  if (t == 0) {
    mbar_arrive_expect_tx(&bar, 2 * nt * TT_TILE);
    for (int c = 0; c < nt; ++c) {
      tma_load_3d(xin + c * TT_TILE, &tm_x, j0, i, 64 * c, &bar);
      tma_load_3d(dyin + c * TT_TILE, &tm_dy, 64 * c, j0, i, &bar);
    }
  }
  for (int c = t; c < C; c += blockDim.x) gs[c] = gamma[c];
  const bool ok = __syncthreads_and(mbar_wait(&bar, 0, &s_abort));
  if (!ok) {
    if (t == 0) mbar_drain(&bar, 0);
    return;
  }
  cm_tile_stats(xin, C, red, mu, rs);
  auto xat = [&](int c, int jj) { return lds16(xin + (c >> 6) * TT_TILE + sw128(c & 63, jj >> 3) + (jj & 7) * 2); };
  auto dyat = [&](int c, int jj) {
    return lds16(dyin + (c >> 6) * TT_TILE + sw128(jj, (c & 63) >> 3) + (c & 7) * 2);
  };
  // a1 = mean_c(dy gamma), a2 = mean_c(dy gamma xhat) per position
  {
    const float m = mu[j], r = rs[j];
    float s1 = 0.f, s2 = 0.f;
    for (int c = qt * cpq; c < (qt + 1) * cpq; ++c) {
      const float gd = dyat(c, j) * gs[c];
      s1 += gd;
      s2 += gd * (xat(c, j) - m) * r;
    }
    red[qt * 64 + j] = s1;
    __syncthreads();
    if (t < 64) a1[t] = (red[t] + red[64 + t] + red[128 + t] + red[192 + t]) / C;
    __syncthreads();
    red[qt * 64 + j] = s2;
    __syncthreads();
    if (t < 64) a2[t] = (red[t] + red[64 + t] + red[128 + t] + red[192 + t]) / C;
    __syncthreads();
  }
  // gamma / beta gradients: 256 / C threads per channel, each over a slice of
  // the tile's positions, combined in shared memory (red2: 2 x 256 floats)
  {
    const int tpc = 256 / C, c = t % C, part = t / C, per = 64 / tpc;
    float sg = 0.f, sb = 0.f;
    for (int jj = part * per; jj < (part + 1) * per; ++jj) {
      const float d = dyat(c, jj);
      sg += d * (xat(c, jj) - mu[jj]) * rs[jj];
      sb += d;
    }
    red2[t] = sg;
    red2[256 + t] = sb;
    __syncthreads();
    if (t < C) {
      float g = 0.f, b = 0.f;
      for (int k = 0; k < tpc; ++k) g += red2[k * C + t], b += red2[256 + k * C + t];
      atomicAdd(dgamma + t, g);
      atomicAdd(dbeta + t, b);
    }
  }
  __syncthreads();  // every read of x is done before dx overwrites it
  for (int e = t; e < 64 * C; e += blockDim.x) {
    const int jj = e & 63, c = e >> 6;
    const uint32_t a = xin + (c >> 6) * TT_TILE + sw128(c & 63, jj >> 3) + (jj & 7) * 2;
    const float xh = (lds16(a) - mu[jj]) * rs[jj];
    sts16(a, rs[jj] * (dyat(c, jj) * gs[c] - a1[jj] - xh * a2[jj]));
  }
  fence_proxy_async();
  __syncthreads();
  if (t == 0) {
    for (int c = 0; c < nt; ++c) tma_store_3d(&tm_dx, xin + c * TT_TILE, j0, i, 64 * c);
    bulk_commit();
    bulk_wait_read_all();
  }
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

cudaError_t ln_fwd_cm_tma_launch(const void *x, int64_t pitch, const float *gamma, const float *beta, void *y, int R,
                                 int C, cudaStream_t s) {
  CUtensorMap tx, ty;
  if (!map_cm(&tx, x, pitch, R, C) || !map_rows(&ty, y, R, C)) return cudaErrorNotSupported;
  const int smem = 2 * (C / 64) * TT_TILE + 1024;
  static int attr = 0;
  if (attr < smem) {
    cudaError_t e = cudaFuncSetAttribute(ln_fwd_cm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  return launch_k(ln_fwd_cm_tma, dim3((R + 63) / 64, R), 256, smem, s, tx, ty, gamma, beta, C);
}

cudaError_t ln_fwd_cm_rows(const void *x, int64_t pitch, int64_t cstride, const float *gamma, const float *beta,
                           void *y, int rows, int R, int C, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (!ln_cm_tma_supported(x, pitch, y, R, C) || cstride % 8) return cudaErrorNotSupported;
  Prof p("ln_fwd_cm", s, 0, 4.0 * rows * (double)R * C);
  CUtensorMap tx, ty;
  if (!map_cm(&tx, x, pitch, R, C, rows, cstride) || !map_rows(&ty, y, R, C, rows)) return cudaErrorNotSupported;
  const int smem = 2 * (C / 64) * TT_TILE + 1024;
  static int attr = 0;
  if (attr < smem) {
    cudaError_t e = cudaFuncSetAttribute(ln_fwd_cm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  return launch_k(ln_fwd_cm_tma, dim3((R + 63) / 64, rows), 256, smem, s, tx, ty, gamma, beta, C);
}

cudaError_t ln_bwd_cm_tma_launch(const void *dy, const void *x, int64_t pitch, const float *gamma, void *dx, int R,
                                 int C, float *dgamma, float *dbeta, cudaStream_t s) {
  CUtensorMap tx, tdy, tdx;
  if (!map_cm(&tx, x, pitch, R, C) || !map_rows(&tdy, dy, R, C) || !map_cm(&tdx, dx, pitch, R, C))
    return cudaErrorNotSupported;
  const int smem = 2 * (C / 64) * TT_TILE + 1024;
  static int attr = 0;
  if (attr < smem) {
    cudaError_t e = cudaFuncSetAttribute(ln_bwd_cm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  return launch_k(ln_bwd_cm_tma, dim3((R + 63) / 64, R), 256, smem, s, tx, tdy, tdx, gamma, C, dgamma, dbeta);
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
