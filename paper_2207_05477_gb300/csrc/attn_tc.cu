// Gated self-attention forward on the 5th-generation tensor cores (sm_103a)
// for head dim 32 and at most 256 keys: the MSA row / column and triangle
// attentions of the Evoformer block at training-crop sizes (AF2 Alg. 7, 8,
// 13, 14; the fused operator of Sec. 3.1).
//
// One CTA of eight warps per (128 queries, head, batch item):
//   * TMA brings Q [128 x 32], K and V [Ypad x 32] (64-byte swizzle); each
//     warp streams its 32 rows of the pair-bias tile in 32-key chunks (fp32,
//     128-byte swizzle) through a ring of its own, so the softmax warps never
//     wait for one another;
//   * one tcgen05.mma pair computes S = Q K^T (M 128, N Ypad, K 32) into
//     TMEM columns [0, Ypad);
//   * thread = query row (warps w and w + 4 read TMEM lanes 32(w % 4).. and
//     take half of the key chunks each): pass 1 turns S into log2-domain
//     logits (scale, pair bias, key mask) stored back in place and takes the
//     row max; pass 2 writes P = 2^(logit - max) as bf16 pairs into TMEM
//     columns [0, Ypad / 2) (over logits every warp has consumed) and sums
//     it; partial maxima and sums meet in shared memory;
//   * tcgen05.mma with A = P from TMEM and B = V from shared memory
//     accumulates O = P V (M 128, N 32, K Ypad) in TMEM columns [128, 160);
//   * the epilogue divides by the row sum, writes the attention output and its
//     sigmoid-gated copy (bf16) and the row log-sum-exp (log2 domain) for the
//     backward.
// Keys are padded to a multiple of 32 (the pad and masked keys get a logit of
// -inf).  Every mbarrier wait is bounded (about a second); a wait that runs
// out records EVO_ERR_TIMEOUT in this unit's error word and the CTA returns.
#include <algorithm>
#include <cstring>

#include "prof.h"
#include "tc.cuh"

namespace evo {

using namespace tc;

bool tc::make_tmap_nd(CUtensorMap *tm, CUtensorMapDataType dt, int rank, const void *base, const uint64_t *dims,
                      const uint64_t *stride_bytes, const uint32_t *box, CUtensorMapSwizzle swz) {
  typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  if (!fn || rank < 1 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
    if (i > 0) st[i - 1] = stride_bytes[i - 1];
  }
  return fn(tm, dt, (cuuint32_t)rank, const_cast<void *>(base), d, st, b, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

constexpr int AT_C = 32;      // channels of a shared-memory q / k / v row (head dims 8 and 16 zero-padded)
constexpr int AT_WARPS = 8;   // backward: two per TMEM lane quarter, splitting the key chunks

constexpr float NEG_INF_F = -__builtin_huge_valf();
constexpr float POS_INF_F = __builtin_huge_valf();

// 2^x on the SFU (ex2.approx: relative error about 2^-22, far below the bf16
// rounding P receives next)
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Coordinates of a q/k/v tile in its 4-D map (d, then h / row / batch ordered by stride).
struct QkvPos {
  int row, h, b;  // which map dimension (1..3) holds the row, head and batch coordinate
};

__device__ __forceinline__ void tile_coords(const QkvPos &p, int row, int h, int b, int (&c)[4]) {
  c[0] = 0;
  c[p.row] = row;
  c[p.h] = h;
  c[p.b] = b;
}

// byte offset of 16-byte piece q of row r in a tile of 64-byte rows with the
// 64-byte swizzle (tile base 512-byte aligned)
__device__ __forceinline__ uint32_t sw64_off(int r, int q) { return (uint32_t)(r * 64 + (((q ^ (r >> 1)) & 3) << 4)); }

__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}

// -------------------------------------------------- forward, at most 256 keys
// At most 256 keys (the training-crop attentions, and the extra-MSA and
// template rows): all of a row's logits fit one TMEM tile, so one pass needs
// no online rescaling.  Head dims 8 and 16 arrive zero-padded to 32 channels
// (the TMA box is 32 channels wide; the copy fills the rest).
// One CTA of eight warps per (128 queries, head, batch item):
//   * TMA brings Q [128 x 32], K and V [Ypad x 32] (64-byte swizzle); each
//     warp streams its 32 rows of the pair-bias tile in 64-key boxes through
//     a ring of its own, so the softmax warps never wait for one another;
//   * one tcgen05.mma pair computes S = Q K^T (M 128, N Ypad, K 32) into
//     TMEM columns [0, Ypad);
//   * thread = query row (warps w and w + 4 read TMEM lanes 32(w % 4).. and
//     take half of the key chunks each): pass 1 turns S into log2-domain
//     logits (scale, pair bias, key mask) stored back in place and takes the
//     row max; pass 2 writes P = 2^(logit - max) as bf16 pairs into TMEM
//     columns [0, Ypad / 2) (over logits every warp has consumed) and sums
//     it; partial maxima and sums meet in shared memory;
//   * tcgen05.mma with A = P from TMEM and B = V from shared memory
//     accumulates O = P V (M 128, N 32, K Ypad) in TMEM columns [128, 160);
//   * the epilogue divides by the row sum, writes the attention output and its
//     sigmoid-gated copy (bf16) and the row log-sum-exp (log2 domain) for the
//     backward.
// Keys are padded to a multiple of 32 (the pad and masked keys get a logit of
// -inf).
constexpr int AT_QROWS = 128;
constexpr int AT_MAXKEYS = 256;
constexpr int AT_TMEM_COLS = 256;
constexpr int AT_O_COL = 128;  // O accumulator columns [128, 160)
// dynamic shared memory (offsets from a 1 KB aligned base)
constexpr int AT_Q_OFF = 0;                               // 128 x 64 B
constexpr int AT_K_OFF = AT_Q_OFF + AT_QROWS * 64;        // 256 x 64 B
constexpr int AT_V_OFF = AT_K_OFF + AT_MAXKEYS * 64;      // 256 x 64 B
// pair bias (bf16): per warp AT_BRING boxes of [32 rows x 64 keys] (4 KB each)
constexpr int AT_BRING = 2;
constexpr int AT_B_OFF = AT_V_OFF + AT_MAXKEYS * 64;
constexpr int AT_R_OFF = AT_B_OFF + AT_WARPS * AT_BRING * 4096;  // [2][128] row max, [2][128] row sum
constexpr int AT_M_OFF = AT_R_OFF + 4 * AT_QROWS * 4;            // 256 floats: additive key mask
constexpr int AT_SMEM = AT_M_OFF + AT_MAXKEYS * 4 + 1024;


struct AttnTcArgs {
  AttnArgs a;
  QkvPos pq, pk;  // q (and g) / k, v map dimension positions
  int ypad;       // keys padded to a multiple of 32 (<= 256)
  int has_bias;
};


__global__ void __launch_bounds__(AT_WARPS * 32, 2) attn_fwd_short(const __grid_constant__ CUtensorMap tmQ,
                                                             const __grid_constant__ CUtensorMap tmK,
                                                             const __grid_constant__ CUtensorMap tmV,
                                                             const __grid_constant__ CUtensorMap tmB, AttnTcArgs A) {
  pdl_trigger();
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar_qk, bar_v, bar_s, bar_o, bar_b[AT_WARPS][AT_BRING];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  const AttnArgs &a = A.a;
  const uint32_t raw = smem_u32(dsm);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = dsm + (base - raw);
  float *maskadd = reinterpret_cast<float *>(gbase + AT_M_OFF);
  float *red = reinterpret_cast<float *>(gbase + AT_R_OFF);  // [0..255] max, [256..511] sum
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int quarter = warp & 3, half = warp >> 2;
  const int x0 = blockIdx.x * AT_QROWS, h = blockIdx.y, b = blockIdx.z;
  const int ypad = A.ypad, nch = ypad / 32;
  // this warp's key chunks [c_lo, c_hi)
  const int c_mid = (nch + 1) / 2;
  const int c_lo = half ? c_mid : 0, c_hi = half ? nch : c_mid;

  if (tid == 0) {
    mbar_init(&bar_qk, 1);
    mbar_init(&bar_v, 1);
    mbar_init(&bar_s, 1);
    mbar_init(&bar_o, 1);
    for (int w = 0; w < AT_WARPS; ++w)
      for (int k = 0; k < AT_BRING; ++k) mbar_init(&bar_b[w][k], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)AT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // global memory only from here on: wait for the kernels before this one
  pdl_wait();
  // what this thread put in flight (drained after an abort): lane 0 of each
  // warp streams the pair bias of its rows and chunks; thread 0 issues the rest
  int bias_issued = 0, bias_done = 0;
  bool s_issued = false, o_issued = false;
  // the warp's pair bias (bf16): one [32 rows x 64 keys] box per pair of its
  // key chunks, all requested at once
  const uint32_t bring = base + AT_B_OFF + (uint32_t)warp * AT_BRING * 4096u;
  if (A.has_bias && lane == 0)
    for (int bx = 0; bx < AT_BRING && c_lo + 2 * bx < c_hi; ++bx) {
      mbar_arrive_expect_tx(&bar_b[warp][bx], 4096);
      tma_load_3d(bring + bx * 4096u, &tmB, (c_lo + 2 * bx) * 32, x0 + quarter * 32, h, &bar_b[warp][bx]);
      ++bias_issued;
    }

  if (tid == 0) {
    int c[4];
    mbar_arrive_expect_tx(&bar_qk, (uint32_t)(AT_QROWS * 64 + ypad * 64));
    tile_coords(A.pq, x0, h, b, c);
    tma_load_4d(base + AT_Q_OFF, &tmQ, c[0], c[1], c[2], c[3], &bar_qk);
    tile_coords(A.pk, 0, h, b, c);
    tma_load_4d(base + AT_K_OFF, &tmK, c[0], c[1], c[2], c[3], &bar_qk);
    mbar_arrive_expect_tx(&bar_v, (uint32_t)(ypad * 64));
    tma_load_4d(base + AT_V_OFF, &tmV, c[0], c[1], c[2], c[3], &bar_v);
  }
  // additive key mask (0 for a valid key, -inf for a masked or padding key),
  // read while the copies are in flight
  for (int y = tid; y < ypad; y += blockDim.x) {
    bool valid = y < a.Y;
    if (valid && a.mask) valid = a.mask[(int64_t)b * a.sMb + (int64_t)y * a.sMy] != 0.f;
    maskadd[y] = valid ? 0.f : NEG_INF_F;
  }
  __syncthreads();
  if (tid == 0) {
    // S = Q K^T
    if (mbar_wait(&bar_qk, 0, &s_abort)) {
      tc_fence_after();
      const uint32_t idesc = instr_desc(128, ypad, false, false);
#pragma unroll
      for (int ks = 0; ks < AT_C / 16; ++ks) {
        const uint64_t qd = smem_desc(base + AT_Q_OFF + ks * 32, 16, 512, 4);
        const uint64_t kd = smem_desc(base + AT_K_OFF + ks * 32, 16, 512, 4);
        mma_ss(tmem, qd, kd, idesc, ks > 0 ? 1u : 0u);
      }
      mma_commit(&bar_s);
      s_issued = true;
    }
  }
  const int row = quarter * 32 + lane;  // query row within the tile (TMEM lane)
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  const float sl2 = a.scale * EVO_LOG2E;
  // tcgen05.ld / st are warp-collective: every decision that guards them is
  // made uniform across the warp
  bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_s, 0, &s_abort));
  tc_fence_after();

  // pass 1 over this warp's chunks: logits (log2 domain) in place, partial row
  // max; the TMEM load of the next chunk is in flight while this one is worked
  float mx = NEG_INF_F;
  uint32_t ra[32], rb[32];
  if (ok && c_lo < c_hi) {
    tmem_ld32_async(lane_base + (uint32_t)(c_lo * 32), ra);
    tmem_wait_ld(ra);
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int j = c_lo + t;
    if (j >= c_hi) break;
    uint32_t(&r)[32] = (t & 1) ? rb : ra;
    uint32_t(&nx)[32] = (t & 1) ? ra : rb;
    const int bx = t >> 1, hh = t & 1;  // box and its half holding chunk j
    if (A.has_bias && hh == 0) ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_b[warp][bx], 0, &s_abort));
    if (ok) bias_done = bx + 1;
    if (ok) {
      if (j + 1 < c_hi) tmem_ld32_async(lane_base + (uint32_t)((j + 1) * 32), nx);
      float v[32];
      const float4 *ma = reinterpret_cast<const float4 *>(maskadd + j * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 mv = ma[q];
        v[4 * q] = __uint_as_float(r[4 * q]) * sl2 + mv.x;
        v[4 * q + 1] = __uint_as_float(r[4 * q + 1]) * sl2 + mv.y;
        v[4 * q + 2] = __uint_as_float(r[4 * q + 2]) * sl2 + mv.z;
        v[4 * q + 3] = __uint_as_float(r[4 * q + 3]) * sl2 + mv.w;
      }
      if (A.has_bias) {
        // this lane's 128-byte row of the box (64 keys, 128-byte swizzle: 16-byte
        // piece k at k ^ (lane & 7)); chunk j is pieces 4 hh .. 4 hh + 3
        const uint32_t rbox = bring + bx * 4096u + lane * 128u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint4 w;
          asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                       : "r"(rbox + (uint32_t)(((4 * hh + k) ^ (lane & 7)) << 4)));
          const __nv_bfloat162 *hv = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(hv[q]);
            v[8 * k + 2 * q] = fmaf(f.x, EVO_LOG2E, v[8 * k + 2 * q]);
            v[8 * k + 2 * q + 1] = fmaf(f.y, EVO_LOG2E, v[8 * k + 2 * q + 1]);
          }
        }
      }
      uint32_t w32[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        mx = fmaxf(mx, v[jj]);
        w32[jj] = __float_as_uint(v[jj]);
      }
      tmem_st32(lane_base + (uint32_t)(j * 32), w32);
      if (j + 1 < c_hi) tmem_wait_ld(nx);
    }
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");  // nothing left in flight after an abort
  red[half * AT_QROWS + row] = mx;
  tmem_wait_st();
  __syncthreads();
  mx = fmaxf(red[row], red[AT_QROWS + row]);

  // pass 2: P = 2^(logit - max) of this warp's chunks, held as bf16 pairs
  // until every warp has read its logits (P for chunk j lands in columns
  // [16j, 16j + 16), over logits of chunk j / 2, which may be the other warp's)
  const float muse = mx == NEG_INF_F ? 0.f : mx;
  float l = 0.f;
  uint32_t pk[4][16];
  if (ok && c_lo < c_hi) {
    tmem_ld32_async(lane_base + (uint32_t)(c_lo * 32), ra);
    tmem_wait_ld(ra);
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int j = c_lo + t;
    if (ok && j < c_hi) {
      uint32_t(&r)[32] = (t & 1) ? rb : ra;
      uint32_t(&nx)[32] = (t & 1) ? ra : rb;
      if (j + 1 < c_hi) tmem_ld32_async(lane_base + (uint32_t)((j + 1) * 32), nx);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float p0 = ex2(__uint_as_float(r[2 * i]) - muse);
        const float p1 = ex2(__uint_as_float(r[2 * i + 1]) - muse);
        l += p0 + p1;
        __nv_bfloat162 hv = __floats2bfloat162_rn(p0, p1);
        pk[t][i] = *reinterpret_cast<uint32_t *>(&hv);
      }
      if (j + 1 < c_hi) tmem_wait_ld(nx);
    }
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  red[2 * AT_QROWS + half * AT_QROWS + row] = l;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int j = c_lo + t;
    if (ok && j < c_hi) tmem_st16(lane_base + (uint32_t)(j * 16), pk[t]);
  }
  l = red[2 * AT_QROWS + row] + red[3 * AT_QROWS + row];
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();

  if (tid == 0 && ok && !s_abort) {
    // O = P V
    tc_fence_after();
    if (mbar_wait(&bar_v, 0, &s_abort)) {
      const uint32_t idesc = instr_desc(128, AT_C, false, true);
      for (int ks = 0; ks < ypad / 16; ++ks) {
        const uint64_t vd = smem_desc(base + AT_V_OFF + ks * 1024, 16384, 512, 4);
        mma_ts(tmem + AT_O_COL, tmem + (uint32_t)(ks * 8), vd, idesc, ks > 0 ? 1u : 0u);
      }
      mma_commit(&bar_o);
      o_issued = true;
    }
  }
  // epilogue: the two warps of a quarter take 16 output channels each; the
  // gate row is requested before the wait for O
  const int x = x0 + row;
  const int c = a.c, d0 = half * 16;
  const bool mine = d0 < c;  // this warp's 16 output channels hold any of the head's c
  uint4 gwv[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
  if (x < a.X && mine) {
    const bf16 *gp = (const bf16 *)a.g + (int64_t)b * a.sQb + (int64_t)x * a.sQx + h * c + d0;
    gwv[0] = *reinterpret_cast<const uint4 *>(gp);
    if (c - d0 > 8) gwv[1] = *reinterpret_cast<const uint4 *>(gp + 8);
  }
  __syncthreads();
  ok = __all_sync(0xffffffffu, ok && !s_abort && mbar_wait(&bar_o, 0, &s_abort));
  tc_fence_after();
  uint32_t r[16];
  if (ok) tmem_ld16(lane_base + AT_O_COL + (uint32_t)d0, r);
  if (ok && x < a.X) {
    const float inv = l > 0.f ? 1.f / l : 0.f;
    bf16 *op = (bf16 *)a.o_att + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * c + d0;
    bf16 *gop = (bf16 *)a.o_gate + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * c + d0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q * 8 >= c - d0) continue;  // channels past the head dim (none at c = 32)
      const uint4 gw = gwv[q];
      const bf16 *gh = reinterpret_cast<const bf16 *>(&gw);
      uint4 ow, gow;
      uint32_t *o32 = reinterpret_cast<uint32_t *>(&ow), *g32 = reinterpret_cast<uint32_t *>(&gow);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float v0 = __uint_as_float(r[q * 8 + 2 * i]) * inv;
        const float v1 = __uint_as_float(r[q * 8 + 2 * i + 1]) * inv;
        __nv_bfloat162 o2 = __floats2bfloat162_rn(v0, v1);
        __nv_bfloat162 g2 =
            __floats2bfloat162_rn(v0 * __bfloat162float(gh[2 * i]), v1 * __bfloat162float(gh[2 * i + 1]));
        o32[i] = *reinterpret_cast<uint32_t *>(&o2);
        g32[i] = *reinterpret_cast<uint32_t *>(&g2);
      }
      *reinterpret_cast<uint4 *>(op + q * 8) = ow;
      *reinterpret_cast<uint4 *>(gop + q * 8) = gow;
    }
    if (half == 0) a.lse2[((int64_t)b * a.H + h) * a.X + x] = l > 0.f ? muse + log2f(l) : POS_INF_F;
  }
  // drain (after an abort) anything still in flight before the CTA exits
  if (s_abort) {
    if (tid == 0) {
      mbar_drain(&bar_qk, 0);
      mbar_drain(&bar_v, 0);
      if (s_issued) mbar_drain(&bar_s, 0);
      if (o_issued) mbar_drain(&bar_o, 0);
    }
    if (lane == 0)
      for (int bx = bias_done; bx < bias_issued; ++bx) mbar_drain(&bar_b[warp][bx], 0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)AT_TMEM_COLS)
                 : "memory");
  }
}


// ------------------------------------------------------------------- forward
// Any number of keys, head dim c in {8, 16, 32}.  Persistent: two CTAs per
// SM, each looping over tiles of (128 queries, head, batch item).  The keys
// of a tile are streamed in blocks of 64 with an online softmax (the logits
// of a row never exist in full anywhere), and the blocks of all of a CTA's
// tiles form one stream, so the copies and MMAs of the next tile run under
// the softmax and epilogue of this one:
//   * warp SW (control): loads block G's K, V, pair-bias tile and key mask
//     into ring slot G % 3 (TMA for K, V at c = 32 and for the bias; its
//     lanes write the mask and, at c < 32, the zero-padded K / V rows, all
//     fetched into registers one block ahead so that no global load sits on
//     its path) and each tile's Q into one of four Q slots; lane 0 issues
//     S_G = Q K_G^T (M 128, N 64) into TMEM S buffer G % 2 and, once the
//     softmax warps have read S_G and written P_G into P buffer G % 2,
//     O += P_G V_G (A = P from TMEM; a tile's first block starts O afresh)
//     and at once S_{G+2} into the S buffer just read;
//   * the SW softmax warps (thread = query row = TMEM lane): with SW = 8,
//     warps w and w + 4 share a lane quarter and take 32 keys of each block
//     each, and the two warps of a row meet at a named barrier for the
//     block's row max; with SW = 4 (long key streams) one warp per lane
//     quarter takes all 64 keys and needs no exchange.  They form the
//     logits in the log2 domain (scale, pair bias, key mask), the block's
//     row max, the running max m and the partial sums l, and write
//     P = 2^(logit - m) as bf16 pairs into the P buffer.
//     m only moves when a block's row max exceeds it by more than 8 (so
//     P <= 2^8): then the accumulated O (its columns of the row, after the
//     last O += P V has finished) and l are rescaled, which after a tile's
//     first block happens rarely;
//   * tile epilogue: O / l, the sigmoid-gated copy (bf16; the gate row is
//     read at the start of the tile) and the row log-sum-exp (log2 domain;
//     +inf for a row with no valid key, whose output is 0).
// TMEM: 256 columns (S buffers [0, 64) and [64, 128), P buffers [128, 160)
// and [160, 192), O [192, 224)).  Ordering facts the waits rely on: the
// MMAs of the control lane complete in issue order, so S_{G+2} done means
// O += P_G V_G done (P buffer G % 2 may be rewritten), and a softmax warp at
// block G has S_G, so every product before P_{G-1} is done.  Every wait is
// bounded; a wait that runs out records EVO_ERR_TIMEOUT and the CTA drains
// what it put in flight and returns.
constexpr int FW_Q = 128;
constexpr int FW_KB = 64;
constexpr int FW_NS = 3;   // ring slots of key blocks
constexpr int FW_NQ = 4;   // Q slots (tiles of one key block still keep two S in flight)
constexpr int FW_SOFT_WARPS = 8;
constexpr int FW_THREADS = (FW_SOFT_WARPS + 1) * 32;
constexpr int FW_TMEM_COLS = 256;
constexpr int FW_P_COL = 128;
constexpr int FW_O_COL = 192;
constexpr float FW_RESCALE = 8.f;
// shared memory (offsets from a 1 KB aligned base): Q slots ([128 rows]
// [64 B], 64-byte swizzle); ring slots of K, V ([64 keys][64 B], 64-byte
// swizzle) and the bias tile ([128 rows][128 B], 128-byte swizzle); the
// additive key masks [3][64]; the row-max / row-sum exchange [4][128]
constexpr int FW_Q_OFF = 0;
constexpr int FW_SK = 0, FW_SV = FW_KB * 64, FW_SB = 2 * FW_KB * 64;
constexpr int FW_SLOT = FW_SB + FW_Q * FW_KB * 2;
constexpr int FW_RING_OFF = FW_NQ * FW_Q * 64;
constexpr int FW_M_OFF = FW_RING_OFF + FW_NS * FW_SLOT;
constexpr int FW_X_OFF = FW_M_OFF + FW_NS * FW_KB * 4;
constexpr int FW_SMEM = FW_X_OFF + 4 * FW_Q * 4 + 1024;
static_assert(FW_SMEM * 2 + 2048 <= 233472, "two CTAs per SM");

struct AttnFwdArgs {
  AttnArgs a;
  QkvPos pq, pk;  // q / k, v map dimension positions (TMA path)
  int tma_qkv;    // q, k, v by TMA (head dim 32); else the control warp loads rows
  int has_bias;
  int nb;         // key blocks of 64 per tile
  int nxt;        // query tiles per (head, batch item)
  int tiles;      // nxt * H * B1
};

// What the control warp fetches for one key block before it writes the
// block into its ring slot: the lane's two key-mask values and, without TMA,
// its pieces of the K and V rows.
struct FwFetch {
  float m[2];
  uint4 k[4], v[4];
};

// Rows [row0, row0 + nrows) of a q view into a 64-byte-swizzled tile (c / 8
// data pieces per row; rows at or past `valid` as zeros); the pieces past
// c / 8 are left as they are (zeroed once per CTA).
__device__ __forceinline__ void load_rows(uint32_t tile, const bf16 *src, int64_t stride, int row0, int nrows, int valid,
                                          int c, int lane) {
  const int per = c >> 3;
  for (int idx = lane; idx < nrows * per; idx += 32) {
    const int r = idx / per, q = idx - r * per;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (row0 + r < valid) v = *reinterpret_cast<const uint4 *>(src + (int64_t)(row0 + r) * stride + q * 8);
    sts128(tile + sw64_off(r, q), v);
  }
}

struct TileId {
  int x0, h, b;
};
__device__ __forceinline__ TileId tile_id(const AttnFwdArgs &A, int t) {
  TileId r;
  const int xt = t % A.nxt, rest = t / A.nxt;
  r.x0 = xt * FW_Q;
  r.h = rest % A.a.H;
  r.b = rest / A.a.H;
  return r;
}

template <int SW>
__global__ void __launch_bounds__((SW + 1) * 32, 2) attn_fwd_stream(const __grid_constant__ CUtensorMap tmQ,
                                                             const __grid_constant__ CUtensorMap tmK,
                                                             const __grid_constant__ CUtensorMap tmV,
                                                             const __grid_constant__ CUtensorMap tmB, AttnFwdArgs A) {
  pdl_trigger();
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar_q[FW_NQ], bar_full[FW_NS], bar_s[2], bar_p[2], bar_o[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  const AttnArgs &a = A.a;
  const uint32_t raw = smem_u32(dsm);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = dsm + (base - raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = A.nb, c = a.c;
  // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int ntile = blockIdx.x < A.tiles ? (A.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int NG = ntile * nb;  // key blocks of all of them, one stream

  if (threadIdx.x == 0) {
    for (int i = 0; i < FW_NQ; ++i) mbar_init(&bar_q[i], 1);
    for (int i = 0; i < FW_NS; ++i) mbar_init(&bar_full[i], 2);  // TMA bytes + the control warp's arrival
    for (int i = 0; i < 2; ++i)
      mbar_init(&bar_s[i], 1), mbar_init(&bar_p[i], SW), mbar_init(&bar_o[i], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)FW_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // global memory only from here on: wait for the kernels before this one
  pdl_wait();

  if (warp == SW) {
    // ------------------------------------------------------------ control warp
    const bool leader = lane == 0;
    const int per = c >> 3;  // 16-byte pieces of a K / V row
    bool ok = true;
    int loaded = 0, waited = 0;       // key blocks put in flight / seen complete
    int q_loaded = 0, q_waited = 0;   // tiles whose Q was put in flight / seen complete
    uint64_t *last_bar = nullptr;     // the last MMA commit and its phase
    uint32_t last_par = 0;
    if (!A.tma_qkv) {
      // the pieces past the head dim stay zero for every row of the Q and K / V slots
      for (int i = lane; i < FW_NQ * FW_Q * 4; i += 32)
        if ((i & 3) >= per) sts128(base + FW_Q_OFF + (i >> 9) * (FW_Q * 64) + sw64_off((i >> 2) & 127, i & 3),
                                   make_uint4(0, 0, 0, 0));
      for (int sl = 0; sl < FW_NS; ++sl)
        for (int i = lane; i < 2 * FW_KB * 4; i += 32) {
          const int r = (i >> 2) & (FW_KB - 1), q = i & 3, kv = i / (FW_KB * 4);
          if (q >= per) sts128(base + FW_RING_OFF + sl * FW_SLOT + kv * FW_SV + sw64_off(r, q), make_uint4(0, 0, 0, 0));
        }
    }
    // issue the global loads of block G (the values are used a block later)
    auto fetch = [&](int G, FwFetch &f, bool rows) {
      const TileId t = tile_id(A, (int)blockIdx.x + (G / nb) * (int)gridDim.x);
      const int j = G % nb;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int y = j * FW_KB + u * 32 + lane;
        f.m[u] = y < a.Y ? (a.mask ? a.mask[(int64_t)t.b * a.sMb + (int64_t)y * a.sMy] : 1.f) : 0.f;
      }
      if (rows && !A.tma_qkv) {
        const int64_t kvoff = (int64_t)t.b * a.sKb + (int64_t)t.h * c;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = lane + 32 * u, r = idx / per, q = idx - r * per, y = j * FW_KB + r;
          const bool in = u < 2 * per && y < a.Y;
          f.k[u] = in ? *reinterpret_cast<const uint4 *>((const bf16 *)a.k + kvoff + (int64_t)y * a.sKy + q * 8)
                      : make_uint4(0, 0, 0, 0);
          f.v[u] = in ? *reinterpret_cast<const uint4 *>((const bf16 *)a.v + kvoff + (int64_t)y * a.sKy + q * 8)
                      : make_uint4(0, 0, 0, 0);
        }
      }
    };
    // block G into its ring slot: TMA copies, then the fetched mask and rows
    auto store = [&](int G, const FwFetch &f) {
      const TileId t = tile_id(A, (int)blockIdx.x + (G / nb) * (int)gridDim.x);
      const int j = G % nb, sl = G % FW_NS;
      const uint32_t slot = base + FW_RING_OFF + sl * FW_SLOT;
      const uint32_t tx = (A.tma_qkv ? 2u * FW_KB * 64u : 0u) + (A.has_bias ? (uint32_t)(FW_Q * FW_KB * 2) : 0u);
      if (leader) {
        mbar_arrive_expect_tx(&bar_full[sl], tx);
        if (A.tma_qkv) {
          int cc[4];
          tile_coords(A.pk, j * FW_KB, t.h, t.b, cc);
          tma_load_4d(slot + FW_SK, &tmK, cc[0], cc[1], cc[2], cc[3], &bar_full[sl]);
          tma_load_4d(slot + FW_SV, &tmV, cc[0], cc[1], cc[2], cc[3], &bar_full[sl]);
        }
        if (A.has_bias) tma_load_3d(slot + FW_SB, &tmB, j * FW_KB, t.x0, t.h, &bar_full[sl]);
      }
      if (!A.tma_qkv) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < 2 * per) {
            const int idx = lane + 32 * u, r = idx / per, q = idx - r * per;
            sts128(slot + FW_SK + sw64_off(r, q), f.k[u]);
            sts128(slot + FW_SV + sw64_off(r, q), f.v[u]);
          }
        }
      }
      float *maskadd = reinterpret_cast<float *>(gbase + FW_M_OFF) + sl * FW_KB;
#pragma unroll
      for (int u = 0; u < 2; ++u) maskadd[u * 32 + lane] = f.m[u] != 0.f ? 0.f : NEG_INF_F;
      fence_proxy_async();  // the generic-proxy rows are read by the tensor cores
      __syncwarp();
      if (leader) mbar_arrive(&bar_full[sl]);
      ++loaded;
    };
    // Q of tile i into Q slot i % 4
    auto load_q = [&](int i) {
      const TileId t = tile_id(A, (int)blockIdx.x + i * (int)gridDim.x);
      const uint32_t qs = base + FW_Q_OFF + (uint32_t)((i % FW_NQ) * FW_Q * 64);
      if (A.tma_qkv) {
        if (leader) {
          int cc[4];
          mbar_arrive_expect_tx(&bar_q[i % FW_NQ], FW_Q * 64);
          tile_coords(A.pq, t.x0, t.h, t.b, cc);
          tma_load_4d(qs, &tmQ, cc[0], cc[1], cc[2], cc[3], &bar_q[i % FW_NQ]);
        }
      } else {
        load_rows(qs, (const bf16 *)a.q + (int64_t)t.b * a.sQb + (int64_t)t.h * c, a.sQx, t.x0, FW_Q, a.X, c, lane);
        fence_proxy_async();
        __syncwarp();
        if (leader) mbar_arrive(&bar_q[i % FW_NQ]);
      }
      ++q_loaded;
    };
    // S_G = Q K_G^T into buffer G % 2 (waits for the tile's Q at its first block)
    // every wait of the control warp is made warp-uniform: its lanes must take
    // the same path through the __syncwarp of store() and load_q()
    auto issue_s = [&](int G) {
      const int i = G / nb;
      if (G % nb == 0) {
        ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_q[i % FW_NQ], (uint32_t)((i / FW_NQ) & 1), &s_abort));
        if (ok) q_waited = i + 1;
      }
      ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_full[G % FW_NS], (uint32_t)((G / FW_NS) & 1), &s_abort));
      if (!ok) return;
      waited = G + 1;
      if (leader) {
        tc_fence_after();
        const uint32_t qs = base + FW_Q_OFF + (uint32_t)((i % FW_NQ) * FW_Q * 64);
        const uint32_t slot = base + FW_RING_OFF + (G % FW_NS) * FW_SLOT;
        const uint32_t idesc = instr_desc(128, FW_KB, false, false);
        for (int ks = 0; ks < (c + 15) / 16; ++ks) {
          const uint64_t qd = smem_desc(qs + ks * 32, 16, 512, 4);
          const uint64_t kd = smem_desc(slot + FW_SK + ks * 32, 16, 512, 4);
          mma_ss(tmem + (uint32_t)((G & 1) * FW_KB), qd, kd, idesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(&bar_s[G & 1]);
      }
      last_bar = &bar_s[G & 1];
      last_par = (uint32_t)((G >> 1) & 1);
    };

    {
      // the first ring slots and Q tiles: every mask load in flight before
      // any is stored (the rows of the untiled path are fetched block by block)
      float m0[FW_NS], m1[FW_NS];
#pragma unroll
      for (int G = 0; G < FW_NS; ++G) {
        FwFetch f;
        f.m[0] = f.m[1] = 0.f;
        if (G < NG) fetch(G, f, false);
        m0[G] = f.m[0], m1[G] = f.m[1];
      }
      for (int i = 0; i < FW_NQ && i < ntile; ++i) load_q(i);
#pragma unroll
      for (int G = 0; G < FW_NS; ++G) {
        if (G < NG) {
          FwFetch f;
          if (!A.tma_qkv) fetch(G, f, true);
          f.m[0] = m0[G], f.m[1] = m1[G];
          store(G, f);
        }
      }
    }
    FwFetch nxt;  // block FW_NS + (refills so far), fetched a block ahead
    if (FW_NS < NG) fetch(FW_NS, nxt, true);
    for (int G = 0; G < NG && G < 2 && ok; ++G) issue_s(G);
    for (int G = 0; G < NG && ok; ++G) {
      // the softmax warps have read S_G and written P_G (and rescaled O)
      ok = __all_sync(0xffffffffu, mbar_wait(&bar_p[G & 1], (uint32_t)((G >> 1) & 1), &s_abort));
      if (!ok) break;
      // every S up to S_G is done with its Q slot
      while (q_loaded < ntile && (q_loaded - FW_NQ) * nb + nb - 1 <= G) load_q(q_loaded);
      if (leader) {
        tc_fence_after();
        const uint32_t slot = base + FW_RING_OFF + (G % FW_NS) * FW_SLOT;
        const uint32_t idesc = instr_desc(128, AT_C, false, true);
        for (int ks = 0; ks < FW_KB / 16; ++ks) {
          const uint64_t vd = smem_desc(slot + FW_SV + ks * 1024, 16384, 512, 4);
          mma_ts(tmem + FW_O_COL, tmem + (uint32_t)(FW_P_COL + (G & 1) * (FW_KB / 2) + ks * 8), vd, idesc,
                 (G % nb > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(&bar_o[G & 1]);
      }
      last_bar = &bar_o[G & 1];
      last_par = (uint32_t)((G >> 1) & 1);
      if (G + 2 < NG) {
        issue_s(G + 2);  // into the S buffer the softmax warps have just read
        if (!ok) break;
      }
      if (G + FW_NS < NG) {
        // ring slot G % 3 is free once O += P_G V_G is done
        ok = __all_sync(0xffffffffu, mbar_wait(&bar_o[G & 1], (uint32_t)((G >> 1) & 1), &s_abort));
        if (!ok) break;
        store(G + FW_NS, nxt);
        if (G + FW_NS + 1 < NG) fetch(G + FW_NS + 1, nxt, true);
      }
    }
    if (s_abort && leader) {
      // drain what this CTA put in flight before its memory goes away
      for (int i = q_waited; i < q_loaded; ++i) mbar_drain(&bar_q[i % FW_NQ], (uint32_t)((i / FW_NQ) & 1));
      for (int G = waited; G < loaded; ++G) mbar_drain(&bar_full[G % FW_NS], (uint32_t)((G / FW_NS) & 1));
      if (last_bar) mbar_drain(last_bar, last_par);
    }
  } else if constexpr (SW == 4) {
    // ---------------------------------------- softmax warps, one per lane quarter
    // thread = query row, all 64 keys of a block: no exchange with a partner
    const int quarter = warp;
    const int row = quarter * 32 + lane;  // query row within the tile (TMEM lane)
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const float sl2 = a.scale * EVO_LOG2E;
    bool ok = true;
    for (int i = 0; i < ntile; ++i) {
      const TileId t = tile_id(A, (int)blockIdx.x + i * (int)gridDim.x);
      const int x = t.x0 + row;
      // the gate row of this tile, needed at its end
      uint4 gw[4] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0),
                     make_uint4(0, 0, 0, 0)};
      if (x < a.X) {
        const uint4 *gp =
            reinterpret_cast<const uint4 *>((const bf16 *)a.g + (int64_t)t.b * a.sQb + (int64_t)x * a.sQx + t.h * c);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q * 8 < c) gw[q] = gp[q];
      }
      float m_run = NEG_INF_F, l = 0.f;
      for (int j = 0; j < nb; ++j) {
        const int G = i * nb + j, sl = G % FW_NS;
        const uint32_t slot = base + FW_RING_OFF + sl * FW_SLOT;
        const uint32_t sbuf = lane_base + (uint32_t)((G & 1) * FW_KB);
        // tcgen05.ld / st are warp-collective: the guards around them are warp-uniform
        ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_s[G & 1], (uint32_t)((G >> 1) & 1), &s_abort));
        ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_full[sl], (uint32_t)((G / FW_NS) & 1), &s_abort));
        float v[64];
        float mloc = NEG_INF_F;
        if (ok) {
          tc_fence_after();
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            uint32_t r[32];
            tmem_ld32(sbuf + (uint32_t)(hf * 32), r);
            const float4 *ma = reinterpret_cast<const float4 *>(gbase + FW_M_OFF) + sl * (FW_KB / 4) + hf * 8;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 mv = ma[q];
              v[32 * hf + 4 * q] = fmaf(__uint_as_float(r[4 * q]), sl2, mv.x);
              v[32 * hf + 4 * q + 1] = fmaf(__uint_as_float(r[4 * q + 1]), sl2, mv.y);
              v[32 * hf + 4 * q + 2] = fmaf(__uint_as_float(r[4 * q + 2]), sl2, mv.z);
              v[32 * hf + 4 * q + 3] = fmaf(__uint_as_float(r[4 * q + 3]), sl2, mv.w);
            }
          }
          if (A.has_bias) {
            // this row's 128-byte line of the bias tile (64 keys; piece k at k ^ (row & 7))
            const uint32_t rb = slot + FW_SB + (uint32_t)row * 128u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const uint4 w = lds128(rb + (uint32_t)((k ^ (row & 7)) << 4));
              const __nv_bfloat162 *hv = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float2 f = __bfloat1622float2(hv[q]);
                v[8 * k + 2 * q] = fmaf(f.x, EVO_LOG2E, v[8 * k + 2 * q]);
                v[8 * k + 2 * q + 1] = fmaf(f.y, EVO_LOG2E, v[8 * k + 2 * q + 1]);
              }
            }
          }
#pragma unroll
          for (int k = 0; k < 64; ++k) mloc = fmaxf(mloc, v[k]);
          const bool need = m_run == NEG_INF_F ? mloc > NEG_INF_F : mloc > m_run + FW_RESCALE;
          if (__any_sync(0xffffffffu, need)) {
            float corr = 1.f;
            if (need) {
              corr = m_run == NEG_INF_F ? 0.f : ex2(m_run - mloc);
              m_run = mloc;
            }
            l *= corr;
            if (j > 0) {
              // O holds the tile's blocks before this one: rescale the row once their product is done
              ok = __all_sync(0xffffffffu,
                              mbar_wait(&bar_o[(G - 1) & 1], (uint32_t)(((G - 1) >> 1) & 1), &s_abort));
              if (ok) {
                tc_fence_after();
                uint32_t r[32];
                tmem_ld32(lane_base + FW_O_COL, r);
#pragma unroll
                for (int k = 0; k < 32; ++k) r[k] = __float_as_uint(__uint_as_float(r[k]) * corr);
                tmem_st32(lane_base + FW_O_COL, r);
              }
            }
          }
        }
        if (ok) {
          const float muse = m_run == NEG_INF_F ? 0.f : m_run;
          uint32_t pk[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float p0 = ex2(v[2 * k] - muse), p1 = ex2(v[2 * k + 1] - muse);
            l += p0 + p1;
            __nv_bfloat162 hv = __floats2bfloat162_rn(p0, p1);
            pk[k] = *reinterpret_cast<uint32_t *>(&hv);
          }
          // P buffer G % 2: its last reader, O += P_{G-2} V_{G-2}, finished before S_G did
          tmem_st32(lane_base + (uint32_t)(FW_P_COL + (G & 1) * (FW_KB / 2)), pk);
          tmem_wait_st();
          tc_fence_before();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_p[G & 1]);
      }
      // tile epilogue
      const int Glast = i * nb + nb - 1;
      ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_o[Glast & 1], (uint32_t)((Glast >> 1) & 1), &s_abort));
      if (ok) {
        tc_fence_after();
        uint32_t r[32];
        tmem_ld32(lane_base + FW_O_COL, r);
        if (x < a.X) {
          const float inv = l > 0.f ? 1.f / l : 0.f;
          bf16 *op = (bf16 *)a.o_att + (int64_t)t.b * a.sOb + (int64_t)x * a.sOx + t.h * c;
          bf16 *gop = (bf16 *)a.o_gate + (int64_t)t.b * a.sOb + (int64_t)x * a.sOx + t.h * c;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (q * 8 < c) {
              const __nv_bfloat162 *gh = reinterpret_cast<const __nv_bfloat162 *>(&gw[q]);
              uint4 ow, gow;
              uint32_t *o32 = reinterpret_cast<uint32_t *>(&ow), *g32 = reinterpret_cast<uint32_t *>(&gow);
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float v0 = __uint_as_float(r[q * 8 + 2 * k]) * inv;
                const float v1 = __uint_as_float(r[q * 8 + 2 * k + 1]) * inv;
                const float2 gf = __bfloat1622float2(gh[k]);
                __nv_bfloat162 o2 = __floats2bfloat162_rn(v0, v1);
                __nv_bfloat162 g2 = __floats2bfloat162_rn(v0 * gf.x, v1 * gf.y);
                o32[k] = *reinterpret_cast<uint32_t *>(&o2);
                g32[k] = *reinterpret_cast<uint32_t *>(&g2);
              }
              *reinterpret_cast<uint4 *>(op + q * 8) = ow;
              *reinterpret_cast<uint4 *>(gop + q * 8) = gow;
            }
          }
          a.lse2[((int64_t)t.b * a.H + t.h) * a.X + x] = l > 0.f ? m_run + log2f(l) : POS_INF_F;
        }
      }
    }
  } else {
    // ------------------------------------------------------------ softmax warps
    const int quarter = warp & 3, hf = warp >> 2;
    const int row = quarter * 32 + lane;  // query row within the tile (TMEM lane)
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    float *xmax = reinterpret_cast<float *>(gbase + FW_X_OFF);  // [2][128]
    float *lsum = xmax + 2 * FW_Q;                               // [2][128]
    const float sl2 = a.scale * EVO_LOG2E;
    const int d0 = hf * 16;  // this warp's 16 output channels
    const bool mine = d0 < c;
    bool ok = true;
    // Both warps of a lane quarter pass the named barriers of every block and
    // tile, so no early exit: after an abort the rest is skipped in place.
    for (int i = 0; i < ntile; ++i) {
      const TileId t = tile_id(A, (int)blockIdx.x + i * (int)gridDim.x);
      const int x = t.x0 + row;
      // the gate row of this tile, needed at its end
      uint4 gw[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
      if (x < a.X && mine) {
        const bf16 *gp = (const bf16 *)a.g + (int64_t)t.b * a.sQb + (int64_t)x * a.sQx + t.h * c + d0;
        gw[0] = *reinterpret_cast<const uint4 *>(gp);
        if (c - d0 > 8) gw[1] = *reinterpret_cast<const uint4 *>(gp + 8);
      }
      float m_run = NEG_INF_F, l = 0.f;
      for (int j = 0; j < nb; ++j) {
        const int G = i * nb + j, sl = G % FW_NS;
        const uint32_t slot = base + FW_RING_OFF + sl * FW_SLOT;
        const uint32_t sbuf = lane_base + (uint32_t)((G & 1) * FW_KB);
        // tcgen05.ld / st are warp-collective: the guards around them are warp-uniform
        ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_s[G & 1], (uint32_t)((G >> 1) & 1), &s_abort));
        ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_full[sl], (uint32_t)((G / FW_NS) & 1), &s_abort));
        float v[32];
        float mloc = NEG_INF_F;
        if (ok) {
          tc_fence_after();
          uint32_t r[32];
          tmem_ld32(sbuf + (uint32_t)(hf * 32), r);
          const float4 *ma = reinterpret_cast<const float4 *>(gbase + FW_M_OFF) + sl * (FW_KB / 4) + hf * 8;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 mv = ma[q];
            v[4 * q] = fmaf(__uint_as_float(r[4 * q]), sl2, mv.x);
            v[4 * q + 1] = fmaf(__uint_as_float(r[4 * q + 1]), sl2, mv.y);
            v[4 * q + 2] = fmaf(__uint_as_float(r[4 * q + 2]), sl2, mv.z);
            v[4 * q + 3] = fmaf(__uint_as_float(r[4 * q + 3]), sl2, mv.w);
          }
          if (A.has_bias) {
            // this row's 128-byte line of the bias tile (64 keys; piece k at k ^ (row & 7)); this warp's half
            const uint32_t rb = slot + FW_SB + (uint32_t)row * 128u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint4 w = lds128(rb + (uint32_t)(((4 * hf + k) ^ (row & 7)) << 4));
              const __nv_bfloat162 *hv = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float2 f = __bfloat1622float2(hv[q]);
                v[8 * k + 2 * q] = fmaf(f.x, EVO_LOG2E, v[8 * k + 2 * q]);
                v[8 * k + 2 * q + 1] = fmaf(f.y, EVO_LOG2E, v[8 * k + 2 * q + 1]);
              }
            }
          }
#pragma unroll
          for (int k = 0; k < 32; ++k) mloc = fmaxf(mloc, v[k]);
        }
        // the row's block max over both halves (the partner has read its
        // logits before it arrives here, so P may then land over them)
        xmax[hf * FW_Q + row] = mloc;
        asm volatile("bar.sync %0, %1;" ::"r"(1 + quarter), "r"(64) : "memory");
        mloc = fmaxf(mloc, xmax[(hf ^ 1) * FW_Q + row]);
        if (ok) {
          const bool need = m_run == NEG_INF_F ? mloc > NEG_INF_F : mloc > m_run + FW_RESCALE;
          if (__any_sync(0xffffffffu, need)) {
            float corr = 1.f;
            if (need) {
              corr = m_run == NEG_INF_F ? 0.f : ex2(m_run - mloc);
              m_run = mloc;
            }
            l *= corr;
            if (j > 0) {
              // O holds the tile's blocks before this one: rescale this warp's
              // 16 columns once their product is done
              ok = __all_sync(0xffffffffu,
                              mbar_wait(&bar_o[(G - 1) & 1], (uint32_t)(((G - 1) >> 1) & 1), &s_abort));
              if (ok) {
                tc_fence_after();
                uint32_t r[16];
                tmem_ld16(lane_base + FW_O_COL + (uint32_t)d0, r);
#pragma unroll
                for (int k = 0; k < 16; ++k) r[k] = __float_as_uint(__uint_as_float(r[k]) * corr);
                tmem_st16(lane_base + FW_O_COL + (uint32_t)d0, r);
              }
            }
          }
        }
        if (ok) {
          const float muse = m_run == NEG_INF_F ? 0.f : m_run;
          uint32_t pk[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float p0 = ex2(v[2 * k] - muse), p1 = ex2(v[2 * k + 1] - muse);
            l += p0 + p1;
            __nv_bfloat162 hv = __floats2bfloat162_rn(p0, p1);
            pk[k] = *reinterpret_cast<uint32_t *>(&hv);
          }
          // P buffer G % 2: its last reader, O += P_{G-2} V_{G-2}, finished before S_G did
          tmem_st16(lane_base + (uint32_t)(FW_P_COL + (G & 1) * (FW_KB / 2) + hf * 16), pk);
          tmem_wait_st();
          tc_fence_before();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_p[G & 1]);
        // the next block's max exchange reuses xmax: the partner must have read it
        asm volatile("bar.sync %0, %1;" ::"r"(1 + quarter), "r"(64) : "memory");
      }
      // tile epilogue: the partial sums meet (the block barriers above order
      // this exchange after the partner's read of the previous tile's)
      lsum[hf * FW_Q + row] = l;
      asm volatile("bar.sync %0, %1;" ::"r"(1 + quarter), "r"(64) : "memory");
      l += lsum[(hf ^ 1) * FW_Q + row];
      const int Glast = i * nb + nb - 1;
      ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_o[Glast & 1], (uint32_t)((Glast >> 1) & 1), &s_abort));
      if (ok) {
        tc_fence_after();
        uint32_t r[16];
        tmem_ld16(lane_base + FW_O_COL + (uint32_t)d0, r);
        if (x < a.X && mine) {
          const float inv = l > 0.f ? 1.f / l : 0.f;
          bf16 *op = (bf16 *)a.o_att + (int64_t)t.b * a.sOb + (int64_t)x * a.sOx + t.h * c + d0;
          bf16 *gop = (bf16 *)a.o_gate + (int64_t)t.b * a.sOb + (int64_t)x * a.sOx + t.h * c + d0;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            if (q * 8 < c - d0) {
              const __nv_bfloat162 *gh = reinterpret_cast<const __nv_bfloat162 *>(&gw[q]);
              uint4 ow, gow;
              uint32_t *o32 = reinterpret_cast<uint32_t *>(&ow), *g32 = reinterpret_cast<uint32_t *>(&gow);
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float v0 = __uint_as_float(r[q * 8 + 2 * k]) * inv;
                const float v1 = __uint_as_float(r[q * 8 + 2 * k + 1]) * inv;
                const float2 gf = __bfloat1622float2(gh[k]);
                __nv_bfloat162 o2 = __floats2bfloat162_rn(v0, v1);
                __nv_bfloat162 g2 = __floats2bfloat162_rn(v0 * gf.x, v1 * gf.y);
                o32[k] = *reinterpret_cast<uint32_t *>(&o2);
                g32[k] = *reinterpret_cast<uint32_t *>(&g2);
              }
              *reinterpret_cast<uint4 *>(op + q * 8) = ow;
              *reinterpret_cast<uint4 *>(gop + q * 8) = gow;
            }
          }
        }
        if (x < a.X && hf == 0)
          a.lse2[((int64_t)t.b * a.H + t.h) * a.X + x] = l > 0.f ? m_run + log2f(l) : POS_INF_F;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)FW_TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------------ backward
// One CTA of eight warps per (head, batch item), all X <= 256 queries and
// Y <= 256 keys; head dims 8 and 16 arrive zero-padded to 32 channels (the
// 32-channel TMA box fills past the head dim) and only the head's channels
// of the gradients are stored.  Query tiles of 128 (qt) and key halves of
// 128 (kh):
//   for kh: for qt:
//     S = Q_qt K_kh^T, dP = dO_qt V_kh^T                     (TMEM [0,128), [128,256))
//     P = 2^(logit - lse2), dS = P (dP - D)     thread = query row, two warps
//                                                per TMEM lane quarter on 64 keys each
//     P, dS (bf16) -> shared memory as the MN-major A operands of
//       dV_kh += P^T dO_qt, dK_kh += dS^T Q_qt                (TMEM [256,288), [288,320))
//     dS (bf16 pairs) -> TMEM [128,192) as the A operand of
//       dQ_qt += dS K_kh                                      (TMEM [320 + 32 qt, ...))
//     dbias[h][x][y] += dS (fp32 vector atomics, one warp per query row, read
//       back from the shared dS copy so that a warp covers 128 contiguous keys)
//   dK_kh, dV_kh -> k/v gradient rows (bf16); finally dQ -> q gradient rows.
// Logit scale: S holds raw q.k; dQ and dK carry the softmax scale.
constexpr int BT_TMEM_COLS = 512;
constexpr int BT_S_COL = 0, BT_DP_COL = 128, BT_DK_COL = 256, BT_DV_COL = 288, BT_DQ_COL = 320;
// dynamic shared memory (1 KB aligned base)
constexpr int BT_Q_OFF = 0;                      // 2 x [128 q][64 B]
constexpr int BT_DO_OFF = BT_Q_OFF + 2 * 8192;   // 2 x [128 q][64 B]
constexpr int BT_K_OFF = BT_DO_OFF + 2 * 8192;   // 2 x [128 keys][64 B]
constexpr int BT_V_OFF = BT_K_OFF + 2 * 8192;    // 2 x [128 keys][64 B]
constexpr int BT_P_OFF = BT_V_OFF + 2 * 8192;    // [2 kb][2 mc][64 q][128 B]  (P^T operand)
constexpr int BT_DS_OFF = BT_P_OFF + 32768;      // same layout (dS^T operand)
constexpr int BT_B_OFF = BT_DS_OFF + 32768;      // per warp 2 x [32 rows][32 keys] fp32
constexpr int BT_L_OFF = BT_B_OFF + AT_WARPS * 2 * 4096;  // lse2 [256], D [256], maskadd [256]
constexpr int BT_SMEM = BT_L_OFF + 3 * 256 * 4 + 1024;

struct AttnTcBwdArgs {
  AttnArgs a;
  QkvPos pq, pk, po;  // q (and g) / k, v / dO (and dog, o) map dimension positions
  int nq, nkh;        // query tiles of 128, key halves of 128
  int has_bias;
  int fused_gate;     // dO slots hold dog; g and o tiles are loaded too
};

// Byte offset of element (key, q) in a [2 key chunks][128 q][64 keys] bf16
// tile with the 128-byte swizzle: rows of 64 keys, one per query.  Read as
// P^T / dS^T (M = keys, K = queries) it is the MN-major operand of dV and
// dK (key chunks LBO = 16 KB apart); read as dS (M = queries, K = keys) it is
// the K-major operand of dQ (a 16-key k-step 32 bytes into a row).
__device__ __forceinline__ uint32_t ds_off(int key, int q) {
  const int mc = key >> 6, m = key & 63;
  return (uint32_t)(mc * 16384 + q * 128 + ((((m >> 3) ^ (q & 7)) & 7) << 4) + (m & 7) * 2);
}

__global__ void __launch_bounds__(AT_WARPS * 32, 1) attn_bwd_tc(const __grid_constant__ CUtensorMap tmQ,
                                                                const __grid_constant__ CUtensorMap tmK,
                                                                const __grid_constant__ CUtensorMap tmV,
                                                                const __grid_constant__ CUtensorMap tmO,
                                                                const __grid_constant__ CUtensorMap tmB,
                                                                const __grid_constant__ CUtensorMap tmG,
                                                                const __grid_constant__ CUtensorMap tmOa,
                                                                AttnTcBwdArgs A) {
  pdl_trigger();
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar_in, bar_sd, bar_mm, bar_b[AT_WARPS][2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  const AttnArgs &a = A.a;
  const uint32_t raw = smem_u32(dsm);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = dsm + (base - raw);
  float *lse_s = reinterpret_cast<float *>(gbase + BT_L_OFF);
  float *d_s = lse_s + 256;
  float *maskadd = lse_s + 512;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int quarter = warp & 3, half = warp >> 2;
  const int h = blockIdx.x, b = blockIdx.y;
  const int nq = A.nq, nkh = A.nkh;

  if (tid == 0) {
    mbar_init(&bar_in, 1);
    mbar_init(&bar_sd, 1);
    mbar_init(&bar_mm, 1);
    for (int w = 0; w < AT_WARPS; ++w) mbar_init(&bar_b[w][0], 1), mbar_init(&bar_b[w][1], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)BT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // global memory only from here on: wait for the kernels before this one
  pdl_wait();
  bool in_issued = false;
  int nsd = 0, nmm = 0;  // commits issued on bar_sd / bar_mm (thread 0)
  if (tid == 0) {
    int c[4];
    mbar_arrive_expect_tx(&bar_in, (uint32_t)(nq * (A.fused_gate ? 4 : 2) * 8192 + nkh * 2 * 8192));
    for (int qt = 0; qt < nq; ++qt) {
      tile_coords(A.pq, qt * 128, h, b, c);
      tma_load_4d(base + BT_Q_OFF + qt * 8192, &tmQ, c[0], c[1], c[2], c[3], &bar_in);
      if (A.fused_gate)  // the gate tile (q layout) waits in the P^T buffer
        tma_load_4d(base + BT_P_OFF + qt * 8192, &tmG, c[0], c[1], c[2], c[3], &bar_in);
      tile_coords(A.po, qt * 128, h, b, c);
      tma_load_4d(base + BT_DO_OFF + qt * 8192, &tmO, c[0], c[1], c[2], c[3], &bar_in);
      if (A.fused_gate)  // and the attention output tile in the dS^T buffer
        tma_load_4d(base + BT_DS_OFF + qt * 8192, &tmOa, c[0], c[1], c[2], c[3], &bar_in);
    }
    for (int kh = 0; kh < nkh; ++kh) {
      tile_coords(A.pk, kh * 128, h, b, c);
      tma_load_4d(base + BT_K_OFF + kh * 8192, &tmK, c[0], c[1], c[2], c[3], &bar_in);
      tma_load_4d(base + BT_V_OFF + kh * 8192, &tmV, c[0], c[1], c[2], c[3], &bar_in);
    }
    in_issued = true;
  }
  // row statistics of the forward (padding rows get lse2 = +inf: P = 0) and the key mask
  for (int i = tid; i < 256; i += blockDim.x) {
    const bool xin = i < a.X;
    lse_s[i] = xin ? a.lse2[((int64_t)b * a.H + h) * a.X + i] : POS_INF_F;
    d_s[i] = xin && !A.fused_gate ? a.Dsum[((int64_t)b * a.H + h) * a.X + i] : 0.f;
    bool valid = i < a.Y;
    if (valid && a.mask) valid = a.mask[(int64_t)b * a.sMb + (int64_t)i * a.sMy] != 0.f;
    maskadd[i] = valid ? 0.f : NEG_INF_F;
  }
  __syncthreads();
  bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_in, 0, &s_abort));
  if (A.fused_gate) {
    // thread = query row x = tid (X <= 256): do_att = dog * g in place of dog,
    // D = sum_c do_att * o, dgpre = dog * o * g (1 - g); rows of 64 B with the
    // 64-byte swizzle (16-byte piece j of row r at j ^ ((r >> 1) & 3))
    const int qt = tid >> 7, r = tid & 127, x = tid;
    if (ok && qt < nq) {
      const uint32_t rowb = (uint32_t)(qt * 8192 + r * 64);
      float dsum = 0.f;
      uint4 dgw[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t off = rowb + (uint32_t)((j ^ ((r >> 1) & 3)) << 4);
        uint4 wdog, wg, wo;
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(wdog.x), "=r"(wdog.y), "=r"(wdog.z), "=r"(wdog.w) : "r"(base + BT_DO_OFF + off));
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(wg.x), "=r"(wg.y), "=r"(wg.z), "=r"(wg.w) : "r"(base + BT_P_OFF + off));
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(wo.x), "=r"(wo.y), "=r"(wo.z), "=r"(wo.w) : "r"(base + BT_DS_OFF + off));
        const bf16 *hd = reinterpret_cast<const bf16 *>(&wdog), *hg = reinterpret_cast<const bf16 *>(&wg),
                   *ho = reinterpret_cast<const bf16 *>(&wo);
        uint4 wa;
        uint32_t *pa = reinterpret_cast<uint32_t *>(&wa), *pg = reinterpret_cast<uint32_t *>(&dgw[j]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float d0 = __bfloat162float(hd[2 * i]), d1 = __bfloat162float(hd[2 * i + 1]);
          const float g0 = __bfloat162float(hg[2 * i]), g1 = __bfloat162float(hg[2 * i + 1]);
          const float o0 = __bfloat162float(ho[2 * i]), o1 = __bfloat162float(ho[2 * i + 1]);
          const float a0 = d0 * g0, a1 = d1 * g1;
          dsum += a0 * o0 + a1 * o1;
          __nv_bfloat162 va = __floats2bfloat162_rn(a0, a1);
          __nv_bfloat162 vg = __floats2bfloat162_rn(d0 * o0 * g0 * (1.f - g0), d1 * o1 * g1 * (1.f - g1));
          pa[i] = *reinterpret_cast<uint32_t *>(&va);
          pg[i] = *reinterpret_cast<uint32_t *>(&vg);
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + BT_DO_OFF + off), "r"(wa.x), "r"(wa.y),
                     "r"(wa.z), "r"(wa.w)
                     : "memory");
      }
      if (x < a.X) {
        d_s[x] = dsum;
        bf16 *gp = (bf16 *)a.dgpre + (int64_t)b * a.sQb + (int64_t)x * a.sQx + h * a.c;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (8 * j < a.c) *reinterpret_cast<uint4 *>(gp + 8 * j) = dgw[j];
      }
    }
    // do_att is read by the tensor cores (async proxy) and D by every row below
    fence_proxy_async();
    __syncthreads();
  }
  const float sl2 = a.scale * EVO_LOG2E;
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  const uint32_t bring = base + BT_B_OFF + (uint32_t)warp * 2 * 4096u;
  int bias_issued = 0, bias_done = 0;

  const int nit = nkh * nq;  // sub-tiles
  // S = Q_qt K_kh^T and dP = dO_qt V_kh^T of sub-tile `it` (thread 0)
  auto issue_sdp = [&](int it) {
    const int kh = it / nq, qt = it - kh * nq;
    tc_fence_after();
    const uint32_t idesc = instr_desc(128, 128, false, false);
#pragma unroll
    for (int ks = 0; ks < AT_C / 16; ++ks) {
      const uint64_t qd = smem_desc(base + BT_Q_OFF + qt * 8192 + ks * 32, 16, 512, 4);
      const uint64_t kd = smem_desc(base + BT_K_OFF + kh * 8192 + ks * 32, 16, 512, 4);
      mma_ss(tmem + BT_S_COL, qd, kd, idesc, ks > 0 ? 1u : 0u);
    }
#pragma unroll
    for (int ks = 0; ks < AT_C / 16; ++ks) {
      const uint64_t od = smem_desc(base + BT_DO_OFF + qt * 8192 + ks * 32, 16, 512, 4);
      const uint64_t vd = smem_desc(base + BT_V_OFF + kh * 8192 + ks * 32, 16, 512, 4);
      mma_ss(tmem + BT_DP_COL, od, vd, idesc, ks > 0 ? 1u : 0u);
    }
    mma_commit(&bar_sd);
    ++nsd;
  };
  // this warp's pair-bias box of sub-tile `it` (its 32 query rows x its 64
  // keys, bf16) into its ring slot it % 2 (lane 0)
  auto issue_bias = [&](int it) {
    const int kh = it / nq, qt = it - kh * nq;
    mbar_arrive_expect_tx(&bar_b[warp][it & 1], 4096);
    tma_load_3d(bring + (uint32_t)(it & 1) * 4096u, &tmB, kh * 128 + half * 64, qt * 128 + quarter * 32, h,
                &bar_b[warp][it & 1]);
    ++bias_issued;
  };
  if (a.bias && lane == 0 && ok)
    for (int it = 0; it < 2 && it < nit; ++it) issue_bias(it);
  if (tid == 0 && ok && !s_abort) issue_sdp(0);

  for (int kh = 0; kh < nkh; ++kh) {
    for (int qt = 0; qt < nq; ++qt) {
      const int it = kh * nq + qt;  // sub-tile counter (barrier phases)
      ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_sd, (uint32_t)(it & 1), &s_abort));
      tc_fence_after();
      const int row = quarter * 32 + lane;  // query row in the tile
      const int xq = qt * 128 + row;
      const float lse = lse_s[xq < 256 ? xq : 255], dd = d_s[xq < 256 ? xq : 255];
      // this warp's two 32-key chunks: the TMEM loads of the second are in
      // flight while the first is worked
      uint32_t sa[32], pa[32], sb[32], pb[32];
      if (a.bias) ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_b[warp][it & 1], (uint32_t)((it >> 1) & 1), &s_abort));
      if (ok && a.bias) bias_done = it + 1;
      if (ok) {
        tmem_ld32_async(lane_base + BT_S_COL + (uint32_t)(half * 64), sa);
        tmem_ld32_async(lane_base + BT_DP_COL + (uint32_t)(half * 64), pa);
        tmem_wait_ld(sa);
        tmem_wait_ld(pa);
      }
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int cl = half * 2 + t;           // 32-key chunk within the key half
        const int y0 = kh * 128 + cl * 32;     // first key of the chunk
        if (ok) {
          uint32_t(&sr)[32] = t ? sb : sa;
          uint32_t(&pr)[32] = t ? pb : pa;
          if (t == 0) {
            tmem_ld32_async(lane_base + BT_S_COL + (uint32_t)(cl * 32 + 32), sb);
            tmem_ld32_async(lane_base + BT_DP_COL + (uint32_t)(cl * 32 + 32), pb);
          }
          float bv[32];
          if (a.bias) {
            // pieces 4t .. 4t + 3 of this lane's 128-byte (64-key) row, 128-byte swizzle
            const uint32_t rb = bring + (uint32_t)(it & 1) * 4096u + lane * 128u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              uint4 w;
              asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                           : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                           : "r"(rb + (uint32_t)(((4 * t + k) ^ (lane & 7)) << 4)));
              const bf16 *hv = reinterpret_cast<const bf16 *>(&w);
#pragma unroll
              for (int q = 0; q < 8; ++q) bv[8 * k + q] = __bfloat162float(hv[q]);
            }
          } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) bv[k] = 0.f;
          }
          float p[32], ds[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float lg = fmaf(__uint_as_float(sr[k]), sl2, fmaf(bv[k], EVO_LOG2E, maskadd[y0 + k]));
            p[k] = ex2(lg - lse);
            ds[k] = p[k] * (__uint_as_float(pr[k]) - dd);
          }
          // P and dS into the operand tiles (element (key, query) at ds_off)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t wp[4], wd[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              __nv_bfloat162 a2 = __floats2bfloat162_rn(p[8 * j + 2 * i], p[8 * j + 2 * i + 1]);
              __nv_bfloat162 d2 = __floats2bfloat162_rn(ds[8 * j + 2 * i], ds[8 * j + 2 * i + 1]);
              wp[i] = *reinterpret_cast<uint32_t *>(&a2);
              wd[i] = *reinterpret_cast<uint32_t *>(&d2);
            }
            const uint32_t off = ds_off(cl * 32 + 8 * j, row);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + BT_P_OFF + off), "r"(wp[0]),
                         "r"(wp[1]), "r"(wp[2]), "r"(wp[3])
                         : "memory");
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + BT_DS_OFF + off), "r"(wd[0]),
                         "r"(wd[1]), "r"(wd[2]), "r"(wd[3])
                         : "memory");
          }
          if (t == 0) {
            tmem_wait_ld(sb);
            tmem_wait_ld(pb);
          }
        }
      }
      // every warp has read S and dP and written its P / dS rows (read by the
      // tensor cores: async proxy); the next pair-bias box may reuse the slot
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      if (a.bias && lane == 0 && ok && it + 2 < nit) issue_bias(it + 2);
      if (tid == 0 && ok && !s_abort) {
        tc_fence_after();
        const uint32_t id_kv = instr_desc(128, AT_C, true, true);   // A = P^T / dS^T (MN-major), B = dO / Q (MN-major)
        const uint32_t id_q = instr_desc(128, AT_C, false, true);   // A = dS (K-major), B = K (MN-major)
        for (int ks = 0; ks < 8; ++ks) {
          const uint64_t pd = smem_desc(base + BT_P_OFF + ks * 2048, 16384, 1024, 2);
          const uint64_t dsd = smem_desc(base + BT_DS_OFF + ks * 2048, 16384, 1024, 2);
          const uint64_t dsk = smem_desc(base + BT_DS_OFF + (ks >> 2) * 16384 + (ks & 3) * 32, 16, 1024, 2);
          const uint64_t od = smem_desc(base + BT_DO_OFF + qt * 8192 + ks * 1024, 16384, 512, 4);
          const uint64_t qd = smem_desc(base + BT_Q_OFF + qt * 8192 + ks * 1024, 16384, 512, 4);
          const uint64_t kd = smem_desc(base + BT_K_OFF + kh * 8192 + ks * 1024, 16384, 512, 4);
          const uint32_t acc_kv = (qt > 0 || ks > 0) ? 1u : 0u;
          mma_ss(tmem + BT_DV_COL, pd, od, id_kv, acc_kv);
          mma_ss(tmem + BT_DK_COL, dsd, qd, id_kv, acc_kv);
          mma_ss(tmem + BT_DQ_COL + (uint32_t)(qt * 32), dsk, kd, id_q, (kh > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(&bar_mm);
        ++nmm;
        // the next sub-tile's S and dP (their TMEM columns were read above;
        // the tensor cores run these after the products just issued)
        if (it + 1 < nit) issue_sdp(it + 1);
      }
      // pair-bias gradient from the shared dS copy: warp w takes query rows w, w + 8, ..
      if (a.dbias && ok) {
        for (int r = warp; r < 128; r += AT_WARPS) {
          const int x = qt * 128 + r;
          const int y = kh * 128 + lane * 4;
          if (x >= a.X || y >= a.Y) continue;
          const uint32_t off = ds_off(lane * 4, r);
          uint32_t w0, w1;
          asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(w0), "=r"(w1) : "r"(base + BT_DS_OFF + off));
          const float2 f0 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w0));
          const float2 f1 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w1));
          float *dst = a.dbias + (int64_t)h * a.sBh + (int64_t)x * a.sBx + y;
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(f0.x), "f"(f0.y), "f"(f1.x),
                       "f"(f1.y)
                       : "memory");
        }
      }
      ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_mm, (uint32_t)(it & 1), &s_abort));
      // every warp is done with this sub-tile's shared P / dS copies and TMEM
      // columns before the next sub-tile rewrites them
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
    // dK, dV of this key half: thread = key row, the two warps of a quarter take 16 channels each
    {
      const int y = kh * 128 + quarter * 32 + lane;
      uint32_t rk[16], rv[16];
      if (ok) {
        tmem_ld16(lane_base + BT_DK_COL + (uint32_t)(half * 16), rk);
        tmem_ld16(lane_base + BT_DV_COL + (uint32_t)(half * 16), rv);
      }
      if (ok && y < a.Y) {
        bf16 *dk = (bf16 *)a.dk + (int64_t)b * a.sKb + (int64_t)y * a.sKy + h * a.c + half * 16;
        bf16 *dv = (bf16 *)a.dv + (int64_t)b * a.sKb + (int64_t)y * a.sKy + h * a.c + half * 16;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (half * 16 + 8 * q >= a.c) continue;  // channels past the head dim
          uint4 wk, wv;
          uint32_t *k32 = reinterpret_cast<uint32_t *>(&wk), *v32 = reinterpret_cast<uint32_t *>(&wv);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 k2 = __floats2bfloat162_rn(__uint_as_float(rk[8 * q + 2 * i]) * a.scale,
                                                      __uint_as_float(rk[8 * q + 2 * i + 1]) * a.scale);
            __nv_bfloat162 v2 =
                __floats2bfloat162_rn(__uint_as_float(rv[8 * q + 2 * i]), __uint_as_float(rv[8 * q + 2 * i + 1]));
            k32[i] = *reinterpret_cast<uint32_t *>(&k2);
            v32[i] = *reinterpret_cast<uint32_t *>(&v2);
          }
          *reinterpret_cast<uint4 *>(dk + 8 * q) = wk;
          *reinterpret_cast<uint4 *>(dv + 8 * q) = wv;
        }
      }
      tc_fence_before();
      __syncthreads();  // the next key half restarts the dK / dV accumulators
      tc_fence_after();
    }
  }
  // dQ of every query tile
  for (int qt = 0; qt < nq; ++qt) {
    const int x = qt * 128 + quarter * 32 + lane;
    uint32_t rq[16];
    if (ok) tmem_ld16(lane_base + BT_DQ_COL + (uint32_t)(qt * 32 + half * 16), rq);
    if (ok && x < a.X) {
      bf16 *dq = (bf16 *)a.dq + (int64_t)b * a.sQb + (int64_t)x * a.sQx + h * a.c + half * 16;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (half * 16 + 8 * q >= a.c) continue;  // channels past the head dim
        uint4 w;
        uint32_t *w32 = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          __nv_bfloat162 q2 = __floats2bfloat162_rn(__uint_as_float(rq[8 * q + 2 * i]) * a.scale,
                                                    __uint_as_float(rq[8 * q + 2 * i + 1]) * a.scale);
          w32[i] = *reinterpret_cast<uint32_t *>(&q2);
        }
        *reinterpret_cast<uint4 *>(dq + 8 * q) = w;
      }
    }
  }
  // drain (after an abort) anything still in flight before the CTA exits
  if (s_abort) {
    if (tid == 0) {
      if (in_issued) mbar_drain(&bar_in, 0);
      for (int i = 0; i < nsd; ++i) mbar_drain(&bar_sd, (uint32_t)(i & 1));
      for (int i = 0; i < nmm; ++i) mbar_drain(&bar_mm, (uint32_t)(i & 1));
    }
    if (lane == 0)
      for (int j = bias_done; j < bias_issued; ++j) mbar_drain(&bar_b[warp][j & 1], (uint32_t)((j >> 1) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BT_TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------- backward, any length
// Any number of queries and keys, head dim c in {8, 16, 32} (rows zero-padded
// to 32 channels in shared memory).  One CTA of eight warps per (128-key
// block, head, batch item), looping over the query tiles of 128:
//   S = Q_t K^T, dP = dO_t V^T                                (TMEM [0,128), [128,256))
//   P = 2^(logit - lse2), dS = P (dP - D)     thread = query row, two warps
//                                              per TMEM lane quarter on 64 keys each
//   P, dS (bf16) -> shared memory (ds_off layout): the MN-major A operands of
//     dV += P^T dO_t, dK += dS^T Q_t                          (TMEM [256,288), [288,320))
//   and the K-major A operand of dQ_t = dS K                  (TMEM [320,352))
//   dQ_t is added into the fp32 dQ accumulator with vector atomics (every key
//   block of the row adds its share); dbias[h][x][y] += dS likewise.
// do_att (the gradient of the ungated output) and D = rowsum(do_att * o)
// come from the gate pass before this kernel.  The next tile's Q, dO (TMA,
// or at c < 32 rows fetched into registers a tile ahead) and the pair-bias
// boxes (per warp, two slots) are in flight while a tile is processed.
constexpr int BS_TMEM_COLS = 512;
constexpr int BS_S_COL = 0, BS_DP_COL = 128, BS_DK_COL = 256, BS_DV_COL = 288, BS_DQ_COL = 320;
// dynamic shared memory (1 KB aligned base)
constexpr int BS_K_OFF = 0;                               // [128 keys][64 B]
constexpr int BS_V_OFF = 8192;                            // [128 keys][64 B]
constexpr int BS_Q_OFF = 16384;                           // 2 x [128 q][64 B]
constexpr int BS_DO_OFF = BS_Q_OFF + 2 * 8192;            // 2 x [128 q][64 B]
constexpr int BS_P_OFF = BS_DO_OFF + 2 * 8192;            // [2 key chunks][128 q][128 B]
constexpr int BS_DS_OFF = BS_P_OFF + 32768;               // same layout
constexpr int BS_B_OFF = BS_DS_OFF + 32768;               // per warp 2 x [32 rows][64 keys] bf16
constexpr int BS_M_OFF = BS_B_OFF + AT_WARPS * 2 * 4096;  // maskadd [128]
constexpr int BS_SMEM = BS_M_OFF + 128 * 4 + 1024;

struct AttnBwdStreamArgs {
  AttnArgs a;
  QkvPos pq, pk, po;  // q / k, v / do_att map dimension positions (TMA path)
  int tma;            // q, k, v, do_att by TMA (head dim 32); else rows loaded by the threads
  int nq;             // query tiles of 128
  int has_bias;
};

__global__ void __launch_bounds__(AT_WARPS * 32, 1) attn_bwd_stream(const __grid_constant__ CUtensorMap tmQ,
                                                                    const __grid_constant__ CUtensorMap tmK,
                                                                    const __grid_constant__ CUtensorMap tmV,
                                                                    const __grid_constant__ CUtensorMap tmO,
                                                                    const __grid_constant__ CUtensorMap tmB,
                                                                    AttnBwdStreamArgs A) {
  pdl_trigger();
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bar_kv, bar_in[2], bar_sd, bar_mm, bar_b[AT_WARPS][2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  const AttnArgs &a = A.a;
  const uint32_t raw = smem_u32(dsm);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = dsm + (base - raw);
  float *maskadd = reinterpret_cast<float *>(gbase + BS_M_OFF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int quarter = warp & 3, half = warp >> 2;
  const int kb = blockIdx.x, h = blockIdx.y, b = blockIdx.z;
  const int y0 = kb * 128, nq = A.nq, c = a.c, per = c >> 3;

  if (tid == 0) {
    mbar_init(&bar_kv, 1);
    mbar_init(&bar_in[0], 1);
    mbar_init(&bar_in[1], 1);
    mbar_init(&bar_sd, 1);
    mbar_init(&bar_mm, 1);
    for (int w = 0; w < AT_WARPS; ++w) mbar_init(&bar_b[w][0], 1), mbar_init(&bar_b[w][1], 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)BS_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  pdl_wait();

  const int64_t qoff = (int64_t)b * a.sQb + (int64_t)h * c;   // q rows
  const int64_t ooff = (int64_t)b * a.sOb + (int64_t)h * c;   // do_att rows
  const int64_t koff = (int64_t)b * a.sKb + (int64_t)h * c;   // k, v rows
  int in_issued = 0, in_done = 0, bias_issued = 0, bias_done = 0;
  bool kv_issued = false;
  int nsd = 0, nmm = 0;
  // Q_t and dO_t into slot t % 2 (thread 0, TMA)
  auto issue_in = [&](int t) {
    int cc[4];
    mbar_arrive_expect_tx(&bar_in[t & 1], 2 * 8192);
    tile_coords(A.pq, t * 128, h, b, cc);
    tma_load_4d(base + BS_Q_OFF + (t & 1) * 8192, &tmQ, cc[0], cc[1], cc[2], cc[3], &bar_in[t & 1]);
    tile_coords(A.po, t * 128, h, b, cc);
    tma_load_4d(base + BS_DO_OFF + (t & 1) * 8192, &tmO, cc[0], cc[1], cc[2], cc[3], &bar_in[t & 1]);
    ++in_issued;
  };
  // this warp's pair-bias box of tile t (its 32 query rows x its 64 keys) into slot t % 2 (lane 0)
  const uint32_t bring = base + BS_B_OFF + (uint32_t)warp * 2 * 4096u;
  auto issue_bias = [&](int t) {
    mbar_arrive_expect_tx(&bar_b[warp][t & 1], 4096);
    tma_load_3d(bring + (uint32_t)(t & 1) * 4096u, &tmB, y0 + half * 64, t * 128 + quarter * 32, h,
                &bar_b[warp][t & 1]);
    ++bias_issued;
  };
  // rows of the untiled path: thread tid owns pieces tid and tid + 256 of a 128-row tile
  uint4 pq_reg[2], po_reg[2];
  auto fetch_in = [&](int t) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 256 * u, r = idx / per, q = idx - r * per, x = t * 128 + r;
      const bool in = idx < 128 * per && x < a.X;
      pq_reg[u] = in ? *reinterpret_cast<const uint4 *>((const bf16 *)a.q + qoff + (int64_t)x * a.sQx + q * 8)
                     : make_uint4(0, 0, 0, 0);
      po_reg[u] = in ? *reinterpret_cast<const uint4 *>((const bf16 *)a.do_att + ooff + (int64_t)x * a.sOx + q * 8)
                     : make_uint4(0, 0, 0, 0);
    }
  };
  auto store_in = [&](int t) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 256 * u, r = idx / per, q = idx - r * per;
      if (idx < 128 * per) {
        sts128(base + BS_Q_OFF + (t & 1) * 8192 + sw64_off(r, q), pq_reg[u]);
        sts128(base + BS_DO_OFF + (t & 1) * 8192 + sw64_off(r, q), po_reg[u]);
      }
    }
  };

  if (A.tma) {
    if (tid == 0) {
      int cc[4];
      mbar_arrive_expect_tx(&bar_kv, 2 * 8192);
      tile_coords(A.pk, y0, h, b, cc);
      tma_load_4d(base + BS_K_OFF, &tmK, cc[0], cc[1], cc[2], cc[3], &bar_kv);
      tma_load_4d(base + BS_V_OFF, &tmV, cc[0], cc[1], cc[2], cc[3], &bar_kv);
      kv_issued = true;
      issue_in(0);
      if (nq > 1) issue_in(1);
    }
  } else {
    // zero-padded rows: pieces past the head dim stay zero in every tile
    for (int i = tid; i < 128 * 4; i += blockDim.x) {
      const int r = i >> 2, q = i & 3;
      if (q >= per) {
        const uint4 z = make_uint4(0, 0, 0, 0);
        sts128(base + BS_K_OFF + sw64_off(r, q), z);
        sts128(base + BS_V_OFF + sw64_off(r, q), z);
        for (int sl = 0; sl < 2; ++sl) {
          sts128(base + BS_Q_OFF + sl * 8192 + sw64_off(r, q), z);
          sts128(base + BS_DO_OFF + sl * 8192 + sw64_off(r, q), z);
        }
      }
    }
    for (int idx = tid; idx < 128 * per; idx += blockDim.x) {
      const int r = idx / per, q = idx - r * per, y = y0 + r;
      uint4 kv = make_uint4(0, 0, 0, 0), vv = kv;
      if (y < a.Y) {
        kv = *reinterpret_cast<const uint4 *>((const bf16 *)a.k + koff + (int64_t)y * a.sKy + q * 8);
        vv = *reinterpret_cast<const uint4 *>((const bf16 *)a.v + koff + (int64_t)y * a.sKy + q * 8);
      }
      sts128(base + BS_K_OFF + sw64_off(r, q), kv);
      sts128(base + BS_V_OFF + sw64_off(r, q), vv);
    }
    fetch_in(0);
    store_in(0);
    if (nq > 1) fetch_in(1);
    fence_proxy_async();
    if (tid == 0) {
      mbar_arrive(&bar_kv);
      mbar_arrive(&bar_in[0]);
    }
  }
  if (a.bias && lane == 0)
    for (int t = 0; t < 2 && t < nq; ++t) issue_bias(t);
  // the key mask of the block
  if (tid < 128) {
    const int y = y0 + tid;
    bool valid = y < a.Y;
    if (valid && a.mask) valid = a.mask[(int64_t)b * a.sMb + (int64_t)y * a.sMy] != 0.f;
    maskadd[tid] = valid ? 0.f : NEG_INF_F;
  }
  __syncthreads();
  bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_kv, 0, &s_abort));

  const float sl2 = a.scale * EVO_LOG2E;
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  const int row = quarter * 32 + lane;  // query row in the tile (TMEM lane)
  float lse_n = POS_INF_F, d_n = 0.f;   // the row statistics of tile t, read a tile ahead
  if (row < a.X) {
    lse_n = a.lse2[((int64_t)b * a.H + h) * a.X + row];
    d_n = a.Dsum[((int64_t)b * a.H + h) * a.X + row];
  }

  for (int t = 0; t < nq; ++t) {
    const float lse = lse_n, dd = d_n;
    {
      const int xn = (t + 1) * 128 + row;
      lse_n = POS_INF_F, d_n = 0.f;
      if (t + 1 < nq && xn < a.X) {
        lse_n = a.lse2[((int64_t)b * a.H + h) * a.X + xn];
        d_n = a.Dsum[((int64_t)b * a.H + h) * a.X + xn];
      }
    }
    if (!A.tma && t > 0) {
      // this tile's rows, fetched during the last one, into its slot (free:
      // the last products that read it finished before the last tile ended)
      store_in(t);
      fence_proxy_async();
      __syncthreads();
      if (t + 1 < nq) fetch_in(t + 1);
      if (tid == 0) mbar_arrive(&bar_in[t & 1]);
    }
    if (tid == 0 && ok && !s_abort) {
      ok = mbar_wait(&bar_in[t & 1], (uint32_t)((t >> 1) & 1), &s_abort);
      if (ok) {
        in_done = t + 1;
        tc_fence_after();
        const uint32_t idesc = instr_desc(128, 128, false, false);
        for (int ks = 0; ks < (c + 15) / 16; ++ks) {
          const uint64_t qd = smem_desc(base + BS_Q_OFF + (t & 1) * 8192 + ks * 32, 16, 512, 4);
          const uint64_t kd = smem_desc(base + BS_K_OFF + ks * 32, 16, 512, 4);
          mma_ss(tmem + BS_S_COL, qd, kd, idesc, ks > 0 ? 1u : 0u);
        }
        for (int ks = 0; ks < (c + 15) / 16; ++ks) {
          const uint64_t od = smem_desc(base + BS_DO_OFF + (t & 1) * 8192 + ks * 32, 16, 512, 4);
          const uint64_t vd = smem_desc(base + BS_V_OFF + ks * 32, 16, 512, 4);
          mma_ss(tmem + BS_DP_COL, od, vd, idesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(&bar_sd);
        ++nsd;
      }
    }
    ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_sd, (uint32_t)(t & 1), &s_abort));
    tc_fence_after();
#pragma unroll
    for (int tt = 0; tt < 2; ++tt) {
      const int cl = half * 2 + tt;  // 32-key chunk of the block
      if (a.bias && tt == 0)
        ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_b[warp][t & 1], (uint32_t)((t >> 1) & 1), &s_abort));
      if (ok && a.bias) bias_done = t + 1;
      if (ok) {
        uint32_t sr[32], pr[32];
        tmem_ld32(lane_base + BS_S_COL + (uint32_t)(cl * 32), sr);
        tmem_ld32(lane_base + BS_DP_COL + (uint32_t)(cl * 32), pr);
        float bv[32];
        if (a.bias) {
          const uint32_t rb = bring + (uint32_t)(t & 1) * 4096u + lane * 128u;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint4 w = lds128(rb + (uint32_t)(((4 * tt + k) ^ (lane & 7)) << 4));
            const __nv_bfloat162 *hv = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float2 f = __bfloat1622float2(hv[q]);
              bv[8 * k + 2 * q] = f.x, bv[8 * k + 2 * q + 1] = f.y;
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k) bv[k] = 0.f;
        }
        float p[32], ds[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const float lg = fmaf(__uint_as_float(sr[k]), sl2, fmaf(bv[k], EVO_LOG2E, maskadd[cl * 32 + k]));
          p[k] = ex2(lg - lse);
          ds[k] = p[k] * (__uint_as_float(pr[k]) - dd);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint4 wp, wd;
          uint32_t *pp = reinterpret_cast<uint32_t *>(&wp), *pd = reinterpret_cast<uint32_t *>(&wd);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 a2 = __floats2bfloat162_rn(p[8 * j + 2 * i], p[8 * j + 2 * i + 1]);
            __nv_bfloat162 d2 = __floats2bfloat162_rn(ds[8 * j + 2 * i], ds[8 * j + 2 * i + 1]);
            pp[i] = *reinterpret_cast<uint32_t *>(&a2);
            pd[i] = *reinterpret_cast<uint32_t *>(&d2);
          }
          const uint32_t off = ds_off(cl * 32 + 8 * j, row);
          sts128(base + BS_P_OFF + off, wp);
          sts128(base + BS_DS_OFF + off, wd);
        }
      }
    }
    // every warp has read S and dP and written its P / dS rows (read by the
    // tensor cores: async proxy); the pair-bias slot of this tile is free
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (a.bias && lane == 0 && ok && t + 2 < nq) issue_bias(t + 2);
    if (tid == 0 && ok && !s_abort) {
      tc_fence_after();
      const uint32_t id_kv = instr_desc(128, AT_C, true, true);  // A = P^T / dS^T (MN-major), B = dO / Q (MN-major)
      const uint32_t id_q = instr_desc(128, AT_C, false, true);  // A = dS (K-major), B = K (MN-major)
      for (int ks = 0; ks < 8; ++ks) {
        const uint64_t pd = smem_desc(base + BS_P_OFF + ks * 2048, 16384, 1024, 2);
        const uint64_t dsd = smem_desc(base + BS_DS_OFF + ks * 2048, 16384, 1024, 2);
        const uint64_t dsk = smem_desc(base + BS_DS_OFF + (ks >> 2) * 16384 + (ks & 3) * 32, 16, 1024, 2);
        const uint64_t od = smem_desc(base + BS_DO_OFF + (t & 1) * 8192 + ks * 1024, 16384, 512, 4);
        const uint64_t qd = smem_desc(base + BS_Q_OFF + (t & 1) * 8192 + ks * 1024, 16384, 512, 4);
        const uint64_t kd = smem_desc(base + BS_K_OFF + ks * 1024, 16384, 512, 4);
        const uint32_t acc_kv = (t > 0 || ks > 0) ? 1u : 0u;
        mma_ss(tmem + BS_DV_COL, pd, od, id_kv, acc_kv);
        mma_ss(tmem + BS_DK_COL, dsd, qd, id_kv, acc_kv);
        mma_ss(tmem + BS_DQ_COL, dsk, kd, id_q, ks > 0 ? 1u : 0u);
      }
      mma_commit(&bar_mm);
      ++nmm;
    }
    // pair-bias gradient from the shared dS copy: warp w takes query rows w, w + 8, ..
    if (a.dbias && ok) {
      const bool vec = (a.Y & 3) == 0;
      for (int r = warp; r < 128; r += AT_WARPS) {
        const int x = t * 128 + r, y = y0 + lane * 4;
        if (x >= a.X || y >= a.Y) continue;
        uint32_t w0, w1;
        asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(w0), "=r"(w1) : "r"(base + BS_DS_OFF + ds_off(lane * 4, r)));
        const float2 f0 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w0));
        const float2 f1 = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w1));
        float *dst = a.dbias + (int64_t)h * a.sBh + (int64_t)x * a.sBx + y;
        if (vec) {
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(f0.x), "f"(f0.y), "f"(f1.x),
                       "f"(f1.y)
                       : "memory");
        } else {
          const float fv[4] = {f0.x, f0.y, f1.x, f1.y};
          for (int e = 0; e < 4 && y + e < a.Y; ++e) atomicAdd(dst + e, fv[e]);
        }
      }
    }
    ok = __all_sync(0xffffffffu, ok && mbar_wait(&bar_mm, (uint32_t)(t & 1), &s_abort));
    tc_fence_after();
    // dQ_t into the fp32 accumulator: thread = query row, the two warps of a quarter 16 channels each
    {
      const int x = t * 128 + row, d0 = half * 16;
      uint32_t rq[16];
      if (ok) tmem_ld16(lane_base + BS_DQ_COL + (uint32_t)d0, rq);
      if (ok && x < a.X && d0 < c) {
        float *dst = a.dq_acc + (int64_t)b * a.sOb + (int64_t)x * a.sOx + (int64_t)h * c + d0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (4 * q < c - d0)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * q),
                         "f"(__uint_as_float(rq[4 * q])), "f"(__uint_as_float(rq[4 * q + 1])),
                         "f"(__uint_as_float(rq[4 * q + 2])), "f"(__uint_as_float(rq[4 * q + 3]))
                         : "memory");
      }
    }
    // the next tile rewrites the shared P / dS copies, the TMEM S / dP / dQ
    // columns and this tile's Q, dO slot
    tc_fence_before();
    __syncthreads();
    if (A.tma && tid == 0 && ok && t + 2 < nq) issue_in(t + 2);
  }
  // dK, dV of the block: thread = key row, the two warps of a quarter take 16 channels each
  {
    const int y = y0 + quarter * 32 + lane, d0 = half * 16;
    uint32_t rk[16], rv[16];
    if (ok) {
      tmem_ld16(lane_base + BS_DK_COL + (uint32_t)d0, rk);
      tmem_ld16(lane_base + BS_DV_COL + (uint32_t)d0, rv);
    }
    if (ok && y < a.Y && d0 < c) {
      bf16 *dk = (bf16 *)a.dk + koff + (int64_t)y * a.sKy + d0;
      bf16 *dv = (bf16 *)a.dv + koff + (int64_t)y * a.sKy + d0;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (8 * q < c - d0) {
          uint4 wk, wv;
          uint32_t *k32 = reinterpret_cast<uint32_t *>(&wk), *v32 = reinterpret_cast<uint32_t *>(&wv);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 k2 = __floats2bfloat162_rn(__uint_as_float(rk[8 * q + 2 * i]) * a.scale,
                                                      __uint_as_float(rk[8 * q + 2 * i + 1]) * a.scale);
            __nv_bfloat162 v2 =
                __floats2bfloat162_rn(__uint_as_float(rv[8 * q + 2 * i]), __uint_as_float(rv[8 * q + 2 * i + 1]));
            k32[i] = *reinterpret_cast<uint32_t *>(&k2);
            v32[i] = *reinterpret_cast<uint32_t *>(&v2);
          }
          *reinterpret_cast<uint4 *>(dk + 8 * q) = wk;
          *reinterpret_cast<uint4 *>(dv + 8 * q) = wv;
        }
      }
    }
  }
  // drain (after an abort) anything still in flight before the CTA exits
  if (s_abort) {
    if (tid == 0) {
      if (kv_issued) mbar_drain(&bar_kv, 0);
      for (int i = in_done; i < in_issued; ++i) mbar_drain(&bar_in[i & 1], (uint32_t)((i >> 1) & 1));
      if (nmm > 0) mbar_drain(&bar_mm, (uint32_t)((nmm - 1) & 1));
      if (nsd > 0) mbar_drain(&bar_sd, (uint32_t)((nsd - 1) & 1));
    }
    if (lane == 0)
      for (int j = bias_done; j < bias_issued; ++j) mbar_drain(&bar_b[warp][j & 1], (uint32_t)((j >> 1) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BS_TMEM_COLS)
                 : "memory");
  }
}

// 4-D map of a q/k/v view: element (d, h, row, b) at base + b*s_b + row*s_row + h*c + d,
// outer dimensions ordered by stride (TMA takes them in any order; ascending
// strides keep every dimension's span inside the next stride).
bool qkv_map(CUtensorMap *tm, const void *base, int H, int rows, int B1, int64_t s_row, int64_t s_b, int box_rows,
             QkvPos *pos, int c = AT_C) {
  // head dim c <= 32: the box is 32 channels wide all the same, so a row
  // lands as 64 bytes with channels c..31 filled with zeros by the copy
  struct D {
    uint64_t n, stride;
    uint32_t box;
    int which;  // 0 row, 1 h, 2 b
  } ds[3] = {{(uint64_t)rows, (uint64_t)s_row, (uint32_t)box_rows, 0}, {(uint64_t)H, (uint64_t)c, 1, 1},
             {(uint64_t)B1, (uint64_t)s_b, 1, 2}};
  // extent-1 dimensions go last (their stride is never stepped); the rest by stride
  std::stable_sort(ds, ds + 3, [](const D &x, const D &y) {
    if ((x.n == 1) != (y.n == 1)) return y.n == 1;
    return x.stride < y.stride;
  });
  for (int i = 1; i < 3; ++i)
    if (ds[i].n == 1) ds[i].stride = std::max<uint64_t>(ds[i].stride, ds[i - 1].stride * ds[i - 1].n);
  uint64_t dims[4] = {(uint64_t)c, ds[0].n, ds[1].n, ds[2].n};
  uint64_t st[3] = {ds[0].stride * 2, ds[1].stride * 2, ds[2].stride * 2};
  uint32_t box[4] = {AT_C, ds[0].box, ds[1].box, ds[2].box};
  for (int i = 0; i < 3; ++i) {
    if (ds[i].stride % 8) return false;  // 16-byte strides
    if (i > 0 && ds[i].stride < ds[i - 1].stride * ds[i - 1].n) return false;
    if (ds[i].which == 0) pos->row = i + 1;
    else if (ds[i].which == 1) pos->h = i + 1;
    else pos->b = i + 1;
  }
  if (c <= 0 || c > AT_C || c % 8 || ds[0].stride < (uint64_t)c) return false;
  return make_tmap_nd(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, st, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

}  // namespace

bool attn_tc_supported(const AttnArgs &a) {
  auto a16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if ((a.c != 8 && a.c != 16 && a.c != 32) || a.Y <= 0 || a.X <= 0) return false;
  if (!a16(a.q) || !a16(a.k) || !a16(a.v) || !a16(a.g) || !a16(a.o_att) || !a16(a.o_gate)) return false;
  if (a.sOx % 8 || a.sOb % 8 || a.sQx % 8 || a.sQb % 8 || a.sKy % 8 || a.sKb % 8) return false;
  if (a.bias && (!a.bias_bf16 || !a16(a.bias) || a.sBx % 8 || a.sBh % 8 || a.sBx < a.Y ||
                 a.sBh < a.sBx * (int64_t)a.X))
    return false;
  return true;
}

namespace {

cudaError_t attn_fwd_short_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes) {
  AttnTcArgs A{};
  A.a = a;
  A.ypad = (a.Y + 31) / 32 * 32;
  A.has_bias = a.bias != nullptr;
  CUtensorMap tq, tk, tv, tb;
  std::memset(&tb, 0, sizeof(tb));
  QkvPos pv;
  if (!qkv_map(&tq, a.q, a.H, a.X, a.B1, a.sQx, a.sQb, AT_QROWS, &A.pq, a.c) ||
      !qkv_map(&tk, a.k, a.H, a.Y, a.B1, a.sKy, a.sKb, A.ypad, &A.pk, a.c) ||
      !qkv_map(&tv, a.v, a.H, a.Y, a.B1, a.sKy, a.sKb, A.ypad, &pv, a.c))
    return cudaErrorNotSupported;
  if (a.bias) {
    const uint64_t dims[3] = {(uint64_t)a.Y, (uint64_t)a.X, (uint64_t)a.H};
    const uint64_t st[2] = {(uint64_t)a.sBx * 2, (uint64_t)a.sBh * 2};
    const uint32_t box[3] = {64, 32, 1};
    if (!make_tmap_nd(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, a.bias, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorNotSupported;
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(attn_fwd_short, cudaFuncAttributeMaxDynamicSharedMemorySize, AT_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.X + AT_QROWS - 1) / AT_QROWS, a.H, a.B1);
  Prof p("attn_fwd_tc", s, flops, bytes);
  launch_k(attn_fwd_short, grid, AT_WARPS * 32, AT_SMEM, s, tq, tk, tv, tb, A);
  return cudaGetLastError();
}

cudaError_t attn_fwd_stream_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes) {
  AttnFwdArgs A{};
  A.a = a;
  A.nb = (a.Y + FW_KB - 1) / FW_KB;
  A.nxt = (a.X + FW_Q - 1) / FW_Q;
  const long long tiles = (long long)A.nxt * a.H * a.B1;
  if (tiles >= (1ll << 31)) return cudaErrorNotSupported;
  A.tiles = (int)tiles;
  A.has_bias = a.bias != nullptr;
  CUtensorMap tq, tk, tv, tb;
  std::memset(&tq, 0, sizeof(tq));
  std::memset(&tk, 0, sizeof(tk));
  std::memset(&tv, 0, sizeof(tv));
  std::memset(&tb, 0, sizeof(tb));
  // q, k, v by TMA where the views allow it (at head dims 8 and 16 the copy
  // fills channels c..31 of each 64-byte row with zeros); otherwise the
  // control warp loads the rows
  QkvPos pv;
  A.tma_qkv = qkv_map(&tq, a.q, a.H, a.X, a.B1, a.sQx, a.sQb, FW_Q, &A.pq, a.c) &&
              qkv_map(&tk, a.k, a.H, a.Y, a.B1, a.sKy, a.sKb, FW_KB, &A.pk, a.c) &&
              qkv_map(&tv, a.v, a.H, a.Y, a.B1, a.sKy, a.sKb, FW_KB, &pv, a.c);
  if (a.bias) {
    const uint64_t dims[3] = {(uint64_t)a.Y, (uint64_t)a.X, (uint64_t)a.H};
    const uint64_t st[2] = {(uint64_t)a.sBx * 2, (uint64_t)a.sBh * 2};
    const uint32_t box[3] = {FW_KB, FW_Q, 1};
    if (!make_tmap_nd(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, a.bias, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorNotSupported;
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(attn_fwd_stream<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // persistent: two CTAs per SM (TMEM, shared memory and registers allow two)
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<long long>(tiles, 2ll * sms);
  Prof p("attn_fwd_tc", s, flops, bytes);
  // long key streams (12 blocks of 64 or more) take one softmax warp per TMEM
  // lane quarter (a thread works all 64 keys of a block and needs no
  // partner's row max): 4 % faster at 2048 keys; shorter streams keep two
  // warps per quarter, whose extra warps hide more of the per-tile latency
  // (1.4 % faster at 384 keys)
  if (A.nb >= 12) {
    static bool attr4 = false;
    if (!attr4) {
      cudaError_t e = cudaFuncSetAttribute(attn_fwd_stream<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM);
      if (e != cudaSuccess) return e;
      attr4 = true;
    }
    launch_k(attn_fwd_stream<4>, grid, 5 * 32, FW_SMEM, s, tq, tk, tv, tb, A);
  } else {
    launch_k(attn_fwd_stream<8>, grid, FW_THREADS, FW_SMEM, s, tq, tk, tv, tb, A);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t attn_fwd_tc_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes) {
  // the training-crop shapes (head dim 32, at most 256 keys) take the
  // one-pass kernel when TMA can describe the views; everything else streams
  if (a.Y <= AT_MAXKEYS) {
    const cudaError_t e = attn_fwd_short_launch(a, s, flops, bytes);
    if (e != cudaErrorNotSupported) return e;
  }
  return attn_fwd_stream_launch(a, s, flops, bytes);
}

bool attn_bwd_tc_supported(const AttnArgs &a) {
  auto a16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (!attn_tc_supported(a) || a.Y > 256 || a.X > 256 || !a.dq || !a.dk || !a.dv) return false;
  if (!a16(a.dq) || !a16(a.dk) || !a16(a.dv) || a.sKy % 8 || a.sKb % 8) return false;
  if (a.dog ? (!a.dgpre || !a16(a.dog) || !a16(a.dgpre)) : (!a.do_att || !a.Dsum || !a16(a.do_att))) return false;
  if (a.bias && (!a.dbias || !a16(a.dbias) || a.Y % 4)) return false;
  return true;
}

cudaError_t attn_bwd_tc_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes) {
  AttnTcBwdArgs A{};
  A.a = a;
  A.nq = (a.X + 127) / 128;
  A.nkh = (a.Y + 127) / 128;
  A.has_bias = a.bias != nullptr;
  CUtensorMap tq, tk, tv, to, tb, tg, toa;
  std::memset(&tb, 0, sizeof(tb));
  std::memset(&tg, 0, sizeof(tg));
  std::memset(&toa, 0, sizeof(toa));
  QkvPos pv, px;
  A.fused_gate = a.dog != nullptr;
  if (!qkv_map(&tq, a.q, a.H, a.X, a.B1, a.sQx, a.sQb, 128, &A.pq, a.c)) return cudaErrorNotSupported;
  if (!qkv_map(&tk, a.k, a.H, a.Y, a.B1, a.sKy, a.sKb, 128, &A.pk, a.c)) return cudaErrorNotSupported;
  if (!qkv_map(&tv, a.v, a.H, a.Y, a.B1, a.sKy, a.sKb, 128, &pv, a.c)) return cudaErrorNotSupported;
  if (!qkv_map(&to, A.fused_gate ? a.dog : a.do_att, a.H, a.X, a.B1, a.sOx, a.sOb, 128, &A.po, a.c))
    return cudaErrorNotSupported;
  if (A.fused_gate) {
    if (!qkv_map(&tg, a.g, a.H, a.X, a.B1, a.sQx, a.sQb, 128, &px, a.c)) return cudaErrorNotSupported;
    if (!qkv_map(&toa, a.o_att, a.H, a.X, a.B1, a.sOx, a.sOb, 128, &px, a.c)) return cudaErrorNotSupported;
  }
  if (a.bias) {
    const uint64_t dims[3] = {(uint64_t)a.Y, (uint64_t)a.X, (uint64_t)a.H};
    const uint64_t st[2] = {(uint64_t)a.sBx * 2, (uint64_t)a.sBh * 2};
    const uint32_t box[3] = {64, 32, 1};
    if (!make_tmap_nd(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, a.bias, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorNotSupported;
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(attn_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(a.H, a.B1);
  Prof p("attn_bwd_tc", s, flops, bytes);
  launch_k(attn_bwd_tc, grid, AT_WARPS * 32, BT_SMEM, s, tq, tk, tv, to, tb, tg, toa, A);
  return cudaGetLastError();
}

namespace {
__global__ void attn_tc_debug_wait_kernel(int64_t limit_ns) {
  pdl_entry();
  debug_wait_body(limit_ns);
}
}  // namespace

cudaError_t attn_tc_debug_wait(int64_t limit_ns, cudaStream_t s) {
  launch_k(attn_tc_debug_wait_kernel, 1, 32, 0, s, limit_ns);
  return cudaGetLastError();
}

bool attn_bwd_stream_supported(const AttnArgs &a) {
  auto a16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (!attn_tc_supported(a) || !a.dq_acc || !a.dk || !a.dv || !a.do_att || !a.Dsum) return false;
  if (!a16(a.dq_acc) || !a16(a.dk) || !a16(a.dv) || !a16(a.do_att)) return false;
  if (a.bias && !a.dbias) return false;
  return a.Y <= 65535 * 128;
}

cudaError_t attn_bwd_stream_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes) {
  AttnBwdStreamArgs A{};
  A.a = a;
  A.nq = (a.X + 127) / 128;
  A.has_bias = a.bias != nullptr;
  CUtensorMap tq, tk, tv, to, tb;
  std::memset(&tq, 0, sizeof(tq));
  std::memset(&tk, 0, sizeof(tk));
  std::memset(&tv, 0, sizeof(tv));
  std::memset(&to, 0, sizeof(to));
  std::memset(&tb, 0, sizeof(tb));
  QkvPos pv;
  A.tma = a.c == AT_C && qkv_map(&tq, a.q, a.H, a.X, a.B1, a.sQx, a.sQb, 128, &A.pq) &&
          qkv_map(&tk, a.k, a.H, a.Y, a.B1, a.sKy, a.sKb, 128, &A.pk) &&
          qkv_map(&tv, a.v, a.H, a.Y, a.B1, a.sKy, a.sKb, 128, &pv) &&
          qkv_map(&to, a.do_att, a.H, a.X, a.B1, a.sOx, a.sOb, 128, &A.po);
  if (a.bias) {
    const uint64_t dims[3] = {(uint64_t)a.Y, (uint64_t)a.X, (uint64_t)a.H};
    const uint64_t st[2] = {(uint64_t)a.sBx * 2, (uint64_t)a.sBh * 2};
    const uint32_t box[3] = {64, 32, 1};
    if (!make_tmap_nd(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, a.bias, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorNotSupported;
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(attn_bwd_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, BS_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.Y + 127) / 128, a.H, a.B1);
  Prof p("attn_bwd_tc", s, flops, bytes);
  launch_k(attn_bwd_stream, grid, AT_WARPS * 32, BS_SMEM, s, tq, tk, tv, to, tb, A);
  return cudaGetLastError();
}

cudaError_t attn_tc_error_read_clear(int *out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, tc_error_word, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(tc_error_word, &zero, sizeof(int));
}

}  // namespace evo
