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

constexpr int AT_QROWS = 128;
constexpr int AT_C = 32;
constexpr int AT_MAXKEYS = 256;
constexpr int AT_TMEM_COLS = 256;
constexpr int AT_O_COL = 128;  // O accumulator columns [128, 160)
constexpr int AT_WARPS = 8;    // two per TMEM lane quarter, splitting the key chunks
// dynamic shared memory (offsets from a 1 KB aligned base)
constexpr int AT_Q_OFF = 0;                               // 128 x 64 B
constexpr int AT_K_OFF = AT_Q_OFF + AT_QROWS * 64;        // 256 x 64 B
constexpr int AT_V_OFF = AT_K_OFF + AT_MAXKEYS * 64;      // 256 x 64 B
// pair bias: per warp a ring of AT_BRING [32 rows x 32 keys] fp32 chunks (4 KB each)
constexpr int AT_BRING = 2;
constexpr int AT_B_OFF = AT_V_OFF + AT_MAXKEYS * 64;
constexpr int AT_R_OFF = AT_B_OFF + AT_WARPS * AT_BRING * 4096;  // [2][128] row max, [2][128] row sum
constexpr int AT_M_OFF = AT_R_OFF + 4 * AT_QROWS * 4;            // 256 floats: additive key mask
constexpr int AT_SMEM = AT_M_OFF + AT_MAXKEYS * 4 + 1024;

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

struct AttnTcArgs {
  AttnArgs a;
  QkvPos pq, pk;  // q (and g) / k, v map dimension positions
  int ypad;       // keys padded to a multiple of 32 (<= 256)
  int has_bias;
};

__device__ __forceinline__ void tile_coords(const QkvPos &p, int row, int h, int b, int (&c)[4]) {
  c[0] = 0;
  c[p.row] = row;
  c[p.h] = h;
  c[p.b] = b;
}

__global__ void __launch_bounds__(AT_WARPS * 32) attn_fwd_tc(const __grid_constant__ CUtensorMap tmQ,
                                                             const __grid_constant__ CUtensorMap tmK,
                                                             const __grid_constant__ CUtensorMap tmV,
                                                             const __grid_constant__ CUtensorMap tmB, AttnTcArgs A) {
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
  // what this thread put in flight (drained after an abort): lane 0 of each
  // warp streams the pair bias of its rows and chunks; thread 0 issues the rest
  int bias_issued = 0, bias_done = 0;
  bool s_issued = false, o_issued = false;
  const uint32_t bring = base + AT_B_OFF + (uint32_t)warp * AT_BRING * 4096u;
  auto bias_chunk = [&](int j) {  // lane 0: chunk j (keys 32j..) of this warp's rows, slot (j - c_lo) % ring
    const int k = (j - c_lo) % AT_BRING;
    mbar_arrive_expect_tx(&bar_b[warp][k], 4096);
    tma_load_3d(bring + k * 4096u, &tmB, j * 32, x0 + quarter * 32, h, &bar_b[warp][k]);
    ++bias_issued;
  };
  if (A.has_bias && lane == 0)
    for (int j = c_lo; j < c_hi && j < c_lo + AT_BRING; ++j) bias_chunk(j);

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

  // pass 1 over this warp's chunks: logits (log2 domain) in place, partial row max
  float mx = NEG_INF_F;
  for (int j = c_lo; j < c_hi; ++j) {
    const int sl = (j - c_lo) % AT_BRING;
    if (A.has_bias)
      ok = __all_sync(0xffffffffu,
                      ok && mbar_wait(&bar_b[warp][sl], (uint32_t)(((j - c_lo) / AT_BRING) & 1), &s_abort));
    if (ok) bias_done = j - c_lo + 1;
    if (ok) {
      uint32_t r[32];
      tmem_ld32(lane_base + (uint32_t)(j * 32), r);
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
        // this lane's row of the warp's 128-byte-swizzled chunk: 16-byte piece k at k ^ (lane & 7)
        const uint32_t rb = bring + sl * 4096u + lane * 128u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          float4 bv;
          asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                       : "=f"(bv.x), "=f"(bv.y), "=f"(bv.z), "=f"(bv.w)
                       : "r"(rb + (uint32_t)((k ^ (lane & 7)) << 4)));
          v[4 * k] = fmaf(bv.x, EVO_LOG2E, v[4 * k]);
          v[4 * k + 1] = fmaf(bv.y, EVO_LOG2E, v[4 * k + 1]);
          v[4 * k + 2] = fmaf(bv.z, EVO_LOG2E, v[4 * k + 2]);
          v[4 * k + 3] = fmaf(bv.w, EVO_LOG2E, v[4 * k + 3]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        mx = fmaxf(mx, v[jj]);
        r[jj] = __float_as_uint(v[jj]);
      }
      tmem_st32(lane_base + (uint32_t)(j * 32), r);
    }
    if (A.has_bias) {
      // the slot is refilled once the warp has read it
      __syncwarp();
      if (lane == 0 && ok && j + AT_BRING < c_hi) bias_chunk(j + AT_BRING);
    }
  }
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
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int j = c_lo + t;
    if (ok && j < c_hi) {
      uint32_t r[32];
      tmem_ld32(lane_base + (uint32_t)(j * 32), r);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float p0 = ex2(__uint_as_float(r[2 * i]) - muse);
        const float p1 = ex2(__uint_as_float(r[2 * i + 1]) - muse);
        l += p0 + p1;
        __nv_bfloat162 hv = __floats2bfloat162_rn(p0, p1);
        pk[t][i] = *reinterpret_cast<uint32_t *>(&hv);
      }
    }
  }
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
  const int d0 = half * 16;
  uint4 gwv[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
  if (x < a.X) {
    const bf16 *gp = (const bf16 *)a.g + (int64_t)b * a.sQb + (int64_t)x * a.sQx + h * AT_C + d0;
    gwv[0] = *reinterpret_cast<const uint4 *>(gp);
    gwv[1] = *reinterpret_cast<const uint4 *>(gp + 8);
  }
  __syncthreads();
  ok = __all_sync(0xffffffffu, ok && !s_abort && mbar_wait(&bar_o, 0, &s_abort));
  tc_fence_after();
  uint32_t r[16];
  if (ok) tmem_ld16(lane_base + AT_O_COL + (uint32_t)d0, r);
  if (ok && x < a.X) {
    const float inv = l > 0.f ? 1.f / l : 0.f;
    bf16 *op = (bf16 *)a.o_att + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * AT_C + d0;
    bf16 *gop = (bf16 *)a.o_gate + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * AT_C + d0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
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
      for (int j = bias_done; j < bias_issued; ++j)
        mbar_drain(&bar_b[warp][j % AT_BRING], (uint32_t)((j / AT_BRING) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)AT_TMEM_COLS)
                 : "memory");
  }
}

// 4-D map of a q/k/v view: element (d, h, row, b) at base + b*s_b + row*s_row + h*c + d,
// outer dimensions ordered by stride (TMA takes them in any order; ascending
// strides keep every dimension's span inside the next stride).
bool qkv_map(CUtensorMap *tm, const void *base, int H, int rows, int B1, int64_t s_row, int64_t s_b, int box_rows,
             QkvPos *pos) {
  struct D {
    uint64_t n, stride;
    uint32_t box;
    int which;  // 0 row, 1 h, 2 b
  } ds[3] = {{(uint64_t)rows, (uint64_t)s_row, (uint32_t)box_rows, 0}, {(uint64_t)H, AT_C, 1, 1},
             {(uint64_t)B1, (uint64_t)s_b, 1, 2}};
  // extent-1 dimensions go last (their stride is never stepped); the rest by stride
  std::stable_sort(ds, ds + 3, [](const D &x, const D &y) {
    if ((x.n == 1) != (y.n == 1)) return y.n == 1;
    return x.stride < y.stride;
  });
  for (int i = 1; i < 3; ++i)
    if (ds[i].n == 1) ds[i].stride = std::max<uint64_t>(ds[i].stride, ds[i - 1].stride * ds[i - 1].n);
  uint64_t dims[4] = {AT_C, ds[0].n, ds[1].n, ds[2].n};
  uint64_t st[3] = {ds[0].stride * 2, ds[1].stride * 2, ds[2].stride * 2};
  uint32_t box[4] = {AT_C, ds[0].box, ds[1].box, ds[2].box};
  for (int i = 0; i < 3; ++i) {
    if (ds[i].stride % 8) return false;  // 16-byte strides
    if (i > 0 && ds[i].stride < ds[i - 1].stride * ds[i - 1].n) return false;
    if (ds[i].which == 0) pos->row = i + 1;
    else if (ds[i].which == 1) pos->h = i + 1;
    else pos->b = i + 1;
  }
  if (ds[0].stride < AT_C) return false;
  return make_tmap_nd(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, st, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

}  // namespace

bool attn_tc_supported(const AttnArgs &a) {
  auto a16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (a.c != AT_C || a.Y <= 0 || a.Y > AT_MAXKEYS || a.X <= 0) return false;
  if (!a16(a.q) || !a16(a.k) || !a16(a.v) || !a16(a.g) || !a16(a.o_att) || !a16(a.o_gate)) return false;
  if (a.sOx % 8 || a.sOb % 8 || a.sQx % 8 || a.sQb % 8) return false;
  if (a.bias && (!a16(a.bias) || a.sBx % 4 || a.sBh % 4 || a.sBx < a.Y || a.sBh < a.sBx * (int64_t)a.X))
    return false;
  return true;
}

cudaError_t attn_fwd_tc_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes) {
  AttnTcArgs A{};
  A.a = a;
  A.ypad = (a.Y + 31) / 32 * 32;
  A.has_bias = a.bias != nullptr;
  CUtensorMap tq, tk, tv, tb;
  std::memset(&tb, 0, sizeof(tb));
  // views TMA cannot describe: the caller falls back to the mma.sync kernel
  if (!qkv_map(&tq, a.q, a.H, a.X, a.B1, a.sQx, a.sQb, AT_QROWS, &A.pq)) return cudaErrorNotSupported;
  if (!qkv_map(&tk, a.k, a.H, a.Y, a.B1, a.sKy, a.sKb, A.ypad, &A.pk)) return cudaErrorNotSupported;
  QkvPos pv;
  if (!qkv_map(&tv, a.v, a.H, a.Y, a.B1, a.sKy, a.sKb, A.ypad, &pv)) return cudaErrorNotSupported;
  if (a.bias) {
    const uint64_t dims[3] = {(uint64_t)a.Y, (uint64_t)a.X, (uint64_t)a.H};
    const uint64_t st[2] = {(uint64_t)a.sBx * 4, (uint64_t)a.sBh * 4};
    const uint32_t box[3] = {32, 32, 1};
    if (!make_tmap_nd(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.bias, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorNotSupported;
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(attn_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, AT_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.X + AT_QROWS - 1) / AT_QROWS, a.H, a.B1);
  Prof p("attn_fwd_tc", s, flops, bytes);
  attn_fwd_tc<<<grid, AT_WARPS * 32, AT_SMEM, s>>>(tq, tk, tv, tb, A);
  return cudaGetLastError();
}

cudaError_t attn_tc_error_read_clear(int *out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, tc_error_word, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(tc_error_word, &zero, sizeof(int));
}

}  // namespace evo
