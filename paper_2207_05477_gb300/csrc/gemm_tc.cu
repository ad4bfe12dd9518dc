// BF16 GEMM on the 5th-generation tensor cores (sm_103a): TMA loads 128x64 /
// BNx64 operand tiles (128-byte swizzle) into a STAGES-deep shared-memory ring,
// one elected thread issues tcgen05.mma (M=128, N=BN, K=16) accumulating FP32
// in tensor memory, and sixteen epilogue warps drain TMEM with tcgen05.ld
// through the shared epilogue (bias, scales, gates, residual, layout-changing
// stores).
//
// The kernel is persistent (one CTA per SM) and warp-specialised: lane 0 of
// warp 0 streams A/B k-tiles with TMA through a STAGES-deep ring, running
// ahead across output tiles; lane 0 of warp 1 issues the MMAs into one of two
// TMEM accumulators; warps 2-17 drain the other accumulator through the
// epilogue, so a tile's epilogue overlaps the next tile's loads and MMAs.
// The epilogue is latency-bound (few instructions per byte, each waiting on
// TMEM or global loads), hence four warps per TMEM lane quarter, each on
// 32-column chunks, with the row operands of a chunk (gate, residual, ReLU
// reference) requested before the accumulator wait.
//
// Operands may be K-major or MN-major (the transpose bits of the instruction
// descriptor); backward GEMMs (dX = dY W, dW = dY^T X) use MN-major views of
// the forward tensors instead of transposed copies.
//
// Every wait on an mbarrier is bounded (about one second of %globaltimer); a
// wait that runs out sets the library's device error word, the CTA drains its
// in-flight copies with bounded waits, frees its TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "tc.cuh"

namespace evo {

namespace {

using namespace tc;

constexpr int BM = 128, BK = 64;

// Persistent kernel configuration: a ring of A/B k-tiles, sixteen epilogue
// warps with a small shared-memory region each, and two TMEM accumulators of
// BN columns (tile i drains while tile i+1 accumulates).  The depth of the
// k-tile ring is chosen at launch: whatever shared memory the epilogue
// regions leave.
constexpr int EPI_WARPS = 16;  // four per TMEM lane quarter, 32-column slots at a 128-column stride
constexpr int MAX_STAGES = 6;
constexpr int SMEM_LIMIT = 232448;  // bytes of dynamic shared memory one CTA may use

template <int BN, bool AMN, bool BMN>
struct TcCfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;
  // A K-major tile: rows of 128 B, k-step of 16 elements = 32 B.
  // An MN-major tile: 64-element (128 B) MN chunks of 64 K-rows (8 KB each);
  // a k-step of 16 rows = 2 KB.
  static constexpr uint32_t A_KSTEP = AMN ? 2048u : 32u;
  static constexpr uint32_t B_KSTEP = BMN ? 2048u : 32u;
  static constexpr uint32_t A_LBO = AMN ? 8192u : 16u;
  static constexpr uint32_t B_LBO = BMN ? 8192u : 16u;
  static constexpr uint32_t IDESC = instr_desc(BM, BN, AMN, BMN);
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N");
  static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM columns");
};

// Epilogue region of one warp (1 KB aligned):
//   [0, 4 KB)    two 2 KB slots: the chunk's residual tile, loaded by TMA and
//                overwritten in place by the bf16 result the TMA store reads
//                (the output staging when there is no residual);
//   [4 KB, 8 KB) two 2 KB slots for the gate or ReLU-reference tile (only
//                when the epilogue has one);
//   the general path instead stages 32 x 33 floats from offset 0.
// Tiles are 32 rows x 64 B with the 64-byte swizzle.
__host__ __device__ constexpr int epi_warp_bytes(bool has_opa) { return has_opa ? 8192 : 5120; }

struct TcLaunch {
  int stages;     // depth of the k-tile ring
  int epi_bytes;  // per epilogue warp
  int tma_store;  // 0: general epilogue; 1: 3-D row-major map; 2, 3: 4-D two-level maps
  int has_opa;    // gate or ReLU reference tile loaded by TMA
  int has_res;    // residual tile loaded by TMA
};

struct TileCoord {
  int m0, n0, b, split, kt0, nk;
};

constexpr int EK_PLAIN = 0, EK_OPS = 1, EK_GENERAL = 2;

__device__ __forceinline__ TileCoord decode_tile(const GemmOp &g, int t, int bn) {
  const int ntn = (g.N + bn - 1) / bn, ntm = (g.M + BM - 1) / BM;
  TileCoord c;
  const int nn = t % ntn;
  int rest = t / ntn;
  const int mm = rest % ntm;
  rest /= ntm;
  c.b = rest / g.splits;
  c.split = rest % g.splits;
  c.m0 = mm * BM;
  c.n0 = nn * bn;
  const int kt_total = (g.K + BK - 1) / BK;
  const int per = (kt_total + g.splits - 1) / g.splits;
  c.kt0 = c.split * per;
  c.nk = max(0, min(kt_total, c.kt0 + per) - c.kt0);
  return c;
}

// General epilogue of one staged 32-row x 32-column chunk (rows mrow0..,
// columns nbase..): lane = column, rows in turn (split-K partials are plain
// coalesced fp32 rows; everything else goes through epi_store).
__device__ __forceinline__ void epi_chunk(const GemmOp &g, const float *mine, int lane, int mrow0, int nbase, int b,
                                          int split) {
  const Epi &e = g.e;
  if (e.atomic && e.map.mdiv >= (1ll << 31) && e.map.ndiv >= (1ll << 31) && e.map.s_n0 == 1 &&
      e.map.s_m0 % 4 == 0 && e.c_bstride % 4 == 0 && (((uintptr_t)e.C) & 15u) == 0) {
    // split-K partial products added into a row-major fp32 output with
    // 16-byte vector reductions: lane = (row r0 + lane / 8 + 4 i, columns
    // 4 (lane % 8) .. + 3), a quarter of the reduction requests of one per
    // element
    const int rq = lane >> 3, cq = lane & 7;
    const int n0 = nbase + 4 * cq;
    float *cbase = (float *)e.C + (int64_t)b * e.c_bstride;
    for (int i = 0; i < 8; ++i) {
      const int rr = rq + 4 * i, m = mrow0 + rr;
      if (m >= g.M) break;
      const float *src = mine + rr * 33 + 4 * cq;
      const float v0 = src[0] * e.alpha, v1 = src[1] * e.alpha, v2 = src[2] * e.alpha, v3 = src[3] * e.alpha;
      float *dst = cbase + (int64_t)m * e.map.s_m0 + n0;
      if (n0 + 3 < g.N) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(v0), "f"(v1), "f"(v2), "f"(v3)
                     : "memory");
      } else {
        if (n0 < g.N) atomicAdd(dst, v0);
        if (n0 + 1 < g.N) atomicAdd(dst + 1, v1);
        if (n0 + 2 < g.N) atomicAdd(dst + 2, v2);
      }
    }
    return;
  }
  const int n = nbase + lane;
  if (n >= g.N) return;
  for (int rr = 0; rr < 32; ++rr) {
    const int m = mrow0 + rr;
    if (m >= g.M) break;
    const float acc = mine[rr * 33 + lane];
    if (e.partial) e.partial[((int64_t)split * e.M + m) * e.N + n] = acc;
    else if (e.atomic) atomicAdd((float *)e.C + (int64_t)b * e.c_bstride + e.map(m, n), acc * e.alpha);
    else epi_store<bf16>(e, b, split, m, n, acc);
  }
}

// Four 16-byte vectors of row m, columns nb..nb+31 of a bf16 matrix (zero
// past column N or row M).
__device__ __forceinline__ void ld_row32(const void *base, int64_t ld, int m, bool mok, int nb, int N, uint4 (&o)[4]) {
  const bf16 *p = (const bf16 *)base + (int64_t)m * ld + nb;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (mok && nb + j * 8 + 7 < N) {
      o[j] = *reinterpret_cast<const uint4 *>(p + j * 8);
    } else {
      bf16 *h = reinterpret_cast<bf16 *>(&o[j]);
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) h[jj] = (mok && nb + j * 8 + jj < N) ? p[j * 8 + jj] : __float2bfloat16_rn(0.f);
    }
  }
}

__device__ __forceinline__ float bf_at(const uint4 (&o)[4], int k) {
  return __bfloat162float(reinterpret_cast<const bf16 *>(&o[k >> 3])[k & 7]);
}

// Persistent warp-specialised GEMM: grid = min(#tiles, #SMs), tiles taken
// round-robin (N fastest, so CTAs working at the same time share A tiles in L2).
// warp 0 lane 0: TMA producer (runs ahead through the stage ring across tiles)
// warp 1 lane 0: MMA issuer (accumulator buffer alternates per tile)
// warps 2-17: epilogue (warp w drains TMEM lane quarter w % 4 and takes the
//             32-column slot (w - 2) / 4 of every 128 columns)
// EK selects the epilogue compiled in: EK_PLAIN (TMA store; bias, scales and
// activation only), EK_OPS (TMA store with row operands: residual, gate,
// ReLU reference, aux copy) or EK_GENERAL (per-element stores: split-K
// partials and atomics, fp32 outputs, maps TMA cannot describe).  A smaller
// epilogue is a smaller, faster-issuing loop.
template <int BN, bool AMN, bool BMN, int EK>
__global__ void __launch_bounds__(576, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmOpA,
                   const __grid_constant__ CUtensorMap tmRes, GemmOp g, TcLaunch L) {
  pdl_trigger();
  using C = TcCfg<BN, AMN, BMN>;
  extern __shared__ uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t op_bar[EPI_WARPS][2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const uint32_t raw = smem_u32(dsmem);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = ((g.N + BN - 1) / BN) * ((g.M + BM - 1) / BM) * g.batch * g.splits;
  const int stages = L.stages;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf_bar[a], 1);
      mbar_init(&acce_bar[a], EPI_WARPS);
    }
    for (int w = 0; w < EPI_WARPS; ++w) {
      mbar_init(&op_bar[w][0], 1);
      mbar_init(&op_bar[w][1], 1);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // global memory only from here on: wait for the kernels before this one
  pdl_wait();

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    uint32_t it = 0, stage = 0, phase = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      const TileCoord tc = decode_tile(g, t, BN);
      for (int i = 0; i < tc.nk; ++i, ++it) {
        if (it >= (uint32_t)stages && !mbar_wait(&empty_bar[stage], phase ^ 1u, &s_abort)) {
          stop = true;
          break;
        }
        const uint32_t sa = sbase + stage * C::STAGE_BYTES;
        const uint32_t sb = sa + C::A_BYTES;
        const int kc = (tc.kt0 + i) * BK;
        mbar_arrive_expect_tx(&full_bar[stage], C::STAGE_BYTES);
        if (AMN) {
          tma_load_3d(sa, &tmA, tc.m0, kc, tc.b, &full_bar[stage]);
          tma_load_3d(sa + 8192, &tmA, tc.m0 + 64, kc, tc.b, &full_bar[stage]);
        } else {
          tma_load_3d(sa, &tmA, kc, tc.m0, tc.b, &full_bar[stage]);
        }
        if (BMN) {
#pragma unroll
          for (int cpart = 0; cpart < BN / 64; ++cpart)
            tma_load_3d(sb + cpart * 8192, &tmB, tc.n0 + cpart * 64, kc, tc.b, &full_bar[stage]);
        } else {
          tma_load_3d(sb, &tmB, kc, tc.n0, tc.b, &full_bar[stage]);
        }
        if (++stage == (uint32_t)stages) stage = 0, phase ^= 1u;
      }
    }
    if (s_abort) {
      // drain: wait (bounded) for every load that may still be in flight
      const uint32_t first = it > (uint32_t)stages ? it - stages : 0u;
      for (uint32_t i = first; i < it; ++i) {
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(&full_bar[i % stages], (i / stages) & 1u) && globaltimer_ns() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    uint32_t stage = 0, phase = 0, ai = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      const TileCoord tc = decode_tile(g, t, BN);
      if (tc.nk == 0) continue;
      const uint32_t ab = ai & 1u, u = ai >> 1;
      if (ai >= 2 && !mbar_wait(&acce_bar[ab], (u - 1) & 1u, &s_abort)) break;
      tc_fence_after();
      const uint32_t dacc = tmem + ab * BN;
      for (int i = 0; i < tc.nk; ++i) {
        if (!mbar_wait(&full_bar[stage], phase, &s_abort)) {
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + stage * C::STAGE_BYTES;
        const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t ad = smem_desc(sa + kk * C::A_KSTEP, C::A_LBO, 1024);
          const uint64_t bd = smem_desc(sb + kk * C::B_KSTEP, C::B_LBO, 1024);
          mma_ss(dacc, ad, bd, C::IDESC, (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty_bar[stage]);
        if (++stage == (uint32_t)stages) stage = 0, phase ^= 1u;
      }
      if (stop) break;
      mma_commit(&accf_bar[ab]);
      ++ai;
    }
    mma_commit(&done_bar);
  } else if (warp >= 2) {
    // ---------------- epilogue warps
    // warp w drains TMEM lane quarter w % 4 (the lanes tcgen05.ld lets it
    // reach); the four warps of a quarter take 32-column slots 0..3 of every
    // 128 columns of the tile.
    const int ew = warp - 2;
    const int quarter = warp & 3, slot = ew >> 2;
    const uint32_t region = sbase + stages * C::STAGE_BYTES + ew * L.epi_bytes;
    float *mine = reinterpret_cast<float *>(dsmem + (region - raw));
    const Epi &e = g.e;
    uint32_t ai = 0;
    if constexpr (EK != EK_GENERAL) {
      // Chunk k of this warp (k counts the warp's chunks over all its tiles)
      // uses slot k & 1.  Its operand tiles are requested by TMA at the end
      // of chunk k - 1 (the first one before the loop), after the store that
      // last read that slot (chunk k - 2) has finished reading.
      const uint32_t op_bytes = EK == EK_OPS ? (L.has_opa ? 2048u : 0u) + (L.has_res ? 2048u : 0u) : 0u;
      int nt = blockIdx.x, nc = slot * 32;  // the next chunk whose operands are requested
      // the chunks of a tile are columns slot*32 + 128 i below BN and N, rows
      // of the warp's quarter below M; advance() moves (nt, nc) to the next
      // one in the order the loop below visits them (nt >= ntiles: none left)
      auto advance = [&]() {
        nc += 128;
        while (nt < ntiles) {
          const TileCoord q = decode_tile(g, nt, BN);
          if (nc < BN && q.n0 + nc < g.N && q.m0 + quarter * 32 < g.M) return;
          nt += gridDim.x;
          nc = slot * 32;
        }
      };
      uint32_t requested = 0;  // chunks whose operand tiles have been requested
      auto request = [&](uint32_t k) {  // lane 0: operand tiles of chunk (nt, nc) into slot k & 1
        if (nt >= ntiles || op_bytes == 0) return;
        requested = k + 1;
        const TileCoord q = decode_tile(g, nt, BN);
        const uint32_t sl = k & 1u;
        mbar_arrive_expect_tx(&op_bar[ew][sl], op_bytes);
        const int n = q.n0 + nc, mq = q.m0 + quarter * 32;
        if (L.has_res) tma_load_3d(region + sl * 2048u, &tmRes, n, mq, q.b, &op_bar[ew][sl]);
        if (L.has_opa) tma_load_3d(region + 4096u + sl * 2048u, &tmOpA, n, mq, 0, &op_bar[ew][sl]);
      };
      nc -= 128;
      advance();
      if (lane == 0) request(0);
      uint32_t k = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileCoord tc = decode_tile(g, t, BN);
        const uint32_t ab = ai & 1u, u = ai >> 1;
        const int mrow0 = tc.m0 + quarter * 32;
        const int m = mrow0 + lane;
        const bool mok = m < g.M;
        bool have = false;
        if (tc.nk > 0) {
          have = mbar_wait(&accf_bar[ab], u & 1u, &s_abort);
          have = __all_sync(0xffffffffu, have);
          if (!have) break;
          tc_fence_after();
        }
        const float rs = (e.row_scale && mok) ? e.row_scale[m] : 1.f;
        bool ok = true;
        for (int c0 = slot * 32; c0 < BN && mrow0 < g.M; c0 += 128) {
          const int nb = tc.n0 + c0;
          if (nb >= g.N) break;
          const uint32_t sl = k & 1u;
          const uint32_t obuf = region + sl * 2048u, abuf = region + 4096u + sl * 2048u;
          // this thread's 64-byte row of a swizzled 32 x 32 bf16 tile: 16-byte
          // chunk j at j ^ ((row >> 1) & 3)
          const uint32_t rowoff = lane * 64u;
          const uint32_t swz = (uint32_t)((lane >> 1) & 3);
          float v[32];
          if (have) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ab * BN + (uint32_t)c0, r);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) v[jj] = __uint_as_float(r[jj]);
            if (e.alpha != 1.f) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj) v[jj] *= e.alpha;
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) v[jj] = 0.f;
          }
          // column conditions are decided per chunk where the whole chunk agrees
          if (e.bias && nb >= e.bias_n0 && nb + 31 < g.N) {
            const float4 *bp = reinterpret_cast<const float4 *>(e.bias + (nb - e.bias_n0));
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 x = bp[q];
              v[4 * q] += x.x, v[4 * q + 1] += x.y, v[4 * q + 2] += x.z, v[4 * q + 3] += x.w;
            }
          } else if (e.bias && nb + 31 >= e.bias_n0) {
            // boundary chunk: columns past N are clipped by the store, so their
            // (clamped) bias index only has to stay inside the bias vector
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int n = min(nb + jj, g.N - 1);
              const float b = e.bias[max(n - e.bias_n0, 0)];
              v[jj] += nb + jj >= e.bias_n0 ? b : 0.f;
            }
          }
          if (e.row_scale) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) v[jj] *= rs;
          }
          if (EK == EK_OPS && (L.has_opa || L.has_res)) {
            if (!mbar_wait(&op_bar[ew][sl], (k >> 1) & 1u, &s_abort)) ok = false;
            if (!__all_sync(0xffffffffu, ok)) break;
          }
          if (EK == EK_OPS && e.relu_ref) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              uint4 w;
              asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                           : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                           : "r"(abuf + rowoff + ((j ^ swz) << 4)));
              const bf16 *h = reinterpret_cast<const bf16 *>(&w);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj)
                if (!(__bfloat162float(h[jj]) > 0.f)) v[j * 8 + jj] = 0.f;
            }
          }
          if (e.act == ACT_RELU) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) v[jj] = fmaxf(v[jj], 0.f);
          } else if (e.act == ACT_SIGMOID && nb >= e.act_n0) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) v[jj] = __fdividef(1.f, 1.f + __expf(-v[jj]));
          } else if (e.act == ACT_SIGMOID && nb + 31 >= e.act_n0) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const float sg = __fdividef(1.f, 1.f + __expf(-v[jj]));
              v[jj] = nb + jj >= e.act_n0 ? sg : v[jj];
            }
          }
          if (EK == EK_OPS && e.aux && mok) {
            bf16 *p = (bf16 *)e.aux + (int64_t)m * e.aux_ld + nb;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (nb + j * 8 + 7 < g.N) {
                uint4 w;
                uint32_t *wp = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                  __nv_bfloat162 h2 = __floats2bfloat162_rn(v[j * 8 + 2 * jj], v[j * 8 + 2 * jj + 1]);
                  wp[jj] = *reinterpret_cast<uint32_t *>(&h2);
                }
                *reinterpret_cast<uint4 *>(p + j * 8) = w;
              } else {
                for (int jj = 0; jj < 8; ++jj)
                  if (nb + j * 8 + jj < g.N) p[j * 8 + jj] = __float2bfloat16_rn(v[j * 8 + jj]);
              }
            }
          }
          if (EK != EK_OPS || !L.has_res) {
            // the output slot was last read by the store of chunk k - 2
            if (lane == 0) bulk_wait_read<1>();
            __syncwarp();
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t off = rowoff + ((j ^ swz) << 4);
            if (EK == EK_OPS && e.gate) {
              uint4 w;
              asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                           : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                           : "r"(abuf + off));
              const bf16 *h = reinterpret_cast<const bf16 *>(&w);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) v[j * 8 + jj] *= __bfloat162float(h[jj]);
            }
            if (EK == EK_OPS && L.has_res) {
              uint4 w;
              asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                           : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                           : "r"(obuf + off));
              const bf16 *h = reinterpret_cast<const bf16 *>(&w);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) v[j * 8 + jj] += __bfloat162float(h[jj]);
            }
            uint32_t w[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              __nv_bfloat162 h2 = __floats2bfloat162_rn(v[j * 8 + 2 * jj], v[j * 8 + 2 * jj + 1]);
              w[jj] = *reinterpret_cast<uint32_t *>(&h2);
            }
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(obuf + off), "r"(w[0]), "r"(w[1]),
                         "r"(w[2]), "r"(w[3])
                         : "memory");
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {  // rows and columns past the tensor are clipped by TMA
            if (L.tma_store == 1) {
              tma_store_3d(&tmC, obuf, nb, mrow0, tc.b);
            } else {
              // 4-D view of a two-level output map (see the host side for the order)
              const int md = e.map.mdiv >= (1ll << 31) ? g.M : (int)e.map.mdiv;
              if (L.tma_store == 2) tma_store_4d(&tmC, obuf, 0, mrow0 % md, nb >> 5, mrow0 / md);
              else tma_store_4d(&tmC, obuf, 0, nb >> 5, mrow0 % md, mrow0 / md);
            }
            bulk_commit();
          }
          if (EK == EK_OPS && op_bytes) {
            // operands of the next chunk into the other slot, once the store
            // of chunk k - 1 (the slot's last reader) has read it
            advance();
            if (lane == 0) {
              bulk_wait_read<1>();
              request(k + 1);
            }
          }
          ++k;
        }
        if (!ok) break;
        if (tc.nk > 0) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce_bar[ab]);
          ++ai;
        }
        if (s_abort) break;
      }
      if (EK == EK_OPS && lane == 0) {
        // drain (after an abort): operand tiles requested but not consumed
        for (uint32_t kk = k; kk < requested; ++kk) {
          const uint64_t t0 = globaltimer_ns();
          while (!mbar_try_wait(&op_bar[ew][kk & 1u], (kk >> 1) & 1u) && globaltimer_ns() - t0 < WAIT_LIMIT_NS) {
          }
        }
      }
    } else {
      (void)tmC, (void)tmOpA, (void)tmRes;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileCoord tc = decode_tile(g, t, BN);
        const uint32_t ab = ai & 1u, u = ai >> 1;
        const int mrow0 = tc.m0 + quarter * 32;
        bool have = false;
        if (tc.nk > 0) {
          have = mbar_wait(&accf_bar[ab], u & 1u, &s_abort);
          have = __all_sync(0xffffffffu, have);
          if (!have) break;
          tc_fence_after();
        }
        for (int c0 = slot * 32; c0 < BN && mrow0 < g.M; c0 += 128) {
          if (tc.n0 + c0 >= g.N) break;
          if (have) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ab * BN + (uint32_t)c0, r);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) mine[lane * 33 + jj] = __uint_as_float(r[jj]);
          } else {
            for (int jj = 0; jj < 32; ++jj) mine[lane * 33 + jj] = 0.f;
          }
          __syncwarp();
          epi_chunk(g, mine, lane, mrow0, tc.n0 + c0, tc.b, tc.split);
          __syncwarp();
        }
        if (tc.nk > 0) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce_bar[ab]);
          ++ai;
        }
        if (s_abort) break;
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  __syncwarp();
  // every MMA issued has completed before TMEM is released
  if (threadIdx.x == 0) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(&done_bar, 0) && globaltimer_ns() - t0 < WAIT_LIMIT_NS) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
}

__global__ void debug_wait_kernel(int64_t limit_ns) {
  pdl_entry();
  debug_wait_body(limit_ns);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
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
  return fn;
}

// 3-D bf16 tensor {inner, outer, batch} with strides ld, bs (elements).
bool make_tmap(CUtensorMap *tm, const void *base, uint64_t inner, uint64_t outer, uint64_t batch, uint64_t ld,
               uint64_t bs, uint32_t box_inner, uint32_t box_outer,
               CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  if (batch <= 1) bs = ld * outer;
  cuuint64_t dims[3] = {inner, outer, batch < 1 ? 1 : batch};
  cuuint64_t strides[2] = {ld * 2, bs * 2};
  cuuint32_t box[3] = {box_inner, box_outer, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 148;
  }
  return n;
}

// 4-D bf16 tensor {d0, d1, d2, d3} with element strides s1, s2, s3 (any order).
bool make_tmap4(CUtensorMap *tm, const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3, uint64_t s1,
                uint64_t s2, uint64_t s3, uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3, CUtensorMapSwizzle swz) {
  // strides must be non-decreasing and each must span the previous dimension
  if (s1 < d0 || s2 < s1 * d1 || s3 < s2 * d2) return false;
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[4] = {d0, d1, d2, d3};
  cuuint64_t strides[3] = {s1 * 2, s2 * 2, s3 * 2};
  cuuint32_t box[4] = {b0, b1, b2, b3};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, bool AMN, bool BMN, int EK>
cudaError_t run_tc(int grid, int smem, cudaStream_t s, const CUtensorMap &ta, const CUtensorMap &tb,
                   const CUtensorMap &tc, const CUtensorMap &topa, const CUtensorMap &tres, const GemmOp &g,
                   const TcLaunch &L) {
  static bool attr_set = false;
  if (!attr_set) {
    // the opt-in limit covers static shared memory (the barriers) as well
    cudaError_t err = cudaFuncSetAttribute(gemm_tc_kernel<BN, AMN, BMN, EK>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT - 2048);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  return launch_k(gemm_tc_kernel<BN, AMN, BMN, EK>, grid, 32 * (2 + EPI_WARPS), smem, s, ta, tb, tc, topa, tres, g,
                  L);
}

template <int BN, bool AMN, bool BMN>
cudaError_t launch_tc(const GemmOp &g, cudaStream_t s) {
  using C = TcCfg<BN, AMN, BMN>;
  CUtensorMap ta, tb;
  bool ok = AMN ? make_tmap(&ta, g.A, g.M, g.K, g.batch, g.lda, g.a_bs, 64, 64)
                : make_tmap(&ta, g.A, g.K, g.M, g.batch, g.lda, g.a_bs, 64, BM);
  ok = ok && (BMN ? make_tmap(&tb, g.B, g.N, g.K, g.batch, g.ldb, g.b_bs, 64, 64)
                  : make_tmap(&tb, g.B, g.K, g.N, g.batch, g.ldb, g.b_bs, 64, BN));
  if (!ok) return cudaErrorInvalidValue;
  // TMA-store epilogue.  Kind 1: plain row-major bf16 output (3-D map over
  // n, m, batch).  Kind 2: a two-level map with 32-wide column groups,
  // offset = (n / 32) s_n1 + n % 32 + (m / mdiv) s_m1 + (m % mdiv) s_m0, stored
  // through a 4-D map whose box is one warp's 32 x 32 sub-tile.  The row
  // operands (residual, gate or ReLU reference) arrive by TMA as 32 x 32
  // tiles too, so they need 16-byte aligned bases and row strides.
  const Epi &e = g.e;
  auto a16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  const bool operands_ok = !e.partial && !e.atomic && !e.c_f32 && !e.accumulate && !(e.gate && e.relu_ref) && a16(e.C) &&
                           (!e.residual || a16(e.residual)) &&
                           (!e.relu_ref || (a16(e.relu_ref) && e.relu_ld % 8 == 0)) &&
                           (!e.aux || (a16(e.aux) && e.aux_ld % 8 == 0)) &&
                           (!e.gate || (a16(e.gate) && e.gate_ld % 8 == 0)) &&
                           (!e.bias || (a16(e.bias) && e.bias_n0 % 4 == 0));
  const bool plain = e.map.mdiv >= (1ll << 31) && e.map.ndiv >= (1ll << 31) && e.map.s_n0 == 1;
  TcLaunch L{};
  CUtensorMap tc, topa, tres;
  std::memset(&tc, 0, sizeof(tc));
  std::memset(&topa, 0, sizeof(topa));
  std::memset(&tres, 0, sizeof(tres));
  if (operands_ok && plain && e.map.s_m0 % 8 == 0 && (g.batch == 1 || e.c_bstride % 8 == 0)) {
    if (make_tmap(&tc, e.C, g.N, g.M, g.batch, e.map.s_m0, g.batch > 1 ? e.c_bstride : 0, 32, 32,
                  CU_TENSOR_MAP_SWIZZLE_64B))
      L.tma_store = 1;
  } else if (operands_ok && !plain && g.batch == 1 && !e.residual && e.map.ndiv == 32 && e.map.s_n0 == 1 &&
             g.N % 32 == 0 && e.map.s_n1 % 8 == 0 && e.map.s_m0 % 8 == 0 &&
             (e.map.mdiv >= (1ll << 31) || (e.map.mdiv % 32 == 0 && g.M % e.map.mdiv == 0 && e.map.s_m1 % 8 == 0))) {
    // TMA wants each dimension's stride to cover the previous dimensions, so the
    // four index parts are ordered by stride: d (1) first, then the smaller of
    // m % md and n / 32, then the other, then m / md.
    const uint64_t md = e.map.mdiv >= (1ll << 31) ? (uint64_t)g.M : (uint64_t)e.map.mdiv;
    const uint64_t s_nhi = (uint64_t)e.map.s_n1, s_mlo = (uint64_t)e.map.s_m0;
    const uint64_t nhi = (uint64_t)g.N / 32, mhi = (uint64_t)g.M / md;
    // a single m / md group never steps its stride: give it one past the others
    const uint64_t s_mhi = mhi == 1 ? std::max(s_mlo * md, s_nhi * nhi)
                                    : (e.map.mdiv >= (1ll << 31) ? s_mlo * md : (uint64_t)e.map.s_m1);
    if (s_mlo >= 32 && s_mlo <= s_nhi && s_nhi >= s_mlo * md && s_mhi >= s_nhi * nhi) {
      if (make_tmap4(&tc, e.C, 32, md, nhi, mhi, s_mlo, s_nhi, s_mhi, 32, 32, 1, 1, CU_TENSOR_MAP_SWIZZLE_64B))
        L.tma_store = 2;
    } else if (s_nhi >= 32 && s_nhi <= s_mlo && s_mlo >= s_nhi * nhi && s_mhi >= s_mlo * md) {
      if (make_tmap4(&tc, e.C, 32, nhi, md, mhi, s_nhi, s_mlo, s_mhi, 32, 1, 32, 1, CU_TENSOR_MAP_SWIZZLE_64B))
        L.tma_store = 3;
    }
  }
  if (L.tma_store) {
    const void *opa = e.gate ? e.gate : e.relu_ref;
    const int64_t opa_ld = e.gate ? e.gate_ld : e.relu_ld;
    bool ops = true;
    if (opa) {
      ops = make_tmap(&topa, opa, g.N, g.M, 1, opa_ld, 0, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B);
      L.has_opa = 1;
    }
    if (ops && e.residual) {
      ops = make_tmap(&tres, e.residual, g.N, g.M, g.batch, e.map.s_m0, g.batch > 1 ? e.c_bstride : 0, 32, 32,
                      CU_TENSOR_MAP_SWIZZLE_64B);
      L.has_res = 1;
    }
    if (!ops) L.tma_store = L.has_opa = L.has_res = 0;
  }
  L.epi_bytes = epi_warp_bytes(L.has_opa);
  L.stages = std::min(MAX_STAGES, (SMEM_LIMIT - 2048 - EPI_WARPS * L.epi_bytes) / C::STAGE_BYTES);
  if (L.stages < 2) return cudaErrorInvalidValue;
  const int smem = L.stages * C::STAGE_BYTES + EPI_WARPS * L.epi_bytes + 1024;
  // more than half of the SM's shared memory: one resident CTA per SM, so a
  // CTA's TMEM allocation never waits on another CTA's
  if (smem <= SMEM_LIMIT / 2 + 1024 || smem > SMEM_LIMIT - 2048) return cudaErrorInvalidValue;

  const long long tiles =
      (long long)((g.N + BN - 1) / BN) * ((g.M + BM - 1) / BM) * (long long)g.batch * g.splits;
  const int grid = (int)std::min<long long>(tiles, sm_count());
  // algorithmic bytes: operands once, the output once, and every epilogue
  // operand (residual, gate, ReLU reference, aux copy) once
  double cbytes = g.e.partial ? 4.0 * g.splits : (g.e.c_f32 ? (g.e.accumulate ? 8.0 : 4.0) : 2.0);
  cbytes += 2.0 * ((g.e.residual ? 1 : 0) + (g.e.gate ? 1 : 0) + (g.e.relu_ref ? 1 : 0) + (g.e.aux ? 1 : 0));
  Prof p(prof_detail() ? prof_name("g%dx%dx%d*%ds%dn%d%s%se%d", (int)g.M, (int)g.N, (int)g.K, (int)g.batch, g.splits,
                                    BN, AMN ? "T" : "", BMN ? "t" : "", L.tma_store)
                      : (g.cls ? g.cls : "gemm_tc"),
         s, 2.0 * g.M * g.N * (double)g.K * g.batch,
         g.batch * (2.0 * ((double)g.M * g.K + (double)g.N * g.K) + cbytes * g.M * g.N));
  const int ek = !L.tma_store ? EK_GENERAL : (L.has_opa || L.has_res || e.aux) ? EK_OPS : EK_PLAIN;
  if (ek == EK_PLAIN) return run_tc<BN, AMN, BMN, EK_PLAIN>(grid, smem, s, ta, tb, tc, topa, tres, g, L);
  if (ek == EK_OPS) return run_tc<BN, AMN, BMN, EK_OPS>(grid, smem, s, ta, tb, tc, topa, tres, g, L);
  return run_tc<BN, AMN, BMN, EK_GENERAL>(grid, smem, s, ta, tb, tc, topa, tres, g, L);
}

template <int BN>
cudaError_t dispatch_major(const GemmOp &g, cudaStream_t s) {
  if (g.a_mn) {
    return g.b_mn ? launch_tc<BN, true, true>(g, s) : launch_tc<BN, true, false>(g, s);
  }
  return g.b_mn ? launch_tc<BN, false, true>(g, s) : launch_tc<BN, false, false>(g, s);
}

}  // namespace

cudaError_t error_word_read_clear(int *out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, tc_error_word, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(tc_error_word, &zero, sizeof(int));
}

cudaError_t debug_wait(int64_t limit_ns, cudaStream_t s) {
  Prof p("debug_wait", s);
  launch_k(debug_wait_kernel, 1, 32, 0, s, limit_ns);
  return cudaGetLastError();
}

bool gemm_tc_supported(const GemmOp &g) {
  auto al16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (!al16(g.A) || !al16(g.B)) return false;
  if ((g.lda * 2) % 16 || (g.ldb * 2) % 16) return false;
  if (g.batch > 1 && ((g.a_bs * 2) % 16 || (g.b_bs * 2) % 16)) return false;
  if (g.splits > 1 && (g.batch != 1 || !(g.e.partial || g.e.atomic))) return false;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return false;
  return true;
}

cudaError_t gemm_tc_bf16(const GemmOp &g0, cudaStream_t s) {
  if (!gemm_tc_supported(g0)) return cudaErrorInvalidValue;
  // one persistent CTA per SM; the tile width (and, for atomic split-K, the
  // split count) is the autotuner's once it has timed this shape
  const int bn0 = g0.N > 128 && g0.N % 256 == 0 ? 256 : g0.N > 64 ? 128 : 64;
  const TuneChoice c = tune_choose(g0, bn0, s);
  GemmOp g = g0;
  g.splits = c.splits;
  const cudaError_t err = c.bn == 256   ? dispatch_major<256>(g, s)
                          : c.bn == 128 ? dispatch_major<128>(g, s)
                                        : dispatch_major<64>(g, s);
  tune_done(c, s);
  return err;
}

}  // namespace evo
