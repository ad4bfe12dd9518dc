// BF16 GEMM on the 5th-generation tensor cores (sm_103a): TMA loads 128x64 /
// BNx64 operand tiles (128-byte swizzle) into a STAGES-deep shared-memory ring,
// one elected thread issues tcgen05.mma (M=128, N=BN, K=16) accumulating FP32
// in tensor memory, and the four warps drain TMEM with tcgen05.ld through the
// shared epilogue (bias, scales, gates, residual, layout-changing stores).
//
// Warp roles (256 threads): warp 0 allocates TMEM, lane 0 of warp 0 is the TMA
// producer, lane 0 of warp 1 issues the MMAs, all eight warps run the epilogue
// (warps w and w+4 read TMEM lanes / tile rows 32w..32w+31, half the columns each).
//
// Operands may be K-major or MN-major (the transpose bits of the instruction
// descriptor); backward GEMMs (dX = dY W, dW = dY^T X) use MN-major views of
// the forward tensors instead of transposed copies.
//
// Every wait on an mbarrier is bounded (about one second of %globaltimer); a
// wait that runs out sets the library's device error word, the CTA drains its
// in-flight copies with bounded waits, frees its TMEM and returns.
#include <cuda.h>

#include "kernels.h"

namespace evo {

__device__ int g_evo_error = 0;

namespace {

constexpr int BM = 128, BK = 64;
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; gives up when the CTA abort flag is raised or the limit passes.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
      *abort_flag = 1;
      atomicExch(&g_evo_error, -6);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle, sm_100-family version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, dense.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN, int STAGES, bool AMN, bool BMN>
struct TcCfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
  // A K-major tile: rows of 128 B, k-step of 16 elements = 32 B.
  // An MN-major tile: 64-element (128 B) MN chunks of 64 K-rows (8 KB each);
  // a k-step of 16 rows = 2 KB.
  static constexpr uint32_t A_KSTEP = AMN ? 2048u : 32u;
  static constexpr uint32_t B_KSTEP = BMN ? 2048u : 32u;
  static constexpr uint32_t A_LBO = AMN ? 8192u : 16u;
  static constexpr uint32_t B_LBO = BMN ? 8192u : 16u;
  static constexpr uint32_t IDESC = instr_desc(BM, BN, AMN, BMN);
  // At most 512 TMEM columns per SM across the CTAs that fit by shared memory.
  static_assert((233472 / (SMEM + 1024)) * TMEM_COLS <= 512, "TMEM oversubscription");
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N");
  // the epilogue stages 8 warps x 32 rows x (64 + 1) floats in the stage buffers
  static_assert(8 * 32 * ((BN < 64 ? BN : 64) + 1) * 4 <= STAGES * STAGE_BYTES, "epilogue staging");
};

template <int BN, int STAGES, bool AMN, bool BMN>
__global__ void __launch_bounds__(256, 2)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmOp g) {
  using C = TcCfg<BN, STAGES, AMN, BMN>;
  extern __shared__ uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const uint32_t raw = smem_u32(dsmem);
  const uint32_t sbase = (raw + 1023u) & ~1023u;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int b = blockIdx.z / g.splits, split = blockIdx.z % g.splits;
  const int kt_total = (g.K + BK - 1) / BK;
  const int per = (kt_total + g.splits - 1) / g.splits;
  const int kt0 = split * per;
  const int nk = max(0, min(kt_total, kt0 + per) - kt0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (nk > 0 && warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      const uint32_t j = (uint32_t)(i / STAGES);
      if (i >= STAGES && !mbar_wait(&empty_bar[s], (j - 1) & 1u, &s_abort)) break;
      const uint32_t sa = sbase + s * C::STAGE_BYTES;
      const uint32_t sb = sa + C::A_BYTES;
      const int kc = (kt0 + i) * BK;
      mbar_arrive_expect_tx(&full_bar[s], C::STAGE_BYTES);
      if (AMN) {
        tma_load_3d(sa, &tmA, m0, kc, b, &full_bar[s]);
        tma_load_3d(sa + 8192, &tmA, m0 + 64, kc, b, &full_bar[s]);
      } else {
        tma_load_3d(sa, &tmA, kc, m0, b, &full_bar[s]);
      }
      if (BMN) {
#pragma unroll
        for (int c = 0; c < BN / 64; ++c) tma_load_3d(sb + c * 8192, &tmB, n0 + c * 64, kc, b, &full_bar[s]);
      } else {
        tma_load_3d(sb, &tmB, kc, n0, b, &full_bar[s]);
      }
      ++issued;
    }
    if (s_abort) {
      // drain: wait (bounded) for every load still in flight before leaving
      for (int i = max(0, issued - STAGES); i < issued; ++i) {
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(&full_bar[i % STAGES], (uint32_t)(i / STAGES) & 1u) &&
               globaltimer_ns() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (nk > 0 && warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      const uint32_t j = (uint32_t)(i / STAGES);
      if (!mbar_wait(&full_bar[s], j & 1u, &s_abort)) break;
      tc_fence_after();
      const uint32_t sa = sbase + s * C::STAGE_BYTES;
      const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ad = smem_desc(sa + kk * C::A_KSTEP, C::A_LBO, 1024);
        const uint64_t bd = smem_desc(sb + kk * C::B_KSTEP, C::B_LBO, 1024);
        tc_mma(tmem, ad, bd, C::IDESC, (i > 0 || kk > 0) ? 1u : 0u);
      }
      tc_commit(&empty_bar[s]);
    }
    tc_commit(&done_bar);
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> shared (64-column chunks, in the idle
  // stage buffers) -> stores with lanes along columns, so every output map
  // used by the block is written in contiguous runs.  Warps w and w+4 share
  // TMEM lane quarter w and split the tile's columns.
  bool have = nk > 0;
  if (have) have = mbar_wait(&done_bar, 0, &s_abort);
  have = __all_sync(0xffffffffu, have);
  tc_fence_after();
  const int quarter = warp & 3, half = warp >> 2;
  constexpr int CH = BN < 64 ? BN : 64;
  constexpr int LDS = CH + 1;
  constexpr int NCH = BN / CH;
  constexpr int CH_PER_HALF = NCH > 1 ? NCH / 2 : 1;
  if (have || (nk == 0 && !s_abort)) {
    float *mine = reinterpret_cast<float *>(dsmem + (sbase - raw)) + warp * 32 * LDS;
    const Epi &e = g.e;
    const bool fast = !e.partial && !e.c_f32 && !e.relu_ref && !e.aux && !e.gate && e.map.mdiv >= (1ll << 31) &&
                      e.map.ndiv >= (1ll << 31) && e.map.s_n0 == 1 && (e.map.s_m0 & 1) == 0 &&
                      (e.c_bstride & 1) == 0;
    for (int ci = 0; ci < CH_PER_HALF; ++ci) {
      const int cidx = NCH > 1 ? half * CH_PER_HALF + ci : ci;
      if (NCH == 1 && half == 1) break;  // a single chunk is drained by warps 0-3
      const int c0 = cidx * CH;
      if (n0 + c0 >= g.N) break;
      if (have) {
#pragma unroll
        for (int q = 0; q < CH; q += 16) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(c0 + q), r);
#pragma unroll
          for (int j = 0; j < 16; ++j) mine[lane * LDS + q + j] = __uint_as_float(r[j]);
        }
      } else {
        for (int j = 0; j < CH; ++j) mine[lane * LDS + j] = 0.f;
      }
      __syncwarp();
      const int cc = 2 * lane;
      const int n = n0 + c0 + cc;
      if (fast && cc < CH) {
        // row-major output: bias / activation decisions per lane, one bf16x2 per row
        const bool ok0 = n < g.N, ok1 = n + 1 < g.N;
        const float b0 = (e.bias && ok0 && n >= e.bias_n0) ? e.bias[n - e.bias_n0] : 0.f;
        const float b1 = (e.bias && ok1 && n + 1 >= e.bias_n0) ? e.bias[n + 1 - e.bias_n0] : 0.f;
        const bool s0 = e.act == ACT_SIGMOID && n >= e.act_n0, s1 = e.act == ACT_SIGMOID && n + 1 >= e.act_n0;
        const bool relu = e.act == ACT_RELU;
        bf16 *cb = (bf16 *)e.C + (int64_t)b * e.c_bstride + n;
        const bf16 *rb = e.residual ? (const bf16 *)e.residual + (int64_t)b * e.c_bstride + n : nullptr;
        for (int rr = 0; rr < 32; ++rr) {
          const int m = m0 + quarter * 32 + rr;
          if (m >= g.M || !ok0) break;
          float v0 = mine[rr * LDS + cc] * e.alpha + b0;
          float v1 = mine[rr * LDS + cc + 1] * e.alpha + b1;
          if (e.row_scale) {
            const float rs = e.row_scale[m];
            v0 *= rs;
            v1 *= rs;
          }
          if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          if (s0) v0 = 1.f / (1.f + __expf(-v0));
          if (s1) v1 = 1.f / (1.f + __expf(-v1));
          const int64_t ro = (int64_t)m * e.map.s_m0;
          if (ok1) {
            if (rb) {
              const __nv_bfloat162 r2 = *reinterpret_cast<const __nv_bfloat162 *>(rb + ro);
              v0 += __low2float(r2);
              v1 += __high2float(r2);
            }
            *reinterpret_cast<__nv_bfloat162 *>(cb + ro) = __floats2bfloat162_rn(v0, v1);
          } else {
            if (rb) v0 += __bfloat162float(rb[ro]);
            cb[ro] = __float2bfloat16_rn(v0);
          }
        }
      } else if (cc < CH) {
        for (int rr = 0; rr < 32; ++rr) {
          const int m = m0 + quarter * 32 + rr;
          if (m >= g.M) break;
          const int64_t rowoff = (int64_t)b * e.c_bstride + e.map.row(m);
          if (n < g.N) epi_pair<bf16>(e, b, split, m, n, rowoff, mine[rr * LDS + cc], mine[rr * LDS + cc + 1]);
        }
      }
      __syncwarp();
    }
  }
  if (s_abort && nk > 0 && threadIdx.x == 0) {
    // MMAs may still be in flight: wait (bounded) for their commit before freeing TMEM
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(&done_bar, 0) && globaltimer_ns() - t0 < WAIT_LIMIT_NS) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
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
               uint64_t bs, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  if (batch <= 1) bs = ld * outer;
  cuuint64_t dims[3] = {inner, outer, batch < 1 ? 1 : batch};
  cuuint64_t strides[2] = {ld * 2, bs * 2};
  cuuint32_t box[3] = {box_inner, box_outer, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int STAGES, bool AMN, bool BMN>
cudaError_t launch_tc(const GemmOp &g, cudaStream_t s) {
  using C = TcCfg<BN, STAGES, AMN, BMN>;
  CUtensorMap ta, tb;
  bool ok = AMN ? make_tmap(&ta, g.A, g.M, g.K, g.batch, g.lda, g.a_bs, 64, 64)
                : make_tmap(&ta, g.A, g.K, g.M, g.batch, g.lda, g.a_bs, 64, BM);
  ok = ok && (BMN ? make_tmap(&tb, g.B, g.N, g.K, g.batch, g.ldb, g.b_bs, 64, 64)
                  : make_tmap(&tb, g.B, g.K, g.N, g.batch, g.ldb, g.b_bs, 64, BN));
  if (!ok) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<BN, STAGES, AMN, BMN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch * g.splits);
  const double cbytes = g.e.partial ? 4.0 * g.splits : (g.e.c_f32 ? 4.0 : 2.0);
  Prof p("gemm_tc", s, 2.0 * g.M * g.N * (double)g.K * g.batch,
         g.batch * (2.0 * ((double)g.M * g.K + (double)g.N * g.K) + cbytes * g.M * g.N));
  gemm_tc_kernel<BN, STAGES, AMN, BMN><<<grid, 256, C::SMEM, s>>>(ta, tb, g);
  return cudaGetLastError();
}

template <int BN, int STAGES>
cudaError_t dispatch_major(const GemmOp &g, cudaStream_t s) {
  if (g.a_mn) {
    return g.b_mn ? launch_tc<BN, STAGES, true, true>(g, s) : launch_tc<BN, STAGES, true, false>(g, s);
  }
  return g.b_mn ? launch_tc<BN, STAGES, false, true>(g, s) : launch_tc<BN, STAGES, false, false>(g, s);
}

__global__ void debug_wait_kernel(int64_t limit_ns) {
  // One mbarrier that nothing ever arrives on: the bounded wait runs out,
  // records the timeout in the device error word and the kernel returns.
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  abort_flag = 0;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(&bar, 0)) {
    if ((int64_t)(globaltimer_ns() - t0) > limit_ns) {
      atomicExch(&g_evo_error, -6);
      return;
    }
  }
}

}  // namespace

cudaError_t error_word_read_clear(int *out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_evo_error, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_evo_error, &zero, sizeof(int));
}

cudaError_t debug_wait(int64_t limit_ns, cudaStream_t s) {
  Prof p("debug_wait", s);
  debug_wait_kernel<<<1, 32, 0, s>>>(limit_ns);
  return cudaGetLastError();
}

bool gemm_tc_supported(const GemmOp &g) {
  auto al16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (!al16(g.A) || !al16(g.B)) return false;
  if ((g.lda * 2) % 16 || (g.ldb * 2) % 16) return false;
  if (g.batch > 1 && ((g.a_bs * 2) % 16 || (g.b_bs * 2) % 16)) return false;
  if (g.splits > 1 && (g.batch != 1 || !g.e.partial)) return false;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return false;
  return true;
}

cudaError_t gemm_tc_bf16(const GemmOp &g, cudaStream_t s) {
  if (!gemm_tc_supported(g)) return cudaErrorInvalidValue;
  // stage counts keep two CTAs resident per SM (shared memory and 512 TMEM columns)
  if (g.N > 128 && g.N % 256 == 0) return dispatch_major<256, 2>(g, s);
  if (g.N > 64) return dispatch_major<128, 3>(g, s);
  return dispatch_major<64, 4>(g, s);
}

}  // namespace evo
