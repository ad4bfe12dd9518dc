// Fused transition MLP (AF2 Alg. 9 and 15, the MSA and pair transitions; the
// operator fusion of Sec. 3.1 carried over to the MLP) on the 5th-generation
// tensor cores:
//
//   out = x + b2 + relu(xn W1^T + b1) W2^T        (xn = LayerNorm(x), C -> N1 -> C)
//
// for a tile of 128 rows at a time, with the N1-wide hidden layer kept on the
// SM: it is produced 128 columns (a chunk) at a time into tensor memory by
// the first product, turned into BF16 (bias, ReLU) by the epilogue warps and
// written back into the same tensor memory (two BF16 per 32-bit column), and
// consumed there as the A operand of the second product, whose FP32
// accumulator O (128 x C) stays in tensor memory across the chunks.  Shared
// memory holds only the tile's xn rows and a deep ring of weight slices.  The hidden layer never goes to global memory: the kernel serves
// the paths that do not keep it (the backward's recompute keeps it for dW2
// and the ReLU mask and runs the two products as separate GEMMs).
//
// One persistent CTA per SM (tiles round-robin), warp-specialised:
//   warp 0 lane 0: TMA producer: the tile's xn rows once, then the weight
//                  slices through a ring of 16 KB stages in the order the
//                  MMAs take them: W1_0, W1_1, W2_0, W1_2, W2_1, ..., W2_last;
//   warp 1 lane 0: MMA issuer: GEMM1 of chunk j into hidden buffer j % 2,
//                  then GEMM2 of chunk j - 1, so that the epilogue of a
//                  chunk overlaps the next chunk's first product;
//   warps 2-17:    epilogue: hidden chunks (bias, ReLU, BF16 back into
//                  tensor memory), then the tile's output (bias, residual,
//                  BF16);
//                  each warp's global operands (biases, residual rows) are
//                  requested before it waits for the accumulator they meet.
// Tensor memory: O in columns [0, C), the two hidden buffers at 256 and 384
// (each 128 FP32 columns; the warp that reads hidden columns 32 s .. 32 s + 31
// writes their BF16 pairs into the first 16 of them).
// Every mbarrier wait is bounded; a wait that runs out sets this unit's error
// word and the CTA drains its copies and MMAs, frees its tensor memory and
// returns.
#include "tc.cuh"

namespace evo {
using namespace tc;
namespace {

constexpr int MB = 128;                  // rows per tile (the MMA's M)
constexpr int NH = 128;                  // hidden columns per chunk (GEMM1's N, GEMM2's K)
constexpr int SLICE = 128 * 64 * 2;      // one [128 rows x 64 k] BF16 operand slice (16 KB)
constexpr int MLP_EPI_WARPS = 16;        // four per TMEM lane quarter
constexpr int MLP_THREADS = 32 * (2 + MLP_EPI_WARPS);
constexpr int MLP_SMEM_LIMIT = 232448;   // dynamic shared memory one CTA may use
constexpr int MLP_MAX_STAGES = 12;

template <int C>
struct MlpCfg {
  static constexpr int KS1 = C / 64;         // k-slices of xn and of a W1 chunk
  static constexpr int W2S = 2 * (C / 128);  // W2 slices of a chunk: C / 128 row halves x 2 k-slices
  static constexpr int A1_BYTES = KS1 * SLICE;
  static constexpr int FIXED = A1_BYTES;
  static constexpr int FIT = (MLP_SMEM_LIMIT - 2048 - FIXED) / SLICE;
  static constexpr int STAGES = FIT > MLP_MAX_STAGES ? MLP_MAX_STAGES : FIT;
  static constexpr int SMEM = FIXED + STAGES * SLICE + 1024;
  static constexpr uint32_t IDESC = instr_desc(MB, 128, false, false);
  static constexpr uint32_t TM_O = 0, TM_H = 256;
  static_assert(STAGES >= 3, "ring too shallow");
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

template <int C>
__global__ void __launch_bounds__(MLP_THREADS, 1)
    mlp_fused_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                     const __grid_constant__ CUtensorMap tmW2, const float *b1, const float *b2, const bf16 *res,
                     bf16 *out, int M, int N1) {
  pdl_trigger();
  using Cf = MlpCfg<C>;
  constexpr int STAGES = Cf::STAGES;
  extern __shared__ uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t a1_full, a1_empty, h_full[2], hs_full[2], hs_empty[2];
  __shared__ __align__(8) uint64_t o_full, o_empty, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const uint32_t raw = smem_u32(dsmem);
  const uint32_t sA1 = (raw + 1023u) & ~1023u, sRing = sA1 + Cf::A1_BYTES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (M + MB - 1) / MB, NCH = N1 / NH;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&a1_full, 1);
    mbar_init(&a1_empty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&h_full[b], 1);
      mbar_init(&hs_full[b], MLP_EPI_WARPS);
      mbar_init(&hs_empty[b], 1);
    }
    mbar_init(&o_full, 1);
    mbar_init(&o_empty, MLP_EPI_WARPS);
    mbar_init(&done_bar, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  pdl_wait();  // global memory only from here on

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    uint32_t it = 0, stage = 0, phase = 0, ti = 0, a1_loads = 0;
    bool stop = false;
    auto put = [&](const CUtensorMap *tm, int c0, int c1) {
      if (it >= (uint32_t)STAGES && !mbar_wait(&empty_bar[stage], phase ^ 1u, &s_abort)) return false;
      mbar_arrive_expect_tx(&full_bar[stage], SLICE);
      tma_load_3d(sRing + stage * SLICE, tm, c0, c1, 0, &full_bar[stage]);
      ++it;
      if (++stage == (uint32_t)STAGES) stage = 0, phase ^= 1u;
      return true;
    };
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++ti) {
      // the previous tile's first products have read the xn tile
      if (ti >= 1 && !mbar_wait(&a1_empty, (ti - 1) & 1u, &s_abort)) break;
      mbar_arrive_expect_tx(&a1_full, Cf::A1_BYTES);
#pragma unroll
      for (int ks = 0; ks < Cf::KS1; ++ks) tma_load_3d(sA1 + ks * SLICE, &tmX, 64 * ks, t * MB, 0, &a1_full);
      ++a1_loads;
      for (int j = 0; j <= NCH && !stop; ++j) {
        if (j < NCH)
          for (int ks = 0; ks < Cf::KS1 && !stop; ++ks) stop = !put(&tmW1, 64 * ks, NH * j);
        if (j >= 1)
          for (int q = 0; q < Cf::W2S && !stop; ++q) stop = !put(&tmW2, NH * (j - 1) + 64 * (q & 1), 128 * (q >> 1));
      }
    }
    if (s_abort) {
      // drain: wait (bounded) for every load that may still be in flight
      const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
      for (uint32_t i = first; i < it; ++i) mbar_drain(&full_bar[i % STAGES], (i / STAGES) & 1u);
      if (a1_loads) mbar_drain(&a1_full, (a1_loads - 1) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    uint32_t stage = 0, phase = 0, ti = 0, g = 0;
    bool stop = false;
    auto take = [&](uint32_t &addr) {
      if (!mbar_wait(&full_bar[stage], phase, &s_abort)) return false;
      tc_fence_after();
      addr = sRing + stage * SLICE;
      return true;
    };
    auto release = [&]() {
      mma_commit(&empty_bar[stage]);
      if (++stage == (uint32_t)STAGES) stage = 0, phase ^= 1u;
    };
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++ti) {
      if (!mbar_wait(&a1_full, ti & 1u, &s_abort)) break;
      tc_fence_after();
      for (int j = 0; j <= NCH && !stop; ++j) {
        if (j < NCH) {
          // GEMM1 of chunk j: H[hb] = xn W1_j^T, once GEMM2 of the buffer's
          // previous chunk (gj - 2) has read its BF16 pairs
          const uint32_t gj = g + j, hb = gj & 1u, u = gj >> 1;
          if (gj >= 2 && !mbar_wait(&hs_empty[hb], (u - 1) & 1u, &s_abort)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t dH = tmem + Cf::TM_H + hb * NH;
          for (int ks = 0; ks < Cf::KS1; ++ks) {
            uint32_t b;
            if (!take(b)) {
              stop = true;
              break;
            }
            const uint32_t a = sA1 + ks * SLICE;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_ss(dH, smem_desc(a + kk * 32, 16, 1024), smem_desc(b + kk * 32, 16, 1024), Cf::IDESC,
                     (ks > 0 || kk > 0) ? 1u : 0u);
            release();
          }
          if (stop) break;
          mma_commit(&h_full[hb]);
          if (j == NCH - 1) mma_commit(&a1_empty);
        }
        if (j >= 1) {
          // GEMM2 of chunk j - 1: O += H[pb] (BF16 in tensor memory) W2_{j-1}^T
          const uint32_t gp = g + j - 1, pb = gp & 1u, up = gp >> 1;
          if (j == 1 && ti >= 1 && !mbar_wait(&o_empty, (ti - 1) & 1u, &s_abort)) {
            stop = true;
            break;
          }
          if (!mbar_wait(&hs_full[pb], up & 1u, &s_abort)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t aH = tmem + Cf::TM_H + pb * NH;
          for (int q = 0; q < Cf::W2S; ++q) {
            uint32_t b;
            if (!take(b)) {
              stop = true;
              break;
            }
            const int s = q & 1, half = q >> 1;
            // k step 4 s + kk (hidden columns 64 s + 16 kk ..): the BF16 pairs
            // the warp of slot (4 s + kk) / 2 wrote, 8 columns from the start
            // of its 32-column region for odd steps
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_ts(tmem + Cf::TM_O + 128 * half, aH + (uint32_t)(64 * s + 32 * (kk >> 1) + 8 * (kk & 1)),
                     smem_desc(b + kk * 32, 16, 1024), Cf::IDESC, (j > 1 || s > 0 || kk > 0) ? 1u : 0u);
            release();
          }
          if (stop) break;
          mma_commit(&hs_empty[pb]);
        }
      }
      if (stop) break;
      mma_commit(&o_full);
      g += NCH;
    }
    mma_commit(&done_bar);
  } else if (warp >= 2) {
    // ---------------- epilogue warps: warp w reaches TMEM lane quarter w % 4
    // (rows quarter * 32 + lane); its slot (w - 2) / 4 picks hidden columns
    // 32 slot .. + 31 of each chunk and output columns (C / 4) slot .. + C / 4
    constexpr int OC = C / 128;  // 32-column output pieces per warp
    const int quarter = warp & 3, slot = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t ti = 0, g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++ti) {
      const int r = quarter * 32 + lane, m = t * MB + r;
      const bool mok = m < M;
      for (int j = 0; j < NCH; ++j) {
        const uint32_t gj = g + j, hb = gj & 1u, u = gj >> 1;
        float4 bq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) bq[q] = reinterpret_cast<const float4 *>(b1 + NH * j + 32 * slot)[q];
        ok = __all_sync(0xffffffffu, mbar_wait(&h_full[hb], u & 1u, &s_abort));
        if (!ok) break;
        tc_fence_after();
        uint32_t v[32];
        const uint32_t hcol = lane_base + Cf::TM_H + hb * NH + 32 * slot;
        tmem_ld32(hcol, v);
        // hidden columns 32 slot + 2 i, + 1: bias, ReLU, a BF16 pair into
        // column 32 slot + i of the same buffer (this warp's own columns)
        uint32_t pk[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float4 bb = bq[i >> 1];
          const float b0 = (i & 1) ? bb.z : bb.x, b1v = (i & 1) ? bb.w : bb.y;
          pk[i] = pack_bf16x2(fmaxf(__uint_as_float(v[2 * i]) + b0, 0.f), fmaxf(__uint_as_float(v[2 * i + 1]) + b1v, 0.f));
        }
        tmem_st16(hcol, pk);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&hs_full[hb]);
      }
      if (!ok) break;
      // the tile's output, columns (C / 4) slot + 32 c + 8 q .. + 7: the
      // residual row requested before the accumulator wait
      const int col0 = (C / 4) * slot;
      uint4 rq[OC][4];
#pragma unroll
      for (int c = 0; c < OC; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          rq[c][q] = mok ? reinterpret_cast<const uint4 *>(res + (int64_t)m * C + col0 + 32 * c)[q]
                         : make_uint4(0u, 0u, 0u, 0u);
      ok = __all_sync(0xffffffffu, mbar_wait(&o_full, ti & 1u, &s_abort));
      if (!ok) break;
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < OC; ++c) {
        uint32_t v[32];
        tmem_ld32(lane_base + Cf::TM_O + col0 + 32 * c, v);
        if (mok) {
          uint4 *op = reinterpret_cast<uint4 *>(out + (int64_t)m * C + col0 + 32 * c);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t rr[4] = {rq[c][q].x, rq[c][q].y, rq[c][q].z, rq[c][q].w};
            const float4 bl = reinterpret_cast<const float4 *>(b2 + col0 + 32 * c + 8 * q)[0];
            const float4 bh = reinterpret_cast<const float4 *>(b2 + col0 + 32 * c + 8 * q)[1];
            const float bv[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
            float f[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float rv = __uint_as_float(e & 1 ? (rr[e >> 1] & 0xffff0000u) : (rr[e >> 1] << 16));
              f[e] = (__uint_as_float(v[8 * q + e]) + bv[e]) + rv;
            }
            op[q] = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                               pack_bf16x2(f[6], f[7]));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&o_empty);
      g += NCH;
    }
  }
  __syncwarp();
  // every MMA issued has completed before tensor memory is released
  if (threadIdx.x == 0) mbar_drain(&done_bar, 0);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

__global__ void mlp_debug_wait_kernel(int64_t limit_ns) {
  pdl_entry();
  debug_wait_body(limit_ns);
}

bool map_rows_k64(CUtensorMap *tm, const void *p, uint64_t inner, uint64_t rows) {
  const uint64_t dims[3] = {inner, rows, 1};
  const uint64_t st[2] = {inner * 2, inner * rows * 2};
  const uint32_t box[3] = {64, 128, 1};
  return make_tmap_nd(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, p, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

template <int C>
cudaError_t mlp_go(const CUtensorMap &tx, const CUtensorMap &t1, const CUtensorMap &t2, const float *b1,
                   const float *b2, const void *res, void *out, int M, int N1, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(mlp_fused_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, MlpCfg<C>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidValue;
  const int ntiles = (M + MB - 1) / MB;
  return launch_k(mlp_fused_kernel<C>, std::min(ntiles, sms), MLP_THREADS, MlpCfg<C>::SMEM, s, tx, t1, t2, b1, b2,
                  (const bf16 *)res, (bf16 *)out, M, N1);
}

bool a16p(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

bool mlp_fused_supported(int64_t M, int C, int N1, const void *xn, const void *w1, const float *b1, const void *w2,
                         const float *b2, const void *res, const void *out) {
  return M > 0 && M < (1ll << 31) && (C == 128 || C == 256) && N1 > 0 && N1 % NH == 0 && a16p(xn) && a16p(w1) &&
         a16p(b1) && a16p(w2) && a16p(b2) && a16p(res) && a16p(out);
}

cudaError_t mlp_fused_tc(const void *xn, const void *w1, const float *b1, const void *w2, const float *b2,
                         const void *res, void *out, int64_t M, int C, int N1, cudaStream_t s) {
  if (!mlp_fused_supported(M, C, N1, xn, w1, b1, w2, b2, res, out)) return cudaErrorInvalidValue;
  // algorithmic bytes: xn, the residual and the output once, the weights once
  Prof p("mlp_fused", s, 4.0 * (double)M * N1 * C, 2.0 * (3.0 * (double)M * C + 2.0 * (double)N1 * C));
  CUtensorMap tx, t1, t2;
  if (!map_rows_k64(&tx, xn, (uint64_t)C, (uint64_t)M) || !map_rows_k64(&t1, w1, (uint64_t)C, (uint64_t)N1) ||
      !map_rows_k64(&t2, w2, (uint64_t)N1, (uint64_t)C))
    return cudaErrorInvalidValue;
  return C == 256 ? mlp_go<256>(tx, t1, t2, b1, b2, res, out, (int)M, N1, s)
                  : mlp_go<128>(tx, t1, t2, b1, b2, res, out, (int)M, N1, s);
}

cudaError_t mlp_tc_error_read_clear(int *out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, tc_error_word, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(tc_error_word, &zero, sizeof(int));
}

cudaError_t mlp_tc_debug_wait(int64_t limit_ns, cudaStream_t s) {
  Prof p("debug_wait", s);
  launch_k(mlp_debug_wait_kernel, 1, 32, 0, s, limit_ns);
  return cudaGetLastError();
}

}  // namespace evo
