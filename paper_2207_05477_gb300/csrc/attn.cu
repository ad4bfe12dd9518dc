// Gated self-attention with pair bias and key mask, one attention axis at a
// time (MSA row, MSA column, triangle start / end node): the operator that the
// paper fuses ("Fused Gated Self-Attention", Sec. 3.1, Fig. 2).  Unlike the
// paper's operator, which keeps the softmax as a separate kernel and stores
// the logits in place (Sec. 3.4.3), the logits never reach memory here: the
// forward is an online-softmax pass over key tiles that adds the pair bias and
// mask in registers and applies the sigmoid gate in the epilogue, saving only
// the row log-sum-exp (log2 domain) for the backward, which recomputes the
// probabilities tile by tile.
//
// Two implementations of the same arithmetic:
//  * BF16 tensor-core path: mma.sync m16n8k16 (BF16 in, FP32 accumulate),
//    64 queries x 64 keys per tile, 4 warps of 16 rows, cp.async double
//    buffering.  Head dims 8/16/32 (padded to a multiple of 16).
//  * FP32 plain path: SIMT, one thread per query (forward, dq) or per key
//    (dk, dv).
// dQ and the pair-bias gradient (summed over the batch axis: MSA rows for row
// attention, the fixed node for triangle attention) are accumulated with FP32
// atomics into caller-zeroed buffers.
#include "kernels.h"

namespace evo {
namespace {

constexpr float POS_INF = __builtin_huge_valf();
constexpr float NEG_INF = -__builtin_huge_valf();

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(su32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(su32(p)));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// Coalesced copy of the pair-bias tile bias[h][x0 + r][y0 + q] (r, q < 64) into
// shared memory, pre-scaled by log2(e); zero outside [X, Y).  The bias is bf16
// or fp32 (a.bias_bf16).
__device__ __forceinline__ void load_bias_tile(float (*dst)[68], const AttnArgs &a, int h, int x0, int y0) {
  for (int idx = threadIdx.x; idx < 64 * 16; idx += blockDim.x) {
    const int r = idx >> 4, q4 = (idx & 15) * 4;
    const int x = x0 + r, y = y0 + q4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (x < a.X) {
      const int64_t o = (int64_t)h * a.sBh + (int64_t)x * a.sBx + y;
      if (a.bias_bf16) {
        const bf16 *p = (const bf16 *)a.bias + o;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (y + k < a.Y) v[k] = __bfloat162float(p[k]);
      } else {
        const float *p = (const float *)a.bias + o;
        const bool vec = ((a.sBx & 3) == 0) && ((a.sBh & 3) == 0) && (((uintptr_t)a.bias & 15u) == 0);
        if (vec && y + 3 < a.Y) {
          const float4 f = *reinterpret_cast<const float4 *>(p);
          v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (y + k < a.Y) v[k] = p[k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[r][q4 + k] = v[k] * EVO_LOG2E;
  }
}

__device__ __forceinline__ void red_add_v2(float *p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Copies a [64 x c] bf16 tile (rows r0.., row stride ld elements) into smem
// rows of LD elements, zero-filling rows >= nrows and columns >= c.
template <int CP, int LD>
__device__ __forceinline__ void load_tile(bf16 (*dst)[LD], const bf16 *src, int64_t ld, int r0, int nrows, int c) {
  constexpr int CH = CP / 8;
  for (int idx = threadIdx.x; idx < 64 * CH; idx += blockDim.x) {
    const int r = idx / CH, ch = idx % CH;
    bf16 *d = &dst[r][ch * 8];
    if (r0 + r < nrows && ch * 8 < c) cp_async16(d, src + (int64_t)(r0 + r) * ld + ch * 8);
    else *reinterpret_cast<uint4 *>(d) = make_uint4(0, 0, 0, 0);
  }
}

// ------------------------------------------------------------------ BF16 fwd
template <int CP>
__global__ void __launch_bounds__(128) attn_fwd_mma(AttnArgs a) {
  pdl_entry();
  constexpr int LD = CP + 8;
  __shared__ __align__(16) bf16 Qs[64][LD];
  __shared__ __align__(16) bf16 Ks[2][64][LD];
  __shared__ __align__(16) bf16 Vs[2][64][LD];
  __shared__ float Ms[2][64];
  __shared__ float Bs[64][68];  // pair-bias tile (log2 units) of the current key tile
  const int b = blockIdx.z, h = blockIdx.y, x0 = blockIdx.x * 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  const int c = a.c;
  const bf16 *qb = (const bf16 *)a.q + (int64_t)b * a.sQb + h * c;
  const bf16 *kb = (const bf16 *)a.k + (int64_t)b * a.sKb + h * c;
  const bf16 *vb = (const bf16 *)a.v + (int64_t)b * a.sKb + h * c;
  const float sl2 = a.scale * EVO_LOG2E;
  const int nkt = (a.Y + 63) / 64;

  auto load_kv = [&](int kt, int buf) {
    const int y0 = kt * 64;
    load_tile<CP, LD>(Ks[buf], kb, a.sKy, y0, a.Y, c);
    load_tile<CP, LD>(Vs[buf], vb, a.sKy, y0, a.Y, c);
    for (int r = threadIdx.x; r < 64; r += blockDim.x) {
      const int y = y0 + r;
      float ok = y < a.Y ? 1.f : 0.f;
      if (ok != 0.f && a.mask) ok = a.mask[(int64_t)b * a.sMb + (int64_t)y * a.sMy] != 0.f ? 1.f : 0.f;
      Ms[buf][r] = ok;
    }
  };

  load_tile<CP, LD>(Qs, qb, a.sQx, x0, a.X, c);
  load_kv(0, 0);
  cp_commit();

  uint32_t qa[CP / 16][4];
  float o[CP / 8][4];
#pragma unroll
  for (int i = 0; i < CP / 8; ++i) o[i][0] = o[i][1] = o[i][2] = o[i][3] = 0.f;
  float mrow[2] = {NEG_INF, NEG_INF}, lrow[2] = {0.f, 0.f};
  const int xr[2] = {x0 + warp * 16 + gq, x0 + warp * 16 + gq + 8};

  for (int kt = 0; kt < nkt; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nkt) {
      load_kv(kt + 1, buf ^ 1);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    if (a.bias) load_bias_tile(Bs, a, h, x0, kt * 64);
    __syncthreads();
    if (kt == 0) {
#pragma unroll
      for (int ks = 0; ks < CP / 16; ++ks) {
        const int j = lane >> 3;
        ldsm_x4(qa[ks], &Qs[warp * 16 + (j & 1) * 8 + (lane & 7)][ks * 16 + (j >> 1) * 8]);
      }
    }
    float s[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) s[nt][0] = s[nt][1] = s[nt][2] = s[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < CP / 16; ++ks) {
#pragma unroll
      for (int nt = 0; nt < 8; nt += 2) {
        uint32_t r[4];
        const int j = lane >> 3;
        ldsm_x4(r, &Ks[buf][(nt + (j >> 1)) * 8 + (lane & 7)][ks * 16 + (j & 1) * 8]);
        mma16816(s[nt], qa[ks], r[0], r[1]);
        mma16816(s[nt + 1], qa[ks], r[2], r[3]);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int kc = nt * 8 + 2 * t + (e & 1);
        float v = s[nt][e] * sl2;
        if (a.bias) v += Bs[warp * 16 + gq + 8 * (e >> 1)][kc];
        s[nt][e] = Ms[buf][kc] != 0.f ? v : NEG_INF;
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float mt = NEG_INF;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) mt = fmaxf(mt, fmaxf(s[nt][2 * r], s[nt][2 * r + 1]));
      mt = fmaxf(mt, __shfl_xor_sync(0xffffffffu, mt, 1));
      mt = fmaxf(mt, __shfl_xor_sync(0xffffffffu, mt, 2));
      const float mnew = fmaxf(mrow[r], mt);
      const float muse = mnew == NEG_INF ? 0.f : mnew;
      const float alpha = exp2f(mrow[r] - muse);
      float sum = 0.f;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        s[nt][2 * r] = exp2f(s[nt][2 * r] - muse);
        s[nt][2 * r + 1] = exp2f(s[nt][2 * r + 1] - muse);
        sum += s[nt][2 * r] + s[nt][2 * r + 1];
      }
      lrow[r] = lrow[r] * alpha + sum;
#pragma unroll
      for (int dn = 0; dn < CP / 8; ++dn) {
        o[dn][2 * r] *= alpha;
        o[dn][2 * r + 1] *= alpha;
      }
      mrow[r] = mnew;
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t pa[4];
      pa[0] = pack_bf16(s[2 * kk][0], s[2 * kk][1]);
      pa[1] = pack_bf16(s[2 * kk][2], s[2 * kk][3]);
      pa[2] = pack_bf16(s[2 * kk + 1][0], s[2 * kk + 1][1]);
      pa[3] = pack_bf16(s[2 * kk + 1][2], s[2 * kk + 1][3]);
#pragma unroll
      for (int dp = 0; dp < CP / 8; dp += 2) {
        uint32_t r[4];
        const int j = lane >> 3;
        ldsm_x4_t(r, &Vs[buf][kk * 16 + (j & 1) * 8 + (lane & 7)][(dp + (j >> 1)) * 8]);
        mma16816(o[dp], pa, r[0], r[1]);
        mma16816(o[dp + 1], pa, r[2], r[3]);
      }
    }
    __syncthreads();
  }

  bf16 *oatt = (bf16 *)a.o_att + (int64_t)b * a.sOb + h * c;
  bf16 *ogate = (bf16 *)a.o_gate + (int64_t)b * a.sOb + h * c;
  const bf16 *gb = (const bf16 *)a.g + (int64_t)b * a.sQb + h * c;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    float l = lrow[r];
    l += __shfl_xor_sync(0xffffffffu, l, 1);
    l += __shfl_xor_sync(0xffffffffu, l, 2);
    const int x = xr[r];
    if (x >= a.X) continue;
    const float inv = l > 0.f ? 1.f / l : 0.f;
    const float muse = mrow[r] == NEG_INF ? 0.f : mrow[r];
    if (t == 0) a.lse2[((int64_t)b * a.H + h) * a.X + x] = l > 0.f ? muse + log2f(l) : POS_INF;
#pragma unroll
    for (int dn = 0; dn < CP / 8; ++dn) {
      const int d = dn * 8 + 2 * t;
      if (d >= c) continue;
      const float v0 = o[dn][2 * r] * inv, v1 = o[dn][2 * r + 1] * inv;
      const __nv_bfloat162 gg = *reinterpret_cast<const __nv_bfloat162 *>(gb + (int64_t)x * a.sQx + d);
      *reinterpret_cast<uint32_t *>(oatt + (int64_t)x * a.sOx + d) = pack_bf16(v0, v1);
      *reinterpret_cast<uint32_t *>(ogate + (int64_t)x * a.sOx + d) =
          pack_bf16(v0 * __low2float(gg), v1 * __high2float(gg));
    }
  }
}

// ------------------------------------------------------------------ BF16 bwd
// CTA = (key tile of 64, head, batch); warp w owns keys 16w..16w+15 and loops
// over all query tiles: S^T = K Q^T, dP^T = V dO^T, P^T = exp2(S^T - lse),
// dS^T = P^T (dP^T - D); dV += P^T dO, dK += dS^T Q; dQ = dS K via shared
// memory and atomics; dbias += dS via atomics.
template <int CP>
__global__ void __launch_bounds__(128) attn_bwd_mma(AttnArgs a) {
  pdl_entry();
  constexpr int LD = CP + 8;
  __shared__ __align__(16) bf16 Ks[64][LD];
  __shared__ __align__(16) bf16 Vs[64][LD];
  __shared__ __align__(16) bf16 Qs[64][LD];
  __shared__ __align__(16) bf16 dOs[64][LD];
  __shared__ __align__(16) bf16 dSs[64][64 + 8];  // [query][key]
  __shared__ float dSf[64][68];                    // [query][key]: bias tile, then dS
  __shared__ float lse_s[64], D_s[64], kval[64];
  const int b = blockIdx.z, h = blockIdx.y, y0 = blockIdx.x * 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  const int c = a.c;
  const float sl2 = a.scale * EVO_LOG2E;
  const bf16 *qb = (const bf16 *)a.q + (int64_t)b * a.sQb + h * c;
  const bf16 *kb = (const bf16 *)a.k + (int64_t)b * a.sKb + h * c;
  const bf16 *vb = (const bf16 *)a.v + (int64_t)b * a.sKb + h * c;
  const bf16 *dob = (const bf16 *)a.do_att + (int64_t)b * a.sOb + h * c;

  load_tile<CP, LD>(Ks, kb, a.sKy, y0, a.Y, c);
  load_tile<CP, LD>(Vs, vb, a.sKy, y0, a.Y, c);
  cp_commit();
  for (int r = threadIdx.x; r < 64; r += blockDim.x) {
    const int y = y0 + r;
    float ok = y < a.Y ? 1.f : 0.f;
    if (ok != 0.f && a.mask) ok = a.mask[(int64_t)b * a.sMb + (int64_t)y * a.sMy] != 0.f ? 1.f : 0.f;
    kval[r] = ok;
  }
  cp_wait<0>();
  __syncthreads();
  uint32_t ka[CP / 16][4], va[CP / 16][4];
#pragma unroll
  for (int ks = 0; ks < CP / 16; ++ks) {
    const int j = lane >> 3;
    ldsm_x4(ka[ks], &Ks[warp * 16 + (j & 1) * 8 + (lane & 7)][ks * 16 + (j >> 1) * 8]);
    ldsm_x4(va[ks], &Vs[warp * 16 + (j & 1) * 8 + (lane & 7)][ks * 16 + (j >> 1) * 8]);
  }
  float dk[CP / 8][4], dv[CP / 8][4];
#pragma unroll
  for (int i = 0; i < CP / 8; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) dk[i][e] = dv[i][e] = 0.f;

  const int kr[2] = {warp * 16 + gq, warp * 16 + gq + 8};
  for (int x0 = 0; x0 < a.X; x0 += 64) {
    load_tile<CP, LD>(Qs, qb, a.sQx, x0, a.X, c);
    load_tile<CP, LD>(dOs, dob, a.sOx, x0, a.X, c);
    cp_commit();
    for (int r = threadIdx.x; r < 64; r += blockDim.x) {
      const int x = x0 + r;
      const int64_t li = ((int64_t)b * a.H + h) * a.X + x;
      lse_s[r] = x < a.X ? a.lse2[li] : POS_INF;
      D_s[r] = x < a.X ? a.Dsum[li] : 0.f;
    }
    if (a.bias) load_bias_tile(dSf, a, h, x0, y0);
    cp_wait<0>();
    __syncthreads();
    float st[8][4], dp[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) st[nt][e] = dp[nt][e] = 0.f;
#pragma unroll
    for (int ks = 0; ks < CP / 16; ++ks) {
#pragma unroll
      for (int nt = 0; nt < 8; nt += 2) {
        uint32_t r[4];
        const int j = lane >> 3;
        ldsm_x4(r, &Qs[(nt + (j >> 1)) * 8 + (lane & 7)][ks * 16 + (j & 1) * 8]);
        mma16816(st[nt], ka[ks], r[0], r[1]);
        mma16816(st[nt + 1], ka[ks], r[2], r[3]);
        ldsm_x4(r, &dOs[(nt + (j >> 1)) * 8 + (lane & 7)][ks * 16 + (j & 1) * 8]);
        mma16816(dp[nt], va[ks], r[0], r[1]);
        mma16816(dp[nt + 1], va[ks], r[2], r[3]);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int qc = nt * 8 + 2 * t + (e & 1);
        const int krow = kr[e >> 1];
        const int x = x0 + qc, y = y0 + krow;
        float p = 0.f;
        if (kval[krow] != 0.f && x < a.X) {
          float v = st[nt][e] * sl2;
          if (a.bias) v += dSf[qc][krow];
          p = exp2f(v - lse_s[qc]);
        }
        const float ds = p * (dp[nt][e] - D_s[qc]);
        st[nt][e] = p;
        dp[nt][e] = ds;
        dSs[qc][krow] = __float2bfloat16_rn(ds);
      }
    }
    if (a.bias) {
      __syncthreads();  // every thread has read its bias values
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) dSf[nt * 8 + 2 * t + (e & 1)][kr[e >> 1]] = dp[nt][e];
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t pa[4], sa[4];
      pa[0] = pack_bf16(st[2 * kk][0], st[2 * kk][1]);
      pa[1] = pack_bf16(st[2 * kk][2], st[2 * kk][3]);
      pa[2] = pack_bf16(st[2 * kk + 1][0], st[2 * kk + 1][1]);
      pa[3] = pack_bf16(st[2 * kk + 1][2], st[2 * kk + 1][3]);
      sa[0] = pack_bf16(dp[2 * kk][0], dp[2 * kk][1]);
      sa[1] = pack_bf16(dp[2 * kk][2], dp[2 * kk][3]);
      sa[2] = pack_bf16(dp[2 * kk + 1][0], dp[2 * kk + 1][1]);
      sa[3] = pack_bf16(dp[2 * kk + 1][2], dp[2 * kk + 1][3]);
#pragma unroll
      for (int dd = 0; dd < CP / 8; dd += 2) {
        uint32_t r[4];
        const int j = lane >> 3;
        ldsm_x4_t(r, &dOs[kk * 16 + (j & 1) * 8 + (lane & 7)][(dd + (j >> 1)) * 8]);
        mma16816(dv[dd], pa, r[0], r[1]);
        mma16816(dv[dd + 1], pa, r[2], r[3]);
        ldsm_x4_t(r, &Qs[kk * 16 + (j & 1) * 8 + (lane & 7)][(dd + (j >> 1)) * 8]);
        mma16816(dk[dd], sa, r[0], r[1]);
        mma16816(dk[dd + 1], sa, r[2], r[3]);
      }
    }
    __syncthreads();
    // dQ rows 16w..16w+15 of this query tile = dS[16 x 64 keys] K[64 keys x c]
    {
      float dq[CP / 8][4];
#pragma unroll
      for (int i = 0; i < CP / 8; ++i) dq[i][0] = dq[i][1] = dq[i][2] = dq[i][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        uint32_t af[4];
        const int j = lane >> 3;
        ldsm_x4(af, &dSs[warp * 16 + (j & 1) * 8 + (lane & 7)][kk * 16 + (j >> 1) * 8]);
#pragma unroll
        for (int dd = 0; dd < CP / 8; dd += 2) {
          uint32_t r[4];
          ldsm_x4_t(r, &Ks[kk * 16 + (j & 1) * 8 + (lane & 7)][(dd + (j >> 1)) * 8]);
          mma16816(dq[dd], af, r[0], r[1]);
          mma16816(dq[dd + 1], af, r[2], r[3]);
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int x = x0 + warp * 16 + gq + 8 * r;
        if (x >= a.X) continue;
        float *dst = a.dq_acc + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * c;
#pragma unroll
        for (int dd = 0; dd < CP / 8; ++dd) {
          const int d = dd * 8 + 2 * t;
          if (d < c) red_add_v2(dst + d, dq[dd][2 * r], dq[dd][2 * r + 1]);
        }
      }
    }
    if (a.dbias) {
      const bool vec = ((a.sBx & 3) == 0) && ((a.sBh & 3) == 0) && (((uintptr_t)a.dbias & 15u) == 0);
      for (int idx = threadIdx.x; idx < 64 * 16; idx += blockDim.x) {
        const int qc = idx >> 4, k4 = (idx & 15) * 4;
        const int x = x0 + qc, y = y0 + k4;
        if (x >= a.X || y >= a.Y) continue;
        float *dst = a.dbias + (int64_t)h * a.sBh + (int64_t)x * a.sBx + y;
        const float v0 = dSf[qc][k4], v1 = dSf[qc][k4 + 1], v2 = dSf[qc][k4 + 2], v3 = dSf[qc][k4 + 3];
        if (vec && y + 3 < a.Y) {
          if (v0 != 0.f || v1 != 0.f || v2 != 0.f || v3 != 0.f) red_add_v4(dst, v0, v1, v2, v3);
        } else {
          if (v0 != 0.f) atomicAdd(dst, v0);
          if (y + 1 < a.Y && v1 != 0.f) atomicAdd(dst + 1, v1);
          if (y + 2 < a.Y && v2 != 0.f) atomicAdd(dst + 2, v2);
          if (y + 3 < a.Y && v3 != 0.f) atomicAdd(dst + 3, v3);
        }
      }
    }
    __syncthreads();
  }
  bf16 *dkb = (bf16 *)a.dk + (int64_t)b * a.sKb + h * c;
  bf16 *dvb = (bf16 *)a.dv + (int64_t)b * a.sKb + h * c;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int y = y0 + kr[r];
    if (y >= a.Y) continue;
#pragma unroll
    for (int dd = 0; dd < CP / 8; ++dd) {
      const int d = dd * 8 + 2 * t;
      if (d >= c) continue;
      *reinterpret_cast<uint32_t *>(dkb + (int64_t)y * a.sKy + d) =
          pack_bf16(dk[dd][2 * r] * a.scale, dk[dd][2 * r + 1] * a.scale);
      *reinterpret_cast<uint32_t *>(dvb + (int64_t)y * a.sKy + d) = pack_bf16(dv[dd][2 * r], dv[dd][2 * r + 1]);
    }
  }
}

// ------------------------------------------------------------------ FP32 plain
template <int CM>
__global__ void __launch_bounds__(128) attn_fwd_simt(AttnArgs a) {
  pdl_entry();
  __shared__ float Ks[32][CM], Vs[32][CM];
  __shared__ float Mk[32];
  const int b = blockIdx.z, h = blockIdx.y;
  const int x = blockIdx.x * 128 + threadIdx.x;
  const int c = a.c;
  const float *qp = (const float *)a.q + (int64_t)b * a.sQb + (int64_t)x * a.sQx + h * c;
  const float *kb = (const float *)a.k + (int64_t)b * a.sKb + h * c;
  const float *vb = (const float *)a.v + (int64_t)b * a.sKb + h * c;
  const float sl2 = a.scale * EVO_LOG2E;
  float q[CM], o[CM];
  const bool live = x < a.X;
#pragma unroll
  for (int d = 0; d < CM; ++d) {
    q[d] = (live && d < c) ? qp[d] : 0.f;
    o[d] = 0.f;
  }
  float mrow = NEG_INF, l = 0.f;
  for (int y0 = 0; y0 < a.Y; y0 += 32) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * CM; idx += blockDim.x) {
      const int r = idx / CM, d = idx % CM, y = y0 + r;
      const bool ok = y < a.Y && d < c;
      Ks[r][d] = ok ? kb[(int64_t)y * a.sKy + d] : 0.f;
      Vs[r][d] = ok ? vb[(int64_t)y * a.sKy + d] : 0.f;
    }
    for (int r = threadIdx.x; r < 32; r += blockDim.x) {
      const int y = y0 + r;
      float ok = y < a.Y ? 1.f : 0.f;
      if (ok != 0.f && a.mask) ok = a.mask[(int64_t)b * a.sMb + (int64_t)y * a.sMy] != 0.f ? 1.f : 0.f;
      Mk[r] = ok;
    }
    __syncthreads();
    if (!live) continue;
    for (int r = 0; r < 32 && y0 + r < a.Y; ++r) {
      if (Mk[r] == 0.f) continue;
      float sdot = 0.f;
#pragma unroll
      for (int d = 0; d < CM; ++d) sdot = fmaf(q[d], Ks[r][d], sdot);
      float s = sdot * sl2;
      if (a.bias) s += ((const float *)a.bias)[(int64_t)h * a.sBh + (int64_t)x * a.sBx + y0 + r] * EVO_LOG2E;
      const float mnew = fmaxf(mrow, s);
      const float alpha = exp2f(mrow - mnew);
      const float p = exp2f(s - mnew);
      l = l * alpha + p;
#pragma unroll
      for (int d = 0; d < CM; ++d) o[d] = o[d] * alpha + p * Vs[r][d];
      mrow = mnew;
    }
  }
  if (!live) return;
  const float inv = l > 0.f ? 1.f / l : 0.f;
  float *oatt = (float *)a.o_att + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * c;
  float *ogate = (float *)a.o_gate + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * c;
  const float *gp = (const float *)a.g + (int64_t)b * a.sQb + (int64_t)x * a.sQx + h * c;
  for (int d = 0; d < c; ++d) {
    const float v = o[d] * inv;
    oatt[d] = v;
    ogate[d] = v * gp[d];
  }
  a.lse2[((int64_t)b * a.H + h) * a.X + x] = l > 0.f ? mrow + log2f(l) : POS_INF;
}

// dq (unscaled, into dq_acc) and dbias: one thread per query.
template <int CM>
__global__ void __launch_bounds__(128) attn_bwd_dq_simt(AttnArgs a) {
  pdl_entry();
  __shared__ float Ks[32][CM], Vs[32][CM];
  __shared__ float Mk[32];
  const int b = blockIdx.z, h = blockIdx.y;
  const int x = blockIdx.x * 128 + threadIdx.x;
  const int c = a.c;
  const bool live = x < a.X;
  const float sl2 = a.scale * EVO_LOG2E;
  const float *kb = (const float *)a.k + (int64_t)b * a.sKb + h * c;
  const float *vb = (const float *)a.v + (int64_t)b * a.sKb + h * c;
  float q[CM], dO[CM], dq[CM];
  const float *qp = (const float *)a.q + (int64_t)b * a.sQb + (int64_t)x * a.sQx + h * c;
  const float *dop = (const float *)a.do_att + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * c;
#pragma unroll
  for (int d = 0; d < CM; ++d) {
    q[d] = (live && d < c) ? qp[d] : 0.f;
    dO[d] = (live && d < c) ? dop[d] : 0.f;
    dq[d] = 0.f;
  }
  const int64_t li = ((int64_t)b * a.H + h) * a.X + x;
  const float lse = live ? a.lse2[li] : POS_INF;
  const float Dx = live ? a.Dsum[li] : 0.f;
  for (int y0 = 0; y0 < a.Y; y0 += 32) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * CM; idx += blockDim.x) {
      const int r = idx / CM, d = idx % CM, y = y0 + r;
      const bool ok = y < a.Y && d < c;
      Ks[r][d] = ok ? kb[(int64_t)y * a.sKy + d] : 0.f;
      Vs[r][d] = ok ? vb[(int64_t)y * a.sKy + d] : 0.f;
    }
    for (int r = threadIdx.x; r < 32; r += blockDim.x) {
      const int y = y0 + r;
      float ok = y < a.Y ? 1.f : 0.f;
      if (ok != 0.f && a.mask) ok = a.mask[(int64_t)b * a.sMb + (int64_t)y * a.sMy] != 0.f ? 1.f : 0.f;
      Mk[r] = ok;
    }
    __syncthreads();
    if (!live) continue;
    for (int r = 0; r < 32 && y0 + r < a.Y; ++r) {
      if (Mk[r] == 0.f) continue;
      float sdot = 0.f, dpv = 0.f;
#pragma unroll
      for (int d = 0; d < CM; ++d) {
        sdot = fmaf(q[d], Ks[r][d], sdot);
        dpv = fmaf(dO[d], Vs[r][d], dpv);
      }
      float s = sdot * sl2;
      if (a.bias) s += ((const float *)a.bias)[(int64_t)h * a.sBh + (int64_t)x * a.sBx + y0 + r] * EVO_LOG2E;
      const float p = exp2f(s - lse);
      const float ds = p * (dpv - Dx);
#pragma unroll
      for (int d = 0; d < CM; ++d) dq[d] = fmaf(ds, Ks[r][d], dq[d]);
      if (a.dbias && ds != 0.f) atomicAdd(a.dbias + (int64_t)h * a.sBh + (int64_t)x * a.sBx + y0 + r, ds);
    }
  }
  if (!live) return;
  float *dst = a.dq_acc + (int64_t)b * a.sOb + (int64_t)x * a.sOx + h * c;
  for (int d = 0; d < c; ++d) dst[d] += dq[d];
}

// dk, dv: one thread per key.
template <int CM>
__global__ void __launch_bounds__(128) attn_bwd_dkv_simt(AttnArgs a) {
  pdl_entry();
  __shared__ float Qs[32][CM], dOs[32][CM];
  __shared__ float Ls[32], Ds[32];
  const int b = blockIdx.z, h = blockIdx.y;
  const int y = blockIdx.x * 128 + threadIdx.x;
  const int c = a.c;
  bool live = y < a.Y;
  if (live && a.mask) live = a.mask[(int64_t)b * a.sMb + (int64_t)y * a.sMy] != 0.f;
  const float sl2 = a.scale * EVO_LOG2E;
  const float *qb = (const float *)a.q + (int64_t)b * a.sQb + h * c;
  const float *dob = (const float *)a.do_att + (int64_t)b * a.sOb + h * c;
  float k[CM], v[CM], dk[CM], dv[CM];
  const float *kp = (const float *)a.k + (int64_t)b * a.sKb + (int64_t)y * a.sKy + h * c;
  const float *vp = (const float *)a.v + (int64_t)b * a.sKb + (int64_t)y * a.sKy + h * c;
#pragma unroll
  for (int d = 0; d < CM; ++d) {
    const bool ok = live && d < c;
    k[d] = ok ? kp[d] : 0.f;
    v[d] = ok ? vp[d] : 0.f;
    dk[d] = dv[d] = 0.f;
  }
  for (int x0 = 0; x0 < a.X; x0 += 32) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * CM; idx += blockDim.x) {
      const int r = idx / CM, d = idx % CM, x = x0 + r;
      const bool ok = x < a.X && d < c;
      Qs[r][d] = ok ? qb[(int64_t)x * a.sQx + d] : 0.f;
      dOs[r][d] = ok ? dob[(int64_t)x * a.sOx + d] : 0.f;
    }
    for (int r = threadIdx.x; r < 32; r += blockDim.x) {
      const int x = x0 + r;
      const int64_t li = ((int64_t)b * a.H + h) * a.X + x;
      Ls[r] = x < a.X ? a.lse2[li] : POS_INF;
      Ds[r] = x < a.X ? a.Dsum[li] : 0.f;
    }
    __syncthreads();
    if (!live) continue;
    for (int r = 0; r < 32 && x0 + r < a.X; ++r) {
      float sdot = 0.f, dpv = 0.f;
#pragma unroll
      for (int d = 0; d < CM; ++d) {
        sdot = fmaf(Qs[r][d], k[d], sdot);
        dpv = fmaf(dOs[r][d], v[d], dpv);
      }
      float s = sdot * sl2;
      if (a.bias) s += ((const float *)a.bias)[(int64_t)h * a.sBh + (int64_t)(x0 + r) * a.sBx + y] * EVO_LOG2E;
      const float p = exp2f(s - Ls[r]);
      const float ds = p * (dpv - Ds[r]);
#pragma unroll
      for (int d = 0; d < CM; ++d) {
        dv[d] = fmaf(p, dOs[r][d], dv[d]);
        dk[d] = fmaf(ds, Qs[r][d], dk[d]);
      }
    }
  }
  if (y >= a.Y) return;
  float *dkp = (float *)a.dk + (int64_t)b * a.sKb + (int64_t)y * a.sKy + h * c;
  float *dvp = (float *)a.dv + (int64_t)b * a.sKb + (int64_t)y * a.sKy + h * c;
  for (int d = 0; d < c; ++d) {
    dkp[d] = dk[d] * a.scale;
    dvp[d] = dv[d];
  }
}

bool mma_ok(const AttnArgs &a) {
  // 16-byte cp.async rows: head offsets, row strides and bases in multiples of 8 bf16
  auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
  if (a.c % 8 || a.c > 32) return false;
  if (a.sQb % 8 || a.sQx % 8 || a.sKb % 8 || a.sKy % 8 || a.sOb % 8 || a.sOx % 8) return false;
  return al(a.q) && al(a.k) && al(a.v) && al(a.g) && al(a.o_att) && al(a.o_gate);
}

}  // namespace

cudaError_t attn_fwd(const AttnArgs &a, int use_bf16, cudaStream_t s) {
  if (a.B1 <= 0 || a.X <= 0 || a.H <= 0) return cudaSuccess;
  const double inner = (double)a.B1 * a.H * a.X * (double)a.Y * a.c;
  const double ts = use_bf16 ? 2.0 : 4.0;
  const double io = (double)a.B1 * a.H * a.c * ((double)a.X * 4 + (double)a.Y * 2) * ts +
                    (a.bias ? 4.0 * a.H * (double)a.X * a.Y : 0.0);
  if (use_bf16 && attn_tc_supported(a)) {
    const cudaError_t e = attn_fwd_tc_launch(a, s, 4.0 * inner, io);
    if (e != cudaErrorNotSupported) return e;
  }
  Prof p(use_bf16 ? "attn_fwd_mma" : "attn_fwd_simt", s, 4.0 * inner, io);
  if (use_bf16) {
    if (!mma_ok(a)) return cudaErrorInvalidValue;
    dim3 grid((a.X + 63) / 64, a.H, a.B1);
    if (a.c <= 16) launch_k(attn_fwd_mma<16>, grid, 128, 0, s, a);
    else launch_k(attn_fwd_mma<32>, grid, 128, 0, s, a);
  } else {
    dim3 grid((a.X + 127) / 128, a.H, a.B1);
    if (a.c <= 8) launch_k(attn_fwd_simt<8>, grid, 128, 0, s, a);
    else if (a.c <= 32) launch_k(attn_fwd_simt<32>, grid, 128, 0, s, a);
    else return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// mma.sync (bf16) or SIMT (fp32) backward: dq accumulates, unscaled, in fp32
// with atomics and is then scaled into its destination.
static cudaError_t attn_bwd_accumulating(const AttnArgs &a, int use_bf16, cudaStream_t s, double flops, double io) {
  cudaError_t e = cudaMemsetAsync(a.dq_acc, 0, (size_t)a.B1 * a.X * a.H * a.c * sizeof(float), s);
  if (e != cudaSuccess) return e;
  bool done = false;
  if (use_bf16 && attn_bwd_stream_supported(a)) {
    e = attn_bwd_stream_launch(a, s, flops, io);
    if (e != cudaErrorNotSupported && e != cudaSuccess) return e;
    done = e == cudaSuccess;
  }
  if (!done) {
    Prof p(use_bf16 ? "attn_bwd_mma" : "attn_bwd_simt", s, flops, io, use_bf16 ? 1 : 2);
    if (use_bf16) {
      if (!mma_ok(a)) return cudaErrorInvalidValue;
      dim3 grid((a.Y + 63) / 64, a.H, a.B1);
      if (a.c <= 16) launch_k(attn_bwd_mma<16>, grid, 128, 0, s, a);
      else launch_k(attn_bwd_mma<32>, grid, 128, 0, s, a);
    } else {
      dim3 gq((a.X + 127) / 128, a.H, a.B1), gk((a.Y + 127) / 128, a.H, a.B1);
      if (a.c <= 8) {
        launch_k(attn_bwd_dq_simt<8>, gq, 128, 0, s, a);
        launch_k(attn_bwd_dkv_simt<8>, gk, 128, 0, s, a);
      } else if (a.c <= 32) {
        launch_k(attn_bwd_dq_simt<32>, gq, 128, 0, s, a);
        launch_k(attn_bwd_dkv_simt<32>, gk, 128, 0, s, a);
      } else {
        return cudaErrorInvalidValue;
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return attn_dq_store(a, a.dq, use_bf16, s);
}

cudaError_t attn_bwd(const AttnArgs &a, int use_bf16, cudaStream_t s) {
  if (a.B1 <= 0 || a.X <= 0 || a.H <= 0) return cudaSuccess;
  const double inner = (double)a.B1 * a.H * a.X * (double)a.Y * a.c;
  const double ts = use_bf16 ? 2.0 : 4.0;
  const double io = (double)a.B1 * a.H * a.c * ((double)a.X * (2 * ts + 4) + (double)a.Y * 4 * ts) +
                    (a.bias ? 8.0 * a.H * (double)a.X * a.Y : 0.0);
  if (use_bf16 && attn_bwd_tc_supported(a)) {
    const cudaError_t e = attn_bwd_tc_launch(a, s, 10.0 * inner, io);
    if (e != cudaErrorNotSupported) return e;
  }
  if (a.dog) {
    // the other kernels take do_att and D from a separate gate-backward pass
    const cudaError_t e = attn_gate_bwd(a, a.dog, a.dgpre, a.sQb, a.sQx, const_cast<void *>(a.do_att),
                                        const_cast<float *>(a.Dsum), use_bf16, s);
    if (e != cudaSuccess) return e;
  }
  return attn_bwd_accumulating(a, use_bf16, s, 10.0 * inner, io);
}

}  // namespace evo
