// MSA global column attention of the extra-MSA stack (AlphaFold2 Alg. 19,
// used by the ExtraMSAStack the paper trains, Sec. 2 and Table "model
// settings"): per residue column i, the query is the masked mean over the
// sequences of the H-head projection q, keys and values are single-head
// (width c), and every sequence row s receives the same attention output,
// gated by its own sigmoid gate.  The work per column is tiny (H x S logits
// of width c), so one CTA owns one column and keeps the S x H logits in
// shared memory; the cost is reading q, k, v, g and writing the gated output.
//
// Row layout of the fused projection (width ld):
//   [ q (H*c) | k (c) | v (c) | g (H*c) ],  row (s, i) at (s * R + i) * ld.
#include "kernels.h"

namespace evo {
namespace {

constexpr int NT = 256;  // threads per column
constexpr float NEG_INF_G = -__builtin_huge_valf();

template <int HC>
__device__ __forceinline__ void block_reduce_vec(float (&v)[HC], float *red /* [NT/32][HC] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < HC; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < HC; ++k) red[warp * HC + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < HC; ++k) {
    float t = 0.f;
    for (int w = 0; w < NT / 32; ++w) t += red[w * HC + k];
    v[k] = t;
  }
  __syncthreads();
}

// stats layout per column: st[(i*H + h)*2 + {0: max (log2 units), 1: sum}]
template <typename T, int H, int CD>
__global__ void __launch_bounds__(NT) gattn_fwd_k(const T *qkvg, int64_t ld, int S, int R, const float *mask,
                                                  float scale, float *qbar_out, float *obar_out, float *stats,
                                                  T *o_gate) {
  pdl_entry();
  constexpr int HC = H * CD;
  extern __shared__ float lg[];  // [S][H] logits (log2 units)
  __shared__ float red[NT / 32 * HC];
  __shared__ float qb[HC], ob[HC], mx[H], sm[H];
  const int i = blockIdx.x;
  const float sl2 = scale * EVO_LOG2E;
  // 1. masked mean of q over the sequences
  float acc[HC];
#pragma unroll
  for (int k = 0; k < HC; ++k) acc[k] = 0.f;
  float cnt = 0.f;
  for (int s = threadIdx.x; s < S; s += NT) {
    const float mk = mask[(int64_t)s * R + i];
    if (mk == 0.f) continue;
    const T *row = qkvg + ((int64_t)s * R + i) * ld;
#pragma unroll
    for (int k = 0; k < HC; ++k) acc[k] += mk * ldf(row + k);
    cnt += mk;
  }
  cnt = warp_sum(cnt);
  __shared__ float cred[NT / 32];
  if ((threadIdx.x & 31) == 0) cred[threadIdx.x >> 5] = cnt;
  block_reduce_vec<HC>(acc, red);
  float ctot = 0.f;
  for (int w = 0; w < NT / 32; ++w) ctot += cred[w];
  if (threadIdx.x < HC) qb[threadIdx.x] = acc[threadIdx.x] / (ctot + 1e-10f);
  __syncthreads();
  // 2. logits and per-head maxima
  float lmax[H];
#pragma unroll
  for (int h = 0; h < H; ++h) lmax[h] = NEG_INF_G;
  for (int t = threadIdx.x; t < S; t += NT) {
    const T *row = qkvg + ((int64_t)t * R + i) * ld + HC;
    float kv[CD];
#pragma unroll
    for (int d = 0; d < CD; ++d) kv[d] = ldf(row + d);
    const bool valid = mask[(int64_t)t * R + i] != 0.f;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      float l = 0.f;
#pragma unroll
      for (int d = 0; d < CD; ++d) l += qb[h * CD + d] * kv[d];
      l = valid ? l * sl2 : NEG_INF_G;
      lg[t * H + h] = l;
      lmax[h] = fmaxf(lmax[h], l);
    }
  }
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      lmax[h] = warp_max(lmax[h]);
      if (lane == 0) red[warp * H + h] = lmax[h];
    }
    __syncthreads();
    if (threadIdx.x < H) {
      float m = NEG_INF_G;
      for (int w = 0; w < NT / 32; ++w) m = fmaxf(m, red[w * H + threadIdx.x]);
      mx[threadIdx.x] = m == NEG_INF_G ? 0.f : m;
    }
    __syncthreads();
  }
  // 3. unnormalised probabilities, their sums, and sum_t p v
  float pv[HC], ps[H];
#pragma unroll
  for (int k = 0; k < HC; ++k) pv[k] = 0.f;
#pragma unroll
  for (int h = 0; h < H; ++h) ps[h] = 0.f;
  for (int t = threadIdx.x; t < S; t += NT) {
    const T *row = qkvg + ((int64_t)t * R + i) * ld + HC + CD;
    float vv[CD];
#pragma unroll
    for (int d = 0; d < CD; ++d) vv[d] = ldf(row + d);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float p = exp2f(lg[t * H + h] - mx[h]);
      ps[h] += p;
#pragma unroll
      for (int d = 0; d < CD; ++d) pv[h * CD + d] += p * vv[d];
    }
  }
  block_reduce_vec<HC>(pv, red);
  block_reduce_vec<H>(ps, red);
  if (threadIdx.x < HC) {
    const int h = threadIdx.x / CD;
    ob[threadIdx.x] = ps[h] > 0.f ? pv[threadIdx.x] / ps[h] : 0.f;
    qbar_out[(int64_t)i * HC + threadIdx.x] = qb[threadIdx.x];
    obar_out[(int64_t)i * HC + threadIdx.x] = ob[threadIdx.x];
  }
  if (threadIdx.x < H) {
    stats[((int64_t)i * H + threadIdx.x) * 2] = mx[threadIdx.x];
    stats[((int64_t)i * H + threadIdx.x) * 2 + 1] = ps[threadIdx.x];
    sm[threadIdx.x] = ps[threadIdx.x];
  }
  __syncthreads();
  // 4. gated output rows
  for (int s = threadIdx.x; s < S; s += NT) {
    const T *g = qkvg + ((int64_t)s * R + i) * ld + HC + 2 * CD;
    T *o = o_gate + ((int64_t)s * R + i) * HC;
#pragma unroll
    for (int k = 0; k < HC; ++k) stf(o + k, ldf(g + k) * ob[k]);
  }
}

template <typename T, int H, int CD>
__global__ void __launch_bounds__(NT) gattn_bwd_k(const T *qkvg, int64_t ld, int S, int R, const float *mask,
                                                  float scale, const float *qbar_in, const float *obar_in,
                                                  const float *stats, const T *dog, T *dqkvg) {
  pdl_entry();
  constexpr int HC = H * CD;
  extern __shared__ float lg[];  // [S][H] probabilities
  __shared__ float red[NT / 32 * HC];
  __shared__ float qb[HC], ob[HC], dob[HC], dqb[HC], Dh[H], cred[NT / 32];
  const int i = blockIdx.x;
  const float sl2 = scale * EVO_LOG2E;
  if (threadIdx.x < HC) {
    qb[threadIdx.x] = qbar_in[(int64_t)i * HC + threadIdx.x];
    ob[threadIdx.x] = obar_in[(int64_t)i * HC + threadIdx.x];
  }
  __syncthreads();
  // 1. gate gradient and d(obar) = sum_s dog * g
  float acc[HC];
#pragma unroll
  for (int k = 0; k < HC; ++k) acc[k] = 0.f;
  float cnt = 0.f;
  for (int s = threadIdx.x; s < S; s += NT) {
    const int64_t r = (int64_t)s * R + i;
    const T *g = qkvg + r * ld + HC + 2 * CD;
    const T *dg = dog + r * HC;
    T *dgp = dqkvg + r * ld + HC + 2 * CD;
#pragma unroll
    for (int k = 0; k < HC; ++k) {
      const float gv = ldf(g + k), d = ldf(dg + k);
      acc[k] += d * gv;
      stf(dgp + k, d * ob[k] * gv * (1.f - gv));
    }
    cnt += mask[r];
  }
  cnt = warp_sum(cnt);
  if ((threadIdx.x & 31) == 0) cred[threadIdx.x >> 5] = cnt;
  block_reduce_vec<HC>(acc, red);
  if (threadIdx.x < HC) dob[threadIdx.x] = acc[threadIdx.x];
  float ctot = 0.f;
  for (int w = 0; w < NT / 32; ++w) ctot += cred[w];
  __syncthreads();
  // 2. probabilities again, dp = dobar . v, and D_h = sum_t p dp
  float Dl[H];
#pragma unroll
  for (int h = 0; h < H; ++h) Dl[h] = 0.f;
  for (int t = threadIdx.x; t < S; t += NT) {
    const int64_t r = (int64_t)t * R + i;
    const T *row = qkvg + r * ld + HC;
    float kv[CD], vv[CD];
#pragma unroll
    for (int d = 0; d < CD; ++d) {
      kv[d] = ldf(row + d);
      vv[d] = ldf(row + CD + d);
    }
    const bool valid = mask[r] != 0.f;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      float p = 0.f;
      const float sum = stats[((int64_t)i * H + h) * 2 + 1];
      if (valid && sum > 0.f) {
        float l = 0.f;
#pragma unroll
        for (int d = 0; d < CD; ++d) l += qb[h * CD + d] * kv[d];
        p = exp2f(l * sl2 - stats[((int64_t)i * H + h) * 2]) / sum;
      }
      float dp = 0.f;
#pragma unroll
      for (int d = 0; d < CD; ++d) dp += dob[h * CD + d] * vv[d];
      lg[t * H + h] = p;
      Dl[h] += p * dp;
    }
  }
  block_reduce_vec<H>(Dl, red);
  if (threadIdx.x < H) Dh[threadIdx.x] = Dl[threadIdx.x];
  __syncthreads();
  // 3. dv, dk per key row, and d(qbar)
#pragma unroll
  for (int k = 0; k < HC; ++k) acc[k] = 0.f;
  for (int t = threadIdx.x; t < S; t += NT) {
    const int64_t r = (int64_t)t * R + i;
    const T *row = qkvg + r * ld + HC;
    float kv[CD], vv[CD], dk[CD], dv[CD];
#pragma unroll
    for (int d = 0; d < CD; ++d) {
      kv[d] = ldf(row + d);
      vv[d] = ldf(row + CD + d);
      dk[d] = dv[d] = 0.f;
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float p = lg[t * H + h];
      float dp = 0.f;
#pragma unroll
      for (int d = 0; d < CD; ++d) dp += dob[h * CD + d] * vv[d];
      const float dl = p * (dp - Dh[h]) * scale;
#pragma unroll
      for (int d = 0; d < CD; ++d) {
        dv[d] += p * dob[h * CD + d];
        dk[d] += dl * qb[h * CD + d];
        acc[h * CD + d] += dl * kv[d];
      }
    }
    T *drow = dqkvg + r * ld + HC;
#pragma unroll
    for (int d = 0; d < CD; ++d) {
      stf(drow + d, dk[d]);
      stf(drow + CD + d, dv[d]);
    }
  }
  block_reduce_vec<HC>(acc, red);
  if (threadIdx.x < HC) dqb[threadIdx.x] = acc[threadIdx.x] / (ctot + 1e-10f);
  __syncthreads();
  // 4. dq rows: the masked mean spreads d(qbar) over the valid sequences
  for (int s = threadIdx.x; s < S; s += NT) {
    const int64_t r = (int64_t)s * R + i;
    const float mk = mask[r];
    T *dq = dqkvg + r * ld;
#pragma unroll
    for (int k = 0; k < HC; ++k) stf(dq + k, mk * dqb[k]);
  }
}

template <typename T>
cudaError_t launch_fwd(const GlobalAttnArgs &a, cudaStream_t s) {
  const size_t sm = (size_t)a.S * a.H * sizeof(float);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  if (a.H == 8 && a.c == 8) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(gattn_fwd_k<T, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    launch_k(gattn_fwd_k<T, 8, 8>, a.R, NT, sm, s, (const T *)a.qkvg, a.ld, a.S, a.R, a.mask, a.scale, a.qbar,
                                            (float *)a.o_att_bar, a.lse2, (T *)a.o_gate);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_bwd(const GlobalAttnArgs &a, const void *dog, void *dqkvg, cudaStream_t s) {
  const size_t sm = (size_t)a.S * a.H * sizeof(float);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  if (a.H == 8 && a.c == 8) {
    if (sm > 48 * 1024) cudaFuncSetAttribute(gattn_bwd_k<T, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    launch_k(gattn_bwd_k<T, 8, 8>, a.R, NT, sm, s, (const T *)a.qkvg, a.ld, a.S, a.R, a.mask, a.scale, a.qbar,
                                            (const float *)a.o_att_bar, a.lse2, (const T *)dog, (T *)dqkvg);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool global_attn_supported(int H, int c) { return H == 8 && c == 8; }

cudaError_t global_attn_fwd(const GlobalAttnArgs &a, int use_bf16, cudaStream_t s) {
  const double ts = use_bf16 ? 2.0 : 4.0;
  Prof p("gattn_fwd", s, 4.0 * a.S * (double)a.R * a.H * a.c,
         ts * (double)a.S * a.R * (2.0 * a.H * a.c + 2.0 * a.c) + ts * (double)a.S * a.R * a.H * a.c);
  return use_bf16 ? launch_fwd<bf16>(a, s) : launch_fwd<float>(a, s);
}

cudaError_t global_attn_bwd(const GlobalAttnArgs &a, const void *dog, void *dqkvg, float *scratch, int use_bf16,
                            cudaStream_t s) {
  (void)scratch;
  const double ts = use_bf16 ? 2.0 : 4.0;
  Prof p("gattn_bwd", s, 8.0 * a.S * (double)a.R * a.H * a.c,
         ts * (double)a.S * a.R * (4.0 * a.H * a.c + 4.0 * a.c));
  return use_bf16 ? launch_bwd<bf16>(a, dog, dqkvg, s) : launch_bwd<float>(a, dog, dqkvg, s);
}

}  // namespace evo
