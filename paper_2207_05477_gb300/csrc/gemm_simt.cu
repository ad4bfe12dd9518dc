// SIMT FP32 GEMM: the plain path's projection / contraction kernel (no tensor
// cores, no TF32).  64x64 output tile per CTA, 256 threads with a 4x4 register
// tile each, K staged through shared memory 16 at a time.
#include "kernels.h"

namespace evo {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(GemmOp g) {
  pdl_entry();
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int b = blockIdx.z / g.splits, split = blockIdx.z % g.splits;
  const T *A = (const T *)g.A + (int64_t)b * g.a_bs;
  const T *B = (const T *)g.B + (int64_t)b * g.b_bs;
  int kchunk = (g.K + g.splits - 1) / g.splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int kbeg = split * kchunk;
  const int kend = min(g.K, kbeg + kchunk);

  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + r * 256;
      int mm, kk;
      if (g.a_mn) { kk = idx / BM; mm = idx % BM; } else { mm = idx / BK; kk = idx % BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float va = 0.f;
      if (gm < g.M && gk < kend)
        va = ldf(A + (g.a_mn ? (int64_t)gk * g.lda + gm : (int64_t)gm * g.lda + gk));
      As[kk][mm] = va;
      int nn;
      if (g.b_mn) { kk = idx / BN; nn = idx % BN; } else { nn = idx / BK; kk = idx % BK; }
      const int gn = n0 + nn, gk2 = k0 + kk;
      float vb = 0.f;
      if (gn < g.N && gk2 < kend)
        vb = ldf(B + (g.b_mn ? (int64_t)gk2 * g.ldb + gn : (int64_t)gn * g.ldb + gk2));
      Bs[kk][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n < g.N) epi_store<T>(g.e, b, split, m, n, acc[i][j]);
    }
  }
}
}  // namespace

cudaError_t gemm_simt_f32(const GemmOp &g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch * g.splits);
  Prof p("gemm_simt", s, 2.0 * g.M * g.N * (double)g.K * g.batch,
         4.0 * g.batch * ((double)g.M * g.K + (double)g.N * g.K + (double)g.M * g.N));
  launch_k(gemm_simt_kernel<float>, grid, 256, 0, s, g);
  return cudaGetLastError();
}

}  // namespace evo
