// Internal launch interface of libevo's kernels (host side).
#pragma once
#include "common.cuh"
#include "prof.h"

namespace evo {

// C = epilogue( sum_k A(m,k) B(n,k) ), batched over blockIdx.z.
//   A(m,k) = A[b*a_bs + m*lda + k]   (a_mn = 0, "K-major")
//          = A[b*a_bs + k*lda + m]   (a_mn = 1, "MN-major")
//   B(n,k) likewise with ldb, b_bs, b_mn.
// With splits > 1 (batch must be 1) each split writes e.partial and the caller
// reduces the partials (reduce_splits).
struct GemmOp {
  int M, N, K, batch;
  const void *A;
  int64_t lda, a_bs;
  int a_mn;
  const void *B;
  int64_t ldb, b_bs;
  int b_mn;
  Epi e;
  int splits;
  const char *cls;  // profiler class of the launch (nullptr: "gemm_tc")
};

// SIMT FP32 GEMM (the plain path; no tensor cores).
cudaError_t gemm_simt_f32(const GemmOp &g, cudaStream_t s);
// tcgen05 + TMA BF16 GEMM (FP32 accumulation in tensor memory).
cudaError_t gemm_tc_bf16(const GemmOp &g, cudaStream_t s);
// Query whether gemm_tc_bf16 accepts the operand strides/alignment.
bool gemm_tc_supported(const GemmOp &g);
// Tile width and split count for one GEMM launch (the autotuner's choice, or
// the defaults passed in); with a and b set the launch is bracketed by that
// event pair (tune_done records b).
struct TuneChoice {
  int bn, splits;
  cudaEvent_t a, b;
};
TuneChoice tune_choose(const GemmOp &g, int default_bn, cudaStream_t s);
void tune_done(const TuneChoice &c, cudaStream_t s);
// Reads and clears the device error word (EVO_OK or EVO_ERR_TIMEOUT); synchronous.
cudaError_t error_word_read_clear(int *out);
// Launches one CTA whose bounded mbarrier wait is made to run out after limit_ns.
cudaError_t debug_wait(int64_t limit_ns, cudaStream_t s);

// Attention over one axis with optional pair bias, key mask and sigmoid gate.
// Batch b in [0,B1), head h, query x in [0,X), key y in [0,Y), head dim c.
//   q(b,x,h,:) = q[b*sQb + x*sQx + h*c + :]   g shares q's strides
//   k(b,y,h,:) = k[b*sKb + y*sKy + h*c + :]   v shares k's strides
//   bias(h,x,y) = bias[h*sBh + x*sBx + y]     (bf16 when bias_bf16, else fp32; may be null)
//   key valid   = mask[b*sMb + y*sMy] != 0    (fp32, may be null)
//   o(b,x,h,:) at o_att/o_gate[b*sOb + x*sOx + h*c + :]
//   lse2[(b*H + h)*X + x] = log2 of the softmax normaliser (+inf: no valid key)
struct AttnArgs {
  const void *q, *k, *v, *g;
  int64_t sQb, sQx, sKb, sKy;
  int B1, H, X, Y, c;
  const void *bias;
  int64_t sBh, sBx;
  int bias_bf16;
  const float *mask;
  int64_t sMb, sMy;
  void *o_att, *o_gate;
  int64_t sOb, sOx;
  float *lse2;
  float scale;
  // backward
  const void *do_att;    // grad of the ungated output, o_att's strides
  const float *Dsum;     // [(b*H+h)*X + x] = sum_d do_att * o_att
  float *dq_acc;         // fp32 [b*sOb + x*sOx + h*c + d] accumulated (unscaled)
  void *dk, *dv;         // k/v strides
  float *dbias;          // fp32 [h*sBh + x*sBx + y] accumulated
  void *dq;              // q strides: the scaled query gradient (activation type)
  // Gate backward in the same pass (tcgen05 path): with dog (grad of the gated
  // output, o strides) the kernel forms do_att = dog * g and D itself and
  // writes the gate pre-activation gradient dgpre = dog * o * g (1 - g) (q
  // strides); do_att and Dsum are then not read.
  const void *dog;
  void *dgpre;
};
cudaError_t attn_fwd(const AttnArgs &a, int use_bf16, cudaStream_t s);
// tcgen05 forward (bf16, head dim 32, at most 256 keys, 16-byte aligned rows);
// cudaErrorNotSupported (nothing launched) when TMA cannot describe the views.
bool attn_tc_supported(const AttnArgs &a);
cudaError_t attn_fwd_tc_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes);
// tcgen05 backward (as the forward, and X <= 256): writes dq, dk, dv and adds
// the pair-bias gradient; cudaErrorNotSupported (nothing launched) as above.
bool attn_bwd_tc_supported(const AttnArgs &a);
cudaError_t attn_bwd_tc_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes);
// tcgen05 backward of any length and head dims 8, 16, 32: reads do_att and
// Dsum (the gate pass), adds the unscaled query gradient into dq_acc (fp32,
// zeroed by the caller) and the pair-bias gradient into dbias, writes dk, dv;
// cudaErrorNotSupported (nothing launched) when the views do not fit.
bool attn_bwd_stream_supported(const AttnArgs &a);
cudaError_t attn_bwd_stream_launch(const AttnArgs &a, cudaStream_t s, double flops, double bytes);
// Reads and clears the error word of the tcgen05 attention kernels; synchronous.
cudaError_t attn_tc_error_read_clear(int *out);
// one CTA whose bounded wait (this unit's own) runs out after limit_ns
cudaError_t attn_tc_debug_wait(int64_t limit_ns, cudaStream_t s);
cudaError_t attn_bwd(const AttnArgs &a, int use_bf16, cudaStream_t s);

// Global column attention (extra-MSA stack): single-head k, v.
struct GlobalAttnArgs {
  const void *qkvg;  // rows (s,i) of width ld: [q (H*c) | k (c) | v (c) | g (H*c)]
  int64_t ld;
  int S, R, H, c;
  const float *mask;  // [S,R]
  void *o_att_bar;    // [R, H*c] fp32 attention output per column (before gate)
  float *qbar;        // [R, H*c] fp32 masked mean of q
  float *lse2;        // [R, H, 2] fp32 softmax max (log2 units) and sum
  void *o_gate;       // [S,R,H*c]
  float scale;
};
bool global_attn_supported(int H, int c);
cudaError_t global_attn_fwd(const GlobalAttnArgs &a, int use_bf16, cudaStream_t s);
// backward: dog [S,R,H*c] grad of gated output -> dqkvg rows (same layout as qkvg)
cudaError_t global_attn_bwd(const GlobalAttnArgs &a, const void *dog, void *dqkvg, float *scratch,
                            int use_bf16, cudaStream_t s);

// LayerNorm over channels of rows x[M, C] (eps 1e-5, biased variance).
cudaError_t ln_fwd(const void *x, const float *gamma, const float *beta, void *y, int64_t M, int C,
                   int use_bf16, cudaStream_t s);
// LayerNorm of a channel-major tensor x[C][R][pitch] (position p = (i,j) at i*pitch+j)
// written row-major y[R*R, C].
cudaError_t ln_fwd_cm(const void *x, int64_t pitch, const float *gamma, const float *beta, void *y,
                      int R, int C, int use_bf16, cudaStream_t s);
// dx = LN backward of dy (rows x[M,C]); dacc (fp32) += dx if dacc else dx_out = dx;
// dcopy (activation type, may be null) = updated dacc; with dinit (activation
// type) the accumulator starts from dinit instead of its old contents (dacc =
// dinit + dx).  Each block adds its sums of the gamma/beta gradients to
// dgamma, dbeta with fp32 atomics.
// With dsum (fp32, may be null) the column sums of what is written (the
// updated accumulator, or dx_out) are added to dsum[0..C): the bias gradient
// of the layer that consumes this gradient next.
cudaError_t ln_bwd(const void *dy, const void *x, const float *gamma, float *dacc, void *dcopy,
                   void *dx_out, int64_t M, int C, int use_bf16, cudaStream_t s, float *dgamma,
                   float *dbeta, const void *dinit = nullptr, float *dsum = nullptr);
// LayerNorm backward for the channel-major input of ln_fwd_cm: dy row-major [R*R, C],
// dx channel-major [C][R][pitch]; dgamma, dbeta accumulated with fp32 atomics.
cudaError_t ln_bwd_cm(const void *dy, const void *x, int64_t pitch, const float *gamma, void *dx,
                      int R, int C, int use_bf16, cudaStream_t s, float *dgamma, float *dbeta);

// Sum of partial rows: out[n] += sum_b part[b*N + n], n < N.
cudaError_t reduce_partials(const float *part, int nblk, int N, float *out, cudaStream_t s);
// out[n] += sum_b part[b*ld + n]
cudaError_t reduce_partials_ld(const float *part, int nblk, int64_t ld, int N, float *out, cudaStream_t s);
// out[n] += sum_m x[m, n] (leading dim ld, activation type); each block adds its
// column sums over a range of rows with fp32 atomics.
cudaError_t colsum(const void *x, int64_t ld, int64_t M, int N, int use_bf16, cudaStream_t s, float *out);
// out[i] += sum_s part[s*n + i]
cudaError_t reduce_splits(const float *part, int splits, int64_t n, float *out, cudaStream_t s);
// bf16 out[map(m, n)] = sum_s part[(s*M + m)*N + n]  (N even)
cudaError_t reduce_splits_map(const float *part, int splits, int M, int N, const OutMap &map, void *out,
                              cudaStream_t s);

// Pair-bias projection: out[h][pos'] = x[pos] . w[h], pos = (p0,p1) in [R,R];
// pos' = p0*R+p1, or p1*R+p0 with transpose.  out is bf16 when use_bf16 (the
// attention kernels read the bias as an activation), else fp32.
cudaError_t head_proj_fwd(const void *x, const float *w, void *out, int R, int C, int H, int transpose,
                          int use_bf16, cudaStream_t s);
// The pair-bias projection of npos consecutive positions (the rows of an
// i-slab, not transposed) into out[h * hstride + pos]; BF16, C = 128, H = 4
// or 8 only (cudaErrorNotSupported otherwise, nothing launched).
cudaError_t head_proj_fwd_rows(const void *x, const float *w, void *out, int64_t npos, int64_t hstride, int C, int H,
                               cudaStream_t s);
// dx[pos] (+)= sum_h dbias[h][pos'] w[h]; dw += sum_pos dbias x (each block adds
// its sum over a range of positions with fp32 atomics).
cudaError_t head_proj_bwd(const float *dbias, const void *x, const float *w, void *dx, int accumulate,
                          int R, int C, int H, int transpose, int use_bf16, cudaStream_t s, float *dw);

// Triangle multiplication gating: abg[P, ld] projections [ap|ag|bp|bg|g] (the
// output gate g already through its sigmoid, by the projection's epilogue);
// a = mask ap sigmoid(ag), b = mask bp sigmoid(bg) written channel-major
// [c][R][pitch] (incoming: transposed positions).
cudaError_t trimul_gate_fwd(const void *abg, int64_t ld, const float *mask, void *A, void *B, int64_t pitch,
                            int R, int cm, int incoming, int use_bf16, cudaStream_t s);
// TMA-tiled BF16 versions (cm a multiple of 64, 16-byte aligned rows); they
// return cudaErrorNotSupported (nothing launched) when a tensor map cannot
// describe the buffers.
bool trimul_gate_tma_supported(const void *abg, int64_t ld, const void *A, const void *B, int64_t pitch, int R,
                               int cm);
cudaError_t trimul_gate_fwd_tma_launch(const void *abg, int64_t ld, const float *mask, void *A, void *B, int64_t pitch,
                                       int R, int cm, int incoming, cudaStream_t s);
// The outgoing gate of `rows` pair rows (an i-slab): abg [rows * R, ld], mask
// [rows][R] (the slab's rows), A and B channel-major [c][rows][pitch] at
// channel strides a_cstride / b_cstride (B may be the slab's rows of a full
// [c][R][pitch] buffer); swap: a from (bp, bg) and b from (ap, ag).  BF16 TMA
// kernel only (cudaErrorNotSupported when it does not apply).
cudaError_t trimul_gate_fwd_rows(const void *abg, int64_t ld, const float *mask, void *A, int64_t a_cstride, void *B,
                                 int64_t b_cstride, int64_t pitch, int rows, int R, int cm, int swap, cudaStream_t s);
cudaError_t trimul_gate_bwd_tma_launch(const void *dA, const void *dB, int64_t pitch, const void *abg, int64_t ld,
                                       const float *mask, void *dabg, int R, int cm, int incoming, cudaStream_t s);
// TMA-tiled BF16 versions of ln_fwd_cm / ln_bwd_cm (C = 64, 128 or 256);
// cudaErrorNotSupported (nothing launched) as above.
bool ln_cm_tma_supported(const void *x, int64_t pitch, const void *y, int R, int C);
cudaError_t ln_fwd_cm_tma_launch(const void *x, int64_t pitch, const float *gamma, const float *beta, void *y, int R,
                                 int C, cudaStream_t s);
// The same for `rows` pair rows of R columns: x [C][rows][pitch] at channel
// stride cstride, y [rows * R, C] (BF16 TMA kernel only).
cudaError_t ln_fwd_cm_rows(const void *x, int64_t pitch, int64_t cstride, const float *gamma, const float *beta,
                           void *y, int rows, int R, int C, cudaStream_t s);
cudaError_t ln_bwd_cm_tma_launch(const void *dy, const void *x, int64_t pitch, const float *gamma, void *dx, int R,
                                 int C, float *dgamma, float *dbeta, cudaStream_t s);
// Reads and clears the error word of the TMA gate kernels; synchronous.
cudaError_t trimul_tc_error_read_clear(int *out);

// Fused transition MLP (tcgen05, BF16): out = res + b2 + relu(xn W1^T + b1) W2^T
// over M rows of C channels (C = 128 or 256), the hidden layer (width N1, a
// multiple of 128) kept on the SM.  W1 is [N1][C], W2 [C][N1] (row-major,
// BF16); all pointers 16-byte aligned.
bool mlp_fused_supported(int64_t M, int C, int N1, const void *xn, const void *w1, const float *b1, const void *w2,
                         const float *b2, const void *res, const void *out);
cudaError_t mlp_fused_tc(const void *xn, const void *w1, const float *b1, const void *w2, const float *b2,
                         const void *res, void *out, int64_t M, int C, int N1, cudaStream_t s);
cudaError_t mlp_tc_error_read_clear(int *out);
cudaError_t mlp_tc_debug_wait(int64_t limit_ns, cudaStream_t s);
cudaError_t trimul_tc_debug_wait(int64_t limit_ns, cudaStream_t s);
cudaError_t trimul_gate_bwd(const void *dA, const void *dB, int64_t pitch, const void *abg, int64_t ld,
                            const float *mask, void *dabg, int R, int cm, int incoming, int use_bf16,
                            cudaStream_t s);
// Output gate backward: dy = dz * g; dgpre = dz * y * g (1 - g).
// With dsum (fp32, may be null): dsum[c] += sum_p dy[p, c].
cudaError_t gate_out_bwd(const void *dz, const void *g, int64_t g_ld, const void *y, void *dy,
                         void *dgpre, int64_t dg_ld, int64_t P, int C, int use_bf16, cudaStream_t s,
                         float *dsum = nullptr);
// Attention gate backward: do_att = dog * g; dgpre = dog * o_att * g (1-g);
// D[(b*H+h)*X+x] = sum_d do_att * o_att.  Rows follow AttnArgs strides.
cudaError_t attn_gate_bwd(const AttnArgs &a, const void *dog, void *dgpre, int64_t sGb_d, int64_t sGx_d,
                          void *do_att, float *D, int use_bf16, cudaStream_t s);
// Training-mode dropout of a residual update: out[p, c] = (res ? res[p, c] : 0)
// + upd[p, c] * scale[q, c] with q = p % R (row-wise) or p / R (column-wise);
// rows of C channels, activation type; scale fp32 [R, C].
cudaError_t dropout_apply(const void *upd, const float *scale, const void *res, void *out, int64_t P, int C, int R,
                          int colwise, int use_bf16, cudaStream_t s);
// dq (activation type, q strides of dst) = scale * dq_acc
cudaError_t attn_dq_store(const AttnArgs &a, void *dq, int use_bf16, cudaStream_t s);
// inv_norm[i*R+j] = 1 / (eps + sum_s mask[s,i] mask[s,j])
cudaError_t opm_inv_norm(const float *mask, float *inv_norm, int S, int R, float eps, cudaStream_t s);
// y[m, :] = x[m, :] * scale[m]   (x, y activation type; rows of width C)
// With dsum (fp32, may be null): dsum[c] += sum_m y[m, c].
cudaError_t row_scale(const void *x, const float *scale, void *y, int64_t M, int C, int use_bf16, cudaStream_t s,
                      float *dsum = nullptr);
// dst = (float) src  and  dst = (T) src conversions; fill.
cudaError_t to_f32(const void *src, float *dst, int64_t n, int use_bf16, cudaStream_t s);
cudaError_t from_f32(const float *src, void *dst, int64_t n, int use_bf16, cudaStream_t s);
cudaError_t f32_to_bf16(const float *src, bf16 *dst, int64_t n, cudaStream_t s);
// dst[b * dst_ld + a][.] = src[a * Bd + b][.] over an A x Bd grid of rows of
// W 32-bit words (the pair grid transposed: A = Bd = dst_ld = R; a slab of A
// rows put back into the columns of an R x R grid: Bd = dst_ld = R).
cudaError_t transpose_rows(const void *src, void *dst, int64_t A, int64_t Bd, int W, int64_t dst_ld, cudaStream_t s);
// Copies A x B rows of W 32-bit words between row-major [.][src_B][W] and
// [.][dst_B][W] layouts (the staging of a padded protein).
cudaError_t copy_rows_strided(const void *src, void *dst, int64_t A, int64_t B, int64_t src_B, int64_t dst_B, int W,
                              cudaStream_t s);

}  // namespace evo
