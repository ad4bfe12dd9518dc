/*
 * evo.h -- C ABI of the GB300 (sm_103a) Evoformer block library (libevo.so).
 *
 * The operation is one AlphaFold2 Evoformer block, the unit that HelixFold
 * (arXiv 2207.05477) optimises: MSA row attention with pair bias, MSA column
 * attention, MSA transition, outer product mean, triangle multiplication
 * (outgoing, incoming), triangle attention (starting, ending node) and pair
 * transition, in that order (paper Sec. 3.1 and Fig. 1-2 name the modules;
 * the arithmetic is that of AlphaFold2's published Evoformer, Algorithms 6-15
 * and 19 of its supplement).  Forward and backward; the backward recomputes
 * the forward of the block from its inputs (per-block recompute, Sec. 3.4.1).
 *
 * Conventions for every entry point:
 *  - Every pointer argument named *_in/*_out, m, z, masks, params, dparams,
 *    workspace is a DEVICE pointer owned by the caller.  The library never
 *    allocates or frees device memory and never synchronises the stream,
 *    except evo_get_error which reads the device error word.
 *  - Tensors are dense, row-major, channel innermost:
 *      m        [n_seq, n_res, c_m]     activation dtype (act_dtype)
 *      z        [n_res, n_res, c_z]     activation dtype
 *      msa_mask [n_seq, n_res]          fp32, 1 = valid, 0 = padded
 *      pair_mask[n_res, n_res]          fp32, 1 = valid, 0 = padded
 *    A masked key is excluded from its softmax exactly; a query with no valid
 *    key receives an attention output of 0 (its update is the output bias).
 *  - params is the flat fp32 parameter buffer of one block (evo_param_layout
 *    lists each tensor; each starts on a 256-byte boundary, the alignment of
 *    the paper's fused parameter tensors, Sec. 3.2 "Tensor Fusion").
 *  - params_bf16 is evo_params_to_bf16's copy of params (same offsets); it is
 *    required when act_dtype == EVO_BF16 and ignored for EVO_F32.
 *  - Every call returns 0 (EVO_OK) or a negative EVO_ERR_* code.  Calls never
 *    abort and never print.  Launch errors are reported as EVO_ERR_CUDA.
 *  - The stream argument is a cudaStream_t (0 = legacy default stream).
 */
#ifndef EVO_H
#define EVO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *evo_stream_t; /* same type as cudaStream_t */

enum {
  EVO_OK = 0,
  EVO_ERR_INVALID_ARG = -1,  /* null pointer, non-positive size, bad enum   */
  EVO_ERR_UNSUPPORTED = -2,  /* dims the kernels do not implement           */
  EVO_ERR_ALIGNMENT = -3,    /* device pointer not 256-byte aligned         */
  EVO_ERR_WORKSPACE = -4,    /* ws_bytes below evo_workspace_size           */
  EVO_ERR_CUDA = -5,         /* a CUDA runtime call or launch failed        */
  EVO_ERR_TIMEOUT = -6       /* a bounded device wait gave up (error word)  */
};

enum { EVO_F32 = 0, EVO_BF16 = 1 };           /* act_dtype */
enum { EVO_COL_ATTENTION = 0, EVO_COL_GLOBAL = 1 }; /* msa_col_mode */
enum { EVO_MODE_FWD = 0, EVO_MODE_BWD = 1, EVO_MODE_INFER = 2 };  /* workspace query mode */

/* Sizes of one block.  Defaults of the paper's Evoformer (Table "model
 * settings", Table "FastFold vs PPFold": C_m=256, C_z=128, 8 heads):
 * c_m 256, c_z 128, h_msa 8, c_msa 32, h_tri 4, c_tri 32, c_mul 128,
 * c_opm 32, trans_n 4.  The extra-MSA block uses c_m 64, c_msa 8 and
 * msa_col_mode EVO_COL_GLOBAL. */
typedef struct evo_dims {
  int32_t n_seq, n_res, c_m, c_z;
  int32_t h_msa, c_msa, h_tri, c_tri;
  int32_t c_mul, c_opm, trans_n;
  int32_t msa_col_mode; /* EVO_COL_ATTENTION | EVO_COL_GLOBAL */
  int32_t act_dtype;    /* EVO_F32 | EVO_BF16: storage of m, z, intermediates */
  /* i-slab subbatching of the pair stack (Sec. 3.4.4), read by the inference
   * plan only (evo_block_fwd_infer, evo_block_fwd_noalloc and their
   * evo_workspace_size): 0 (or >= n_res) runs every pair step on the whole
   * n_res x n_res grid; 0 < pair_slab < n_res runs it pair_slab rows at a
   * time, so that the pair-sized scratch shrinks by n_res / pair_slab and
   * what stays full-size is z (two buffers), its transpose, the b operand of
   * a triangle product and the pair biases.  The result is the unsliced
   * forward's, bit for bit.  Requires EVO_BF16, c_z = 128, h_msa and h_tri
   * 4 or 8 and c_mul 64, 128 or 256 (EVO_ERR_UNSUPPORTED otherwise);
   * negative: EVO_ERR_INVALID_ARG. */
  int32_t pair_slab;
} evo_dims;

typedef struct evo_param_entry {
  char name[48];     /* e.g. "row.w_qkvg"                                    */
  int64_t offset;    /* in floats from the start of params                  */
  int32_t ndim;      /* 1 or 2                                              */
  int64_t shape[4];  /* weights are [out, in]                               */
} evo_param_entry;

/* Number of fp32 scalars in one block's flat parameter buffer, padding
 * included (1,829,952 at the paper's Evoformer dims).  0 on bad dims. */
size_t evo_param_count(const evo_dims *d);

/* Fills up to cap entries of the parameter table (Sec. 3.2 flat buffer) and
 * returns the total number of entries, or a negative error.  Host only. */
int evo_param_layout(const evo_dims *d, evo_param_entry *out, int cap);

/* Bytes of the BF16 parameter copy (evo_param_count * 2). */
int evo_params_bf16_size(const evo_dims *d, size_t *bytes);

/* Rounds params (fp32, device) to bfloat16 (round to nearest even) into
 * params_bf16 (device, evo_params_bf16_size bytes). */
int evo_params_to_bf16(const evo_dims *d, const float *params, void *params_bf16,
                       evo_stream_t stream);

/* Workspace bytes for evo_block_fwd (mode EVO_MODE_FWD), evo_block_bwd
 * (EVO_MODE_BWD) or evo_block_fwd_infer (EVO_MODE_INFER), and for
 * evo_stack_fwd over `batch` proteins padded to d's sizes (EVO_MODE_FWD):
 * batch 1 is the block's plan; batch > 1 adds the staging of one protein
 * (its m, z and masks in compact layout, see evo_stack_fwd).  The workspace
 * is scratch owned by the caller; its content on entry is irrelevant and on
 * exit undefined.  EVO_ERR_INVALID_ARG for batch < 1 or an unknown mode. */
int evo_workspace_size(const evo_dims *d, int batch, int mode, size_t *bytes);

/* Forward of one block: (m_out, z_out) = Evoformer(m_in, z_in).
 * m_out may equal m_in and z_out may equal z_in (in-place update).
 * All device pointers must be 256-byte aligned. */
int evo_block_fwd(const evo_dims *d, const float *params, const void *params_bf16,
                  const void *m_in, const void *z_in, void *m_out, void *z_out,
                  const float *msa_mask, const float *pair_mask,
                  void *workspace, size_t ws_bytes, evo_stream_t stream);

/* Forward of one block for inference, with the same arguments, layouts,
 * in-place rules and errors as evo_block_fwd and the same result, bit for
 * bit, in a workspace about a quarter of EVO_MODE_FWD's: size it with
 * evo_workspace_size(d, EVO_MODE_INFER, ...).  The sub-modules' scratch
 * buffers share one region, each dead once its sub-module has written its
 * output, and the residual streams alternate between two buffers each, so
 * the workspace is the largest sub-module's scratch plus two m and two z
 * buffers (about 3.8 KB per pair position at the paper's dims in BF16
 * instead of 15 KB).  It carries the paper's memory read/write in-place
 * (Sec. 3.4.3: one allocation reused instead of one per intermediate) across
 * the block's sub-modules, which lets one GPU run a block on sequences of
 * several thousand residues without subbatching; with d->pair_slab set it
 * also subbatches the pair stack (Sec. 3.4.4), which takes the workspace
 * from about 3.3 KB to about 1.35 KB per pair position at the paper's dims
 * (N_seq 128, N_res 4096, slabs of 1/8 of the rows).  Evaluation mode only. */
int evo_block_fwd_infer(const evo_dims *d, const float *params, const void *params_bf16,
                        const void *m_in, const void *z_in, void *m_out, void *z_out,
                        const float *msa_mask, const float *pair_mask,
                        void *workspace, size_t ws_bytes, evo_stream_t stream);

/* Training-mode dropout of the block (AF2 Alg. 6): each non-null pointer is
 * the scale of one site's residual update, fp32 on the device, 256-byte
 * aligned, entries 0 (dropped) or 1 / (1 - rate), drawn by the caller (the
 * random draw is an input).  Row-wise sites share one draw over the rows of
 * the update: msa_row [n_res, c_m] (MSA row attention, same for every
 * sequence), tri_out, tri_in, att_start [n_res, c_z] (indexed by the pair
 * column j, same for every row i); the column-wise site att_end [n_res, c_z]
 * is indexed by the pair row i, same for every column j.  A null site is
 * not dropped; a null evo_dropout pointer is evaluation mode. */
typedef struct evo_dropout {
  const float *msa_row;
  const float *tri_out;
  const float *tri_in;
  const float *att_start;
  const float *att_end;
} evo_dropout;

/* Backward of one block with per-block recompute (Sec. 3.4.1): recomputes
 * the forward from (m_in, z_in) inside the workspace, then propagates the
 * cotangents dm_out [n_seq,n_res,c_m] and dz_out [n_res,n_res,c_z]
 * (activation dtype) back to dm_in, dz_in (activation dtype, overwritten)
 * and ADDS the parameter gradient to dparams (fp32, evo_param_count). */
int evo_block_bwd(const evo_dims *d, const float *params, const void *params_bf16,
                  const void *m_in, const void *z_in,
                  const float *msa_mask, const float *pair_mask,
                  const void *dm_out, const void *dz_out,
                  void *dm_in, void *dz_in, float *dparams,
                  void *workspace, size_t ws_bytes, evo_stream_t stream);

/* evo_block_fwd / evo_block_bwd with training-mode dropout (see
 * evo_dropout; NULL gives exactly the plain calls).  The backward recomputes
 * the forward with the same scales, which must be unchanged between the two
 * calls. */
int evo_block_fwd_dropout(const evo_dims *d, const float *params, const void *params_bf16,
                          const void *m_in, const void *z_in, void *m_out, void *z_out,
                          const float *msa_mask, const float *pair_mask, const evo_dropout *dropout,
                          void *workspace, size_t ws_bytes, evo_stream_t stream);
int evo_block_bwd_dropout(const evo_dims *d, const float *params, const void *params_bf16,
                          const void *m_in, const void *z_in, const float *msa_mask,
                          const float *pair_mask, const evo_dropout *dropout,
                          const void *dm_out, const void *dz_out, void *dm_in, void *dz_in,
                          float *dparams, void *workspace, size_t ws_bytes, evo_stream_t stream);

/* Forward through n_blocks consecutive blocks (the EvoformerStack, Fig. 1)
 * of a batch of proteins, updating m and z in place.
 *  - d holds the padded sizes Smax = d->n_seq, Rmax = d->n_res and the
 *    channels; protein i has n_seq_b[i] sequences and n_res_b[i] residues
 *    (host arrays; 1 <= n_seq_b[i] <= Smax, 1 <= n_res_b[i] <= Rmax).  With
 *    batch 1 they may be NULL and the protein has the padded sizes.
 *  - Device buffers padded per protein (row-major, channel innermost):
 *    m [batch][Smax][Rmax][c_m], z [batch][Rmax][Rmax][c_z],
 *    msa_mask [batch][Smax][Rmax], pair_mask [batch][Rmax][Rmax] (fp32 0/1;
 *    the masks mark padding inside a protein's own sizes, as for a block).
 *    Entries outside a protein's sizes are neither read nor written.
 *  - Block k reads params + k*param_stride and params_bf16 + k*param_stride
 *    (bf16 elements); every protein runs the same blocks.
 *  - Workspace: evo_workspace_size(d, batch, EVO_MODE_FWD).  A protein at
 *    the padded sizes with batch 1 runs in place; in a batch each protein is
 *    staged into the workspace in compact layout, run through the blocks at
 *    its own sizes (no work on the padding) and written back.  The proteins
 *    run one after another on `stream`; results equal those of
 *    evo_stack_fwd on each protein alone, bit for bit.
 * Returns EVO_ERR_INVALID_ARG for a bad size or stride, EVO_ERR_WORKSPACE
 * when ws_bytes is too small. */
int evo_stack_fwd(const evo_dims *d, int n_blocks, int batch, const int32_t *n_seq_b,
                  const int32_t *n_res_b, const float *params, const void *params_bf16,
                  size_t param_stride, void *m, void *z, const float *msa_mask,
                  const float *pair_mask, void *workspace, size_t ws_bytes, evo_stream_t stream);

/* Forward of one block, as evo_block_fwd, but allocating nothing and taking
 * no workspace: its scratch is a 128 MiB array inside the library, reserved
 * on every GPU that loads it until the process exits.  This is a library
 * convenience with no counterpart in the paper.  It is meant for callers that
 * cannot allocate device memory when they call (a server whose device memory
 * was divided up at start-up, a host callback or latency-critical loop where
 * cudaMalloc's possible device synchronisation is not acceptable) and do not
 * want to hold a workspace of their own.
 *  - It runs the inference workspace plan (as evo_block_fwd_infer), whose
 *    outputs equal evo_block_fwd's bit for bit.
 *  - Inputs and outputs are caller-owned device buffers, exactly as for
 *    evo_block_fwd (256-byte aligned; m_out may equal m_in, z_out z_in).
 *  - Returns EVO_ERR_WORKSPACE when the problem needs more scratch than
 *    128 MiB (evo_workspace_size(d, EVO_MODE_INFER) > 128 MiB).  At the
 *    default channels that is N_res above 198 (BF16) / 138 (FP32) at
 *    N_seq = 16, above 181 / 100 at N_seq = 128 and above 55 / 28 at
 *    N_seq = 512.
 *  - The first call on a device (and the first call in a new context on it)
 *    looks up the array's device address in the current context
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address is cached per (device, context): after cudaDeviceReset the
 *    next call looks it up again.
 *  - Every call uses the same array: calls that may overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller.
 *    The forward writes every scratch byte before reading it, so nothing in
 *    the array needs to start at zero. */
int evo_block_fwd_noalloc(const evo_dims *d, const float *params, const void *params_bf16,
                          const void *m_in, const void *z_in, void *m_out, void *z_out,
                          const float *msa_mask, const float *pair_mask, evo_stream_t stream);

/* Template pair stack block (AF2 Alg. 16): the pair half of
 * the block -- triangle multiplication outgoing and incoming, triangle
 * attention starting and ending node, pair transition, with the same
 * dropout sites (msa_row ignored) -- on z alone.  Only the pair fields of
 * evo_dims are read (n_res, c_z, h_tri, c_tri, c_mul, trans_n, act_dtype);
 * the template dims are c_z 64, c_mul 64, h_tri 4, c_tri 16, trans_n 2.
 * Its flat parameter buffer holds the pair-stack tensors only
 * (evo_pair_param_count / evo_pair_param_layout, same names and 256-byte
 * alignment as the block's); evo_pair_workspace_size sizes its scratch.
 * The backward recomputes the forward, writes dz_in and adds the parameter
 * gradient to dparams; errors as for the block. */
size_t evo_pair_param_count(const evo_dims *d);
int evo_pair_param_layout(const evo_dims *d, evo_param_entry *out, int cap);
int evo_pair_workspace_size(const evo_dims *d, int mode, size_t *bytes);
int evo_pair_params_to_bf16(const evo_dims *d, const float *params, void *params_bf16, evo_stream_t stream);
int evo_pair_block_fwd(const evo_dims *d, const float *params, const void *params_bf16,
                       const void *z_in, void *z_out, const float *pair_mask, const evo_dropout *dropout,
                       void *workspace, size_t ws_bytes, evo_stream_t stream);
int evo_pair_block_bwd(const evo_dims *d, const float *params, const void *params_bf16,
                       const void *z_in, const float *pair_mask, const evo_dropout *dropout,
                       const void *dz_out, void *dz_in, float *dparams,
                       void *workspace, size_t ws_bytes, evo_stream_t stream);

/* Fused training update over a flat parameter buffer (Sec. 3.2, tensor
 * fusion: the stages of its table of kernel launches -- gradient clip by
 * global norm, optimizer update, EMA -- over all parameters at once).  For
 * every element, with G the L2 norm of the whole of grad:
 *   g  = grad * (clip_norm > 0 ? clip_norm / max(G, clip_norm) : 1)
 *   m  = beta1 m + (1 - beta1) g,   v = beta2 v + (1 - beta2) g^2
 *   w -= lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps)
 *   e  = ema_decay e + (1 - ema_decay) w          (when ema is given)
 *   params_bf16 = bf16(w), round to nearest even   (when given)
 * (Adam as Kingma and Ba 2015, Algorithm 1; AlphaFold2's settings are lr 1e-3,
 * beta1 0.9, beta2 0.999, eps 1e-6, clip_norm 0.1, ema_decay 0.999.)
 * Two launches: a deterministic partial sum of squares, then one pass that
 * clips, updates and averages; the result does not depend on the run.
 *  - n elements in each buffer (fp32 device buffers params, grad, exp_avg,
 *    exp_avg_sq, ema; bf16 params_bf16), all caller-owned, 256-byte aligned,
 *    none overlapping another.  The flat buffer of one or several blocks
 *    (evo_param_layout, padding included: a zero gradient on the padding
 *    leaves it at zero) is the intended argument.  grad is not modified.
 *  - exp_avg and exp_avg_sq start at zero before step 1; ema (may be NULL)
 *    usually starts as a copy of params; params_bf16 may be NULL.
 *  - grad_norm (may be NULL): a device float that receives G (before the
 *    clip), 4-byte aligned.
 *  - workspace: evo_adam_workspace_size(n) bytes of device scratch.
 *  - n == 0 is a no-op.  EVO_ERR_INVALID_ARG for a NULL required pointer,
 *    step < 1, a beta outside [0, 1), eps <= 0, a non-finite lr or eps, a
 *    NaN clip_norm, or (with ema) a decay outside [0, 1];
 *    EVO_ERR_ALIGNMENT, EVO_ERR_WORKSPACE as for the block. */
typedef struct evo_adam {
  float lr, beta1, beta2, eps;
  float clip_norm;  /* <= 0: no clipping */
  float ema_decay;  /* read only when ema is given */
  int32_t step;     /* Adam step number t, 1 for the first update */
} evo_adam;

size_t evo_adam_workspace_size(size_t n);
int evo_adam_step(const evo_adam *h, size_t n, float *params, const float *grad,
                  float *exp_avg, float *exp_avg_sq, float *ema, void *params_bf16,
                  float *grad_norm, void *workspace, size_t ws_bytes, evo_stream_t stream);

/* Waits for the stream, then returns and clears the device error words of
 * every unit: EVO_OK, or EVO_ERR_TIMEOUT if a bounded in-kernel wait gave up
 * since the last call. */
int evo_get_error(evo_stream_t stream);

/* Units of the library with their own device error word. */
enum { EVO_UNIT_GEMM = 0, EVO_UNIT_ATTENTION = 1, EVO_UNIT_TRIMUL = 2, EVO_UNIT_MLP = 3 };

/* Diagnostics for failure detection: launches one CTA of the given unit
 * (EVO_UNIT_GEMM: the tcgen05 GEMM; EVO_UNIT_ATTENTION: the tcgen05
 * attention kernels; EVO_UNIT_TRIMUL: the TMA triangle-multiplication and
 * channel-major LayerNorm kernels; EVO_UNIT_MLP: the fused transition MLP)
 * whose bounded mbarrier wait -- the same wait code those kernels use -- is
 * never satisfied and gives up after
 * limit_ns (at most 5 s), recording EVO_ERR_TIMEOUT in that unit's device
 * error word exactly as a timed-out wait inside one of its kernels would.
 * The GPU context stays usable; evo_get_error then returns EVO_ERR_TIMEOUT.
 * EVO_ERR_INVALID_ARG for an unknown unit or a limit outside [0, 5 s].  The
 * paper has no counterpart (it describes no failure detection). */
int evo_debug_wait_timeout(int unit, long long limit_ns, evo_stream_t stream);

/* Throughput probe of the special-function unit's exponential, the bound of
 * the attention softmax at small head dims (no counterpart in the paper):
 * `blocks` CTAs of 256 threads each run eight independent chains of
 * `iters` steps x <- 2^(a x + b) and write one float to sink[thread]
 * (caller-owned device buffer of blocks * 256 floats).  variant 0 times
 * ex2.approx.f32 (one result per instruction), variant 1 ex2.approx.bf16x2
 * (two).  The caller times the launch on `stream`; results per launch =
 * blocks * 256 * 8 * iters * (variant + 1).  EVO_ERR_INVALID_ARG for a bad
 * variant, size or pointer. */
int evo_probe_ex2(int variant, int blocks, int iters, float *sink, evo_stream_t stream);

/* Per-kernel timing.  evo_profile_begin starts recording a CUDA event pair
 * around every kernel launch of the library (on the launch stream), with the
 * launch's algorithmic flops and DRAM bytes; evo_profile_end waits for the
 * stream, stops recording and aggregates by kernel name into out (up to cap
 * entries), returning the number of distinct names.  evo_profile_only
 * (called before evo_profile_begin) restricts the next recording to the
 * launches of one kernel name, so that timing a single kernel class adds one
 * event pair per launch of that class and nothing elsewhere; NULL or "" means
 * every kernel.  With EVO_PROFILE_DETAIL=1 in the environment at
 * evo_profile_begin, GEMM entries are named by shape and tile
 * ("g<M>x<N>x<K>*<batch>s<splits>n<BN>..."). */
typedef struct evo_profile_entry {
  char name[32];
  int32_t calls;     /* launch sites that ran                           */
  int32_t launches;  /* kernel launches                                 */
  double total_ms;   /* summed event time                               */
  double flops;      /* algorithmic flops of those launches             */
  double bytes;      /* algorithmic DRAM bytes (inputs read + outputs)  */
} evo_profile_entry;
int evo_profile_only(const char *kernel_name);
/* Pause (1) or resume (0) the timing of launches inside an open recording
 * session, without synchronising: the timed launches of a session can be a
 * sample of the work issued meanwhile. */
int evo_profile_pause(int paused);
int evo_profile_begin(void);
int evo_profile_end(evo_stream_t stream, evo_profile_entry *out, int cap);

/* GEMM tile autotuning.  Between evo_tune_begin and evo_tune_end, every
 * tensor-core GEMM launch of the library is keyed by its shape (M, N, K,
 * batch, operand majors) and epilogue, and each run of n consecutive launches
 * of a key tries each of its n candidate launch configurations once, in an
 * order shuffled from run to run, every launch under a CUDA event pair: the
 * output tile width BN in {64, 128, 256} and, for the weight-gradient
 * products that add into fp32 with atomics, the number of K ranges (the
 * default, twice it, half of it, one).  Every candidate computes the same
 * product, so the work issued meanwhile stays correct; launches captured
 * into a CUDA graph are not timed.  evo_tune_end waits for the stream and the
 * device, then keeps per key the candidate with the lowest median time (the
 * default unless every candidate ran at least once) and returns the number
 * of keys; later launches of a tuned key use its choice.  Run each workload
 * n times between begin and end, n at least the largest candidate count
 * (12).  evo_tune_clear drops the table (back to the built-in choice);
 * evo_tune_entries copies up to cap entries out and returns how many there
 * are.  This scheduling aid has no counterpart in the paper. */
typedef struct evo_tune_entry {
  int64_t M, N, K, batch;
  int32_t default_bn, default_splits; /* the built-in choice                 */
  int32_t bn, splits;                 /* the chosen launch configuration     */
  int32_t candidates;                 /* configurations timed for this key   */
} evo_tune_entry;
int evo_tune_begin(void);
int evo_tune_end(evo_stream_t stream);
int evo_tune_clear(void);
int evo_tune_entries(evo_tune_entry *out, int cap);
/* The tuned table as a text file (one line per shape: its key, the built-in
 * and the chosen configuration), and back: evo_tune_load replaces the table
 * (EVO_ERR_INVALID_ARG, table unchanged, for a missing or malformed file or
 * during a tuning session).  A loaded choice is used only where the tuner
 * could have offered it for that launch.  With EVO_TUNE_CACHE=<path> in the
 * environment the file is loaded before the first GEMM launch and written by
 * every evo_tune_end. */
int evo_tune_save(const char *path);
int evo_tune_load(const char *path);

/* Static description of an EVO_* code. */
const char *evo_strerror(int code);

/* Library build id (sm target and version), static string. */
const char *evo_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EVO_H */
