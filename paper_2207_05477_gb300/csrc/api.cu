// C ABI of libevo (declared in include/evo.h).
#include <cstring>

#include "block.h"

using namespace evo;

namespace {

bool aligned256(const void *p) { return p && ((uintptr_t)p & 255u) == 0; }

}  // namespace

extern "C" {

size_t evo_param_count(const evo_dims *d) {
  if (!d) return 0;
  std::vector<PEntry> t;
  return (size_t)build_param_table(*d, t);
}

int evo_param_layout(const evo_dims *d, evo_param_entry *out, int cap) {
  if (!d) return EVO_ERR_INVALID_ARG;
  std::vector<PEntry> t;
  build_param_table(*d, t);
  for (int i = 0; i < (int)t.size() && i < cap && out; ++i) {
    std::memset(&out[i], 0, sizeof(evo_param_entry));
    std::strncpy(out[i].name, t[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].offset = t[i].offset;
    out[i].ndim = t[i].ndim;
    for (int k = 0; k < 4; ++k) out[i].shape[k] = t[i].shape[k];
  }
  return (int)t.size();
}

int evo_params_bf16_size(const evo_dims *d, size_t *bytes) {
  if (!d || !bytes) return EVO_ERR_INVALID_ARG;
  *bytes = evo_param_count(d) * 2;
  return EVO_OK;
}

int evo_params_to_bf16(const evo_dims *d, const float *params, void *params_bf16, evo_stream_t stream) {
  if (!d || !params || !params_bf16) return EVO_ERR_INVALID_ARG;
  if (!aligned256(params) || !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  const int64_t n = (int64_t)evo_param_count(d);
  return f32_to_bf16(params, (bf16 *)params_bf16, n, (cudaStream_t)stream) == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Staging of one protein of a padded batch: m, z and both masks in compact layout.
size_t staging_bytes(const evo_dims &d) {
  const size_t es = d.act_dtype == EVO_BF16 ? 2 : 4;
  const size_t S = (size_t)d.n_seq, R = (size_t)d.n_res;
  return al256(S * R * d.c_m * es) + al256(R * R * d.c_z * es) + al256(S * R * 4) + al256(R * R * 4);
}

}  // namespace

int evo_workspace_size(const evo_dims *d, int batch, int mode, size_t *bytes) {
  if (!bytes || batch < 1 || (mode != EVO_MODE_FWD && mode != EVO_MODE_BWD && mode != EVO_MODE_INFER))
    return EVO_ERR_INVALID_ARG;
  const int v = mode == EVO_MODE_INFER ? validate_infer_dims(d) : validate_dims(d);
  if (v != EVO_OK) return v;
  *bytes = workspace_bytes(*d, mode) + (batch > 1 ? staging_bytes(*d) : 0);
  return EVO_OK;
}

namespace {

int dropout_ok(const evo_dropout *dr) {
  if (!dr) return EVO_OK;
  for (const float *q : {dr->msa_row, dr->tri_out, dr->tri_in, dr->att_start, dr->att_end})
    if (q && !aligned256(q)) return EVO_ERR_ALIGNMENT;
  return EVO_OK;
}

}  // namespace

int evo_block_fwd(const evo_dims *d, const float *params, const void *params_bf16, const void *m_in, const void *z_in,
                  void *m_out, void *z_out, const float *msa_mask, const float *pair_mask, void *workspace,
                  size_t ws_bytes, evo_stream_t stream) {
  return evo_block_fwd_dropout(d, params, params_bf16, m_in, z_in, m_out, z_out, msa_mask, pair_mask, nullptr,
                               workspace, ws_bytes, stream);
}

int evo_block_bwd(const evo_dims *d, const float *params, const void *params_bf16, const void *m_in, const void *z_in,
                  const float *msa_mask, const float *pair_mask, const void *dm_out, const void *dz_out, void *dm_in,
                  void *dz_in, float *dparams, void *workspace, size_t ws_bytes, evo_stream_t stream) {
  return evo_block_bwd_dropout(d, params, params_bf16, m_in, z_in, msa_mask, pair_mask, nullptr, dm_out, dz_out,
                               dm_in, dz_in, dparams, workspace, ws_bytes, stream);
}

int evo_block_fwd_dropout(const evo_dims *d, const float *params, const void *params_bf16, const void *m_in,
                          const void *z_in, void *m_out, void *z_out, const float *msa_mask, const float *pair_mask,
                          const evo_dropout *dropout, void *workspace, size_t ws_bytes, evo_stream_t stream) {
  const int v = validate_dims(d);
  if (v != EVO_OK) return v;
  const bool bf = d->act_dtype == EVO_BF16;
  if (!params || !m_in || !z_in || !m_out || !z_out || !msa_mask || !pair_mask || !workspace || (bf && !params_bf16))
    return EVO_ERR_INVALID_ARG;
  for (const void *p : {(const void *)params, m_in, z_in, (const void *)m_out, (const void *)z_out,
                        (const void *)msa_mask, (const void *)pair_mask, (const void *)workspace})
    if (!aligned256(p)) return EVO_ERR_ALIGNMENT;
  if (bf && !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  if (dropout_ok(dropout) != EVO_OK) return EVO_ERR_ALIGNMENT;
  return block_forward(*d, params, (const bf16 *)params_bf16, m_in, z_in, m_out, z_out, msa_mask, pair_mask,
                       workspace, ws_bytes, (cudaStream_t)stream, dropout);
}

int evo_block_fwd_infer(const evo_dims *d, const float *params, const void *params_bf16, const void *m_in,
                        const void *z_in, void *m_out, void *z_out, const float *msa_mask, const float *pair_mask,
                        void *workspace, size_t ws_bytes, evo_stream_t stream) {
  const int v = validate_infer_dims(d);
  if (v != EVO_OK) return v;
  const bool bf = d->act_dtype == EVO_BF16;
  if (!params || !m_in || !z_in || !m_out || !z_out || !msa_mask || !pair_mask || !workspace || (bf && !params_bf16))
    return EVO_ERR_INVALID_ARG;
  for (const void *p : {(const void *)params, m_in, z_in, (const void *)m_out, (const void *)z_out,
                        (const void *)msa_mask, (const void *)pair_mask, (const void *)workspace})
    if (!aligned256(p)) return EVO_ERR_ALIGNMENT;
  if (bf && !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  return block_forward_infer(*d, params, (const bf16 *)params_bf16, m_in, z_in, m_out, z_out, msa_mask, pair_mask,
                             workspace, ws_bytes, (cudaStream_t)stream);
}

int evo_block_bwd_dropout(const evo_dims *d, const float *params, const void *params_bf16, const void *m_in,
                          const void *z_in, const float *msa_mask, const float *pair_mask, const evo_dropout *dropout,
                          const void *dm_out, const void *dz_out, void *dm_in, void *dz_in, float *dparams,
                          void *workspace, size_t ws_bytes, evo_stream_t stream) {
  const int v = validate_dims(d);
  if (v != EVO_OK) return v;
  const bool bf = d->act_dtype == EVO_BF16;
  if (!params || !m_in || !z_in || !msa_mask || !pair_mask || !dm_out || !dz_out || !dm_in || !dz_in || !dparams ||
      !workspace || (bf && !params_bf16))
    return EVO_ERR_INVALID_ARG;
  for (const void *p : {(const void *)params, m_in, z_in, (const void *)msa_mask, (const void *)pair_mask, dm_out,
                        dz_out, (const void *)dm_in, (const void *)dz_in, (const void *)dparams,
                        (const void *)workspace})
    if (!aligned256(p)) return EVO_ERR_ALIGNMENT;
  if (bf && !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  if (dropout_ok(dropout) != EVO_OK) return EVO_ERR_ALIGNMENT;
  return block_backward(*d, params, (const bf16 *)params_bf16, m_in, z_in, msa_mask, pair_mask, dm_out, dz_out, dm_in,
                        dz_in, dparams, workspace, ws_bytes, (cudaStream_t)stream, dropout);
}

int evo_stack_fwd(const evo_dims *d, int n_blocks, int batch, const int32_t *n_seq_b, const int32_t *n_res_b,
                  const float *params, const void *params_bf16, size_t param_stride, void *m, void *z,
                  const float *msa_mask, const float *pair_mask, void *workspace, size_t ws_bytes,
                  evo_stream_t stream) {
  const int v = validate_dims(d);
  if (v != EVO_OK) return v;
  if (n_blocks < 0 || batch < 1 || param_stride < evo_param_count(d) || param_stride % 128) return EVO_ERR_INVALID_ARG;
  if (batch > 1 && (!n_seq_b || !n_res_b)) return EVO_ERR_INVALID_ARG;
  const int Smax = d->n_seq, Rmax = d->n_res;
  for (int i = 0; i < batch && n_seq_b && n_res_b; ++i)
    if (n_seq_b[i] < 1 || n_seq_b[i] > Smax || n_res_b[i] < 1 || n_res_b[i] > Rmax) return EVO_ERR_INVALID_ARG;
  if (batch == 1 && n_seq_b && n_res_b && (n_seq_b[0] != Smax || n_res_b[0] != Rmax)) return EVO_ERR_INVALID_ARG;
  if (n_blocks == 0) return EVO_OK;  // the identity: nothing to launch
  if (!params || !m || !z || !msa_mask || !pair_mask || !workspace) return EVO_ERR_INVALID_ARG;
  const bool bf = d->act_dtype == EVO_BF16;
  const cudaStream_t s = (cudaStream_t)stream;
  auto run = [&](const evo_dims *dd, void *mm, void *zz, const float *ms, const float *ps, void *ws, size_t wb) {
    for (int k = 0; k < n_blocks; ++k) {
      const float *p = params + (size_t)k * param_stride;
      const void *p16 = bf ? (const void *)((const bf16 *)params_bf16 + (size_t)k * param_stride) : nullptr;
      const int r = evo_block_fwd(dd, p, p16, mm, zz, mm, zz, ms, ps, ws, wb, stream);
      if (r != EVO_OK) return r;
    }
    return (int)EVO_OK;
  };
  if (batch == 1) return run(d, m, z, msa_mask, pair_mask, workspace, ws_bytes);

  // a padded batch: each protein staged in compact layout after the block plan
  const size_t plan = workspace_bytes(*d, EVO_MODE_FWD);
  if (ws_bytes < plan + staging_bytes(*d)) return EVO_ERR_WORKSPACE;
  const size_t es = bf ? 2 : 4;
  char *st = (char *)workspace + al256(plan);
  if ((uintptr_t)st % 256) return EVO_ERR_ALIGNMENT;
  char *sm = st;
  char *sz = sm + al256((size_t)Smax * Rmax * d->c_m * es);
  char *smm = sz + al256((size_t)Rmax * Rmax * d->c_z * es);
  char *spm = smm + al256((size_t)Smax * Rmax * 4);
  const int mw = d->c_m * (int)es / 4, zw = d->c_z * (int)es / 4;  // 32-bit words per row
  for (int i = 0; i < batch; ++i) {
    const int S = n_seq_b[i], R = n_res_b[i];
    evo_dims di = *d;
    di.n_seq = S, di.n_res = R;
    char *mi = (char *)m + (size_t)i * Smax * Rmax * d->c_m * es;
    char *zi = (char *)z + (size_t)i * Rmax * Rmax * d->c_z * es;
    const float *mmi = msa_mask + (size_t)i * Smax * Rmax;
    const float *pmi = pair_mask + (size_t)i * Rmax * Rmax;
    // gather: [S][R][.] of the padded [Smax][Rmax][.] slot into compact rows
    if (copy_rows_strided(mi, sm, S, R, Rmax, R, mw, s) != cudaSuccess ||
        copy_rows_strided(zi, sz, R, R, Rmax, R, zw, s) != cudaSuccess ||
        copy_rows_strided(mmi, smm, S, R, Rmax, R, 1, s) != cudaSuccess ||
        copy_rows_strided(pmi, spm, R, R, Rmax, R, 1, s) != cudaSuccess)
      return EVO_ERR_CUDA;
    const int r = run(&di, sm, sz, (const float *)smm, (const float *)spm, workspace, plan);
    if (r != EVO_OK) return r;
    // scatter the updated m and z back into the slot
    if (copy_rows_strided(sm, mi, S, R, R, Rmax, mw, s) != cudaSuccess ||
        copy_rows_strided(sz, zi, R, R, R, Rmax, zw, s) != cudaSuccess)
      return EVO_ERR_CUDA;
  }
  return EVO_OK;
}

int evo_get_error(evo_stream_t stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return EVO_ERR_CUDA;
  int h = 0, h2 = 0, h3 = 0, h4 = 0;
  if (error_word_read_clear(&h) != cudaSuccess) return EVO_ERR_CUDA;
  if (attn_tc_error_read_clear(&h2) != cudaSuccess) return EVO_ERR_CUDA;
  if (trimul_tc_error_read_clear(&h3) != cudaSuccess) return EVO_ERR_CUDA;
  if (mlp_tc_error_read_clear(&h4) != cudaSuccess) return EVO_ERR_CUDA;
  return h != EVO_OK ? h : h2 != EVO_OK ? h2 : h3 != EVO_OK ? h3 : h4;
}

int evo_debug_wait_timeout(int unit, long long limit_ns, evo_stream_t stream) {
  if (limit_ns < 0 || limit_ns > 5000000000ll) return EVO_ERR_INVALID_ARG;
  cudaError_t e;
  switch (unit) {
    case EVO_UNIT_GEMM: e = debug_wait(limit_ns, (cudaStream_t)stream); break;
    case EVO_UNIT_ATTENTION: e = attn_tc_debug_wait(limit_ns, (cudaStream_t)stream); break;
    case EVO_UNIT_TRIMUL: e = trimul_tc_debug_wait(limit_ns, (cudaStream_t)stream); break;
    case EVO_UNIT_MLP: e = mlp_tc_debug_wait(limit_ns, (cudaStream_t)stream); break;
    default: return EVO_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

const char *evo_strerror(int code) {
  switch (code) {
    case EVO_OK: return "ok";
    case EVO_ERR_INVALID_ARG: return "invalid argument";
    case EVO_ERR_UNSUPPORTED: return "unsupported dimensions";
    case EVO_ERR_ALIGNMENT: return "device pointer not 256-byte aligned";
    case EVO_ERR_WORKSPACE: return "workspace too small";
    case EVO_ERR_CUDA: return "CUDA error";
    case EVO_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown error";
  }
}

const char *evo_version(void) { return "libevo 0.1 sm_103a"; }

}  // extern "C"

extern "C" {

size_t evo_pair_param_count(const evo_dims *d) {
  if (!d) return 0;
  std::vector<PEntry> t;
  return (size_t)build_param_table(*d, t, true);
}

int evo_pair_param_layout(const evo_dims *d, evo_param_entry *out, int cap) {
  if (!d) return EVO_ERR_INVALID_ARG;
  std::vector<PEntry> t;
  build_param_table(*d, t, true);
  for (int i = 0; i < (int)t.size() && i < cap && out; ++i) {
    std::memset(&out[i], 0, sizeof(evo_param_entry));
    std::strncpy(out[i].name, t[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].offset = t[i].offset;
    out[i].ndim = t[i].ndim;
    for (int k = 0; k < 4; ++k) out[i].shape[k] = t[i].shape[k];
  }
  return (int)t.size();
}

int evo_pair_workspace_size(const evo_dims *d, int mode, size_t *bytes) {
  if (!bytes || (mode != EVO_MODE_FWD && mode != EVO_MODE_BWD)) return EVO_ERR_INVALID_ARG;
  const int v = validate_pair_dims(d);
  if (v != EVO_OK) return v;
  *bytes = workspace_bytes(*d, mode, true);
  return EVO_OK;
}

int evo_pair_params_to_bf16(const evo_dims *d, const float *params, void *params_bf16, evo_stream_t stream) {
  if (!d || !params || !params_bf16) return EVO_ERR_INVALID_ARG;
  if (!aligned256(params) || !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  const int64_t n = (int64_t)evo_pair_param_count(d);
  return f32_to_bf16(params, (bf16 *)params_bf16, n, (cudaStream_t)stream) == cudaSuccess ? EVO_OK : EVO_ERR_CUDA;
}

int evo_pair_block_fwd(const evo_dims *d, const float *params, const void *params_bf16, const void *z_in,
                       void *z_out, const float *pair_mask, const evo_dropout *dropout, void *workspace,
                       size_t ws_bytes, evo_stream_t stream) {
  const int v = validate_pair_dims(d);
  if (v != EVO_OK) return v;
  const bool bf = d->act_dtype == EVO_BF16;
  if (!params || !z_in || !z_out || !pair_mask || !workspace || (bf && !params_bf16)) return EVO_ERR_INVALID_ARG;
  for (const void *p : {(const void *)params, z_in, (const void *)z_out, (const void *)pair_mask,
                        (const void *)workspace})
    if (!aligned256(p)) return EVO_ERR_ALIGNMENT;
  if (bf && !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  if (dropout_ok(dropout) != EVO_OK) return EVO_ERR_ALIGNMENT;
  return pair_block_forward(*d, params, (const bf16 *)params_bf16, z_in, z_out, pair_mask, workspace, ws_bytes,
                            (cudaStream_t)stream, dropout);
}

int evo_pair_block_bwd(const evo_dims *d, const float *params, const void *params_bf16, const void *z_in,
                       const float *pair_mask, const evo_dropout *dropout, const void *dz_out, void *dz_in,
                       float *dparams, void *workspace, size_t ws_bytes, evo_stream_t stream) {
  const int v = validate_pair_dims(d);
  if (v != EVO_OK) return v;
  const bool bf = d->act_dtype == EVO_BF16;
  if (!params || !z_in || !pair_mask || !dz_out || !dz_in || !dparams || !workspace || (bf && !params_bf16))
    return EVO_ERR_INVALID_ARG;
  for (const void *p : {(const void *)params, z_in, (const void *)pair_mask, dz_out, (const void *)dz_in,
                        (const void *)dparams, (const void *)workspace})
    if (!aligned256(p)) return EVO_ERR_ALIGNMENT;
  if (bf && !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  if (dropout_ok(dropout) != EVO_OK) return EVO_ERR_ALIGNMENT;
  return pair_block_backward(*d, params, (const bf16 *)params_bf16, z_in, pair_mask, dz_out, dz_in, dparams,
                             workspace, ws_bytes, (cudaStream_t)stream, dropout);
}

}  // extern "C"
