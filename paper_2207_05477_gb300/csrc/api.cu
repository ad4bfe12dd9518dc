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

int evo_workspace_size(const evo_dims *d, int mode, size_t *bytes) {
  if (!bytes || (mode != EVO_MODE_FWD && mode != EVO_MODE_BWD && mode != EVO_MODE_INFER)) return EVO_ERR_INVALID_ARG;
  const int v = validate_dims(d);
  if (v != EVO_OK) return v;
  *bytes = workspace_bytes(*d, mode);
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
  const int v = validate_dims(d);
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

int evo_stack_fwd(const evo_dims *d, int n_blocks, const float *params, const void *params_bf16, size_t param_stride,
                  void *m, void *z, const float *msa_mask, const float *pair_mask, void *workspace, size_t ws_bytes,
                  evo_stream_t stream) {
  const int v = validate_dims(d);
  if (v != EVO_OK) return v;
  if (n_blocks < 0 || param_stride < evo_param_count(d) || param_stride % 128) return EVO_ERR_INVALID_ARG;
  const bool bf = d->act_dtype == EVO_BF16;
  for (int b = 0; b < n_blocks; ++b) {
    const float *p = params + (size_t)b * param_stride;
    const void *p16 = bf ? (const void *)((const bf16 *)params_bf16 + (size_t)b * param_stride) : nullptr;
    const int r = evo_block_fwd(d, p, p16, m, z, m, z, msa_mask, pair_mask, workspace, ws_bytes, stream);
    if (r != EVO_OK) return r;
  }
  return EVO_OK;
}

int evo_get_error(evo_stream_t stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return EVO_ERR_CUDA;
  int h = 0, h2 = 0, h3 = 0;
  if (error_word_read_clear(&h) != cudaSuccess) return EVO_ERR_CUDA;
  if (attn_tc_error_read_clear(&h2) != cudaSuccess) return EVO_ERR_CUDA;
  if (trimul_tc_error_read_clear(&h3) != cudaSuccess) return EVO_ERR_CUDA;
  return h != EVO_OK ? h : h2 != EVO_OK ? h2 : h3;
}

int evo_debug_wait_timeout(int unit, long long limit_ns, evo_stream_t stream) {
  if (limit_ns < 0 || limit_ns > 5000000000ll) return EVO_ERR_INVALID_ARG;
  cudaError_t e;
  switch (unit) {
    case EVO_UNIT_GEMM: e = debug_wait(limit_ns, (cudaStream_t)stream); break;
    case EVO_UNIT_ATTENTION: e = attn_tc_debug_wait(limit_ns, (cudaStream_t)stream); break;
    case EVO_UNIT_TRIMUL: e = trimul_tc_debug_wait(limit_ns, (cudaStream_t)stream); break;
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
