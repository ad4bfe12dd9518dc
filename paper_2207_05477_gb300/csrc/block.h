// Internal: parameter table, workspace plan and block drivers of libevo.
#pragma once
#include <string>
#include <vector>

#include "evo.h"
#include "kernels.h"

namespace evo {

struct PEntry {
  std::string name;
  int64_t offset;  // floats
  int ndim;
  int64_t shape[4];
};

// The flat parameter buffer of one block (256-byte aligned tensors). Returns
// the padded total in floats.
int64_t build_param_table(const evo_dims &d, std::vector<PEntry> &out, bool pair_only = false);

// 0 if the dims are implemented, else an EVO_ERR_* code (the pair version
// checks only the pair-stack fields).
int validate_dims(const evo_dims *d);
int validate_pair_dims(const evo_dims *d);
// validate_dims plus the requirements of the i-slab inference plan
// (d->pair_slab set): what evo_block_fwd_infer and its workspace size check.
int validate_infer_dims(const evo_dims *d);
bool pair_slabbed(const evo_dims &d);

// Workspace bytes of the forward (EVO_MODE_FWD), the backward (EVO_MODE_BWD)
// or the forward-only inference plan (EVO_MODE_INFER).
size_t workspace_bytes(const evo_dims &d, int mode, bool pair_only = false);

int block_forward(const evo_dims &d, const float *p32, const bf16 *p16, const void *m_in, const void *z_in,
                  void *m_out, void *z_out, const float *msa_mask, const float *pair_mask, void *ws, size_t ws_bytes,
                  cudaStream_t s, const evo_dropout *dropout = nullptr);

// Forward in the inference plan: sub-modules share one scratch region.
int block_forward_infer(const evo_dims &d, const float *p32, const bf16 *p16, const void *m_in, const void *z_in,
                        void *m_out, void *z_out, const float *msa_mask, const float *pair_mask, void *ws,
                        size_t ws_bytes, cudaStream_t s);

int block_backward(const evo_dims &d, const float *p32, const bf16 *p16, const void *m_in, const void *z_in,
                   const float *msa_mask, const float *pair_mask, const void *dm_out, const void *dz_out, void *dm_in,
                   void *dz_in, float *dparams, void *ws, size_t ws_bytes, cudaStream_t s,
                   const evo_dropout *dropout = nullptr);

// Template pair stack block (AF2 Alg. 16): the pair half of the block alone.
int pair_block_forward(const evo_dims &d, const float *p32, const bf16 *p16, const void *z_in, void *z_out,
                       const float *pair_mask, void *ws, size_t ws_bytes, cudaStream_t s,
                       const evo_dropout *dropout = nullptr);
int pair_block_backward(const evo_dims &d, const float *p32, const bf16 *p16, const void *z_in, const float *pair_mask,
                        const void *dz_out, void *dz_in, float *dparams, void *ws, size_t ws_bytes, cudaStream_t s,
                        const evo_dropout *dropout = nullptr);

}  // namespace evo
